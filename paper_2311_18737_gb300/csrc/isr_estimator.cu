// isr_estimator.cu -- learned plasma-line estimator: forward, backward and Adam kernels.
//
// The plasma line's frequency carries the electron density (Eq. 1 of the paper).  A small
// network reads one gate's integrated spectrum (standardised log power over a band) and
// returns the line position and a presence probability:
//   4 x [conv1d 9 taps, 32 channels, zero padding, ReLU] -> location logits z (1x1 conv)
//   and presence logit q from an MLP on [max over bins, mean over bins] of the last layer.
// Loss: BCE(q, present) + present * cross-entropy(softmax(z), Gaussian target of width
// 1 bin at the true position).  Parameters are kept in FP32 (master copy, Adam moments);
// activations and working weights are stored in the plan's precision (FP32 or BF16) and
// every product is accumulated in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>

#include "isr.h"
#include "isr_kernels.cuh"

namespace {

constexpr int CH = 32;      // channels
constexpr int KT = 9;       // taps
constexpr int HALF = KT / 2;
constexpr int WIN = 3;      // soft-argmax half window
constexpr float SIGMA_T = 1.0f;

// flat parameter layout (matches the documented order)
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + CH * 1 * KT;
constexpr int OFF_W2 = OFF_B1 + CH, OFF_B2 = OFF_W2 + CH * CH * KT;
constexpr int OFF_W3 = OFF_B2 + CH, OFF_B3 = OFF_W3 + CH * CH * KT;
constexpr int OFF_W4 = OFF_B3 + CH, OFF_B4 = OFF_W4 + CH * CH * KT;
constexpr int OFF_W5 = OFF_B4 + CH, OFF_B5 = OFF_W5 + CH;
constexpr int OFF_WA = OFF_B5 + 1, OFF_BA = OFF_WA + CH * 2 * CH;
constexpr int OFF_WB = OFF_BA + CH, OFF_BB = OFF_WB + CH;
constexpr int NPARAM = OFF_BB + 1;
static_assert(NPARAM == ISR_EST_N_PARAMS, "parameter count");

__host__ __device__ constexpr int w_off(int l) { return l == 1 ? OFF_W1 : l == 2 ? OFF_W2 : l == 3 ? OFF_W3 : OFF_W4; }
__host__ __device__ constexpr int b_off(int l) { return l == 1 ? OFF_B1 : l == 2 ? OFF_B2 : l == 3 ? OFF_B3 : OFF_B4; }

template <class T> __device__ __forceinline__ float ld(const T* p, size_t i);
template <> __device__ __forceinline__ float ld<float>(const float* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p, size_t i)
{
    return __bfloat162float(p[i]);
}
template <class T> __device__ __forceinline__ T cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// ---------------------------------------------------------------- features
// x[i] = (ln max(P[lo+i], 1e-30) - mean) / (std + 1e-6) over the band; one CTA per gate
__global__ void features_kernel(const float* __restrict__ spectra, int nfft, int lo, int L, float* __restrict__ x)
{
    const float* P = spectra + (size_t)blockIdx.x * nfft + lo;
    float* xo = x + (size_t)blockIdx.x * L;
    double s = 0, s2 = 0;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        double y = log(fmax((double)P[i], 1e-30));
        s += y;
        s2 += y * y;
    }
    __shared__ double r1[32], r2[32];
    for (int o = 16; o; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = s;
        r2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    __shared__ double mean_s, inv_s;
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += r1[w];
            b += r2[w];
        }
        double m = a / L;
        double var = fmax(b / L - m * m, 0.0);
        mean_s = m;
        inv_s = 1.0 / (sqrt(var) + 1e-6);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L; i += blockDim.x)
        xo[i] = (float)((log(fmax((double)P[i], 1e-30)) - mean_s) * inv_s);
}

template <class T>
__global__ void cast_kernel(const float* __restrict__ in, size_t n, T* __restrict__ out)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = cvt<T>(in[i]);
}

// working conv weights: forward layout [ci][k][co] and the backward-data layout of the
// flipped transpose, [co][k'][ci] = W[co][ci][8 - k'] (both in the storage type)
template <class T>
__global__ void relayout_kernel(const float* __restrict__ theta, T* __restrict__ wf, T* __restrict__ wb)
{
    // layers 1..4 packed back to back: layer 1 has Cin = 1
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n1 = CH * KT, n = CH * CH * KT;
    if (i >= n1 + 3 * n) return;
    int l, e, cin;
    if (i < n1) {
        l = 1; e = i; cin = 1;
    } else {
        l = 2 + (i - n1) / n; e = (i - n1) % n; cin = CH;
    }
    // e indexes [co][ci][k]
    int co = e / (cin * KT), rem = e % (cin * KT), ci = rem / KT, k = rem % KT;
    float w = theta[w_off(l) + e];
    size_t base = l == 1 ? 0 : (size_t)n1 + (size_t)(l - 2) * n;
    wf[base + ((size_t)ci * KT + k) * CH + co] = cvt<T>(w);
    if (l > 1) wb[(size_t)(l - 2) * n + ((size_t)co * KT + (KT - 1 - k)) * CH + ci] = cvt<T>(w);
}

// ---------------------------------------------------------------- convolution
// out[b][co][i] = sum_{ci,k} w[ci][k][co] in[b][ci][i + k - 4]  (+ bias, ReLU) or, for the
// backward-data use, times the ReLU mask of `mask` (the layer below's activations).
// CTA: 128 positions of one row; warp = 16 positions, lane = output channel.
constexpr int CT = 128;
constexpr size_t conv_smem_bytes(int cin) { return sizeof(float) * (size_t)cin * ((CT + KT - 1) + KT * CH); }

template <class TIN, class TW, class TOUT, class TM, int CIN, bool FWD>
__global__ void __launch_bounds__(256) conv_kernel(const TIN* __restrict__ in, const TW* __restrict__ w,
                                                   const float* __restrict__ bias, const TM* __restrict__ mask,
                                                   int L, TOUT* __restrict__ out)
{
    constexpr int XW = CT + KT - 1;
    extern __shared__ float conv_smem[];
    float* xs = conv_smem;                 // [CIN][XW]
    float* ws = conv_smem + CIN * XW;      // [CIN][KT][CH]
    const int b = blockIdx.y;
    const int i0 = blockIdx.x * CT;
    const TIN* inb = in + (size_t)b * CIN * L;
    for (int e = threadIdx.x; e < CIN * XW; e += 256) {
        int ci = e / XW, j = e % XW;
        int pos = i0 + j - HALF;
        xs[e] = (pos >= 0 && pos < L) ? ld<TIN>(inb, (size_t)ci * L + pos) : 0.f;
    }
    for (int e = threadIdx.x; e < CIN * KT * CH; e += 256) ws[e] = ld<TW>(w, e);
    __syncthreads();
    const int co = threadIdx.x & 31;
    const int p0 = (threadIdx.x >> 5) * 16;
    float acc[16];
    const float bv = FWD ? bias[co] : 0.f;
#pragma unroll
    for (int p = 0; p < 16; ++p) acc[p] = bv;
    for (int ci = 0; ci < CIN; ++ci) {
        float xv[16 + KT - 1];
#pragma unroll
        for (int j = 0; j < 16 + KT - 1; ++j) xv[j] = xs[ci * XW + p0 + j];
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const float wv = ws[(ci * KT + k) * CH + co];
#pragma unroll
            for (int p = 0; p < 16; ++p) acc[p] = fmaf(wv, xv[p + k], acc[p]);
        }
    }
    TOUT* ob = out + ((size_t)b * CH + co) * L;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int i = i0 + p0 + p;
        if (i < L) {
            float v = acc[p];
            if (FWD) {
                v = fmaxf(v, 0.f);
            } else if (mask) {
                v = ld<TM>(mask, ((size_t)b * CH + co) * L + i) > 0.f ? v : 0.f;
            }
            ob[i] = cvt<TOUT>(v);
        }
    }
}

// dW[co][ci][k] += sum_i da[b][co][i] h[b][ci][i + k - 4];  db[co] += sum_i da[b][co][i]
// CTA: one row b, positions [i0, i0 + WG_SPAN); lane = co, warp = group of CIN/8 input channels
constexpr int WG_SPAN = 1152;

template <class TH, int CIN>
__global__ void __launch_bounds__(256) wgrad_kernel(const TH* __restrict__ h, const float* __restrict__ da, int L,
                                                    float* __restrict__ dW, float* __restrict__ db)
{
    constexpr int CPW = CIN >= 8 ? CIN / 8 : 1;       // input channels per warp
    constexpr int WARPS_USED = CIN >= 8 ? 8 : CIN;
    __shared__ float das[CT][CH + 1];
    __shared__ float hs[CIN][CT + KT - 1];
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool active = warp < WARPS_USED;
    float acc[CPW][KT];
#pragma unroll
    for (int c = 0; c < CPW; ++c)
#pragma unroll
        for (int k = 0; k < KT; ++k) acc[c][k] = 0.f;
    float dbacc = 0.f;
    const int span_end = min(L, (int)(blockIdx.x + 1) * WG_SPAN);
    for (int i0 = blockIdx.x * WG_SPAN; i0 < span_end; i0 += CT) {
        __syncthreads();
        for (int e = threadIdx.x; e < CT * CH; e += 256) {
            int co = e / CT, j = e % CT;
            int pos = i0 + j;
            das[j][co] = pos < span_end ? da[((size_t)b * CH + co) * L + pos] : 0.f;
        }
        for (int e = threadIdx.x; e < CIN * (CT + KT - 1); e += 256) {
            int ci = e / (CT + KT - 1), j = e % (CT + KT - 1);
            int pos = i0 + j - HALF;
            hs[ci][j] = (pos >= 0 && pos < L) ? ld<TH>(h, ((size_t)b * CIN + ci) * L + pos) : 0.f;
        }
        __syncthreads();
        if (active) {
            for (int j = 0; j < CT; j += 4) {
                float d[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] = das[j + q][lane];
                if (warp == 0) dbacc += d[0] + d[1] + d[2] + d[3];
#pragma unroll
                for (int c = 0; c < CPW; ++c) {
                    const float* hr = hs[warp * CPW + c] + j;
                    float hv[4 + KT - 1];
#pragma unroll
                    for (int q = 0; q < 4 + KT - 1; ++q) hv[q] = hr[q];
#pragma unroll
                    for (int k = 0; k < KT; ++k)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[c][k] = fmaf(d[q], hv[q + k], acc[c][k]);
                }
            }
        }
    }
    if (active) {
#pragma unroll
        for (int c = 0; c < CPW; ++c)
#pragma unroll
            for (int k = 0; k < KT; ++k) atomicAdd(&dW[((size_t)lane * CIN + warp * CPW + c) * KT + k], acc[c][k]);
        if (warp == 0) atomicAdd(&db[lane], dbacc);
    }
}

// ---------------------------------------------------------------- head
// per row: z, max/argmax/mean per channel, presence MLP
template <class T>
__global__ void __launch_bounds__(256) head_fwd_kernel(const T* __restrict__ h4, const float* __restrict__ theta, int L,
                                                       float* __restrict__ z, int* __restrict__ amax,
                                                       float* __restrict__ pooled, float* __restrict__ u,
                                                       float* __restrict__ q)
{
    const int b = blockIdx.x;
    const T* hb = h4 + (size_t)b * CH * L;
    __shared__ float w5[CH];
    __shared__ float pool_s[2 * CH];
    __shared__ float u_s[CH];
    if (threadIdx.x < CH) w5[threadIdx.x] = theta[OFF_W5 + threadIdx.x];
    __syncthreads();
    const float b5 = theta[OFF_B5];
    for (int i = threadIdx.x; i < L; i += 256) {
        float s = b5;
#pragma unroll 8
        for (int c = 0; c < CH; ++c) s = fmaf(w5[c], ld<T>(hb, (size_t)c * L + i), s);
        z[(size_t)b * L + i] = s;
    }
    // warp w: channels 4w .. 4w+3
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int cc = 0; cc < 4; ++cc) {
        const int c = warp * 4 + cc;
        float mx = -INFINITY, sum = 0.f;
        int mi = 0;
        for (int i = lane; i < L; i += 32) {
            float v = ld<T>(hb, (size_t)c * L + i);
            if (v > mx) {
                mx = v;
                mi = i;
            }
            sum += v;
        }
        for (int o = 16; o; o >>= 1) {
            float om = __shfl_down_sync(0xffffffffu, mx, o);
            int oi = __shfl_down_sync(0xffffffffu, mi, o);
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (om > mx || (om == mx && oi < mi)) {
                mx = om;
                mi = oi;
            }
        }
        if (lane == 0) {
            pool_s[c] = mx;
            pool_s[CH + c] = sum / L;
            amax[b * CH + c] = mi;
        }
    }
    __syncthreads();
    if (threadIdx.x < CH) {
        const int j = threadIdx.x;
        float s = theta[OFF_BA + j];
        for (int e = 0; e < 2 * CH; ++e) s = fmaf(theta[OFF_WA + j * 2 * CH + e], pool_s[e], s);
        u_s[j] = fmaxf(s, 0.f);
        u[b * CH + j] = u_s[j];
    }
    if (threadIdx.x < 2 * CH) pooled[b * 2 * CH + threadIdx.x] = pool_s[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = theta[OFF_BB];
        for (int j = 0; j < CH; ++j) s = fmaf(theta[OFF_WB + j], u_s[j], s);
        q[b] = s;
    }
}

__device__ __forceinline__ float block_sum(float v, float* red)
{
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__device__ __forceinline__ float block_max(float v, float* red)
{
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    return t;
}

// per row: loss, dz -> da4 (ReLU-masked gradient of h4), head parameter gradients
template <class T>
__global__ void __launch_bounds__(256) head_bwd_kernel(const T* __restrict__ h4, const float* __restrict__ theta, int L,
                                                       int B, const float* __restrict__ z, const int* __restrict__ amax,
                                                       const float* __restrict__ pooled, const float* __restrict__ u,
                                                       const float* __restrict__ q, const float* __restrict__ fpos,
                                                       const float* __restrict__ pres, float* __restrict__ da4,
                                                       float* __restrict__ grad, float* __restrict__ loss)
{
    const int b = blockIdx.x;
    __shared__ float red[8];
    __shared__ float w5[CH], dpool[2 * CH], du_s[CH];
    const float* zb = z + (size_t)b * L;
    const float y = pres[b], f = fpos[b];
    // softmax statistics and target normalisation
    float m = -INFINITY;
    for (int i = threadIdx.x; i < L; i += 256) m = fmaxf(m, zb[i]);
    m = block_max(m, red);
    float se = 0.f, st = 0.f, stz = 0.f;
    for (int i = threadIdx.x; i < L; i += 256) {
        se += __expf(zb[i] - m);
        const float d = (i - f) / SIGMA_T;
        const float t = __expf(-0.5f * d * d);
        st += t;
        stz += t * zb[i];
    }
    se = block_sum(se, red);
    st = block_sum(st, red);
    stz = block_sum(stz, red);
    const float lse = m + logf(se);
    const float invB = 1.f / B;
    const float qb = q[b];
    const float sig = 1.f / (1.f + __expf(-qb));
    const float dq = (sig - y) * invB;
    if (threadIdx.x < CH) w5[threadIdx.x] = theta[OFF_W5 + threadIdx.x];
    if (threadIdx.x == 0) {
        // CE = lse - sum t z / sum t ; BCE in the stable form
        const float ce = (y > 0.f && st > 0.f) ? y * (lse - stz / st) : 0.f;
        const float bce = fmaxf(qb, 0.f) - qb * y + log1pf(__expf(-fabsf(qb)));
        atomicAdd(loss, (bce + ce) * invB);
        atomicAdd(&grad[OFF_BB], dq);
    }
    // presence MLP backward (threads 0..31)
    if (threadIdx.x < CH) {
        const int j = threadIdx.x;
        const float uj = u[b * CH + j];
        atomicAdd(&grad[OFF_WB + j], dq * uj);
        const float du = uj > 0.f ? dq * theta[OFF_WB + j] : 0.f;
        du_s[j] = du;
        atomicAdd(&grad[OFF_BA + j], du);
        for (int e = 0; e < 2 * CH; ++e) atomicAdd(&grad[OFF_WA + j * 2 * CH + e], du * pooled[b * 2 * CH + e]);
    }
    __syncthreads();
    if (threadIdx.x < 2 * CH) {
        float s = 0.f;
        for (int j = 0; j < CH; ++j) s = fmaf(du_s[j], theta[OFF_WA + j * 2 * CH + threadIdx.x], s);
        dpool[threadIdx.x] = s;
    }
    __syncthreads();
    // dz, dw5, db5, da4
    const T* hb = h4 + (size_t)b * CH * L;
    float dw5[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) dw5[c] = 0.f;
    float db5 = 0.f;
    // the location term exists only for gates with a line (its target may lie anywhere,
    // even outside the band, for gates without one)
    const bool loc = y > 0.f && st > 0.f;
    const float inv_st = loc ? 1.f / st : 0.f;
    for (int i = threadIdx.x; i < L; i += 256) {
        const float d = (i - f) / SIGMA_T;
        const float t = loc ? __expf(-0.5f * d * d) * inv_st : 0.f;
        const float dz = loc ? y * (__expf(zb[i] - lse) - t) * invB : 0.f;
        db5 += dz;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const float hv = ld<T>(hb, (size_t)c * L + i);
            dw5[c] = fmaf(dz, hv, dw5[c]);
            float g = w5[c] * dz + dpool[CH + c] / L;
            if (i == amax[b * CH + c]) g += dpool[c];
            da4[((size_t)b * CH + c) * L + i] = hv > 0.f ? g : 0.f;
        }
    }
    db5 = block_sum(db5, red);
    if (threadIdx.x == 0) atomicAdd(&grad[OFF_B5], db5);
    for (int c = 0; c < CH; ++c) {
        float s = block_sum(dw5[c], red);
        if (threadIdx.x == 0) atomicAdd(&grad[OFF_W5 + c], s);
    }
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// per row: position = softmax-weighted mean over the 7 bins around argmax z (+ band_lo),
// presence = sigmoid(q)
__global__ void predict_kernel(const float* __restrict__ z, const float* __restrict__ q, int L, int lo,
                               float* __restrict__ pos, float* __restrict__ pres)
{
    const int b = blockIdx.x;
    const float* zb = z + (size_t)b * L;
    float mx = -INFINITY;
    int mi = 0;
    for (int i = threadIdx.x; i < L; i += 32) {
        if (zb[i] > mx) {
            mx = zb[i];
            mi = i;
        }
    }
    for (int o = 16; o; o >>= 1) {
        float om = __shfl_down_sync(0xffffffffu, mx, o);
        int oi = __shfl_down_sync(0xffffffffu, mi, o);
        if (om > mx || (om == mx && oi < mi)) {
            mx = om;
            mi = oi;
        }
    }
    if (threadIdx.x == 0) {
        const int a = max(0, mi - WIN), e = min(L, mi + WIN + 1);
        double sw = 0, swi = 0;
        for (int i = a; i < e; ++i) {
            const double wgt = exp((double)zb[i] - (double)mx);
            sw += wgt;
            swi += wgt * i;
        }
        pos[b] = (float)(lo + swi / sw);
        pres[b] = 1.f / (1.f + expf(-q[b]));
    }
}

}  // namespace

struct isr_est {
    int nfft = 0, lo = 0, L = 0, max_batch = 0, precision = 0, dev = 0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int64_t step = 0;
    void* wf = nullptr;       // forward working weights (storage type)
    void* wb = nullptr;       // backward-data working weights
    void* act[5] = {};        // x, h1..h4 (storage type)
    float *z = nullptr, *pooled = nullptr, *u = nullptr, *q = nullptr, *loss = nullptr;
    int* amax = nullptr;
    float *da0 = nullptr, *da1 = nullptr; // gradient ping-pong [B][32][L]
};

namespace {

using isr::fail;

#define EST_TRY(expr)                                                                                 \
    do {                                                                                              \
        cudaError_t e_ = (expr);                                                                      \
        if (e_ != cudaSuccess)                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, "%s: %s", #expr, \
                        cudaGetErrorString(e_));                                                      \
    } while (0)

struct Dev {
    int prev = -1;
    explicit Dev(int d)
    {
        cudaGetDevice(&prev);
        cudaSetDevice(d);
    }
    ~Dev()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
isr_status set_smem_attrs()
{
    const int big = (int)conv_smem_bytes(CH);
    EST_TRY(cudaFuncSetAttribute(conv_kernel<T, T, T, T, CH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    EST_TRY(cudaFuncSetAttribute(conv_kernel<float, T, float, T, CH, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    return ISR_OK;
}

template <class T>
isr_status forward_t(isr_est* e, const float* x, int n)
{
    const int L = e->L;
    cudaStream_t s = e->stream;
    T* act[5];
    for (int i = 0; i < 5; ++i) act[i] = static_cast<T*>(e->act[i]);
    const size_t nx = (size_t)n * L;
    cast_kernel<T><<<(unsigned)std::min<size_t>((nx + 255) / 256, 4096), 256, 0, s>>>(x, nx, act[0]);
    relayout_kernel<T><<<(CH * KT + 3 * CH * CH * KT + 255) / 256, 256, 0, s>>>(e->theta, static_cast<T*>(e->wf),
                                                                                 static_cast<T*>(e->wb));
    const T* wf = static_cast<const T*>(e->wf);
    dim3 grid((L + CT - 1) / CT, n);
    conv_kernel<T, T, T, T, 1, true><<<grid, 256, conv_smem_bytes(1), s>>>(act[0], wf, e->theta + OFF_B1, nullptr,
                                                                            L, act[1]);
    for (int l = 2; l <= 4; ++l)
        conv_kernel<T, T, T, T, CH, true><<<grid, 256, conv_smem_bytes(CH), s>>>(act[l - 1], wf + CH * KT + (size_t)(l - 2) * CH * CH * KT,
                                                              e->theta + b_off(l), nullptr, L, act[l]);
    head_fwd_kernel<T><<<n, 256, 0, s>>>(act[4], e->theta, L, e->z, e->amax, e->pooled, e->u, e->q);
    EST_TRY(cudaGetLastError());
    return ISR_OK;
}

template <class T>
isr_status backward_t(isr_est* e, int n, const float* fpos, const float* pres)
{
    const int L = e->L;
    cudaStream_t s = e->stream;
    T* act[5];
    for (int i = 0; i < 5; ++i) act[i] = static_cast<T*>(e->act[i]);
    EST_TRY(cudaMemsetAsync(e->grad, 0, sizeof(float) * NPARAM, s));
    EST_TRY(cudaMemsetAsync(e->loss, 0, sizeof(float), s));
    head_bwd_kernel<T><<<n, 256, 0, s>>>(act[4], e->theta, L, n, e->z, e->amax, e->pooled, e->u, e->q, fpos, pres,
                                         e->da0, e->grad, e->loss);
    const T* wbk = static_cast<const T*>(e->wb);
    float* da = e->da0;
    float* dn = e->da1;
    dim3 gw((L + WG_SPAN - 1) / WG_SPAN, n);
    dim3 gc((L + CT - 1) / CT, n);
    for (int l = 4; l >= 1; --l) {
        if (l == 1) {
            wgrad_kernel<T, 1><<<gw, 256, 0, s>>>(act[0], da, L, e->grad + OFF_W1, e->grad + OFF_B1);
        } else {
            wgrad_kernel<T, CH><<<gw, 256, 0, s>>>(act[l - 1], da, L, e->grad + w_off(l), e->grad + b_off(l));
            // gradient into the layer below, masked by its ReLU: da_{l-1} = (W_l^T * da_l) (h_{l-1} > 0)
            conv_kernel<float, T, float, T, CH, false><<<gc, 256, conv_smem_bytes(CH), s>>>(
                da, wbk + (size_t)(l - 2) * CH * CH * KT, nullptr, act[l - 1], L, dn);
            std::swap(da, dn);
        }
    }
    EST_TRY(cudaGetLastError());
    return ISR_OK;
}

bool dev_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

isr_status check_batch(isr_est* e, const float* x, int n)
{
    if (!e || !x) return fail(ISR_ERR_INVALID_ARG, "estimator and x must not be NULL");
    if (n < 1 || n > e->max_batch) return fail(ISR_ERR_INVALID_ARG, "batch %d outside [1, %d]", n, e->max_batch);
    if (!dev_ptr(x)) return fail(ISR_ERR_INVALID_ARG, "x must be device memory");
    return ISR_OK;
}

}  // namespace

extern "C" {

isr_status isr_est_create(isr_est** out, int32_t nfft, int32_t band_lo, int32_t band_len, int32_t max_batch,
                          int32_t precision, int32_t device, void* stream)
{
    isr::clear_error();
    if (!out) return fail(ISR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nfft < 8 || band_lo < 0 || band_len < 16 || band_lo + band_len > nfft || max_batch < 1)
        return fail(ISR_ERR_INVALID_ARG, "need 0 <= band_lo, band_len >= 16, band_lo + band_len <= nfft, max_batch >= 1");
    if (precision != ISR_EST_FP32 && precision != ISR_EST_BF16) return fail(ISR_ERR_UNSUPPORTED, "unknown precision");
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(ISR_ERR_CUDA, "no current device");
    Dev guard(dev);
    isr_est* e = new (std::nothrow) isr_est();
    if (!e) return fail(ISR_ERR_NO_MEMORY, "host allocation failed");
    e->nfft = nfft;
    e->lo = band_lo;
    e->L = band_len;
    e->max_batch = max_batch;
    e->precision = precision;
    e->dev = dev;
    e->stream = static_cast<cudaStream_t>(stream);
    const size_t es = precision == ISR_EST_BF16 ? 2 : 4;
    const size_t B = max_batch, L = band_len;
    cudaError_t r = cudaSuccess;
    auto A = [&](void** p, size_t bytes) {
        if (r == cudaSuccess) r = cudaMalloc(p, bytes);
    };
    A((void**)&e->theta, 4 * NPARAM);
    A((void**)&e->m, 4 * NPARAM);
    A((void**)&e->v, 4 * NPARAM);
    A((void**)&e->grad, 4 * NPARAM);
    A(&e->wf, es * (CH * KT + 3 * CH * CH * KT));
    A(&e->wb, es * 3 * CH * CH * KT);
    A(&e->act[0], es * B * L);
    for (int i = 1; i < 5; ++i) A(&e->act[i], es * B * CH * L);
    A((void**)&e->z, 4 * B * L);
    A((void**)&e->pooled, 4 * B * 2 * CH);
    A((void**)&e->u, 4 * B * CH);
    A((void**)&e->q, 4 * B);
    A((void**)&e->loss, 4);
    A((void**)&e->amax, 4 * B * CH);
    A((void**)&e->da0, 4 * B * CH * L);
    A((void**)&e->da1, 4 * B * CH * L);
    if (r == cudaSuccess) r = cudaMemset(e->theta, 0, 4 * NPARAM);
    if (r == cudaSuccess) r = cudaMemset(e->m, 0, 4 * NPARAM);
    if (r == cudaSuccess) r = cudaMemset(e->v, 0, 4 * NPARAM);
    if (r == cudaSuccess) {
        isr_status st = precision == ISR_EST_BF16 ? set_smem_attrs<__nv_bfloat16>() : set_smem_attrs<float>();
        if (st != ISR_OK) {
            isr_est_destroy(e);
            return st;
        }
    }
    if (r != cudaSuccess) {
        isr_est_destroy(e);
        return fail(r == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, "allocation failed: %s",
                    cudaGetErrorString(r));
    }
    *out = e;
    return ISR_OK;
}

isr_status isr_est_set_params(isr_est* e, const float* params)
{
    if (!e || !params) return fail(ISR_ERR_INVALID_ARG, "NULL argument");
    Dev guard(e->dev);
    EST_TRY(cudaMemcpyAsync(e->theta, params, 4 * NPARAM, cudaMemcpyDefault, e->stream));
    EST_TRY(cudaMemsetAsync(e->m, 0, 4 * NPARAM, e->stream));
    EST_TRY(cudaMemsetAsync(e->v, 0, 4 * NPARAM, e->stream));
    EST_TRY(cudaStreamSynchronize(e->stream));
    e->step = 0;
    return ISR_OK;
}

isr_status isr_est_get_params(isr_est* e, float* params)
{
    if (!e || !params) return fail(ISR_ERR_INVALID_ARG, "NULL argument");
    Dev guard(e->dev);
    EST_TRY(cudaMemcpyAsync(params, e->theta, 4 * NPARAM, cudaMemcpyDefault, e->stream));
    EST_TRY(cudaStreamSynchronize(e->stream));
    return ISR_OK;
}

isr_status isr_est_features(isr_est* e, const float* spectra, int32_t n, float* x)
{
    if (!e || !spectra || !x || n < 1) return fail(ISR_ERR_INVALID_ARG, "bad arguments");
    Dev guard(e->dev);
    features_kernel<<<n, 256, 0, e->stream>>>(spectra, e->nfft, e->lo, e->L, x);
    EST_TRY(cudaGetLastError());
    return ISR_OK;
}

isr_status isr_est_grad(isr_est* e, const float* x, int32_t n, const float* line_bin, const float* present,
                        float* loss, float* grad)
{
    isr_status st = check_batch(e, x, n);
    if (st != ISR_OK) return st;
    if (!line_bin || !present) return fail(ISR_ERR_INVALID_ARG, "labels must not be NULL");
    Dev guard(e->dev);
    st = e->precision == ISR_EST_BF16 ? forward_t<__nv_bfloat16>(e, x, n) : forward_t<float>(e, x, n);
    if (st == ISR_OK)
        st = e->precision == ISR_EST_BF16 ? backward_t<__nv_bfloat16>(e, n, line_bin, present)
                                          : backward_t<float>(e, n, line_bin, present);
    if (st != ISR_OK) return st;
    if (grad) EST_TRY(cudaMemcpyAsync(grad, e->grad, 4 * NPARAM, cudaMemcpyDefault, e->stream));
    if (loss) EST_TRY(cudaMemcpyAsync(loss, e->loss, 4, cudaMemcpyDefault, e->stream));
    EST_TRY(cudaStreamSynchronize(e->stream));
    return ISR_OK;
}

isr_status isr_est_train_step(isr_est* e, const float* x, int32_t n, const float* line_bin, const float* present,
                              float lr, float* loss)
{
    isr_status st = check_batch(e, x, n);
    if (st != ISR_OK) return st;
    if (!line_bin || !present || !(lr > 0.f)) return fail(ISR_ERR_INVALID_ARG, "labels NULL or lr <= 0");
    Dev guard(e->dev);
    st = e->precision == ISR_EST_BF16 ? forward_t<__nv_bfloat16>(e, x, n) : forward_t<float>(e, x, n);
    if (st == ISR_OK)
        st = e->precision == ISR_EST_BF16 ? backward_t<__nv_bfloat16>(e, n, line_bin, present)
                                          : backward_t<float>(e, n, line_bin, present);
    if (st != ISR_OK) return st;
    e->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, (float)e->step)), c2 = 1.f / (1.f - powf(b2, (float)e->step));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, e->stream>>>(e->theta, e->grad, e->m, e->v, NPARAM, lr, b1, b2, 1e-8f,
                                                              c1, c2);
    EST_TRY(cudaGetLastError());
    if (loss) {
        EST_TRY(cudaMemcpyAsync(loss, e->loss, 4, cudaMemcpyDefault, e->stream));
        EST_TRY(cudaStreamSynchronize(e->stream));
    }
    return ISR_OK;
}

isr_status isr_est_predict(isr_est* e, const float* x, int32_t n, float* line_bin, float* presence)
{
    isr_status st = check_batch(e, x, n);
    if (st != ISR_OK) return st;
    if (!line_bin || !presence) return fail(ISR_ERR_INVALID_ARG, "outputs must not be NULL");
    Dev guard(e->dev);
    st = e->precision == ISR_EST_BF16 ? forward_t<__nv_bfloat16>(e, x, n) : forward_t<float>(e, x, n);
    if (st != ISR_OK) return st;
    predict_kernel<<<n, 32, 0, e->stream>>>(e->z, e->q, e->L, e->lo, line_bin, presence);
    EST_TRY(cudaGetLastError());
    return ISR_OK;
}

void isr_est_destroy(isr_est* e)
{
    if (!e) return;
    Dev guard(e->dev);
    cudaStreamSynchronize(e->stream);
    void* ptrs[] = {e->theta, e->m, e->v, e->grad, e->wf, e->wb, e->act[0], e->act[1], e->act[2], e->act[3],
                    e->act[4], e->z, e->pooled, e->u, e->q, e->loss, e->amax, e->da0, e->da1};
    for (void* p : ptrs) cudaFree(p);
    cudaGetLastError();
    delete e;
}

}  // extern "C"
