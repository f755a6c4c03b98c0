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
#include <type_traits>

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
// whether v, once stored as T, reads back above zero (the test of the backward pass's ReLU mask);
// for BF16 the sign and magnitude bits of the stored pattern: positive and not zero
template <class T> __device__ __forceinline__ bool positive_as_stored(float v);
template <> __device__ __forceinline__ bool positive_as_stored<float>(float v) { return v > 0.f; }
template <> __device__ __forceinline__ bool positive_as_stored<__nv_bfloat16>(float v)
{
    return (int16_t)__bfloat16_as_ushort(__float2bfloat16_rn(v)) > 0;
}

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
// flipped transpose, [co][k'][ci] = W[co][ci][8 - k'] (both in the storage type); with
// tf and tb (tensor-core path, layers 2-4) also the GEMM rows [co][k][ci] of the forward
// weights and [ci][k'][co] of the flipped transpose
template <class T>
__global__ void relayout_kernel(const float* __restrict__ theta, T* __restrict__ wf, T* __restrict__ wb,
                                T* __restrict__ tf, T* __restrict__ tb)
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
    if (l > 1 && tf) {
        tf[(size_t)(l - 2) * n + ((size_t)co * KT + k) * CH + ci] = cvt<T>(w);
        tb[(size_t)(l - 2) * n + ((size_t)ci * KT + (KT - 1 - k)) * CH + co] = cvt<T>(w);
    }
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

// ---------------------------------------------------------------- tensor-core convolution
// Layers 2-4 (32 -> 32 channels) with BF16 storage, as a GEMM on the warp-level tensor-core
// instruction mma.m16n8k16 (BF16 operands, FP32 accumulation):
//   out[co][i] = sum_kk A[co][kk] B[kk][i],   kk = 32 k + ci,   B[kk][i] = in[ci][i + k - 4],
// with A the weights in [co][k][ci] order (K = 288).  B is never formed: the CTA stages its
// input as a position-major tile, one 80-byte row of 32 channels per position (halo included),
// so the 8 x 8 blocks of B at tap k are rows i + k of that tile and ldmatrix reads them as they
// are.  Row pitches of 80 B (tile) and 592 B (weights) put the eight rows an ldmatrix reads on
// 32 distinct banks.  The backward-data convolution is the same GEMM on the flipped transposed
// weights; its FP32 input (the gradient) is split into two BF16 parts, hi + lo, and both are
// multiplied, so the products keep ~16 bits of the gradient and the FP32 accumulation.
// CTA: CF_CT = 512 positions x 32 output channels, 16 warps; warp w: positions [32 w, 32 w + 32),
// all channels (a CTA stages the 18 KB of weights once per 512 positions).
constexpr int CF_CT = 512;                 // positions per convolution CTA
constexpr int CF_THREADS = 16 * 32;
constexpr int CF_XW = CF_CT + KT - 1;      // staged positions, halo included
constexpr int CF_OR = CF_CT + 8;           // output staging row (elements)
constexpr int TC_CT = 256;                 // positions per weight-gradient chunk
constexpr int TC_XW = TC_CT + KT - 1;
constexpr int TC_XR = CH + 8;              // bf16 per staged position (80 B)
constexpr int TC_K = KT * CH;              // GEMM depth
constexpr int TC_WR = TC_K + 8;            // bf16 per staged weight row (592 B)
constexpr size_t tc_smem_bytes(bool fwd)
{
    return (size_t)2 * ((fwd ? 1 : 2) * CF_XW * TC_XR + CH * TC_WR);
}
static_assert(CF_CT == CF_THREADS, "a warp per 32 positions");
static_assert((size_t)CH * CF_OR * 4 <= (size_t)2 * 2 * CF_XW * TC_XR, "FP32 output tile fits the input tiles");
static_assert((size_t)CH * CF_OR * 2 <= (size_t)2 * CF_XW * TC_XR, "BF16 output tile fits the input tile");

// BF16 storage runs the 32 -> 32 channel convolutions on the tensor cores
template <class T> constexpr bool kTensorConv = false;
template <> constexpr bool kTensorConv<__nv_bfloat16> = true;

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// Position-major staging of one row's 32 channels, positions i0 - 4 + j for j < XW (zero
// outside [0, L)): xs[j][c] at a TC_XR-element pitch.  With L a multiple of 8 every channel row
// is read in 16-byte pieces along the positions (lane = channel, so the 2-byte shared stores of
// a warp fill 64 contiguous bytes); otherwise two channels per 32-bit word, element by element.
template <int XW>
__device__ __forceinline__ void stage_act_tile(const unsigned short* __restrict__ rows, int L, int i0,
                                               unsigned short* xs)
{
    static_assert(XW % 8 == 0 && XW * (CH / 2) % 32 == 0, "staging pieces tile the halo'd window");
    if ((L & 7) == 0) {
        // pieces v cover positions i0 - 8 + 8 v .. +7, v < XW / 8 + 1
        for (int e = threadIdx.x; e < CH * (XW / 8 + 1); e += blockDim.x) {
            const int c = e & (CH - 1), v = e / CH;
            const int pos0 = i0 - 8 + 8 * v;
            const unsigned short* src = rows + (size_t)c * L;
            unsigned short t[8];
            if (pos0 >= 0 && pos0 + 8 <= L) {
                const uint4 q = *reinterpret_cast<const uint4*>(src + pos0);
                const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    t[2 * k] = (unsigned short)(w[k] & 0xffffu);
                    t[2 * k + 1] = (unsigned short)(w[k] >> 16);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) t[k] = (pos0 + k >= 0 && pos0 + k < L) ? src[pos0 + k] : 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int j = 8 * v - HALF + k;
                if (j >= 0 && j < XW) xs[j * TC_XR + c] = t[k];
            }
        }
    } else {
        uint32_t* xw = reinterpret_cast<uint32_t*>(xs);
        for (int w = threadIdx.x; w < XW * (CH / 2); w += blockDim.x) {
            const int grp = w >> 5, l = w & 31;
            const int j = (grp >> 2) * 8 + (l & 7), cp = (grp & 3) * 4 + (l >> 3);
            const int pos = i0 - HALF + j;
            const size_t o = (size_t)(2 * cp) * L + pos;
            const bool inside = pos >= 0 && pos < L;
            const uint32_t v0 = inside ? rows[o] : 0u, v1 = inside ? rows[o + L] : 0u;
            xw[j * (TC_XR / 2) + cp] = v0 | (v1 << 16);
        }
    }
}

// The same tile from FP32 rows, split into BF16 hi and lo tiles (with L a multiple of 4, read
// in 16-byte pieces; positions i0 - 4 + 4 v .. +3, v < XW / 4).
template <int XW>
__device__ __forceinline__ void stage_split_tile(const float* __restrict__ rows, int L, int i0, unsigned short* xh,
                                                 unsigned short* xl)
{
    for (int e = threadIdx.x; e < CH * (XW / 4); e += blockDim.x) {
        const int c = e & (CH - 1), v = e / CH;
        const int pos0 = i0 - HALF + 4 * v;
        const float* src = rows + (size_t)c * L;
        float t[4];
        if ((L & 3) == 0 && pos0 >= 0 && pos0 + 4 <= L) {
            const float4 q = *reinterpret_cast<const float4*>(src + pos0);
            t[0] = q.x; t[1] = q.y; t[2] = q.z; t[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] = (pos0 + k >= 0 && pos0 + k < L) ? src[pos0 + k] : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 4; k += 2) {
            uint32_t hi, lo;
            isr::split2<true>(t[k], t[k + 1], hi, lo);
            const int j = 4 * v + k;
            xh[j * TC_XR + c] = (unsigned short)(hi & 0xffffu);
            xh[(j + 1) * TC_XR + c] = (unsigned short)(hi >> 16);
            xl[j * TC_XR + c] = (unsigned short)(lo & 0xffffu);
            xl[(j + 1) * TC_XR + c] = (unsigned short)(lo >> 16);
        }
    }
}


// FWD: in = BF16 activations [B][32][L], out = BF16 relu(conv + bias).
// !FWD: in = FP32 gradient [B][32][L], out = FP32 conv masked by mask > 0 (BF16 activations
// of the layer below), no bias.
template <bool FWD>
__global__ void __launch_bounds__(CF_THREADS) conv_tc_kernel(const void* __restrict__ in, const __nv_bfloat16* __restrict__ wt,
                                                      const float* __restrict__ bias,
                                                      const __nv_bfloat16* __restrict__ mask, int L,
                                                      void* __restrict__ out)
{
    constexpr int NX = FWD ? 1 : 2;                    // staged input parts
    constexpr int XWORDS = CF_XW * TC_XR / 2;          // 32-bit words per staged part
    extern __shared__ __align__(16) unsigned char tc_smem[];
    uint32_t* xs = reinterpret_cast<uint32_t*>(tc_smem);
    uint4* ws = reinterpret_cast<uint4*>(tc_smem + (size_t)4 * NX * XWORDS);
    const int b = blockIdx.y, i0 = blockIdx.x * CF_CT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // weights: [co][288] rows, 16-byte copies into 592-byte rows
    const uint4* w4 = reinterpret_cast<const uint4*>(wt);
    for (int e = tid; e < CH * (TC_K / 8); e += CF_THREADS) {
        const int co = e / (TC_K / 8), q = e - co * (TC_K / 8);
        ws[co * (TC_WR / 8) + q] = w4[e];
    }
    // input: position-major tile of positions i0 - 4 + j (FP32 input: hi and lo tiles)
    if constexpr (FWD)
        stage_act_tile<CF_XW>(static_cast<const unsigned short*>(in) + (size_t)b * CH * L, L, i0,
                              reinterpret_cast<unsigned short*>(xs));
    else
        stage_split_tile<CF_XW>(static_cast<const float*>(in) + (size_t)b * CH * L, L, i0,
                                reinterpret_cast<unsigned short*>(xs), reinterpret_cast<unsigned short*>(xs + XWORDS));
    __syncthreads();

    float acc[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
    const uint32_t xs_s = isr::smem_u32(xs), ws_s = isr::smem_u32(ws);
    const int r8 = lane & 7, mq = lane >> 3;
    // ldmatrix rows: weights, matrix mq = (rows +8 if mq odd, columns +8 if mq >= 2), giving
    // the A fragment registers in order; tile, matrix mq = (n-tile mq / 2, channels +8 if mq
    // odd), giving (b0, b1) of two n-tiles
    const uint32_t a_row = ws_s + 2u * (uint32_t)(((mq & 1) * 8 + r8) * TC_WR + (mq >> 1) * 8);
    const uint32_t b_row = xs_s + 2u * (uint32_t)((warp * 32 + (mq >> 1) * 8 + r8) * TC_XR + (mq & 1) * 8);
#pragma unroll 2
    for (int s = 0; s < TC_K / 16; ++s) {              // k-step s: tap s / 2, channels 16 (s % 2) ..
        const int tap = s >> 1, ci0 = (s & 1) * 16;
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) ldsm_x4(a[mt], a_row + 2u * (uint32_t)(mt * 16 * TC_WR + s * 16));
#pragma unroll
        for (int part = 0; part < NX; ++part) {
            uint32_t bq[2][4];
#pragma unroll
            for (int p = 0; p < 2; ++p)
                ldsm_x4(bq[p], b_row + 4u * (uint32_t)(part * XWORDS) + 2u * (uint32_t)((p * 16 + tap) * TC_XR + ci0));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const uint4 af = make_uint4(a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    isr::mma16816<true>(acc[mt][nt], af, bq[nt >> 1][(nt & 1) * 2], bq[nt >> 1][(nt & 1) * 2 + 1]);
            }
        }
    }
    __syncthreads();   // every warp is done with the tiles: the output tile reuses them

    // accumulator (mt, nt, q): channel mt 16 + g + 8 (q >= 2), position 32 warp + 8 nt + 2 t + (q & 1)
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int co = mt * 16 + h * 8 + g;
            const float bv = FWD ? __ldg(bias + co) : 0.f;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int pl = warp * 32 + nt * 8 + 2 * t4;
                const float v0 = acc[mt][nt][2 * h] + bv, v1 = acc[mt][nt][2 * h + 1] + bv;
                if constexpr (FWD)
                    reinterpret_cast<uint32_t*>(tc_smem)[(co * CF_OR + pl) / 2] =
                        isr::pack2<true>(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
                else
                    reinterpret_cast<float2*>(tc_smem)[(co * CF_OR + pl) / 2] = make_float2(v0, v1);
            }
        }
    __syncthreads();
    // coalesced rows: warp w writes channels w and w + 16
    for (int co = warp; co < CH; co += CF_THREADS / 32) {
        const size_t row = ((size_t)b * CH + co) * L;
        for (int q = lane; q < CF_CT; q += 32) {
            const int i = i0 + q;
            if (i >= L) break;
            if constexpr (FWD) {
                static_cast<__nv_bfloat16*>(out)[row + i] = reinterpret_cast<const __nv_bfloat16*>(tc_smem)[co * CF_OR + q];
            } else {
                const float v = reinterpret_cast<const float*>(tc_smem)[co * CF_OR + q];
                static_cast<float*>(out)[row + i] = __bfloat162float(mask[row + i]) > 0.f ? v : 0.f;
            }
        }
    }
}

// ---------------------------------------------------------------- tcgen05 convolution
// Layers 2-4 with BF16 storage on the fifth-generation tensor cores: the same GEMM as
// conv_tc_kernel with positions as M,
//   D[i][co] = sum_{k, ci} X[i + k - 4][ci] W[co][ci][k]     (M = 128 positions per tile, N = 32, K = 288),
// issued by one thread as tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32
// accumulator in tensor memory).  The input tile is staged position-major in four "planes" of
// eight channels, [rows][8 ch] with 16-byte rows, so every 8 x 16-byte core matrix of the
// K-major no-swizzle layout is eight consecutive rows of one plane (SBO = 128 B between 8-row
// groups, LBO = plane stride between the two 8-channel halves of a K = 16 step), and the A
// operand of tap k is the same tile started k rows later: descriptor start + 16 k bytes.  The
// weights are 36 planes [tap][8-channel group] of [32 co][8 ci].  A tile is TPC M tiles of 128
// positions (128 TPC threads; 18 MMAs per M tile, 36 in the backward-data pass, which multiplies
// the hi and lo parts of its FP32 input) and 32 TPC TMEM columns; warp w reads M tile w / 4 at its
// lane quarter and writes the epilogue (bias + ReLU to BF16, or the FP32 gradient masked by the
// layer below) straight from registers, one coalesced 32-position store per channel.  Every
// thread issues all of its staging loads before its first shared store.
// TPC = M tiles of 128 positions per tile (1, 2 or 4): 128 TPC threads, four warps per M tile
template <int TPC> struct C5 {
    static constexpr int CT = 128 * TPC;                   // positions per CTA
    static constexpr int THREADS = 128 * TPC;
    static constexpr int XW = CT + KT - 1;                 // staged rows (halo included)
    static constexpr int PLANE = XW * 16 + 16;             // bytes per channel plane (+16: planes 4 banks apart)
    static constexpr int PART = 4 * PLANE;                 // one staged part (32 channels)
    static constexpr int COLS = TPC <= 1 ? 32 : 32 * TPC;  // TMEM columns: one N = 32 tile per M tile
    // the persistent convolution: two staging buffers of 1 (forward) or 2 (hi, lo) parts, the
    // weight planes, two mbarriers and the TMEM address slot
    static constexpr size_t smem(bool fwd) { return (size_t)2 * (fwd ? 1 : 2) * PART + KT * 4 * 512 + 32; }
    static_assert(PLANE % 16 == 0 && (PLANE / 4) % 32 == 4, "planes 16-byte aligned, four banks apart");
};
constexpr int C5_WBYTES = KT * 4 * 512;                    // weight planes
constexpr int C5_TPC = 2;                                  // the launched shape

// 16-bit index of (row j, channel c) in a staged part of plane size PLANE bytes
template <int PLANE>
__device__ __forceinline__ int c5_idx(int j, int c) { return (c >> 3) * (PLANE / 2) + j * 8 + (c & 7); }

// Staging of one row's 32 channels, positions i0 - 4 + j for j < XW (zero outside [0, L)), into
// planes, in two phases so that a pipelined caller keeps the global loads in flight while it does
// other work: c5_act_load issues every global load of the thread into registers, c5_act_store
// writes them to the planes.  When L is not a multiple of 8 the 16-byte loads do not apply:
// c5_act_load does nothing and c5_act_store stages word by word.  Called by THREADS threads.
// NT = the calling threads (C5<TPC>::THREADS unless a caller stages with more).
template <int TPC, int NT = C5<TPC>::THREADS> struct C5Act {
    static constexpr int NITEM = CH * (C5<TPC>::XW / 8 + 1);   // (channel, 8-position block) pieces
    static constexpr int PER = (NITEM + NT - 1) / NT;
};

template <int TPC, int NT = C5<TPC>::THREADS>
__device__ __forceinline__ void c5_act_load(const unsigned short* __restrict__ rows, int L, int i0,
                                            uint4 (&q)[C5Act<TPC, NT>::PER])
{
    constexpr int NITEM = C5Act<TPC, NT>::NITEM, PER = C5Act<TPC, NT>::PER, THREADS = NT;
    if ((L & 7) != 0) return;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * THREADS;
        const int c = e & (CH - 1), v = e / CH;
        const int pos0 = i0 - 8 + 8 * v;   // a multiple of 8 (i0 is): the piece lies inside [0, L) or outside
        q[u] = make_uint4(0u, 0u, 0u, 0u);
        if (e < NITEM && pos0 >= 0 && pos0 + 8 <= L) q[u] = *reinterpret_cast<const uint4*>(rows + (size_t)c * L + pos0);
    }
}

template <int TPC, int NT = C5<TPC>::THREADS>
__device__ __forceinline__ void c5_act_store(const unsigned short* __restrict__ rows, int L, int i0,
                                             const uint4 (&q)[C5Act<TPC, NT>::PER], unsigned short* xs)
{
    using G = C5<TPC>;
    constexpr int XW = G::XW, THREADS = NT, P = G::PLANE;
    constexpr int NITEM = C5Act<TPC, NT>::NITEM, PER = C5Act<TPC, NT>::PER;
    static_assert(NITEM % 32 == 0 && THREADS % 32 == 0, "whole warps per item round (the shuffles)");
    if ((L & 7) == 0) {
        // lane = channel c; lanes c, c ^ 1 swap halves of their 8 positions, so that the even lane
        // holds positions 0-3 and the odd lane positions 4-7 of both channels and writes one 32-bit
        // word (channels c & ~1, c | 1) per position: per store the even lanes fill rows j (16
        // banks over the four planes) and the odd lanes rows j + 4 (the other 16)
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = threadIdx.x + u * THREADS;
            if (e >= NITEM) break;
            const int c = e & (CH - 1), v = e / CH, odd = c & 1;
            const uint32_t r0 = __shfl_xor_sync(0xffffffffu, odd ? q[u].x : q[u].z, 1);
            const uint32_t r1 = __shfl_xor_sync(0xffffffffu, odd ? q[u].y : q[u].w, 1);
            const uint32_t m0 = odd ? q[u].z : q[u].x, m1 = odd ? q[u].w : q[u].y;
            const uint32_t e0 = odd ? r0 : m0, o0 = odd ? m0 : r0;   // even / odd channel, positions 0-1 of the half
            const uint32_t e1 = odd ? r1 : m1, o1 = odd ? m1 : r1;   // positions 2-3
            const uint32_t w[4] = {__byte_perm(e0, o0, 0x5410), __byte_perm(e0, o0, 0x7632),
                                   __byte_perm(e1, o1, 0x5410), __byte_perm(e1, o1, 0x7632)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int j = 8 * v - HALF + 4 * odd + k;
                if (j >= 0 && j < XW) *reinterpret_cast<uint32_t*>(xs + c5_idx<P>(j, c & ~1)) = w[k];
            }
        }
    } else {
        for (int e = threadIdx.x; e < XW * (CH / 2); e += THREADS) {
            const int j = e / (CH / 2), cp = e - j * (CH / 2);
            const int pos = i0 - HALF + j;
            const size_t o = (size_t)(2 * cp) * L + pos;
            const bool inside = pos >= 0 && pos < L;
            const uint32_t v0 = inside ? rows[o] : 0u, v1 = inside ? rows[o + L] : 0u;
            *reinterpret_cast<uint32_t*>(xs + c5_idx<P>(j, 2 * cp)) = v0 | (v1 << 16);
        }
    }
}

template <int TPC>
__device__ __forceinline__ void c5_stage_act(const unsigned short* __restrict__ rows, int L, int i0, unsigned short* xs)
{
    uint4 q[C5Act<TPC>::PER];
    c5_act_load<TPC>(rows, L, i0, q);
    c5_act_store<TPC>(rows, L, i0, q, xs);
}

// The same from FP32 rows, split into BF16 hi (part xh) and lo (part xl), in the same two phases.
template <int TPC> struct C5Split {
    static constexpr int NITEM = CH * (C5<TPC>::XW / 4);        // (channel, 4-position block) pieces
    static constexpr int PER = (NITEM + C5<TPC>::THREADS - 1) / C5<TPC>::THREADS;
};

template <int TPC>
__device__ __forceinline__ void c5_split_load(const float* __restrict__ rows, int L, int i0,
                                              float4 (&q)[C5Split<TPC>::PER])
{
    constexpr int NITEM = C5Split<TPC>::NITEM, PER = C5Split<TPC>::PER, THREADS = C5<TPC>::THREADS;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * THREADS;
        const int c = e & (CH - 1), v = e / CH;
        const int pos0 = i0 - HALF + 4 * v;
        const float* src = rows + (size_t)c * L;
        q[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < NITEM) {
            if ((L & 3) == 0 && pos0 >= 0 && pos0 + 4 <= L) {
                q[u] = *reinterpret_cast<const float4*>(src + pos0);
            } else {
                q[u].x = (pos0 >= 0 && pos0 < L) ? src[pos0] : 0.f;
                q[u].y = (pos0 + 1 >= 0 && pos0 + 1 < L) ? src[pos0 + 1] : 0.f;
                q[u].z = (pos0 + 2 >= 0 && pos0 + 2 < L) ? src[pos0 + 2] : 0.f;
                q[u].w = (pos0 + 3 >= 0 && pos0 + 3 < L) ? src[pos0 + 3] : 0.f;
            }
        }
    }
}

template <int TPC>
__device__ __forceinline__ void c5_split_store(const float4 (&q)[C5Split<TPC>::PER], unsigned short* xh,
                                               unsigned short* xl)
{
    constexpr int NITEM = C5Split<TPC>::NITEM, PER = C5Split<TPC>::PER, THREADS = C5<TPC>::THREADS;
    constexpr int P = C5<TPC>::PLANE;
    static_assert(NITEM % 32 == 0 && THREADS % 32 == 0, "whole warps per item round (the shuffles)");
    static_assert((C5<TPC>::PART / 4) % 32 == 16, "the hi and lo parts 16 banks apart");
    // lane = channel c; lanes c, c ^ 1 swap parts: the even lane gets the hi words of both
    // channels and the odd lane the lo words, and each writes one 32-bit word (channels c & ~1,
    // c | 1) per position, so every store fills rows j of both parts, 32 distinct banks
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = threadIdx.x + u * THREADS;
        if (e >= NITEM) break;
        const int c = e & (CH - 1), v = e / CH, odd = c & 1;
        uint32_t hi0, lo0, hi1, lo1;
        isr::split2<true>(q[u].x, q[u].y, hi0, lo0);
        isr::split2<true>(q[u].z, q[u].w, hi1, lo1);
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, odd ? hi0 : lo0, 1);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, odd ? hi1 : lo1, 1);
        const uint32_t m0 = odd ? lo0 : hi0, m1 = odd ? lo1 : hi1;
        const uint32_t e0 = odd ? r0 : m0, o0 = odd ? m0 : r0;   // even / odd channel, positions 0-1
        const uint32_t e1 = odd ? r1 : m1, o1 = odd ? m1 : r1;   // positions 2-3
        const uint32_t w[4] = {__byte_perm(e0, o0, 0x5410), __byte_perm(e0, o0, 0x7632),
                               __byte_perm(e1, o1, 0x5410), __byte_perm(e1, o1, 0x7632)};
        unsigned short* x = odd ? xl : xh;
#pragma unroll
        for (int k = 0; k < 4; ++k) *reinterpret_cast<uint32_t*>(x + c5_idx<P>(4 * v + k, c & ~1)) = w[k];
    }
}

// FWD: in = BF16 activations [B][32][L], out = BF16 relu(conv + bias); with BITS (a training pass)
//   also the ReLU mask, bits[b * L + i] bit co = (stored output [b][co][i] > 0).
// !FWD: in = FP32 gradient [B][32][L], out = FP32 conv masked by the layer below's ReLU, read as
//   those bits (one word per position, loaded before the epilogue waits for the tile's MMAs), no bias.
// wt: GEMM rows [out channel][tap][in channel] (BF16), as for conv_tc_kernel.
// Persistent: CTA c takes tiles c, c + gridDim.x, ... of the n_rows x ceil(L / CT) tiles (row-major)
// with a two-deep pipeline over two staging buffers, two TMEM accumulators and two mbarriers.  In
// the iteration of tile t: the global loads of tile t + gridDim.x are issued into registers, the
// epilogue of tile t runs (its MMAs were issued one iteration earlier), the registers are written
// to the other staging buffer (whose MMAs completed before the previous epilogue), and after one
// barrier thread 0 issues that tile's MMAs into the other accumulator.  The weights are staged
// once per CTA.  A wait that runs out of polls ends the CTA's loop (the vote at the barrier makes
// that uniform) and the tiles left are not written.
constexpr int C5_CTAS_PER_SM = 2;
static_assert(C5_CTAS_PER_SM * 2 * C5<C5_TPC>::COLS <= 512, "TMEM columns of the resident CTAs");
template <bool FWD, bool BITS = !FWD>
__global__ void __launch_bounds__(C5<C5_TPC>::THREADS, C5_CTAS_PER_SM) conv_tc05_kernel(const void* __restrict__ in,
                                                                         const __nv_bfloat16* __restrict__ wt,
                                                                         const float* __restrict__ bias,
                                                                         uint32_t* __restrict__ bits, int L,
                                                                         int n_rows, void* __restrict__ out)
{
    using G = C5<C5_TPC>;
    constexpr int NX = FWD ? 1 : 2;
    constexpr int C5_CT = G::CT, CF_THREADS = G::THREADS, C5_PART = G::PART, C5_PLANE = G::PLANE, C5_COLS = G::COLS;
    static_assert(C5_PLANE % 16 == 0 && C5_PART % 16 == 0, "descriptor steps are whole 16-byte units");
    extern __shared__ __align__(128) unsigned char c5_smem[];
    unsigned char* xs = c5_smem;                                  // [2 buffers][NX parts of 4 planes]
    unsigned char* ws = c5_smem + 2 * NX * C5_PART;               // 36 weight planes
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ws + C5_WBYTES); // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_row = (L + C5_CT - 1) / C5_CT, n_tiles = n_rows * tiles_per_row;
    if ((int)blockIdx.x >= n_tiles) return;   // uniform per CTA, before any barrier or allocation

    if (tid == 0) {
        isr::mbar_init(isr::smem_u32(&mbar[0]), 1);
        isr::mbar_init(isr::smem_u32(&mbar[1]), 1);
    }
    if (warp == 0) isr::tmem_alloc(isr::smem_u32(tslot), 2 * C5_COLS);
    // weights: 16-byte piece (co, tap, 8-channel group g) of row co to plane (tap, g), row co
    {
        const uint4* w4 = reinterpret_cast<const uint4*>(wt);
        constexpr int WPER = (CH * KT * 4 + CF_THREADS - 1) / CF_THREADS;
        uint4 wq[WPER];
#pragma unroll
        for (int u = 0; u < WPER; ++u) {
            const int e = tid + u * CF_THREADS;
            if (e < CH * KT * 4) wq[u] = w4[e];
        }
#pragma unroll
        for (int u = 0; u < WPER; ++u) {
            const int e = tid + u * CF_THREADS;
            if (e >= CH * KT * 4) break;
            const int co = e / (KT * 4), r = e - co * (KT * 4);  // r = tap * 4 + g
            *reinterpret_cast<uint4*>(ws + (r * CH + co) * 16) = wq[u];
        }
    }

    // staging of tile t: global loads into registers, then shared stores into buffer `buf`
    uint4 qa[FWD ? C5Act<C5_TPC>::PER : 1];
    float4 qs[FWD ? 1 : C5Split<C5_TPC>::PER];
    auto load = [&](int t) {
        const int b = t / tiles_per_row, i0 = (t - b * tiles_per_row) * C5_CT;
        if constexpr (FWD)
            c5_act_load<C5_TPC>(static_cast<const unsigned short*>(in) + (size_t)b * CH * L, L, i0, qa);
        else
            c5_split_load<C5_TPC>(static_cast<const float*>(in) + (size_t)b * CH * L, L, i0, qs);
    };
    auto store = [&](int t, int buf) {
        const int b = t / tiles_per_row, i0 = (t - b * tiles_per_row) * C5_CT;
        unsigned char* x = xs + buf * NX * C5_PART;
        if constexpr (FWD)
            c5_act_store<C5_TPC>(static_cast<const unsigned short*>(in) + (size_t)b * CH * L, L, i0, qa,
                                 reinterpret_cast<unsigned short*>(x));
        else
            c5_split_store<C5_TPC>(qs, reinterpret_cast<unsigned short*>(x), reinterpret_cast<unsigned short*>(x + C5_PART));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the tile, for the tensor cores
    };
    // thread 0: the MMAs of the tile in buffer `buf` into accumulator `buf`, committed to mbar[buf]
    auto issue = [&](uint32_t tbase, int buf) {
        constexpr uint32_t idesc = isr::tc05_idesc<true>();      // BF16, FP32 accumulate, M 128, N 32
        // descriptors built once and stepped in 16-byte units of the start field (addresses stay
        // below 0x40000 B, so the 14-bit field never carries): tap k starts the A tile k rows
        // (16 B each) later and B at weight plane 4 k; K-step ks moves A by two channel planes
        // and B by two weight planes (512 B each)
        const uint64_t bd0 = isr::tc05_desc(isr::smem_u32(ws), 512, 128);
        const uint32_t xb = isr::smem_u32(xs) + buf * NX * C5_PART;
#pragma unroll 1
        for (int m = 0; m < C5_CT / 128; ++m) {
            const uint32_t d = tbase + (uint32_t)(buf * C5_COLS) + 32u * m;
            uint32_t acc = 0;
#pragma unroll 1
            for (int part = 0; part < NX; ++part) {
                // rows 128 m + tap of the tile, channels 16 ks .. (planes 2 ks, 2 ks + 1)
                const uint64_t ad0 = isr::tc05_desc(xb + part * C5_PART + 128 * m * 16, C5_PLANE, 128);
#pragma unroll
                for (int tap = 0; tap < KT; ++tap)
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        isr::tc05_mma(d, ad0 + (uint32_t)(tap + ks * (2 * C5_PLANE / 16)),
                                      bd0 + (uint32_t)((tap * 4 + 2 * ks) * (512 / 16)), idesc, acc);
                        acc = 1;
                    }
            }
        }
        isr::tc05_commit(isr::smem_u32(&mbar[buf]));
    };

    int t = blockIdx.x;
    load(t);
    store(t, 0);
    isr::fence_barrier_init();
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    if (tid == 0) issue(tbase, 0);

    // epilogue: warp w, tile m = w / 4, lane quarter w % 4 -> position i
    const int m = warp >> 2;
    for (int k = 0;; ++k) {
        const int buf = k & 1, tn = t + (int)gridDim.x;
        const bool more = tn < n_tiles;
        if (more) load(tn);
        uint32_t mbits = 0;   // backward: the ReLU mask of this thread's position, in flight during the wait
        if constexpr (!FWD) {
            const int b = t / tiles_per_row, i = (t - b * tiles_per_row) * C5_CT + 128 * m + 32 * (warp & 3) + lane;
            if (i < L) mbits = bits[(size_t)b * L + i];
        }
        const bool done = isr::mbar_wait(isr::smem_u32(&mbar[buf]), (uint32_t)(k >> 1) & 1u, 1u << 26);
        isr::tmem_fence_after_sync();
        {
            const int b = t / tiles_per_row, i0 = (t - b * tiles_per_row) * C5_CT;
            const int i = i0 + 128 * m + 32 * (warp & 3) + lane;
            uint32_t r[32];
            isr::tmem_ld32(isr::tmem_warp_lane_base(tbase) + (uint32_t)(buf * C5_COLS) + 32u * m, r);
            isr::tmem_wait_ld32(r);
            if (done && i < L) {
                const size_t row = (size_t)b * CH * L + i;
                uint32_t fbits = 0;
#pragma unroll
                for (int co = 0; co < CH; ++co) {
                    const float v = __uint_as_float(r[co]);
                    if constexpr (FWD) {
                        const __nv_bfloat16 hv = __float2bfloat16_rn(fmaxf(v + __ldg(bias + co), 0.f));
                        static_cast<__nv_bfloat16*>(out)[row + (size_t)co * L] = hv;
                        if constexpr (BITS) fbits |= (uint32_t)((int16_t)__bfloat16_as_ushort(hv) > 0) << co;
                    } else {
                        static_cast<float*>(out)[row + (size_t)co * L] = (mbits >> co) & 1u ? v : 0.f;
                    }
                }
                if constexpr (FWD && BITS) bits[(size_t)b * L + i] = fbits;
            }
        }
        // the other staging buffer and accumulator were last used by tile t - gridDim.x, whose
        // MMAs completed (waited on in the previous iteration) and whose epilogue is done
        if (more) store(tn, buf ^ 1);
        isr::tmem_fence_before_sync();
        const bool ok = __syncthreads_and(done) != 0;
        isr::tmem_fence_after_sync();
        if (!more || !ok) break;
        if (tid == 0) issue(tbase, buf ^ 1);
        t = tn;
    }
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    if (warp == 0) isr::tmem_dealloc(tbase, 2 * C5_COLS);
}

// Persistent CTAs of conv_tc05_kernel: one per tile, up to `slots` (the resident count on all SMs).
inline int conv_tc05_grid(int L, int n_rows, int slots)
{
    const int tiles = n_rows * ((L + C5<C5_TPC>::CT - 1) / C5<C5_TPC>::CT);
    return std::max(1, std::min(tiles, slots));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2_trans(uint32_t (&r)[2], uint32_t addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}

// Weight gradient of layers 2-4 with BF16 storage on the tensor cores:
//   dW[co][ci][k] = sum_{b,i} da[b][co][i] h[b][ci][i + k - 4],  db[co] = sum_{b,i} da[b][co][i],
// the GEMM D[co][kk] = sum_i A[co][i] B[i][kk] with kk = (k, ci), A = da (FP32, split into BF16
// hi + lo, both multiplied) and B[i][(k, ci)] = h[ci][i + k - 4].  B's 8 x 8 blocks are read
// transposed (ldmatrix.trans) from the position-major activation tile of the forward kernel,
// whose rows i + k start on 16-byte boundaries for every tap k.  CTA: `span` positions of one
// row in chunks of TC_CT; warp w: output channels 16 (w % 2) .., input channels 8 (w / 2) ..
// at all 9 taps; the CTA's partial dW and db are added with one atomic per element.  Four
// CTAs per SM (64 registers, 55 KB of shared memory each) hide the staging loads.
constexpr int WT_DR = TC_CT + 8;   // bf16 per staged gradient row (528 B)
constexpr size_t wgrad_tc_smem_bytes() { return (size_t)2 * (2 * CH * WT_DR + TC_XW * TC_XR); }

// Chunks per CTA for n rows of L positions with `slots` resident CTAs: the shortest span whose
// CTAs fit in one wave (else one CTA per row).  Every CTA ends with an atomic add to each of the
// same 9216 weights, so more, shorter CTAs contend there: at 128 rows x 4608 positions 2, 4 and 5
// chunks per CTA took 235, 195 and 157 us per launch.
int wgrad_span_chunks(int L, int n, int slots)
{
    const int cpr = (L + TC_CT - 1) / TC_CT;
    for (int k = 1; k <= cpr; ++k)
        if ((int64_t)n * ((cpr + k - 1) / k) <= slots) return k;
    return cpr;
}

__global__ void __launch_bounds__(256, 4) wgrad_tc_kernel(const __nv_bfloat16* __restrict__ h, const float* __restrict__ da,
                                                       int L, int span, float* __restrict__ dW,
                                                       float* __restrict__ db)
{
    extern __shared__ __align__(16) unsigned char wt_smem[];
    uint32_t* dah = reinterpret_cast<uint32_t*>(wt_smem);   // [CH][WT_DR / 2] words, hi parts
    uint32_t* dal = dah + CH * WT_DR / 2;                   // lo parts
    uint32_t* xs = dal + CH * WT_DR / 2;                    // [TC_XW][TC_XR / 2] words
    __shared__ float db_s[CH];
    const int b = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < CH) db_s[tid] = 0.f;
    const int mt = warp & 1, ci0 = (warp >> 1) * 8;
    const int r8 = lane & 7, mq = lane >> 3;
    const uint32_t a_hi = isr::smem_u32(dah) + 2u * (uint32_t)((mt * 16 + (mq & 1) * 8 + r8) * WT_DR + (mq >> 1) * 8);
    const uint32_t a_lo = a_hi + 2u * (uint32_t)(CH * WT_DR);
    // transposed B blocks: matrix mq = (positions +8 if mq odd, tap +1 if mq >= 2)
    const uint32_t b_row = isr::smem_u32(xs) + 2u * (uint32_t)(((mq >> 1) + (mq & 1) * 8 + r8) * TC_XR + ci0);
    float acc[KT][4];
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[k][q] = 0.f;
    const int span_end = min(L, (int)(blockIdx.x + 1) * span);
    for (int p0 = blockIdx.x * span; p0 < span_end; p0 += TC_CT) {
        __syncthreads();   // the previous chunk's tiles are consumed (and db_s is initialised)
        // gradient: word (co, pp) = positions p0 + 2 pp, +1 of channel co (zero past the span);
        // the 32 lanes of a warp share co, so the bias gradient reduces per warp first
        for (int e = tid; e < CH * TC_CT / 2; e += 256) {
            const int co = e / (TC_CT / 2), pp = e - co * (TC_CT / 2);
            const int pos = p0 + 2 * pp;
            const float* src = da + ((size_t)b * CH + co) * L;
            const float v0 = pos < span_end ? src[pos] : 0.f;
            const float v1 = pos + 1 < span_end ? src[pos + 1] : 0.f;
            uint32_t hi, lo;
            isr::split2<true>(v0, v1, hi, lo);
            dah[co * (WT_DR / 2) + pp] = hi;
            dal[co * (WT_DR / 2) + pp] = lo;
            float s = v0 + v1;
            for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) atomicAdd(&db_s[co], s);
        }
        // activations: position-major tile of positions p0 - 4 + j (zero outside the row)
        stage_act_tile<TC_XW>(reinterpret_cast<const unsigned short*>(h) + (size_t)b * CH * L, L, p0,
                              reinterpret_cast<unsigned short*>(xs));
        __syncthreads();
#pragma unroll 2
        for (int s = 0; s < TC_CT / 16; ++s) {   // k-step: positions p0 + 16 s ..
            uint32_t ah[4], al[4];
            ldsm_x4(ah, a_hi + 2u * (uint32_t)(16 * s));
            ldsm_x4(al, a_lo + 2u * (uint32_t)(16 * s));
            const uint4 fh = make_uint4(ah[0], ah[1], ah[2], ah[3]), fl = make_uint4(al[0], al[1], al[2], al[3]);
#pragma unroll
            for (int tp = 0; tp < KT - 1; tp += 2) {
                uint32_t bq[4];
                ldsm_x4_trans(bq, b_row + 2u * (uint32_t)((16 * s + tp) * TC_XR));
                isr::mma16816<true>(acc[tp], fh, bq[0], bq[1]);
                isr::mma16816<true>(acc[tp], fl, bq[0], bq[1]);
                isr::mma16816<true>(acc[tp + 1], fh, bq[2], bq[3]);
                isr::mma16816<true>(acc[tp + 1], fl, bq[2], bq[3]);
            }
            uint32_t b8[2];   // tap 8: matrices 0 and 1 only (lanes 0-15 give the rows)
            ldsm_x2_trans(b8, b_row + 2u * (uint32_t)((16 * s + KT - 1 - (mq >> 1)) * TC_XR));
            isr::mma16816<true>(acc[KT - 1], fh, b8[0], b8[1]);
            isr::mma16816<true>(acc[KT - 1], fl, b8[0], b8[1]);
        }
    }
    // accumulator (k, q): output channel 16 mt + g + 8 (q >= 2), input channel ci0 + 2 t + (q & 1)
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int co = mt * 16 + g + (q >> 1) * 8, ci = ci0 + 2 * t4 + (q & 1);
            atomicAdd(&dW[((size_t)co * CH + ci) * KT + k], acc[k][q]);
        }
    __syncthreads();
    if (tid < CH) atomicAdd(&db[tid], db_s[tid]);
}

// Weight gradient of layers 2-4 on tcgen05 (ISR_EST_BF16):
//   dW[co][ci][k] = sum_p da[co][p] h[ci][p + k - 4]   over the CTA's chunks,
// as D_g[(k, i)][n] = sum_p A_g[(k, i)][p] B[n][p] with K = positions (16 per MMA): A_g = the
// activation planes of channel group g (8 channels per 16-byte row, positions as rows) as an
// MN-major operand whose 8-row M-groups are 16 bytes apart, so M-group k reads channels 8 g + i at
// position p + k, i.e. tap k (groups 9-15 are padding); B = the gradient's BF16 hi parts (rows
// 0-31) and lo parts (rows 32-63; their sum keeps ~16 bits of the FP32 gradient), K-major 8 x 8
// blocks staged from the channel-major rows; N = 64, M = 128, TMEM columns 64 g, 256 in all.  In
// the no-swizzle layouts of both majors the descriptor's leading-byte offset steps along K and its
// stride-byte offset along M or N.  Four 128 x 64 x 16 MMAs per K-step (64 per chunk) read 6 KB of
// shared memory each: 384 KB per chunk, where 32-column MMAs per tap needed 144 MMAs and 720 KB,
// which the tensor pipe could not stream while the CTA staged the next chunk.  Chunks of 256
// positions are double-buffered; 16 warps stage (and run the epilogue), one more issues the MMAs;
// the n_rows x ceil(L / 256) chunks, row after row, are split into gridDim.x contiguous ranges of
// equal length (+-1), so a CTA's range may cross from one row into the next: the sum over
// positions and rows does not care.  One CTA per SM.
// one arrival (release semantics at CTA scope) on the barrier's current phase
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

constexpr int W5_CHUNK = 256;                    // positions per chunk (16 K-steps)
constexpr int W5_THREADS = 512;                  // staging (and epilogue) threads
constexpr int W5_BLOCK = W5_THREADS + 32;        // + one warp that issues the MMAs
constexpr int W5_ASBO = W5_CHUNK / 8 * 128;      // bytes per 8-row group of A (all its 8-position blocks)
constexpr int W5_ABUF = 8 * W5_ASBO;             // one A buffer: 8 real row groups (hi 0-3, lo 4-7)
using W5X = C5<2>;                               // activation tile: 256 + 8 rows, 4 planes
static_assert(W5X::CT == W5_CHUNK, "activation tile matches the chunk");
constexpr size_t w5_smem_bytes() { return (size_t)2 * W5_ABUF + 2 * W5X::PART + 64; }
// dynamic shared memory requested at launch: more than half an SM's, so that one CTA has the SM to
// itself (its 544 threads need the register file)
constexpr size_t W5_SMEM_LAUNCH = 120 * 1024;
constexpr int W5_TMEM_COLS = 4 * 2 * CH;         // D_g of the four channel groups
static_assert(w5_smem_bytes() <= W5_SMEM_LAUNCH, "launch request covers the layout");
// the padding M-groups (taps 9-15) of the last plane of the second buffer read up to 4336 bytes
// from that plane's start: still inside the launch allocation
static_assert((size_t)2 * W5_ABUF + W5X::PART + 3 * W5X::PLANE + (W5_CHUNK - 16) * 16 + 15 * 16 + 256 <= W5_SMEM_LAUNCH,
              "A's padding rows stay in shared memory");
// ... and the 9 real taps stay inside their plane (rows < XW)
static_assert((W5_CHUNK - 16) + 15 + (KT - 1) < W5X::XW, "real taps read staged rows only");

__global__ void __launch_bounds__(W5_BLOCK, 1) wgrad_tc05_kernel(const __nv_bfloat16* __restrict__ h,
                                                                   const float* __restrict__ da, int L, int n_rows,
                                                                   float* __restrict__ dW, float* __restrict__ db)
{
    extern __shared__ __align__(128) unsigned char w5_smem[];
    unsigned char* abuf = w5_smem;                                  // [2][8 row groups][W5_ASBO]
    unsigned char* xbuf = w5_smem + 2 * W5_ABUF;                    // [2][W5X::PART]
    // mbar[b]: the MMAs of the chunk in buffer b completed (one commit); full[b]: buffer b staged
    // (one arrival per staging warp)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(w5_smem + 2 * W5_ABUF + 2 * W5X::PART);   // [2]
    uint64_t* full = mbar + 2;                                                              // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 4);
    __shared__ float db_s[CH];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cpr = (L + W5_CHUNK - 1) / W5_CHUNK;                 // chunks per row
    const int64_t total = (int64_t)n_rows * cpr;
    const int q_begin = (int)((int64_t)blockIdx.x * total / gridDim.x);
    const int nch = (int)((int64_t)(blockIdx.x + 1) * total / gridDim.x) - q_begin;
    if (tid < CH) db_s[tid] = 0.f;
    if (tid == 0) {
        isr::mbar_init(isr::smem_u32(&mbar[0]), 1);
        isr::mbar_init(isr::smem_u32(&mbar[1]), 1);
        isr::mbar_init(isr::smem_u32(&full[0]), W5_THREADS / 32);
        isr::mbar_init(isr::smem_u32(&full[1]), W5_THREADS / 32);
    }
    if (warp == 0) isr::tmem_alloc(isr::smem_u32(tslot), W5_TMEM_COLS);

    // stage chunk c into buffer c & 1: da as hi / lo 8 x 8 blocks, the activations as planes; in
    // two phases, all global loads of the chunk (gradient and activations) into registers first,
    // then the shared stores, so that one round trip to memory per chunk overlaps the MMAs
    // items (8-position block kb, channel co) with the channel fastest: the eight lanes of a
    // 16-byte store phase write one 128-byte core matrix (no bank conflicts)
    constexpr int NITEM = CH * (W5_CHUNK / 8), PER = NITEM / W5_THREADS;
    float4 q0[PER], q1[PER];
    uint4 qa[C5Act<2, W5_THREADS>::PER];
    float dbacc = 0.f;   // bias gradient of channel `lane` (every item of this thread has co = lane)
    static_assert(W5_THREADS % CH == 0, "item e = tid + u W5_THREADS keeps channel e % 32 = lane");
    auto load = [&](int c) {
        const int q = q_begin + c, b = q / cpr, p0 = (q - b * cpr) * W5_CHUNK;
        const int span_end = min(L, p0 + W5_CHUNK);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = tid + u * W5_THREADS;
            const int co = e & (CH - 1), kb = e / CH;
            const int pos = p0 + 8 * kb;
            const float* src = da + ((size_t)b * CH + co) * L + pos;
            if ((L & 3) == 0 && pos + 8 <= span_end) {
                q0[u] = *reinterpret_cast<const float4*>(src);
                q1[u] = *reinterpret_cast<const float4*>(src + 4);
            } else {
                float t[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) t[k] = pos + k < span_end ? src[k] : 0.f;
                q0[u] = make_float4(t[0], t[1], t[2], t[3]);
                q1[u] = make_float4(t[4], t[5], t[6], t[7]);
            }
        }
        c5_act_load<2, W5_THREADS>(reinterpret_cast<const unsigned short*>(h) + (size_t)b * CH * L, L, p0, qa);
    };
    auto store = [&](int c) {
        const int q = q_begin + c, b = q / cpr, p0 = (q - b * cpr) * W5_CHUNK;
        unsigned char* a = abuf + (c & 1) * W5_ABUF;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = tid + u * W5_THREADS;
            const int co = e & (CH - 1), kb = e / CH;
            const float t[8] = {q0[u].x, q0[u].y, q0[u].z, q0[u].w, q1[u].x, q1[u].y, q1[u].z, q1[u].w};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) isr::split2<true>(t[2 * k], t[2 * k + 1], hi[k], lo[k]);
            const uint32_t o = (uint32_t)((co >> 3) * W5_ASBO + kb * 128 + (co & 7) * 16);
            *reinterpret_cast<uint4*>(a + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(a + o + 4 * W5_ASBO) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
            dbacc += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
        }
        c5_act_store<2, W5_THREADS>(reinterpret_cast<const unsigned short*>(h) + (size_t)b * CH * L, L, p0, qa,
                                    reinterpret_cast<unsigned short*>(xbuf + (c & 1) * W5X::PART));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    };

    isr::fence_barrier_init();
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    bool ok = true;
    if (warp < W5_THREADS / 32) {
        // staging warps: chunk c + 1 goes into buffer (c + 1) & 1 once chunk c - 1's MMAs, which
        // read that buffer, have completed; each warp then arrives on full[(c + 1) & 1]
        for (int c = -1; c + 1 < nch; ++c) {
            load(c + 1);
            if (c >= 1 && !isr::mbar_wait(isr::smem_u32(&mbar[(c + 1) & 1]), (uint32_t)((c - 1) >> 1) & 1u, 1u << 26)) {
                ok = false;
                break;
            }
            store(c + 1);
            __syncwarp();
            if (lane == 0) mbar_arrive(isr::smem_u32(&full[(c + 1) & 1]));
        }
    } else if (lane == 0) {
        // the issuing warp: a tcgen05.mma issue holds its thread until the tensor pipe takes it,
        // so this thread does nothing else.  A = the activation planes, MN-major (bit 15): LBO =
        // 128 B along K (8 positions), SBO = 16 B along M, so M-group j (rows 8 j ..) is channel
        // group g started j rows later, i.e. tap j; B = the gradient's hi / lo rows, K-major: LBO =
        // 128 B along K, SBO = W5_ASBO along N (8 rows).  N = 64, M = 128 (M-groups 9-15 unused).
        constexpr uint32_t idesc =
            (isr::tc05_idesc<true>() & ~(0x3Fu << 17)) | ((uint32_t)(2 * CH >> 3) << 17) | (1u << 15);
        for (int c = 0; c < nch; ++c) {
            if (!isr::mbar_wait(isr::smem_u32(&full[c & 1]), (uint32_t)(c >> 1) & 1u, 1u << 26)) {
                ok = false;
                break;
            }
            isr::tmem_fence_after_sync();
            // descriptors built once per chunk; K-step s adds 16 (256 B) to the 16-byte-unit start
            // field of both (addresses stay below 0x40000 B: the field never carries)
            const uint64_t bd0 = isr::tc05_desc(isr::smem_u32(abuf + (c & 1) * W5_ABUF), 128, W5_ASBO);
            const uint32_t xa = isr::smem_u32(xbuf + (c & 1) * W5X::PART);
            uint64_t ad0[4];
#pragma unroll
            for (int g = 0; g < 4; ++g) ad0[g] = isr::tc05_desc(xa + g * W5X::PLANE, 128, 16);
#pragma unroll 1
            for (int s = 0; s < W5_CHUNK / 16; ++s) {
                const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    isr::tc05_mma(tbase + (uint32_t)(2 * CH * g), ad0[g] + 16u * (uint32_t)s, bd0 + 16u * (uint32_t)s,
                                  idesc, acc);
            }
            isr::tc05_commit(isr::smem_u32(&mbar[c & 1]));
        }
    }
    if (warp < W5_THREADS / 32) atomicAdd(&db_s[lane], dbacc);
    // the last commit covers every MMA of this CTA; a thread whose wait ran out skips it
    if (nch > 0 && ok) ok = isr::mbar_wait(isr::smem_u32(&mbar[(nch - 1) & 1]), (uint32_t)((nch - 1) >> 1) & 1u, 1u << 26);
    isr::tmem_fence_before_sync();
    ok = __syncthreads_and(ok) != 0;
    isr::tmem_fence_after_sync();
    // epilogue: D_g (columns 64 g ..) row 8 t + i (TMEM lane) = tap t, input channel 8 g + i;
    // columns 0-31 the hi and 32-63 the lo part of output channel co.  Warp w reads lane quarter
    // w % 4 (taps 4 (w % 4) ..) of channel group g = w / 4; taps 9-15 are padding.
    static_assert(W5_THREADS == 512, "sixteen epilogue warps: four lane quarters x four channel groups");
    const int quarter = warp & 3, g = warp >> 2;
    if (ok && warp < W5_THREADS / 32 && quarter < 3) {
        const int t = 4 * quarter + (lane >> 3), ci = 8 * g + (lane & 7);
        uint32_t rh[32], rl[32];
        isr::tmem_ld32(isr::tmem_warp_lane_base(tbase) + (uint32_t)(2 * CH * g), rh);
        isr::tmem_ld32(isr::tmem_warp_lane_base(tbase) + (uint32_t)(2 * CH * g + CH), rl);
        isr::tmem_wait_ld32(rh);
        isr::tmem_wait_ld32(rl);
        if (t < KT) {
#pragma unroll
            for (int co = 0; co < CH; ++co)
                atomicAdd(&dW[((size_t)co * CH + ci) * KT + t], __uint_as_float(rh[co]) + __uint_as_float(rl[co]));
        }
    }
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    if (warp == 0) isr::tmem_dealloc(tbase, W5_TMEM_COLS);
    if (tid < CH) atomicAdd(&db[tid], db_s[tid]);
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

// Weight gradient of the one-channel first layer:
//   dW1[co][k] += sum_i da[b][co][i] x[b][i + k - 4],  db1[co] += sum_i da[b][co][i]
// The n_rows x ceil(L / W1_SPAN) spans, row after row, are split into gridDim.x contiguous ranges
// (two CTAs per SM), and a CTA keeps its sums in registers over its spans.  Lane l is output
// channel l, so a thread holds only that channel's nine tap sums and its bias sum and the
// registers go to loads in flight.  Spans are short (512 positions) so that CTAs get near-equal
// numbers of them.  Within a span [i0, i0 + W1_SPAN) of row b warp w takes the positions
// i0 + 64 w .. i0 + 64 w + 63 in rounds of eight steps of 8 positions: per step a
// lane reads 8 consecutive positions of its channel's gradient row (two 16-byte loads; a round's
// loads are all issued before the first is used) and the 16 inputs x[p - 4 .. p + 11] as four
// 16-byte broadcast reads of the span's input row in shared memory.  At the end the eight warps'
// sums of each channel are added in shared memory and every weight receives one atomic per CTA.
constexpr int W1_SPAN = 512;
constexpr int W1_STEP = 8;                              // positions per lane and step
constexpr int W1_U = 8;                                 // steps per round (their loads in flight)
constexpr int W1_WSPAN = W1_SPAN / 8;                   // positions per warp and span
static_assert(W1_WSPAN % (W1_STEP * W1_U) == 0, "whole rounds per warp and span");

template <class TH>
__global__ void __launch_bounds__(256, 2) wgrad1_kernel(const TH* __restrict__ x, const float* __restrict__ da, int L,
                                                        int n_rows, float* __restrict__ dW, float* __restrict__ db)
{
    __shared__ __align__(16) float xs[W1_SPAN + 16];    // xs[j] = x[b][i0 - 4 + j]
    __shared__ float red[8][CH * (KT + 1)];             // the warps' sums: [warp][channel][tap, bias]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int spr = (L + W1_SPAN - 1) / W1_SPAN;                 // spans per row
    const int64_t total = (int64_t)n_rows * spr;
    const int q_begin = (int)((int64_t)blockIdx.x * total / gridDim.x);
    const int q_end = (int)((int64_t)(blockIdx.x + 1) * total / gridDim.x);
    float acc[KT], dbacc = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[k] = 0.f;
    const bool vec = (L & 3) == 0;   // 16-byte gradient loads (8-position pieces start at multiples of 8)
    for (int q = q_begin; q < q_end; ++q) {
        const int b = q / spr, i0 = (q - b * spr) * W1_SPAN, iend = min(L, i0 + W1_SPAN);
        __syncthreads();   // the previous span's reads of xs are done
        for (int j = threadIdx.x; j < W1_SPAN + 16; j += 256) {
            const int pos = i0 - HALF + j;
            xs[j] = (pos >= 0 && pos < L) ? ld<TH>(x, (size_t)b * L + pos) : 0.f;
        }
        __syncthreads();
        const float* dar = da + ((size_t)b * CH + lane) * L;
#pragma unroll 1
        for (int r = 0; r < W1_WSPAN / (W1_STEP * W1_U); ++r) {
            const int pbase = i0 + warp * W1_WSPAN + r * W1_STEP * W1_U;
            float d[W1_U][W1_STEP];
#pragma unroll
            for (int u = 0; u < W1_U; ++u) {
                const int p = pbase + W1_STEP * u;
                if (vec && p + W1_STEP <= iend) {
                    const float4 a0 = __ldg(reinterpret_cast<const float4*>(dar + p));
                    const float4 a1 = __ldg(reinterpret_cast<const float4*>(dar + p + 4));
                    d[u][0] = a0.x; d[u][1] = a0.y; d[u][2] = a0.z; d[u][3] = a0.w;
                    d[u][4] = a1.x; d[u][5] = a1.y; d[u][6] = a1.z; d[u][7] = a1.w;
                } else {
#pragma unroll
                    for (int t = 0; t < W1_STEP; ++t) d[u][t] = p + t < iend ? __ldg(dar + p + t) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < W1_U; ++u) {
                const int j = pbase + W1_STEP * u - i0;   // zero gradient past iend: no effect
                const float4* x4 = reinterpret_cast<const float4*>(&xs[j]);
                float xw[16];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float4 t4 = x4[v];
                    xw[4 * v] = t4.x; xw[4 * v + 1] = t4.y; xw[4 * v + 2] = t4.z; xw[4 * v + 3] = t4.w;
                }
#pragma unroll
                for (int t = 0; t < W1_STEP; ++t) {
                    const float dv = d[u][t];
                    dbacc += dv;
#pragma unroll
                    for (int k = 0; k < KT; ++k) acc[k] = fmaf(dv, xw[t + k], acc[k]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < KT; ++k) red[warp][lane * (KT + 1) + k] = acc[k];
    red[warp][lane * (KT + 1) + KT] = dbacc;
    __syncthreads();
    for (int e = threadIdx.x; e < CH * (KT + 1); e += 256) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w][e];
        const int co = e / (KT + 1), k = e - co * (KT + 1);
        atomicAdd(k < KT ? &dW[co * KT + k] : &db[co], t);
    }
}

// ---------------------------------------------------------------- first layer (one input channel)
// h1[b][co][i] = relu(b1[co] + sum_k W1[co][k] x[b][i + k - 4]).  A thread takes two adjacent
// positions and loops over the channels, so every channel row is written in coalesced pairs.
constexpr int L1_CT = 512;   // positions per CTA

template <class T> __device__ __forceinline__ void store_pair(T* o, float a, float b);
template <> __device__ __forceinline__ void store_pair<float>(float* o, float a, float b)
{
    *reinterpret_cast<float2*>(o) = make_float2(a, b);
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* o, float a, float b)
{
    *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(a, b);
}
// the same, returning in bits 0 / 1 whether a / b read back above zero as stored
template <class T> __device__ __forceinline__ uint32_t store_pair_signs(T* o, float a, float b);
template <> __device__ __forceinline__ uint32_t store_pair_signs<float>(float* o, float a, float b)
{
    store_pair<float>(o, a, b);
    return (uint32_t)(a > 0.f) | ((uint32_t)(b > 0.f) << 1);
}
template <> __device__ __forceinline__ uint32_t store_pair_signs<__nv_bfloat16>(__nv_bfloat16* o, float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    *reinterpret_cast<__nv_bfloat162*>(o) = h;
    const uint32_t w = *reinterpret_cast<const uint32_t*>(&h);
    return (uint32_t)((int16_t)(w & 0xffffu) > 0) | ((uint32_t)((int32_t)w > 0x0000ffff) << 1);
}

template <class T, bool BITS>
__global__ void __launch_bounds__(256) conv1_kernel(const T* __restrict__ x, const T* __restrict__ w1,
                                                    const float* __restrict__ b1, int L, T* __restrict__ out,
                                                    uint32_t* __restrict__ bits)
{
    __shared__ float xs[L1_CT + KT - 1];
    __shared__ __align__(16) float ws[CH][12];   // W1[co][0..8], b1[co], 0, 0
    const int b = blockIdx.y, i0 = blockIdx.x * L1_CT;
    const T* xb = x + (size_t)b * L;
    for (int j = threadIdx.x; j < L1_CT + KT - 1; j += 256) {
        const int pos = i0 - HALF + j;
        xs[j] = (pos >= 0 && pos < L) ? ld<T>(xb, pos) : 0.f;
    }
    for (int e = threadIdx.x; e < CH * 12; e += 256) {
        const int co = e / 12, k = e - co * 12;
        ws[co][k] = k < KT ? ld<T>(w1, (size_t)k * CH + co) : (k == KT ? b1[co] : 0.f);   // w1: [k][co]
    }
    __syncthreads();
    const int p = 2 * threadIdx.x, i = i0 + p;
    if (i >= L) return;
    float xv[KT + 1];
#pragma unroll
    for (int j = 0; j < KT + 1; ++j) xv[j] = xs[p + j];
    const bool pair = i + 1 < L && (L & 1) == 0;   // even row offsets: aligned pair stores
    uint32_t m0 = 0, m1 = 0;                        // ReLU mask bits of positions i, i + 1 (BITS)
#pragma unroll 4
    for (int co = 0; co < CH; ++co) {
        const float4 wa = *reinterpret_cast<const float4*>(&ws[co][0]);
        const float4 wb = *reinterpret_cast<const float4*>(&ws[co][4]);
        const float4 wc = *reinterpret_cast<const float4*>(&ws[co][8]);
        const float w[KT] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w, wc.x};
        float s0 = wc.y, s1 = wc.y;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            s0 = fmaf(w[k], xv[k], s0);
            s1 = fmaf(w[k], xv[k + 1], s1);
        }
        s0 = fmaxf(s0, 0.f);
        s1 = fmaxf(s1, 0.f);
        T* o = out + ((size_t)b * CH + co) * L + i;
        if (pair) {
            if constexpr (BITS) {
                const uint32_t sg = store_pair_signs<T>(o, s0, s1);
                m0 |= (sg & 1u) << co;
                m1 |= (sg >> 1) << co;
            } else {
                store_pair<T>(o, s0, s1);
            }
        } else {
            if constexpr (BITS) {
                m0 |= (uint32_t)positive_as_stored<T>(s0) << co;
                m1 |= (uint32_t)positive_as_stored<T>(s1) << co;
            }
            o[0] = cvt<T>(s0);
            if (i + 1 < L) o[1] = cvt<T>(s1);
        }
    }
    if constexpr (BITS) {
        bits[(size_t)b * L + i] = m0;
        if (i + 1 < L) bits[(size_t)b * L + i + 1] = m1;
    }
}

// ---------------------------------------------------------------- head
// Forward head in two kernels.  head_chunk_kernel: CTA (chunk x of HD_CT positions, row b)
// writes z for its positions and, per channel, the chunk's max, first arg-max and sum.
// head_mlp_kernel: per row, the chunk partials -> max / arg-max (first index) / mean per
// channel, then the presence MLP.
constexpr int HD_CT = 512;

template <class T>
__global__ void __launch_bounds__(256) head_chunk_kernel(const T* __restrict__ h4, const float* __restrict__ theta,
                                                         int L, int nx, float* __restrict__ z,
                                                         float* __restrict__ pmax, int* __restrict__ pidx,
                                                         float* __restrict__ psum, float* __restrict__ zmax,
                                                         int* __restrict__ zidx)
{
    const int b = blockIdx.y, xc = blockIdx.x, i0 = xc * HD_CT, iend = min(L, i0 + HD_CT);
    const T* hb = h4 + (size_t)b * CH * L;
    __shared__ float w5[CH];
    if (threadIdx.x < CH) w5[threadIdx.x] = theta[OFF_W5 + threadIdx.x];
    __syncthreads();
    const float b5 = theta[OFF_B5];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float zm = -INFINITY;   // the chunk's largest z and its first position
    int zi = i0;
    // BF16 rows with L a multiple of 8 are read once: warp w loads its channels 4w .. 4w + 3 with
    // 16-byte loads (lane: positions p = i0 + 8 lane + 256 r, all loads issued first), keeps their
    // max / first arg-max / sum and adds their part of z into zp[w]; z = b5 + the eight parts.
    // Other rows: z over all channels per position, then each channel's statistics, scalar loads.
    bool vec = false;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) vec = (L & 7) == 0;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) if (vec) {
        constexpr int HV = 8, HR = HD_CT / (32 * HV);
        __shared__ __align__(16) float zp[8][HD_CT];
        const T* hw = hb + (size_t)warp * 4 * L;
        uint4 hq[HR][4];
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const int p = i0 + HV * lane + 32 * HV * r;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                hq[r][cc] = p < iend ? *reinterpret_cast<const uint4*>(hw + (size_t)cc * L + p) : make_uint4(0u, 0u, 0u, 0u);
        }
        float mx[4], sum[4];
        int mi[4];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            mx[cc] = -INFINITY;
            sum[cc] = 0.f;
            mi[cc] = i0;
        }
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const int p = i0 + HV * lane + 32 * HV * r;
            if (p >= iend) break;
            float zpart[HV];
#pragma unroll
            for (int k = 0; k < HV; ++k) {
                zpart[k] = 0.f;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const uint32_t w = (&hq[r][cc].x)[k >> 1];
                    const float v = __uint_as_float((k & 1) ? (w & 0xffff0000u) : (w << 16));   // BF16 -> FP32
                    zpart[k] = fmaf(w5[warp * 4 + cc], v, zpart[k]);
                    if (v > mx[cc]) {
                        mx[cc] = v;
                        mi[cc] = p + k;
                    }
                    sum[cc] += v;
                }
            }
            float4* zq = reinterpret_cast<float4*>(&zp[warp][p - i0]);
            zq[0] = make_float4(zpart[0], zpart[1], zpart[2], zpart[3]);
            zq[1] = make_float4(zpart[4], zpart[5], zpart[6], zpart[7]);
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            for (int o = 16; o; o >>= 1) {
                const float om = __shfl_down_sync(0xffffffffu, mx[cc], o);
                const int oi = __shfl_down_sync(0xffffffffu, mi[cc], o);
                sum[cc] += __shfl_down_sync(0xffffffffu, sum[cc], o);
                if (om > mx[cc] || (om == mx[cc] && oi < mi[cc])) {
                    mx[cc] = om;
                    mi[cc] = oi;
                }
            }
            if (lane == 0) {
                const size_t o = ((size_t)b * nx + xc) * CH + warp * 4 + cc;
                pmax[o] = mx[cc];
                pidx[o] = mi[cc];
                psum[o] = sum[cc];
            }
        }
        __syncthreads();
        for (int i = i0 + threadIdx.x; i < iend; i += 256) {
            float s = b5;
#pragma unroll
            for (int w = 0; w < 8; ++w) s += zp[w][i - i0];
            z[(size_t)b * L + i] = s;
            if (s > zm) {
                zm = s;
                zi = i;
            }
        }
    }
    if (!vec) {
        for (int i = i0 + threadIdx.x; i < iend; i += 256) {
            float s = b5;
#pragma unroll 8
            for (int c = 0; c < CH; ++c) s = fmaf(w5[c], ld<T>(hb, (size_t)c * L + i), s);
            z[(size_t)b * L + i] = s;
            if (s > zm) {
                zm = s;
                zi = i;
            }
        }
    }
    for (int o = 16; o; o >>= 1) {
        const float om = __shfl_down_sync(0xffffffffu, zm, o);
        const int oi = __shfl_down_sync(0xffffffffu, zi, o);
        if (om > zm || (om == zm && oi < zi)) {
            zm = om;
            zi = oi;
        }
    }
    __shared__ float zm_s[8];
    __shared__ int zi_s[8];
    if (lane == 0) {
        zm_s[warp] = zm;
        zi_s[warp] = zi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w)
            if (zm_s[w] > zm_s[0] || (zm_s[w] == zm_s[0] && zi_s[w] < zi_s[0])) {
                zm_s[0] = zm_s[w];
                zi_s[0] = zi_s[w];
            }
        zmax[(size_t)b * nx + xc] = zm_s[0];
        zidx[(size_t)b * nx + xc] = zi_s[0];
    }
    // warp w: channels 4w .. 4w+3 (done above for the vector path)
    if (!vec) for (int cc = 0; cc < 4; ++cc) {
        const int c = warp * 4 + cc;
        float mx = -INFINITY, sum = 0.f;
        int mi = i0;
        for (int i = i0 + lane; i < iend; i += 32) {
            const float v = ld<T>(hb, (size_t)c * L + i);
            if (v > mx) {
                mx = v;
                mi = i;
            }
            sum += v;
        }
        for (int o = 16; o; o >>= 1) {
            const float om = __shfl_down_sync(0xffffffffu, mx, o);
            const int oi = __shfl_down_sync(0xffffffffu, mi, o);
            sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (om > mx || (om == mx && oi < mi)) {
                mx = om;
                mi = oi;
            }
        }
        if (lane == 0) {
            const size_t o = ((size_t)b * nx + xc) * CH + c;
            pmax[o] = mx;
            pidx[o] = mi;
            psum[o] = sum;
        }
    }
}

// With pos and pres (inference) it also gives the prediction: position = softmax-weighted mean
// over the 7 bins around the first arg-max of z (+ band_lo), presence = sigmoid(q).
__global__ void __launch_bounds__(64) head_mlp_kernel(const float* __restrict__ theta, int L, int nx,
                                                      const float* __restrict__ pmax, const int* __restrict__ pidx,
                                                      const float* __restrict__ psum, const float* __restrict__ z,
                                                      const float* __restrict__ zmax, const int* __restrict__ zidx,
                                                      int lo, int* __restrict__ amax, float* __restrict__ pooled,
                                                      float* __restrict__ u, float* __restrict__ q,
                                                      float* __restrict__ pos, float* __restrict__ pres)
{
    const int b = blockIdx.x;
    __shared__ float pool_s[2 * CH];
    __shared__ float u_s[CH];
    if (pos && threadIdx.x == CH) {
        float mx = -INFINITY;
        int mi = 0;
        for (int xc = 0; xc < nx; ++xc)   // chunks in position order: ties keep the first
            if (zmax[(size_t)b * nx + xc] > mx) {
                mx = zmax[(size_t)b * nx + xc];
                mi = zidx[(size_t)b * nx + xc];
            }
        const float* zb = z + (size_t)b * L;
        const int a = max(0, mi - WIN), e = min(L, mi + WIN + 1);
        double sw = 0, swi = 0;
        for (int i = a; i < e; ++i) {
            const double wgt = exp((double)zb[i] - (double)mx);
            sw += wgt;
            swi += wgt * i;
        }
        pos[b] = (float)(lo + swi / sw);
    }
    if (threadIdx.x < CH) {
        const int c = threadIdx.x;
        float mx = -INFINITY, sum = 0.f;
        int mi = 0;
        for (int xc = 0; xc < nx; ++xc) {   // chunks in position order: ties keep the first
            const size_t o = ((size_t)b * nx + xc) * CH + c;
            if (pmax[o] > mx) {
                mx = pmax[o];
                mi = pidx[o];
            }
            sum += psum[o];
        }
        pool_s[c] = mx;
        pool_s[CH + c] = sum / L;
        amax[b * CH + c] = mi;
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
        if (pres) pres[b] = 1.f / (1.f + expf(-s));
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

// Head backward in two kernels.  head_bwd_row_kernel (per row): softmax statistics of z, the
// loss, the presence-MLP gradients and d(pooled); it leaves per row the scalars the location
// term needs (lse, 1 / sum t, y / B for gates with a line else 0, the line position) and
// d(pooled).  head_bwd_chunk_kernel (CTA = HD_CT positions of one row): dz, the ReLU-masked
// gradient of h4 and the CTA's partial dw5, db5.
constexpr int HB_SCAL = 4;   // per-row scalars: lse, 1 / sum t, y / B (0 without a line), f

__global__ void __launch_bounds__(256) head_bwd_row_kernel(const float* __restrict__ theta, int L, int B,
                                                           const float* __restrict__ z, const float* __restrict__ pooled,
                                                           const float* __restrict__ u, const float* __restrict__ q,
                                                           const float* __restrict__ fpos, const float* __restrict__ pres,
                                                           float* __restrict__ scal, float* __restrict__ dpool,
                                                           float* __restrict__ grad, float* __restrict__ loss)
{
    const int b = blockIdx.x;
    __shared__ float red[8];
    __shared__ float du_s[CH];
    const float* zb = z + (size_t)b * L;
    const float y = pres[b], f = fpos[b];
    // softmax statistics and target normalisation.  Rows of up to 4 x 256 x RV positions (L a
    // multiple of 4) are read once, as float4 pieces all in flight together, and kept in registers
    // for both passes; longer or unaligned rows are read twice with scalar loads.
    constexpr int RV = 5;
    const bool in_regs = (L & 3) == 0 && L <= 4 * 256 * RV;
    float4 zr[RV];
    float m = -INFINITY;
    if (in_regs) {
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const int i = 4 * (threadIdx.x + 256 * v);
            zr[v] = i < L ? __ldg(reinterpret_cast<const float4*>(zb + i)) : make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        }
#pragma unroll
        for (int v = 0; v < RV; ++v) m = fmaxf(m, fmaxf(fmaxf(zr[v].x, zr[v].y), fmaxf(zr[v].z, zr[v].w)));
    } else {
        for (int i = threadIdx.x; i < L; i += 256) m = fmaxf(m, zb[i]);
    }
    m = block_max(m, red);
    float se = 0.f, st = 0.f, stz = 0.f;
    auto term = [&](int i, float zi) {
        se += __expf(zi - m);
        const float d = (i - f) / SIGMA_T;
        const float t = __expf(-0.5f * d * d);
        st += t;
        stz += t * zi;
    };
    if (in_regs) {
#pragma unroll
        for (int v = 0; v < RV; ++v) {
            const int i = 4 * (threadIdx.x + 256 * v);
            if (i < L) {
                term(i, zr[v].x);
                term(i + 1, zr[v].y);
                term(i + 2, zr[v].z);
                term(i + 3, zr[v].w);
            }
        }
    } else {
        for (int i = threadIdx.x; i < L; i += 256) term(i, zb[i]);
    }
    se = block_sum(se, red);
    st = block_sum(st, red);
    stz = block_sum(stz, red);
    const float lse = m + logf(se);
    const float invB = 1.f / B;
    const float qb = q[b];
    const float sig = 1.f / (1.f + __expf(-qb));
    const float dq = (sig - y) * invB;
    // the location term exists only for gates with a line (its target may lie anywhere,
    // even outside the band, for gates without one)
    const bool loc = y > 0.f && st > 0.f;
    if (threadIdx.x == 0) {
        // CE = lse - sum t z / sum t ; BCE in the stable form
        const float ce = loc ? y * (lse - stz / st) : 0.f;
        const float bce = fmaxf(qb, 0.f) - qb * y + log1pf(__expf(-fabsf(qb)));
        atomicAdd(loss, (bce + ce) * invB);
        atomicAdd(&grad[OFF_BB], dq);
        float* sc = scal + (size_t)b * HB_SCAL;
        sc[0] = lse;
        sc[1] = loc ? 1.f / st : 0.f;
        sc[2] = loc ? y * invB : 0.f;
        sc[3] = f;
    }
    // presence MLP backward (du by threads 0..31; the 32 x 64 weight gradient by all threads)
    if (threadIdx.x < CH) {
        const int j = threadIdx.x;
        const float uj = u[b * CH + j];
        atomicAdd(&grad[OFF_WB + j], dq * uj);
        const float du = uj > 0.f ? dq * theta[OFF_WB + j] : 0.f;
        du_s[j] = du;
        atomicAdd(&grad[OFF_BA + j], du);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CH * 2 * CH; e += 256)
        atomicAdd(&grad[OFF_WA + e], du_s[e / (2 * CH)] * pooled[b * 2 * CH + e % (2 * CH)]);
    if (threadIdx.x < 2 * CH) {
        float s = 0.f;
        for (int j = 0; j < CH; ++j) s = fmaf(du_s[j], theta[OFF_WA + j * 2 * CH + threadIdx.x], s);
        dpool[(size_t)b * 2 * CH + threadIdx.x] = s;
    }
}

// warp w: channels 4w .. 4w+3 of the chunk, lanes along the positions (each warp evaluates dz
// itself), so a thread keeps four partial dw5 sums and every warp adds its own channels
template <class T>
__global__ void __launch_bounds__(256, 2) head_bwd_chunk_kernel(const T* __restrict__ h4, const float* __restrict__ theta,
                                                             int L, const float* __restrict__ z,
                                                             const int* __restrict__ amax,
                                                             const float* __restrict__ scal,
                                                             const float* __restrict__ dpool, float* __restrict__ da4,
                                                             float* __restrict__ grad)
{
    const int b = blockIdx.y, i0 = blockIdx.x * HD_CT, iend = min(L, i0 + HD_CT);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* sc = scal + (size_t)b * HB_SCAL;
    const float lse = sc[0], inv_st = sc[1], ys = sc[2], f = sc[3];
    float w5[4], gmean[4], gmax[4];
    int am[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
        const int c = warp * 4 + cc;
        w5[cc] = theta[OFF_W5 + c];
        gmax[cc] = dpool[(size_t)b * 2 * CH + c];
        gmean[cc] = dpool[(size_t)b * 2 * CH + CH + c] / L;
        am[cc] = amax[b * CH + c];
    }
    const float* zb = z + (size_t)b * L;
    const T* hb = h4 + ((size_t)b * CH + warp * 4) * L;
    float* ob = da4 + ((size_t)b * CH + warp * 4) * L;
    // BF16 rows with L a multiple of 8: lane takes positions p = i0 + 8 lane + 256 r, 8 at a time,
    // and every activation load of the chunk is issued here, before dz is computed (iend is a
    // multiple of 8: a piece is whole or absent)
    constexpr int HV = 8;                       // positions per lane and round (one 16-byte BF16 load)
    constexpr int HR = HD_CT / (32 * HV);       // rounds per chunk
    static_assert(HD_CT % (32 * HV) == 0, "whole rounds per chunk");
    bool vec = false;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) vec = (L & 7) == 0;
    uint4 hq[HR][4];
    if (vec) {
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const int p = i0 + HV * lane + 32 * HV * r;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                hq[r][cc] = p < iend ? *reinterpret_cast<const uint4*>(hb + (size_t)cc * L + p) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    // dL/dz once per position (every warp needs it for its four channels)
    __shared__ __align__(16) float dz_s[HD_CT];   // read as float4 by the vector path
    float db5 = 0.f;
    for (int i = i0 + threadIdx.x; i < iend; i += 256) {
        const float d = (i - f) / SIGMA_T;
        const float dz = ys != 0.f ? ys * (__expf(zb[i] - lse) - __expf(-0.5f * d * d) * inv_st) : 0.f;
        dz_s[i - i0] = dz;
        db5 += dz;
    }
    __syncthreads();
    float dw5[4] = {0.f, 0.f, 0.f, 0.f};
    // one position's four channels: dw5 += dz h, da4 = (w5 dz + mean and max pooling terms) (h > 0)
    auto position = [&](int i, float dz, const float (&hv)[4], float (&o)[4]) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
            dw5[cc] = fmaf(dz, hv[cc], dw5[cc]);
            float g = w5[cc] * dz + gmean[cc];
            if (i == am[cc]) g += gmax[cc];
            o[cc] = hv[cc] > 0.f ? g : 0.f;
        }
    };
    if constexpr (std::is_same<T, __nv_bfloat16>::value) if (vec) {
#pragma unroll
        for (int r = 0; r < HR; ++r) {
            const int p = i0 + HV * lane + 32 * HV * r;
            if (p >= iend) break;
            const float4 z0 = *reinterpret_cast<const float4*>(&dz_s[p - i0]);
            const float4 z1 = *reinterpret_cast<const float4*>(&dz_s[p - i0 + 4]);
            const float dzv[HV] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            float o[4][HV];
#pragma unroll
            for (int k = 0; k < HV; ++k) {
                float hv[4], ok[4];
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const uint32_t w = (&hq[r][cc].x)[k >> 1];
                    hv[cc] = __uint_as_float((k & 1) ? (w & 0xffff0000u) : (w << 16));   // BF16 -> FP32
                }
                position(p + k, dzv[k], hv, ok);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) o[cc][k] = ok[cc];
            }
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                float4* d = reinterpret_cast<float4*>(ob + (size_t)cc * L + p);
                d[0] = make_float4(o[cc][0], o[cc][1], o[cc][2], o[cc][3]);
                d[1] = make_float4(o[cc][4], o[cc][5], o[cc][6], o[cc][7]);
            }
        }
    }
    if (!vec) {
        for (int i = i0 + lane; i < iend; i += 32) {
            float hv[4], o[4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) hv[cc] = ld<T>(hb, (size_t)cc * L + i);
            position(i, dz_s[i - i0], hv, o);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) ob[(size_t)cc * L + i] = o[cc];
        }
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc)
        for (int o = 16; o; o >>= 1) dw5[cc] += __shfl_down_sync(0xffffffffu, dw5[cc], o);
    if (lane == 0) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) atomicAdd(&grad[OFF_W5 + warp * 4 + cc], dw5[cc]);
    }
    // db5: one sum per CTA (every CTA adds into the same address, so one atomic each, not one per warp)
    __shared__ float db5_s[8];
    for (int o = 16; o; o >>= 1) db5 += __shfl_down_sync(0xffffffffu, db5, o);
    if (lane == 0) db5_s[warp] = db5;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += db5_s[w];
        atomicAdd(&grad[OFF_B5], t);   // the chunk's positions
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

}  // namespace

struct isr_est {
    int nfft = 0, lo = 0, L = 0, max_batch = 0, precision = 0, dev = 0;
    cudaStream_t stream = nullptr;
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    int64_t step = 0;
    void* wf = nullptr;       // forward working weights (storage type)
    void* wb = nullptr;       // backward-data working weights
    void* tf = nullptr;       // tensor-core GEMM rows of the forward weights (BF16 only)
    void* tb = nullptr;       // ... and of the backward-data weights
    void* act[5] = {};        // x, h1..h4 (storage type)
    float *z = nullptr, *pooled = nullptr, *u = nullptr, *q = nullptr, *loss = nullptr;
    int* amax = nullptr;
    float *pmax = nullptr, *psum = nullptr;   // head partials per (row, chunk, channel)
    float *hscal = nullptr, *dpool = nullptr; // head backward: per-row scalars and d(pooled)
    float* zmax = nullptr;                    // per (row, chunk): largest location logit ...
    int* zidx = nullptr;                      // ... and its first position
    bool weights_stale = true;                // the working weights need the master copy's values
    int wgrad_slots = 0;                      // resident tensor-core weight-gradient CTAs (all SMs)
    bool conv05 = false;                      // BF16 convolutions on tcgen05 (else mma.sync)
    int sms = 0;                              // multiprocessors of the device
    int c5_slots[2] = {1, 1};                 // persistent tcgen05 convolution CTAs, backward / forward
    int* pidx = nullptr;
    float *da0 = nullptr, *da1 = nullptr; // gradient ping-pong [B][32][L]
    // tcgen05 engine: ReLU masks of h1..h3 as written by a training forward pass, [3][B][L] words,
    // bit co of word (b, i) set when h_l[b][co][i] > 0 as stored
    uint32_t* hbits = nullptr;
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
    if constexpr (kTensorConv<T>) {
        EST_TRY(cudaFuncSetAttribute(conv_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes(true)));
        EST_TRY(cudaFuncSetAttribute(conv_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)tc_smem_bytes(false)));
        EST_TRY(cudaFuncSetAttribute(wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wgrad_tc_smem_bytes()));
        EST_TRY(cudaFuncSetAttribute(wgrad_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)W5_SMEM_LAUNCH));
        for (auto k : {conv_tc05_kernel<true, false>, conv_tc05_kernel<true, true>}) {
            EST_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C5<C5_TPC>::smem(true)));
            EST_TRY(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared));
        }
        EST_TRY(cudaFuncSetAttribute(conv_tc05_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)C5<C5_TPC>::smem(false)));
        EST_TRY(cudaFuncSetAttribute(conv_tc05_kernel<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared));
    }
    return ISR_OK;
}

// pos / pres: the prediction outputs (inference), or NULL
template <class T>
isr_status forward_t(isr_est* e, const float* x, int n, float* pos = nullptr, float* pres = nullptr)
{
    const int L = e->L;
    cudaStream_t s = e->stream;
    T* act[5];
    for (int i = 0; i < 5; ++i) act[i] = static_cast<T*>(e->act[i]);
    const size_t nx = (size_t)n * L;
    cast_kernel<T><<<(unsigned)std::min<size_t>((nx + 255) / 256, 4096), 256, 0, s>>>(x, nx, act[0]);
    if (e->weights_stale) {   // working weights follow the master copy only after it changed
        relayout_kernel<T><<<(CH * KT + 3 * CH * CH * KT + 255) / 256, 256, 0, s>>>(
            e->theta, static_cast<T*>(e->wf), static_cast<T*>(e->wb), static_cast<T*>(e->tf), static_cast<T*>(e->tb));
        e->weights_stale = false;
    }
    const T* wf = static_cast<const T*>(e->wf);
    dim3 grid((L + CT - 1) / CT, n);
    // a training pass (no prediction outputs) of the tcgen05 engine leaves the ReLU masks of h1..h3
    // as bits for the backward-data convolutions
    auto hbits = [&](int l) -> uint32_t* {
        return (pos == nullptr && e->hbits && l <= 3) ? e->hbits + (size_t)(l - 1) * e->max_batch * L : nullptr;
    };
    (hbits(1) ? conv1_kernel<T, true> : conv1_kernel<T, false>)<<<dim3((L + L1_CT - 1) / L1_CT, n), 256, 0, s>>>(
        act[0], wf, e->theta + OFF_B1, L, act[1], hbits(1));
    for (int l = 2; l <= 4; ++l) {
        if constexpr (kTensorConv<T>) {
            const T* w = static_cast<const T*>(e->tf) + (size_t)(l - 2) * CH * CH * KT;
            if (e->conv05)
                (hbits(l) ? conv_tc05_kernel<true, true> : conv_tc05_kernel<true, false>)<<<
                    conv_tc05_grid(L, n, e->c5_slots[1]), C5<C5_TPC>::THREADS, C5<C5_TPC>::smem(true), s>>>(
                    act[l - 1], w, e->theta + b_off(l), hbits(l), L, n, act[l]);
            else
                conv_tc_kernel<true><<<dim3((L + CF_CT - 1) / CF_CT, n), CF_THREADS, tc_smem_bytes(true), s>>>(
                    act[l - 1], w, e->theta + b_off(l), nullptr, L, act[l]);
        } else {
            conv_kernel<T, T, T, T, CH, true><<<grid, 256, conv_smem_bytes(CH), s>>>(
                act[l - 1], wf + CH * KT + (size_t)(l - 2) * CH * CH * KT, e->theta + b_off(l), nullptr, L, act[l]);
        }
    }
    const int nxh = (L + HD_CT - 1) / HD_CT;
    head_chunk_kernel<T><<<dim3(nxh, n), 256, 0, s>>>(act[4], e->theta, L, nxh, e->z, e->pmax, e->pidx, e->psum,
                                                      e->zmax, e->zidx);
    head_mlp_kernel<<<n, 64, 0, s>>>(e->theta, L, nxh, e->pmax, e->pidx, e->psum, e->z, e->zmax, e->zidx, e->lo,
                                     e->amax, e->pooled, e->u, e->q, pos, pres);
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
    head_bwd_row_kernel<<<n, 256, 0, s>>>(e->theta, L, n, e->z, e->pooled, e->u, e->q, fpos, pres, e->hscal,
                                          e->dpool, e->grad, e->loss);
    head_bwd_chunk_kernel<T><<<dim3((L + HD_CT - 1) / HD_CT, n), 256, 0, s>>>(act[4], e->theta, L, e->z, e->amax,
                                                                              e->hscal, e->dpool, e->da0, e->grad);
    const T* wbk = static_cast<const T*>(e->wb);
    float* da = e->da0;
    float* dn = e->da1;
    dim3 gw((L + WG_SPAN - 1) / WG_SPAN, n);
    dim3 gc((L + CT - 1) / CT, n);
    const int span = TC_CT * wgrad_span_chunks(L, n, std::max(1, e->wgrad_slots));
    for (int l = 4; l >= 1; --l) {
        if (l == 1) {
            const int spans = n * ((L + W1_SPAN - 1) / W1_SPAN);
            wgrad1_kernel<T><<<std::min(spans, 2 * std::max(1, e->sms)), 256, 0, s>>>(act[0], da, L, n,
                                                                                     e->grad + OFF_W1, e->grad + OFF_B1);
        } else {
            if constexpr (kTensorConv<T>) {
                if (e->conv05) {
                    const int chunks = n * ((L + W5_CHUNK - 1) / W5_CHUNK);
                    wgrad_tc05_kernel<<<std::min(chunks, e->sms), W5_BLOCK, W5_SMEM_LAUNCH, s>>>(
                        reinterpret_cast<const __nv_bfloat16*>(act[l - 1]), da, L, n, e->grad + w_off(l),
                        e->grad + b_off(l));
                } else {
                    wgrad_tc_kernel<<<dim3((L + span - 1) / span, n), 256, wgrad_tc_smem_bytes(), s>>>(
                        act[l - 1], da, L, span, e->grad + w_off(l), e->grad + b_off(l));
                }
            } else
                wgrad_kernel<T, CH><<<gw, 256, 0, s>>>(act[l - 1], da, L, e->grad + w_off(l), e->grad + b_off(l));
            // gradient into the layer below, masked by its ReLU: da_{l-1} = (W_l^T * da_l) (h_{l-1} > 0)
            if constexpr (kTensorConv<T>) {
                const T* w = static_cast<const T*>(e->tb) + (size_t)(l - 2) * CH * CH * KT;
                if (e->conv05)
                    conv_tc05_kernel<false><<<conv_tc05_grid(L, n, e->c5_slots[0]), C5<C5_TPC>::THREADS,
                                              C5<C5_TPC>::smem(false), s>>>(
                        da, w, nullptr, e->hbits + (size_t)(l - 2) * e->max_batch * L, L, n, dn);
                else
                    conv_tc_kernel<false><<<dim3((L + CF_CT - 1) / CF_CT, n), CF_THREADS, tc_smem_bytes(false), s>>>(
                        da, w, nullptr, act[l - 1], L, dn);
            } else
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
    if (precision != ISR_EST_FP32 && precision != ISR_EST_BF16 && precision != ISR_EST_BF16_MMASYNC)
        return fail(ISR_ERR_UNSUPPORTED, "unknown precision");
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
    e->conv05 = precision == ISR_EST_BF16;
    e->dev = dev;
    e->stream = static_cast<cudaStream_t>(stream);
    const bool bf16 = precision != ISR_EST_FP32;
    const size_t es = bf16 ? 2 : 4;
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
    if (bf16) {
        A(&e->tf, es * 3 * CH * CH * KT);
        A(&e->tb, es * 3 * CH * CH * KT);
    }
    A(&e->act[0], es * B * L);
    for (int i = 1; i < 5; ++i) A(&e->act[i], es * B * CH * L);
    A((void**)&e->z, 4 * B * L);
    A((void**)&e->pooled, 4 * B * 2 * CH);
    A((void**)&e->u, 4 * B * CH);
    A((void**)&e->q, 4 * B);
    A((void**)&e->loss, 4);
    A((void**)&e->amax, 4 * B * CH);
    const size_t nxh = (L + HD_CT - 1) / HD_CT;
    A((void**)&e->pmax, 4 * B * nxh * CH);
    A((void**)&e->pidx, 4 * B * nxh * CH);
    A((void**)&e->psum, 4 * B * nxh * CH);
    A((void**)&e->hscal, 4 * B * HB_SCAL);
    A((void**)&e->dpool, 4 * B * 2 * CH);
    A((void**)&e->zmax, 4 * B * nxh);
    A((void**)&e->zidx, 4 * B * nxh);
    A((void**)&e->da0, 4 * B * CH * L);
    A((void**)&e->da1, 4 * B * CH * L);
    if (e->conv05) A((void**)&e->hbits, 4 * 3 * B * L);
    if (r == cudaSuccess) r = cudaMemset(e->theta, 0, 4 * NPARAM);
    if (r == cudaSuccess) r = cudaMemset(e->m, 0, 4 * NPARAM);
    if (r == cudaSuccess) r = cudaMemset(e->v, 0, 4 * NPARAM);
    if (r == cudaSuccess) {
        isr_status st = bf16 ? set_smem_attrs<__nv_bfloat16>() : set_smem_attrs<float>();
        if (st != ISR_OK) {
            isr_est_destroy(e);
            return st;
        }
        int sms = 0;
        r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e->sms = std::max(1, sms);
        if (bf16 && r == cudaSuccess) {
            int occ = 0;
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_tc_kernel, 256, wgrad_tc_smem_bytes());
            e->wgrad_slots = std::max(1, occ) * e->sms;
            // two CTAs per SM, the shape the kernel is built for (__launch_bounds__ minimum): 128
            // registers x 256 threads, at most 86 KB of shared memory and 128 TMEM columns each
            e->c5_slots[0] = e->c5_slots[1] = C5_CTAS_PER_SM * e->sms;
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
    e->weights_stale = true;
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
    st = e->precision != ISR_EST_FP32 ? forward_t<__nv_bfloat16>(e, x, n) : forward_t<float>(e, x, n);
    if (st == ISR_OK)
        st = e->precision != ISR_EST_FP32 ? backward_t<__nv_bfloat16>(e, n, line_bin, present)
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
    st = e->precision != ISR_EST_FP32 ? forward_t<__nv_bfloat16>(e, x, n) : forward_t<float>(e, x, n);
    if (st == ISR_OK)
        st = e->precision != ISR_EST_FP32 ? backward_t<__nv_bfloat16>(e, n, line_bin, present)
                                          : backward_t<float>(e, n, line_bin, present);
    if (st != ISR_OK) return st;
    e->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - powf(b1, (float)e->step)), c2 = 1.f / (1.f - powf(b2, (float)e->step));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, e->stream>>>(e->theta, e->grad, e->m, e->v, NPARAM, lr, b1, b2, 1e-8f,
                                                              c1, c2);
    e->weights_stale = true;
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
    return e->precision != ISR_EST_FP32 ? forward_t<__nv_bfloat16>(e, x, n, line_bin, presence)
                                        : forward_t<float>(e, x, n, line_bin, presence);
}

void isr_est_destroy(isr_est* e)
{
    if (!e) return;
    Dev guard(e->dev);
    cudaStreamSynchronize(e->stream);
    void* ptrs[] = {e->theta, e->m, e->v, e->grad, e->wf, e->wb, e->tf, e->tb, e->act[0], e->act[1], e->act[2], e->act[3],
                    e->act[4], e->z, e->pooled, e->u, e->q, e->loss, e->amax, e->da0, e->da1,
                    e->pmax, e->pidx, e->psum, e->hscal, e->dpool, e->zmax, e->zidx, e->hbits};
    for (void* p : ptrs) cudaFree(p);
    cudaGetLastError();
    delete e;
}

}  // extern "C"
