// isr_paired.cuh -- FFT arithmetic on pairs of butterflies with the paired FP32 instructions
// of sm_100+ (FADD2 / FMUL2 / FFMA2: two FP32 operations per thread per instruction).
//
// A thread transforms two butterflies in lock step: a CP holds the same complex element of
// both, real parts in one float2 and imaginary parts in another ("structure of arrays"), so
// every add, multiply and fused multiply-add of the radix-R DFT, the twiddles and the
// |X|^2 accumulation is one paired instruction for two butterflies.  Subtraction is an FFMA2
// with -1 (exact), so no separate negation is ever issued.
#pragma once

#include <cstdint>

#include "isr_fft.cuh"

namespace isr {

struct CP {
    float2 re, im;   // (butterfly 0, butterfly 1)
};

__device__ __forceinline__ float2 bc(float c) { return make_float2(c, c); }

__device__ __forceinline__ CP padd(const CP& a, const CP& b)
{
    return CP{__fadd2_rn(a.re, b.re), __fadd2_rn(a.im, b.im)};
}

// a - b as b * (-1) + a (exact)
__device__ __forceinline__ CP psub(const CP& a, const CP& b)
{
    return CP{__ffma2_rn(b.re, bc(-1.f), a.re), __ffma2_rn(b.im, bc(-1.f), a.im)};
}

// a - i b and a + i b (the rotated add/sub of a radix-4 butterfly), one instruction each part
__device__ __forceinline__ CP psub_ib(const CP& a, const CP& b)   // a - i b = (a.re + b.im, a.im - b.re)
{
    return CP{__fadd2_rn(a.re, b.im), __ffma2_rn(b.re, bc(-1.f), a.im)};
}
__device__ __forceinline__ CP padd_ib(const CP& a, const CP& b)   // a + i b = (a.re - b.im, a.im + b.re)
{
    return CP{__ffma2_rn(b.im, bc(-1.f), a.re), __fadd2_rn(a.im, b.re)};
}

// z * exp(-2 pi i I / LEN) for compile-time I, LEN
template <int I, int LEN>
__device__ __forceinline__ CP pmul_w(const CP& z)
{
    constexpr int i = ((I % LEN) + LEN) % LEN;
    if constexpr (i == 0) {
        return z;
    } else if constexpr (2 * i == LEN) {                 // -1
        return CP{__fmul2_rn(z.re, bc(-1.f)), __fmul2_rn(z.im, bc(-1.f))};
    } else if constexpr (4 * i == LEN) {                 // -i: (re, im) -> (im, -re)
        return CP{z.im, __fmul2_rn(z.re, bc(-1.f))};
    } else if constexpr (4 * i == 3 * LEN) {             // +i: (re, im) -> (-im, re)
        return CP{__fmul2_rn(z.im, bc(-1.f)), z.re};
    } else {
        constexpr float c = float(ct_cos2pi(i, LEN));
        constexpr float s = float(ct_sin2pi(i, LEN));
        // (x + iy)(c - is) = (xc + ys) + i(yc - xs)
        return CP{__ffma2_rn(z.im, bc(s), __fmul2_rn(z.re, bc(c))), __ffma2_rn(z.re, bc(-s), __fmul2_rn(z.im, bc(c)))};
    }
}

// z * w for a runtime twiddle pair w = (wre + i wim), nwim = -wim
__device__ __forceinline__ CP pmul(const CP& z, const float2 wre, const float2 wim, const float2 nwim)
{
    return CP{__ffma2_rn(z.im, nwim, __fmul2_rn(z.re, wre)), __ffma2_rn(z.re, wim, __fmul2_rn(z.im, wre))};
}

// radix-4 DFT of (x0, x1, x2, x3), outputs in natural order
__device__ __forceinline__ void pdft4(CP& x0, CP& x1, CP& x2, CP& x3)
{
    const CP t0 = padd(x0, x2), t1 = psub(x0, x2), t2 = padd(x1, x3), t3 = psub(x1, x3);
    x0 = padd(t0, t2);
    x2 = psub(t0, t2);
    x1 = psub_ib(t1, t3);   // t1 - i t3
    x3 = padd_ib(t1, t3);   // t1 + i t3
}

// radix-16 DFT as 4 x 4: v[k] in, V[q] = sum_k v[k] W16^{qk} out in natural order
__device__ __forceinline__ void pdft16(CP (&v)[16])
{
    // first radix-4 over stride 4: for k1 < 4, inputs v[k1 + 4 k2], outputs Y[k1][q1]
    static_for<4>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        pdft4(v[k1], v[k1 + 4], v[k1 + 8], v[k1 + 12]);
        // v[k1 + 4 q1] now holds Y[k1][q1]; twiddle W16^{k1 q1}
        v[k1 + 4] = pmul_w<k1 * 1, 16>(v[k1 + 4]);
        v[k1 + 8] = pmul_w<k1 * 2, 16>(v[k1 + 8]);
        v[k1 + 12] = pmul_w<k1 * 3, 16>(v[k1 + 12]);
    });
    // second radix-4 over k1 for each q1: X[q1 + 4 q2] = sum_k1 Y'[k1][q1] W4^{k1 q2}
    static_for<4>([&](auto Q1) {
        constexpr int q1 = decltype(Q1)::value;
        pdft4(v[4 * q1 + 0], v[4 * q1 + 1], v[4 * q1 + 2], v[4 * q1 + 3]);
        // v[4 q1 + q2] holds X[q1 + 4 q2]
    });
    // reorder to natural order: X[q] at v[q]; currently X[q1 + 4 q2] sits at v[4 q1 + q2]
    CP t[16];
    static_for<16>([&](auto I) {
        constexpr int i = decltype(I)::value;
        t[(i & 3) * 4 + (i >> 2)] = v[i];
    });
    static_for<16>([&](auto I) {
        constexpr int i = decltype(I)::value;
        v[i] = t[i];
    });
}

}  // namespace isr

#include "isr_kernel.cuh"

namespace isr {

// ---------------------------------------------------------------- paired schedule, nfft 16384
// Radix order 4: Stockham passes [4, 16, 16, 16]; thread t transforms the butterfly pair
// (j, j + 1), j = 2 t (pass 0: four pairs j = 2 (t + 512 m)).  The exchange buffer is two
// planes (real, imaginary) with two pad floats per 32, so a pair is one 8-byte access per
// plane and every paired access is free of bank conflicts (pass 0's scalar stores: 2-way).
struct SchedP {
    static constexpr int N = 16384;
    static constexpr int PLANE = N + N / 16;
    static constexpr int OFF_MBAR = 0;
    static constexpr int OFF_BASE = 64;                        // float4 [t]: W_N^j, W_N^{j+1}
    static constexpr int OFF_TAB1 = OFF_BASE + 16 * 512;       // float4 [k-1][jm/2], Ns = 4
    static constexpr int OFF_TAB2 = OFF_TAB1 + 16 * 15 * 2;    // float4 [k-1][jm/2], Ns = 64
    static constexpr int OFF_STAGE = OFF_TAB2 + 16 * 15 * 32;
    static constexpr int STAGE_WORDS = Sched<14>::STAGE_WORDS;
    static constexpr int OFF_XRE = OFF_STAGE + 4 * STAGE_WORDS;
    static constexpr int OFF_XIM = OFF_XRE + 4 * PLANE;
    static constexpr int SMEM = OFF_XIM + 4 * PLANE;
};

__device__ __forceinline__ int pph(int i) { return i + 2 * (i >> 5); }

// twiddle pair table entry: (re W^{a}, re W^{a'}, im W^{a}, im W^{a'}) with W = exp(-2 pi i / n)
__device__ __forceinline__ float4 tw_pair(int a0, int a1, int n)
{
    double s0, c0, s1, c1;
    sincospi(-2.0 * (double)a0 / (double)n, &s0, &c0);
    sincospi(-2.0 * (double)a1 / (double)n, &s1, &c1);
    return make_float4((float)c0, (float)c1, (float)s0, (float)s1);
}

template <bool FULL>
__device__ __forceinline__ bool integrate_unit_p(const KArgs a, const int gx, const int c, unsigned char* smem,
                                                 const uint32_t phase0, const bool setup)
{
    using S = SchedP;
    constexpr int N = S::N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    float4* base = reinterpret_cast<float4*>(smem + S::OFF_BASE);
    float4* tab1 = reinterpret_cast<float4*>(smem + S::OFF_TAB1);
    float4* tab2 = reinterpret_cast<float4*>(smem + S::OFF_TAB2);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + S::OFF_STAGE);
    float* xre = reinterpret_cast<float*>(smem + S::OFF_XRE);
    float* xim = reinterpret_cast<float*>(smem + S::OFF_XIM);

    const int t = threadIdx.x;
    const int r = gx;
    const bool valid = r < a.n_ranges;
    const int64_t s_r = (int64_t)a.range_start + (int64_t)(valid ? r : a.n_ranges - 1) * a.range_step;
    const int p_begin = c * a.chunk_len;
    const int p_end = min(p_begin + a.chunk_len, a.n_ipp);
    const uint32_t bar = smem_u32(&mbar[0]);
    const int off = (int)(s_r & 3);
    const uint32_t copy_bytes = (uint32_t)(((off + a.code_len + 3) & ~3) * 4);
    const bool dbg_ok = debug_window_ok(a, s_r, off, copy_bytes, S::STAGE_WORDS, t);
    auto issue = [&](int p) {
        const uint32_t* src = a.echo + (int64_t)p * a.echo_stride + (s_r - off);
        bulk_load(smem_u32(stage), src, copy_bytes, bar);
    };

    if (setup) __syncthreads();
    if (setup) {
        base[t] = tw_pair(2 * t, 2 * t + 1, N);                      // pass 3: W_N^j, W_N^{j+1}
        for (int i = t; i < 15 * 2 + 15 * 32; i += kThreads) {
            if (i < 30) {                                             // pass 1: Ns 4, radix 16
                const int k = i / 2 + 1, jm = 2 * (i % 2);
                tab1[i] = tw_pair(jm * k, (jm + 1) * k, 64);
            } else {                                                  // pass 2: Ns 64, radix 16
                const int e = i - 30, k = e / 32 + 1, jm = 2 * (e % 32);
                tab2[e] = tw_pair(jm * k, (jm + 1) * k, 1024);
            }
        }
    }
    __syncthreads();
    if (t == 0 && dbg_ok && p_begin < p_end && p_begin != a.drop_ipp) issue(p_begin);

    const int8_t* code = reinterpret_cast<const int8_t*>(a.tx);
    // chips of pass 0: bit (2 m + e) * 4 + k for position 2 (t + 512 m) + e + 4096 k
    auto signs_of = [&](const int8_t* row) {
        uint32_t sg = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int pos = 2 * (t + 512 * m) + e + 4096 * k;
                    if ((FULL || pos < a.code_len) && row[pos] < 0) sg |= 1u << ((2 * m + e) * 4 + k);
                }
        return sg;
    };
    uint32_t signs = a.tx_stride == 0 ? signs_of(code) : 0u;

    float2 acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = make_float2(0.f, 0.f);
    const int j = 2 * t;
    bool timed_out = false;
    int it = 0;
    for (int p = p_begin; p < p_end; ++p, ++it) {
        const bool ok = mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (a.tx_stride != 0) signs = signs_of(code + (size_t)p * (size_t)a.tx_stride);

        // ---- pass 0: decode, radix 4 over stride 4096 (Ns = 1), scalar stores y[4 j' + q]
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int jm = 2 * (t + 512 * m);
            CP x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 rr, ii;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int pos = jm + e + 4096 * k;
                    float2 z = make_float2(0.f, 0.f);
                    if (FULL || pos < a.code_len)
                        z = decode<TX_PM1>(stage[off + pos], nullptr, pos,
                                           (signs << (31 - ((2 * m + e) * 4 + k))) & 0x80000000u);
                    if (e == 0) {
                        rr.x = z.x;
                        ii.x = z.y;
                    } else {
                        rr.y = z.x;
                        ii.y = z.y;
                    }
                }
                x[k] = CP{rr, ii};
            }
            pdft4(x[0], x[1], x[2], x[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i0 = pph(4 * jm + q), i1 = pph(4 * jm + 4 + q);
                xre[i0] = x[q].re.x;
                xim[i0] = x[q].im.x;
                xre[i1] = x[q].re.y;
                xim[i1] = x[q].im.y;
            }
        }
        __syncthreads();   // pass-0 outputs complete; the window is consumed
        if (t == 0 && dbg_ok && p + 1 < p_end && p + 1 != a.drop_ipp) {
            fence_proxy_async();
            issue(p + 1);
        }

        CP v[16];
        // ---- passes 1 and 2: radix 16 with table twiddles, read all / barrier / write all
#pragma unroll
        for (int ps = 1; ps <= 2; ++ps) {
            const int NS = ps == 1 ? 4 : 64;
            const float4* tb = ps == 1 ? tab1 : tab2;
            const int jmq = (j % NS) >> 1;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int i = pph(j + 1024 * k);
                v[k] = CP{*reinterpret_cast<const float2*>(&xre[i]), *reinterpret_cast<const float2*>(&xim[i])};
            }
#pragma unroll
            for (int k = 1; k < 16; ++k) {
                const float4 w = tb[(k - 1) * (NS / 2) + jmq];
                const float2 wre = make_float2(w.x, w.y), wim = make_float2(w.z, w.w);
                v[k] = pmul(v[k], wre, wim, __fmul2_rn(wim, bc(-1.f)));
            }
            pdft16(v);
            __syncthreads();
            const int idxD = (j / NS) * NS * 16 + (j % NS);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int i = pph(idxD + q * NS);
                *reinterpret_cast<float2*>(&xre[i]) = v[q].re;
                *reinterpret_cast<float2*>(&xim[i]) = v[q].im;
            }
            __syncthreads();
        }
        // ---- pass 3: radix 16, Ns = 1024, recurrence twiddles, accumulate |X|^2
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int i = pph(j + 1024 * k);
            v[k] = CP{*reinterpret_cast<const float2*>(&xre[i]), *reinterpret_cast<const float2*>(&xim[i])};
        }
        {
            const float4 b = base[t];
            const float2 wre = make_float2(b.x, b.y), wim = make_float2(b.z, b.w);
            const float2 nwim = __fmul2_rn(wim, bc(-1.f));
            float2 cre = wre, cim = wim;
#pragma unroll
            for (int k = 1; k < 16; ++k) {
                v[k] = pmul(v[k], cre, cim, __fmul2_rn(cim, bc(-1.f)));
                if (k < 15) {
                    const CP nc = pmul(CP{cre, cim}, wre, wim, nwim);
                    cre = nc.re;
                    cim = nc.im;
                }
            }
        }
        pdft16(v);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            acc[q] = __ffma2_rn(v[q].im, v[q].im, __ffma2_rn(v[q].re, v[q].re, acc[q]));
    }

    if (timed_out) {
        if (t == 0) atomicOr(a.status, 1);
        mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        return false;
    }
    // bins j + 1024 q and j + 1 + 1024 q
    if (valid) {
        float* out = a.partial + ((int64_t)c * a.n_ranges + r) * N;
#pragma unroll
        for (int q = 0; q < 16; ++q) *reinterpret_cast<float2*>(&out[j + 1024 * q]) = acc[q];
    }
    return true;
}

template <bool FULL>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_p(KArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) mbar_init(smem_u32(&mbar[0]), 1);
    fence_barrier_init();
    integrate_unit_p<FULL>(a, blockIdx.x, blockIdx.y, smem, 0u, true);
}

// ---------------------------------------------------------------- paired schedule [16, 32, 32]
// Radix order 5 (nfft 16384): the Stockham passes of radix order 1 with paired arithmetic.
//  pass 0 (radix 16, Ns = 1): thread t transforms butterflies t and t + 512 as one CP
//    stream.  Their outputs y[16 j + q] lie N/2 apart, so the first exchange layout keeps
//    y[s] and y[s + N/2] in one 16-byte slot s < N/2, (re, re', im, im'): one 16-byte store
//    per output pair.
//  pass 1 (radix 32, Ns = 16) and pass 2 (radix 32, Ns = 512): butterfly t.  With input
//    twiddles w^k the first radix-2 DIF stage of the 32-point DFT is
//        A_k = w^k (x_k + w^16 x_{k+16}),   B_k = (w W_32)^k (x_k - w^16 x_{k+16}),  k < 16,
//    computed as scalar FP32 for s_k = x_k + w^16 x_{k+16} and d_k = x_k - w^16 x_{k+16},
//    then (s_k, d_k) times the twiddle pair (w^k, (w W_32)^k) as one CP; a paired 16-point
//    DFT of (A, B) gives X[2u] (lane 0) and X[2u + 1] (lane 1).  Pass 1 reads its inputs
//    k, k + 16 (N/2 apart) as one slot of the first layout and writes the plain padded
//    complex layout of radix order 1, which pass 2 reads; pass 2 accumulates |X|^2 for
//    the bin pair (2u, 2u + 1) in one paired register.
struct SchedQ {
    static constexpr int N = 16384;
    static constexpr int SLOTS = N / 2 + N / 32;   // first layout: 16-byte slots, one pad per 16
    static constexpr int NPAD = N + N / 16;        // second layout: float2, one pad per 16
    static constexpr int OFF_MBAR = 0;
    static constexpr int OFF_BASE = 64;                      // float4 [t]: (w, w W_32), w = W_N^t
    static constexpr int OFF_W16 = OFF_BASE + 16 * 512;      // float2 [t]: W_1024^t (= w^16, pass 2)
    static constexpr int OFF_TAB1 = OFF_W16 + 8 * 512;       // float4 [k - 1][jm], pass 1, k = 1..15
    static constexpr int OFF_T16 = OFF_TAB1 + 16 * 15 * 16;  // float2 [jm]: W_32^jm (= w^16, pass 1)
    static constexpr int OFF_STAGE = OFF_T16 + 8 * 16;
    static constexpr int STAGE_WORDS = N + 4;
    static constexpr int OFF_XCH = OFF_STAGE + 4 * STAGE_WORDS;
    static constexpr int XCH_BYTES = 16 * SLOTS > 8 * NPAD ? 16 * SLOTS : 8 * NPAD;
    static constexpr int SMEM = OFF_XCH + XCH_BYTES;
    static_assert(OFF_STAGE % 16 == 0 && OFF_XCH % 16 == 0, "bulk copies and 16-byte slots need alignment");
};

// first exchange layout: slot s -> s + s / 16 (16-byte units)
__device__ __forceinline__ int qslot(int s) { return s + (s >> 4); }

// first DIF stage of a 32-point DFT for inputs a = x_k, b = x_{k+16} (scalar FP32):
// (s, d) = (a + w16 b, a - w16 b) as one CP
__device__ __forceinline__ CP dif_first(const float2 a, const float2 b, const float2 w16)
{
    const float2 y = cmul(b, w16);
    return CP{make_float2(a.x + y.x, a.x - y.x), make_float2(a.y + y.y, a.y - y.y)};
}

template <bool FULL>
__device__ __forceinline__ bool integrate_unit_q(const KArgs a, const int gx, const int c, unsigned char* smem,
                                                 const uint32_t phase0, const bool setup)
{
    using S = SchedQ;
    constexpr int N = S::N;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    float4* base = reinterpret_cast<float4*>(smem + S::OFF_BASE);
    float2* w16t = reinterpret_cast<float2*>(smem + S::OFF_W16);
    float4* tab1 = reinterpret_cast<float4*>(smem + S::OFF_TAB1);
    float2* t16 = reinterpret_cast<float2*>(smem + S::OFF_T16);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + S::OFF_STAGE);
    float4* x1 = reinterpret_cast<float4*>(smem + S::OFF_XCH);   // first layout
    float2* x2 = reinterpret_cast<float2*>(smem + S::OFF_XCH);   // second layout

    const int t = threadIdx.x;
    const int r = gx;
    const bool valid = r < a.n_ranges;
    const int64_t s_r = (int64_t)a.range_start + (int64_t)(valid ? r : a.n_ranges - 1) * a.range_step;
    const int p_begin = c * a.chunk_len;
    const int p_end = min(p_begin + a.chunk_len, a.n_ipp);
    const uint32_t bar = smem_u32(&mbar[0]);
    const int off = (int)(s_r & 3);
    const uint32_t copy_bytes = (uint32_t)(((off + a.code_len + 3) & ~3) * 4);
    const bool dbg_ok = debug_window_ok(a, s_r, off, copy_bytes, S::STAGE_WORDS, t);
    auto issue = [&](int p) {
        const uint32_t* src = a.echo + (int64_t)p * a.echo_stride + (s_r - off);
        bulk_load(smem_u32(stage), src, copy_bytes, bar);
    };

    if (setup) __syncthreads();
    if (setup) {
        base[t] = tw_pair(t, t + 512, N);                       // (w, w W_32), w = W_N^t
        {
            double sn, cs;
            sincospi(-2.0 * (double)t / 1024.0, &sn, &cs);     // w^16 = W_1024^t
            w16t[t] = make_float2((float)cs, (float)sn);
        }
        if (t < 15 * 16) {                                      // pass 1: w = W_512^jm
            const int k = t / 16 + 1, jm = t % 16;
            tab1[t] = tw_pair(jm * k, (jm + 16) * k, 512);     // (w^k, (w W_32)^k)
        } else if (t < 15 * 16 + 16) {
            const int jm = t - 15 * 16;
            double sn, cs;
            sincospi(-2.0 * (double)jm / 32.0, &sn, &cs);       // w^16 = W_32^jm
            t16[jm] = make_float2((float)cs, (float)sn);
        }
    }
    __syncthreads();
    if (t == 0 && dbg_ok && p_begin < p_end && p_begin != a.drop_ipp) issue(p_begin);

    const int8_t* code = reinterpret_cast<const int8_t*>(a.tx);
    // chips of pass 0: bit b * 16 + k for position t + 512 b + 1024 k (radix order 1's layout)
    uint32_t signs = a.tx_stride == 0 ? load_signs<14, 1>(code, t, a.code_len) : 0u;

    float2 acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = make_float2(0.f, 0.f);
    const int jm = t & 15;
    bool timed_out = false;
    int it = 0;
    for (int p = p_begin; p < p_end; ++p, ++it) {
        const bool ok = mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        if (a.tx_stride != 0) signs = load_signs<14, 1>(code + (size_t)p * (size_t)a.tx_stride, t, a.code_len);

        CP v[16];
        // ---- pass 0: decode, two radix-16 butterflies (t, t + 512) in lock step
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float2 rr, ii;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int pos = t + 512 * b + 1024 * k;
                float2 z = make_float2(0.f, 0.f);
                if (FULL || pos < a.code_len)
                    z = decode<TX_PM1>(stage[off + pos], nullptr, pos, (signs << (31 - (b * 16 + k))) & 0x80000000u);
                if (b == 0) {
                    rr.x = z.x;
                    ii.x = z.y;
                } else {
                    rr.y = z.x;
                    ii.y = z.y;
                }
            }
            v[k] = CP{rr, ii};
        }
        pdft16(v);
#pragma unroll
        for (int q = 0; q < 16; ++q) x1[qslot(16 * t) + q] = make_float4(v[q].re.x, v[q].re.y, v[q].im.x, v[q].im.y);
        __syncthreads();   // pass-0 outputs complete; the window is consumed
        if (t == 0 && dbg_ok && p + 1 < p_end && p + 1 != a.drop_ipp) {
            fence_proxy_async();
            issue(p + 1);
        }

        // ---- pass 1: radix 32, Ns = 16, twiddles from the table
        const float2 w16p1 = t16[jm];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float4 e = x1[qslot(t) + 544 * k];   // inputs k and k + 16
            v[k] = dif_first(make_float2(e.x, e.z), make_float2(e.y, e.w), w16p1);
        }
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const float4 w = tab1[(k - 1) * 16 + jm];
            const float2 wim = make_float2(w.z, w.w);
            v[k] = pmul(v[k], make_float2(w.x, w.y), wim, __fmul2_rn(wim, bc(-1.f)));
        }
        pdft16(v);
        __syncthreads();
        {
            // X[q] of butterfly t at (t / 16) 512 + t % 16 + 16 q, padded one per 16
            float2* o = x2 + (t >> 4) * 544 + (t & 15);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                o[17 * (2 * u)] = make_float2(v[u].re.x, v[u].im.x);
                o[17 * (2 * u + 1)] = make_float2(v[u].re.y, v[u].im.y);
            }
        }
        __syncthreads();

        // ---- pass 2: radix 32, Ns = 512, twiddles by a paired recurrence; accumulate |X|^2
        {
            const float2* in = x2 + t + (t >> 4);
            const float2 w16p2 = w16t[t];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = dif_first(in[544 * k], in[544 * (k + 16)], w16p2);
            const float4 b2 = base[t];
            const float2 c1re = make_float2(b2.x, b2.y), c1im = make_float2(b2.z, b2.w);
            const float2 c1nim = __fmul2_rn(c1im, bc(-1.f));
            float2 cre = c1re, cim = c1im;
#pragma unroll
            for (int k = 1; k < 16; ++k) {
                v[k] = pmul(v[k], cre, cim, __fmul2_rn(cim, bc(-1.f)));
                if (k < 15) {
                    const CP nc = pmul(CP{cre, cim}, c1re, c1im, c1nim);
                    cre = nc.re;
                    cim = nc.im;
                }
            }
        }
        pdft16(v);
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = __ffma2_rn(v[u].im, v[u].im, __ffma2_rn(v[u].re, v[u].re, acc[u]));
    }

    if (timed_out) {
        if (t == 0) atomicOr(a.status, 1);
        mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        return false;
    }
    // bins t + 512 q: acc[u] holds q = 2u (x) and q = 2u + 1 (y)
    if (valid) {
        float* out = a.partial + ((int64_t)c * a.n_ranges + r) * N;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            out[t + 1024 * u] = acc[u].x;
            out[t + 1024 * u + 512] = acc[u].y;
        }
    }
    return true;
}

template <bool FULL>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_q(KArgs a)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) mbar_init(smem_u32(&mbar[0]), 1);
    fence_barrier_init();
    integrate_unit_q<FULL>(a, blockIdx.x, blockIdx.y, smem, 0u, true);
}

}  // namespace isr
