// isr_kernel.cuh -- fused decode -> FFT -> |X|^2 integration kernel for sm_103a.
//
// One CTA (512 threads) owns G = 16384 / nfft range gates for one chunk of IPPs (for
// nfft = 16384: one gate).  Per IPP and gate it
//   1. waits for the gate's int16 IQ echo window, staged into shared memory by a bulk
//      asynchronous copy (cp.async.bulk + mbarrier) that was issued one IPP ahead;
//   2. decodes x[k] = conj(eps[k]) * m[s_r + k] on the fly while loading the first
//      radix pass (Eq. 7 of the paper, the "complex multiplication" kernel of Sec. 3.2.1);
//   3. runs a three-pass Stockham FFT (radices 8..32 in one of several orders): each thread
//      owns 32 points, every pass is a register-resident radix-R DFT, passes exchange data
//      through a padded (bank-conflict-free) shared-memory buffer, and the middle pass works
//      in place so that only three barriers of the gate separate the passes of an IPP (the
//      transform of Sec. 3.2.2);
//   4. adds |X[f]|^2 into 32 FP32 accumulators per thread that stay in registers for the
//      whole IPP chunk (Eq. 8, the "spectrum accumulation" kernel of Sec. 3.2.3).
// At the end of the chunk each thread writes its 32 partial sums once; a separate
// reduction adds the chunk partials into FP64 accumulators.
#pragma once

#include <cstdint>

#include "isr_fft.cuh"
#include "isr_tc.cuh"
#include "isr_tc05.cuh"
#include "isr_tmem.cuh"

namespace isr {

enum TxKind { TX_CI16 = 0, TX_C32 = 1, TX_PM1 = 2 };

constexpr int kThreads = 512;

// ---------------------------------------------------------------- per-size schedule
// Radix orders of the three-pass sizes (nfft 2048 .. 16384).  ORDER 0 is the default;
// Plan.autotune and the batched launch time them on the caller's data and pick per size.
__host__ __device__ constexpr int radix_of(int log2n, int order, int p)
{
    if (log2n <= 5) return p == 0 ? (1 << log2n) : 1;
    if (log2n <= 10) {
        constexpr int a0[5] = {8, 16, 16, 32, 32}, a1[5] = {8, 8, 16, 16, 32};
        return p == 0 ? a0[log2n - 6] : p == 1 ? a1[log2n - 6] : 1;
    }
    constexpr int t11[3][3] = {{16, 16, 8}, {8, 16, 16}, {32, 8, 8}};
    constexpr int t12[3][3] = {{16, 16, 16}, {32, 16, 8}, {8, 16, 32}};
    constexpr int t13[3][3] = {{32, 16, 16}, {16, 16, 32}, {16, 32, 16}};
    constexpr int t14[3][3] = {{32, 32, 16}, {16, 32, 32}, {32, 16, 32}};
    return log2n == 11 ? t11[order][p] : log2n == 12 ? t12[order][p] : log2n == 13 ? t13[order][p] : t14[order][p];
}
constexpr int kOrders = 4;   // 0..2 Stockham orders, 3 the warp-local schedule

// TMT: the inter-pass twiddles of passes 1 and 2 are precomputed per thread into tensor
// memory once per CTA (three-pass sizes with a first radix >= 16) instead of being formed
// from tables and recurrences in every IPP.
template <int LOG2N, int ORDER = 0, bool TMT = false>
struct Sched {
    static constexpr int N = 1 << LOG2N;
    static constexpr int E = N < 32 ? N : 32;   // points per thread
    static constexpr int T = N / E;             // threads per transform
    static constexpr int G = kThreads / T;      // transforms (gates) per CTA
    // radices of the Stockham passes, first to last
    static constexpr int NP = LOG2N <= 5 ? 1 : LOG2N <= 10 ? 2 : 3;
    static constexpr int R0 = radix_of(LOG2N, ORDER, 0);
    static constexpr int R1 = radix_of(LOG2N, ORDER, 1);
    static constexpr int R2 = radix_of(LOG2N, ORDER, 2);
    static_assert(R0 * R1 * R2 == N, "radix product must equal nfft");
    __host__ __device__ static constexpr int radix(int p) { return p == 0 ? R0 : p == 1 ? R1 : R2; }
    // Twiddles of pass p >= 1: w^k with w = exp(-2 pi i (j mod Ns) / (Ns R)).  A pass whose
    // distinct values fit a small table (Ns (R - 1) <= 1024) reads them from a per-CTA
    // table laid out [k - 1][j mod Ns] (consecutive lanes, consecutive entries); other
    // passes build w^k by recurrence from a per-thread base w kept in a slot table.
    __host__ __device__ static constexpr int ns(int p) { return p == 1 ? R0 : R0 * R1; }
    __host__ __device__ static constexpr bool tab(int p) { return ns(p) * (radix(p) - 1) <= 1024; }
    // table entries (float2), stored as pairs (w^{2p+1}, w^{2p+2}) in float4 [p][j mod Ns]
    // radix 16 and 32 keep only (w, w^2), (w^3, w^4), (w^8, w^16) per j mod Ns (6 entries) and
    // form the other powers with one product each; smaller radices keep every power
    __host__ __device__ static constexpr int tabw(int p) { return radix(p) >= 16 ? 6 : radix(p); }
    static constexpr int TAB1 = (!TMT && NP > 1 && tab(1)) ? ns(1) * tabw(1) : 0;
    static constexpr int TAB2 = (!TMT && NP > 2 && tab(2)) ? ns(2) * tabw(2) : 0;
    static constexpr int SLOTS1 = (!TMT && NP > 1 && !tab(1)) ? E / R1 : 0;           // per-thread bases
    static constexpr int SLOTS2 = (!TMT && NP > 2 && !tab(2)) ? E / R2 : 0;
    // TMEM twiddles: per thread and pass, (E / R)(R - 1) <= 31 complex values as [b][k - 1] in
    // 64 columns of the thread's lane; the warps of one lane quarter take 128 columns each
    static_assert(!TMT || (NP == 3 && R0 >= 16 && kThreads == 512), "TMEM twiddles: three-pass sizes, first radix >= 16");
    static constexpr int TM_COLS = 512;
    static constexpr int NSLOT = SLOTS1 + SLOTS2;
    // shared-memory exchange buffer: one pad element per PADP keeps every access pattern
    // of the passes free of bank conflicts (stride R0 + 1 for the first pass' writes)
    static constexpr int PADP = R0 < 16 ? 16 : R0;
    // the middle pass writes its outputs back into the slots it read (in place, no barrier
    // between its reads and writes); the last pass then reads through the index permutation.
    // Needs Ns = R0 = PADP for conflict-free, constant-offset permuted reads.
    static constexpr bool INPLACE = NP == 3 && R0 >= 16;
    static constexpr int NPAD = NP > 1 ? N + N / PADP : 0;
    // window + alignment slack (16-byte multiple); at nfft 16384 room for the padded
    // 16-row layout of the tensor-core first pass
    static constexpr int STAGE_WORDS = LOG2N == 14 ? 16 * kTcSeg : N + 4;
    // dynamic shared-memory layout (bytes)
    static constexpr int OFF_MBAR = 0;
    // at least 8 mbarrier slots: the batched launch keeps slots 0..7 alive across shapes
    static constexpr int OFF_TW = 16 * ((8 * (G < 8 ? 8 : G) + 15) / 16);
    static constexpr int OFF_TMEMADDR = OFF_TW;   // the CTA's TMEM base address (TMT)
    static constexpr int OFF_TAB = OFF_TW + 16 * ((8 * NSLOT * T + 15) / 16) + (TMT ? 16 : 0);
    static constexpr int OFF_STAGE = OFF_TAB + 16 * ((8 * (TAB1 + TAB2) + 15) / 16);
    static constexpr int OFF_XCH = OFF_STAGE + 4 * STAGE_WORDS * G;
    static constexpr int SMEM = OFF_XCH + 8 * NPAD * G;
};

__device__ __forceinline__ int pidx(int i, int padp) { return i + i / padp; }

// u[k] = buf[padded(j + k * STRIDE)], k < R.  When STRIDE is a multiple of the pad period
// the padded addresses are one base plus compile-time offsets.
template <int STRIDE, int R, int PADP>
__device__ __forceinline__ void load_strided(float2* u, const float2* buf, int j)
{
    if constexpr (STRIDE % PADP == 0) {
        const float2* b = buf + pidx(j, PADP);
        static_for<R>([&](auto Kc) {
            constexpr int k = decltype(Kc)::value;
            u[k] = b[k * (STRIDE + STRIDE / PADP)];
        });
    } else {
        static_for<R>([&](auto Kc) {
            constexpr int k = decltype(Kc)::value;
            u[k] = buf[pidx(j + k * STRIDE, PADP)];
        });
    }
}

// buf[padded(base + q * STRIDE)] = X[q] = u[bitrev(q)], q < R (the DFT output order).
// base is a multiple of R when STRIDE == 1 and R >= PADP or STRIDE is a multiple of PADP.
template <int STRIDE, int R, int PADP>
__device__ __forceinline__ void store_strided(float2* buf, int base, const float2* u)
{
    if constexpr ((STRIDE == 1 && R == PADP) || (STRIDE % PADP == 0)) {
        float2* b = buf + pidx(base, PADP);
        static_for<R>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            constexpr int o = STRIDE == 1 ? q : q * (STRIDE + STRIDE / PADP);
            b[o] = u[BitRev<R>::at(q)];
        });
    } else {
        static_for<R>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            buf[pidx(base + q * STRIDE, PADP)] = u[BitRev<R>::at(q)];
        });
    }
}

struct KArgs {
    const uint32_t* echo;   // complex int16 samples as 32-bit words, 16-byte aligned
    int64_t echo_stride;    // words per IPP row (multiple of 4)
    const void* tx;         // code rows
    int64_t tx_stride;      // chips between code rows (0 = shared)
    float* partial;         // [n_chunks][n_ranges][N]
    int* status;            // bit 0: a wait timed out
    int n_ranges;
    int range_start;
    int range_step;
    int code_len;
    int n_ipp;              // IPPs in this launch (rows of echo)
    int chunk_len;          // IPPs per chunk (blockIdx.y)
    unsigned wait_limit;    // try_wait polls before giving up
    int drop_ipp;           // test hook: never stage this IPP (launch-relative), -1 = off
    // debug builds: [5] = SM cycles of the IPP loop's phases summed over CTAs as seen by thread 0
    // (window wait + barrier, pass 0, middle pass, last pass) and the IPPs counted; NULL = off
    unsigned long long* phase_cycles = nullptr;
};

// ---------------------------------------------------------------- async-copy primitives
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// arm the barrier for `bytes` and start one bulk global->shared copy completing on it
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// bounded wait for phase `parity` of the barrier; false if it did not complete in time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---------------------------------------------------------------- decode helpers
__device__ __forceinline__ float2 iq_of(uint32_t w)
{
    return make_float2((float)(int16_t)(w & 0xffffu), (float)(int16_t)(w >> 16));
}

// Binary-phase codes: CVT picks how a sample's int16 pair becomes floats.  The first passes decode
// even samples with the conversion instruction and odd ones with the magic-number form below, so
// that both pipes share the work: at nfft 16384 either form alone took 320-323 ms per
// integration of the realistic workload (order 6), the split 312.5 ms.
template <int TXT, bool CVT = false>
__device__ __forceinline__ float2 decode(uint32_t w, const void* txrow, int pos, uint32_t sbit)
{
    if constexpr (TXT == TX_PM1 && CVT) {
        // the conversion instruction, then sbit (the chip's sign in bit 31) flips both signs
        const float2 m = iq_of(w);
        return make_float2(__int_as_float(__float_as_int(m.x) ^ sbit), __int_as_float(__float_as_int(m.y) ^ sbit));
    } else if constexpr (TXT == TX_PM1) {
        // sbit holds the chip's sign in bit 31.  Exact int16 -> float conversion on the integer
        // and FMA pipes (the conversion instruction runs on a narrower pipe): XOR 0x8000 turns
        // each int16 into the offset-binary
        // u = v + 2^15 in [0, 2^16); placed in the low mantissa bits of 1.5 * 2^23 it gives the
        // float 1.5 * 2^23 + u exactly, and adding -(1.5 * 2^23 + 2^15) leaves v (all integers
        // below 2^24).  The chip's sign goes into both magic constants, so the sum is +-v.
        const uint32_t cs = 0x4B400000u ^ sbit;       //  1.5 * 2^23, with the chip's sign
        const uint32_t ks = 0xCB408000u ^ sbit;       // -(1.5 * 2^23 + 2^15), with the chip's sign
        const uint32_t wb = w ^ 0x80008000u;
        const float fi = __int_as_float(__byte_perm(wb, cs, 0x7610));   // bytes wb.0, wb.1, cs.2, cs.3
        const float fq = __int_as_float(__byte_perm(wb, cs, 0x7632));   // bytes wb.2, wb.3, cs.2, cs.3
        return make_float2(fi + __int_as_float(ks), fq + __int_as_float(ks));
    } else if constexpr (TXT == TX_CI16) {
        float2 m = iq_of(w);
        float2 e = iq_of(__ldg(reinterpret_cast<const uint32_t*>(txrow) + pos));
        // conj(e) * m = (ex mx + ey my) + i (ex my - ey mx)
        return make_float2(fmaf(e.x, m.x, e.y * m.y), fmaf(e.x, m.y, -e.y * m.x));
    } else {
        float2 m = iq_of(w);
        float2 e = __ldg(reinterpret_cast<const float2*>(txrow) + pos);
        return make_float2(fmaf(e.x, m.x, e.y * m.y), fmaf(e.x, m.y, -e.y * m.x));
    }
}

// sign bits of the code chips a thread decodes in the first pass (bit b*R0 + k)
template <int LOG2N, int ORDER>
__device__ __forceinline__ uint32_t load_signs(const int8_t* row, int t, int code_len)
{
    using S = Sched<LOG2N, ORDER>;
    uint32_t m = 0;
    static_for<S::E / S::R0>([&](auto Bc) {
        constexpr int b = decltype(Bc)::value;
        static_for<S::R0>([&](auto Kc) {
            constexpr int k = decltype(Kc)::value;
            int pos = t + S::T * b + k * (S::N / S::R0);
            if (pos < code_len && row[pos] < 0) m |= 1u << (b * S::R0 + k);
        });
    });
    return m;
}

// apply the Stockham twiddles w^k (k = 1..R-1) to v[0..R) given w.  Radix <= 8: a chain
// w^{k+1} = w^k w.  Radix 16 and 32: the same R - 2 products arranged as a shallow tree,
// w^2..w^7 from w, then w^{8 m + i} = w^{8 m} w^i with w^8 = (w^4)^2, w^16 = (w^8)^2 and
// w^24 = w^16 w^8, so no power is more than six products from w.
template <int R>
__device__ __forceinline__ void twiddle(float2* v, float2 w)
{
    if constexpr (R < 16) {
        float2 cur = w;
        static_for<R - 1>([&](auto Kc) {
            constexpr int k = decltype(Kc)::value + 1;
            v[k] = cmul(v[k], cur);
            if constexpr (k + 1 < R) cur = cmul(cur, w);
        });
    } else {
        float2 p[8];
        p[1] = w;
        p[2] = cmul(w, w);
        p[3] = cmul(p[2], w);
        p[4] = cmul(p[2], p[2]);
        p[5] = cmul(p[4], w);
        p[6] = cmul(p[4], p[2]);
        p[7] = cmul(p[4], p[3]);
        static_for<7>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value + 1;
            v[i] = cmul(v[i], p[i]);
        });
        const float2 w8 = cmul(p[4], p[4]);
        v[8] = cmul(v[8], w8);
        static_for<7>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value + 1;
            v[8 + i] = cmul(v[8 + i], cmul(w8, p[i]));
        });
        if constexpr (R == 32) {
            const float2 w16 = cmul(w8, w8);
            v[16] = cmul(v[16], w16);
            static_for<7>([&](auto Ic) {
                constexpr int i = decltype(Ic)::value + 1;
                v[16 + i] = cmul(v[16 + i], cmul(w16, p[i]));
            });
            const float2 w24 = cmul(w16, w8);
            v[24] = cmul(v[24], w24);
            static_for<7>([&](auto Ic) {
                constexpr int i = decltype(Ic)::value + 1;
                v[24 + i] = cmul(v[24 + i], cmul(w24, p[i]));
            });
        }
    }
}

// apply w^k (k = 1..R-1) from a pair table: float4 [p][jm] = (w^{2p+1}, w^{2p+2}); one
// 16-byte load brings two twiddles
template <int R, int NS>
__device__ __forceinline__ void twiddle_tab(float2* v, const float2* tab, int jm)
{
    const float4* t = reinterpret_cast<const float4*>(tab) + jm;
    static_for<R / 2>([&](auto Pc) {
        constexpr int pr = decltype(Pc)::value;
        const float4 e = t[pr * NS];
        v[2 * pr + 1] = cmul(v[2 * pr + 1], make_float2(e.x, e.y));
        if constexpr (2 * pr + 2 < R) v[2 * pr + 2] = cmul(v[2 * pr + 2], make_float2(e.z, e.w));
    });
}

// apply w^k (k = 1..R-1, R = 16 or 32) from three table pairs (w, w^2), (w^3, w^4), (w^8, w^16):
// w^5..w^7 = w^4 w^{1..3}, w^{8+i} = w^8 w^i, w^{16+i} = w^16 w^i; every power is at most two
// products from the table (error ~2 ulp), and the table costs 3 of the R/2 16-byte loads
template <int R, int NS>
__device__ __forceinline__ void twiddle_tab3(float2* v, const float2* tab, int jm)
{
    static_assert(R == 16 || R == 32, "three-pair table covers radix 16 and 32");
    const float4* t = reinterpret_cast<const float4*>(tab) + jm;
    const float4 a = t[0], b = t[NS], c = t[2 * NS];
    float2 w[8];
    w[1] = make_float2(a.x, a.y);
    w[2] = make_float2(a.z, a.w);
    w[3] = make_float2(b.x, b.y);
    w[4] = make_float2(b.z, b.w);
    w[5] = cmul(w[4], w[1]);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
    const float2 w8 = make_float2(c.x, c.y);
    static_for<7>([&](auto Ic) {
        constexpr int i = decltype(Ic)::value + 1;
        v[i] = cmul(v[i], w[i]);
    });
    v[8] = cmul(v[8], w8);
    static_for<7>([&](auto Ic) {
        constexpr int i = decltype(Ic)::value + 1;
        v[8 + i] = cmul(v[8 + i], cmul(w8, w[i]));
    });
    if constexpr (R == 32) {
        const float2 w16 = make_float2(c.z, c.w);
        v[16] = cmul(v[16], w16);
        static_for<7>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value + 1;
            v[16 + i] = cmul(v[16 + i], cmul(w16, w[i]));
        });
        const float2 w24 = cmul(w16, w8);
        v[24] = cmul(v[24], w24);
        static_for<7>([&](auto Ic) {
            constexpr int i = decltype(Ic)::value + 1;
            v[24 + i] = cmul(v[24 + i], cmul(w24, w[i]));
        });
    }
}

// apply w^k (k = 1..R-1) to butterfly B of a pass from this thread's TMEM twiddles (complex
// index e = B (R - 1) + k - 1, eight per 16-column load)
template <int R, int B>
__device__ __forceinline__ void twiddle_tmem(float2* u, uint32_t addr)
{
    constexpr int e0 = B * (R - 1), e1 = e0 + R - 1;
    static_for<4>([&](auto Cc) {
        constexpr int c = decltype(Cc)::value;
        if constexpr (8 * c < e1 && 8 * c + 8 > e0) {
            uint32_t r[16];
            tmem_ld16(addr + 16 * c, r);
            tmem_wait_ld(r);
            static_for<8>([&](auto Ec) {
                constexpr int i = decltype(Ec)::value, e = 8 * c + i;
                if constexpr (e >= e0 && e < e1) {
                    constexpr int k = e - e0 + 1;
                    u[k] = cmul(u[k], make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1])));
                }
            });
        }
    });
}

// R-point DFT of a pass of the fused unit: from nfft 1024 up the tangent-form radix-2^2 network
// (sdft: two instead of four instructions per non-trivial twiddle product, same outputs), below
// it the plain radix-2 network, which measured faster there
template <int R, int LOG2N>
__device__ __forceinline__ void unit_dft(float2* u)
{
    if constexpr (LOG2N >= 10 && R >= 8) sdft<R>(u);
    else dft<R, LOG2N >= 10>(u);
}

// ---------------------------------------------------------------- debug-build window check
// With -DISR_DEBUG every gate checks, before it stages anything, that its window copy lies
// inside the echo row (s_r >= 0, s_r + code_len <= echo_stride, the 16-byte-rounded copy
// [s_r - off, s_r - off + words) within the row) and fits the stage buffer.  A gate that
// fails sets bit 1 of the status word and never issues a copy: its bounded waits then run
// out and the unit ends through the timeout path, with no access outside any buffer.  The
// release build checks nothing here (the host validates the geometry before every launch).
template <class A>
__device__ __forceinline__ bool debug_window_ok(const A& a, int64_t s_r, int off, uint32_t copy_bytes,
                                                int stage_words, int t)
{
#ifdef ISR_DEBUG
    const int64_t first = s_r - off, words = (int64_t)(copy_bytes / 4);
    const bool ok = s_r >= 0 && a.code_len >= 1 && s_r + a.code_len <= a.echo_stride && first >= 0 &&
                    (first & 3) == 0 && first + words <= a.echo_stride && off + a.code_len <= stage_words &&
                    words <= stage_words;
    if (!ok && t == 0) atomicOr(a.status, 2);
    return ok;
#else
    (void)a, (void)s_r, (void)off, (void)copy_bytes, (void)stage_words, (void)t;
    return true;
#endif
}

// ---------------------------------------------------------------- the fused work unit
// One unit = gates [gx G, gx G + G) of IPP chunk c of the launch `a`.  Each gate group g
// owns mbarrier slot g (initialised by the caller); phase0 is the number of phases that
// slot has completed before this unit (units run back to back in the batched launch).
// setup = false reuses the twiddle tables left by the previous unit of the same shape.
// FULL = true promises code_len == nfft (no zero padding, no per-sample bound check).
// Returns false if a staged-window wait ran out.
// P0 selects the engine of the first pass: the SIMT radix-R0 DFT, or (nfft 16384, radix
// order 1, binary-phase, full-length codes only) a split-precision tensor-core GEMM.
// A is how the arguments arrive: by value from a kernel parameter, or (persistent kernels) as a
// reference to a shared-memory copy, read where needed rather than held in registers.
// TMT: twiddles of passes 1 and 2 from tensor memory at tmem (the CTA's allocation of
// Sched::TM_COLS columns); setup writes them.
// SPLITDEC: binary-phase samples of the first pass decoded half with the conversion instruction,
// half in the magic-number form (see decode); false: all with the conversion instruction.
template <int LOG2N, int TXT, int ORDER = 0, bool FULL = false, int P0 = P0_SIMT, class A = const KArgs,
          bool TMT = false, bool SPLITDEC = true>
__device__ __forceinline__ bool integrate_unit(A a, const int gx, const int c, unsigned char* smem,
                                               const uint32_t phase0, const bool setup, const uint32_t tmem = 0)
{
    using S = Sched<LOG2N, ORDER, TMT>;
    constexpr int N = S::N, E = S::E, T = S::T, G = S::G, NP = S::NP;
    constexpr int R0 = S::R0;
    constexpr int RL = S::radix(NP - 1);  // radix of the last pass
    // transforms of 32 or fewer threads live inside one warp and sync per warp; with several
    // gates per CTA each gate's threads sync on a named barrier of their own (1 + g), so the
    // gates of a CTA run their passes independently and their FFT and exchange phases overlap
    constexpr bool CTA_SYNC = T > 32;
    static_assert(P0 == P0_SIMT || (LOG2N == 14 && ORDER == 1 && TXT == TX_PM1 && FULL),
                  "the tensor-core first pass exists for nfft 16384, radix order 1, full binary-phase codes");
    uint4* afrag = reinterpret_cast<uint4*>(smem + S::SMEM);   // tensor-core A fragments (mma.sync)
    unsigned char* ftile = smem + S::SMEM;                      // DFT operator tiles (tcgen05)
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    float2* twb = reinterpret_cast<float2*>(smem + S::OFF_TW);
    float2* tab = reinterpret_cast<float2*>(smem + S::OFF_TAB);

    const int tid = threadIdx.x;
    const int g = tid / T;
    const int t = tid - g * T;
    const int r = gx * G + g;
    const uint32_t mma_bar = smem_u32(&mbar[G]); // tcgen05 first pass: the MMAs of this IPP completed
    auto gsync = [&]() {
        if constexpr (!CTA_SYNC) __syncwarp();
        else if constexpr (G == 1) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(T) : "memory");
    };
    auto gsync_or = [&](bool pred) -> bool {
        if constexpr (!CTA_SYNC) {
            return __any_sync(0xffffffffu, pred);
        } else if constexpr (G == 1) {
            return __syncthreads_or(pred) != 0;
        } else {
            uint32_t any;
            asm volatile(
                "{\n\t.reg .pred p, q;\n\t"
                "setp.ne.u32 p, %1, 0;\n\t"
                "bar.red.or.pred q, %2, %3, p;\n\t"
                "selp.u32 %0, 1, 0, q;\n\t}"
                : "=r"(any)
                : "r"((uint32_t)pred), "r"(1 + g), "n"(T)
                : "memory");
            return any != 0;
        }
    };
    const bool valid = r < a.n_ranges;
    const int64_t s_r = (int64_t)a.range_start + (int64_t)(valid ? r : a.n_ranges - 1) * a.range_step;
    const int p_begin = c * a.chunk_len;
    const int p_end = min(p_begin + a.chunk_len, a.n_ipp);

    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + S::OFF_STAGE) + g * S::STAGE_WORDS;
    float2* xch = reinterpret_cast<float2*>(smem + S::OFF_XCH) + g * S::NPAD;
    const uint32_t bar = smem_u32(&mbar[g]);

    // window geometry: the copy starts at the 16-byte boundary at or below s_r
    const int off = (int)(s_r & 3);
    const uint32_t copy_bytes = (uint32_t)(((off + a.code_len + 3) & ~3) * 4);
    const bool dbg_ok = debug_window_ok(a, s_r, off, copy_bytes, S::STAGE_WORDS, t);
    auto issue = [&](int p) {
        const uint32_t* src = a.echo + (int64_t)p * a.echo_stride + (s_r - off);
        if constexpr (!p0_is_mmasync(P0)) {
            bulk_load(smem_u32(stage), src, copy_bytes, bar);
        } else {
            // 16 rows of 1024 samples (+4 words of alignment slack, inside the window's row),
            // each at a 1028-word pitch so the GEMM's column loads hit distinct banks
            const uint32_t last = off > 0 ? 4u * kTcSeg : 4u * 1024u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                         "r"(15u * 4u * kTcSeg + last) : "memory");
            for (int k = 0; k < 16; ++k)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_u32(stage + k * kTcSeg)),
                    "l"(src + 1024 * k), "r"(k < 15 ? 4u * kTcSeg : last), "r"(bar)
                    : "memory");
        }
    };

    // the previous unit of this CTA may still read the tables and the exchange buffer
    if (setup) __syncthreads();
    // per-thread twiddle bases of the recurrence passes, slot-major: [slot][t]
    for (int i = setup ? tid : S::NSLOT * T; i < S::NSLOT * T; i += kThreads) {
        int slot = i / T, tt = i - slot * T;
        int pass = slot < S::SLOTS1 ? 1 : 2;
        int b = pass == 1 ? slot : slot - S::SLOTS1;
        int ns = S::ns(pass), R = S::radix(pass);
        int j = tt + T * b;
        float sn, cs;   // the argument is an exact dyadic fraction; FP32 keeps setup off the FP64 pipe
        sincospif(-2.f * (float)(j % ns) / (float)(ns * R), &sn, &cs);
        twb[i] = make_float2(cs, sn);
    }
    if constexpr (p0_is_mmasync(P0)) {
        if (setup) tc_setup_afrags<P0>(afrag);
    } else if constexpr (p0_is_tc05(P0)) {
        if (setup) tc05_setup_f<P0>(ftile);
    }
    // this thread's TMEM twiddles: lane quarter of the warp, 128 columns per warp of the quarter
    const uint32_t tw_tm = TMT ? tmem_warp_lane_base(tmem) + 128u * (uint32_t)(tid >> 7) : 0u;
    if constexpr (TMT) {
        if (setup) {
            static_for<2>([&](auto Pc) {
                constexpr int pass = decltype(Pc)::value + 1;
                constexpr int R = S::radix(pass), NS = S::ns(pass), NB = E / R;
                static_for<4>([&](auto Cc) {
                    constexpr int cc = decltype(Cc)::value;
                    uint32_t rr[16];
                    static_for<8>([&](auto Ec) {
                        constexpr int i = decltype(Ec)::value, e = 8 * cc + i;
                        constexpr int b = e / (R - 1), k = e % (R - 1) + 1;
                        float sn = 0.f, cs = 0.f;
                        if constexpr (b < NB) {
                            const int jm = (t + T * b) % NS;   // exact dyadic argument
                            sincospif(-2.f * (float)((jm * k) % (NS * R)) / (float)(NS * R), &sn, &cs);
                        }
                        rr[2 * i] = __float_as_uint(cs);
                        rr[2 * i + 1] = __float_as_uint(sn);
                    });
                    tmem_st16(tw_tm + 64u * (pass - 1) + 16u * cc, rr);
                });
            });
            tmem_wait_st();
        }
    }
    // twiddle tables of the small passes, w^k = exp(-2 pi i jm k / (Ns R)): float4 [p][jm] =
    // (w^{2p+1}, w^{2p+2}) for radix <= 8; for radix 16 and 32 the three pairs (w, w^2),
    // (w^3, w^4), (w^8, w^16)
    for (int i = setup ? tid : S::TAB1 + S::TAB2; i < S::TAB1 + S::TAB2; i += kThreads) {
        int pass = i < S::TAB1 ? 1 : 2;
        int e = pass == 1 ? i : i - S::TAB1;
        int ns = S::ns(pass), R = S::radix(pass);
        int e4 = e >> 1, pr = e4 / ns, jm = e4 - pr * ns;
        int k = R >= 16 ? (pr < 2 ? 2 * pr + 1 + (e & 1) : 8 << (e & 1)) : 2 * pr + 1 + (e & 1);
        float sn = 0.f, cs = 0.f;
        if (k < R) sincospif(-2.f * (float)(jm * k) / (float)(ns * R), &sn, &cs);
        tab[i] = make_float2(cs, sn);
    }
    __syncthreads();

    if (t == 0 && dbg_ok && p_begin < p_end && p_begin != a.drop_ipp) issue(p_begin);

    const char* txbase = reinterpret_cast<const char*>(a.tx);
    constexpr int CHIP = TXT == TX_CI16 ? 4 : TXT == TX_C32 ? 8 : 1;
    uint32_t signs = 0;
    if constexpr (p0_is_mmasync(P0)) {
        if (a.tx_stride == 0) signs = tc_load_signs(reinterpret_cast<const int8_t*>(txbase));
    } else if constexpr (TXT == TX_PM1) {
        if (a.tx_stride == 0) signs = load_signs<LOG2N, ORDER>(reinterpret_cast<const int8_t*>(txbase), t, a.code_len);
    }

    float acc[E];
#pragma unroll
    for (int i = 0; i < E; ++i) acc[i] = 0.f;

    float2 v[E];
    bool timed_out = false;
    int it = 0;
#ifdef ISR_DEBUG
    long long ph[4] = {0, 0, 0, 0}, tq0 = 0, tq1 = 0, tq2 = 0;   // phase cycles (thread 0 reports)
#endif
    for (int p = p_begin; p < p_end; ++p, ++it) {
#ifdef ISR_DEBUG
        const long long tq = clock64();
        if (p > p_begin) ph[3] += tq - tq2;
#endif
        bool ok = mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        // every thread of the gate agrees before anyone leaves; this barrier also orders the
        // previous IPP's last-pass reads of xch before this IPP's first-pass writes
        {
            const bool any_fail = gsync_or(!ok);
            if (any_fail) {
                timed_out = true;
                break;
            }
        }
#ifdef ISR_DEBUG
        tq0 = clock64();
        ph[0] += tq0 - tq;
#endif
        const char* txrow = txbase + (size_t)p * (size_t)a.tx_stride * CHIP;
        if constexpr (p0_is_mmasync(P0)) {
            if (a.tx_stride != 0) signs = tc_load_signs(reinterpret_cast<const int8_t*>(txrow));
        } else if constexpr (TXT == TX_PM1) {
            if (a.tx_stride != 0) signs = load_signs<LOG2N, ORDER>(reinterpret_cast<const int8_t*>(txrow), t, a.code_len);
        }

        // ---- pass 0: decode from the staged window, radix-R0 DFT
        if constexpr (p0_is_mmasync(P0)) {
            tc_pass0<P0, S::PADP>(stage, off, signs, afrag, xch);
        } else if constexpr (p0_is_tc05(P0)) {
            // operand rows into the (free) exchange buffer, one thread issues the GEMM, every
            // warp stores its rows of the result in Stockham order
            tc05_build_operands<P0>(stage, off, signs, reinterpret_cast<unsigned char*>(xch));
            gsync();
            if (tid == 0) tc05_issue<P0>(smem_u32(xch), smem_u32(ftile), tmem, mma_bar);
            ok = mbar_wait(mma_bar, (uint32_t)it & 1u, a.wait_limit) && ok;
            tmem_fence_after_sync();
            tc05_store_outputs<S::PADP>(tmem, xch);
            tmem_fence_before_sync();
        } else static_for<E / R0>([&](auto Bc) {
            constexpr int b = decltype(Bc)::value;
            const int j = t + T * b;
            float2* u = v + b * R0;
            static_for<R0>([&](auto Kc) {
                constexpr int k = decltype(Kc)::value;
                const int pos = j + k * (N / R0);
                // chips at or past code_len are the zero padding (and are never read)
                u[k] = make_float2(0.f, 0.f);
                if (FULL || pos < a.code_len)
                    u[k] = decode<TXT, SPLITDEC ? (k & 1) == 0 : true>(stage[off + pos], txrow, pos,
                                                                       (signs << (31 - (b * R0 + k))) & 0x80000000u);
            });
            unit_dft<R0, LOG2N>(u);
            if constexpr (NP == 1) {
                static_for<R0>([&](auto Qc) {
                    constexpr int q = decltype(Qc)::value;
                    float2 X = u[BitRev<R0>::at(q)];
                    acc[b * R0 + q] = fmaf(X.x, X.x, fmaf(X.y, X.y, acc[b * R0 + q]));
                });
            } else {
                // Stockham output of the first pass (Ns = 1): y[j R0 + q]
                store_strided<1, R0, S::PADP>(xch, j * R0, u);
            }
        });

        // window fully consumed and first-pass outputs visible (tcgen05 first pass: also the
        // vote on its bounded wait for the GEMM)
        if constexpr (p0_is_tc05(P0)) {
            if (gsync_or(!ok)) {
                timed_out = true;
                break;
            }
        } else {
            gsync();
        }
        if (t == 0 && dbg_ok && p + 1 < p_end && p + 1 != a.drop_ipp) {
            fence_proxy_async();
            issue(p + 1);
        }
#ifdef ISR_DEBUG
        tq1 = clock64();
        ph[1] += tq1 - tq0;
        tq2 = tq1;
#endif
        if constexpr (NP == 1) continue;

        // ---- middle pass (three-pass sizes), in place: butterfly j reads x[j + (N/R) k] and
        // writes its output X_j[q] to the same slots, j + (N/R) q, so no other thread touches
        // them and no barrier separates the reads from the writes.  (Stockham element
        // D = (j / Ns) Ns R + j % Ns + q Ns is X_j[q]; the last pass finds it there.)
        if constexpr (S::INPLACE) {
            constexpr int R = S::R1, NS = R0;
            static_for<E / R>([&](auto Bc) {
                constexpr int b = decltype(Bc)::value;
                const int j = t + T * b;
                float2* u = v + b * R;
                load_strided<N / R, R, S::PADP>(u, xch, j);
                if constexpr (TMT) twiddle_tmem<R, b>(u, tw_tm);
                else if constexpr (S::tab(1) && R >= 16) twiddle_tab3<R, NS>(u, tab, j % NS);
                else if constexpr (S::tab(1)) twiddle_tab<R, NS>(u, tab, j % NS);
                else twiddle<R>(u, twb[b * T + t]);
                unit_dft<R, LOG2N>(u);
                store_strided<N / R, R, S::PADP>(xch, j, u);
            });
            gsync();
        } else if constexpr (NP == 3) {
            // read all, barrier, write all (Stockham order)
            constexpr int R = S::R1, NS = R0;
            static_for<E / R>([&](auto Bc) {
                constexpr int b = decltype(Bc)::value;
                const int j = t + T * b;
                float2* u = v + b * R;
                load_strided<N / R, R, S::PADP>(u, xch, j);
                if constexpr (S::tab(1) && R >= 16) twiddle_tab3<R, NS>(u, tab, j % NS);
                else if constexpr (S::tab(1)) twiddle_tab<R, NS>(u, tab, j % NS);
                else twiddle<R>(u, twb[b * T + t]);
                unit_dft<R, LOG2N>(u);
            });
            gsync();
            static_for<E / R>([&](auto Bc) {
                constexpr int b = decltype(Bc)::value;
                const int j = t + T * b;
                const int idxD = (j / NS) * NS * R + (j % NS);
                store_strided<NS, R, S::PADP>(xch, idxD, v + b * R);
            });
            gsync();
        }

#ifdef ISR_DEBUG
        tq2 = clock64();
        ph[2] += tq2 - tq1;
#endif
        // ---- last pass: read, twiddle, DFT, accumulate |X|^2 in registers
        {
            constexpr int R = RL;
            constexpr int PL = NP - 1;                        // index of the last pass
            constexpr int SLOT0 = PL == 2 ? S::SLOTS1 : 0;
            constexpr int TAB0 = PL == 2 ? S::TAB1 : 0;
            static_for<E / R>([&](auto Bc) {
                constexpr int b = decltype(Bc)::value;
                const int j = t + T * b;
                float2* u = v + b * R;
                if constexpr (S::INPLACE) {
                    // Stockham element D = j + (N/R) k sits at k Ns1 + j % Ns1 + (N/R1) (j / Ns1)
                    constexpr int NS1 = R0;
                    load_strided<NS1, R, S::PADP>(u, xch, (j % NS1) + (N / S::R1) * (j / NS1));
                } else {
                    load_strided<N / R, R, S::PADP>(u, xch, j);
                }
                if constexpr (TMT) twiddle_tmem<R, b>(u, tw_tm + 64u);
                else if constexpr (S::tab(PL) && R >= 16) twiddle_tab3<R, S::ns(PL)>(u, tab + TAB0, j % S::ns(PL));
                else if constexpr (S::tab(PL)) twiddle_tab<R, S::ns(PL)>(u, tab + TAB0, j % S::ns(PL));
                else twiddle<R>(u, twb[(SLOT0 + b) * T + t]);
                unit_dft<R, LOG2N>(u);
                static_for<R>([&](auto Qc) {
                    constexpr int q = decltype(Qc)::value;
                    float2 X = u[BitRev<R>::at(q)];
                    acc[b * R + q] = fmaf(X.x, X.x, fmaf(X.y, X.y, acc[b * R + q]));
                });
            });
        }
    }

#ifdef ISR_DEBUG
    if (!timed_out && a.phase_cycles && threadIdx.x == 0 && p_end > p_begin) {
        ph[3] += clock64() - tq2;
        for (int i = 0; i < 4; ++i) atomicAdd(a.phase_cycles + i, (unsigned long long)ph[i]);
        atomicAdd(a.phase_cycles + 4, (unsigned long long)(p_end - p_begin));
    }
#endif
    if (timed_out) {
        if (t == 0) atomicOr(a.status, 1);
        // let the copy still in flight land before the CTA's shared memory is released
        mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        return false;
    }

    // ---- chunk partials: bin of acc[b*RL + q] is j + q * N / RL, j = t + T b
    if (valid) {
        float* out = a.partial + ((int64_t)c * a.n_ranges + r) * N;
        static_for<E / RL>([&](auto Bc) {
            constexpr int b = decltype(Bc)::value;
            const int j = t + T * b;
            static_for<RL>([&](auto Qc) {
                constexpr int q = decltype(Qc)::value;
                out[j + q * (N / RL)] = acc[b * RL + q];
            });
        });
    }
    return true;
}

// ---------------------------------------------------------------- warp-local schedule
// Radix order 3 of nfft = M x 1024 (M = 2, 4, 8, 16): a decimation-in-frequency first pass,
//   Z_q[n] = W_N^{n q} sum_{k<M} x[n + 1024 k] W_M^{k q}      (n < 1024, q < M),
// spread over the gate's 32 M threads, then M independent 1024-point transforms,
//   X[q + M m] = sum_n Z_q[n] W_1024^{n m},
// one per warp, as a two-pass radix-32 Stockham FFT inside the warp.  Only the first pass
// needs the whole gate's data, so an IPP takes two CTA barriers instead of four and the
// warps run the rest independently.
template <int LOG2N>
struct SchedWL {
    static constexpr int N = 1 << LOG2N;
    static constexpr int M = N / 1024;          // first-pass radix = warps per gate
    static constexpr int T = N / 32;            // threads per gate
    static constexpr int G = kThreads / T;      // gates per CTA
    static constexpr int BF = 32 / M;           // first-pass butterflies per thread
    static constexpr int RPAD = 1024 + 64;      // one region (padded 2 per 32: 16-byte pairs)
    static constexpr int STAGE_WORDS = Sched<LOG2N>::STAGE_WORDS;
    static constexpr int OFF_MBAR = 0;
    static constexpr int OFF_TWB = 64;                        // [b][t] bases W_N^n (per CTA)
    static constexpr int OFF_TABC = OFF_TWB + 8 * 1024;       // float4 [3][l]: (w, w^2), (w^3, w^4), (w^8, w^16)
    static constexpr int OFF_STAGE = OFF_TABC + 8 * 32 * 32;
    static constexpr int OFF_REG = OFF_STAGE + 4 * STAGE_WORDS * G;
    static constexpr int SMEM = OFF_REG + 8 * RPAD * M * G;
    static_assert(LOG2N >= 11 && LOG2N <= 14, "warp-local schedule covers nfft 2048 .. 16384");
};

// two pad elements per 32 keep even elements 16-byte aligned for paired stores
__device__ __forceinline__ int pid32(int i) { return i + 2 * (i >> 5); }

// TMT: the first pass's twiddles W_N^{n q} and the last pass's W_1024^{l k} precomputed per thread
// in tensor memory at tmem, and a thread's two first-pass columns n = t and t + T (instead of two
// adjacent columns): the window reads become unit-stride (no bank conflicts) and the first-pass
// outputs go out as single complex stores.
template <int LOG2N, int TXT, bool FULL, class A = const KArgs, bool TMT = false>
__device__ __forceinline__ bool integrate_unit_wl(A a, const int gx, const int c, unsigned char* smem,
                                                  const uint32_t phase0, const bool setup, const uint32_t tmem = 0)
{
    using S = SchedWL<LOG2N>;
    constexpr int N = S::N, M = S::M, T = S::T, G = S::G, BF = S::BF;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    float2* twb = reinterpret_cast<float2*>(smem + S::OFF_TWB);
    float2* tabc = reinterpret_cast<float2*>(smem + S::OFF_TABC);

    const int tid = threadIdx.x;
    const int g = tid / T;
    const int t = tid - g * T;
    const int lane = t & 31, wg = t >> 5;
    const int r = gx * G + g;
    const bool valid = r < a.n_ranges;
    const int64_t s_r = (int64_t)a.range_start + (int64_t)(valid ? r : a.n_ranges - 1) * a.range_step;
    const int p_begin = c * a.chunk_len;
    const int p_end = min(p_begin + a.chunk_len, a.n_ipp);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + S::OFF_STAGE) + g * S::STAGE_WORDS;
    float2* reg = reinterpret_cast<float2*>(smem + S::OFF_REG) + g * M * S::RPAD;
    const uint32_t bar = smem_u32(&mbar[g]);
    const int off = (int)(s_r & 3);
    const uint32_t copy_bytes = (uint32_t)(((off + a.code_len + 3) & ~3) * 4);
    const bool dbg_ok = debug_window_ok(a, s_r, off, copy_bytes, S::STAGE_WORDS, t);
    auto issue = [&](int p) {
        const uint32_t* src = a.echo + (int64_t)p * a.echo_stride + (s_r - off);
        bulk_load(smem_u32(stage), src, copy_bytes, bar);
    };
    // first-pass column of butterfly b of thread tt
    auto col = [&](int tt, int b) { return TMT ? tt + T * b : 2 * (tt + T * (b >> 1)) + (b & 1); };
    static_assert(!TMT || (G == 1 && (M - 1) * BF <= 32), "TMEM twiddles: one gate per CTA, <= 32 first-pass twiddles");
    const uint32_t tw_tm = TMT ? tmem_warp_lane_base(tmem) + 128u * (uint32_t)(tid >> 7) : 0u;

    if (setup) __syncthreads();
    if constexpr (TMT) {
        if (setup) {
            // columns [0, 64): first pass, entry b (M - 1) + i - 1 = W_N^{n bitrev(i)} for the
            // register i that holds output bitrev(i); columns [64, 128): W_1024^{l k}, k = 1..31
            static_for<8>([&](auto Cc) {
                constexpr int cc = decltype(Cc)::value;
                uint32_t rr[16];
                static_for<8>([&](auto Ec) {
                    constexpr int i8 = decltype(Ec)::value, e = 8 * (cc & 3) + i8;
                    float sn = 0.f, cs = 0.f;
                    if constexpr (cc < 4) {
                        constexpr int b = e / (M - 1), i = e % (M - 1) + 1;
                        if constexpr (b < BF) {
                            const int n = col(t, b);
                            sincospif(-2.f * (float)((n * BitRev<M>::at(i)) % N) / (float)N, &sn, &cs);
                        }
                    } else if constexpr (e < 31) {
                        sincospif(-2.f * (float)((lane * (e + 1)) % 1024) / 1024.f, &sn, &cs);
                    }
                    rr[2 * i8] = __float_as_uint(cs);
                    rr[2 * i8 + 1] = __float_as_uint(sn);
                });
                tmem_st16(tw_tm + 16u * cc, rr);
            });
            tmem_wait_st();
        }
    }
    for (int i = (setup && !TMT) ? tid : 1024; i < 1024; i += kThreads) {   // bases W_N^n, slot [b][t]
        const int b = i / T, tt = i - b * T;
        const int n = col(tt, b);
        float sn, cs;
        sincospif(-2.f * (float)n / (float)N, &sn, &cs);
        twb[i] = make_float2(cs, sn);
    }
    // three pairs per lane (w, w^2), (w^3, w^4), (w^8, w^16), w = W_1024^l (see twiddle_tab3)
    for (int i = (setup && !TMT) ? tid : 6 * 32; i < 6 * 32; i += kThreads) {
        const int e4 = i >> 1, pr = e4 / 32, l = e4 % 32;
        const int k = pr < 2 ? 2 * pr + 1 + (i & 1) : 8 << (i & 1);
        float sn, cs;
        sincospif(-2.f * (float)(l * k) / 1024.f, &sn, &cs);
        tabc[i] = make_float2(cs, sn);
    }
    __syncthreads();
    if (t == 0 && dbg_ok && p_begin < p_end && p_begin != a.drop_ipp) issue(p_begin);

    const char* txbase = reinterpret_cast<const char*>(a.tx);
    constexpr int CHIP = TXT == TX_CI16 ? 4 : TXT == TX_C32 ? 8 : 1;
    // first-pass chips of this thread: bit b M + k for position col(t, b) + 1024 k
    auto signs_of = [&](const int8_t* row) {
        uint32_t m = 0;
        static_for<BF>([&](auto Bc) {
            constexpr int b = decltype(Bc)::value;
            static_for<M>([&](auto Kc) {
                constexpr int k = decltype(Kc)::value;
                const int pos = col(t, b) + 1024 * k;
                if (pos < a.code_len && row[pos] < 0) m |= 1u << (b * M + k);
            });
        });
        return m;
    };
    uint32_t signs = 0;
    if constexpr (TXT == TX_PM1) {
        if (a.tx_stride == 0) signs = signs_of(reinterpret_cast<const int8_t*>(txbase));
    }

    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    float2 v[32];
    bool timed_out = false;
    int it = 0;
    for (int p = p_begin; p < p_end; ++p, ++it) {
        const bool ok = mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        // also orders the previous IPP's last reads of the regions before this IPP's writes
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const char* txrow = txbase + (size_t)p * (size_t)a.tx_stride * CHIP;
        if constexpr (TXT == TX_PM1) {
            if (a.tx_stride != 0) signs = signs_of(reinterpret_cast<const int8_t*>(txrow));
        }
        // ---- pass A: decode, radix-M DFT over stride 1024, DIF twiddles, scatter to regions;
        // butterflies b and b + 1 of a thread are the adjacent columns n, n + 1
        float2 zp[M] = {};   // even butterflies fill it before the odd ones read it
        static_for<BF>([&](auto Bc) {
            constexpr int b = decltype(Bc)::value;
            const int n = col(t, b);
            float2 u[M];
            static_for<M>([&](auto Kc) {
                constexpr int k = decltype(Kc)::value;
                const int pos = n + 1024 * k;
                u[k] = make_float2(0.f, 0.f);
                if (FULL || pos < a.code_len)
                    u[k] = decode<TXT, (k & 1) == 0>(stage[off + pos], txrow, pos, (signs << (31 - (b * M + k))) & 0x80000000u);
            });
            sdft<M>(u);
            if constexpr (TMT) {
                twiddle_tmem<M, b>(u, tw_tm);   // u[i] *= W_N^{n bitrev(i)}
                static_for<M>([&](auto Qc) {
                    constexpr int q = decltype(Qc)::value;
                    reg[q * S::RPAD + pid32(n)] = u[BitRev<M>::at(q)];
                });
                return;
            }
            const float2 w = twb[b * T + t];
            float2 cur = w;
            static_for<M>([&](auto Qc) {
                constexpr int q = decltype(Qc)::value;
                float2 z = u[BitRev<M>::at(q)];
                if constexpr (q > 0) {
                    z = cmul(z, cur);
                    if constexpr (q + 1 < M) cur = cmul(cur, w);
                }
                if constexpr (b & 1) {
                    *reinterpret_cast<float4*>(&reg[q * S::RPAD + pid32(n - 1)]) =
                        make_float4(zp[q].x, zp[q].y, z.x, z.y);
                } else {
                    zp[q] = z;
                }
            });
        });
        __syncthreads();   // regions complete; the window is consumed
        if (t == 0 && dbg_ok && p + 1 < p_end && p + 1 != a.drop_ipp) {
            fence_proxy_async();
            issue(p + 1);
        }
        // ---- pass B (warp wg, region wg): radix-32 over stride 32, Stockham Ns = 1, in place
        float2* rw = reg + wg * S::RPAD;
        static_for<32>([&](auto Kc) {                       // rw[pid32(l + 32 k)] = rw[l + 34 k]
            constexpr int k = decltype(Kc)::value;
            v[k] = rw[lane + 34 * k];
        });
        sdft<32>(v);
        __syncwarp();
        static_for<16>([&](auto Qc) {                       // y[32 l + q], q pairs: rw[34 l + q]
            constexpr int q = 2 * decltype(Qc)::value;
            const float2 x0 = v[BitRev<32>::at(q)], x1 = v[BitRev<32>::at(q + 1)];
            *reinterpret_cast<float4*>(&rw[34 * lane + q]) = make_float4(x0.x, x0.y, x1.x, x1.y);
        });
        __syncwarp();
        // ---- pass C: twiddle W_1024^{l k}, radix-32, accumulate |X|^2 (bin wg + M (l + 32 q))
        static_for<32>([&](auto Kc) {
            constexpr int k = decltype(Kc)::value;
            v[k] = rw[lane + 34 * k];
        });
        if constexpr (TMT) twiddle_tmem<32, 0>(v, tw_tm + 64u);
        else twiddle_tab3<32, 32>(v, tabc, lane);
        sdft<32>(v);
        static_for<32>([&](auto Qc) {
            constexpr int q = decltype(Qc)::value;
            const float2 X = v[BitRev<32>::at(q)];
            acc[q] = fmaf(X.x, X.x, fmaf(X.y, X.y, acc[q]));
        });
    }

    if (timed_out) {
        if (tid == 0) atomicOr(a.status, 1);
        mbar_wait(bar, (phase0 + (uint32_t)it) & 1u, a.wait_limit);
        return false;
    }
    if (valid) {
        float* out = a.partial + ((int64_t)c * a.n_ranges + r) * N;
#pragma unroll
        for (int q = 0; q < 32; ++q) out[wg + M * (lane + 32 * q)] = acc[q];
    }
    return true;
}

// The warp-local schedule with its twiddles in tensor memory (512 columns, one CTA per SM).
template <int LOG2N, int TXT, bool FULL>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_wl_tm(KArgs a)
{
    using S = SchedWL<LOG2N>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_MBAR + 8 * 7);
    if (threadIdx.x < S::G) mbar_init(smem_u32(&mbar[threadIdx.x]), 1);
    if (threadIdx.x < 32) tmem_alloc(smem_u32(tslot), 512);
    fence_barrier_init();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    integrate_unit_wl<LOG2N, TXT, FULL, const KArgs, true>(a, blockIdx.x, blockIdx.y, smem, 0u, true, tbase);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (threadIdx.x < 32) tmem_dealloc(tbase, 512);
}

template <int LOG2N, int TXT, bool FULL>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_wl(KArgs a)
{
    using S = SchedWL<LOG2N>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    if (threadIdx.x < S::G) mbar_init(smem_u32(&mbar[threadIdx.x]), 1);
    fence_barrier_init();
    integrate_unit_wl<LOG2N, TXT, FULL>(a, blockIdx.x, blockIdx.y, smem, 0u, true);
}

// One-shot launch with the inter-pass twiddles in tensor memory: warp 0 allocates all 512
// columns (one CTA per SM: the shared memory admits no second one), every thread writes its
// twiddles once, and warp 0 frees the columns after the unit, timed out or not.
template <int LOG2N, int TXT, bool FULL, int ORDER>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_tm(KArgs a)
{
    using S = Sched<LOG2N, ORDER, true>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_TMEMADDR);
    if (threadIdx.x < S::G) mbar_init(smem_u32(&mbar[threadIdx.x]), 1);
    if (threadIdx.x < 32) tmem_alloc(smem_u32(tslot), S::TM_COLS);
    fence_barrier_init();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    integrate_unit<LOG2N, TXT, ORDER, FULL, P0_SIMT, const KArgs, true>(a, blockIdx.x, blockIdx.y, smem, 0u, true,
                                                                         tbase);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (threadIdx.x < 32) tmem_dealloc(tbase, S::TM_COLS);
}

// One-shot launch with the first pass on tcgen05 (MODE one of P0_TC05_*): warp 0 allocates
// the accumulator columns of the GEMM, mbarrier slot 1 tracks the GEMM of each IPP.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel_tc05(KArgs a)
{
    using S = Sched<14, 1>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::OFF_MBAR + 8 * 7);   // slot 7 holds the address
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);   // staged window
        mbar_init(smem_u32(&mbar[1]), 1);   // GEMM committed
    }
    if (threadIdx.x < 32) tmem_alloc(smem_u32(tslot), kTc05Cols);
    fence_barrier_init();
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;
    integrate_unit<14, TX_PM1, 1, true, MODE>(a, blockIdx.x, blockIdx.y, smem, 0u, true, tbase);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (threadIdx.x < 32) tmem_dealloc(tbase, kTc05Cols);
}

// One-shot launch: grid = (gate groups, IPP chunks), one unit per CTA.
template <int LOG2N, int TXT, bool FULL = false, int ORDER = 0, int P0 = P0_SIMT>
__global__ void __launch_bounds__(kThreads, 1) integrate_kernel(KArgs a)
{
    using S = Sched<LOG2N, ORDER>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::OFF_MBAR);
    if (threadIdx.x < S::G) mbar_init(smem_u32(&mbar[threadIdx.x]), 1);
    fence_barrier_init();
    integrate_unit<LOG2N, TXT, ORDER, FULL, P0>(a, blockIdx.x, blockIdx.y, smem, 0u, true);
}

}  // namespace isr
