// isr_tc05.cuh -- the first FFT pass of nfft = 16384 as tcgen05 tensor-core GEMMs.
//
// Radix order [16, 32, 32]: for every column j < 1024 of the window the first pass is the
// 16-point DFT  V_j[q] = sum_{k<16} W16^{qk} x[j + 1024 k].  In real arithmetic, with the row
// X_j = [Re x(j + 1024 k), k < 16 | Im x(j + 1024 k), k < 16] (K = 32), it is
//     D[j][n] = sum_k X_j[k] F[n][k],   F = [[Fr, -Fi]; [Fi, Fr]]  (N = 32: Re V_j | Im V_j)
// i.e. D = X F^T with M = 1024 positions (eight M = 128 tiles), N = 32, K = 32.
//
// Per IPP: every thread decodes its two columns from the staged window, splits each decoded
// sample (an integer of at most 16 bits) exactly into hi + lo in BF16 or FP16, and writes the
// rows into K-major operand tiles in shared memory (the exchange buffer, free at that point);
// one thread issues the MMAs (accumulator in tensor memory, FP32) and commits them to an
// mbarrier; each warp then reads its rows of D with tcgen05.ld -- row j holds the 16 outputs of
// butterfly j -- and stores them in Stockham order for the SIMT passes that follow.
// Split modes add X_hi F_hi + X_lo F_hi + X_hi F_lo (the dropped X_lo F_lo is below FP32
// rounding); single modes X_hi F_hi only.
//
// Operand layout (no swizzle, K-major): 8-row x 16-byte core matrices; within a tile the core
// matrix of rows 8 i.. and elements 8 c.. sits at i * 512 + c * 128 bytes (LBO = 128 B between
// K-neighbours, SBO = 512 B between 8-row groups).  One M = 128 tile of X is 8 KB; F is 2 KB.
#pragma once

#include <cstdint>

#include "isr_tc.cuh"
#include "isr_tmem.cuh"

namespace isr {

// tensor-core first-pass engines: the warp-level mma.sync modes (isr_tc.cuh) and these
enum P0Tc05Mode { P0_TC05_BF16_SPLIT = 5, P0_TC05_FP16_SPLIT = 6, P0_TC05_BF16 = 7, P0_TC05_FP16 = 8 };

__host__ __device__ constexpr bool p0_is_tc05(int mode) { return mode >= P0_TC05_BF16_SPLIT && mode <= P0_TC05_FP16; }
__host__ __device__ constexpr bool p0_is_mmasync(int mode) { return mode >= P0_BF16_SPLIT && mode <= P0_FP16; }

template <int MODE> struct Tc05Fmt {
    static constexpr bool bf16 = MODE == P0_TC05_BF16_SPLIT || MODE == P0_TC05_BF16;
    static constexpr bool split = MODE == P0_TC05_BF16_SPLIT || MODE == P0_TC05_FP16_SPLIT;
};

constexpr int kTc05TileBytes = 8192;          // one M = 128 tile of X (K = 32, 16-bit)
constexpr int kTc05XBytes = 8 * kTc05TileBytes;  // one operand part (hi or lo) of all 1024 rows
constexpr int kTc05FBytes = 2048;             // F (N = 32, K = 32, 16-bit)
constexpr int kTc05Cols = 256;                // TMEM columns of D: eight tiles of N = 32

// shared-memory matrix descriptor, K-major, no swizzle (sm_100 format: version 1 at bit 46)
__device__ __forceinline__ uint64_t tc05_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16 (1) or FP16 (0), both K-major,
// N = 32 (bits 17-22: N / 8), M = 128 (bits 24-28: M / 16)
template <bool BF>
__host__ __device__ constexpr uint32_t tc05_idesc()
{
    return (1u << 4) | ((BF ? 1u : 0u) << 7) | ((BF ? 1u : 0u) << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc05_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive once on the mbarrier when every MMA this thread issued before has completed
__device__ __forceinline__ void tc05_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld32(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// byte offset of row r, K-element c (multiple of 8) in a K-major no-swizzle tile of K = 32
__device__ __forceinline__ uint32_t tc05_row_chunk(int r, int c)
{
    return (uint32_t)((r >> 3) * 512 + (c >> 3) * 128 + (r & 7) * 16);
}

// F_hi and F_lo, [n][k] K-major (n < 32 output rows, k < 32 inputs), at f (4 KB); one warp.
// Ends with the proxy fence that makes the tiles visible to the tensor cores.
template <int MODE>
__device__ __forceinline__ void tc05_setup_f(unsigned char* f)
{
    constexpr bool BF = Tc05Fmt<MODE>::bf16;
    if (threadIdx.x >= 32) return;
    const int n = threadIdx.x;
#pragma unroll 1
    for (int c = 0; c < 32; c += 8) {
        uint32_t hi[4], lo[4];
        for (int e = 0; e < 4; ++e) split2<BF>(tc_a_elem(n, c + 2 * e), tc_a_elem(n, c + 2 * e + 1), hi[e], lo[e]);
        *reinterpret_cast<uint4*>(f + tc05_row_chunk(n, c)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(f + kTc05FBytes + tc05_row_chunk(n, c)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Operand rows of this thread's two columns j = t + 512 b (b < 2) into xs (hi part at xs, lo
// at xs + kTc05XBytes), decoded from the staged window with the chip signs in `signs` (bit
// 16 b + k for position j + 1024 k).  Ends with the proxy fence for the tensor cores.
template <int MODE>
__device__ __forceinline__ void tc05_build_operands(const uint32_t* stage, int off, uint32_t signs, unsigned char* xs)
{
    constexpr bool BF = Tc05Fmt<MODE>::bf16;
    constexpr bool SPLIT = Tc05Fmt<MODE>::split;
    const int t = threadIdx.x;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int j = t + 512 * b;
        unsigned char* row_hi = xs + (j >> 7) * kTc05TileBytes;
        unsigned char* row_lo = row_hi + kTc05XBytes;
        float re[16], im[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t w = stage[off + j + 1024 * k];
            const uint32_t sb = (signs << (31 - (16 * b + k))) & 0x80000000u;
            re[k] = __int_as_float(__float_as_int((float)(int16_t)(w & 0xffffu)) ^ sb);
            im[k] = __int_as_float(__float_as_int((float)(int16_t)(w >> 16)) ^ sb);
        }
#pragma unroll
        for (int c = 0; c < 32; c += 8) {
            const float* src = c < 16 ? re + c : im + (c - 16);
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if constexpr (SPLIT) split2<BF>(src[2 * e], src[2 * e + 1], hi[e], lo[e]);
                else hi[e] = pack2<BF>(src[2 * e], src[2 * e + 1]);
            }
            const uint32_t o = tc05_row_chunk(j & 127, c);
            *reinterpret_cast<uint4*>(row_hi + o) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            if constexpr (SPLIT) *reinterpret_cast<uint4*>(row_lo + o) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Issued by one thread: D tile m (TMEM columns 32 m) = X tile m times F^T, then commit to mbar.
template <int MODE>
__device__ __forceinline__ void tc05_issue(uint32_t xs, uint32_t fs, uint32_t d_tmem, uint32_t mbar)
{
    constexpr bool BF = Tc05Fmt<MODE>::bf16;
    constexpr bool SPLIT = Tc05Fmt<MODE>::split;
    constexpr uint32_t idesc = tc05_idesc<BF>();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
    for (int m = 0; m < 8; ++m) {
        const uint32_t d = d_tmem + 32u * m;
        uint32_t acc = 0;
        // products (X part, F part): hi hi, then lo hi and hi lo for the split modes
#pragma unroll
        for (int pr = 0; pr < (SPLIT ? 3 : 1); ++pr) {
            const uint32_t xa = xs + (pr == 1 ? kTc05XBytes : 0) + m * kTc05TileBytes;
            const uint32_t fa = fs + (pr == 2 ? kTc05FBytes : 0);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {   // K = 16 per instruction: two core matrices of 128 B
                tc05_mma(d, tc05_desc(xa + 256u * ks, 128u, 512u), tc05_desc(fa + 256u * ks, 128u, 512u), idesc, acc);
                acc = 1;
            }
        }
    }
    tc05_commit(mbar);
}

// After the MMAs completed: this warp's rows of D (tiles w / 4 and w / 4 + 4 of its lane
// quarter) in Stockham order y[16 j + q] = V_j[q] (Ns = 1) in the padded exchange buffer.
template <int PADP>
__device__ __forceinline__ void tc05_store_outputs(uint32_t d_tmem, float2* xch)
{
    static_assert(PADP == 16, "one pad element per 16: outputs q < 16 of column j at 17 j + q");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tq = tmem_warp_lane_base(d_tmem);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = (warp >> 2) + 4 * h;
        uint32_t r[32];
        tmem_ld32(tq + 32u * m, r);
        tmem_wait_ld32(r);
        const int j = 128 * m + 32 * (warp & 3) + lane;
        float2* b = xch + 17 * j;
#pragma unroll
        for (int q = 0; q < 16; ++q) b[q] = make_float2(__uint_as_float(r[q]), __uint_as_float(r[16 + q]));
    }
}

}  // namespace isr
