// isr_tc.cuh -- the first FFT pass of nfft = 16384 as split-precision tensor-core GEMMs.
//
// Radix order [16, 32, 32]: the first pass is, for every column j < 1024 of the window,
//   V_j[q] = sum_{k<16} W16^{qk} x[j + 1024 k]          (a 16-point DFT, W16 = e^{-2 pi i/16})
// i.e. one complex GEMM  Y[16 x 1024] = F16[16 x 16] X[16 x 1024]  per window and IPP, done in
// real arithmetic as  [Yr; Yi] = [[Fr, -Fi]; [Fi, Fr]] [Xr; Xi]  (M = 32, K = 32, N = 1024).
// Operands are BF16 or FP16 with FP32 accumulation (mma.sync m16n8k16).  Every decoded
// sample is an integer of at most 16 bits, so it splits exactly into hi + lo in either
// format; the DFT matrix splits into hi + lo with a residual of 2^-17 (BF16) or 2^-22
// (FP16).  SPLIT modes accumulate A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo
// is below FP32 rounding); single modes use A_hi B_hi only, to show what the split buys.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace isr {

enum P0Mode { P0_SIMT = 0, P0_BF16_SPLIT = 1, P0_FP16_SPLIT = 2, P0_BF16 = 3, P0_FP16 = 4 };

constexpr int kTcSeg = 1028;          // staged window: 16 rows of 1024 samples + 4 slack words
constexpr int kTcAfragBytes = 8 * 32 * 16;

template <int MODE> struct TcFmt {
    static constexpr bool bf16 = MODE == P0_BF16_SPLIT || MODE == P0_BF16;
    static constexpr bool split = MODE == P0_BF16_SPLIT || MODE == P0_FP16_SPLIT;
};

// pack two floats (first in the low half) into the 16-bit format, round to nearest
template <bool BF>
__device__ __forceinline__ uint32_t pack2(float lo_elem, float hi_elem)
{
    if constexpr (BF) {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
        return *reinterpret_cast<uint32_t*>(&v);
    } else {
        __half2 v = __floats2half2_rn(lo_elem, hi_elem);
        return *reinterpret_cast<uint32_t*>(&v);
    }
}

template <bool BF>
__device__ __forceinline__ float2 unpack2(uint32_t p)
{
    if constexpr (BF) {
        __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162*>(&p);
        return __bfloat1622float2(v);
    } else {
        __half2 v = *reinterpret_cast<__half2*>(&p);
        return __half22float2(v);
    }
}

// hi = round(x, y); lo = round of the residual (exact for integers of <= 16 bits)
template <bool BF>
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo)
{
    hi = pack2<BF>(x, y);
    const float2 h = unpack2<BF>(hi);
    lo = pack2<BF>(x - h.x, y - h.y);
}

template <bool BF>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint4& a, uint32_t b0, uint32_t b1)
{
    if constexpr (BF) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
    }
}

// Element (r, c) of the real 32 x 32 operator [[Fr, -Fi]; [Fi, Fr]], F = the 16-point DFT.
__device__ __forceinline__ float tc_a_elem(int r, int c)
{
    const int q = r & 15, k = c & 15;
    double s, co;
    sincospi(2.0 * (double)((q * k) & 15) / 16.0, &s, &co);   // W16^{qk} = cos - i sin
    const double fr = co, fi = -s;
    if (r < 16) return (float)(c < 16 ? fr : -fi);
    return (float)(c < 16 ? fi : fr);
}

// Per-lane A fragments in shared memory, [frag][lane] uint4, frag = ((mt * 2 + ks) * 2 + part):
// rows 16 mt + {g, g + 8}, columns 16 ks + {2t, 2t + 1, 2t + 8, 2t + 9} (g = lane / 4, t = lane % 4).
template <int MODE>
__device__ __forceinline__ void tc_setup_afrags(uint4* af)
{
    constexpr bool BF = TcFmt<MODE>::bf16;
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x, g = lane >> 2, t = lane & 3;
    for (int mt = 0; mt < 2; ++mt)
        for (int ks = 0; ks < 2; ++ks) {
            uint32_t hi[4], lo[4];
            const int r0 = 16 * mt + g, c0 = 16 * ks + 2 * t;
            const int rr[4] = {r0, r0 + 8, r0, r0 + 8};
            const int cc[4] = {c0, c0, c0 + 8, c0 + 8};
            for (int i = 0; i < 4; ++i) split2<BF>(tc_a_elem(rr[i], cc[i]), tc_a_elem(rr[i], cc[i] + 1), hi[i], lo[i]);
            af[((mt * 2 + ks) * 2 + 0) * 32 + lane] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            af[((mt * 2 + ks) * 2 + 1) * 32 + lane] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
}

// sign bits of the code chips a thread decodes in the tensor-core first pass:
// bit nt * 4 + kk for column j = 64 warp + 8 nt + g and row k = {2t, 2t+1, 2t+8, 2t+9}[kk]
__device__ __forceinline__ uint32_t tc_load_signs(const int8_t* row)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    uint32_t m = 0;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int k = 2 * t + (kk & 1) + 8 * (kk >> 1);
            const int pos = 64 * warp + 8 * nt + g + 1024 * k;
            if (row[pos] < 0) m |= 1u << (nt * 4 + kk);
        }
    return m;
}

// The first pass for one window (one gate per CTA): decode from the padded stage
// (row k at k * kTcSeg + off), GEMM on the tensor cores, Stockham output y[16 j + q].
template <int MODE, int PADP>
__device__ __forceinline__ void tc_pass0(const uint32_t* stage, int off, uint32_t signs, const uint4* af,
                                         float2* xch)
{
    constexpr bool BF = TcFmt<MODE>::bf16;
    constexpr bool SPLIT = TcFmt<MODE>::split;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    uint4 A[2][2][2];
#pragma unroll
    for (int f = 0; f < 8; ++f) A[f >> 2][(f >> 1) & 1][f & 1] = af[f * 32 + lane];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int j = 64 * warp + 8 * nt + g;
        // decoded samples x[j + 1024 k] for k = 2t, 2t+1, 2t+8, 2t+9
        float re[4], im[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int k = 2 * t + (kk & 1) + 8 * (kk >> 1);
            const uint32_t w = stage[k * kTcSeg + off + j];
            const uint32_t sb = (signs << (31 - (nt * 4 + kk))) & 0x80000000u;
            re[kk] = __int_as_float(__float_as_int((float)(int16_t)(w & 0xffffu)) ^ sb);
            im[kk] = __int_as_float(__float_as_int((float)(int16_t)(w >> 16)) ^ sb);
        }
        // B fragments (rows k, column j): ks 0 = real parts, ks 1 = imaginary parts
        uint32_t bh[2][2], bl[2][2];
        split2<BF>(re[0], re[1], bh[0][0], bl[0][0]);
        split2<BF>(re[2], re[3], bh[0][1], bl[0][1]);
        split2<BF>(im[0], im[1], bh[1][0], bl[1][0]);
        split2<BF>(im[2], im[3], bh[1][1], bl[1][1]);
        float D[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int i = 0; i < 4; ++i) D[mt][i] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                mma16816<BF>(D[mt], A[mt][ks][0], bh[ks][0], bh[ks][1]);
                if constexpr (SPLIT) {
                    mma16816<BF>(D[mt], A[mt][ks][0], bl[ks][0], bl[ks][1]);
                    mma16816<BF>(D[mt], A[mt][ks][1], bh[ks][0], bh[ks][1]);
                }
            }
        }
        // D[0] = Re V, D[1] = Im V at rows q = g, g + 8 and columns j0 + 2t, j0 + 2t + 1
        const int jc = 64 * warp + 8 * nt + 2 * t;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = g + 8 * (i >> 1);
            const int jj = jc + (i & 1);
            const int e = 16 * jj + q;
            xch[e + e / PADP] = make_float2(D[0][i], D[1][i]);
        }
    }
}

}  // namespace isr
