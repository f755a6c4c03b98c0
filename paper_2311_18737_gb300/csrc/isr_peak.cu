// isr_peak.cu -- measured FP32 fused multiply-add throughput of the device.
//
// The integrate kernel is bound by the FP32 SIMT pipe, so its roofline denominator is the FP32
// peak: SMs x 128 FMA lanes x 2 FLOP x SM clock.  This microkernel measures that rate: every
// thread runs independent FMA dependency chains (enough of them to cover the pipe latency) and
// nothing else, 4 CTAs of 256 threads per SM.  The paired variant issues FFMA2 (two FP32 FMAs per
// lane and instruction) to show whether pairing raises the lane throughput or only saves issue
// slots.
//
// isr_tc05_rate measures the tensor pipe the same way for one tcgen05.mma shape (kind::f16, BF16
// operands from shared memory, FP32 accumulator in TMEM, M = 128, K = 16, N given): one thread
// per CTA issues the MMAs back to back, one CTA per SM.  The estimator's convolutions use
// N = 32 and N = 64 shapes, whose rate is well below the N = 256 peak.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "isr.h"
#include "isr_kernels.cuh"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;     // independent chains per thread
constexpr int kInner = 128;    // FMAs per chain per outer iteration (unrolled)

__global__ void __launch_bounds__(kPeakThreads) fma_chain_kernel(float* sink, int outer, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
    for (int o = 0; o < outer; ++o) {
#pragma unroll
        for (int k = 0; k < kInner; ++k)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.f) sink[0] = s;   // never true for b, c > 0 and a >= 0: keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) fma2_chain_kernel(float* sink, int outer, float b, float c)
{
    float2 a[kChains];
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = make_float2((float)(threadIdx.x + i) * 1e-3f, (float)i * 2e-3f);
    for (int o = 0; o < outer; ++o) {
#pragma unroll
        for (int k = 0; k < kInner; ++k)
#pragma unroll
            for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
    if (s == -1.f) sink[0] = s;
}

constexpr int kRateThreads = 128;
constexpr int kRateIters = 4096;   // MMAs per CTA

// Operands: A (128 x 16 BF16, K-major) 4 KB and B (N x 16, K-major) N * 32 bytes of zeros, no
// swizzle (LBO 128 B along K, SBO 256 B between 8-row groups); D = TMEM columns [0, N) of 256.
// cycles[blockIdx.x] = clock64 cycles from the first issue to the commit's completion; a wait that
// runs out of polls increments *fail.
template <int N>
__global__ void __launch_bounds__(kRateThreads, 1) tc05_rate_kernel(unsigned long long* cycles, int* fail)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr int BYTES = 4096 + N * 32;
    for (int i = tid; i < BYTES / 16; i += kRateThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) isr::mbar_init(isr::smem_u32(&bar), 1);
    if (warp == 0) isr::tmem_alloc(isr::smem_u32(&tslot), 256);
    isr::fence_proxy_async();
    isr::fence_barrier_init();
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    const uint32_t tbase = tslot;
    if (tid == 0) {
        const uint64_t ad = isr::tc05_desc(isr::smem_u32(sm), 128, 256);
        const uint64_t bd = isr::tc05_desc(isr::smem_u32(sm + 4096), 128, 256);
        const uint32_t idesc = (isr::tc05_idesc<true>() & ~(0x3Fu << 17)) | ((uint32_t)(N >> 3) << 17);
        const unsigned long long t0 = clock64();
        for (int i = 0; i < kRateIters; ++i) isr::tc05_mma(tbase, ad, bd, idesc, i > 0 ? 1u : 0u);
        isr::tc05_commit(isr::smem_u32(&bar));
        const bool ok = isr::mbar_wait(isr::smem_u32(&bar), 0, 1u << 26);
        cycles[blockIdx.x] = clock64() - t0;
        if (!ok) atomicAdd(fail, 1);
    }
    isr::tmem_fence_before_sync();
    __syncthreads();
    isr::tmem_fence_after_sync();
    if (warp == 0) isr::tmem_dealloc(tbase, 256);
}

template <int N>
cudaError_t tc05_rate_launch(int sms, cudaStream_t st, unsigned long long* cycles, int* fail)
{
    const int smem = 4096 + N * 32;
    tc05_rate_kernel<N><<<sms, kRateThreads, smem, st>>>(cycles, fail);
    return cudaGetLastError();
}

}  // namespace

extern "C" isr_status isr_tc05_rate(int32_t device, int32_t n, double* tflops, double* cycles_per_mma)
{
    isr::clear_error();
    if (!tflops || !cycles_per_mma) return isr::fail(ISR_ERR_INVALID_ARG, "isr_tc05_rate: NULL output");
    if (n != 32 && n != 64 && n != 128 && n != 256)
        return isr::fail(ISR_ERR_INVALID_ARG, "isr_tc05_rate: n must be 32, 64, 128 or 256");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return isr::fail(ISR_ERR_CUDA, "isr_tc05_rate: cudaSetDevice: %s", cudaGetErrorString(e));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    unsigned long long* cycles = nullptr;
    int* fail = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&cycles, sizeof(unsigned long long) * sms);
    if (e == cudaSuccess) e = cudaMalloc(&fail, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(fail, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = -1.f;
    for (int run = 0; run < 3 && e == cudaSuccess; ++run) {   // run 0 warms up
        cudaEventRecord(e0, st);
        e = n == 32 ? tc05_rate_launch<32>(sms, st, cycles, fail)
            : n == 64 ? tc05_rate_launch<64>(sms, st, cycles, fail)
            : n == 128 ? tc05_rate_launch<128>(sms, st, cycles, fail)
                       : tc05_rate_launch<256>(sms, st, cycles, fail);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && run > 0 && (best < 0.f || t < best)) best = t;
    }
    std::vector<unsigned long long> h(sms > 0 ? sms : 1);
    int failed = 0;
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), cycles, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&failed, fail, sizeof(int), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (cycles) cudaFree(cycles);
    if (fail) cudaFree(fail);
    if (e != cudaSuccess) return isr::fail(ISR_ERR_CUDA, "isr_tc05_rate: %s", cudaGetErrorString(e));
    if (failed) return isr::fail(ISR_ERR_TIMEOUT, "isr_tc05_rate: %d CTAs timed out waiting for their MMAs", failed);
    double mean = 0.0;
    for (int i = 0; i < sms; ++i) mean += (double)h[i] / sms;
    *cycles_per_mma = mean / kRateIters;
    *tflops = 2.0 * 128.0 * n * 16.0 * kRateIters * sms / (best * 1e-3) / 1e12;
    return ISR_OK;
}

extern "C" isr_status isr_fp32_peak(int32_t device, int32_t paired, double* tflops, double* ms)
{
    isr::clear_error();
    if (!tflops || !ms) return isr::fail(ISR_ERR_INVALID_ARG, "isr_fp32_peak: NULL output");
    if (paired != 0 && paired != 1) return isr::fail(ISR_ERR_INVALID_ARG, "isr_fp32_peak: paired must be 0 or 1");
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return isr::fail(ISR_ERR_CUDA, "isr_fp32_peak: cudaSetDevice: %s", cudaGetErrorString(e));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    float* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMalloc(&sink, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int blocks = 4 * sms;
    const int outer = 8000;   // ~20 ms per run (scalar) at the nominal rate
    float best = -1.f;
    for (int run = 0; run < 4 && e == cudaSuccess; ++run) {   // run 0 warms up
        cudaEventRecord(e0, st);
        if (paired)
            fma2_chain_kernel<<<blocks, kPeakThreads, 0, st>>>(sink, outer, 0.999999f, 1e-6f);
        else
            fma_chain_kernel<<<blocks, kPeakThreads, 0, st>>>(sink, outer, 0.999999f, 1e-6f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && run > 0 && (best < 0.f || t < best)) best = t;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return isr::fail(ISR_ERR_CUDA, "isr_fp32_peak: %s", cudaGetErrorString(e));
    const double fmas = (double)blocks * kPeakThreads * outer * kInner * kChains * (paired ? 2.0 : 1.0);
    *ms = best;
    *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
    return ISR_OK;
}
