// isr_peak.cu -- measured FP32 fused multiply-add throughput of the device.
//
// The integrate kernel is bound by the FP32 SIMT pipe, so its roofline denominator is the FP32
// peak: SMs x 128 FMA lanes x 2 FLOP x SM clock.  This microkernel measures that rate: every
// thread runs independent FMA dependency chains (enough of them to cover the pipe latency) and
// nothing else, 4 CTAs of 256 threads per SM.  The paired variant issues FFMA2 (two FP32 FMAs per
// lane and instruction) to show whether pairing raises the lane throughput or only saves issue
// slots.
#include <cuda_runtime.h>

#include <cstdint>

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

}  // namespace

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
