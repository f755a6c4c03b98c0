// isr_linefit.cu -- plasma-line frequency by spectral peak fit on integrated spectra.
//
// The plasma line's frequency carries the electron density (Eq. 1 of the paper: f_r^2 =
// f_p^2 + thermal and magnetic terms, f_p ~ sqrt(n_e)), so the product of an integration is
// the line position per gate.  Per gate: the largest bin of the band, refined by a
// three-point parabola through the logarithm of the power (exact for a Gaussian-shaped
// peak), in double precision; plus the ratio of the peak to the band's mean power.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "isr.h"
#include "isr_kernels.cuh"

namespace {

constexpr int kFitThreads = 256;

__global__ void __launch_bounds__(kFitThreads) peak_fit_kernel(const float* __restrict__ spectra, int nfft,
                                                               int band_lo, int band_hi, double* __restrict__ freq_bin,
                                                               float* __restrict__ snr)
{
    const int r = blockIdx.x;
    const float* P = spectra + (size_t)r * nfft;
    float best = -INFINITY;
    int best_i = band_lo;
    double sum = 0.0;
    for (int i = band_lo + threadIdx.x; i < band_hi; i += kFitThreads) {
        float v = P[i];
        if (v > best) {  // strided scan in increasing i keeps the lowest index on ties
            best = v;
            best_i = i;
        }
        sum += (double)v;
    }
    // block reduction: max value, lowest index among equal maxima; double sum
    __shared__ float s_best[kFitThreads / 32];
    __shared__ int s_idx[kFitThreads / 32];
    __shared__ double s_sum[kFitThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        float ob = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, best_i, o);
        double os = __shfl_down_sync(0xffffffffu, sum, o);
        if (ob > best || (ob == best && oi < best_i)) {
            best = ob;
            best_i = oi;
        }
        sum += os;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        s_best[w] = best;
        s_idx[w] = best_i;
        s_sum[w] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        best = s_best[0];
        best_i = s_idx[0];
        sum = s_sum[0];
        for (int k = 1; k < kFitThreads / 32; ++k) {
            if (s_best[k] > best || (s_best[k] == best && s_idx[k] < best_i)) {
                best = s_best[k];
                best_i = s_idx[k];
            }
            sum += s_sum[k];
        }
        const double mean = sum / (double)(band_hi - band_lo);
        const double pm = P[(best_i - 1 + nfft) % nfft], p0 = best, pp = P[(best_i + 1) % nfft];
        double delta = 0.0;
        if (pm > 0.0 && p0 > 0.0 && pp > 0.0) {
            const double ym = log(pm), y0 = log(p0), yp = log(pp);
            const double d = ym - 2.0 * y0 + yp;
            if (d < 0.0) delta = 0.5 * (ym - yp) / d;
            delta = fmin(0.5, fmax(-0.5, delta));
        }
        freq_bin[r] = (double)best_i + delta;
        snr[r] = mean > 0.0 ? (float)(p0 / mean) : 0.f;
    }
}

}  // namespace

extern "C" isr_status isr_peak_fit(const float* spectra, int32_t n_ranges, int32_t nfft, int32_t band_lo,
                                   int32_t band_hi, double* freq_bin, float* snr, void* stream)
{
    isr::clear_error();
    if (!spectra || !freq_bin || !snr) return isr::fail(ISR_ERR_INVALID_ARG, "isr_peak_fit: NULL pointer");
    if (n_ranges < 1 || nfft < 8 || band_lo < 0 || band_hi > nfft || band_hi - band_lo < 1)
        return isr::fail(ISR_ERR_INVALID_ARG, "isr_peak_fit: need n_ranges >= 1, nfft >= 8, 0 <= band_lo < band_hi <= nfft");
    peak_fit_kernel<<<n_ranges, kFitThreads, 0, static_cast<cudaStream_t>(stream)>>>(spectra, nfft, band_lo, band_hi,
                                                                                   freq_bin, snr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return isr::fail(ISR_ERR_CUDA, "isr_peak_fit: %s", cudaGetErrorString(e));
    return ISR_OK;
}
