/*
 * synth_gpu.cu -- device (nvcc) build of the seeded synthetic echo generator, for inputs
 * too large to make on the host (the 10,000-IPP workload is 1.66 GB of int16 IQ).
 * All arithmetic is in synth_core.h; compiled with -fmad=false so each sample equals the
 * host build's bit for bit.  Not part of the integration library and never timed.
 */
#include <cuda_runtime.h>
#include "synth_core.h"

__global__ void syn_table_kernel(float* table)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < SYN_TABLE_SIZE) syn_table_entry(j, &table[2 * j], &table[2 * j + 1]);
}

__global__ void syn_params_kernel(syn_cfg c, const double* f_base, const double* amp_gate, int64_t row_begin,
                                  int64_t n_rows, syn_rp* rp)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rows * c.n_ranges) return;
    int64_t pr = i / c.n_ranges;
    int r = (int)(i - pr * c.n_ranges);
    rp[i] = syn_range_params(&c, f_base[r], amp_gate ? amp_gate[r] : c.amp, r, (int)(row_begin + pr));
}

__global__ void syn_echo_kernel(syn_cfg c, const syn_rp* rp, const int8_t* code,
                                const float* table, int64_t row_begin, int16_t* out)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t pr = blockIdx.y;
    if (t >= c.echo_stride) return;
    int64_t p = row_begin + pr;
    const int8_t* crow = code + (c.per_ipp_code ? p * c.code_len : 0);
    int16_t I, Q;
    syn_sample(&c, rp + pr * c.n_ranges, crow, table, t, (int)p, &I, &Q);
    int16_t* o = out + (pr * c.echo_stride + t) * 2;
    o[0] = I;
    o[1] = Q;
}

/*
 * Generate rows [row_begin, row_end) into echo_dev (row_begin maps to echo_dev row 0).
 * f_base_host: [n_ranges] doubles; amp_host: [n_ranges] doubles or NULL (cfg->amp for every
 * gate); code_dev: device chips as for syn_echo_rows.
 * Synchronous.  Returns a cudaError_t value (0 = success).
 */
extern "C" int syn_gpu_echo(const syn_cfg* cfg, const double* f_base_host, const double* amp_host,
                            const int8_t* code_dev, int64_t row_begin, int64_t row_end, int16_t* echo_dev)
{
    syn_cfg c = *cfg;
    cudaError_t e;
    float* table = nullptr;
    double* fb = nullptr;
    double* ab = nullptr;
    syn_rp* rp = nullptr;
    int64_t rows_per_batch = 512;
    int nr = c.n_ranges > 0 ? c.n_ranges : 1;
    if ((e = cudaMalloc(&table, sizeof(float) * 2 * SYN_TABLE_SIZE)) != cudaSuccess) goto done;
    if ((e = cudaMalloc(&fb, sizeof(double) * nr)) != cudaSuccess) goto done;
    if (amp_host && (e = cudaMalloc(&ab, sizeof(double) * nr)) != cudaSuccess) goto done;
    if (amp_host && c.n_ranges > 0 &&
        (e = cudaMemcpy(ab, amp_host, sizeof(double) * c.n_ranges, cudaMemcpyHostToDevice)) != cudaSuccess)
        goto done;
    if ((e = cudaMalloc(&rp, sizeof(syn_rp) * nr * rows_per_batch)) != cudaSuccess) goto done;
    if (c.n_ranges > 0 &&
        (e = cudaMemcpy(fb, f_base_host, sizeof(double) * c.n_ranges, cudaMemcpyHostToDevice)) != cudaSuccess)
        goto done;
    syn_table_kernel<<<SYN_TABLE_SIZE / 256, 256>>>(table);
    for (int64_t b = row_begin; b < row_end; b += rows_per_batch) {
        int64_t n = row_end - b < rows_per_batch ? row_end - b : rows_per_batch;
        if (c.n_ranges > 0) {
            int64_t tot = n * c.n_ranges;
            syn_params_kernel<<<(unsigned)((tot + 255) / 256), 256>>>(c, fb, ab, b, n, rp);
        }
        dim3 grid((unsigned)((c.echo_stride + 255) / 256), (unsigned)n);
        syn_echo_kernel<<<grid, 256>>>(c, rp, code_dev, table, b, echo_dev + (b - row_begin) * c.echo_stride * 2);
        if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    }
    e = cudaDeviceSynchronize();
done:
    cudaFree(table);
    cudaFree(fb);
    cudaFree(ab);
    cudaFree(rp);
    return (int)e;
}
