// isr_api.cu -- host side of the C ABI declared in include/isr.h.
//
// A plan holds the persistent FP64 accumulators, the IPP-chunk scratch and the launch
// shape.  isr_integrate splits the requested IPPs into chunks (each summed in FP32 by
// one CTA per gate group), launches the fused kernel once per block of chunks and adds
// the chunk partials into the FP64 accumulators with a reduction kernel.  Host inputs
// are streamed through two device staging buffers on a copy stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "isr.h"
#include "isr_kernels.cuh"

namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace isr {
isr_status fail(isr_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}
void clear_error() { g_err[0] = 0; }
}  // namespace isr

namespace {
using isr::fail;

#define CUDA_TRY(expr)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, \
                        "%s: %s", #expr, cudaGetErrorString(e_));                        \
    } while (0)

// restores the caller's current device on scope exit
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr unsigned kDefaultWaitLimit = 1u << 22;
constexpr int kDefaultChunk = 256;
constexpr int64_t kScratchBudget = int64_t(4) << 30;   // bytes of chunk partials
constexpr int64_t kHostStageBytes = int64_t(1) << 30;   // per host-input staging buffer
constexpr int64_t kHostFirstBytes = int64_t(64) << 20;   // first block of a host-input call

int chip_bytes(int tx_type) { return tx_type == ISR_TX_CI16 ? 4 : tx_type == ISR_TX_C32 ? 8 : 1; }

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// sum of chunk partials into the FP64 accumulators: acc[i] += sum_c part[c][i]
// s + x with the rounding error carried in c (Kahan compensated summation, FP32)
__device__ __forceinline__ void kahan_add(float& s, float& c, float x)
{
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// acc[i] += sum_c part[c][i]: the chunk partials are summed in FP32 with compensation (error
// ~2 ulp whatever the chunk count) and added once per bin into the FP64 accumulator, so the
// kernel streams at memory speed instead of waiting on FP64 conversions and additions
__global__ void reduce_partials_kernel(const float* __restrict__ part, int n_chunks, int64_t n,
                                       double* __restrict__ acc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += stride) {
        float s[4] = {0.f, 0.f, 0.f, 0.f}, cp[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c = 0; c < n_chunks; ++c) {
            const float4 v = __ldcs(reinterpret_cast<const float4*>(part + (int64_t)c * n + i));
            kahan_add(s[0], cp[0], v.x);
            kahan_add(s[1], cp[1], v.y);
            kahan_add(s[2], cp[2], v.z);
            kahan_add(s[3], cp[3], v.w);
        }
        double2* a = reinterpret_cast<double2*>(acc + i);
        double2 a0 = a[0], a1 = a[1];
        a0.x += (double)s[0] - (double)cp[0];
        a0.y += (double)s[1] - (double)cp[1];
        a1.x += (double)s[2] - (double)cp[2];
        a1.y += (double)s[3] - (double)cp[3];
        a[0] = a0;
        a[1] = a1;
    }
}

__global__ void convert_kernel(const double* __restrict__ acc, int64_t n, double scale, float* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(acc[i] * scale);
}

}  // namespace

struct isr_plan {
    isr_plan_desc d{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int log2n = 0;
    isr::KernelEntry ke{};
    double* acc = nullptr;       // [R][N]
    float* partial = nullptr;    // [max_chunks][R][N]
    int max_chunks = 0;
    int ipp_chunk = 0;
    int* status = nullptr;       // device word, bit 0 = timed-out wait
    float* out_stage = nullptr;  // [R][N] for host readback
    int64_t n_ipp_total = 0;
    int64_t launches = 0;
    unsigned wait_limit = kDefaultWaitLimit;
    int drop_ipp = -1;
    int order = 0;  // radix order of the full-length binary-phase kernel
    int precision = 0;  // ISR_PREC_*: engine of the first FFT pass
    // profiling of the fused kernel
    bool prof = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    double kernel_ms = 0;
    int64_t kernel_timed = 0;
    // host-input streaming
    cudaStream_t copy_stream = nullptr;
    uint32_t* hs_echo[2] = {nullptr, nullptr};
    char* hs_tx[2] = {nullptr, nullptr};
    int64_t hs_rows = 0;
    cudaEvent_t hs_copied[2] = {nullptr, nullptr};
    cudaEvent_t hs_free[2] = {nullptr, nullptr};
    cudaEvent_t hs_t[4] = {nullptr, nullptr, nullptr, nullptr};   // block 0: copy start / end, kernels start / end
    int64_t hs_growth = 0;    // block growth the last multi-block host-input call measured (0: none yet)
    unsigned long long* phase = nullptr;   // debug builds: [5] phase cycles of the fused kernel
};

namespace {

cudaEvent_t take_event(isr_plan* p)
{
    if (!p->ev_free.empty()) {
        cudaEvent_t e = p->ev_free.back();
        p->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// after the stream has drained: fold recorded kernel times into the counters
void harvest_events(isr_plan* p)
{
    for (auto& pr : p->ev_pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
            p->kernel_ms += ms;
            p->kernel_timed += 1;
        }
        p->ev_free.push_back(pr.first);
        p->ev_free.push_back(pr.second);
    }
    p->ev_pending.clear();
    cudaGetLastError();
}

isr_status check_geometry(const isr_plan_desc& d, int64_t start, int64_t step)
{
    if (start < 0 || step < 1) return fail(ISR_ERR_INVALID_ARG, "range_start must be >= 0 and range_step >= 1");
    int64_t last_end = start + (int64_t)(d.n_ranges - 1) * step + d.code_len;
    if (last_end > d.echo_stride)
        return fail(ISR_ERR_OUT_OF_RANGE,
                    "last gate window [%lld, %lld) runs past echo_stride %lld", (long long)(last_end - d.code_len),
                    (long long)last_end, (long long)d.echo_stride);
    return ISR_OK;
}

// Launch the fused kernel and the reduction for n rows of device-resident input.
isr_status launch_block(isr_plan* p, const uint32_t* echo, const char* tx, int64_t n, int64_t start, int64_t step)
{
    const int R = p->d.n_ranges;
    const int64_t N = p->d.nfft;
    const int64_t RN = (int64_t)R * N;
    const int rg = (R + p->ke.gates - 1) / p->ke.gates;
    const int cb = chip_bytes(p->d.tx_type);
    int64_t done = 0;
    while (done < n) {
        int64_t n_l = std::min<int64_t>(n - done, (int64_t)p->max_chunks * p->ipp_chunk);
        // chunks: enough for the FP32 sum length cap, and enough CTAs for two waves
        int64_t c_min = (n_l + p->ipp_chunk - 1) / p->ipp_chunk;
        int64_t c_fill = (2 * (int64_t)p->sm_count + rg - 1) / rg;
        int64_t C = std::max(c_min, std::min(c_fill, n_l));
        C = std::min<int64_t>(C, p->max_chunks);
        int64_t chunk = (n_l + C - 1) / C;
        C = (n_l + chunk - 1) / chunk;

        isr::KArgs a;
        a.echo = echo + done * p->d.echo_stride;
        a.echo_stride = p->d.echo_stride;
        a.tx = tx + (size_t)(done * p->d.tx_stride) * cb;
        a.tx_stride = p->d.tx_stride;
        a.partial = p->partial;
        a.status = p->status;
        a.n_ranges = R;
        a.range_start = (int)start;
        a.range_step = (int)step;
        a.code_len = p->d.code_len;
        a.n_ipp = (int)n_l;
        a.chunk_len = (int)chunk;
        a.wait_limit = p->wait_limit;
        a.drop_ipp = (p->drop_ipp >= done && p->drop_ipp < done + n_l) ? (int)(p->drop_ipp - done) : -1;
        a.phase_cycles = p->phase;

        std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
        if (p->prof) {
            ev.first = take_event(p);
            ev.second = take_event(p);
            if (ev.first && ev.second) CUDA_TRY(cudaEventRecord(ev.first, p->stream));
        }
        void* args[] = {&a};
        const bool full = p->d.code_len == p->d.nfft;
        const void* fn = full ? p->ke.fn_order[p->order] : p->ke.fn;
        int smem = full ? p->ke.smem_order[p->order] : p->ke.smem;
        if (p->precision != ISR_PREC_FP32) {
            fn = p->ke.fn_tc[p->precision];
            smem = p->ke.smem_tc;
        }
        CUDA_TRY(cudaLaunchKernel(fn, dim3((unsigned)rg, (unsigned)C), dim3((unsigned)p->ke.threads), args,
                                  (size_t)smem, p->stream));
        if (p->prof && ev.first && ev.second) {
            CUDA_TRY(cudaEventRecord(ev.second, p->stream));
            p->ev_pending.push_back(ev);
        }
        p->launches += 1;
        int threads = 256;
        int64_t blocks = std::min<int64_t>((RN / 4 + threads - 1) / threads, (int64_t)p->sm_count * 8);
        reduce_partials_kernel<<<(unsigned)blocks, threads, 0, p->stream>>>(p->partial, (int)C, RN, p->acc);
        CUDA_TRY(cudaGetLastError());
        done += n_l;
    }
    return ISR_OK;
}

isr_status ensure_host_staging(isr_plan* p, int64_t rows)
{
    if (p->hs_rows >= rows && p->hs_echo[0]) return ISR_OK;
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->hs_echo[b]);
        cudaFree(p->hs_tx[b]);
        p->hs_echo[b] = nullptr;
        p->hs_tx[b] = nullptr;
    }
    p->hs_rows = 0;
    const int64_t tx_rows = p->d.tx_stride ? rows : 1;
    const int64_t tx_bytes = ((tx_rows - 1) * p->d.tx_stride + p->d.code_len) * chip_bytes(p->d.tx_type);
    for (int b = 0; b < 2; ++b) {
        CUDA_TRY(cudaMalloc(&p->hs_echo[b], (size_t)(rows * p->d.echo_stride * 4)));
        CUDA_TRY(cudaMalloc(&p->hs_tx[b], (size_t)((tx_bytes + 15) & ~int64_t(15))));
        if (!p->hs_copied[b]) CUDA_TRY(cudaEventCreateWithFlags(&p->hs_copied[b], cudaEventDisableTiming));
        if (!p->hs_free[b]) CUDA_TRY(cudaEventCreateWithFlags(&p->hs_free[b], cudaEventDisableTiming));
    }
    for (auto& e : p->hs_t)
        if (!e) CUDA_TRY(cudaEventCreate(&e));
    if (!p->copy_stream) CUDA_TRY(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    p->hs_rows = rows;
    return ISR_OK;
}

// Host-resident input: double-buffered H2D copies on the copy stream, kernels on the
// plan stream; returns when every host row has been copied.
isr_status integrate_host(isr_plan* p, const int16_t* echo, const void* tx, int64_t n, int64_t start, int64_t step)
{
    const int64_t row_bytes = p->d.echo_stride * 4;
    int64_t rows = std::max<int64_t>(1, std::min<int64_t>(n, kHostStageBytes / row_bytes));
    isr_status st = ensure_host_staging(p, rows);
    if (st != ISR_OK) return st;
    rows = p->hs_rows;
    const int cb = chip_bytes(p->d.tx_type);
    const char* txc = static_cast<const char*>(tx);
    bool tx_dev = is_device_ptr(tx);
    // A call larger than one staging buffer starts with a small block, so the kernels get going
    // after a short copy, and the blocks then grow up to a buffer, with few launches (each ends
    // with a partly filled wave).  The copy of block i + 1 stays hidden behind block i's kernels
    // while growth <= (kernel time) / (copy time) of equal blocks; the host link differs from box
    // to box, so block 0's copy and kernels are timed, block 1 doubles meanwhile, and once block 1
    // is queued the host waits for block 0's kernels and takes growth = that ratio, within 1..4.
    // A call that fits one buffer is one block.
    const bool several = n > rows;
    int64_t cur = several ? std::max<int64_t>(1, std::min<int64_t>(rows, kHostFirstBytes / row_bytes)) : rows;
    int64_t growth = 2;
    int blk = 0;
    for (int64_t done = 0, nb = 0; done < n; done += nb, ++blk, cur = std::min<int64_t>(rows, growth * cur)) {
        const int b = blk & 1;
        nb = std::min(cur, n - done);
        const bool time0 = several && blk == 0;
        CUDA_TRY(cudaStreamWaitEvent(p->copy_stream, p->hs_free[b], 0));
        if (time0) CUDA_TRY(cudaEventRecord(p->hs_t[0], p->copy_stream));
        CUDA_TRY(cudaMemcpyAsync(p->hs_echo[b], echo + done * p->d.echo_stride * 2, (size_t)(nb * row_bytes),
                                 cudaMemcpyHostToDevice, p->copy_stream));
        const char* txblk;
        if (tx_dev) {
            txblk = txc + (size_t)(done * p->d.tx_stride) * cb;
        } else {
            const int64_t tx_rows = p->d.tx_stride ? nb : 1;
            const int64_t tx_bytes = ((tx_rows - 1) * p->d.tx_stride + p->d.code_len) * cb;
            CUDA_TRY(cudaMemcpyAsync(p->hs_tx[b], txc + (size_t)(done * p->d.tx_stride) * cb, (size_t)tx_bytes,
                                     cudaMemcpyHostToDevice, p->copy_stream));
            txblk = p->hs_tx[b];
        }
        CUDA_TRY(cudaEventRecord(p->hs_copied[b], p->copy_stream));
        if (time0) CUDA_TRY(cudaEventRecord(p->hs_t[1], p->copy_stream));
        CUDA_TRY(cudaStreamWaitEvent(p->stream, p->hs_copied[b], 0));
        if (time0) CUDA_TRY(cudaEventRecord(p->hs_t[2], p->stream));
        st = launch_block(p, p->hs_echo[b], txblk, nb, start, step);
        if (st != ISR_OK) return st;
        if (time0) CUDA_TRY(cudaEventRecord(p->hs_t[3], p->stream));
        CUDA_TRY(cudaEventRecord(p->hs_free[b], p->stream));
        if (several && blk == 1) {
            // block 1 is queued, so the GPU stays busy while the host waits for block 0's kernels
            float tc = 0.f, tk = 0.f;
            CUDA_TRY(cudaEventSynchronize(p->hs_t[3]));
            CUDA_TRY(cudaEventElapsedTime(&tc, p->hs_t[0], p->hs_t[1]));
            CUDA_TRY(cudaEventElapsedTime(&tk, p->hs_t[2], p->hs_t[3]));
            growth = tc > 0.f ? std::max<int64_t>(1, std::min<int64_t>(4, (int64_t)(tk / tc))) : 4;
            p->hs_growth = growth;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(p->copy_stream));
    return ISR_OK;
}

}  // namespace

extern "C" {

const char* isr_last_error(void) { return g_err; }

isr_status isr_plan_create(isr_plan** out, const isr_plan_desc* desc)
{
    g_err[0] = 0;
    if (!out) return fail(ISR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(ISR_ERR_INVALID_ARG, "desc is NULL");
    const isr_plan_desc& d = *desc;
    if (d.nfft < 8 || d.nfft > 16384 || (d.nfft & (d.nfft - 1)))
        return fail(ISR_ERR_UNSUPPORTED, "nfft %d is not a power of two in [8, 16384]", d.nfft);
    if (d.tx_type != ISR_TX_CI16 && d.tx_type != ISR_TX_C32 && d.tx_type != ISR_TX_PM1)
        return fail(ISR_ERR_UNSUPPORTED, "unknown tx_type %d", d.tx_type);
    if (d.code_len < 1 || d.code_len > d.nfft) return fail(ISR_ERR_INVALID_ARG, "code_len must be in [1, nfft]");
    if (d.n_ranges < 1) return fail(ISR_ERR_INVALID_ARG, "n_ranges must be >= 1");
    if (d.echo_stride < 4 || d.echo_stride % 4) return fail(ISR_ERR_INVALID_ARG, "echo_stride must be a positive multiple of 4");
    if (d.echo_stride > (int64_t(1) << 40)) return fail(ISR_ERR_INVALID_ARG, "echo_stride too large");
    if (d.tx_stride < 0 || (d.tx_stride > 0 && d.tx_stride < d.code_len))
        return fail(ISR_ERR_INVALID_ARG, "tx_stride must be 0 or >= code_len");
    if (d.ipp_chunk < 0 || d.max_chunks < 0 || d.max_chunks > 65535 || d.flags != 0)
        return fail(ISR_ERR_INVALID_ARG, "ipp_chunk must be >= 0, max_chunks in [0, 65535], flags 0");
    if (d.range_start > (1 << 30) || d.range_step > (1 << 30))
        return fail(ISR_ERR_INVALID_ARG, "range_start and range_step must be < 2^30");
    isr_status st = check_geometry(d, d.range_start, d.range_step);
    if (st != ISR_OK) return st;

    int dev = d.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(ISR_ERR_CUDA, "no current CUDA device");
    DeviceGuard guard(dev);
    if (!guard.ok) return fail(ISR_ERR_CUDA, "cannot select CUDA device %d", dev);

    isr_plan* p = new (std::nothrow) isr_plan();
    if (!p) return fail(ISR_ERR_NO_MEMORY, "host allocation failed");
    p->d = d;
    p->dev = dev;
    p->stream = static_cast<cudaStream_t>(d.stream);
    int lg = 0;
    while ((1 << lg) < d.nfft) ++lg;
    p->log2n = lg;
    p->ke = isr::kernel_entry(lg, d.tx_type);
    p->ipp_chunk = d.ipp_chunk > 0 ? d.ipp_chunk : kDefaultChunk;

    auto bail = [&](isr_status s) {
        isr_destroy(p);
        return s;
    };
    cudaError_t e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "device query failed: %s", cudaGetErrorString(e)));
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (p->ke.smem > smem_optin)
        return bail(fail(ISR_ERR_UNSUPPORTED, "kernel needs %d B shared memory, device allows %d", p->ke.smem, smem_optin));
    e = cudaFuncSetAttribute(p->ke.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, p->ke.smem);
    for (int o = 0; o < isr::kNumOrders && e == cudaSuccess; ++o)
        e = cudaFuncSetAttribute(p->ke.fn_order[o], cudaFuncAttributeMaxDynamicSharedMemorySize, p->ke.smem_order[o]);
    if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));

    const int64_t RN = (int64_t)d.n_ranges * d.nfft;
    int64_t mc = d.max_chunks > 0 ? d.max_chunks : std::min<int64_t>(64, std::max<int64_t>(1, kScratchBudget / (RN * 4)));
    p->max_chunks = (int)mc;
    e = cudaMalloc(&p->acc, (size_t)(RN * 8));
    if (e == cudaSuccess) e = cudaMalloc(&p->partial, (size_t)(mc * RN * 4));
    if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int));
#ifdef ISR_DEBUG
    if (e == cudaSuccess) e = cudaMalloc(&p->phase, 5 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->phase, 0, 5 * sizeof(unsigned long long), p->stream);
#endif
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(e == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, "device allocation failed: %s",
                         cudaGetErrorString(e)));
    }
    e = cudaMemsetAsync(p->acc, 0, (size_t)(RN * 8), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->status, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "initialisation failed: %s", cudaGetErrorString(e)));
    *out = p;
    return ISR_OK;
}

isr_status isr_integrate(isr_plan* p, const int16_t* echo, const void* tx, int32_t n_ipp, const isr_ranges* ranges,
                         int32_t nfft)
{
    g_err[0] = 0;
    if (!p) return fail(ISR_ERR_INVALID_ARG, "plan is NULL");
    if (nfft != p->d.nfft) return fail(ISR_ERR_INVALID_ARG, "nfft %d does not match the plan's %d", nfft, p->d.nfft);
    if (n_ipp < 0) return fail(ISR_ERR_INVALID_ARG, "n_ipp < 0");
    if (n_ipp == 0) return ISR_OK;
    if (!echo || !tx) return fail(ISR_ERR_INVALID_ARG, "echo and tx_code must not be NULL");
    if (reinterpret_cast<uintptr_t>(echo) % 16) return fail(ISR_ERR_INVALID_ARG, "echo must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(tx) % chip_bytes(p->d.tx_type))
        return fail(ISR_ERR_INVALID_ARG, "tx_code must be aligned to its chip size");
    int64_t start = p->d.range_start, step = p->d.range_step;
    if (ranges) {
        if (ranges->count != p->d.n_ranges)
            return fail(ISR_ERR_INVALID_ARG, "ranges->count %d differs from the plan's n_ranges %d", ranges->count,
                        p->d.n_ranges);
        if (ranges->start > (1 << 30) || ranges->step > (1 << 30))
            return fail(ISR_ERR_INVALID_ARG, "range start and step must be < 2^30");
        start = ranges->start;
        step = ranges->step;
    }
    isr_status st = check_geometry(p->d, start, step);
    if (st != ISR_OK) return st;

    DeviceGuard guard(p->dev);
    if (!guard.ok) return fail(ISR_ERR_CUDA, "cannot select CUDA device %d", p->dev);
    if (is_device_ptr(echo)) {
        st = launch_block(p, reinterpret_cast<const uint32_t*>(echo), static_cast<const char*>(tx), n_ipp, start, step);
    } else {
        st = integrate_host(p, echo, tx, n_ipp, start, step);
    }
    if (st == ISR_OK) p->n_ipp_total += n_ipp;
    return st;
}

isr_status isr_spectra(isr_plan* p, float* out, int32_t flags, int64_t* n_ipp_out)
{
    g_err[0] = 0;
    if (!p) return fail(ISR_ERR_INVALID_ARG, "plan is NULL");
    if (flags & ~(ISR_RESET_AFTER | ISR_MEAN)) return fail(ISR_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    DeviceGuard guard(p->dev);
    if (!guard.ok) return fail(ISR_ERR_CUDA, "cannot select CUDA device %d", p->dev);
    const int64_t RN = (int64_t)p->d.n_ranges * p->d.nfft;
    const double scale = ((flags & ISR_MEAN) && p->n_ipp_total > 0) ? 1.0 / (double)p->n_ipp_total : 1.0;
    if (out) {
        const bool dev_out = is_device_ptr(out);
        float* dst = out;
        if (!dev_out) {
            if (!p->out_stage) CUDA_TRY(cudaMalloc(&p->out_stage, (size_t)(RN * 4)));
            dst = p->out_stage;
        }
        int threads = 256;
        int64_t blocks = std::min<int64_t>((RN + threads - 1) / threads, (int64_t)p->sm_count * 8);
        convert_kernel<<<(unsigned)blocks, threads, 0, p->stream>>>(p->acc, RN, scale, dst);
        CUDA_TRY(cudaGetLastError());
        if (!dev_out) CUDA_TRY(cudaMemcpyAsync(out, dst, (size_t)(RN * 4), cudaMemcpyDeviceToHost, p->stream));
    }
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(&status, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    harvest_events(p);
    if (n_ipp_out) *n_ipp_out = p->n_ipp_total;
    if (flags & ISR_RESET_AFTER) {
        CUDA_TRY(cudaMemsetAsync(p->acc, 0, (size_t)(RN * 8), p->stream));
        p->n_ipp_total = 0;
    }
    if (status) {
        CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
        CUDA_TRY(cudaStreamSynchronize(p->stream));
        if (status & 2)
            return fail(ISR_ERR_OUT_OF_RANGE, "a kernel found a gate window outside its echo row (debug build check)");
        return fail(ISR_ERR_TIMEOUT, "a kernel timed out waiting for its staged echo window");
    }
    return ISR_OK;
}

isr_status isr_plan_query(const isr_plan* p, isr_plan_info* info)
{
    if (!p || !info) return fail(ISR_ERR_INVALID_ARG, "plan and info must not be NULL");
    info->nfft = p->d.nfft;
    info->n_ranges = p->d.n_ranges;
    info->ranges_per_cta = p->ke.gates;
    info->threads_per_cta = p->ke.threads;
    info->smem_bytes = p->ke.smem;
    info->max_chunks = p->max_chunks;
    info->ipp_chunk = p->ipp_chunk;
    info->sm_count = p->sm_count;
    info->n_ipp_integrated = p->n_ipp_total;
    info->kernel_launches = p->launches;
    info->kernel_ms = p->kernel_ms;
    info->kernel_timed = p->kernel_timed;
    info->host_block_growth = p->hs_growth;
    return ISR_OK;
}

isr_status isr_plan_set_profiling(isr_plan* p, int32_t enable)
{
    if (!p) return fail(ISR_ERR_INVALID_ARG, "plan is NULL");
    p->prof = enable != 0;
    return ISR_OK;
}

isr_status isr_plan_phase_cycles(isr_plan* p, uint64_t* out)
{
    if (!p || !out) return fail(ISR_ERR_INVALID_ARG, "plan or out is NULL");
    if (!p->phase) return fail(ISR_ERR_UNSUPPORTED, "phase cycles are recorded by the debug build only (-DISR_DEBUG)");
    DeviceGuard guard(p->dev);
    CUDA_TRY(cudaStreamSynchronize(p->stream));
    unsigned long long h[5];
    CUDA_TRY(cudaMemcpy(h, p->phase, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < 5; ++i) out[i] = (uint64_t)h[i];
    return ISR_OK;
}

isr_status isr_plan_set_wait_limit(isr_plan* p, uint32_t polls)
{
    if (!p || polls == 0) return fail(ISR_ERR_INVALID_ARG, "plan is NULL or polls is 0");
    p->wait_limit = polls;
    return ISR_OK;
}

isr_status isr_plan_set_order(isr_plan* p, int32_t order)
{
    if (!p || order < 0 || order >= isr::kNumOrders)
        return fail(ISR_ERR_INVALID_ARG, "plan is NULL or order not in 0..%d", isr::kNumOrders - 1);
    if (p->d.nfft < 2048 && order != 0) return fail(ISR_ERR_UNSUPPORTED, "radix orders exist for nfft >= 2048 only");
    if (order >= 4 && (p->d.nfft != 16384 || p->d.tx_type != ISR_TX_PM1))
        return fail(ISR_ERR_UNSUPPORTED, "radix orders 4 to 9 exist for nfft 16384 with ISR_TX_PM1 only");
    p->order = order;
    return ISR_OK;
}

isr_status isr_plan_set_precision(isr_plan* p, int32_t precision)
{
    if (!p || precision < ISR_PREC_FP32 || precision > ISR_PREC_TC05_FP16)
        return fail(ISR_ERR_INVALID_ARG, "plan is NULL or unknown precision %d", precision);
    if (precision != ISR_PREC_FP32) {
        if (p->d.nfft != 16384 || p->d.tx_type != ISR_TX_PM1 || p->d.code_len != p->d.nfft || !p->ke.fn_tc[precision])
            return fail(ISR_ERR_UNSUPPORTED, "tensor-core first pass: nfft 16384, ISR_TX_PM1, code_len == nfft only");
        DeviceGuard guard(p->dev);
        cudaError_t e = cudaFuncSetAttribute(p->ke.fn_tc[precision], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             p->ke.smem_tc);
        if (e != cudaSuccess) return fail(ISR_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    }
    p->precision = precision;
    return ISR_OK;
}

isr_status isr_plan_test_drop_window(isr_plan* p, int32_t ipp)
{
    if (!p || ipp < -1) return fail(ISR_ERR_INVALID_ARG, "plan is NULL or ipp < -1");
    p->drop_ipp = ipp;
    return ISR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- allocation-free variant
namespace {

// IPP-chunk partials of isr_integrate_static: [chunks][n_ranges][nfft] floats, plus the
// variant's own status word.  Host code must not use these names as addresses (they are
// host-side shadows); it looks up each device's copy with cudaGetSymbolAddress.
__device__ __align__(256) float g_static_scratch[ISR_STATIC_SCRATCH_FLOATS];
__device__ __align__(16) int g_static_status[4];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_scratch_ptr[kMaxDevices] = {};
int* g_static_status_ptr[kMaxDevices] = {};

// out[i] = (float) sum_c part[c][i] (first block of IPPs) or (float)(out[i] + sum_c part[c][i])
// (later blocks), summed in double: one FP32 rounding of the running sum per block
__global__ void reduce_to_spectra_kernel(const float* __restrict__ part, int n_chunks, int64_t n,
                                         float* __restrict__ out, int accumulate)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double s = accumulate ? (double)out[i] : 0.0;
        for (int c = 0; c < n_chunks; ++c) s += part[(int64_t)c * n + i];
        out[i] = (float)s;
    }
}

// device addresses of the file-scope arrays on `dev` (looked up once per device)
isr_status static_buffers(int dev, float** scratch, int** status)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(ISR_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_scratch_ptr[dev]) {
        void* a = nullptr;
        void* b = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&a, g_static_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&b, g_static_status);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ISR_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        }
        g_static_scratch_ptr[dev] = static_cast<float*>(a);
        g_static_status_ptr[dev] = static_cast<int*>(b);
    }
    *scratch = g_static_scratch_ptr[dev];
    *status = g_static_status_ptr[dev];
    return ISR_OK;
}

}  // namespace

extern "C" {

isr_status isr_integrate_static(const isr_plan_desc* desc, const int16_t* echo, const void* tx, int32_t n_ipp,
                                float* out)
{
    g_err[0] = 0;
    if (!desc) return fail(ISR_ERR_INVALID_ARG, "desc is NULL");
    const isr_plan_desc& d = *desc;
    if (d.nfft < 8 || d.nfft > 16384 || (d.nfft & (d.nfft - 1)))
        return fail(ISR_ERR_UNSUPPORTED, "nfft %d is not a power of two in [8, 16384]", d.nfft);
    if (d.tx_type != ISR_TX_CI16 && d.tx_type != ISR_TX_C32 && d.tx_type != ISR_TX_PM1)
        return fail(ISR_ERR_UNSUPPORTED, "unknown tx_type %d", d.tx_type);
    if (d.code_len < 1 || d.code_len > d.nfft) return fail(ISR_ERR_INVALID_ARG, "code_len must be in [1, nfft]");
    if (d.n_ranges < 1) return fail(ISR_ERR_INVALID_ARG, "n_ranges must be >= 1");
    if (d.echo_stride < 4 || d.echo_stride % 4) return fail(ISR_ERR_INVALID_ARG, "echo_stride must be a positive multiple of 4");
    if (d.tx_stride < 0 || (d.tx_stride > 0 && d.tx_stride < d.code_len))
        return fail(ISR_ERR_INVALID_ARG, "tx_stride must be 0 or >= code_len");
    if (d.range_start > (1 << 30) || d.range_step > (1 << 30) || d.flags != 0)
        return fail(ISR_ERR_INVALID_ARG, "range_start and range_step must be < 2^30, flags 0");
    isr_status st = check_geometry(d, d.range_start, d.range_step);
    if (st != ISR_OK) return st;
    const int64_t RN = (int64_t)d.n_ranges * d.nfft;
    if (RN > ISR_STATIC_SCRATCH_FLOATS)
        return fail(ISR_ERR_INVALID_ARG, "n_ranges * nfft = %lld exceeds the static scratch of %d floats",
                    (long long)RN, ISR_STATIC_SCRATCH_FLOATS);
    if (n_ipp < 1) return fail(ISR_ERR_INVALID_ARG, "n_ipp must be >= 1");
    if (!echo || !tx || !out) return fail(ISR_ERR_INVALID_ARG, "echo, tx_code and out must not be NULL");
    if (reinterpret_cast<uintptr_t>(echo) % 16) return fail(ISR_ERR_INVALID_ARG, "echo must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(tx) % chip_bytes(d.tx_type))
        return fail(ISR_ERR_INVALID_ARG, "tx_code must be aligned to its chip size");
    if (!is_device_ptr(echo) || !is_device_ptr(tx) || !is_device_ptr(out))
        return fail(ISR_ERR_INVALID_ARG, "echo, tx_code and out must be device memory");

    int dev = d.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(ISR_ERR_CUDA, "no current CUDA device");
    DeviceGuard guard(dev);
    if (!guard.ok) return fail(ISR_ERR_CUDA, "cannot select CUDA device %d", dev);
    float* scratch = nullptr;
    int* status = nullptr;
    st = static_buffers(dev, &scratch, &status);
    if (st != ISR_OK) return st;

    int lg = 0;
    while ((1 << lg) < d.nfft) ++lg;
    isr::KernelEntry ke = isr::kernel_entry(lg, d.tx_type);
    CUDA_TRY(cudaFuncSetAttribute(ke.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ke.smem));
    int sm_count = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t stream = static_cast<cudaStream_t>(d.stream);

    // Chunks: FP32 sums of at most kDefaultChunk IPPs (the bound the per-bin tolerance rests
    // on), at most c_cap of them in the scratch at once.  The IPPs run in blocks of at most
    // c_cap * kDefaultChunk: one fused launch and one reduction per block, the reduction of
    // every block after the first adding into `out`.  Within a block, two waves of CTAs when
    // the IPP count allows.
    const int rg = (d.n_ranges + ke.gates - 1) / ke.gates;
    const int64_t c_cap = std::min<int64_t>(65535, ISR_STATIC_SCRATCH_FLOATS / RN);
    const int64_t block_cap = c_cap * kDefaultChunk;
    const int64_t c_fill = (2 * (int64_t)sm_count + rg - 1) / rg;

    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), stream));
    const int cb = chip_bytes(d.tx_type);
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((RN + threads - 1) / threads, (int64_t)sm_count * 8);
    for (int64_t done = 0; done < n_ipp;) {
        const int64_t n_l = std::min<int64_t>(n_ipp - done, block_cap);
        const int64_t c_min = (n_l + kDefaultChunk - 1) / kDefaultChunk;
        int64_t C = std::min(c_cap, std::max(c_min, std::min<int64_t>(c_fill, n_l)));
        const int64_t chunk = (n_l + C - 1) / C;
        C = (n_l + chunk - 1) / chunk;

        isr::KArgs a;
        a.echo = reinterpret_cast<const uint32_t*>(echo) + done * d.echo_stride;
        a.echo_stride = d.echo_stride;
        a.tx = static_cast<const char*>(tx) + (size_t)(done * d.tx_stride) * cb;
        a.tx_stride = d.tx_stride;
        a.partial = scratch;
        a.status = status;
        a.n_ranges = d.n_ranges;
        a.range_start = d.range_start;
        a.range_step = d.range_step;
        a.code_len = d.code_len;
        a.n_ipp = (int)n_l;
        a.chunk_len = (int)chunk;
        a.wait_limit = kDefaultWaitLimit;
        a.drop_ipp = -1;
        void* args[] = {&a};
        CUDA_TRY(cudaLaunchKernel(ke.fn, dim3((unsigned)rg, (unsigned)C), dim3((unsigned)ke.threads), args,
                                  (size_t)ke.smem, stream));
        reduce_to_spectra_kernel<<<(unsigned)blocks, threads, 0, stream>>>(scratch, (int)C, RN, out, done > 0);
        CUDA_TRY(cudaGetLastError());
        done += n_l;
    }
    int flag = 0;
    CUDA_TRY(cudaMemcpyAsync(&flag, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    if (flag & 2)
        return fail(ISR_ERR_OUT_OF_RANGE, "a kernel found a gate window outside its echo row (debug build check)");
    if (flag) return fail(ISR_ERR_TIMEOUT, "a kernel timed out waiting for its staged echo window");
    return ISR_OK;
}

void isr_destroy(isr_plan* p)
{
    if (!p) return;
    DeviceGuard guard(p->dev);
    if (p->stream || p->acc) cudaStreamSynchronize(p->stream);
    if (p->copy_stream) {
        cudaStreamSynchronize(p->copy_stream);
        cudaStreamDestroy(p->copy_stream);
    }
    for (auto& pr : p->ev_pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : p->ev_free) cudaEventDestroy(e);
    for (int b = 0; b < 2; ++b) {
        cudaFree(p->hs_echo[b]);
        cudaFree(p->hs_tx[b]);
        if (p->hs_copied[b]) cudaEventDestroy(p->hs_copied[b]);
        if (p->hs_free[b]) cudaEventDestroy(p->hs_free[b]);
    }
    for (auto e : p->hs_t)
        if (e) cudaEventDestroy(e);
    cudaFree(p->acc);
    cudaFree(p->partial);
    cudaFree(p->status);
    cudaFree(p->phase);
    cudaFree(p->out_stage);
    cudaGetLastError();
    delete p;
}

}  // extern "C"
