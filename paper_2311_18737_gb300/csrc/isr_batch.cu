// isr_batch.cu -- many integration windows of uneven shape in one persistent launch.
//
// A radar usually integrates several windows at once: up- and down-shifted plasma-line
// channels (the line sits at +-f_r, Sec. 2.1 of the paper), different range extents and
// spectral resolutions.  Here every window's (gate group, IPP chunk) work units form one
// queue, ordered longest first; one CTA per SM pulls units from the queue with an atomic
// counter and runs the fused decode -> FFT -> |X|^2 unit of the matching transform length.
// The launch and the chunk reduction can be captured once in a CUDA graph and replayed.
// The Stockham radix order of each transform length can be picked by timing the
// candidates on the windows themselves (autotuning).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "isr.h"
#include "isr_kernels.cuh"

namespace {

using isr::fail;

constexpr int kMinLog2 = 11, kMaxLog2 = 14;
constexpr int kChunk = 256;
constexpr unsigned kWaitLimit = 1u << 22;

struct BatchWin {
    isr::KArgs a;
    int log2n;
    int order;
    int n_gx;   // gate groups
    int n_cy;   // IPP chunks
};

struct BatchUnit {
    int win, gx, cy, pad;
};

template <int L, int O>
constexpr int smem_of() { return isr::Sched<L, O>::SMEM; }

constexpr int max_smem()
{
    int m = 0;
    int v[] = {smem_of<11, 0>(), smem_of<11, 1>(), smem_of<11, 2>(), smem_of<12, 0>(), smem_of<12, 1>(),
               smem_of<12, 2>(), smem_of<13, 0>(), smem_of<13, 1>(), smem_of<13, 2>(), smem_of<14, 0>(),
               smem_of<14, 1>(), smem_of<14, 2>(), isr::SchedWL<11>::SMEM, isr::SchedWL<12>::SMEM,
               isr::SchedWL<13>::SMEM, isr::SchedWL<14>::SMEM};
    for (int x : v) m = x > m ? x : m;
    return m;
}
constexpr int kBatchSmem = max_smem();

// one call per shape: each shape keeps its own register allocation instead of sharing one
template <int L, int O>
__device__ __noinline__ bool run_unit(const BatchWin& w, const BatchUnit& u, unsigned char* smem,
                                      const uint32_t* s_phase, bool setup)
{
    if constexpr (O == 3) {
        using S = isr::SchedWL<L>;
        return isr::integrate_unit_wl<L, isr::TX_PM1, false, const isr::KArgs&>(w.a, u.gx, u.cy, smem, s_phase[threadIdx.x / S::T],
                                                             setup);
    } else {
        using S = isr::Sched<L, O>;
        // every sample on the conversion instruction: the persistent kernel holds all window
        // shapes at the 128-register cap, where the split decode measured slower
        return isr::integrate_unit<L, isr::TX_PM1, O, false, isr::P0_SIMT, const isr::KArgs&, false, false>(
            w.a, u.gx, u.cy, smem, s_phase[threadIdx.x / S::T], setup);
    }
}

// Persistent: one CTA per SM pulls work units until the queue is empty.
__global__ void __launch_bounds__(isr::kThreads, 1) batch_kernel(const BatchWin* __restrict__ wins,
                                                                 const BatchUnit* __restrict__ units, int n_units,
                                                                 int* __restrict__ counter)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_phase[8];
    __shared__ int s_unit;
    // the current unit and its window's arguments: read from shared memory where a unit needs
    // them instead of being held in registers for the whole unit
    __shared__ BatchUnit s_u;
    __shared__ BatchWin s_w;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);   // slot g at byte 8 g for every shape
    if (threadIdx.x < 8) {
        isr::mbar_init(isr::smem_u32(&mbar[threadIdx.x]), 1);
        s_phase[threadIdx.x] = 0;
    }
    isr::fence_barrier_init();
    int prev_key = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int ui = atomicAdd(counter, 1);
            s_unit = ui;
            if (ui < n_units) {
                s_u = units[ui];
                s_w = wins[s_u.win];
            }
        }
        __syncthreads();
        if (s_unit >= n_units) break;
        const BatchUnit& u = s_u;
        const BatchWin& w = s_w;
        const int key = w.log2n * 4 + w.order;
        const bool setup = key != prev_key;
        bool ok = true;
        switch (key) {
        case 11 * 4 + 0: ok = run_unit<11, 0>(w, u, smem, s_phase, setup); break;
        case 11 * 4 + 1: ok = run_unit<11, 1>(w, u, smem, s_phase, setup); break;
        case 11 * 4 + 2: ok = run_unit<11, 2>(w, u, smem, s_phase, setup); break;
        case 11 * 4 + 3: ok = run_unit<11, 3>(w, u, smem, s_phase, setup); break;
        case 12 * 4 + 0: ok = run_unit<12, 0>(w, u, smem, s_phase, setup); break;
        case 12 * 4 + 1: ok = run_unit<12, 1>(w, u, smem, s_phase, setup); break;
        case 12 * 4 + 2: ok = run_unit<12, 2>(w, u, smem, s_phase, setup); break;
        case 12 * 4 + 3: ok = run_unit<12, 3>(w, u, smem, s_phase, setup); break;
        case 13 * 4 + 0: ok = run_unit<13, 0>(w, u, smem, s_phase, setup); break;
        case 13 * 4 + 1: ok = run_unit<13, 1>(w, u, smem, s_phase, setup); break;
        case 13 * 4 + 2: ok = run_unit<13, 2>(w, u, smem, s_phase, setup); break;
        case 13 * 4 + 3: ok = run_unit<13, 3>(w, u, smem, s_phase, setup); break;
        case 14 * 4 + 0: ok = run_unit<14, 0>(w, u, smem, s_phase, setup); break;
        case 14 * 4 + 1: ok = run_unit<14, 1>(w, u, smem, s_phase, setup); break;
        case 14 * 4 + 2: ok = run_unit<14, 2>(w, u, smem, s_phase, setup); break;
        case 14 * 4 + 3: ok = run_unit<14, 3>(w, u, smem, s_phase, setup); break;
        default: break;
        }
        prev_key = key;
        // gates sync on their own barriers inside a unit: agree on the outcome CTA-wide
        const bool all_ok = __syncthreads_and(ok) != 0;
        if (threadIdx.x == 0) {
            // every gate-group slot of this shape completed one phase per IPP of the unit
            const int G = isr::kThreads / (1 << (w.log2n - 5));
            const int p0 = u.cy * w.a.chunk_len;
            const int n = min(p0 + w.a.chunk_len, w.a.n_ipp) - p0;
            for (int g = 0; g < G; ++g) s_phase[g] += (uint32_t)n;
        }
        if (!all_ok) break;   // a wait ran out: the status word is set, stop pulling work
    }
}

struct RedSeg {
    const float* part;
    float* out;
    int64_t n;
    int chunks;
};

// out[i] = sum_c part[c][i], FP32 with Kahan compensation (error ~2 ulp for any chunk count);
// one window per blockIdx.y
__global__ void batch_reduce_kernel(const RedSeg* __restrict__ segs)
{
    const RedSeg s = segs[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x) {
        float sum = 0.f, comp = 0.f;
        for (int c = 0; c < s.chunks; ++c) {
            const float y = s.part[(int64_t)c * s.n + i] - comp;
            const float t = sum + y;
            comp = (t - sum) - y;
            sum = t;
        }
        s.out[i] = (float)((double)sum - (double)comp);
    }
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

#define B_TRY(expr)                                                                                     \
    do {                                                                                                \
        cudaError_t e_ = (expr);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return fail(e_ == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, "%s: %s", #expr, \
                        cudaGetErrorString(e_));                                                        \
    } while (0)

}  // namespace

struct isr_batch {
    int dev = 0, sm_count = 0, flags = 0;
    cudaStream_t user_stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::vector<isr_window> w;
    std::vector<BatchWin> hw;
    std::vector<BatchUnit> hu;
    BatchWin* d_wins = nullptr;
    BatchUnit* d_units = nullptr;
    RedSeg* d_segs = nullptr;
    float* partial = nullptr;
    int* counter = nullptr;
    int* status = nullptr;
    int order[4] = {0, 0, 0, 0};
    float tune_ms[4][4] = {};
    int64_t transforms = 0;
    int64_t max_bins = 0;   // largest window's n_ranges x nfft
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// unit list of the chosen windows (all if only < 0), longest work first
void build_units(isr_batch* b, int only_log2n, std::vector<BatchUnit>& out)
{
    out.clear();
    for (int i = 0; i < (int)b->hw.size(); ++i) {
        const BatchWin& w = b->hw[i];
        if (only_log2n >= 0 && w.log2n != only_log2n) continue;
        for (int c = 0; c < w.n_cy; ++c)
            for (int g = 0; g < w.n_gx; ++g) out.push_back(BatchUnit{i, g, c, 0});
    }
    auto cost = [&](const BatchUnit& u) {
        const BatchWin& w = b->hw[u.win];
        const int p0 = u.cy * w.a.chunk_len;
        const int n = std::min(p0 + w.a.chunk_len, w.a.n_ipp) - p0;
        return (double)n * w.log2n;   // 16384 points per CTA per IPP for every shape
    };
    std::stable_sort(out.begin(), out.end(), [&](const BatchUnit& x, const BatchUnit& y) { return cost(x) > cost(y); });
}

isr_status upload(isr_batch* b, const std::vector<BatchUnit>& units, cudaStream_t s)
{
    B_TRY(cudaMemcpyAsync(b->d_wins, b->hw.data(), sizeof(BatchWin) * b->hw.size(), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemcpyAsync(b->d_units, units.data(), sizeof(BatchUnit) * units.size(), cudaMemcpyHostToDevice, s));
    return ISR_OK;
}

isr_status enqueue(isr_batch* b, int n_units, bool reduce, cudaStream_t s)
{
    B_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), s));
    batch_kernel<<<b->sm_count, isr::kThreads, kBatchSmem, s>>>(b->d_wins, b->d_units, n_units, b->counter);
    B_TRY(cudaGetLastError());
    if (reduce) {
        // memory-bound: about four waves of 256-thread CTAs over all windows (8 per SM resident),
        // at most one CTA per 256 elements of the largest window
        const int64_t want = (4 * 8 * (int64_t)b->sm_count + (int64_t)b->w.size() - 1) / (int64_t)b->w.size();
        const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(want, (b->max_bins + 255) / 256));
        batch_reduce_kernel<<<dim3((unsigned)gx, (unsigned)b->w.size()), 256, 0, s>>>(b->d_segs);
        B_TRY(cudaGetLastError());
    }
    return ISR_OK;
}

isr_status autotune(isr_batch* b)
{
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    std::vector<BatchUnit> units;
    for (int L = kMinLog2; L <= kMaxLog2; ++L) {
        bool used = false;
        for (auto& w : b->hw) used |= w.log2n == L;
        if (!used) continue;
        float best = 1e30f;
        int best_o = 0;
        bool forced = false;
        for (size_t i = 0; i < b->hw.size(); ++i) forced |= b->hw[i].log2n == L && b->w[i].order >= 0;
        if (forced) continue;
        for (int o = 0; o < isr::kOrders; ++o) {
            for (auto& w : b->hw)
                if (w.log2n == L) w.order = o;
            build_units(b, L, units);
            // a probe of a few waves is enough to rank the orders
            units.resize(std::min<size_t>(units.size(), (size_t)b->sm_count * 3));
            isr_status st = upload(b, units, b->cap_stream);
            if (st != ISR_OK) return st;
            st = enqueue(b, (int)units.size(), false, b->cap_stream);   // warm-up
            if (st != ISR_OK) return st;
            B_TRY(cudaEventRecord(e0, b->cap_stream));
            st = enqueue(b, (int)units.size(), false, b->cap_stream);
            if (st != ISR_OK) return st;
            B_TRY(cudaEventRecord(e1, b->cap_stream));
            B_TRY(cudaEventSynchronize(e1));
            float ms = 0;
            B_TRY(cudaEventElapsedTime(&ms, e0, e1));
            b->tune_ms[L - kMinLog2][o] = ms;
            if (ms < best) {
                best = ms;
                best_o = o;
            }
        }
        b->order[L - kMinLog2] = best_o;
        for (auto& w : b->hw)
            if (w.log2n == L) w.order = best_o;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ISR_OK;
}

}  // namespace

extern "C" {

isr_status isr_batch_create(isr_batch** out, const isr_window* windows, int32_t n_windows, int32_t flags,
                            int32_t device, void* stream)
{
    isr::clear_error();
    if (!out) return fail(ISR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!windows || n_windows < 1 || n_windows > 65535) return fail(ISR_ERR_INVALID_ARG, "need 1..65535 windows");
    if (flags & ~(ISR_BATCH_GRAPH | ISR_BATCH_AUTOTUNE)) return fail(ISR_ERR_INVALID_ARG, "unknown flags");
    for (int i = 0; i < n_windows; ++i) {
        const isr_window& w = windows[i];
        if (w.nfft < 2048 || w.nfft > 16384 || (w.nfft & (w.nfft - 1)))
            return fail(ISR_ERR_UNSUPPORTED, "window %d: nfft %d not in {2048, 4096, 8192, 16384}", i, w.nfft);
        if (w.code_len < 1 || w.code_len > w.nfft || w.n_ranges < 1 || w.n_ipp < 1 || w.range_start < 0 ||
            w.range_step < 1 || w.echo_stride % 4 || w.echo_stride < 4 || w.tx_stride < 0 || w.order < -1 ||
            w.order >= isr::kOrders ||
            (w.tx_stride > 0 && w.tx_stride < w.code_len))
            return fail(ISR_ERR_INVALID_ARG, "window %d: bad geometry", i);
        if ((int64_t)w.range_start + (int64_t)(w.n_ranges - 1) * w.range_step + w.code_len > w.echo_stride)
            return fail(ISR_ERR_OUT_OF_RANGE, "window %d: last gate runs past the echo row", i);
        if (!w.echo || !w.tx_code || !w.out || reinterpret_cast<uintptr_t>(w.echo) % 16)
            return fail(ISR_ERR_INVALID_ARG, "window %d: NULL or misaligned buffer", i);
        if (!dev_ptr(w.echo) || !dev_ptr(w.tx_code) || !dev_ptr(w.out))
            return fail(ISR_ERR_INVALID_ARG, "window %d: buffers must be device memory", i);
    }
    int dev = device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(ISR_ERR_CUDA, "no current device");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    isr_batch* b = new (std::nothrow) isr_batch();
    if (!b) return fail(ISR_ERR_NO_MEMORY, "host allocation failed");
    auto bail = [&](isr_status s) {
        isr_batch_destroy(b);
        if (prev >= 0) cudaSetDevice(prev);
        return s;
    };
    b->dev = dev;
    b->flags = flags;
    b->user_stream = static_cast<cudaStream_t>(stream);
    b->w.assign(windows, windows + n_windows);
    if (cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bail(fail(ISR_ERR_CUDA, "device query failed"));
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem);
    if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(ISR_ERR_CUDA, "stream creation failed"));

    // chunking and scratch layout
    int64_t part_floats = 0;
    std::vector<int64_t> part_off(n_windows);
    for (int i = 0; i < n_windows; ++i) {
        const isr_window& w = windows[i];
        int lg = 0;
        while ((1 << lg) < w.nfft) ++lg;
        BatchWin bw{};
        const int G = isr::kThreads / (w.nfft / 32);
        bw.log2n = lg;
        bw.order = w.order >= 0 ? w.order : 0;
        bw.n_gx = (w.n_ranges + G - 1) / G;
        const int chunk = std::min(kChunk, w.n_ipp);
        bw.n_cy = (w.n_ipp + chunk - 1) / chunk;
        bw.a.echo = reinterpret_cast<const uint32_t*>(w.echo);
        bw.a.echo_stride = w.echo_stride;
        bw.a.tx = w.tx_code;
        bw.a.tx_stride = w.tx_stride;
        bw.a.n_ranges = w.n_ranges;
        bw.a.range_start = w.range_start;
        bw.a.range_step = w.range_step;
        bw.a.code_len = w.code_len;
        bw.a.n_ipp = w.n_ipp;
        bw.a.chunk_len = chunk;
        bw.a.wait_limit = kWaitLimit;
        bw.a.drop_ipp = -1;
        part_off[i] = part_floats;
        part_floats += (int64_t)bw.n_cy * w.n_ranges * w.nfft;
        b->hw.push_back(bw);
        b->transforms += (int64_t)w.n_ranges * w.n_ipp;
        b->max_bins = std::max<int64_t>(b->max_bins, (int64_t)w.n_ranges * w.nfft);
    }
    e = cudaMalloc(&b->partial, sizeof(float) * part_floats);
    if (e == cudaSuccess) e = cudaMalloc(&b->counter, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_wins, sizeof(BatchWin) * n_windows);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_segs, sizeof(RedSeg) * n_windows);
    int64_t max_units = 0;
    for (auto& bw : b->hw) max_units += (int64_t)bw.n_gx * bw.n_cy;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_units, sizeof(BatchUnit) * max_units);
    if (e != cudaSuccess)
        return bail(fail(e == cudaErrorMemoryAllocation ? ISR_ERR_NO_MEMORY : ISR_ERR_CUDA, "allocation failed: %s",
                         cudaGetErrorString(e)));
    std::vector<RedSeg> segs(n_windows);
    for (int i = 0; i < n_windows; ++i) {
        b->hw[i].a.partial = b->partial + part_off[i];
        b->hw[i].a.status = b->status;
        segs[i] = RedSeg{b->partial + part_off[i], windows[i].out, (int64_t)windows[i].n_ranges * windows[i].nfft,
                         b->hw[i].n_cy};
    }
    e = cudaMemcpy(b->d_segs, segs.data(), sizeof(RedSeg) * n_windows, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, sizeof(int));
    if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "upload failed: %s", cudaGetErrorString(e)));

    isr_status st = ISR_OK;
    if (flags & ISR_BATCH_AUTOTUNE) st = autotune(b);
    if (st != ISR_OK) return bail(st);
    build_units(b, -1, b->hu);
    st = upload(b, b->hu, b->cap_stream);
    if (st == ISR_OK && cudaStreamSynchronize(b->cap_stream) != cudaSuccess) st = fail(ISR_ERR_CUDA, "upload failed");
    if (st != ISR_OK) return bail(st);
    if (flags & ISR_BATCH_GRAPH) {
        e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e)));
        st = enqueue(b, (int)b->hu.size(), true, b->cap_stream);
        e = cudaStreamEndCapture(b->cap_stream, &b->graph);
        if (st != ISR_OK) return bail(st);
        if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "end capture: %s", cudaGetErrorString(e)));
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) return bail(fail(ISR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)));
    }
    if (prev >= 0) cudaSetDevice(prev);
    *out = b;
    return ISR_OK;
}

isr_status isr_batch_run(isr_batch* b)
{
    isr::clear_error();
    if (!b) return fail(ISR_ERR_INVALID_ARG, "batch is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->dev);
    isr_status st = ISR_OK;
    if (b->exec) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->user_stream);
        if (e != cudaSuccess) st = fail(ISR_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    } else {
        st = enqueue(b, (int)b->hu.size(), true, b->user_stream);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

isr_status isr_batch_wait(isr_batch* b)
{
    if (!b) return fail(ISR_ERR_INVALID_ARG, "batch is NULL");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->dev);
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->user_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user_stream);
    if (e == cudaSuccess && status) e = cudaMemsetAsync(b->status, 0, sizeof(int), b->user_stream);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return fail(ISR_ERR_CUDA, "isr_batch_wait: %s", cudaGetErrorString(e));
    if (status & 2)
        return fail(ISR_ERR_OUT_OF_RANGE, "a batched unit found a gate window outside its echo row (debug build check)");
    if (status) return fail(ISR_ERR_TIMEOUT, "a batched unit timed out waiting for its staged window");
    return ISR_OK;
}

isr_status isr_batch_query(const isr_batch* b, isr_batch_info* info)
{
    if (!b || !info) return fail(ISR_ERR_INVALID_ARG, "NULL argument");
    info->n_windows = (int32_t)b->w.size();
    info->graph = b->exec != nullptr;
    info->n_units = (int64_t)b->hu.size();
    info->transforms = b->transforms;
    for (int i = 0; i < 4; ++i) {
        info->order[i] = b->order[i];
        for (int o = 0; o < 4; ++o) info->tune_ms[i][o] = b->tune_ms[i][o];
    }
    return ISR_OK;
}

void isr_batch_destroy(isr_batch* b)
{
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->dev);
    if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    cudaStreamSynchronize(b->user_stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->partial);
    cudaFree(b->counter);
    cudaFree(b->status);
    cudaFree(b->d_wins);
    cudaFree(b->d_units);
    cudaFree(b->d_segs);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
}

}  // extern "C"
