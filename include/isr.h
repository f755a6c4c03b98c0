/*
 * isr.h -- C ABI of the GB300 plasma-line spectrum integrator.
 *
 * Operation (Hilliard, Vierinen & Erickson, "GPGPU Acceleration of Incoherent Scatter
 * Radar Plasma Line Analysis", Sec. 2.2 Eqs. 7-8 and Sec. 3.2): for every inter-pulse
 * period (IPP) p and every range gate r, with window start s_r = start + r * step,
 *
 *     x[k]    = conj(eps_p[k]) * m_p[s_r + k]          (k < code_len; zero up to nfft)
 *     X[f]    = sum_k x[k] exp(-2 pi i f k / nfft)     (forward, unnormalised, bins 0..nfft-1)
 *     A[r][f] += |X[f]|^2                              (sum over IPPs)
 *
 * The decode multiply, the transform and the power accumulation run fused in one kernel
 * on the GPU; decoded batches never leave the SM.  All calls return an isr_status; on
 * failure isr_last_error() gives a one-line reason (per calling thread).  No C++
 * exception crosses this interface.  Device pointers are plain CUDA device addresses
 * (for example torch tensor data_ptr()); streams are cudaStream_t passed as void*.
 */
#ifndef ISR_H
#define ISR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ISR_OK = 0,
    ISR_ERR_INVALID_ARG = 1,  /* NULL pointer, bad size, misaligned buffer, n_ipp < 0 ...   */
    ISR_ERR_UNSUPPORTED = 2,  /* nfft not a power of two in [8, 16384], unknown tx type     */
    ISR_ERR_OUT_OF_RANGE = 3, /* a gate's window runs past the end of an echo row           */
    ISR_ERR_NO_MEMORY = 4,    /* device or host allocation failed                            */
    ISR_ERR_CUDA = 5,         /* a CUDA call or kernel launch failed (see isr_last_error)    */
    ISR_ERR_TIMEOUT = 6       /* a kernel gave up waiting for its staged input; the result
                                 of that integration is incomplete                          */
} isr_status;

/* Transmit-code chip formats. */
typedef enum {
    ISR_TX_CI16 = 0, /* complex int16: interleaved (I, Q), 4 bytes per chip             */
    ISR_TX_C32 = 1,  /* complex float: interleaved (re, im), 8 bytes per chip           */
    ISR_TX_PM1 = 2   /* binary phase: one int8 per chip, -1 where negative, else +1     */
} isr_tx_type;

/* Plan description.  Geometry is fixed for the life of a plan. */
typedef struct {
    int32_t nfft;        /* transform length: power of two, 8 <= nfft <= 16384 (Sec. 3.2.2) */
    int32_t code_len;    /* chips per code, 1 <= code_len <= nfft; the window is zero-padded */
    int32_t n_ranges;    /* R range gates, >= 1                                               */
    int32_t range_start; /* s_0 in samples, >= 0                                              */
    int32_t range_step;  /* gate spacing in samples, >= 1 (Sec. 4: 25)                        */
    int32_t tx_type;     /* isr_tx_type                                                       */
    int64_t echo_stride; /* complex samples per echo row (IPP); multiple of 4                 */
    int64_t tx_stride;   /* chips between per-IPP code rows; 0 = one code for every IPP       */
    int32_t ipp_chunk;   /* max IPPs summed in FP32 before the FP64 reduction; 0 = 256        */
    int32_t max_chunks;  /* IPP chunks in flight per launch (scratch = max_chunks * R * nfft
                            floats); 0 = automatic (<= 64, <= 4 GiB)                          */
    int32_t device;      /* CUDA device ordinal; -1 = the calling thread's current device     */
    int32_t flags;       /* reserved, must be 0                                               */
    void* stream;        /* cudaStream_t for all work of this plan; NULL = legacy default     */
} isr_plan_desc;

/* Optional per-call gate geometry (overrides the plan's start and step for one call). */
typedef struct {
    int32_t start;
    int32_t step;
    int32_t count; /* must equal the plan's n_ranges */
} isr_ranges;

/* Flags of isr_spectra. */
#define ISR_RESET_AFTER 1 /* zero the accumulators (and the IPP count) after reading them */
#define ISR_MEAN 2        /* divide by the number of integrated IPPs (Eq. 8's mean)       */

/* Read-only plan facts, for callers that size buffers or report launch shapes. */
typedef struct {
    int32_t nfft;
    int32_t n_ranges;
    int32_t ranges_per_cta;    /* gates one CTA transforms side by side */
    int32_t threads_per_cta;
    int32_t smem_bytes;        /* dynamic shared memory per CTA */
    int32_t max_chunks;
    int32_t ipp_chunk;
    int32_t sm_count;
    int64_t n_ipp_integrated;  /* IPPs summed since creation or the last reset */
    int64_t kernel_launches;   /* fused-kernel launches since creation */
    double kernel_ms;          /* summed fused-kernel time of timed launches (profiling) */
    int64_t kernel_timed;      /* launches counted in kernel_ms */
    int64_t host_block_growth; /* growth of the host-input blocks the last call with host rows
                                  beyond one staging buffer measured (1..4; 0: no such call) */
} isr_plan_info;

typedef struct isr_plan isr_plan;

/*
 * Create a plan: validates the description and allocates, on the plan's device, the
 * persistent [n_ranges][nfft] accumulators (FP64, zeroed) and the IPP-chunk scratch.
 * The plan owns that memory until isr_destroy.  On failure *out is set to NULL.
 * Errors: ISR_ERR_INVALID_ARG, ISR_ERR_UNSUPPORTED, ISR_ERR_OUT_OF_RANGE (the last gate's
 * window, range_start + (n_ranges-1)*range_step + code_len, exceeds echo_stride),
 * ISR_ERR_NO_MEMORY, ISR_ERR_CUDA.
 */
isr_status isr_plan_create(isr_plan** out, const isr_plan_desc* desc);

/*
 * Add n_ipp IPPs to the plan's accumulators (Eqs. 7-8; the paper's kernel pipeline of
 * Sec. 3.2 fused into one launch).  Repeated calls continue one integration.
 *   echo    : int16 [n_ipp][echo_stride][2] (I, Q), 16-byte aligned.  Device memory: the
 *             call is asynchronous on the plan's stream and the caller keeps echo and
 *             tx_code alive until the stream passes.  Host memory (pageable or pinned):
 *             the call streams the rows to the GPU through plan-owned staging buffers,
 *             overlapping copies with the kernels, and returns when the host buffers
 *             may be reused.
 *   tx_code : the code(s) in the plan's tx_type, [1 or n_ipp rows] with row p at
 *             p * tx_stride chips; same memory kind rules as echo.
 *   ranges  : NULL = the plan's (range_start, range_step); else that geometry for this
 *             call (count must equal n_ranges; window bounds are re-checked).
 *   nfft    : must equal the plan's nfft (guards against mixing plans).
 * n_ipp == 0 is a no-op.  Arguments are checked on the host before anything is
 * launched.  Errors: ISR_ERR_INVALID_ARG, ISR_ERR_OUT_OF_RANGE, ISR_ERR_NO_MEMORY,
 * ISR_ERR_CUDA.
 */
isr_status isr_integrate(isr_plan* plan, const int16_t* echo, const void* tx_code, int32_t n_ipp,
                         const isr_ranges* ranges, int32_t nfft);

/*
 * Synchronise the plan's stream and copy the [n_ranges][nfft] spectra, as float, to out
 * (device or host memory, caller-owned).  flags: ISR_MEAN divides by the IPP count
 * (no-op when it is 0), ISR_RESET_AFTER zeroes the accumulators afterwards.
 * *n_ipp_out (optional) receives the number of IPPs integrated.  Returns
 * ISR_ERR_TIMEOUT if any kernel since the last call reported a timed-out wait.
 */
isr_status isr_spectra(isr_plan* plan, float* out, int32_t flags, int64_t* n_ipp_out);

/* Fill *info with the plan's launch shape and counters.  Does not synchronise. */
isr_status isr_plan_query(const isr_plan* plan, isr_plan_info* info);

/* Turn per-launch CUDA-event timing of the fused kernel on (1) or off (0). */
isr_status isr_plan_set_profiling(isr_plan* plan, int32_t enable);

/* Tracing, debug build only (-DISR_DEBUG): the Stockham fused kernels (every nfft; at nfft 16384
 * radix orders 0-2 and 6-8) time the phases of their IPP loop with the SM clock, as seen by
 * thread 0 of each CTA, and add them up over all CTAs and launches of the plan:
 *   out[0] waiting for the staged window + the first barrier, out[1] pass 0 (decode, first DFT,
 *   exchange stores), out[2] the middle pass, out[3] the last pass (DFT, |X|^2 accumulation),
 *   out[4] the IPPs those CTAs processed (so out[i] / out[4] = cycles per IPP of one CTA).
 * Synchronises the plan's stream.  The release build records nothing and returns
 * ISR_ERR_UNSUPPORTED.  Errors: ISR_ERR_INVALID_ARG (NULL), ISR_ERR_UNSUPPORTED, ISR_ERR_CUDA. */
isr_status isr_plan_phase_cycles(isr_plan* plan, uint64_t out[5]);

/* Bound of every wait on a staged echo window, in mbarrier polls (default 2^22, on the
 * order of a second).  A wait that runs out makes the kernel stop, record the failure
 * and return; the next isr_spectra reports ISR_ERR_TIMEOUT.  polls must be > 0. */
isr_status isr_plan_set_wait_limit(isr_plan* plan, uint32_t polls);

/* Radix order (0..9) of the kernel used for binary-phase codes with code_len == nfft, for
 * nfft >= 2048 (smaller sizes have one order): 0..2 are three-pass Stockham orders, 3 is a
 * radix-(nfft/1024) decimation-in-frequency pass followed by one 1024-point transform per
 * warp; 4 and 5 (nfft 16384 only) use paired FP32 instructions (two operations each):
 * 4 the passes [4, 16, 16, 16] with each thread transforming two butterflies at once,
 * 5 the passes [16, 32, 32] of order 1 with two butterflies per thread in the first pass
 * and each radix-32 butterfly split into two paired 16-point halves; 6, 7 and 8 (nfft
 * 16384 only) are orders 0, 1 and 2 with every thread's inter-pass twiddles computed once
 * per CTA into tensor memory (all 512 columns of the SM's TMEM, freed when the CTA ends)
 * instead of being formed from tables and recurrences in every IPP; 9 (nfft 16384 only) is
 * order 3 with its twiddles in tensor memory likewise and unit-stride first-pass columns.
 * Every order gives the same spectra up to FP32 rounding; they differ in speed, so a caller (or the
 * binding's autotuner) may time them and keep the fastest.  Default 0. */
isr_status isr_plan_set_order(isr_plan* plan, int32_t order);

/* Engine of the first FFT pass.  ISR_PREC_FP32 (default): SIMT FP32 everywhere.  The
 * tensor-core modes (nfft 16384, ISR_TX_PM1, code_len == nfft) compute the first pass
 * (radix 16 over the window, then radix 32, 32 on the SIMT pipe) as a DFT-matrix GEMM on
 * the tensor cores with FP32 accumulation: *_SPLIT modes use hi + lo operand splits
 * (A_hi B_hi + A_hi B_lo + A_lo B_hi) in BF16 or FP16, the others a single BF16 or FP16
 * product.  ISR_PREC_TC_* issue the warp-level mma.sync instruction with register
 * fragments; ISR_PREC_TC05_* issue tcgen05.mma from one thread with both operands in shared
 * memory (decoded samples split once into K-major operand tiles) and the FP32 accumulator
 * in tensor memory (256 columns per CTA, freed when the CTA ends).  Accumulation over IPPs
 * stays FP32 per chunk and FP64 across chunks. */
#define ISR_PREC_FP32 0
#define ISR_PREC_TC_BF16_SPLIT 1
#define ISR_PREC_TC_FP16_SPLIT 2
#define ISR_PREC_TC_BF16 3
#define ISR_PREC_TC_FP16 4
#define ISR_PREC_TC05_BF16_SPLIT 5
#define ISR_PREC_TC05_FP16_SPLIT 6
#define ISR_PREC_TC05_BF16 7
#define ISR_PREC_TC05_FP16 8
isr_status isr_plan_set_precision(isr_plan* plan, int32_t precision);

/* Test hook: the kernels of the following isr_integrate calls never stage the window of
 * IPP `ipp` (counted from the first IPP of each call; -1 turns the hook off), so its wait
 * runs out and exercises the timeout path above without any fault. */
isr_status isr_plan_test_drop_window(isr_plan* plan, int32_t ipp);

/*
 * Allocation-free integration (the paper has no counterpart; this serves callers that
 * cannot allocate device memory, for example a real-time pipeline that reserves all of
 * its GPU memory at start-up, or a process whose device memory belongs to another
 * allocator such as a framework's caching allocator, where a cudaMalloc could fail or
 * stall).  It computes, for the geometry in *desc, the sum over n_ipp IPPs of the same
 * power spectra as a plan would (Eqs. 7-8), writing float [n_ranges][nfft] to `out`.
 * echo, tx_code and out are caller-owned DEVICE buffers (echo 16-byte aligned); desc's
 * ipp_chunk and max_chunks are ignored.  The IPP-chunk partial sums live in one
 * file-scope device array of ISR_STATIC_SCRATCH_FLOATS floats (16 MiB) that every GPU
 * which loads this library keeps until the process exits; n_ranges * nfft must not
 * exceed it (ISR_ERR_INVALID_ARG otherwise).  Nothing is allocated: no cudaMalloc, no
 * cudaFree, no allocating library routine.  As in a plan, every FP32 partial sums at
 * most 256 IPPs; the array holds C = min(65535, ISR_STATIC_SCRATCH_FLOATS / (n_ranges *
 * nfft)) of them, so the IPPs run in blocks of at most C * 256 (one fused launch and one
 * reduction each).  The first block's reduction writes `out`; each later block adds its
 * sum (formed in double) to `out` with one FP32 rounding, so a call of B blocks carries at
 * most B extra roundings of 2^-24 relative per bin (B = 1 whenever n_ipp <= C * 256).
 * The first call on a device looks up the array's device address (once per device, with
 * that device current), so make that first call before any stream capture.  Every call
 * shares the array and its contents stay from the last call: calls that overlap on the
 * GPU (other host threads or other streams) race and corrupt each other's results.  The
 * call is synchronous: it enqueues its work on desc->stream and then waits for that
 * stream (so it can report ISR_ERR_TIMEOUT from a bounded wait that ran out); a stream
 * that is being captured does not allow that wait, so no call belongs inside a capture.
 */
#define ISR_STATIC_SCRATCH_FLOATS (4 * 1024 * 1024)
isr_status isr_integrate_static(const isr_plan_desc* desc, const int16_t* echo, const void* tx_code,
                                int32_t n_ipp, float* out);

/*
 * Plasma-line position per gate by spectral peak fit (the line frequency gives the
 * electron density through Eq. 1).  spectra: device float [n_ranges][nfft] (a sum or
 * mean from isr_spectra).  For each gate r, within bins [band_lo, band_hi):
 *   b      = the largest bin (lowest index on ties, compared in float),
 *   delta  = 0.5 (y[b-1] - y[b+1]) / (y[b-1] - 2 y[b] + y[b+1]) with y = ln P in double
 *            (neighbours taken modulo nfft; 0 unless the parabola opens downwards and all
 *            three powers are positive; clamped to [-0.5, 0.5]),
 *   freq_bin[r] = b + delta   (double; Hz = freq_bin * fs / nfft, negative frequencies
 *                              are bins above nfft/2),
 *   snr[r]      = P[b] / mean of P over the band (float).
 * freq_bin and snr are device arrays of n_ranges.  Stream-ordered on `stream`, asynchronous.
 */
isr_status isr_peak_fit(const float* spectra, int32_t n_ranges, int32_t nfft, int32_t band_lo, int32_t band_hi,
                        double* freq_bin, float* snr, void* stream);

/*
 * Measured FP32 fused multiply-add throughput of `device`: the denominator of the integrate
 * kernel's roofline (the kernel is bound by the FP32 SIMT pipe, whose nominal rate is SMs x 128
 * lanes x 2 FLOP x SM clock).  An FMA-only kernel (8 independent dependency chains per thread,
 * 4 CTAs of 256 threads per SM) runs 4 times on an internal stream; the best of runs 2-4 is
 * reported.  paired = 0 issues FFMA (one FMA per lane and instruction), paired = 1 FFMA2 (two
 * per lane and instruction).  Writes *tflops (2 FLOP per FMA) and *ms (duration of the best
 * run).  Blocking; allocates 4 bytes of device memory for the duration of the call.  The paper
 * has no counterpart.  Errors: ISR_ERR_INVALID_ARG (NULL output, paired not 0/1; checked before
 * any CUDA call), ISR_ERR_CUDA.
 */
isr_status isr_fp32_peak(int32_t device, int32_t paired, double* tflops, double* ms);

/*
 * Measured tcgen05 tensor-pipe rate of `device` for one MMA shape: kind::f16 (BF16 operands read
 * from shared memory, FP32 accumulator in tensor memory), M = 128, K = 16 and N = n (32, 64, 128
 * or 256).  One thread per CTA issues 4096 MMAs back to back, one CTA per SM; 3 runs on an
 * internal stream, the best of runs 2-3 reported.  Writes *tflops (2 FLOP per multiply-add over
 * all SMs) and *cycles_per_mma (SM clock cycles per MMA, mean over the CTAs).  The learned
 * estimator's convolutions issue N = 32 and N = 64 MMAs, so this is their tensor roofline.
 * Blocking; allocates a few bytes of device memory for the duration of the call.  The paper has
 * no counterpart.  Errors: ISR_ERR_INVALID_ARG (NULL output, n not one of the four; checked
 * before any CUDA call), ISR_ERR_CUDA, ISR_ERR_TIMEOUT (an MMA commit did not complete within the
 * bounded wait).
 */
isr_status isr_tc05_rate(int32_t device, int32_t n, double* tflops, double* cycles_per_mma);

/*
 * Learned plasma-line estimator (the network maps an integrated spectrum to the line's
 * position and presence; Eq. 1 links that position to the electron density).  Network:
 * four 9-tap, 32-channel 1-D convolutions with ReLU over the band's standardised log
 * power, location logits by a 1x1 convolution, presence by an MLP on the per-channel max
 * and mean; parameters as a flat float vector of ISR_EST_N_PARAMS in the order
 * W1[32][1][9] b1[32] W2[32][32][9] b2 W3 b3 W4 b4 w5[32] b5[1] Wa[32][64] ba[32] wb[32] bb[1].
 * Training keeps FP32 master weights and Adam moments; activations and working weights
 * use `precision` (ISR_EST_FP32 or one of the BF16 values below) with FP32 accumulation.
 * With BF16 storage the 32-channel convolutions (forward, backward-data, weight gradient) run
 * on the tensor cores, as tcgen05.mma GEMMs (one thread issues them, the accumulators live in
 * tensor memory) or as warp-level mma.sync, per the constants below;
 * the FP32 gradient entering the backward passes is split into two BF16 parts (~16
 * significant bits) for them.  All array arguments are device memory except where noted;
 * calls are ordered on `stream`.
 */
#define ISR_EST_N_PARAMS 30210
#define ISR_EST_FP32 0
#define ISR_EST_BF16 1         /* BF16 storage, the 32-channel convolutions on tcgen05 (TMEM accumulators) */
#define ISR_EST_BF16_MMASYNC 2 /* BF16 storage, the same convolutions on the warp-level mma.sync path */
typedef struct isr_est isr_est;

/* Estimator for spectra of nfft bins; band [band_lo, band_lo + band_len); batches of up
 * to max_batch gates.  Parameters start at zero: set them with isr_est_set_params. */
isr_status isr_est_create(isr_est** out, int32_t nfft, int32_t band_lo, int32_t band_len, int32_t max_batch,
                          int32_t precision, int32_t device, void* stream);
/* Copy ISR_EST_N_PARAMS floats in (host or device; resets the Adam state) or out. */
isr_status isr_est_set_params(isr_est* est, const float* params);
isr_status isr_est_get_params(isr_est* est, float* params);
/* x[n][band_len] = (ln P - mean) / (std + 1e-6) over the band, from spectra[n][nfft]. */
isr_status isr_est_features(isr_est* est, const float* spectra, int32_t n, float* x);
/* Batch loss and its gradient (no update).  line_bin: true position in bins from band_lo;
 * present: 1 or 0.  loss (one float) and grad (ISR_EST_N_PARAMS floats) may be host or
 * device memory or NULL.  Synchronises the stream. */
isr_status isr_est_grad(isr_est* est, const float* x, int32_t n, const float* line_bin, const float* present,
                        float* loss, float* grad);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the batch; loss (host or device) optional. */
isr_status isr_est_train_step(isr_est* est, const float* x, int32_t n, const float* line_bin, const float* present,
                              float lr, float* loss);
/* line_bin[n]: position in bins of the full spectrum (band_lo + soft-argmax over the 7 bins
 * around the largest location logit); presence[n]: sigmoid of the presence logit. */
isr_status isr_est_predict(isr_est* est, const float* x, int32_t n, float* line_bin, float* presence);
void isr_est_destroy(isr_est* est);

/*
 * Batched integration of many windows of uneven shape in one persistent launch.  Radars
 * integrate several windows at once, e.g. the up- and down-shifted plasma-line channels
 * (the line appears at +-f_r, Sec. 2.1) with different range extents and resolutions.
 * Each window is an independent integration (Eqs. 7-8) with its own echo, code and
 * geometry; isr_batch_run writes, for every window, the sum over its n_ipp IPPs as float
 * [n_ranges][nfft] into its `out`.  All (gate group, IPP chunk) units of all windows
 * form one queue, longest first, served by one CTA per SM.  Buffers are device memory and
 * stay bound to the batch: refill them between runs.  Limits: nfft in {2048, 4096, 8192,
 * 16384}; binary-phase codes (ISR_TX_PM1) only.
 */
typedef struct {
    const int16_t* echo;  /* [n_ipp][echo_stride][2], 16-byte aligned */
    const void* tx_code;  /* int8 chips, [1 or n_ipp rows][tx_stride] */
    float* out;           /* [n_ranges][nfft] sums */
    int64_t echo_stride;  /* multiple of 4 */
    int64_t tx_stride;    /* 0 = one code for every IPP */
    int32_t nfft;
    int32_t code_len;
    int32_t n_ranges;
    int32_t range_start;
    int32_t range_step;
    int32_t n_ipp;
    int32_t order;        /* radix order 0..3 (see isr_plan_set_order), or -1 = default / autotuned */
    int32_t reserved;
} isr_window;

#define ISR_BATCH_GRAPH 1    /* capture launch + reduction in a CUDA graph; runs replay it */
#define ISR_BATCH_AUTOTUNE 2 /* at creation, time the radix orders of each nfft on these windows */

typedef struct {
    int32_t n_windows;
    int32_t graph;          /* 1 if runs replay a captured graph */
    int64_t n_units;        /* work units per run */
    int64_t transforms;     /* gate-IPP transforms per run */
    int32_t order[4];       /* radix order used for nfft 2048, 4096, 8192, 16384 */
    float tune_ms[4][4];    /* probe time of each order (0 if not tuned) */
} isr_batch_info;

typedef struct isr_batch isr_batch;

isr_status isr_batch_create(isr_batch** out, const isr_window* windows, int32_t n_windows, int32_t flags,
                            int32_t device, void* stream);
/* Enqueue one run on the batch's stream (asynchronous). */
isr_status isr_batch_run(isr_batch* batch);
/* Wait for the batch's stream; ISR_ERR_TIMEOUT if a unit's bounded wait ran out. */
isr_status isr_batch_wait(isr_batch* batch);
isr_status isr_batch_query(const isr_batch* batch, isr_batch_info* info);
void isr_batch_destroy(isr_batch* batch);

/* Release the plan and its device memory (synchronises its stream first); NULL is safe. */
void isr_destroy(isr_plan* plan);

/* Reason for the last failed call made by this thread ("" if none). */
const char* isr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ISR_H */
