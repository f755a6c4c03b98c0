"""Thin ctypes binding of ``include/isr.h`` (argument marshalling only).

Every computation happens in ``lib/libisr.so``; this module converts Python arguments
(torch tensors, numpy arrays or raw integer addresses) into the C structs and pointers
the library expects and turns non-zero status codes into ``IsrError``.  There is no
fallback: if the library is missing the import of the binding fails loudly.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# ISR_LIBRARY selects another build of the library (for example lib/libisr_debug.so, whose
# kernels check every staged window against its echo row)
LIB_PATH = os.environ.get("ISR_LIBRARY") or os.path.join(_HERE, "lib", "libisr.so")

ISR_OK = 0
ISR_ERR_INVALID_ARG = 1
ISR_ERR_UNSUPPORTED = 2
ISR_ERR_OUT_OF_RANGE = 3
ISR_ERR_NO_MEMORY = 4
ISR_ERR_CUDA = 5
ISR_ERR_TIMEOUT = 6

ISR_TX_CI16 = 0
ISR_TX_C32 = 1
ISR_TX_PM1 = 2

ISR_RESET_AFTER = 1
ISR_MEAN = 2

STATUS_NAMES = {0: "ISR_OK", 1: "ISR_ERR_INVALID_ARG", 2: "ISR_ERR_UNSUPPORTED", 3: "ISR_ERR_OUT_OF_RANGE",
                4: "ISR_ERR_NO_MEMORY", 5: "ISR_ERR_CUDA", 6: "ISR_ERR_TIMEOUT"}

# every entry point declared in include/isr.h
EXPORTS = ("isr_plan_create", "isr_integrate", "isr_spectra", "isr_plan_query", "isr_plan_set_profiling",
           "isr_plan_set_wait_limit", "isr_plan_set_order", "isr_plan_set_precision", "isr_plan_test_drop_window", "isr_destroy", "isr_last_error",
           "isr_integrate_static", "isr_peak_fit", "isr_fp32_peak", "isr_tc05_rate", "isr_plan_phase_cycles", "isr_est_create", "isr_est_set_params", "isr_est_get_params",
           "isr_est_features", "isr_est_grad", "isr_est_train_step", "isr_est_predict", "isr_est_destroy",
           "isr_batch_create", "isr_batch_run", "isr_batch_wait", "isr_batch_query", "isr_batch_destroy")

# radix orders of isr_plan_set_order (4..8 at nfft 16384 with binary-phase codes only)
N_ORDERS = 10

ISR_PREC_FP32 = 0
ISR_PREC_TC_BF16_SPLIT = 1
ISR_PREC_TC_FP16_SPLIT = 2
ISR_PREC_TC_BF16 = 3
ISR_PREC_TC_FP16 = 4
ISR_PREC_TC05_BF16_SPLIT = 5
ISR_PREC_TC05_FP16_SPLIT = 6
ISR_PREC_TC05_BF16 = 7
ISR_PREC_TC05_FP16 = 8
PRECISION_NAMES = {0: "fp32-simt", 1: "tc-bf16-split", 2: "tc-fp16-split", 3: "tc-bf16", 4: "tc-fp16",
                   5: "tc05-bf16-split", 6: "tc05-fp16-split", 7: "tc05-bf16", 8: "tc05-fp16"}

ISR_BATCH_GRAPH = 1
ISR_BATCH_AUTOTUNE = 2

ISR_EST_N_PARAMS = 30210
ISR_EST_FP32 = 0
ISR_EST_BF16 = 1
ISR_EST_BF16_MMASYNC = 2

# floats of the allocation-free variant's file-scope scratch array
ISR_STATIC_SCRATCH_FLOATS = 4 * 1024 * 1024


class IsrPlanDesc(ctypes.Structure):
    _fields_ = [
        ("nfft", ctypes.c_int32),
        ("code_len", ctypes.c_int32),
        ("n_ranges", ctypes.c_int32),
        ("range_start", ctypes.c_int32),
        ("range_step", ctypes.c_int32),
        ("tx_type", ctypes.c_int32),
        ("echo_stride", ctypes.c_int64),
        ("tx_stride", ctypes.c_int64),
        ("ipp_chunk", ctypes.c_int32),
        ("max_chunks", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class IsrRanges(ctypes.Structure):
    _fields_ = [("start", ctypes.c_int32), ("step", ctypes.c_int32), ("count", ctypes.c_int32)]


class IsrPlanInfo(ctypes.Structure):
    _fields_ = [
        ("nfft", ctypes.c_int32),
        ("n_ranges", ctypes.c_int32),
        ("ranges_per_cta", ctypes.c_int32),
        ("threads_per_cta", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32),
        ("max_chunks", ctypes.c_int32),
        ("ipp_chunk", ctypes.c_int32),
        ("sm_count", ctypes.c_int32),
        ("n_ipp_integrated", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("kernel_ms", ctypes.c_double),
        ("kernel_timed", ctypes.c_int64),
        ("host_block_growth", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IsrWindow(ctypes.Structure):
    _fields_ = [
        ("echo", ctypes.c_void_p),
        ("tx_code", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
        ("echo_stride", ctypes.c_int64),
        ("tx_stride", ctypes.c_int64),
        ("nfft", ctypes.c_int32),
        ("code_len", ctypes.c_int32),
        ("n_ranges", ctypes.c_int32),
        ("range_start", ctypes.c_int32),
        ("range_step", ctypes.c_int32),
        ("n_ipp", ctypes.c_int32),
        ("order", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class IsrBatchInfo(ctypes.Structure):
    _fields_ = [
        ("n_windows", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("n_units", ctypes.c_int64),
        ("transforms", ctypes.c_int64),
        ("order", ctypes.c_int32 * 4),
        ("tune_ms", (ctypes.c_float * 4) * 4),
    ]

    def as_dict(self):
        return {"n_windows": self.n_windows, "graph": bool(self.graph), "n_units": self.n_units,
                "transforms": self.transforms, "order": list(self.order),
                "tune_ms": [list(r) for r in self.tune_ms]}


class IsrError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libisr.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.isr_plan_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(IsrPlanDesc)]
    lib.isr_integrate.argtypes = [P, P, P, ctypes.c_int32, ctypes.POINTER(IsrRanges), ctypes.c_int32]
    lib.isr_spectra.argtypes = [P, P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
    lib.isr_plan_query.argtypes = [P, ctypes.POINTER(IsrPlanInfo)]
    lib.isr_plan_set_profiling.argtypes = [P, ctypes.c_int32]
    lib.isr_plan_set_wait_limit.argtypes = [P, ctypes.c_uint32]
    lib.isr_plan_test_drop_window.argtypes = [P, ctypes.c_int32]
    lib.isr_plan_set_order.argtypes = [P, ctypes.c_int32]
    lib.isr_plan_set_precision.argtypes = [P, ctypes.c_int32]
    lib.isr_integrate_static.argtypes = [ctypes.POINTER(IsrPlanDesc), P, P, ctypes.c_int32, P]
    lib.isr_peak_fit.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P, P]
    lib.isr_fp32_peak.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.isr_tc05_rate.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    lib.isr_plan_phase_cycles.argtypes = [P, P]
    lib.isr_est_create.argtypes = [ctypes.POINTER(P), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_int32, P]
    lib.isr_est_set_params.argtypes = [P, P]
    lib.isr_est_get_params.argtypes = [P, P]
    lib.isr_est_features.argtypes = [P, P, ctypes.c_int32, P]
    lib.isr_est_grad.argtypes = [P, P, ctypes.c_int32, P, P, P, P]
    lib.isr_est_train_step.argtypes = [P, P, ctypes.c_int32, P, P, ctypes.c_float, P]
    lib.isr_est_predict.argtypes = [P, P, ctypes.c_int32, P, P]
    lib.isr_est_destroy.argtypes = [P]
    lib.isr_est_destroy.restype = None
    lib.isr_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(IsrWindow), ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, P]
    lib.isr_batch_run.argtypes = [P]
    lib.isr_batch_wait.argtypes = [P]
    lib.isr_batch_query.argtypes = [P, ctypes.POINTER(IsrBatchInfo)]
    lib.isr_batch_destroy.argtypes = [P]
    lib.isr_batch_destroy.restype = None
    lib.isr_destroy.argtypes = [P]
    lib.isr_destroy.restype = None
    lib.isr_last_error.argtypes = []
    lib.isr_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("isr_destroy", "isr_last_error", "isr_est_destroy", "isr_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != ISR_OK:
        msg = load_library().isr_last_error().decode(errors="replace")
        raise IsrError(status, where, msg)


def _addr(x) -> int | None:
    """Address of a torch tensor, numpy array or integer (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


# ---------------------------------------------------------------- C-named entry points
def isr_plan_create(desc: IsrPlanDesc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().isr_plan_create(ctypes.byref(h), ctypes.byref(desc)), "isr_plan_create")
    return h


def isr_integrate(plan, echo, tx_code, n_ipp: int, ranges: IsrRanges | None, nfft: int) -> None:
    _check(load_library().isr_integrate(plan, _addr(echo), _addr(tx_code), int(n_ipp),
                                        None if ranges is None else ctypes.byref(ranges), int(nfft)),
           "isr_integrate")


def isr_spectra(plan, out, flags: int = 0) -> int:
    n = ctypes.c_int64()
    _check(load_library().isr_spectra(plan, _addr(out), int(flags), ctypes.byref(n)), "isr_spectra")
    return n.value


def isr_plan_query(plan) -> IsrPlanInfo:
    info = IsrPlanInfo()
    _check(load_library().isr_plan_query(plan, ctypes.byref(info)), "isr_plan_query")
    return info


def isr_plan_set_profiling(plan, enable: bool) -> None:
    _check(load_library().isr_plan_set_profiling(plan, 1 if enable else 0), "isr_plan_set_profiling")


def isr_plan_set_wait_limit(plan, polls: int) -> None:
    _check(load_library().isr_plan_set_wait_limit(plan, int(polls)), "isr_plan_set_wait_limit")


def isr_plan_set_order(plan, order: int) -> None:
    _check(load_library().isr_plan_set_order(plan, int(order)), "isr_plan_set_order")


def isr_plan_set_precision(plan, precision: int) -> None:
    _check(load_library().isr_plan_set_precision(plan, int(precision)), "isr_plan_set_precision")


def isr_plan_test_drop_window(plan, ipp: int) -> None:
    _check(load_library().isr_plan_test_drop_window(plan, int(ipp)), "isr_plan_test_drop_window")


def isr_integrate_static(desc: IsrPlanDesc, echo, tx_code, n_ipp: int, out) -> None:
    """Allocation-free integration into ``out`` (device buffers only; synchronous).

    For callers that cannot allocate device memory: the chunk partials live in a fixed
    16 MiB device array inside the library, shared by every call, so calls must not
    overlap on the GPU.  The first call on a device should come before any stream capture.
    """
    _check(load_library().isr_integrate_static(ctypes.byref(desc), _addr(echo), _addr(tx_code), int(n_ipp),
                                               _addr(out)), "isr_integrate_static")


def isr_peak_fit(spectra, n_ranges: int, nfft: int, band_lo: int, band_hi: int, freq_bin, snr,
                 stream=None) -> None:
    _check(load_library().isr_peak_fit(_addr(spectra), int(n_ranges), int(nfft), int(band_lo), int(band_hi),
                                       _addr(freq_bin), _addr(snr), _stream_handle(stream)), "isr_peak_fit")


def isr_fp32_peak(device: int = 0, paired: bool = False) -> tuple:
    """Measured FP32 FMA throughput of the device: (TFLOP/s, ms of the best run)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(load_library().isr_fp32_peak(int(device), int(bool(paired)), ctypes.byref(tf), ctypes.byref(ms)),
           "isr_fp32_peak")
    return tf.value, ms.value


def isr_plan_phase_cycles(plan) -> list:
    """Debug build only: summed SM cycles of the fused kernel's IPP-loop phases (window wait,
    pass 0, middle pass, last pass) as seen by thread 0 of each CTA, and the IPPs counted."""
    out = (ctypes.c_uint64 * 5)()
    _check(load_library().isr_plan_phase_cycles(plan, out), "isr_plan_phase_cycles")
    return [int(v) for v in out]


def isr_tc05_rate(n: int, device: int = 0) -> tuple:
    """Measured tcgen05 rate for BF16 MMAs of shape M = 128, N = n, K = 16 on all SMs:
    (TFLOP/s, SM cycles per MMA)."""
    tf, cyc = ctypes.c_double(), ctypes.c_double()
    _check(load_library().isr_tc05_rate(int(device), int(n), ctypes.byref(tf), ctypes.byref(cyc)), "isr_tc05_rate")
    return tf.value, cyc.value


def isr_est_create(nfft: int, band_lo: int, band_len: int, max_batch: int, precision: int = ISR_EST_BF16,
                   device: int = -1, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().isr_est_create(ctypes.byref(h), int(nfft), int(band_lo), int(band_len), int(max_batch),
                                         int(precision), int(device), _stream_handle(stream)), "isr_est_create")
    return h


def isr_est_set_params(est, params) -> None:
    _check(load_library().isr_est_set_params(est, _addr(params)), "isr_est_set_params")


def isr_est_get_params(est, params) -> None:
    _check(load_library().isr_est_get_params(est, _addr(params)), "isr_est_get_params")


def isr_est_features(est, spectra, n: int, x) -> None:
    _check(load_library().isr_est_features(est, _addr(spectra), int(n), _addr(x)), "isr_est_features")


def isr_est_grad(est, x, n: int, line_bin, present, loss=None, grad=None) -> None:
    _check(load_library().isr_est_grad(est, _addr(x), int(n), _addr(line_bin), _addr(present), _addr(loss),
                                       _addr(grad)), "isr_est_grad")


def isr_est_train_step(est, x, n: int, line_bin, present, lr: float, loss=None) -> None:
    _check(load_library().isr_est_train_step(est, _addr(x), int(n), _addr(line_bin), _addr(present), float(lr),
                                             _addr(loss)), "isr_est_train_step")


def isr_est_predict(est, x, n: int, line_bin, presence) -> None:
    _check(load_library().isr_est_predict(est, _addr(x), int(n), _addr(line_bin), _addr(presence)),
           "isr_est_predict")


def isr_est_destroy(est) -> None:
    load_library().isr_est_destroy(est)


def isr_batch_create(windows, flags: int = 0, device: int = -1, stream=None) -> ctypes.c_void_p:
    arr = (IsrWindow * len(windows))(*windows)
    h = ctypes.c_void_p()
    _check(load_library().isr_batch_create(ctypes.byref(h), arr, len(windows), int(flags), int(device),
                                           _stream_handle(stream)), "isr_batch_create")
    return h


def isr_batch_run(batch) -> None:
    _check(load_library().isr_batch_run(batch), "isr_batch_run")


def isr_batch_wait(batch) -> None:
    _check(load_library().isr_batch_wait(batch), "isr_batch_wait")


def isr_batch_query(batch) -> IsrBatchInfo:
    info = IsrBatchInfo()
    _check(load_library().isr_batch_query(batch, ctypes.byref(info)), "isr_batch_query")
    return info


def isr_batch_destroy(batch) -> None:
    load_library().isr_batch_destroy(batch)


def isr_destroy(plan) -> None:
    load_library().isr_destroy(plan)


def isr_last_error() -> str:
    return load_library().isr_last_error().decode(errors="replace")


# ---------------------------------------------------------------- convenience wrapper
class Plan:
    """Owns one ``isr_plan``; ``integrate`` and ``spectra`` forward to the C calls."""

    def __init__(self, *, nfft: int, n_ranges: int, echo_stride: int, code_len: int | None = None,
                 range_start: int = 0, range_step: int = 25, tx_type: int = ISR_TX_PM1, tx_stride: int = 0,
                 ipp_chunk: int = 0, max_chunks: int = 0, device: int = -1, stream=None):
        d = IsrPlanDesc()
        d.nfft = nfft
        d.code_len = nfft if code_len is None else code_len
        d.n_ranges = n_ranges
        d.range_start = range_start
        d.range_step = range_step
        d.tx_type = tx_type
        d.echo_stride = echo_stride
        d.tx_stride = tx_stride
        d.ipp_chunk = ipp_chunk
        d.max_chunks = max_chunks
        d.device = device
        d.flags = 0
        d.stream = _stream_handle(stream)
        self.desc = d
        self.handle = isr_plan_create(d)

    def integrate(self, echo, tx_code, n_ipp: int, ranges: tuple[int, int] | None = None) -> None:
        rg = None
        if ranges is not None:
            rg = IsrRanges(int(ranges[0]), int(ranges[1]), self.desc.n_ranges)
        isr_integrate(self.handle, echo, tx_code, n_ipp, rg, self.desc.nfft)

    def spectra(self, out=None, flags: int = 0):
        """Copy the spectra into ``out`` (tensor/array, device or host) or a new CPU float32
        torch tensor; returns (out, n_ipp_integrated)."""
        if out is None:
            import torch
            out = torch.empty((self.desc.n_ranges, self.desc.nfft), dtype=torch.float32, pin_memory=False)
        n = isr_spectra(self.handle, out, flags)
        return out, n

    def info(self) -> dict:
        return isr_plan_query(self.handle).as_dict()

    def autotune(self, echo, tx_code, n_ipp: int, reps: int = 2) -> dict:
        """Time the radix orders on ``n_ipp`` IPPs of the caller's data (device buffers) and
        keep the fastest; the accumulators are left as they were.  Returns the times."""
        import torch
        if self.desc.nfft < 2048:
            return {"order": 0, "ms": [0.0]}
        stream = torch.cuda.ExternalStream(self.desc.stream) if self.desc.stream else torch.cuda.current_stream()
        scratch = Plan(nfft=self.desc.nfft, n_ranges=self.desc.n_ranges, echo_stride=self.desc.echo_stride,
                       code_len=self.desc.code_len, range_start=self.desc.range_start, range_step=self.desc.range_step,
                       tx_type=self.desc.tx_type, tx_stride=self.desc.tx_stride, ipp_chunk=self.desc.ipp_chunk,
                       max_chunks=self.desc.max_chunks, device=self.desc.device, stream=self.desc.stream)
        times = []
        try:
            n_orders = N_ORDERS if (self.desc.nfft == 16384 and self.desc.tx_type == ISR_TX_PM1) else 4
            for order in range(n_orders):
                isr_plan_set_order(scratch.handle, order)
                scratch.integrate(echo, tx_code, n_ipp)   # warm-up
                isr_spectra(scratch.handle, None, ISR_RESET_AFTER)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    scratch.integrate(echo, tx_code, n_ipp)
                e1.record(stream)
                isr_spectra(scratch.handle, None, ISR_RESET_AFTER)
                times.append(e0.elapsed_time(e1) / reps)
        finally:
            scratch.close()
        best = int(min(range(len(times)), key=lambda o: times[o]))
        isr_plan_set_order(self.handle, best)
        return {"order": best, "ms": times}

    def set_profiling(self, enable: bool = True) -> None:
        isr_plan_set_profiling(self.handle, enable)

    def close(self) -> None:
        if self.handle:
            isr_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
