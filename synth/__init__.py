"""Seeded synthetic inputs: binary-phase codes and int16 IQ radar echoes.

This module holds no decoding, transform or power arithmetic: only the input model of
the paper's measurement equation (Sec. 2.2, Eqs. 2-3) and the simulated workloads of
Sec. 4 (the paper used SciPy-simulated echoes; these are seeded Philox equivalents).
Both the oracle side (host generator, gcc) and the GPU side (device generator, nvcc)
draw their inputs from here; the two builds are bit-identical (see ``synth_core.h``).

Workloads (sizes from the paper's Sec. 4 and the stated benchmark configurations):

* ``small``     : 64 gates, nfft = code = 1024, 100 IPPs, step 25; noise sigma 1000
                  counts plus one code-modulated tone per gate, frequency uniform in
                  +-0.4 fs, SNR -10 dB per sample.
* ``realistic`` : 1000 gates, nfft = code = 16384, 10,000 IPPs, step 25, 50 MS/s;
                  noise plus a Langmuir line per gate whose frequency follows a Chapman
                  layer (peak 5e11 m^-3 at gate 400) mapped to 1-15 MHz, Lorentzian
                  width 2 bins (FWHM), SNR -20 dB per sample.
* ``paper``     : the paper's own timing shape (4096 gates, nfft 16384, 100 IPPs,
                  echo rows of 250,000 samples) with noise plus tones.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_HOST_LIB = os.path.join(_LIBDIR, "libisr_synth.so")
_GPU_LIB = os.path.join(_LIBDIR, "libisr_synth_gpu.so")
_lock = threading.Lock()
_host = None
_gpu = None

NOISE_ONLY, TONE, LINE = 0, 1, 2


class SynCfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("echo_stride", ctypes.c_int64),
        ("n_ipp", ctypes.c_int32),
        ("code_len", ctypes.c_int32),
        ("n_ranges", ctypes.c_int32),
        ("range_start", ctypes.c_int32),
        ("range_step", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("per_ipp_code", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("sigma", ctypes.c_double),
        ("amp", ctypes.c_double),
        ("hwhm", ctypes.c_double),
        ("max_jitter", ctypes.c_double),
    ]


def _newer(target, *srcs):
    return os.path.exists(target) and all(os.path.getmtime(target) >= os.path.getmtime(s) for s in srcs)


def build_host(force: bool = False) -> str:
    os.makedirs(_LIBDIR, exist_ok=True)
    srcs = [os.path.join(_HERE, "synth_host.c"), os.path.join(_HERE, "synth_core.h")]
    if not force and _newer(_HOST_LIB, *srcs):
        return _HOST_LIB
    tmp = _HOST_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", srcs[0], "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _HOST_LIB)
    return _HOST_LIB


def build_gpu(force: bool = False) -> str:
    """Compile the device generator for sm_103a (cross-compiles without a GPU)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    srcs = [os.path.join(_HERE, "synth_gpu.cu"), os.path.join(_HERE, "synth_core.h")]
    if not force and _newer(_GPU_LIB, *srcs):
        return _GPU_LIB
    tmp = _GPU_LIB + f".tmp{os.getpid()}"
    subprocess.run(["nvcc", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-fmad=false",
                    "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", srcs[0], "-o", tmp], check=True)
    os.replace(tmp, _GPU_LIB)
    return _GPU_LIB


def _host_lib():
    global _host
    with _lock:
        if _host is None:
            build_host()
            lib = ctypes.CDLL(_HOST_LIB)
            lib.syn_philox_kat.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
            lib.syn_fill_table.argtypes = [ctypes.c_void_p]
            lib.syn_fill_code.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p]
            lib.syn_tone_freqs.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            lib.syn_fill_params.argtypes = [ctypes.POINTER(SynCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p]
            lib.syn_echo_rows.argtypes = [ctypes.POINTER(SynCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int]
            lib.syn_echo_rows.restype = ctypes.c_int
            _host = lib
    return _host


def _gpu_lib():
    global _gpu
    with _lock:
        if _gpu is None:
            build_gpu()
            lib = ctypes.CDLL(_GPU_LIB)
            lib.syn_gpu_echo.argtypes = [ctypes.POINTER(SynCfg), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            lib.syn_gpu_echo.restype = ctypes.c_int
            _gpu = lib
    return _gpu


@dataclasses.dataclass
class Workload:
    """A seeded synthetic workload: geometry plus generator settings."""
    name: str
    n_ranges: int
    nfft: int
    code_len: int
    n_ipp: int
    range_start: int
    range_step: int
    echo_stride: int
    seed: int
    kind: int
    sigma: float = 1000.0
    snr_db: float = -10.0
    fs_hz: float = 50e6
    per_ipp_code: bool = False
    # Langmuir-line settings (kind == LINE)
    chapman_peak_gate: float = 400.0
    chapman_scale_gates: float = 100.0
    f_lo_hz: float = 1e6
    f_hi_hz: float = 15e6
    fwhm_bins: float = 2.0
    snap_to_bins: bool = False
    # optional per-gate overrides: frequency (cycles/sample) and SNR in dB (-inf: no signal)
    gate_freq: np.ndarray | None = None
    gate_snr_db: np.ndarray | None = None

    @property
    def amp(self) -> float:
        # per-sample signal power / per-sample noise power (2 sigma^2)
        return math.sqrt(10.0 ** (self.snr_db / 10.0) * 2.0 * self.sigma ** 2)

    def cfg(self) -> SynCfg:
        c = SynCfg()
        c.seed = self.seed
        c.echo_stride = self.echo_stride
        c.n_ipp = self.n_ipp
        c.code_len = self.code_len
        c.n_ranges = self.n_ranges
        c.range_start = self.range_start
        c.range_step = self.range_step
        c.kind = self.kind
        c.per_ipp_code = 1 if self.per_ipp_code else 0
        c.sigma = self.sigma
        c.amp = self.amp
        c.hwhm = 0.5 * self.fwhm_bins / self.nfft
        c.max_jitter = 64.0 / self.nfft
        return c

    def gate_amps(self) -> np.ndarray | None:
        """Per-gate signal amplitude (None: ``amp`` for every gate)."""
        if self.gate_snr_db is None:
            return None
        snr = np.asarray(self.gate_snr_db, dtype=np.float64)
        lin = np.where(np.isfinite(snr), 10.0 ** (np.where(np.isfinite(snr), snr, 0.0) / 10.0), 0.0)
        return np.ascontiguousarray(np.sqrt(lin * 2.0 * self.sigma ** 2), dtype=np.float64)

    def base_freqs(self) -> np.ndarray:
        """Per-gate line/tone frequency in cycles per sample."""
        if self.gate_freq is not None:
            f = np.asarray(self.gate_freq, dtype=np.float64)
        elif self.kind == LINE:
            r = np.arange(self.n_ranges, dtype=np.float64)
            z = (r - self.chapman_peak_gate) / self.chapman_scale_gates
            ne_rel = np.exp(0.5 * (1.0 - z - np.exp(-z)))  # Chapman layer, n_e / n_max
            f_hz = self.f_lo_hz + (self.f_hi_hz - self.f_lo_hz) * np.sqrt(ne_rel)
            f = f_hz / self.fs_hz
        elif self.kind == TONE:
            f = np.zeros(self.n_ranges, dtype=np.float64)
            _host_lib().syn_tone_freqs(self.seed, self.n_ranges, f.ctypes.data)
        else:
            f = np.zeros(self.n_ranges, dtype=np.float64)
        if self.snap_to_bins:
            f = np.round(f * self.nfft) / self.nfft
        return np.ascontiguousarray(f, dtype=np.float64)

    def code(self) -> np.ndarray:
        """Binary-phase code(s) as int8 +-1: [code_len] shared or [n_ipp, code_len]."""
        rows = self.n_ipp if self.per_ipp_code else 1
        out = np.empty((rows, self.code_len), dtype=np.int8)
        _host_lib().syn_fill_code(self.seed, self.code_len, 0, rows, out.ctypes.data)
        return out if self.per_ipp_code else out[0]

    def echo_host(self, row_begin: int = 0, row_end: int | None = None, n_threads: int = 0) -> np.ndarray:
        """Echo rows [row_begin, row_end) as int16 [rows, echo_stride, 2] (host build)."""
        if row_end is None:
            row_end = self.n_ipp
        code = np.ascontiguousarray(self.code())
        fb = self.base_freqs()
        out = np.empty((row_end - row_begin, self.echo_stride, 2), dtype=np.int16)
        amps = self.gate_amps()
        rc = _host_lib().syn_echo_rows(ctypes.byref(self.cfg()), fb.ctypes.data,
                                       None if amps is None else amps.ctypes.data, code.ctypes.data,
                                       row_begin, row_end, out.ctypes.data, n_threads)
        if rc != 0:
            raise MemoryError("synthetic echo generation failed")
        return out

    def echo_device(self, out_ptr: int, code_dev_ptr: int, row_begin: int = 0,
                    row_end: int | None = None) -> None:
        """Echo rows into device memory at ``out_ptr`` (device build, synchronous).

        ``code_dev_ptr`` points to the device copy of ``self.code()``.
        """
        if row_end is None:
            row_end = self.n_ipp
        fb = self.base_freqs()
        amps = self.gate_amps()
        rc = _gpu_lib().syn_gpu_echo(ctypes.byref(self.cfg()), fb.ctypes.data,
                                     None if amps is None else amps.ctypes.data, code_dev_ptr,
                                     row_begin, row_end, out_ptr)
        if rc != 0:
            raise RuntimeError(f"device echo generation failed (cudaError {rc})")


def philox4x32_10(ctr, key64: int):
    c = (ctypes.c_uint32 * 4)(*ctr)
    o = (ctypes.c_uint32 * 4)()
    _host_lib().syn_philox_kat(c, key64, o)
    return list(o)


def phase_table() -> np.ndarray:
    t = np.empty(2 * (1 << 16), dtype=np.float32)
    _host_lib().syn_fill_table(t.ctypes.data)
    return t


def _round_up(x: int, m: int) -> int:
    return (x + m - 1) // m * m


def small(seed: int = 1, **kw) -> Workload:
    R, N, step = kw.get("n_ranges", 64), 1024, 25
    stride = _round_up((R - 1) * step + N, 128)
    base = dict(name="small", n_ranges=R, nfft=N, code_len=N, n_ipp=100, range_start=0,
                range_step=step, echo_stride=stride, seed=seed, kind=TONE, snr_db=-10.0)
    base.update(kw)
    return Workload(**base)


def realistic(seed: int = 2, **kw) -> Workload:
    R, N, step = kw.get("n_ranges", 1000), 16384, 25
    stride = _round_up((R - 1) * step + N, 128)
    base = dict(name="realistic", n_ranges=R, nfft=N, code_len=N, n_ipp=10000, range_start=0,
                range_step=step, echo_stride=stride, seed=seed, kind=LINE, snr_db=-20.0)
    base.update(kw)
    return Workload(**base)


def paper(seed: int = 3, **kw) -> Workload:
    base = dict(name="paper", n_ranges=4096, nfft=16384, code_len=16384, n_ipp=100, range_start=0,
                range_step=25, echo_stride=250000, seed=seed, kind=TONE, snr_db=-10.0)
    base.update(kw)
    return Workload(**base)
