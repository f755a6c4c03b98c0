"""Plain FP64 CPU oracle for decoded power-spectrum integration.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` are the only callers.  The product path never imports this package.

The arithmetic lives in ``isr_oracle.c`` (plain C, double precision, textbook radix-2
FFT); this module only compiles it with gcc and marshals numpy arrays through ctypes.
It follows the paper's Sec. 2.2 (Eqs. 7-8) and the kernel descriptions of Sec. 3.2:
decode ``conj(eps) * echo window``, forward DFT, add ``|X|^2`` over IPPs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libisr_oracle.so")
_SRC = os.path.join(_HERE, "isr_oracle.c")
_lock = threading.Lock()
_lib = None

TX_CI16, TX_C32, TX_PM1 = 0, 1, 2


def _compile(src: str, out: str) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/lib/libisr_oracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return _compile(_SRC, _LIB)


class OracleLib:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_fft.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_fft.restype = ctypes.c_int
        lib.oracle_integrate.argtypes = [
            ctypes.c_void_p, ctypes.c_int64,                # echo, echo_stride
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,  # tx, tx_type, tx_stride
            ctypes.c_int, ctypes.c_int, ctypes.c_int,       # n_ipp, nfft, code_len
            ctypes.c_int, ctypes.c_int64, ctypes.c_int64,   # n_ranges, start, step
            ctypes.c_void_p, ctypes.c_int,                  # sel, n_sel
            ctypes.c_void_p, ctypes.c_int]                  # P, n_threads
        lib.oracle_integrate.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def fft(self, x):
        return _fft(self.lib, x)

    def integrate(self, echo, tx, **kw):
        return _integrate(self.lib, echo, tx, **kw)


def load_variant(src_text: str, tag: str) -> OracleLib:
    """Compile a modified copy of the oracle source (used by tests that plant a mistake
    in the oracle and check that its pins catch it)."""
    d = os.path.join(_LIBDIR, "variants")
    os.makedirs(d, exist_ok=True)
    src = os.path.join(d, f"{tag}.c")
    with open(src, "w") as fh:
        fh.write(src_text)
    return OracleLib(_compile(src, os.path.join(d, f"lib{tag}.so")))


def source_text() -> str:
    with open(_SRC) as fh:
        return fh.read()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = OracleLib(_LIB)
    return _lib


def fft(x: np.ndarray) -> np.ndarray:
    """Forward unnormalised DFT of a power-of-two-length complex vector (FP64)."""
    return _load().fft(x)


def integrate(echo, tx, **kw) -> np.ndarray:
    """Sum over IPPs of |DFT(conj(eps) * echo window)|^2 per range gate (FP64).

    See ``_integrate`` for the arguments."""
    return _load().integrate(echo, tx, **kw)


def _fft(lib, x):
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real, dtype=np.float64)
    im = np.ascontiguousarray(x.imag, dtype=np.float64)
    rc = lib.oracle_fft(re.ctypes.data, im.ctypes.data, int(x.size))
    if rc != 0:
        raise ValueError(f"oracle_fft failed ({rc})")
    return re + 1j * im


def _tx_type_of(tx: np.ndarray) -> int:
    if tx.dtype == np.int16:
        return TX_CI16
    if tx.dtype == np.float32:
        return TX_C32
    if tx.dtype == np.int8:
        return TX_PM1
    raise TypeError(f"unsupported tx dtype {tx.dtype}")


def _integrate(lib, echo: np.ndarray, tx: np.ndarray, *, nfft: int, n_ranges: int,
              range_start: int = 0, range_step: int = 25, code_len: int | None = None,
              n_ipp: int | None = None, per_ipp_tx: bool = False,
              sel=None, out: np.ndarray | None = None, n_threads: int = 0) -> np.ndarray:
    """Sum over IPPs of |DFT(conj(eps) * echo window)|^2 per range gate (FP64).

    echo : int16 array shaped [n_ipp, echo_stride, 2] (interleaved I, Q).
    tx   : one code [code_len(, 2)] or per-IPP codes [n_ipp, code_len(, 2)];
           int16 pairs (complex int16), float32 pairs (complex float) or int8 (+-1).
    sel  : optional list of gate indices; the result has one row per selected gate.
    out  : optional float64 [n_sel, nfft] array to add into.
    """
    echo = np.ascontiguousarray(echo, dtype=np.int16)
    if echo.ndim != 3 or echo.shape[2] != 2:
        raise ValueError("echo must be [n_ipp, echo_stride, 2] int16")
    n_rows, echo_stride = echo.shape[0], echo.shape[1]
    if n_ipp is None:
        n_ipp = n_rows
    if n_ipp > n_rows:
        raise ValueError("n_ipp exceeds echo rows")
    tx = np.ascontiguousarray(tx)
    tx_type = _tx_type_of(tx)
    rows_shape = tx.shape if tx_type == TX_PM1 else tx.shape[:-1]
    if tx_type != TX_PM1 and tx.shape[-1] != 2:
        raise ValueError("complex tx must end in a (re, im) axis of size 2")
    if per_ipp_tx:
        if len(rows_shape) != 2 or rows_shape[0] < n_ipp:
            raise ValueError("per-IPP tx must be [n_ipp, code_len(,2)]")
        tx_len = rows_shape[1]
        tx_stride = tx_len
    else:
        if len(rows_shape) != 1:
            raise ValueError("shared tx must be [code_len(,2)]")
        tx_len = rows_shape[0]
        tx_stride = 0
    if code_len is None:
        code_len = tx_len
    if code_len > tx_len:
        raise ValueError("code_len exceeds tx length")
    if sel is None:
        sel_arr = None
        n_sel = n_ranges
    else:
        sel_arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int32))
        n_sel = int(sel_arr.size)
    if out is None:
        out = np.zeros((n_sel, nfft), dtype=np.float64)
    if out.dtype != np.float64 or out.shape != (n_sel, nfft) or not out.flags.c_contiguous:
        raise ValueError("out must be C-contiguous float64 [n_sel, nfft]")
    rc = lib.oracle_integrate(
        echo.ctypes.data, echo_stride, tx.ctypes.data, tx_type, tx_stride,
        int(n_ipp), int(nfft), int(code_len), int(n_ranges), int(range_start), int(range_step),
        None if sel_arr is None else sel_arr.ctypes.data, n_sel, out.ctypes.data, int(n_threads))
    if rc != 0:
        raise ValueError(f"oracle_integrate failed ({rc})")
    return out
