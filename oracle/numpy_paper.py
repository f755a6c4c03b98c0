"""The paper's CPU comparison implementation, written with NumPy (test and baseline infrastructure).

Sec. 3.3 of the paper times a NumPy implementation of the same steps on one CPU core (the CPU
row of Table 1).  This module follows those steps per IPP, vectorised over range gates as the
paper's GPU kernels are (Sec. 3.2):

  1. complex multiplication: batch[r, k] = conj(eps_p[k]) * m_p[s_r + k] for k < L, zero-padded
     to nfft (Eq. 7, the "complex multiplication" kernel),
  2. one FFT per batch row (numpy.fft.fft along k, double precision),
  3. spectrum accumulation: spectrum[r, f] += |batch_fft[r, f]|^2 (Eq. 8).

It is a timing baseline beside the FP64 oracle (``bench.py`` reports it as the paper-style CPU
figure) and a second, independent CPU implementation that the tests compare with the oracle.
It shares nothing with the CUDA path.
"""
from __future__ import annotations

import numpy as np

TX_CI16, TX_C32, TX_PM1 = 0, 1, 2


def _code_rows(tx, tx_type: int, code_len: int):
    tx = np.asarray(tx)
    if tx_type == TX_PM1:
        eps = np.where(tx.reshape(-1, code_len) < 0, -1.0, 1.0).astype(np.complex128)
    elif tx_type == TX_CI16:
        t = tx.reshape(-1, code_len, 2).astype(np.float64)
        eps = t[..., 0] + 1j * t[..., 1]
    else:
        t = tx.reshape(-1, code_len, 2).astype(np.float64)
        eps = t[..., 0] + 1j * t[..., 1]
    return eps


def integrate(echo, tx, nfft: int, n_ranges: int, range_start: int = 0, range_step: int = 1,
              code_len: int | None = None, tx_type: int = TX_PM1, per_ipp_code: bool = False,
              gates=None):
    """Summed power spectra [len(gates)][nfft] (float64) of the int16 IQ echo
    [n_ipp][echo_stride][2] decoded with the code rows ``tx``; ``gates`` selects range gates
    (default: all n_ranges)."""
    echo = np.asarray(echo)
    n_ipp = echo.shape[0]
    L = nfft if code_len is None else int(code_len)
    eps = _code_rows(tx, tx_type, L)
    gates = np.arange(n_ranges) if gates is None else np.asarray(gates)
    idx = range_start + gates[:, None] * range_step + np.arange(L)[None, :]
    spectrum = np.zeros((len(gates), nfft))
    batch = np.zeros((len(gates), nfft), dtype=np.complex128)
    for p in range(n_ipp):
        m = echo[p, :, 0].astype(np.float64) + 1j * echo[p, :, 1].astype(np.float64)
        e = eps[p] if per_ipp_code else eps[0]
        batch[:, :L] = np.conj(e)[None, :] * m[idx]
        X = np.fft.fft(batch, axis=1)
        spectrum += X.real ** 2 + X.imag ** 2
    return spectrum
