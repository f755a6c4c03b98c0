"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and compare it
with the FP64 oracle bin by bin."""
from __future__ import annotations

import numpy as np
import torch

from paper_2311_18737_gb300 import isr

# Relative tolerance per bin (FP32 transform and FP32 chunk sums against the FP64
# oracle; the derivation of this bound is in the design notes).
RTOL = 1e-5

TX_OF_DTYPE = {np.dtype(np.int8): isr.ISR_TX_PM1, np.dtype(np.int16): isr.ISR_TX_CI16,
               np.dtype(np.float32): isr.ISR_TX_C32}


def gpu_integrate(echo: np.ndarray, tx: np.ndarray, *, nfft: int, n_ranges: int, range_start: int = 0,
                  range_step: int = 25, code_len: int | None = None, per_ipp_tx: bool = False,
                  ipp_chunk: int = 0, max_chunks: int = 0, calls=None, host_input: bool = False,
                  flags: int = 0):
    """Integrate on cuda:0; ``calls`` optionally splits the IPPs into several isr_integrate calls."""
    dev = torch.device("cuda:0")
    n_ipp, stride = echo.shape[0], echo.shape[1]
    tx_type = TX_OF_DTYPE[tx.dtype]
    L = code_len if code_len is not None else (tx.shape[-1] if tx_type == isr.ISR_TX_PM1 else tx.shape[-2])
    tx_len = tx.shape[-1] if tx_type == isr.ISR_TX_PM1 else tx.shape[-2]
    tx_stride = tx_len if per_ipp_tx else 0
    stream = torch.cuda.current_stream(dev)
    if host_input:
        e_in, t_in = np.ascontiguousarray(echo), np.ascontiguousarray(tx)
    else:
        e_in = torch.from_numpy(np.ascontiguousarray(echo)).to(dev)
        t_in = torch.from_numpy(np.ascontiguousarray(tx)).to(dev)
    with isr.Plan(nfft=nfft, n_ranges=n_ranges, echo_stride=stride, code_len=L, range_start=range_start,
                  range_step=range_step, tx_type=tx_type, tx_stride=tx_stride, ipp_chunk=ipp_chunk,
                  max_chunks=max_chunks, device=0, stream=stream) as plan:
        splits = calls or [n_ipp]
        p0 = 0
        for n in splits:
            if host_input:
                e_part = e_in[p0:]
                t_part = t_in[p0:] if per_ipp_tx else t_in
            else:
                e_part = e_in[p0:]
                t_part = t_in[p0:] if per_ipp_tx else t_in
            plan.integrate(e_part, t_part, n)
            p0 += n
        out = torch.empty((n_ranges, nfft), dtype=torch.float32, device=dev)
        _, n_done = plan.spectra(out, flags)
        info = plan.info()
    assert n_done == p0
    return out.cpu().numpy().astype(np.float64), info


def rel_err(got, ref):
    return np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)


def assert_parity(got, ref, rtol=RTOL, what=""):
    rel = rel_err(got, ref)
    worst = np.unravel_index(int(np.argmax(rel)), rel.shape)
    assert rel.max() <= rtol, (f"{what}: max rel err {rel.max():.3e} at {worst} "
                               f"(got {got[worst]:.6e}, ref {ref[worst]:.6e}); p99 {np.quantile(rel, 0.99):.2e}")
    return float(rel.max()), float(np.quantile(rel, 0.99)), float(np.median(rel))
