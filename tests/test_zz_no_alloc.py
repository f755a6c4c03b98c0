"""The allocation-free entry point against the plan-based one.

isr_integrate_static serves callers that cannot allocate device memory (device memory
reserved up front by another allocator or by a real-time pipeline).  Its chunk partials
live in a fixed device array inside the library that every call reuses, so this checks
two calls in a row on the same array (the second must not see the first's leftovers),
each against the plan path within the per-bin tolerance of the other GPU tests.  The
file sorts last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import RTOL, assert_parity
from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu


def _plan_spectra(desc, echo_d, code_d, n_ipp):
    h = isr.isr_plan_create(desc)
    try:
        isr.isr_integrate(h, echo_d, code_d, n_ipp, None, desc.nfft)
        out = torch.empty((desc.n_ranges, desc.nfft), dtype=torch.float32, device=echo_d.device)
        isr.isr_spectra(h, out, 0)
    finally:
        isr.isr_destroy(h)
    return out.cpu().numpy().astype(np.float64)


def _desc(w, stream):
    """Plan description of workload ``w`` (binary-phase code shared by every IPP)."""
    d = isr.IsrPlanDesc()
    d.nfft, d.code_len, d.n_ranges = w.nfft, w.code_len, w.n_ranges
    d.range_start, d.range_step, d.tx_type = w.range_start, w.range_step, isr.ISR_TX_PM1
    d.echo_stride, d.tx_stride, d.ipp_chunk, d.max_chunks = w.echo_stride, 0, 0, 0
    d.device, d.flags, d.stream = 0, 0, stream.cuda_stream
    return d


def test_static_entry_point_matches_plan_twice():
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    cases = [synth.small(n_ipp=100, seed=21), synth.small(n_ipp=37, n_ranges=40, seed=22)]
    for w in cases:
        echo_d = torch.from_numpy(w.echo_host()).to(dev)
        code_d = torch.from_numpy(w.code()).to(dev)
        desc = _desc(w, stream)
        ref = _plan_spectra(desc, echo_d, code_d, w.n_ipp)
        out = torch.full((w.n_ranges, w.nfft), float("nan"), dtype=torch.float32, device=dev)
        isr.isr_integrate_static(desc, echo_d, code_d, w.n_ipp, out)
        assert_parity(out.cpu().numpy().astype(np.float64), ref, rtol=RTOL, what=f"static call, {w.n_ranges} gates")


def test_static_entry_point_rejects_oversize_problem():
    dev = torch.device("cuda:0")
    w = synth.realistic(n_ipp=1, n_ranges=300)       # 300 x 16384 > 4 Mi floats
    d = _desc(w, torch.cuda.current_stream(dev))
    echo_d = torch.zeros((1, w.echo_stride, 2), dtype=torch.int16, device=dev)
    code_d = torch.ones(w.code_len, dtype=torch.int8, device=dev)
    out = torch.empty((w.n_ranges, w.nfft), dtype=torch.float32, device=dev)
    with pytest.raises(isr.IsrError) as ei:
        isr.isr_integrate_static(d, echo_d, code_d, 1, out)
    assert ei.value.status == isr.ISR_ERR_INVALID_ARG


def test_static_entry_point_keeps_fp32_chunks_short_at_the_scratch_limit():
    """256 gates x nfft 16384 fill the whole static array (4 Mi floats), so only one IPP chunk
    fits at a time: 1200 IPPs must run as five blocks of at most 256 IPPs, each block's FP32
    sum added into the output, and stay within the per-bin tolerance of the FP64 oracle (a
    single 1200-IPP FP32 sum would not be guaranteed to).  Two calls in a row."""
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    w = synth.realistic(n_ipp=1200, n_ranges=256, seed=31)
    assert w.n_ranges * w.nfft == isr.ISR_STATIC_SCRATCH_FLOATS
    code = w.code()
    code_d = torch.from_numpy(code).to(dev)
    echo_d = torch.empty((w.n_ipp, w.echo_stride, 2), dtype=torch.int16, device=dev)
    w.echo_device(echo_d.data_ptr(), code_d.data_ptr())
    sel = [0, 1, 127, 128, 254, 255]
    ref = oracle.integrate(echo_d.cpu().numpy(), code, nfft=w.nfft, n_ranges=w.n_ranges,
                           range_start=w.range_start, range_step=w.range_step, sel=sel)
    desc = _desc(w, stream)
    for call in range(2):
        out = torch.full((w.n_ranges, w.nfft), float("nan"), dtype=torch.float32, device=dev)
        isr.isr_integrate_static(desc, echo_d, code_d, w.n_ipp, out)
        got = out.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        assert_parity(got[sel], ref, rtol=RTOL, what=f"static call {call}, 256 gates x 16384, 1200 IPPs")


def test_static_entry_point_zero_padded_code():
    """A code shorter than the transform (700 chips, nfft 1024: zero-padded window) through the
    static entry point, against the FP64 oracle, two calls in a row."""
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    w = synth.small(n_ipp=60, n_ranges=48, code_len=700, seed=23)
    echo = w.echo_host()
    code = w.code()
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_start=w.range_start,
                           range_step=w.range_step)
    echo_d = torch.from_numpy(echo).to(dev)
    code_d = torch.from_numpy(code).to(dev)
    desc = _desc(w, stream)
    assert desc.code_len == 700 and desc.nfft == 1024
    for call in range(2):
        out = torch.full((w.n_ranges, w.nfft), float("nan"), dtype=torch.float32, device=dev)
        isr.isr_integrate_static(desc, echo_d, code_d, w.n_ipp, out)
        assert_parity(out.cpu().numpy().astype(np.float64), ref, rtol=RTOL, what=f"static zero-padded call {call}")
