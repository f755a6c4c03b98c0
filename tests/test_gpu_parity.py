"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on seeded inputs.

Sizes span every transform length the library supports, ragged gate counts, windows
that start off the 16-byte grid, zero-padded codes, every code format, per-IPP codes,
multi-chunk and multi-launch integrations, repeated calls, host-resident inputs and the
timeout path.  The tolerance is the per-bin relative bound RTOL.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import RTOL, assert_parity, gpu_integrate
from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu


def _rand_case(rng, nfft, R, P, start, step, L, kind, per, stride_extra=8):
    stride = start + (R - 1) * step + L + stride_extra
    stride = (stride + 3) // 4 * 4
    # noise-like int16 so every bin has power (relative errors are well defined)
    echo = np.clip(np.rint(rng.standard_normal((P, stride, 2)) * 1000), -32768, 32767).astype(np.int16)
    shape = (P, L) if per else (L,)
    if kind == "pm1":
        tx = np.where(rng.random(shape) < 0.5, -1, 1).astype(np.int8)
    elif kind == "ci16":
        tx = rng.integers(-3, 4, size=shape + (2,)).astype(np.int16)
        tx[..., 0] = np.where(tx[..., 0] == 0, 1, tx[..., 0])
    else:
        tx = (rng.standard_normal(shape + (2,))).astype(np.float32)
    return echo, tx


@pytest.mark.parametrize("log2n", list(range(3, 15)))
def test_every_nfft_pm1(log2n):
    rng = np.random.default_rng(100 + log2n)
    nfft = 1 << log2n
    G = max(1, 16384 // nfft)
    R = G + 3 if G < 64 else 37          # ragged: not a multiple of the gates per CTA
    P = 5 if nfft <= 4096 else 3
    echo, tx = _rand_case(rng, nfft, R, P, start=3, step=7, L=nfft, kind="pm1", per=False)
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=3, range_step=7)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=3, range_step=7)
    assert_parity(got, ref, what=f"nfft={nfft}")


@pytest.mark.parametrize("kind,per", [("ci16", False), ("c32", False), ("pm1", True), ("ci16", True)])
@pytest.mark.parametrize("log2n", [6, 10, 14])
def test_code_formats(kind, per, log2n):
    rng = np.random.default_rng(7 * log2n + len(kind))
    nfft = 1 << log2n
    R, P = 5, 4
    L = nfft - nfft // 8 - 1              # zero-padded window
    echo, tx = _rand_case(rng, nfft, R, P, start=1, step=3, L=L, kind=kind, per=per)
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=1, range_step=3, code_len=L,
                           per_ipp_tx=per)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=1, range_step=3, code_len=L,
                           per_ipp_tx=per)
    assert_parity(got, ref, what=f"{kind} per={per} nfft={nfft}")


# every transform length through the kernels for codes that are not full-length binary phase:
# a zero-padded +-1 code, a full-length complex int16 code and a zero-padded complex float code
@pytest.mark.parametrize("kind,padded", [("pm1", True), ("ci16", False), ("c32", True)])
@pytest.mark.parametrize("log2n", list(range(3, 15)))
def test_every_nfft_general_codes(log2n, kind, padded):
    rng = np.random.default_rng(100 + 3 * log2n + len(kind))
    nfft = 1 << log2n
    R, P = 3, 3
    L = nfft - max(1, nfft // 8) if padded else nfft
    echo, tx = _rand_case(rng, nfft, R, P, start=2, step=5, L=L, kind=kind, per=False)
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=5, code_len=L)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=5, code_len=L)
    assert_parity(got, ref, what=f"{kind} L={L} nfft={nfft}")


@pytest.mark.parametrize("kind", ["pm1", "ci16"])
@pytest.mark.parametrize("log2n", [11, 14])
def test_per_ipp_code_rows_longer_than_the_code(log2n, kind):
    """Per-IPP code rows 32 chips longer than code_len (tx_stride > code_len): each IPP reads
    the first code_len chips of its own row; full-length codes, so +-1 codes take the fast kernel."""
    rng = np.random.default_rng(300 + log2n + len(kind))
    nfft = 1 << log2n
    R, P = 3, 5
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=9, L=nfft + 32, kind=kind, per=True)
    echo = np.ascontiguousarray(echo[:, : ((2 * 9 + nfft + 3) // 4 * 4 + 8)])
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=9, code_len=nfft, per_ipp_tx=True)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=9, code_len=nfft, per_ipp_tx=True)
    assert_parity(got, ref, what=f"{kind} tx_stride {nfft + 32} code_len {nfft}")


@pytest.mark.parametrize("order,log2n", [(o, l) for l in (11, 12, 13, 14) for o in range(4)] +
                         [(o, 14) for o in range(4, isr.N_ORDERS)])
def test_radix_orders(log2n, order):
    rng = np.random.default_rng(31 * log2n + order)
    nfft = 1 << log2n
    R, P = 16384 // nfft + 2, 3
    echo, tx = _rand_case(rng, nfft, R, P, start=2, step=11, L=nfft, kind="pm1", per=False)
    dev = torch.device("cuda:0")
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_start=2, range_step=11, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        isr.isr_plan_set_order(plan.handle, order)
        plan.integrate(torch.from_numpy(echo).to(dev), torch.from_numpy(tx).to(dev), P)
        out, _ = plan.spectra()
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=11)
    assert_parity(out.numpy().astype(np.float64), ref, what=f"nfft={nfft} order={order}")


def test_autotune_keeps_parity():
    rng = np.random.default_rng(8)
    nfft, R, P = 16384, 3, 4
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=25, L=nfft, kind="pm1", per=False)
    dev = torch.device("cuda:0")
    e, t = torch.from_numpy(echo).to(dev), torch.from_numpy(tx).to(dev)
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_step=25, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        res = plan.autotune(e, t, P)
        assert res["order"] in range(isr.N_ORDERS) and len(res["ms"]) == isr.N_ORDERS
        plan.integrate(e, t, P)
        out, n = plan.spectra()
    assert n == P
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25)
    assert_parity(out.numpy().astype(np.float64), ref, what="after autotune")


def test_small_workload_full():
    """64 gates x nfft 1024 x 100 IPPs: every bin of the whole workload."""
    w = synth.small()
    echo, code = w.echo_host(), w.code()
    got, info = gpu_integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    mx, p99, med = assert_parity(got, ref, what="small workload")
    print(f"small workload: max {mx:.2e} p99 {p99:.2e} median {med:.2e}; launch {info}")


def test_chunks_launches_and_calls_agree():
    rng = np.random.default_rng(5)
    nfft, R, P = 2048, 11, 23
    echo, tx = _rand_case(rng, nfft, R, P, start=2, step=5, L=nfft, kind="pm1", per=False)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=5)
    # 3 IPPs per chunk, at most 2 chunks per launch -> 4 launches
    got, info = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=5, ipp_chunk=3,
                              max_chunks=2)
    assert info["kernel_launches"] == 4
    assert_parity(got, ref, what="multi-launch")
    got2, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=2, range_step=5, calls=[1, 9, 13])
    assert_parity(got2, ref, what="three calls")


def test_host_resident_input():
    rng = np.random.default_rng(9)
    nfft, R, P = 4096, 6, 7
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=25, L=nfft, kind="ci16", per=True)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25, per_ipp_tx=True)
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25, per_ipp_tx=True, host_input=True)
    assert_parity(got, ref, what="host input")


def test_host_input_larger_than_a_staging_buffer():
    """Host rows beyond one 1 GiB staging buffer: the library streams them in several blocks
    through two device buffers (the first block smaller), and the sums equal the oracle's."""
    rng = np.random.default_rng(21)
    nfft, R, step = 16384, 3, 25
    stride = ((R - 1) * step + nfft + 3) // 4 * 4
    P = (1 << 30) // (stride * 4) + 1200                  # ~1.07 GiB of host rows
    echo = rng.integers(-3000, 3001, size=(P, stride, 2), dtype=np.int16)
    tx = np.where(rng.random(nfft) < 0.5, -1, 1).astype(np.int8)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=step)
    got, info = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=step, host_input=True)
    assert info["kernel_launches"] >= 3                 # first block, a full buffer, the rest
    # the block growth was measured on block 0's copy and kernels
    assert 1 <= info["host_block_growth"] <= 4, info
    assert_parity(got, ref, what="host input over several staging blocks")


def test_mean_and_reset_flags():
    rng = np.random.default_rng(4)
    nfft, R, P = 256, 9, 6
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=9, L=nfft, kind="pm1", per=False)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=9)
    dev = torch.device("cuda:0")
    e = torch.from_numpy(echo).to(dev)
    t = torch.from_numpy(tx).to(dev)
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_step=9, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        plan.integrate(e, t, P)
        out = torch.empty((R, nfft), dtype=torch.float32, device=dev)
        _, n = plan.spectra(out, isr.ISR_MEAN | isr.ISR_RESET_AFTER)
        assert n == P
        assert_parity(out.cpu().numpy().astype(np.float64), ref / P, what="mean")
        host = np.empty((R, nfft), np.float32)
        _, n = plan.spectra(host)
        assert n == 0 and not host.any()


def test_zero_ipps_is_a_no_op():
    """n_ipp == 0 changes neither the sums nor the IPP count, even with NULL buffers; a
    negative count is an argument error."""
    rng = np.random.default_rng(13)
    nfft, R, P = 1024, 5, 4
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=25, L=nfft, kind="pm1", per=False)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25)
    dev = torch.device("cuda:0")
    e, t = torch.from_numpy(echo).to(dev), torch.from_numpy(tx).to(dev)
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_step=25, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        isr.isr_integrate(plan.handle, None, None, 0, None, nfft)
        plan.integrate(e, t, 2)
        plan.integrate(e, t, 0)
        isr.isr_integrate(plan.handle, None, None, 0, None, nfft)
        plan.integrate(e[2:], t, P - 2)
        with pytest.raises(isr.IsrError) as ei:
            isr.isr_integrate(plan.handle, e, t, -1, None, nfft)
        assert ei.value.status == isr.ISR_ERR_INVALID_ARG
        out, n = plan.spectra()
    assert n == P
    assert_parity(out.numpy().astype(np.float64), ref, what="zero-IPP calls")


def test_ranges_override():
    rng = np.random.default_rng(12)
    nfft, R, P = 512, 7, 4
    echo, tx = _rand_case(rng, nfft, R, P, start=5, step=13, L=nfft, kind="pm1", per=False, stride_extra=200)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=9, range_step=31)
    dev = torch.device("cuda:0")
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_start=5, range_step=13, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        plan.integrate(torch.from_numpy(echo).to(dev), torch.from_numpy(tx).to(dev), P, ranges=(9, 31))
        out, _ = plan.spectra()
    assert_parity(out.numpy().astype(np.float64), ref, what="ranges override")


# 1024: a gate per warp (warp votes); 4096: four gates per CTA on their own named barriers;
# 16384: one gate per CTA (CTA barrier)
@pytest.mark.parametrize("nfft", [1024, 4096, 16384])
def test_timeout_is_reported_and_context_survives(nfft):
    _timeout_case(nfft, 0)


@pytest.mark.parametrize("order", [3, 6, 7, 9])
def test_timeout_every_barrier_kind_at_16384(order):
    # warp-local schedule (CTA + warp barriers) and tensor-memory twiddles (the CTA frees its
    # TMEM on the timeout path)
    _timeout_case(16384, order)


def test_timeout_with_the_tcgen05_first_pass():
    # the dropped window is voted on before that IPP's GEMM is issued; the CTA frees its TMEM
    _timeout_case(16384, 0, isr.ISR_PREC_TC05_FP16_SPLIT)


def _timeout_case(nfft, order, precision=0):
    rng = np.random.default_rng(13)
    R, P = 4, 5
    echo, tx = _rand_case(rng, nfft, R, P, start=0, step=25, L=nfft, kind="pm1", per=False)
    dev = torch.device("cuda:0")
    e = torch.from_numpy(echo).to(dev)
    t = torch.from_numpy(tx).to(dev)
    with isr.Plan(nfft=nfft, n_ranges=R, echo_stride=echo.shape[1], range_step=25, device=0,
                  stream=torch.cuda.current_stream()) as plan:
        if order:
            isr.isr_plan_set_order(plan.handle, order)
        if precision:
            isr.isr_plan_set_precision(plan.handle, precision)
        isr.isr_plan_set_wait_limit(plan.handle, 1 << 12)
        isr.isr_plan_test_drop_window(plan.handle, 2)
        plan.integrate(e, t, P)
        with pytest.raises(isr.IsrError) as ei:
            plan.spectra()
        assert ei.value.status == isr.ISR_ERR_TIMEOUT
        # the context is still usable: a clean integration on a fresh plan matches the oracle
    got, _ = gpu_integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25)
    ref = oracle.integrate(echo, tx, nfft=nfft, n_ranges=R, range_step=25)
    assert_parity(got, ref, what=f"after timeout (order {order})")


def test_device_generator_matches_host_generator():
    w = synth.realistic(n_ipp=3, n_ranges=200)
    dev = torch.device("cuda:0")
    code_d = torch.from_numpy(w.code()).to(dev)
    out = torch.empty((w.n_ipp, w.echo_stride, 2), dtype=torch.int16, device=dev)
    w.echo_device(out.data_ptr(), code_d.data_ptr())
    assert np.array_equal(out.cpu().numpy(), w.echo_host())


def test_allocation_failure_is_reported_and_context_survives():
    # 2^30 gates x 16384 bins of FP64 accumulators (128 TiB) cannot be allocated: the plan
    # reports ISR_ERR_NO_MEMORY and the device stays usable
    nfft, R = 16384, 1 << 30
    with pytest.raises(isr.IsrError) as ei:
        isr.Plan(nfft=nfft, n_ranges=R, echo_stride=R + nfft, range_step=1, device=0,
                 stream=torch.cuda.current_stream())
    assert ei.value.status == isr.ISR_ERR_NO_MEMORY
    rng = np.random.default_rng(14)
    echo, tx = _rand_case(rng, 1024, 4, 3, start=0, step=25, L=1024, kind="pm1", per=False)
    got, _ = gpu_integrate(echo, tx, nfft=1024, n_ranges=4, range_step=25)
    ref = oracle.integrate(echo, tx, nfft=1024, n_ranges=4, range_step=25)
    assert_parity(got, ref, what="after allocation failure")
