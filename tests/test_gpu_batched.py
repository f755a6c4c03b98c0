"""Batched uneven windows (one persistent launch) against one plan per window and against
the FP64 oracle on sampled gates; every radix order, graph replay, autotuning."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import RTOL, assert_parity
from paper_2311_18737_gb300 import batched, isr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bufs():
    ws = batched.config_windows(seed=5, n_windows=8, ipp_scale=0.006, max_gates=300)
    return batched.Buffers(ws)


@pytest.fixture(scope="module")
def reference(bufs):
    outs = batched.per_window(bufs)
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in outs]


@pytest.mark.parametrize("order", [0, 1, 2, 3])
def test_every_radix_order_matches_per_window_plans(bufs, reference, order):
    b = batched.Batch(bufs, flags=0, order=order)
    b.run()
    for i, (o, ref) in enumerate(zip(bufs.out, reference)):
        assert_parity(o.cpu().numpy().astype(np.float64), ref, what=f"order {order} window {i}")
    b.close()


def test_graph_replay_and_autotune(bufs, reference):
    b = batched.Batch(bufs, flags=isr.ISR_BATCH_GRAPH | isr.ISR_BATCH_AUTOTUNE)
    info = b.info()
    assert info["graph"] and info["n_windows"] == 8
    used = {w.nfft for w in bufs.w}
    for k, n in enumerate(batched.NFFTS):
        if n in used:
            assert info["order"][k] in (0, 1, 2, 3) and min(info["tune_ms"][k]) > 0
    b.run()
    first = [o.clone() for o in bufs.out]
    b.run()
    for a, c, ref in zip(first, bufs.out, reference):
        assert torch.equal(a, c)   # replays are deterministic
        assert_parity(c.cpu().numpy().astype(np.float64), ref, what="graph replay")
    b.close()


def test_sampled_gates_against_oracle(bufs):
    b = batched.Batch(bufs, flags=0)
    b.run()
    for i in (0, 1):   # one up-shifted, one down-shifted window
        w = bufs.w[i]
        echo = bufs.echo[i].cpu().numpy()
        code = bufs.code[i].cpu().numpy()
        sel = [0, w.n_ranges // 2, w.n_ranges - 1]
        ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_start=w.range_start,
                               range_step=w.range_step, sel=sel)
        assert_parity(bufs.out[i].cpu().numpy().astype(np.float64)[sel], ref, rtol=RTOL, what=f"window {i}")
    b.close()


def test_bad_window_rejected(bufs):
    ws = bufs.windows()
    ws[3].nfft = 1024
    with pytest.raises(isr.IsrError) as ei:
        isr.isr_batch_create(ws, 0, 0, torch.cuda.current_stream())
    assert ei.value.status == isr.ISR_ERR_UNSUPPORTED


def test_reused_per_window_plans_match_fresh_plans(bufs, reference):
    # the batched comparison's baseline: plans created once and reused over two runs
    pw = batched.PerWindowPlans(bufs, orders={2048: 1, 4096: 0, 8192: 2, 16384: 1})
    try:
        for _ in range(2):
            outs = [torch.empty_like(o) for o in bufs.out]
            pw.run(outs)
            for i, (o, r) in enumerate(zip(outs, reference)):
                assert_parity(o.cpu().numpy().astype(np.float64), r, rtol=RTOL, what=f"reused plan, window {i}")
    finally:
        pw.close()
