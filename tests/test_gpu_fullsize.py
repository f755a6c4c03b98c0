"""Parity at the full realistic workload, in the launch configuration the benchmark times:
1000 gates x nfft 16384 x 10,000 IPPs (1.66 GB of int16 IQ made by the device build of
the input generator, itself checked bit for bit against the host build on sampled rows).

* sampled gates (edges, the Chapman peak and its neighbours, random picks): every bin
  against the FP64 oracle over all 10,000 IPPs;
* every gate: Parseval's identity, sum_f P[r, f] = N sum_p sum_k |m_p[s_r + k]|^2, with the
  right-hand side in exact integer arithmetic;
for every radix order the benchmark's autotuner can pick.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import RTOL, assert_parity
from paper_2311_18737_gb300 import isr

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


# every radix order Plan.autotune (and so bench.py) may pick at this workload
ORDERS = list(range(isr.N_ORDERS))


@pytest.fixture(scope="module")
def realistic_inputs():
    w = synth.realistic()
    dev = torch.device("cuda:0")
    code = w.code()
    code_d = torch.from_numpy(code).to(dev)
    echo_d = torch.empty((w.n_ipp, w.echo_stride, 2), dtype=torch.int16, device=dev)
    w.echo_device(echo_d.data_ptr(), code_d.data_ptr())
    echo = echo_d.cpu().numpy()
    rng = np.random.default_rng(77)
    sel = sorted(set([0, 1, 399, 400, 401, w.n_ranges - 2, w.n_ranges - 1]) |
                 set(rng.choice(w.n_ranges, 9, replace=False).tolist()))
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_start=w.range_start,
                           range_step=w.range_step, sel=sel)
    # Parseval's right-hand side per gate, exact in integers: N sum_p sum_k |m_p[s_r + k]|^2
    L, N = w.code_len, w.nfft
    window_power = np.zeros(w.n_ranges, dtype=np.int64)
    starts = w.range_start + np.arange(w.n_ranges) * w.range_step
    for p0 in range(0, w.n_ipp, 500):
        blk = echo[p0:p0 + 500].astype(np.int64)
        pw = blk[..., 0] ** 2 + blk[..., 1] ** 2
        cs = np.concatenate([np.zeros((pw.shape[0], 1), np.int64), np.cumsum(pw, axis=1)], axis=1)
        window_power += (cs[:, starts + L] - cs[:, starts]).sum(axis=0)
    exact = N * window_power.astype(np.float64)
    yield w, code, code_d, echo_d, echo, sel, ref, exact
    del echo_d


def _integrate(inputs, order):
    w, code, code_d, echo_d = inputs[:4]
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    with isr.Plan(nfft=w.nfft, n_ranges=w.n_ranges, echo_stride=w.echo_stride, range_start=w.range_start,
                  range_step=w.range_step, tx_type=isr.ISR_TX_PM1, device=0, stream=stream) as plan:
        isr.isr_plan_set_order(plan.handle, order)
        plan.integrate(echo_d, code_d, w.n_ipp)
        out = torch.empty((w.n_ranges, w.nfft), dtype=torch.float32, device=dev)
        _, n = plan.spectra(out)
        info = plan.info()
    assert n == w.n_ipp
    return out.cpu().numpy().astype(np.float64), info


def test_device_generator_rows_match_host(realistic_inputs):
    w, echo = realistic_inputs[0], realistic_inputs[4]
    for p in (0, 4999, w.n_ipp - 1):
        assert np.array_equal(echo[p], w.echo_host(p, p + 1)[0]), f"row {p} differs"


@pytest.mark.parametrize("order", ORDERS)
def test_sampled_gates_every_bin_and_parseval(realistic_inputs, order):
    w, sel, ref, exact = realistic_inputs[0], realistic_inputs[5], realistic_inputs[6], realistic_inputs[7]
    got, info = _integrate(realistic_inputs, order)
    mx, p99, med = assert_parity(got[sel], ref, rtol=RTOL, what=f"realistic sampled gates, order {order}")
    print(f"realistic workload, order {order}, {len(sel)} gates x {w.nfft} bins: max {mx:.2e} p99 {p99:.2e} "
          f"median {med:.2e}; launch {info}")
    rel = np.abs(got.sum(axis=1) - exact) / exact
    assert rel.max() <= RTOL, f"order {order}: Parseval off by {rel.max():.2e} at gate {int(np.argmax(rel))}"
