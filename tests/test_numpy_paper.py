"""The paper-style NumPy implementation (the paper's CPU comparison, Sec. 3.3) against the FP64
oracle: two independent CPU implementations of Eqs. 7-8 must agree to double rounding."""
import numpy as np
import pytest

import oracle
import synth
from oracle import numpy_paper


def _rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def test_small_workload_matches_oracle():
    w = synth.small(n_ipp=6)
    echo, code = w.echo_host(), w.code()
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_start=w.range_start,
                           range_step=w.range_step)
    got = numpy_paper.integrate(echo, code, w.nfft, w.n_ranges, w.range_start, w.range_step)
    assert _rel(got, ref) < 1e-10


@pytest.mark.parametrize("kind", ["pm1", "ci16", "c32"])
@pytest.mark.parametrize("per_ipp", [False, True])
def test_code_formats_and_padding(kind, per_ipp):
    rng = np.random.default_rng(11)
    nfft, L, R, P, start, step = 64, 40, 5, 3, 3, 7
    stride = start + (R - 1) * step + L + 5
    echo = rng.integers(-3000, 3000, size=(P, stride, 2), dtype=np.int16)
    rows = P if per_ipp else 1
    if kind == "pm1":
        tx, t = rng.choice(np.array([-1, 1], dtype=np.int8), size=(rows, L)), numpy_paper.TX_PM1
    elif kind == "ci16":
        tx, t = rng.integers(-200, 200, size=(rows, L, 2), dtype=np.int16), numpy_paper.TX_CI16
    else:
        tx, t = rng.standard_normal((rows, L, 2)).astype(np.float32), numpy_paper.TX_C32
    otx = tx if per_ipp else tx[0]
    ref = oracle.integrate(echo, otx, nfft=nfft, n_ranges=R, range_start=start, range_step=step,
                           per_ipp_tx=per_ipp)
    got = numpy_paper.integrate(echo, tx, nfft, R, start, step, code_len=L, tx_type=t, per_ipp_code=per_ipp)
    assert _rel(got, ref) < 1e-10


def test_selected_gates():
    w = synth.small(n_ipp=3)
    echo, code = w.echo_host(), w.code()
    sel = [0, 31, 63]
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step, sel=sel)
    got = numpy_paper.integrate(echo, code, w.nfft, w.n_ranges, 0, w.range_step, gates=sel)
    assert _rel(got, ref) < 1e-10
