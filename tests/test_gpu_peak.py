"""The measured FP32 FMA rate (the integrate kernel's roofline denominator) against the
derived peak: SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock; the measured tcgen05 rate per
MMA shape (the estimator convolutions' tensor roofline) against the nominal dense BF16 rate."""
import pytest

torch = pytest.importorskip("torch")

from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu


def test_fp32_peak_matches_derived_peak():
    props = torch.cuda.get_device_properties(0)
    derived = props.multi_processor_count * 128 * 2 * 2070e6 / 1e12
    ffma, ms = isr.isr_fp32_peak(0, False)
    assert ms > 0
    # at most the derived rate (plus timing noise), at least half of it (clock may drop under load)
    assert 0.5 * derived < ffma < 1.05 * derived
    # pairing two FMAs per instruction does not raise the lane rate beyond the derived peak
    ffma2, _ = isr.isr_fp32_peak(0, True)
    assert 0.5 * derived < ffma2 < 1.05 * derived


def test_tc05_rate_by_shape():
    """M = 128, K = 16 BF16 MMAs: the N = 256 shape runs near the nominal dense rate (2.25
    PFLOP/s for the full part at its boost clock; at most 8192 FLOP per SM and cycle), narrower
    shapes no faster in FLOP/s and no slower per instruction than N = 256."""
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 8192 * 2070e6 / 1e12
    rates = {n: isr.isr_tc05_rate(n) for n in (32, 64, 128, 256)}
    for n, (tf, cyc) in rates.items():
        assert 0 < tf < 1.05 * ceiling, (n, tf)
        assert cyc > 0
    assert rates[256][0] > 0.5 * ceiling
    assert rates[32][0] <= rates[256][0] * 1.05
    assert rates[32][1] <= rates[256][1] * 1.05
