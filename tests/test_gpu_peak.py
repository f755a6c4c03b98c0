"""The measured FP32 FMA rate (the integrate kernel's roofline denominator) against the
derived peak: SMs x 128 FP32 lanes x 2 FLOP x the maximum SM clock."""
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
