"""Plant mistakes in copies of the oracle (on the CPU) and check that the pins catch them.

Each mutation is a plausible slip: a dropped conjugate, a flipped exponent sign, an
off-by-one window, swapped I and Q, a dropped term of |X|^2, a wrong twiddle index,
a per-IPP code read from the wrong row, '=' instead of '+=', non-zero padding.
"""
import numpy as np
import pytest

import oracle
import oracle_pins as pins

MUTATIONS = {
    "no_conj": [("re[k] = er * mr + ei * mi;", "re[k] = er * mr - ei * mi;"),
                ("im[k] = er * mi - ei * mr;", "im[k] = er * mi + ei * mr;")],
    "exp_sign": [("double a = -2.0 * ORC_PI", "double a = 2.0 * ORC_PI")],
    "window_off_by_one": [("echo + 2 * ((int64_t)p * echo_stride + s_r)",
                           "echo + 2 * ((int64_t)p * echo_stride + s_r + 1)")],
    "iq_swapped": [("double mr = (double)m[2 * k], mi = (double)m[2 * k + 1];",
                    "double mi = (double)m[2 * k], mr = (double)m[2 * k + 1];")],
    "dropped_im_power": [("Pr[f] += re[f] * re[f] + im[f] * im[f];", "Pr[f] += re[f] * re[f];")],
    "twiddle_index": [("wr[k * tstep], ci = wi[k * tstep]", "wr[k], ci = wi[k]")],
    "tx_row": [("(size_t)((int64_t)p * tx_stride) * cb", "(size_t)0")],
    "assign_not_add": [("Pr[f] += re[f]", "Pr[f] = re[f]")],
    "pad_nonzero": [("re[k] = 0.0;\n                    im[k] = 0.0;",
                     "re[k] = 1.0;\n                    im[k] = 0.0;")],
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name):
    src = oracle.source_text()
    for old, new in MUTATIONS[name]:
        assert old in src, f"mutation anchor missing for {name}: {old!r}"
        src = src.replace(old, new)
    mutant = oracle.load_variant(src, f"mut_{name}")
    with pytest.raises(AssertionError):
        pins.run_cheap_pins(mutant, np.random.default_rng(3))


def test_unmutated_copy_passes():
    clean = oracle.load_variant(oracle.source_text(), "clean_copy")
    pins.run_cheap_pins(clean, np.random.default_rng(3))
