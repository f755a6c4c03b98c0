"""The seeded input generator (host build): Philox known answers and the sample model."""
import numpy as np
from scipy import stats

import synth


def test_philox4x32_10_known_answers():
    # known-answer vectors published with the Random123 library (Salmon et al., SC'11)
    assert synth.philox4x32_10([0, 0, 0, 0], 0) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert synth.philox4x32_10([0xFFFFFFFF] * 4, 0xFFFFFFFFFFFFFFFF) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                               0x299F31D0A4093822) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_phase_table_matches_exponential():
    t = synth.phase_table().reshape(-1, 2)
    j = np.arange(t.shape[0])
    ref = np.exp(2j * np.pi * j / t.shape[0])
    err = np.abs(t[:, 0] + 1j * t[:, 1] - ref).max()
    assert err < 1.2e-7


def test_noise_is_circular_gaussian():
    w = synth.small(kind=synth.NOISE_ONLY, n_ipp=8, seed=5)
    e = w.echo_host().astype(np.float64)
    var = w.sigma ** 2 + 1.0 / 12.0
    for comp in (0, 1):
        x = e[..., comp].ravel()
        assert abs(x.var() / var - 1) < 4 * np.sqrt(2.0 / x.size)
        assert abs(x.mean()) < 4 * np.sqrt(var / x.size)
        assert stats.kstest(x[::7] / np.sqrt(var), "norm").pvalue > 1e-3
    assert abs(np.corrcoef(e[..., 0].ravel(), e[..., 1].ravel())[0, 1]) < 0.01


def test_deterministic_and_row_addressable():
    w = synth.small(n_ipp=6)
    a = w.echo_host()
    b = w.echo_host(2, 5)
    assert np.array_equal(a[2:5], b)
    assert np.array_equal(a, w.echo_host(n_threads=1))


def test_code_is_binary_phase():
    w = synth.realistic()
    c = w.code()
    assert c.shape == (16384,) and set(np.unique(c)) == {-1, 1}
    assert abs(int(c.astype(np.int64).sum())) < 5 * np.sqrt(c.size)


def test_line_frequencies_follow_chapman_profile():
    w = synth.realistic()
    f_hz = w.base_freqs() * w.fs_hz
    assert int(np.argmax(f_hz)) == 400
    assert abs(f_hz.max() - 15e6) < 1.0 and f_hz.min() >= 1e6
