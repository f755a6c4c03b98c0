"""Pins of the FP64 oracle (CPU only).

The paper prints no spectra, so the oracle is pinned to the mathematics: brute-force
DFTs on tiny inputs, a library FFT at full length, Parseval's identity in exact integer
arithmetic, exactly representable tones, the conjugate-code convention, the range-gate
delay, additivity over IPPs and the noise floor of circular Gaussian noise.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import oracle_pins as pins
import synth


def test_fft_matches_brute_force_dft():
    pins.check_fft_vs_direct(oracle, np.random.default_rng(0))


def test_fft_matches_numpy_at_16384():
    # library special case: numpy's FFT (the paper's CPU path used NumPy)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(16384) + 1j * rng.standard_normal(16384)
    ref = np.fft.fft(x)
    got = oracle.fft(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_integrate_matches_brute_force():
    pins.check_integrate_vs_brute(oracle, np.random.default_rng(2))


def test_exact_tones_land_in_their_bins():
    pins.check_tone_bins(oracle)


def test_complex_code_is_conjugated():
    pins.check_conj_with_complex_code(oracle)


def test_delay_selects_the_right_gate():
    pins.check_delay(oracle)


@pytest.fixture(scope="module")
def small_workload():
    w = synth.small(n_ipp=20)
    return w, w.echo_host(), w.code()


def test_parseval_exact(small_workload):
    w, echo, code = small_workload
    pins.check_parseval(oracle, echo, code, w.nfft, w.n_ranges, w.range_start, w.range_step)


def test_additivity(small_workload):
    w, echo, code = small_workload
    pins.check_additivity(oracle, echo, code, w.nfft, 8, w.range_start, w.range_step)


def test_selected_gates_equal_full_rows(small_workload):
    w, echo, code = small_workload
    full = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    sel = [0, 17, 63]
    part = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step,
                            sel=sel)
    assert np.array_equal(part, full[sel])


def test_tone_gate_peaks_at_its_frequency(small_workload):
    w, echo, code = small_workload
    out = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    f = w.base_freqs()
    for r in (0, 31, 63):
        b = int(round(f[r] * w.nfft)) % w.nfft
        assert abs(int(np.argmax(out[r])) - b) <= 1


def test_noise_floor():
    # circular Gaussian noise, sigma per component, rounded to int16: per-sample variance
    # per component sigma^2 + 1/12; a +-1 code keeps it white, so every bin of one IPP is
    # exponential with mean N * 2 (sigma^2 + 1/12) and the IPP sum is Gamma(P).
    w = synth.small(kind=synth.NOISE_ONLY, n_ipp=40, seed=11)
    echo, code = w.echo_host(), w.code()
    out = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    P, N = w.n_ipp, w.nfft
    mean = P * N * 2 * (w.sigma ** 2 + 1.0 / 12.0)
    # the bin mean of a gate is its window's sample power (Parseval), and the windows of
    # neighbouring gates share samples, so the standard error follows the number of
    # distinct samples: |m|^2 of a circular Gaussian sample has std equal to its mean.
    unique = P * ((w.n_ranges - 1) * w.range_step + w.code_len)
    se = mean / np.sqrt(unique)
    assert abs(out.mean() - mean) <= 4 * se
    # distribution of one gate's bins (independent within a transform): Gamma(P, mean / P)
    z = out[::9].ravel() / (mean / P)
    assert stats.kstest(z, stats.gamma(a=P).cdf).pvalue > 1e-3


def test_bad_arguments_rejected():
    echo = np.zeros((1, 40, 2), np.int16)
    code = np.ones(16, np.int8)
    with pytest.raises(ValueError):
        oracle.integrate(echo, code, nfft=12, n_ranges=1)          # not a power of two
    with pytest.raises(ValueError):
        oracle.integrate(echo, code, nfft=16, n_ranges=2, range_step=30)  # window overruns row
