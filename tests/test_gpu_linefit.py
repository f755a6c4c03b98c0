"""GPU peak fit (isr_peak_fit through the C ABI) against the FP64 peak-fit oracle."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import gpu_integrate
from oracle import linefit
from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu


def _gpu_fit(P, lo, hi):
    dev = torch.device("cuda:0")
    Pd = torch.from_numpy(np.ascontiguousarray(P, dtype=np.float32)).to(dev)
    R, N = P.shape
    f = torch.empty(R, dtype=torch.float64, device=dev)
    s = torch.empty(R, dtype=torch.float32, device=dev)
    isr.isr_peak_fit(Pd, R, N, lo, hi, f, s, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return f.cpu().numpy(), s.cpu().numpy().astype(np.float64)


def test_random_spectra_with_peaks_and_ties():
    rng = np.random.default_rng(3)
    R, N = 300, 4096
    P = rng.gamma(50.0, 1.0, size=(R, N)).astype(np.float32)
    c = rng.uniform(400, 3600, R)
    f = np.arange(N)
    P += (300.0 * np.exp(-((f[None, :] - c[:, None]) ** 2) / 4.0)).astype(np.float32)
    P[7, 1000] = P[7, 1500] = 1e6          # tie
    P[8, :] = 3.0                          # flat
    got_f, got_s = _gpu_fit(P, 300, 3800)
    ref_f, ref_s = linefit.peak_fit(P, 300, 3800)
    assert np.abs(got_f - ref_f).max() <= 1e-9
    assert np.abs(got_s - ref_s).max() <= 1e-6 * np.abs(ref_s).max()


def test_fit_of_integrated_tones():
    w = synth.small(n_ipp=30, snap_to_bins=True)
    echo, code = w.echo_host(), w.code()
    P, _ = gpu_integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_step=w.range_step)
    got_f, _ = _gpu_fit(P, 0, w.nfft)
    ref_f, _ = linefit.peak_fit(P, 0, w.nfft)
    assert np.abs(got_f - ref_f).max() <= 1e-9
    true_bin = np.mod(np.round(w.base_freqs() * w.nfft), w.nfft)
    assert np.abs(got_f - true_bin).max() <= 0.5
