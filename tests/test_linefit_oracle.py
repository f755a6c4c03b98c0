"""Pins of the FP64 peak fit: exact recovery of a Gaussian peak's centre (ln P is a
parabola), first-index tie breaking, band restriction, wrap-around neighbours."""
import numpy as np

from oracle import linefit


def test_gaussian_peak_centre_recovered_exactly():
    N = 4096
    f = np.arange(N)
    for c in (1000.0, 1000.37, 2047.5, 3000.9):
        P = 5e6 * np.exp(-((f - c) ** 2) / (2 * 3.0 ** 2)) + 0.0
        P = np.maximum(P, 1e-30)
        got, _ = linefit.peak_fit(P[None, :].astype(np.float32), 500, 3500)
        # float32 rounding of P limits the recovery to ~1e-5 bin
        assert abs(got[0] - c) < 2e-4, (c, got[0])


def test_ties_take_lowest_index_and_band_limits():
    P = np.ones((1, 64), np.float32)
    P[0, 10] = P[0, 20] = 7.0
    P[0, 50] = 100.0                    # outside the band
    got, snr = linefit.peak_fit(P, 5, 40)
    assert got[0] == 10.0               # flat neighbours: delta = 0... (1,7,1) parabola is symmetric
    band = P[0, 5:40].astype(np.float64)
    assert abs(snr[0] - 7.0 / band.mean()) < 1e-12


def test_wraparound_neighbour():
    P = np.full((1, 32), 1.0, np.float32)
    P[0, 0], P[0, 31], P[0, 1] = 9.0, 4.0, 2.0
    got, _ = linefit.peak_fit(P, 0, 8)
    ym, y0, yp = np.log(4.0), np.log(9.0), np.log(2.0)
    assert abs(got[0] - 0.5 * (ym - yp) / (ym - 2 * y0 + yp)) < 1e-12
