"""Plain FP64 peak fit of integrated spectra (test infrastructure only).

The plasma line's frequency follows the electron density (the paper's Eq. 1, f_p grows as
sqrt(n_e)), so each gate's integrated spectrum is reduced to a line position: the largest
bin of the band, refined by a three-point parabola through ln P (the standard quadratic
peak interpolation; exact for a Gaussian-shaped peak), and the ratio of the peak to the
band's mean power.  Written out gate by gate with numpy in double precision; the argmax
compares float32 values, as the spectra are float32.
"""
from __future__ import annotations

import math

import numpy as np


def peak_fit(P, band_lo: int, band_hi: int):
    """Returns (freq_bin [R] float64, snr [R] float64) for spectra P [R, N]."""
    P32 = np.asarray(P, dtype=np.float32)
    R, N = P32.shape
    freq = np.zeros(R)
    snr = np.zeros(R)
    for r in range(R):
        band = P32[r, band_lo:band_hi]
        b = band_lo + int(np.argmax(band))          # first index of the maximum
        mean = float(np.sum(band.astype(np.float64))) / (band_hi - band_lo)
        pm, p0, pp = float(P32[r, (b - 1) % N]), float(P32[r, b]), float(P32[r, (b + 1) % N])
        delta = 0.0
        if pm > 0 and p0 > 0 and pp > 0:
            ym, y0, yp = math.log(pm), math.log(p0), math.log(pp)
            d = ym - 2.0 * y0 + yp
            if d < 0:
                delta = 0.5 * (ym - yp) / d
            delta = min(0.5, max(-0.5, delta))
        freq[r] = b + delta
        snr[r] = p0 / mean if mean > 0 else 0.0
    return freq, snr
