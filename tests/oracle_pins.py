"""Checks that pin the FP64 oracle to facts other than itself.

Each check takes an oracle-like object (``integrate(...)``, ``fft(...)``) and raises
AssertionError when it disagrees with the mathematics.  The same checks run against the
real oracle (they must pass) and against copies of the oracle with a planted mistake
(at least one must fail).  Nothing here calls the CUDA library.
"""
from __future__ import annotations

import cmath

import numpy as np


def direct_dft(x):
    """Brute-force O(N^2) forward DFT with Python complex arithmetic."""
    n = len(x)
    return np.array([sum(x[k] * cmath.exp(-2j * cmath.pi * f * k / n) for k in range(n))
                     for f in range(n)], dtype=np.complex128)


def brute_integrate(echo, tx, nfft, n_ranges, start, step, code_len, per_ipp_tx):
    """Plain loops: sum_p |sum_k conj(eps_p[k]) m_p[s_r+k] e^{-2 pi i f k/N}|^2."""
    n_ipp = echo.shape[0]
    out = np.zeros((n_ranges, nfft))
    for r in range(n_ranges):
        s = start + r * step
        for p in range(n_ipp):
            row = tx[p] if per_ipp_tx else tx
            x = []
            for k in range(nfft):
                if k < code_len:
                    if row.dtype == np.int8:
                        eps = -1.0 if row[k] < 0 else 1.0
                    else:
                        eps = complex(float(row[k][0]), float(row[k][1]))
                    m = complex(float(echo[p, s + k, 0]), float(echo[p, s + k, 1]))
                    x.append(eps.conjugate() * m if isinstance(eps, complex) else eps * m)
                else:
                    x.append(0j)
            X = direct_dft(x)
            out[r] += np.abs(X) ** 2
    return out


def check_fft_vs_direct(orc, rng, sizes=(1, 2, 4, 8, 16, 64, 256)):
    for n in sizes:
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        got = orc.fft(x)
        ref = direct_dft(list(x))
        scale = max(1.0, np.abs(ref).max())
        assert np.abs(got - ref).max() <= 1e-12 * scale * max(1, n), f"fft mismatch at n={n}"


def check_integrate_vs_brute(orc, rng):
    cases = [
        # nfft, R, P, start, step, code_len, tx kind, per-IPP
        (8, 3, 2, 1, 3, 8, "ci16", False),
        (16, 2, 3, 0, 5, 11, "ci16", True),
        (16, 4, 2, 2, 1, 16, "pm1", False),
        (8, 2, 3, 0, 2, 5, "pm1", True),
        (32, 2, 2, 3, 7, 32, "c32", False),
    ]
    for nfft, R, P, start, step, L, kind, per in cases:
        stride = start + (R - 1) * step + L + 3
        echo = rng.integers(-3000, 3000, size=(P, stride, 2)).astype(np.int16)
        shape = (P, L) if per else (L,)
        if kind == "pm1":
            tx = np.where(rng.random(shape) < 0.5, -1, 1).astype(np.int8)
        elif kind == "ci16":
            tx = rng.integers(-7, 8, size=shape + (2,)).astype(np.int16)
        else:
            tx = rng.standard_normal(shape + (2,)).astype(np.float32)
        got = orc.integrate(echo, tx, nfft=nfft, n_ranges=R, range_start=start, range_step=step,
                            code_len=L, per_ipp_tx=per)
        ref = brute_integrate(echo, tx, nfft, R, start, step, L, per)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-6 * ref.max()), f"integrate mismatch {kind}"


def check_tone_bins(orc):
    """Noise-free tones at exactly representable frequencies land in their bin only."""
    N, A, P = 64, 1000, 3
    code = np.where(np.arange(N) % 3 == 0, -1, 1).astype(np.int8)
    for b, rot in ((N // 4, (0, 1)), (N // 2, (-1, 0)), (3 * N // 4, (0, -1)), (0, (1, 0))):
        # e^{2 pi i b k / N} for b in {0, N/4, N/2, 3N/4} is i^k, (-1)^k, (-i)^k or 1: exact
        k = np.arange(N)
        ph = np.array([complex(*rot) ** kk for kk in k])
        sig = A * code.astype(np.float64) * ph
        echo = np.zeros((P, N + 10, 2), dtype=np.int16)
        echo[:, 5:5 + N, 0] = np.rint(sig.real).astype(np.int16)
        echo[:, 5:5 + N, 1] = np.rint(sig.imag).astype(np.int16)
        out = orc.integrate(echo, code, nfft=N, n_ranges=1, range_start=5, range_step=1)
        peak = P * (A * N) ** 2
        assert abs(out[0, b] - peak) <= 1e-9 * peak, f"tone power wrong at bin {b}"
        others = np.delete(out[0], b)
        assert others.max() <= 1e-18 * peak * N, f"tone leaked out of bin {b}"


def check_conj_with_complex_code(orc):
    """A complex code e^{-2 pi i b k/N} on a constant echo decodes to a tone at +b."""
    N, b, A = 128, 19, 500
    k = np.arange(N)
    eps = np.exp(-2j * np.pi * b * k / N)
    tx = np.stack([eps.real, eps.imag], -1).astype(np.float32)
    echo = np.zeros((1, N, 2), dtype=np.int16)
    echo[0, :, 0] = A
    out = orc.integrate(echo, tx, nfft=N, n_ranges=1, range_start=0, range_step=1)
    assert int(np.argmax(out[0])) == b, "conjugation or sign convention wrong"
    assert out[0, b] > 0.999 * (A * N) ** 2


def check_parseval(orc, echo, code, nfft, R, start, step):
    """sum_f P[r, f] = N sum_p sum_k |m_p[s_r + k]|^2 for a +-1 code (exact integers)."""
    out = orc.integrate(echo, code, nfft=nfft, n_ranges=R, range_start=start, range_step=step)
    e = echo.astype(np.int64)
    pw = e[..., 0] ** 2 + e[..., 1] ** 2
    L = code.shape[-1]
    for r in range(R):
        s = start + r * step
        exact = nfft * int(pw[:, s:s + L].sum())
        assert abs(out[r].sum() - exact) <= 1e-11 * exact, f"Parseval fails at gate {r}"


def check_delay(orc):
    """A coded echo at delay d decodes coherently (DC bin) only at the gate s_r = d."""
    N, L, A = 64, 64, 100
    rng = np.random.default_rng(7)
    code = np.where(rng.random(L) < 0.5, -1, 1).astype(np.int8)
    d = 3 * 4 + 1
    echo = np.zeros((2, 200, 2), dtype=np.int16)
    echo[:, d:d + L, 0] = A * code.astype(np.int16)
    out = orc.integrate(echo, code, nfft=N, n_ranges=20, range_start=1, range_step=4)
    g = int(np.argmax(out[:, 0]))
    assert 1 + 4 * g == d, "decode picked the wrong range gate"
    assert abs(out[g, 0] - 2 * (A * L) ** 2) <= 1e-9 * out[g, 0]


def check_additivity(orc, echo, code, nfft, R, start, step):
    full = orc.integrate(echo, code, nfft=nfft, n_ranges=R, range_start=start, range_step=step)
    a = echo.shape[0] // 3
    part = orc.integrate(echo[:a], code, nfft=nfft, n_ranges=R, range_start=start, range_step=step)
    orc.integrate(echo[a:], code, nfft=nfft, n_ranges=R, range_start=start, range_step=step, out=part)
    assert np.allclose(part, full, rtol=1e-12), "integration is not additive over IPPs"


ALL_CHEAP = ("fft", "brute", "tone", "conj", "delay")


def run_cheap_pins(orc, rng):
    check_fft_vs_direct(orc, rng, sizes=(1, 2, 8, 32))
    check_integrate_vs_brute(orc, rng)
    check_tone_bins(orc)
    check_conj_with_complex_code(orc)
    check_delay(orc)
