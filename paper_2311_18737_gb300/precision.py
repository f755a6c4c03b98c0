"""Precision study: the first FFT pass on the tensor cores (BF16 / FP16, split or single
products, FP32 accumulation; the warp-level mma.sync engine and the tcgen05 engine) next to
the FP32 SIMT path, at the realistic geometry.

For each engine: integration speed, the per-bin relative difference from the FP32 SIMT
engine on sampled gates over all IPPs, and the line position error of the peak fit against
the injected line frequency.  `run` also returns the sampled gates' spectra of every engine,
so that a caller can compare them with a reference computed elsewhere (the test suite does
so against the FP64 oracle).

    python -m paper_2311_18737_gb300.precision --n-ipp 10000 --out precision.json
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import isr


def run(n_ipp: int = 10000, n_sample_gates: int = 8, reps: int = 2, seed: int = 2):
    """Returns (results, inputs): results as printed by the command line; inputs holds what a
    reference needs ("echo", the device tensor int16 [n_ipp][stride][2], "code", the geometry)
    and "spectra", each engine's sampled-gate spectra (float64 [gates][nfft])."""
    import synth

    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    w = synth.realistic(n_ipp=n_ipp, seed=seed)
    code = w.code()
    code_d = torch.from_numpy(code).to(dev)
    echo = torch.empty((n_ipp, w.echo_stride, 2), dtype=torch.int16, device=dev)
    w.echo_device(echo.data_ptr(), code_d.data_ptr())
    R, N = w.n_ranges, w.nfft
    band = (int(1e6 / 50e6 * N) - 8, int(15e6 / 50e6 * N) + 8)
    rng = np.random.default_rng(9)
    sel = sorted(set([0, 400, R - 1]) | set(rng.choice(R, n_sample_gates - 3, replace=False).tolist()))
    truth = w.base_freqs() * N
    out = torch.empty((R, N), dtype=torch.float32, device=dev)
    fb = torch.empty(R, dtype=torch.float64, device=dev)
    sn = torch.empty(R, dtype=torch.float32, device=dev)
    results, spectra = {}, {}
    for mode in (isr.ISR_PREC_FP32, isr.ISR_PREC_TC_BF16_SPLIT, isr.ISR_PREC_TC_FP16_SPLIT, isr.ISR_PREC_TC_BF16,
                 isr.ISR_PREC_TC_FP16, isr.ISR_PREC_TC05_BF16_SPLIT, isr.ISR_PREC_TC05_FP16_SPLIT,
                 isr.ISR_PREC_TC05_BF16, isr.ISR_PREC_TC05_FP16):
        with isr.Plan(nfft=N, n_ranges=R, echo_stride=w.echo_stride, range_start=w.range_start,
                      range_step=w.range_step, tx_type=isr.ISR_TX_PM1, device=0, stream=stream) as plan:
            if mode == isr.ISR_PREC_FP32:
                isr.isr_plan_set_order(plan.handle, 1)   # same radix order as the tensor-core engine
            else:
                isr.isr_plan_set_precision(plan.handle, mode)
            plan.integrate(echo, code_d, n_ipp)
            plan.spectra(out, isr.ISR_RESET_AFTER)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                plan.integrate(echo, code_d, n_ipp)
                plan.spectra(out, isr.ISR_RESET_AFTER)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            plan.integrate(echo, code_d, n_ipp)
            plan.spectra(out)
        isr.isr_peak_fit(out, R, N, band[0], band[1], fb, sn, stream)
        torch.cuda.synchronize()
        P = out.cpu().numpy().astype(np.float64)
        f = fb.cpu().numpy()
        r = {"ms_per_integration": ms, "spectra_per_s": R * n_ipp / (ms / 1e3),
             "line_bin_err_vs_truth": {"median": float(np.median(np.abs(f - truth))),
                                       "max": float(np.max(np.abs(f - truth)))}}
        name = isr.PRECISION_NAMES[mode]
        spectra[name] = P[sel]
        if mode != isr.ISR_PREC_FP32:
            base = spectra[isr.PRECISION_NAMES[isr.ISR_PREC_FP32]]
            rel = np.abs(P[sel] - base) / base
            r["bin_rel_diff_vs_fp32_simt"] = {"max": float(rel.max()), "median": float(np.median(rel))}
        results[name] = r
    res = {"workload": f"{R} gates x nfft {N} x {n_ipp} IPPs (realistic geometry, seed {seed})",
           "sampled_gates": sel, "band_bins": band, "engines": results}
    inputs = {"echo": echo, "code": code, "nfft": N, "n_ranges": R, "range_start": w.range_start,
              "range_step": w.range_step, "sel": sel, "band": band, "spectra": spectra}
    return res, inputs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-ipp", type=int, default=10000)
    ap.add_argument("--gates", type=int, default=8)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res, _ = run(a.n_ipp, a.gates, a.reps)
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
