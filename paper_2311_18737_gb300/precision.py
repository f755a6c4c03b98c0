"""Precision study: the first FFT pass on the tensor cores (BF16 / FP16, split or single
products, FP32 accumulation) next to the FP32 SIMT path, at the realistic geometry.

For each engine: integration speed, the per-bin relative error against the FP64 oracle on
sampled gates over all IPPs, and the line position error of the peak fit (against the
peak fit of the oracle's spectra, and against the injected line frequency).

    python -m paper_2311_18737_gb300.precision --n-ipp 10000 --out precision.json
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import isr


def run(n_ipp: int = 10000, n_sample_gates: int = 8, reps: int = 2, seed: int = 2, with_oracle: bool = True):
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
    ref = None
    if with_oracle:
        import oracle
        host = echo.cpu().numpy()
        ref = oracle.integrate(host, code, nfft=N, n_ranges=R, range_start=w.range_start, range_step=w.range_step,
                               sel=sel)
        del host
    truth = w.base_freqs() * N
    out = torch.empty((R, N), dtype=torch.float32, device=dev)
    fb = torch.empty(R, dtype=torch.float64, device=dev)
    sn = torch.empty(R, dtype=torch.float32, device=dev)
    results = {}
    for mode in (isr.ISR_PREC_FP32, isr.ISR_PREC_TC_BF16_SPLIT, isr.ISR_PREC_TC_FP16_SPLIT, isr.ISR_PREC_TC_BF16,
                 isr.ISR_PREC_TC_FP16):
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
        if ref is not None:
            from oracle import linefit
            rel = np.abs(P[sel] - ref) / ref
            fo, _ = linefit.peak_fit(ref, band[0], band[1])
            fm, _ = linefit.peak_fit(P[sel], band[0], band[1])
            r["bin_rel_err_vs_fp64_oracle"] = {"max": float(rel.max()), "p99": float(np.quantile(rel, 0.99)),
                                               "median": float(np.median(rel))}
            r["line_bin_err_vs_oracle_peak_fit"] = float(np.max(np.abs(fm - fo)))
        results[isr.PRECISION_NAMES[mode]] = r
    return {"workload": f"{R} gates x nfft {N} x {n_ipp} IPPs (realistic geometry, seed {seed})",
            "sampled_gates": sel, "band_bins": band, "engines": results}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-ipp", type=int, default=10000)
    ap.add_argument("--gates", type=int, default=8)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.n_ipp, a.gates, a.reps, with_oracle=not a.no_oracle)
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
