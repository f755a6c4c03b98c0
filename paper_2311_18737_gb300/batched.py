"""Batched uneven integration windows: workload, batched run and per-window comparison.

Workload (the batched-windows configuration): 32 windows, transform length drawn from
{2048, 4096, 8192, 16384}, gate counts uniform in 100..1500, IPP counts uniform in
500..5000, gate step 25, binary-phase codes; even windows carry the up-shifted plasma
line channel (line at +f_r), odd windows the down-shifted one (line at -f_r, Sec. 2.1 of
the paper), each a Chapman-layer Langmuir line at SNR -20 dB, all from the seeded
synthetic generator.  The batched run (one persistent launch, optionally replayed from a
CUDA graph, radix orders optionally autotuned) is compared with one plan per window.

    python -m paper_2311_18737_gb300.batched --out batched.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import isr

NFFTS = (2048, 4096, 8192, 16384)


def config_windows(seed: int = 3, n_windows: int = 32, ipp_scale: float = 1.0, max_gates: int = 1500):
    """Shapes and generator settings of the batched workload (no buffers yet)."""
    import synth

    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_windows):
        nfft = int(rng.choice(NFFTS))
        R = int(rng.integers(100, max_gates + 1))
        P = max(1, int(round(int(rng.integers(500, 5001)) * ipp_scale)))
        w = synth.realistic(seed=int(rng.integers(1, 2**62)), n_ranges=R, n_ipp=P)
        w.nfft = w.code_len = nfft
        w.echo_stride = ((R - 1) * w.range_step + nfft + 127) // 128 * 128
        w.name = f"window {i} ({'down' if i % 2 else 'up'}-shifted)"
        f = w.base_freqs() if w.gate_freq is None else w.gate_freq
        w.gate_freq = -f if i % 2 else f
        out.append(w)
    return out


class Buffers:
    """Device echo, code and output of every window (echo generated on the device)."""

    def __init__(self, workloads, device: int = 0):
        self.dev = torch.device("cuda", device)
        self.w = workloads
        self.echo, self.code, self.out = [], [], []
        for w in workloads:
            code = torch.from_numpy(w.code()).to(self.dev)
            echo = torch.empty((w.n_ipp, w.echo_stride, 2), dtype=torch.int16, device=self.dev)
            w.echo_device(echo.data_ptr(), code.data_ptr())
            self.echo.append(echo)
            self.code.append(code)
            self.out.append(torch.empty((w.n_ranges, w.nfft), dtype=torch.float32, device=self.dev))

    def windows(self, order: int = -1):
        ws = []
        for w, e, c, o in zip(self.w, self.echo, self.code, self.out):
            x = isr.IsrWindow()
            x.echo, x.tx_code, x.out = e.data_ptr(), c.data_ptr(), o.data_ptr()
            x.echo_stride, x.tx_stride = w.echo_stride, 0
            x.nfft, x.code_len, x.n_ranges = w.nfft, w.code_len, w.n_ranges
            x.range_start, x.range_step, x.n_ipp = w.range_start, w.range_step, w.n_ipp
            x.order, x.reserved = order, 0
            ws.append(x)
        return ws


class Batch:
    def __init__(self, bufs: Buffers, flags: int = isr.ISR_BATCH_GRAPH, order: int = -1, stream=None):
        self.stream = stream if stream is not None else torch.cuda.current_stream(bufs.dev)
        self.h = isr.isr_batch_create(bufs.windows(order), flags, bufs.dev.index, self.stream)

    def run(self, wait: bool = True):
        isr.isr_batch_run(self.h)
        if wait:
            isr.isr_batch_wait(self.h)

    def info(self):
        return isr.isr_batch_query(self.h).as_dict()

    def close(self):
        if self.h:
            isr.isr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def per_window(bufs: Buffers, outs=None, stream=None):
    """The same windows through one plan each, created and destroyed per call."""
    stream = stream if stream is not None else torch.cuda.current_stream(bufs.dev)
    outs = outs if outs is not None else [torch.empty_like(o) for o in bufs.out]
    for w, e, c, o in zip(bufs.w, bufs.echo, bufs.code, outs):
        with isr.Plan(nfft=w.nfft, n_ranges=w.n_ranges, echo_stride=w.echo_stride, range_start=w.range_start,
                      range_step=w.range_step, tx_type=isr.ISR_TX_PM1, device=bufs.dev.index, stream=stream) as p:
            p.integrate(e, c, w.n_ipp)
            p.spectra(o)
    return outs


class PerWindowPlans:
    """The same windows through one plan each, the plans created once and kept (what a caller
    without batching does): a run integrates every window, then reads every window's spectra.
    ``orders`` maps nfft to the radix order the plans use (the batch's autotuned orders)."""

    def __init__(self, bufs: Buffers, orders=None, stream=None):
        self.bufs = bufs
        self.stream = stream if stream is not None else torch.cuda.current_stream(bufs.dev)
        self.plans = []
        for w in bufs.w:
            p = isr.Plan(nfft=w.nfft, n_ranges=w.n_ranges, echo_stride=w.echo_stride, range_start=w.range_start,
                         range_step=w.range_step, tx_type=isr.ISR_TX_PM1, device=bufs.dev.index, stream=self.stream)
            if orders and orders.get(w.nfft):
                isr.isr_plan_set_order(p.handle, orders[w.nfft])
            self.plans.append(p)

    def run(self, outs):
        for p, w, e, c in zip(self.plans, self.bufs.w, self.bufs.echo, self.bufs.code):
            p.integrate(e, c, w.n_ipp)
        for p, o in zip(self.plans, outs):
            p.spectra(o, isr.ISR_RESET_AFTER)

    def close(self):
        for p in self.plans:
            p.close()
        self.plans = []


def _timed(fn, reps):
    """(mean ms per call by CUDA events on the current stream, mean wall ms per call)."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record()
    for _ in range(reps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    wall = 1000 * (time.perf_counter() - t0) / reps
    return ev0.elapsed_time(ev1) / reps, wall


def bench(ipp_scale: float = 1.0, reps: int = 2, seed: int = 3):
    ws = config_windows(seed=seed, ipp_scale=ipp_scale)
    t0 = time.time()
    bufs = Buffers(ws)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    transforms = sum(w.n_ranges * w.n_ipp for w in ws)
    t0 = time.time()
    b = Batch(bufs, flags=isr.ISR_BATCH_GRAPH | isr.ISR_BATCH_AUTOTUNE)
    create_s = time.time() - t0
    b.run()

    def run_batched():
        b.run(wait=False)
        isr.isr_batch_wait(b.h)

    batched_ms, batched_wall = _timed(run_batched, reps)
    # fair baseline: per-window plans created once, before timing, with the batch's radix orders
    binfo = b.info()
    orders = dict(zip((2048, 4096, 8192, 16384), binfo["order"]))
    pw = PerWindowPlans(bufs, orders)
    outs = [torch.empty_like(o) for o in bufs.out]
    pw.run(outs)
    reused_ms, reused_wall = _timed(lambda: pw.run(outs), reps)
    pw.close()
    # context: plans created and destroyed inside every run
    outs2 = per_window(bufs)
    create_ms, create_wall = _timed(lambda: per_window(bufs, outs2), reps)
    diff = max(float(((o - r).abs() / r.abs().clamp_min(1e-30)).max()) for o, r in zip(bufs.out, outs))
    res = {"windows": [{"nfft": w.nfft, "gates": w.n_ranges, "ipps": w.n_ipp,
                        "channel": "down" if i % 2 else "up"} for i, w in enumerate(ws)],
           "transforms": transforms,
           "batched_ms": batched_ms, "batched_wall_ms": batched_wall,
           "per_window_ms": reused_ms, "per_window_wall_ms": reused_wall,
           "per_window_create_each_run_ms": create_ms, "per_window_create_each_run_wall_ms": create_wall,
           "batched_spectra_per_s": transforms / (batched_ms / 1e3),
           "per_window_spectra_per_s": transforms / (reused_ms / 1e3),
           "speedup": reused_ms / batched_ms,
           "speedup_vs_plans_created_each_run": create_ms / batched_ms,
           "max_rel_diff_batched_vs_per_window": diff,
           "batch": binfo, "generation_s": gen_s, "create_s": create_s, "reps": reps}
    b.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ipp-scale", type=float, default=1.0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = bench(a.ipp_scale, a.reps)
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)


if __name__ == "__main__":
    main()
