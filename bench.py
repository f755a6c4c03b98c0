"""Benchmark: range-gate spectra per second of the fused integrator at nfft = 16384.

A step is one integration of the realistic workload through the C ABI: isr_integrate
over all IPPs (decode -> FFT -> |X|^2 accumulate, chunk reduction) followed by
isr_spectra into a device buffer.  The echo is generated on the device before timing
(1.66 GB of int16 IQ, larger than L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--scaling weak|strong]

N > 1 runs one process per GPU under torch.distributed.run (bench.py re-launches itself
that way when started directly with --gpus N; under a launcher whose world size differs
from N it exits with status 2).  --scaling weak (default): every rank integrates its own
problem of the full size (independent gate blocks with their own seeds; no data-path
collective).  --scaling strong: the ranks split ONE workload's gates into contiguous
blocks, each rank keeps only the echo samples its gates read, and the [R_g][nfft] blocks
are gathered to rank 0 at the end of every step.  Rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on host cores on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "range-gate spectra/sec (nfft=16384)"
UNIT = "spectra/s"
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM
# sources that define the fused kernel and its launch (the recorded DRAM traffic is tied to them)
TRAFFIC_SOURCES = ("isr_fft.cuh", "isr_kernel.cuh", "isr_tc.cuh", "isr_tc05.cuh", "isr_tmem.cuh", "isr_paired.cuh",
                   "isr_kernels.cuh", "isr_k_16384.cu", "isr_api.cu")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def _workload(name, rank, n_ranges=None, n_ipp=None):
    import synth
    kw = {}
    if n_ranges:
        kw["n_ranges"] = n_ranges
    if n_ipp:
        kw["n_ipp"] = n_ipp
    if name == "small":
        w = synth.small(seed=1 + 1000 * rank, **kw)
    elif name == "paper":
        w = synth.paper(seed=3 + 1000 * rank, **kw)
    else:
        w = synth.realistic(seed=2 + 1000 * rank, **kw)
    if n_ranges and name != "paper":
        # minimal echo row for the gate count, rounded up to 128 samples
        need = w.range_start + (w.n_ranges - 1) * w.range_step + w.code_len
        w.echo_stride = (need + 127) // 128 * 128
    if n_ranges or n_ipp:
        w.name += " (resized)"
    return w


def _workload_desc(w):
    return (f"{w.name}: {w.n_ranges} gates x nfft {w.nfft} x {w.n_ipp} IPPs, gate step {w.range_step}, "
            f"echo row {w.echo_stride} int16 IQ samples, binary-phase code {w.code_len}, "
            f"{'Langmuir lines' if w.kind == 2 else 'tones'} at SNR {w.snr_db:g} dB per gate")


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.fh = None

    def start(self):
        try:
            self.fh = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", self.gpu_id], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.seek(0)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.fh:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        busy = [s for s, p in zip(sm, power) if p > 0.25 * max(power)] if power else sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def _gpu_selector(torch, dev_index):
    try:
        u = str(torch.cuda.get_device_properties(dev_index).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev_index] if vis else str(dev_index)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(values, device, world, use_dist=None):
    """Element-wise maximum of per-rank timings (no-op without a process group)."""
    if not (world > 1 if use_dist is None else use_dist):
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_throughput(world, n_ranges, n_ipp, ms, strong=False):
    """Whole-job spectra/s; the job takes the slowest rank's time.  Weak scaling: every rank
    integrates its own n_ranges x n_ipp problem.  Strong scaling: n_ranges is the one
    workload's gate count, split over the ranks."""
    return (1 if strong else world) * n_ranges * n_ipp / (ms / 1000.0)


def world_check(gpus, world, launched):
    """What to do with --gpus N given the launcher's world size: "run" (they agree),
    "relaunch" (started directly with N > 1: re-run under torch.distributed.run) or "error"
    (a launcher started a different number of ranks)."""
    if gpus < 1:
        return "error"
    if gpus == world:
        return "run"
    if world == 1 and not launched and gpus > 1:
        return "relaunch"
    return "error"


def _relaunch(gpus):
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def _cpu_sample(w, n_gates, n_ipp, threads):
    """Time the FP64 oracle on n_gates gates (spread over the workload) x n_ipp IPPs."""
    import numpy as np

    import oracle
    echo = w.echo_host(0, n_ipp, n_threads=threads)
    code = w.code()
    sel = np.unique(np.linspace(0, w.n_ranges - 1, n_gates).astype(np.int32))
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.integrate(echo, code, nfft=w.nfft, n_ranges=w.n_ranges, range_start=w.range_start,
                           range_step=w.range_step, sel=sel, n_threads=threads)
    dt = time.perf_counter() - t0
    return len(sel) * n_ipp / dt, len(sel), dt, ref, sel


def _numpy_sample(w, n_gates, n_ipp):
    """Time the paper-style NumPy implementation (the paper's CPU comparison: per IPP a decoded
    batch, numpy.fft.fft per row, |X|^2 added; one core) on n_gates gates x n_ipp IPPs."""
    import numpy as np

    from oracle import numpy_paper
    echo = w.echo_host(0, n_ipp)
    code = w.code()
    sel = np.unique(np.linspace(0, w.n_ranges - 1, n_gates).astype(np.int64))
    t0 = time.perf_counter()
    numpy_paper.integrate(echo, code, w.nfft, w.n_ranges, w.range_start, w.range_step, gates=sel)
    dt = time.perf_counter() - t0
    return len(sel) * n_ipp / dt, len(sel), dt


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    w = _workload(args.workload, 0, args.n_ranges, args.n_ipp)
    gates, ipps = args.ref_gates, args.ref_ipps
    for _ in range(args.warmup):
        _cpu_sample(w, gates, ipps, threads)
    rates, secs = [], 0.0
    for _ in range(args.steps):
        r, ng, dt = _cpu_sample(w, gates, ipps, threads)[:3]
        rates.append(r)
        secs += dt
    value = len(rates) * ng * ipps / secs
    sample = f"{ng} gates spread over the workload x the first {ipps} IPPs per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox echoes)",
            "config": {"workload": _workload_desc(w), "nfft": w.nfft, "n_ranges": w.n_ranges, "n_ipp": w.n_ipp},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_2311_18737_gb300 import isr

    from paper_2311_18737_gb300 import shard

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # the multi-rank path (NCCL barriers and max over ranks) runs whenever torchrun launched the
    # process, one rank included
    use_dist = world > 1 or "TORCHELASTIC_RUN_ID" in os.environ
    if use_dist:
        dist.init_process_group("nccl", device_id=dev)

    strong = args.scaling == "strong"
    # strong scaling: one workload (rank 0's seed) split by gates; weak: a problem per rank
    w = _workload(args.workload, 0 if strong else rank, args.n_ranges, args.n_ipp)
    R_total, N, P = w.n_ranges, w.nfft, w.n_ipp
    echo = torch.empty((P, w.echo_stride, 2), dtype=torch.int16, device=dev)
    code_d = torch.from_numpy(w.code()).to(dev)
    w.echo_device(echo.data_ptr(), code_d.data_ptr())
    R, range_start, echo_stride = R_total, w.range_start, w.echo_stride
    blocks = [(0, R_total)]
    if strong:
        blocks = shard.gate_blocks(R_total, world)
        first, R = blocks[rank]
        if R < 1:
            raise SystemExit(f"--scaling strong: {world} ranks for {R_total} gates leaves rank {rank} without gates")
        span = shard.echo_span(first, R, w.range_start, w.range_step, w.code_len)
        # this rank keeps only the echo samples its gates read
        echo = echo[:, span["s0"]:span["s0"] + span["echo_stride"], :].contiguous()
        range_start, echo_stride = span["range_start"], span["echo_stride"]
        torch.cuda.empty_cache()
    stream = torch.cuda.Stream(dev)
    out = torch.empty((R, N), dtype=torch.float32, device=dev)

    plan = isr.Plan(nfft=N, n_ranges=R, echo_stride=echo_stride, range_start=range_start,
                    range_step=w.range_step, tx_type=isr.ISR_TX_PM1, device=local, stream=stream)
    # radix order: time the candidates on a probe of the workload and keep the fastest
    if args.precision:
        # a tensor-core first-pass engine (nfft 16384, radix order 1): a precision-study run
        isr.isr_plan_set_precision(plan.handle, args.precision)
        tune = {"order": 1, "ms": []}
    elif args.order is not None:
        isr.isr_plan_set_order(plan.handle, args.order)
        tune = {"order": args.order, "ms": []}
    elif args.no_autotune:
        tune = {"order": 0, "ms": []}
    else:
        tune = plan.autotune(echo, code_d, min(P, 512))
    plan.set_profiling(True)

    gathered = {}

    def step(e, c, o):
        plan.integrate(e, c, P)
        if strong and use_dist:
            plan.spectra(out, isr.ISR_RESET_AFTER)
            with torch.cuda.stream(stream):
                g = shard.gather_gate_blocks(out, blocks, rank, world)
            if g is not None and o is not out:
                o.copy_(g, non_blocking=True)
            gathered["last"] = g
        else:
            plan.spectra(o, isr.ISR_RESET_AFTER)

    for _ in range(max(3, args.warmup)):
        step(echo, code_d, out)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(_gpu_selector(torch, local))
    sampler.start()
    time.sleep(0.3)
    info0 = plan.info()
    if use_dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(echo, code_d, out)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if use_dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    info1 = plan.info()
    clocks = sampler.stop()

    launches = info1["kernel_launches"] - info0["kernel_launches"]
    timed = info1["kernel_timed"] - info0["kernel_timed"]
    kernel_ms = (info1["kernel_ms"] - info0["kernel_ms"]) / max(1, timed)
    launches_per_step = launches / args.steps
    # our kernels per step: fused kernel + reduction per launch block, one conversion
    gpu_launches = int(launches * 2 + args.steps)

    # end to end through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        echo_h = torch.empty(echo.shape, dtype=torch.int16, pin_memory=True)
        echo_h.copy_(echo)
        code_h = code_d.cpu().pin_memory()
        out_h = torch.empty((R_total if (strong and rank == 0) else R, N), dtype=torch.float32, pin_memory=True)
        step(echo_h, code_h, out_h)
        torch.cuda.synchronize(dev)
        if use_dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step(echo_h, code_h, out_h)
        e2e_ms = 1000 * (time.perf_counter() - t0) / args.e2e_steps
        e2e_ms = max_over_ranks([e2e_ms], dev, world, use_dist)[0]
        e2e = {"value": job_throughput(world, R_total if strong else R, P, e2e_ms, strong), "unit": UNIT,
               "h2d_bytes_per_step": int(echo_h.numel() * 2 + code_h.numel()),
               "d2h_bytes_per_step": int(out_h.numel() * 4), "ms_per_step": e2e_ms,
               "host_block_growth": plan.info()["host_block_growth"]}
        del echo_h

    ms, kernel_ms = max_over_ranks([ms, kernel_ms], dev, world, use_dist)

    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    fp32_peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    flops_per_transform = 5.0 * N * math.log2(N)
    transforms_per_launch = R * P / max(1.0, launches_per_step)
    achieved = flops_per_transform * transforms_per_launch / (kernel_ms / 1000) / 1e12 if kernel_ms > 0 else None
    traffic = _recorded_traffic(N, R, P, tune["order"])
    # measured FP32 FMA rate (own microkernel, after the timed region): cross-check of the derived peak
    measured = None
    if not args.no_peak:
        ffma, _ = isr.isr_fp32_peak(local, False)
        ffma2, _ = isr.isr_fp32_peak(local, True)
        measured = {"ffma": ffma, "ffma2": ffma2, "unit": "TFLOP/s",
                    "how": "isr_fp32_peak: FMA-only kernel, 8 independent chains per thread, 4 x 256 threads "
                           "per SM, best of 3 runs; ffma2 = paired FP32 instruction"}

    line = {"metric": METRIC, "value": job_throughput(world, R_total if strong else R, P, ms, strong), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong" if strong else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Philox echoes generated on the device, not timed)",
            "config": {"workload": _workload_desc(w), "nfft": N, "n_ranges": R, "n_ipp": P,
                       "gates_per_rank": R, "partition": ("contiguous gate blocks, echo sub-span per rank, "
                                                           "blocks gathered to rank 0 each step") if strong else
                       "independent problem per rank", "l2": "inputs larger than L2 (echo %.2f GB per step)" % (
                           echo.numel() * 2 / 1e9), "kernel": "fused decode+FFT+|X|^2, chunks of %d IPPs" %
                       plan.info()["ipp_chunk"], "first_pass_engine": isr.PRECISION_NAMES[args.precision],
                       "radix_order": tune["order"], "radix_order_probe_ms": tune["ms"],
                       "realtime_factor_at_10ms_ipp": (P * 0.010) / (ms / 1000)},
            "gpu_launches": gpu_launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                         "frac": (achieved / fp32_peak_tflops) if achieved else None, "traffic": traffic,
                         "peak_basis": "derived FP32 SIMT peak: %d SMs x %d lanes x 2 FLOP x %.0f MHz (sm max)"
                                       % (props.multi_processor_count, FP32_LANES_PER_SM, sm_max),
                         "flop_model": "5 N log2 N per transform", "kernel_ms_per_launch": kernel_ms,
                         "peak_measured": measured,
                         "hbm_gbs": (traffic / (kernel_ms / 1000) / 1e9) if (traffic and kernel_ms > 0) else None,
                         "hbm_frac_of_measured": (traffic / (kernel_ms / 1000) / 1e9 / peaks["hbm_gbs"])
                         if (traffic and kernel_ms > 0 and peaks.get("hbm_gbs")) else None,
                         "frac_of_measured": (achieved / measured["ffma"]) if (achieved and measured) else None},
            "clocks": clocks, "e2e": e2e}
    if args.phase_cycles:
        # debug build (ISR_LIBRARY=.../libisr_debug.so): SM cycles per IPP of one CTA, by phase,
        # summed over every launch of the plan (probe, warm-up, timed steps)
        cyc = isr.isr_plan_phase_cycles(plan.handle)
        line["phase_cycles_per_ipp"] = {k: cyc[i] / max(1, cyc[4]) for i, k in
                                        enumerate(("window_wait_and_barrier", "pass0", "middle_pass", "last_pass"))}
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, ng, dt, ref, sel = _cpu_sample(w, args.ref_gates, args.ref_ipps, threads)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{ng} gates spread over the workload x the first {args.ref_ipps} IPPs "
                                          f"({dt:.1f} s wall)"}
        # the library on the same sample (same echo rows, all gates, then the sampled rows):
        # the largest per-bin relative difference from the FP64 oracle
        import numpy as np
        plan.integrate(echo[:args.ref_ipps], code_d, args.ref_ipps)
        plan.spectra(out, isr.ISR_RESET_AFTER)
        got = out[torch.as_tensor(sel, dtype=torch.long, device=out.device)].double().cpu().numpy()
        line["cpu_baseline"]["max_rel_err_vs_oracle"] = float(np.max(np.abs(got - ref) / ref))
        v, ng, dt = _numpy_sample(w, 64, 32)
        line["cpu_baseline_numpy"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "paper-style NumPy (Sec. 3.3)",
                                      "sample": f"{ng} gates spread over the workload x the first 32 IPPs "
                                                f"({dt:.1f} s wall)"}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if use_dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _recorded_traffic(nfft, n_ranges, n_ipp, order):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source, the same workload shape and radix order (else null)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2311_18737_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    if rec.get("kernel_source_sha256") != h.hexdigest():
        return None
    if rec.get("workload") != {"n_ranges": n_ranges, "n_ipp": n_ipp}:
        return None
    return rec.get("bytes_per_launch", {}).get(str(nfft), {}).get(str(order))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--scaling", choices=["weak", "strong"], default="weak",
                    help="weak: a full problem per rank; strong: one workload split by gates")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["realistic", "small", "paper"], default="realistic")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--order", type=int, default=None, help="force a radix order (no autotuning)")
    ap.add_argument("--no-peak", action="store_true", help="skip the FP32 FMA-rate microkernel")
    ap.add_argument("--phase-cycles", action="store_true",
                    help="with the debug library (ISR_LIBRARY): report the fused kernel's cycles per IPP by phase")
    ap.add_argument("--precision", type=int, default=0,
                    help="first-pass engine (isr_plan_set_precision): 0 SIMT FP32; 1-4 mma.sync, 5-8 tcgen05 tensor cores")
    ap.add_argument("--ref-gates", type=int, default=256)
    ap.add_argument("--ref-ipps", type=int, default=256)
    ap.add_argument("--n-ranges", type=int, default=None, help="resize the workload (profiling cases)")
    ap.add_argument("--n-ipp", type=int, default=None, help="resize the workload (profiling cases)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    launched = "TORCHELASTIC_RUN_ID" in os.environ or "RANK" in os.environ
    action = world_check(args.gpus, world, launched)
    if action == "relaunch":
        return _relaunch(args.gpus)
    if action == "error":
        print(f"bench.py: --gpus {args.gpus} but the launcher started {world} rank(s)", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
