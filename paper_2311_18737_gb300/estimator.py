"""Learned plasma-line estimator: training spectra from the integrator, training, evaluation.

The plasma line's frequency follows the electron density (the paper's Eq. 1), so the last
step of plasma-line analysis reduces each gate's integrated spectrum to a line position.
The plain method is the spectral peak fit (``isr_peak_fit``); this module trains the small
network of ``isr_est_*`` (hand-written forward, backward and Adam kernels in the library)
on spectra that the integrator itself produces from seeded synthetic echoes with injected
Langmuir lines, and compares both estimates against the injected truth.

Workload of the training data (per integration): the realistic geometry (1000 gates,
nfft 16384, gate step 25, 50 MS/s, binary-phase code), a random Chapman layer (peak gate
150-850, scale height 60-160 gates, peak plasma-line frequency 3-15 MHz; line frequency
proportional to sqrt(n_e)), per-gate SNR uniform in -30..0 dB, 15 % of gates without a
line (and every gate whose line falls below 1.1 MHz), and 256 IPPs per integration.
Spectra are ``ISR_MEAN`` averages; the network reads the 1-15 MHz band (bins 320-4927), or with
``--net-band full`` all 16384 bins; the peak fit always searches the 1-15 MHz band.

    python -m paper_2311_18737_gb300.estimator --train-integrations 200 --steps 3000 --out results.json
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import isr

FS_HZ = 50e6
NFFT = 16384
BAND_LO = 320
BAND_LEN = 4608
N_GATES = 1000
C, K = 32, 9
# parameter blocks in the flat vector (order of include/isr.h)
SHAPES = [("W1", (C, 1, K)), ("b1", (C,)), ("W2", (C, C, K)), ("b2", (C,)), ("W3", (C, C, K)), ("b3", (C,)),
          ("W4", (C, C, K)), ("b4", (C,)), ("w5", (C,)), ("b5", (1,)), ("Wa", (C, 2 * C)), ("ba", (C,)),
          ("wb", (C,)), ("bb", (1,))]


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases, as one float32 vector of ISR_EST_N_PARAMS."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in SHAPES:
        if name.startswith("W") or name in ("w5", "wb"):
            fan_in = int(np.prod(shp[1:])) if len(shp) > 1 else shp[0]
            parts.append(rng.standard_normal(shp).ravel() * math.sqrt(2.0 / fan_in))
        else:
            parts.append(np.zeros(int(np.prod(shp))))
    v = np.concatenate(parts).astype(np.float32)
    assert v.size == isr.ISR_EST_N_PARAMS
    return v


class Estimator:
    """Owns one ``isr_est`` (device buffers for a batch of up to ``max_batch`` gates)."""

    def __init__(self, max_batch: int = 128, precision: int = isr.ISR_EST_BF16, nfft: int = NFFT,
                 band_lo: int = BAND_LO, band_len: int = BAND_LEN, device: int = 0, stream=None):
        self.dev = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.nfft, self.band_lo, self.band_len, self.max_batch = nfft, band_lo, band_len, max_batch
        self.h = isr.isr_est_create(nfft, band_lo, band_len, max_batch, precision, device, self.stream)
        self._loss = torch.zeros(1, dtype=torch.float32, device=self.dev)

    def set_params(self, theta) -> None:
        t = torch.as_tensor(np.ascontiguousarray(theta, dtype=np.float32))
        isr.isr_est_set_params(self.h, t)

    def get_params(self) -> np.ndarray:
        out = np.empty(isr.ISR_EST_N_PARAMS, dtype=np.float32)
        isr.isr_est_get_params(self.h, out)
        return out

    def features(self, spectra: torch.Tensor) -> torch.Tensor:
        n = spectra.shape[0]
        x = torch.empty((n, self.band_len), dtype=torch.float32, device=self.dev)
        isr.isr_est_features(self.h, spectra, n, x)
        return x

    def grad(self, x, line_bin, present):
        g = np.empty(isr.ISR_EST_N_PARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        isr.isr_est_grad(self.h, x, x.shape[0], line_bin, present, loss, g)
        return float(loss[0]), g

    def train_step(self, x, line_bin, present, lr: float, want_loss: bool = False):
        isr.isr_est_train_step(self.h, x, x.shape[0], line_bin, present, lr, self._loss if want_loss else None)
        return float(self._loss.item()) if want_loss else None

    def predict(self, x):
        n = x.shape[0]
        pos = torch.empty(n, dtype=torch.float32, device=self.dev)
        pres = torch.empty(n, dtype=torch.float32, device=self.dev)
        for b0 in range(0, n, self.max_batch):
            b1 = min(n, b0 + self.max_batch)
            isr.isr_est_predict(self.h, x[b0:b1], b1 - b0, pos[b0:b1], pres[b0:b1])
        return pos, pres

    def close(self):
        if self.h:
            isr.isr_est_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def random_profile(rng, n_gates: int = N_GATES, snr_range=(-30.0, 0.0)):
    """Line frequency (cycles/sample), SNR (dB; -inf = no line) and presence per gate."""
    peak = rng.uniform(150, 850)
    scale = rng.uniform(60, 160)
    f_peak = rng.uniform(3e6, 15e6)
    z = (np.arange(n_gates) - peak) / scale
    ne_rel = np.exp(0.5 * (1.0 - z - np.exp(-z)))
    f_hz = f_peak * np.sqrt(ne_rel)
    snr = rng.uniform(snr_range[0], snr_range[1], n_gates)
    present = (f_hz >= 1.1e6) & (rng.random(n_gates) >= 0.15)
    snr = np.where(present, snr, -np.inf)
    return f_hz / FS_HZ, snr, present


def make_dataset(n_integrations: int, seed: int, n_ipp: int = 256, device: int = 0, est: Estimator | None = None,
                 snr_range=(-30.0, 0.0)):
    """Integrate ``n_integrations`` synthetic echo blocks and return features, labels and the
    peak fit of every gate (all device tensors except the numpy metadata)."""
    import synth

    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(seed)
    feats, labels, pres, snrs, pf_bin, pf_snr = [], [], [], [], [], []
    own = est is None
    if own:
        est = Estimator(max_batch=8, device=device)
    w0 = synth.realistic(n_ipp=n_ipp)
    echo = torch.empty((n_ipp, w0.echo_stride, 2), dtype=torch.int16, device=dev)
    spectra = torch.empty((N_GATES, NFFT), dtype=torch.float32, device=dev)
    fb = torch.empty(N_GATES, dtype=torch.float64, device=dev)
    sr = torch.empty(N_GATES, dtype=torch.float32, device=dev)
    with isr.Plan(nfft=NFFT, n_ranges=N_GATES, echo_stride=w0.echo_stride, range_step=w0.range_step,
                  tx_type=isr.ISR_TX_PM1, device=device, stream=stream) as plan:
        for i in range(n_integrations):
            f, snr, present = random_profile(rng, snr_range=snr_range)
            w = synth.realistic(n_ipp=n_ipp, seed=int(rng.integers(1, 2**62)), gate_freq=f, gate_snr_db=snr)
            code = torch.from_numpy(w.code()).to(dev)
            w.echo_device(echo.data_ptr(), code.data_ptr())
            plan.integrate(echo, code, n_ipp)
            plan.spectra(spectra, isr.ISR_MEAN | isr.ISR_RESET_AFTER)
            feats.append(est.features(spectra))
            isr.isr_peak_fit(spectra, N_GATES, NFFT, BAND_LO, BAND_LO + BAND_LEN, fb, sr, stream)
            # positions in the network's band coordinates; presence means a line inside the
            # 1-15 MHz band whatever the network reads
            pf_bin.append(fb.cpu().numpy() - est.band_lo)
            pf_snr.append(sr.cpu().numpy().astype(np.float64))
            lb = f * NFFT - est.band_lo
            lp = f * NFFT - BAND_LO
            labels.append(lb)
            pres.append(present & (lp >= 4) & (lp <= BAND_LEN - 5))
            snrs.append(snr)
    if own:
        est.close()
    lab = np.concatenate(labels).astype(np.float32)
    pr = np.concatenate(pres)
    return {"x": torch.cat(feats), "line_bin": torch.from_numpy(lab).to(dev),
            "present": torch.from_numpy(pr.astype(np.float32)).to(dev), "line_bin_np": lab, "present_np": pr,
            "snr_db": np.concatenate(snrs), "pf_bin": np.concatenate(pf_bin), "pf_snr": np.concatenate(pf_snr),
            "n_ipp": n_ipp}


def train(est: Estimator, data, steps: int, batch: int = 128, lr: float = 2e-3, seed: int = 0, log_every: int = 0):
    """Adam on random minibatches; cosine-decayed learning rate.  Returns the loss history."""
    g = torch.Generator(device=data["x"].device)
    g.manual_seed(seed)
    n = data["x"].shape[0]
    hist = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), device=data["x"].device, generator=g)
        x = data["x"][idx].contiguous()
        lb = data["line_bin"][idx].contiguous()
        pr = data["present"][idx].contiguous()
        lr_s = lr * 0.5 * (1 + math.cos(math.pi * s / max(1, steps)))
        want = log_every and (s % log_every == 0 or s == steps - 1)
        loss = est.train_step(x, lb, pr, max(lr_s, 1e-5), want_loss=bool(want))
        if want:
            hist.append((s, loss))
    return hist


def presence_threshold(data) -> float:
    """Peak-fit presence rule: the peak-to-band-mean ratio threshold that maximises
    accuracy on the given (training) data."""
    s, y = data["pf_snr"], data["present_np"]
    cands = np.quantile(s, np.linspace(0.01, 0.99, 197))
    acc = [((s > c) == y).mean() for c in cands]
    return float(cands[int(np.argmax(acc))])


def evaluate(est: Estimator, data, pf_threshold: float):
    pos, pres = est.predict(data["x"])
    pos = pos.cpu().numpy().astype(np.float64) - est.band_lo
    pres = pres.cpu().numpy().astype(np.float64)
    y, truth, snr = data["present_np"], data["line_bin_np"].astype(np.float64), data["snr_db"]
    out = {"n_gates": int(y.size), "n_present": int(y.sum()),
           "presence_accuracy": {"network": float(((pres > 0.5) == y).mean()),
                                 "peak_fit": float(((data["pf_snr"] > pf_threshold) == y).mean()),
                                 "peak_fit_threshold": pf_threshold}}
    lo_db = int(np.floor(np.min(snr[np.isfinite(snr)]) / 5.0)) * 5 if np.isfinite(snr).any() else -30
    hi_db = int(np.ceil(np.max(snr[np.isfinite(snr)]) / 5.0)) * 5 if np.isfinite(snr).any() else 0
    bins = [(b, b + 5) for b in range(lo_db, hi_db, 5)]
    rows = []
    for lo, hi in bins:
        m = y & (snr >= lo) & (snr < hi)
        if m.sum() == 0:
            continue
        en = np.abs(pos[m] - truth[m])
        ep = np.abs(data["pf_bin"][m] - truth[m])
        rows.append({"snr_db": [lo, hi], "gates": int(m.sum()),
                     "within_1_bin": {"network": float((en <= 1).mean()), "peak_fit": float((ep <= 1).mean())},
                     "median_abs_err_bins": {"network": float(np.median(en)), "peak_fit": float(np.median(ep))}})
    out["frequency_by_snr"] = rows
    hi = y & (snr >= -10)
    if hi.any():
        out["agreement_with_peak_fit_above_-10dB"] = float((np.abs(pos[hi] - data["pf_bin"][hi]) <= 1).mean())
    # the configuration's criterion: the network's position within one bin of the plain peak fit
    # wherever the peak fit itself is within one bin of the injected line
    ok = y & (np.abs(data["pf_bin"] - truth) <= 1)
    if ok.any():
        out["within_1_bin_of_peak_fit_where_peak_fit_finds_the_line"] = float((np.abs(pos[ok] - data["pf_bin"][ok]) <= 1).mean())
    return out


def conv_flop(band_len: int) -> float:
    """Multiply-add FLOP of the four convolutions per spectrum (2 per product)."""
    return 2.0 * band_len * (C * K + 3 * C * C * K)


def predict_rate(est: Estimator, x, band_len: int, reps: int = 5):
    """Inference rate of isr_est_predict on device-resident features, timed with CUDA events
    on the estimator's stream after one warm-up pass; the convolutions are ~99 % of its FLOP."""
    est.predict(x)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(est.stream)
    for _ in range(reps):
        est.predict(x)
    ev1.record(est.stream)
    ev1.synchronize()
    s = ev0.elapsed_time(ev1) / 1e3 / reps
    n = int(x.shape[0])
    return {"predict_spectra": n, "predict_seconds": s, "predict_spectra_per_s": n / s,
            "predict_conv_tflops": conv_flop(band_len) * n / s / 1e12}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-integrations", type=int, default=200)
    ap.add_argument("--eval-integrations", type=int, default=20)
    ap.add_argument("--n-ipp", type=int, default=256)
    ap.add_argument("--snr-range", type=float, nargs=2, default=(-30.0, 0.0), metavar=("LO", "HI"),
                    help="per-gate line SNR range in dB (uniform)")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--precision", choices=["bf16", "bf16-mmasync", "fp32"], default="bf16",
                    help="bf16: convolutions on tcgen05; bf16-mmasync: on warp-level mma.sync")
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-params", default=None)
    ap.add_argument("--net-band", choices=["band", "full"], default="band",
                    help="network input: the 1-15 MHz band or all nfft bins")
    ap.add_argument("--bench-predict", type=int, default=0, metavar="SPECTRA",
                    help="only time inference on this many seeded standard-normal feature rows")
    a = ap.parse_args()
    prec = {"bf16": isr.ISR_EST_BF16, "bf16-mmasync": isr.ISR_EST_BF16_MMASYNC, "fp32": isr.ISR_EST_FP32}[a.precision]
    lo, ln = (BAND_LO, BAND_LEN) if a.net_band == "band" else (0, NFFT)
    est = Estimator(max_batch=a.batch, precision=prec, band_lo=lo, band_len=ln)
    est.set_params(init_params(0))
    if a.bench_predict > 0:
        g = torch.Generator(device=est.dev)
        g.manual_seed(0)
        x = torch.randn((a.bench_predict, ln), generator=g, device=est.dev)
        res = predict_rate(est, x, ln)
        res.update({"precision": a.precision, "batch": a.batch, "net_band": [lo, lo + ln]})
        if prec == isr.ISR_EST_BF16:
            # the forward convolutions issue M = 128, N = 32, K = 16 MMAs: their measured rate is
            # the tensor roofline of this pass (the N = 256 rate is the part's dense BF16 peak)
            r32, _ = isr.isr_tc05_rate(32)
            r256, _ = isr.isr_tc05_rate(256)
            res.update({"tc05_rate_n32_tflops": r32, "tc05_rate_n256_tflops": r256,
                        "conv_frac_of_n32_rate": res["predict_conv_tflops"] / r32,
                        "conv_frac_of_n256_rate": res["predict_conv_tflops"] / r256})
        print(json.dumps(res, indent=1))
        if a.out:
            with open(a.out, "w") as fh:
                json.dump(res, fh, indent=1)
        return
    t0 = time.time()
    tr = make_dataset(a.train_integrations, seed=1, n_ipp=a.n_ipp, est=est, snr_range=tuple(a.snr_range))
    te = make_dataset(a.eval_integrations, seed=2, n_ipp=a.n_ipp, est=est, snr_range=tuple(a.snr_range))
    t_data = time.time() - t0
    torch.cuda.synchronize()
    t0 = time.time()
    hist = train(est, tr, a.steps, batch=a.batch, lr=a.lr, log_every=max(1, a.steps // 20))
    torch.cuda.synchronize()
    t_train = time.time() - t0
    res = evaluate(est, te, presence_threshold(tr))
    res.update(predict_rate(est, te["x"], ln))
    res.update({"train_spectra": int(tr["x"].shape[0]), "eval_spectra": int(te["x"].shape[0]), "n_ipp": a.n_ipp,
                "steps": a.steps, "batch": a.batch, "precision": a.precision, "net_band": [lo, lo + ln],
                "snr_range_db": list(a.snr_range),
                "data_seconds": t_data,
                "train_seconds": t_train, "loss_history": hist})
    print(json.dumps(res, indent=1))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    if a.save_params:
        np.save(a.save_params, est.get_params())


if __name__ == "__main__":
    main()
