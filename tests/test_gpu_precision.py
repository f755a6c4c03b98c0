"""Tensor-core first pass (split BF16 / FP16 products) against the FP64 oracle; the
single-product modes must be measurably worse, which is what the split buys.  The precision
study's engines at the realistic geometry against the oracle on its sampled gates."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import RTOL, assert_parity, rel_err
from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu


def _run(mode, echo, tx, R, start, step):
    dev = torch.device("cuda:0")
    with isr.Plan(nfft=16384, n_ranges=R, echo_stride=echo.shape[1], range_start=start, range_step=step,
                  device=0, stream=torch.cuda.current_stream()) as plan:
        if mode:
            isr.isr_plan_set_precision(plan.handle, mode)
        plan.integrate(torch.from_numpy(echo).to(dev), torch.from_numpy(tx).to(dev), echo.shape[0])
        out, _ = plan.spectra()
    return out.numpy().astype(np.float64)


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(41)
    R, P, start, step = 4, 5, 3, 17       # start 3: windows off the 16-byte grid
    stride = (start + (R - 1) * step + 16384 + 8 + 3) // 4 * 4
    echo = np.clip(np.rint(rng.standard_normal((P, stride, 2)) * 3000), -32768, 32767).astype(np.int16)
    tx = np.where(rng.random(16384) < 0.5, -1, 1).astype(np.int8)
    ref = oracle.integrate(echo, tx, nfft=16384, n_ranges=R, range_start=start, range_step=step)
    return echo, tx, R, start, step, ref


# Per-bin bounds from the operand precision: FP16 hi + lo carries 22 bits of the DFT matrix
# (relative 2^-22), so the FP32 tolerance holds; BF16 hi + lo carries 16 bits and the dropped
# A_lo B_lo term is 2^-16 of a product, so a single IPP's power can be off by ~2 x 2^-16
# (3e-5); averaging over IPPs shrinks it.
BOUNDS = {isr.ISR_PREC_TC_FP16_SPLIT: RTOL, isr.ISR_PREC_TC_BF16_SPLIT: 5e-5,
          isr.ISR_PREC_TC05_FP16_SPLIT: RTOL, isr.ISR_PREC_TC05_BF16_SPLIT: 5e-5}


@pytest.mark.parametrize("mode", [isr.ISR_PREC_TC_BF16_SPLIT, isr.ISR_PREC_TC_FP16_SPLIT,
                                  isr.ISR_PREC_TC05_BF16_SPLIT, isr.ISR_PREC_TC05_FP16_SPLIT])
def test_split_modes_within_their_bounds(case, mode):
    echo, tx, R, start, step, ref = case
    mx, p99, med = assert_parity(_run(mode, echo, tx, R, start, step), ref, rtol=BOUNDS[mode],
                                 what=isr.PRECISION_NAMES[mode])
    print(f"{isr.PRECISION_NAMES[mode]}: max {mx:.2e} p99 {p99:.2e} median {med:.2e}")


@pytest.mark.parametrize("engine", ["mma.sync", "tcgen05"])
def test_single_products_are_worse(case, engine):
    echo, tx, R, start, step, ref = case
    b_split, b_single, f_single = ((isr.ISR_PREC_TC_BF16_SPLIT, isr.ISR_PREC_TC_BF16, isr.ISR_PREC_TC_FP16)
                                   if engine == "mma.sync" else
                                   (isr.ISR_PREC_TC05_BF16_SPLIT, isr.ISR_PREC_TC05_BF16, isr.ISR_PREC_TC05_FP16))
    err = {m: rel_err(_run(m, echo, tx, R, start, step), ref).max() for m in (b_split, b_single, f_single)}
    assert err[b_single] > 10 * err[b_split]
    assert err[b_single] > err[f_single]
    assert err[b_single] < 0.5


def test_tcgen05_and_mma_sync_engines_agree(case):
    """Both tensor-core engines compute the same GEMM from the same split operands; only the
    FP32 accumulation order inside the tensor core differs."""
    echo, tx, R, start, step, ref = case
    for a, b in ((isr.ISR_PREC_TC_FP16_SPLIT, isr.ISR_PREC_TC05_FP16_SPLIT),
                 (isr.ISR_PREC_TC_BF16, isr.ISR_PREC_TC05_BF16)):
        pa, pb = _run(a, echo, tx, R, start, step), _run(b, echo, tx, R, start, step)
        assert rel_err(pb, pa).max() <= 2e-5, (isr.PRECISION_NAMES[a], isr.PRECISION_NAMES[b])


def test_unsupported_shapes_rejected():
    with isr.Plan(nfft=8192, n_ranges=2, echo_stride=9000, device=0, stream=torch.cuda.current_stream()) as plan:
        with pytest.raises(isr.IsrError) as ei:
            isr.isr_plan_set_precision(plan.handle, isr.ISR_PREC_TC_BF16_SPLIT)
        assert ei.value.status == isr.ISR_ERR_UNSUPPORTED


# per-bin bounds at the realistic geometry (sums over many IPPs); the single-product modes
# carry the 16-bit rounding of the DFT matrix, a fixed error per bin that does not average out
STUDY_BOUNDS = {"fp32-simt": RTOL, "tc-fp16-split": RTOL, "tc-bf16-split": 5e-5, "tc-fp16": 1e-3, "tc-bf16": 1e-2,
                "tc05-fp16-split": RTOL, "tc05-bf16-split": 5e-5, "tc05-fp16": 1e-3, "tc05-bf16": 1e-2}


def test_study_against_fp64_oracle():
    """Every engine of the precision study (1000 gates x nfft 16384) against the FP64 oracle on
    the study's sampled gates over all IPPs.  ISR_PRECISION_STUDY_IPP sets the IPP count
    (default 200; the recorded study uses 10000); `pytest -s` prints the table."""
    import os

    from oracle import linefit
    from paper_2311_18737_gb300 import precision

    n_ipp = int(os.environ.get("ISR_PRECISION_STUDY_IPP", "200"))
    res, inp = precision.run(n_ipp=n_ipp, reps=2 if n_ipp >= 1000 else 1)
    ref = oracle.integrate(inp["echo"].cpu().numpy(), inp["code"], nfft=inp["nfft"], n_ranges=inp["n_ranges"],
                           range_start=inp["range_start"], range_step=inp["range_step"], sel=inp["sel"])
    lo, hi = inp["band"]
    f_ref, _ = linefit.peak_fit(ref, lo, hi)
    rows = []
    for name, P in inp["spectra"].items():
        rel = np.abs(P - ref) / ref
        f_eng, _ = linefit.peak_fit(P, lo, hi)
        e = res["engines"][name]
        t = e["line_bin_err_vs_truth"]
        rows.append(f"| {name} | {e['ms_per_integration']:.1f} | {e['spectra_per_s'] / 1e6:.2f} | {rel.max():.2e} | "
                    f"{np.quantile(rel, 0.99):.2e} | {np.median(rel):.2e} | {np.abs(f_eng - f_ref).max():.1e} | "
                    f"{t['median']:.3f} / {t['max']:.3f} |")
        assert rel.max() <= STUDY_BOUNDS[name], (name, float(rel.max()))
    print(res["workload"], "sampled gates", inp["sel"])
    print("\n".join(rows))
