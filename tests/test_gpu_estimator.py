"""The learned estimator's kernels (through the C ABI) against the FP64 reference:
features, loss and every parameter's gradient (FP32 storage), the BF16 variant (tensor-core
convolutions) against the reference with BF16 storage rounding, the prediction, and a short
end-to-end training on spectra the integrator produces."""
import numpy as np
import pytest
import torch

from oracle import estimator as ref
from paper_2311_18737_gb300 import estimator as est_mod
from paper_2311_18737_gb300 import isr

pytestmark = pytest.mark.gpu

# Both BF16 engines: tcgen05 (convolutions in 256-position CTAs of two M = 128 tiles, the weight
# gradient in 256-position chunks) and mma.sync.
ENGINES = [isr.ISR_EST_BF16, isr.ISR_EST_BF16_MMASYNC]


def _setup(precision, B=4, L=256, seed=0):
    rng = np.random.default_rng(seed)
    theta = (ref.init_params(seed) + 0.05 * rng.standard_normal(ref.N_PARAMS)).astype(np.float32)
    x = rng.standard_normal((B, L)).astype(np.float32)
    f = rng.uniform(3, L - 3, B).astype(np.float32)
    y = np.array([1, 0, 1, 1][:B], dtype=np.float32)
    f[1] = -320.0                      # a gate without a line: its position is meaningless
    e = est_mod.Estimator(max_batch=8, precision=precision, nfft=512, band_lo=0, band_len=L)
    e.set_params(theta)
    dev = torch.device("cuda:0")
    return e, theta, x, f, y, [torch.from_numpy(a).to(dev) for a in (x, f, y)]


def test_gradients_match_fp64_reference_fp32_storage():
    e, theta, x, f, y, (xd, fd, yd) = _setup(isr.ISR_EST_FP32)
    loss, g = e.grad(xd, fd, yd)
    rl, rg = ref.loss_and_grad(theta.astype(np.float64), x, f, y)
    assert abs(loss - rl) <= 1e-5 * abs(rl)
    gd, rd = ref.unpack(g.astype(np.float64)), ref.unpack(rg)
    gmax = np.abs(rg).max()
    for name, _ in ref.SHAPES:
        # b5 shifts every location logit equally, so its exact gradient is 0: measure such
        # blocks against the overall gradient scale
        scale = max(np.abs(rd[name]).max(), 1e-3 * gmax)
        err = np.abs(gd[name] - rd[name]).max() / scale
        assert err <= 2e-4, f"{name}: max error {err:.2e} of the block's largest gradient"
    e.close()


def test_bf16_storage_close_to_reference():
    e, theta, x, f, y, (xd, fd, yd) = _setup(isr.ISR_EST_BF16, seed=1)
    loss, g = e.grad(xd, fd, yd)
    rl, rg = ref.loss_and_grad(theta.astype(np.float64), x, f, y)
    assert abs(loss - rl) <= 3e-2 * abs(rl)
    cos = float(g @ rg / (np.linalg.norm(g) * np.linalg.norm(rg)))
    assert cos > 0.98, cos
    e.close()


@pytest.mark.parametrize("precision", ENGINES)
def test_bf16_gradients_per_block_against_rounding_reference(precision):
    """Random inputs (not dyadic): the BF16 variant against the FP64 reference that rounds to
    BF16 exactly where the variant stores (input, conv weights, activations).  What is left is
    FP32 accumulation order and the hi + lo split of the gradient entering the backward passes
    (~16 significant bits), which can move an activation across a BF16 rounding boundary now and
    then; so every parameter block's gradient must agree in norm to 2 % and in direction to
    cosine 0.999, and the loss to 1e-3."""
    e, theta, x, f, y, (xd, fd, yd) = _setup(precision, seed=3)
    loss, g = e.grad(xd, fd, yd)
    rl, rg = ref.loss_and_grad(theta.astype(np.float64), x, f, y, store=ref.round_bf16)
    assert abs(loss - rl) <= 1e-3 * abs(rl), (loss, rl)
    gd, rd = ref.unpack(g.astype(np.float64)), ref.unpack(rg)
    gmax = np.abs(rg).max()
    for name, _ in ref.SHAPES:
        a, b = gd[name].ravel(), rd[name].ravel()
        nb = np.linalg.norm(b)
        if nb <= 1e-3 * gmax:
            # b5: exactly zero in exact arithmetic; bound it by the overall gradient scale
            assert np.abs(a).max() <= 1e-3 * gmax, name
            continue
        rel = np.linalg.norm(a - b) / nb
        cos = float(a @ b / (np.linalg.norm(a) * nb))
        assert rel <= 2e-2 and cos >= 0.999, f"{name}: relative error {rel:.2e}, cosine {cos:.6f}"
    e.close()


def _dyadic_case(B=4, L=600, seed=7, precision=isr.ISR_EST_BF16):
    """Conv weights and biases in multiples of 1/8 within [-1/4, 1/4] and inputs in multiples
    of 1/4: every product and FP32 partial sum of the convolutions is exact, so the BF16
    variant's activations are the BF16 roundings of exact values on both sides.  L = 600 spans
    two full 256-position tiles of the tensor-core convolution and a ragged third."""
    rng = np.random.default_rng(seed)
    d = ref.unpack(ref.init_params(seed))
    for l in range(1, 5):
        d[f"W{l}"] = rng.integers(-2, 3, d[f"W{l}"].shape) / 8.0
        d[f"b{l}"] = rng.integers(-2, 3, d[f"b{l}"].shape) / 8.0
    theta = ref.pack(d).astype(np.float32)
    x = (rng.integers(-8, 9, (B, L)) / 4.0).astype(np.float32)
    f = rng.uniform(3, L - 3, B).astype(np.float32)
    y = np.resize(np.array([1, 0, 1, 1], dtype=np.float32), B)
    e = est_mod.Estimator(max_batch=max(8, B), precision=precision, nfft=2048, band_lo=0, band_len=L)
    e.set_params(theta)
    dev = torch.device("cuda:0")
    return e, theta, x, f, y, [torch.from_numpy(a).to(dev) for a in (x, f, y)]


# Lengths: 600 spans full tiles and a ragged rest; 37 is odd (unpaired stores), one partial
# tile; 1100 gives three tcgen05 CTAs with a length that is not a multiple of 8 (the
# word-by-word staging path).
@pytest.mark.parametrize("precision", ENGINES)
@pytest.mark.parametrize("L", [600, 37, 1100])
def test_bf16_tensor_core_forward_matches_bf16_storage_reference(L, precision):
    e, theta, x, f, y, (xd, fd, yd) = _dyadic_case(L=L, precision=precision)
    pos, pres = e.predict(xd)
    rpos, rpres = ref.predict(theta.astype(np.float64), x, store=ref.round_bf16)
    assert np.abs(pos.cpu().numpy() - rpos).max() <= 1e-3
    assert np.abs(pres.cpu().numpy() - rpres).max() <= 1e-5
    e.close()


@pytest.mark.parametrize("precision", ENGINES)
@pytest.mark.parametrize("L", [600, 37, 1100])
def test_bf16_tensor_core_gradients_match_bf16_storage_reference(L, precision):
    """The backward-data convolution splits the FP32 gradient into two BF16 parts (~16
    significant bits): every parameter block within 1e-3 of its largest gradient."""
    e, theta, x, f, y, (xd, fd, yd) = _dyadic_case(L=L, seed=8, precision=precision)
    loss, g = e.grad(xd, fd, yd)
    rl, rg = ref.loss_and_grad(theta.astype(np.float64), x, f, y, store=ref.round_bf16)
    assert abs(loss - rl) <= 1e-4 * abs(rl)
    gd, rd = ref.unpack(g.astype(np.float64)), ref.unpack(rg)
    gmax = np.abs(rg).max()
    for name, _ in ref.SHAPES:
        scale = max(np.abs(rd[name]).max(), 1e-3 * gmax)
        err = np.abs(gd[name] - rd[name]).max() / scale
        assert err <= 1e-3, f"{name}: max error {err:.2e} of the block's largest gradient"
    e.close()


def test_prediction_matches_reference():
    e, theta, x, f, y, (xd, fd, yd) = _setup(isr.ISR_EST_FP32, seed=2)
    pos, pres = e.predict(xd)
    rpos, rpres = ref.predict(theta.astype(np.float64), x)
    assert np.abs(pos.cpu().numpy() - rpos).max() <= 1e-3
    assert np.abs(pres.cpu().numpy() - rpres).max() <= 1e-5
    e.close()


def test_features_match_reference():
    rng = np.random.default_rng(5)
    P = rng.gamma(30.0, 2.0, size=(6, 512)).astype(np.float32)
    e = est_mod.Estimator(max_batch=8, precision=isr.ISR_EST_FP32, nfft=512, band_lo=40, band_len=300)
    x = e.features(torch.from_numpy(P).cuda()).cpu().numpy()
    assert np.abs(x - ref.features(P, 40, 300)).max() <= 1e-5
    e.close()


@pytest.mark.slow
def test_training_gains_over_peak_fit():
    """Short training on integrator-made spectra (reduced from the full 200k-spectrum run):
    the network must beat the peak fit's presence decision and agree with the peak fit
    within one bin on strong lines."""
    e = est_mod.Estimator(max_batch=128, precision=isr.ISR_EST_BF16)
    e.set_params(est_mod.init_params(0))
    tr = est_mod.make_dataset(16, seed=11, est=e)
    te = est_mod.make_dataset(4, seed=12, est=e)
    hist = est_mod.train(e, tr, steps=600, batch=128, lr=2e-3, log_every=100)
    assert hist[-1][1] < 0.7 * hist[0][1], hist
    res = est_mod.evaluate(e, te, est_mod.presence_threshold(tr))
    print(res)
    assert res["presence_accuracy"]["network"] >= res["presence_accuracy"]["peak_fit"]
    assert res["agreement_with_peak_fit_above_-10dB"] >= 0.9
    e.close()


@pytest.mark.parametrize("precision", ENGINES)
def test_bf16_gradients_many_rows_several_chunks_per_cta(precision):
    """64 rows x 1100 positions: the tcgen05 weight gradient then spreads 320 chunks of 256
    positions over one CTA per SM (two or three per CTA through its double-buffered staging, most
    ranges crossing from one row into the next), and the persistent tcgen05 convolutions take
    several 256-position tiles per CTA; exact (dyadic) inputs, the same bound as the other BF16
    gradient tests."""
    e, theta, x, f, y, (xd, fd, yd) = _dyadic_case(B=64, L=1100, seed=9, precision=precision)
    loss, g = e.grad(xd, fd, yd)
    rl, rg = ref.loss_and_grad(theta.astype(np.float64), x, f, y, store=ref.round_bf16)
    assert abs(loss - rl) <= 1e-4 * abs(rl)
    gd, rd = ref.unpack(g.astype(np.float64)), ref.unpack(rg)
    gmax = np.abs(rg).max()
    for name, _ in ref.SHAPES:
        scale = max(np.abs(rd[name]).max(), 1e-3 * gmax)
        err = np.abs(gd[name] - rd[name]).max() / scale
        assert err <= 1e-3, f"{name}: max error {err:.2e} of the block's largest gradient"
    e.close()
