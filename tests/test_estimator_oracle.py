"""Pins of the FP64 estimator reference: its hand-written backward pass equals central
finite differences of its forward loss; features are standardised; the soft-argmax
prediction of a sharp logit map lands on the logit peak."""
import numpy as np

from oracle import estimator as est


def _case(seed, B=3, L=40):
    rng = np.random.default_rng(seed)
    theta = est.init_params(seed) + 0.05 * rng.standard_normal(est.N_PARAMS)
    x = rng.standard_normal((B, L))
    f = rng.uniform(3, L - 3, B)
    y = np.array([1.0, 0.0, 1.0])[:B]
    return theta, x, f, y


def test_backward_matches_finite_differences():
    theta, x, f, y = _case(1)
    L0, g = est.loss_and_grad(theta, x, f, y)
    assert abs(L0 - est.loss(theta, x, f, y)) < 1e-12
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(est.N_PARAMS, 60, replace=False),
                          np.arange(est.N_PARAMS - 2200, est.N_PARAMS)[::97]])
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        num = (est.loss(tp, x, f, y) - est.loss(tm, x, f, y)) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, g[i])


def test_gate_without_line_ignores_its_position():
    theta, x, f, y = _case(6)
    f2 = f.copy()
    f2[1] = -500.0                      # y[1] == 0: any position, even far outside the band
    L1, g1 = est.loss_and_grad(theta, x, f, y)
    L2, g2 = est.loss_and_grad(theta, x, f2, y)
    assert np.isfinite(L2) and np.all(np.isfinite(g2))
    assert abs(L1 - L2) < 1e-12 and np.allclose(g1, g2, atol=1e-15)


def test_every_block_has_a_gradient():
    theta, x, f, y = _case(3)
    _, g = est.loss_and_grad(theta, x, f, y)
    d = est.unpack(g)
    for name, _ in est.SHAPES:
        assert np.abs(d[name]).sum() > 0, name


def test_features_standardised():
    rng = np.random.default_rng(4)
    P = rng.gamma(20, 1.0, size=(5, 300))
    x = est.features(P, 10, 256)
    assert np.allclose(x.mean(axis=1), 0, atol=1e-12)
    assert np.allclose(x.std(axis=1), 1, atol=1e-4)


def test_prediction_of_sharp_logits():
    theta = np.zeros(est.N_PARAMS)
    d = est.unpack(theta)
    d["b1"][:] = 0.0
    # identity-like path: channel 0 passes x through 4 layers, w5 reads it
    for l in range(1, 5):
        W = np.zeros_like(d[f"W{l}"])
        W[0, 0, est.HALF] = 1.0
        d[f"W{l}"] = W
    d["w5"][0] = 50.0
    theta = est.pack(d)
    x = np.zeros((1, 64))
    x[0, 20] = 1.0
    pos, pres = est.predict(theta, x)
    assert abs(pos[0] - 20.0) < 1e-9 and abs(pres[0] - 0.5) < 1e-12


def test_round_bf16_definition():
    """BF16 keeps 8 significant bits, ties to the even neighbour: hand-worked values, the
    BF16 grid is left alone, and torch's own FP32 -> BF16 conversion agrees."""
    import torch

    u = 2.0 ** -7                                  # BF16 spacing in [1, 2)
    cases = {1.0: 1.0, 1 + u / 2: 1.0, 1 + 3 * u / 2: 1 + 2 * u, 1 + u / 2 + 2.0 ** -20: 1 + u,
             -(1 + 3 * u / 2): -(1 + 2 * u), 255.0: 255.0, 257.0: 256.0, 259.0: 260.0, 0.0: 0.0}
    for v, r in cases.items():
        assert est.round_bf16(np.array([v]))[0] == r, v
    grid = np.array([1 + k * u for k in range(128)] + [-3.0, 0.5, 2.0 ** -20])
    assert np.array_equal(est.round_bf16(grid), grid)
    rng = np.random.default_rng(9)
    v = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(est.round_bf16(v), want)


def test_storage_rounding_is_applied_where_the_bf16_variant_stores():
    """With store=round_bf16 the forward equals a plain forward whose conv weights and input
    were rounded first, when no activation needs rounding (every value is then on the BF16
    grid), and it differs from the plain forward when the input is off the grid."""
    d = est.unpack(np.zeros(est.N_PARAMS))
    for l in range(1, 5):
        W = np.zeros_like(d[f"W{l}"])
        W[0, 0, est.HALF] = 1.0 + 2.0 ** -10       # rounds to 1 in BF16
        d[f"W{l}"] = W
    d["w5"][0] = 1.0
    theta = est.pack(d)
    x = np.array([[0.0, 1.0, 2.0, -1.0, 3.0, 0.5] + [0.0] * 10])
    z_st, _, c = est.forward(theta, x, est.round_bf16)
    dr = {k: v.copy() for k, v in d.items()}
    for l in range(1, 5):
        dr[f"W{l}"] = est.round_bf16(d[f"W{l}"])
    z_pre, _, _ = est.forward(est.pack(dr), x)
    assert np.array_equal(z_st, z_pre)
    assert np.array_equal(z_st[0, :6], np.maximum(x[0, :6], 0))
    x_off = x + 2.0 ** -12                          # off the BF16 grid near 1, 2, 3
    z_off, _, _ = est.forward(theta, x_off, est.round_bf16)
    assert not np.array_equal(z_off, est.forward(theta, x_off)[0])


def test_presence_head_hand_worked():
    """The presence head at non-zero weights, worked out by hand.

    Channel 0 carries relu(x) through the four layers (centre tap 1), channel 1 carries the
    constant 2 (bias 2 in layer 1, centre tap 1 after); every other channel is zero.  With
    x = [0, 1, 3, -2, 0, 0, 0, 0]: h4[0] = [0, 1, 3, 0, 0, 0, 0, 0], h4[1] = 2 everywhere, so
    the pooled vector is max = (3, 2, 0...), mean = (0.5, 2, 0...).  Head rows:
      u0 = relu(1*3 + 2*0.5 - 1)          = 3
      u1 = relu(-1*2 + 0.5*2 + 0.5)       = relu(-0.5) = 0
      u2 = relu(4*0.5 - 0.25*2 + 0)       = 1.5
      q  = 0.5*3 + 10*0 - 2*1.5 + 0.25    = -1.25,   presence = 1 / (1 + e^1.25) = 0.2227001388...
    Location logits z = 1*h4[0] + 0.5*h4[1] - 1 = [0, 1, 3, 0, 0, 0, 0, 0].
    Gradients of the loss at label 1 (batch of one): dq = presence - 1; d bb = dq,
    d wb = dq u = dq (3, 0, 1.5), d ba = dq wb [u > 0] = dq (0.5, 0, -2),
    d Wa[0][0] = dq 0.5 * 3, d Wa[0][32] = dq 0.5 * 0.5, d Wa[1][*] = 0, d Wa[2][32] = dq (-2) 0.5."""
    d = est.unpack(np.zeros(est.N_PARAMS))
    for l in range(1, 5):
        W = np.zeros_like(d[f"W{l}"])
        W[0, 0, est.HALF] = 1.0
        if l > 1:
            W[1, 1, est.HALF] = 1.0
        d[f"W{l}"] = W
    d["b1"][1] = 2.0
    d["w5"][0], d["w5"][1], d["b5"][0] = 1.0, 0.5, -1.0
    d["Wa"][0, 0], d["Wa"][0, 32], d["ba"][0] = 1.0, 2.0, -1.0
    d["Wa"][1, 1], d["Wa"][1, 33], d["ba"][1] = -1.0, 0.5, 0.5
    d["Wa"][2, 32], d["Wa"][2, 33] = 4.0, -0.25
    d["wb"][0], d["wb"][1], d["wb"][2], d["bb"][0] = 0.5, 10.0, -2.0, 0.25
    theta = est.pack(d)
    x = np.array([[0.0, 1.0, 3.0, -2.0, 0.0, 0.0, 0.0, 0.0]])

    z, q, cache = est.forward(theta, x)
    np.testing.assert_array_equal(cache["pooled"][0, :3], [3.0, 2.0, 0.0])
    np.testing.assert_array_equal(cache["pooled"][0, 32:35], [0.5, 2.0, 0.0])
    np.testing.assert_array_equal(cache["u"][0, :3], [3.0, 0.0, 1.5])
    assert q[0] == -1.25
    np.testing.assert_array_equal(z[0], [0.0, 1.0, 3.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    pos, pres = est.predict(theta, x)
    assert abs(pres[0] - 0.22270013882530884) < 1e-15

    _, g = est.loss_and_grad(theta, x, np.array([2.0]), np.array([1.0]))
    gd = est.unpack(g)
    dq = 0.22270013882530884 - 1.0
    assert abs(gd["bb"][0] - dq) < 1e-14
    np.testing.assert_allclose(gd["wb"][:3], [3 * dq, 0.0, 1.5 * dq], rtol=0, atol=1e-14)
    assert np.all(gd["wb"][3:] == 0)
    np.testing.assert_allclose(gd["ba"][:3], [0.5 * dq, 0.0, -2.0 * dq], rtol=0, atol=1e-14)
    assert abs(gd["Wa"][0, 0] - 1.5 * dq) < 1e-14 and abs(gd["Wa"][0, 32] - 0.25 * dq) < 1e-14
    assert np.all(gd["Wa"][1] == 0)
    assert abs(gd["Wa"][2, 32] - (-1.0 * dq)) < 1e-14 and abs(gd["Wa"][2, 33] - (-4.0 * dq)) < 1e-14
