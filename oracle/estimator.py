"""FP64 reference of the learned plasma-line estimator (test infrastructure only).

The network maps one gate's integrated spectrum to the plasma line's position and its
presence (the line frequency gives the electron density, the paper's Eq. 1).  Written
plainly with numpy in double precision: forward pass, loss, and the backward pass by
hand; the tests pin the backward pass to central finite differences of the forward pass.

Features (per gate, band of L bins starting at bin `lo` of the spectrum P):
    y_i = ln(max(P[lo + i], 1e-30)),   x_i = (y_i - mean(y)) / (std(y) + 1e-6)

Network (parameters in this order in the flat vector):
    W1 [32][1][9]  b1 [32]   h1 = relu(conv(x,  W1) + b1)     (zero padding 4 on each side)
    W2 [32][32][9] b2 [32]   h2 = relu(conv(h1, W2) + b2)
    W3 [32][32][9] b3 [32]   h3 = relu(conv(h2, W3) + b3)
    W4 [32][32][9] b4 [32]   h4 = relu(conv(h3, W4) + b4)
    w5 [32]        b5 [1]    z_i = w5 . h4[:, i] + b5          (location logits)
    Wa [32][64]    ba [32]   u = relu(Wa [max_i h4; mean_i h4] + ba)
    wb [32]        bb [1]    q = wb . u + bb                    (presence logit)
    conv(h, W)[c][i] = sum_{ci, k} W[c][ci][k] h[ci][i + k - 4]

Loss per gate (averaged over the batch), with presence label y and line position f (bins
from `lo`): BCE(q, y) + y * CE(softmax(z), t), t_i proportional to exp(-(i - f)^2 / 2).
Prediction: presence sigmoid(q); position = softmax-weighted mean of i over the 7 bins
around argmax z.

Storage precision: the network's BF16 variant keeps the input, the conv weights W1..W4 and
every activation h1..h4 in BF16 (8 significant bits) and computes in FP32.  `forward`,
`loss_and_grad` and `predict` take an optional `store` function applied at exactly those
points (`round_bf16` for that variant; None keeps every value in double precision).
"""
from __future__ import annotations

import numpy as np

C = 32
K = 9
HALF = K // 2
SHAPES = [("W1", (C, 1, K)), ("b1", (C,)), ("W2", (C, C, K)), ("b2", (C,)), ("W3", (C, C, K)), ("b3", (C,)),
          ("W4", (C, C, K)), ("b4", (C,)), ("w5", (C,)), ("b5", (1,)), ("Wa", (C, 2 * C)), ("ba", (C,)),
          ("wb", (C,)), ("bb", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
WIN = 3          # half-width of the soft-argmax window
SIGMA_T = 1.0    # width of the location target, bins


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_params(seed: int = 0):
    rng = np.random.default_rng(seed)
    d = {}
    for name, shp in SHAPES:
        if name.startswith("W") or name in ("w5", "wb"):
            fan_in = int(np.prod(shp[1:])) if len(shp) > 1 else shp[0]
            d[name] = rng.standard_normal(shp) * np.sqrt(2.0 / fan_in)
        else:
            d[name] = np.zeros(shp)
    return pack(d)


def round_bf16(a):
    """Nearest BF16 value (8 significant bits, ties to even) of FP32-representable values,
    as float64: keep the upper 16 bits of the FP32 encoding after adding half of the
    dropped part, plus one where the kept part is odd (the tie rule)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def features(P, lo: int, L: int):
    y = np.log(np.maximum(np.asarray(P, dtype=np.float64)[:, lo:lo + L], 1e-30))
    m = y.mean(axis=1, keepdims=True)
    s = y.std(axis=1, keepdims=True)
    return (y - m) / (s + 1e-6)


def conv(h, W, b):
    """h [B][Cin][L], W [Cout][Cin][K] -> [B][Cout][L] with zero padding."""
    B, Cin, L = h.shape
    hp = np.zeros((B, Cin, L + 2 * HALF))
    hp[:, :, HALF:HALF + L] = h
    out = np.zeros((B, W.shape[0], L)) + b[None, :, None]
    for k in range(K):
        out += np.einsum("oc,bcl->bol", W[:, :, k], hp[:, :, k:k + L])
    return out


def target(f_true, L):
    """Gaussian location target per gate; all zeros where the line lies too far outside
    the band for the target to be representable (such gates carry no line)."""
    i = np.arange(L)[None, :]
    t = np.exp(-((i - np.asarray(f_true, dtype=np.float64)[:, None]) ** 2) / (2 * SIGMA_T ** 2))
    s = t.sum(axis=1, keepdims=True)
    return np.where(s > 0, t / np.where(s > 0, s, 1.0), 0.0)


def forward(theta, x, store=None):
    p = unpack(theta)
    keep = store if store is not None else (lambda v: v)
    x = keep(np.asarray(x, dtype=np.float64))
    cache = {"h0": x[:, None, :]}
    h = cache["h0"]
    for l in range(1, 5):
        cache[f"W{l}"] = keep(p[f"W{l}"])
        h = keep(np.maximum(conv(h, cache[f"W{l}"], p[f"b{l}"]), 0.0))
        cache[f"h{l}"] = h
    z = np.einsum("c,bcl->bl", p["w5"], h) + p["b5"][0]
    amax = h.argmax(axis=2)                      # first index of the maximum
    pooled = np.concatenate([h.max(axis=2), h.mean(axis=2)], axis=1)
    u = np.maximum(pooled @ p["Wa"].T + p["ba"], 0.0)
    q = u @ p["wb"] + p["bb"][0]
    cache.update(z=z, amax=amax, pooled=pooled, u=u, q=q)
    return z, q, cache


def softmax(z):
    e = np.exp(z - z.max(axis=1, keepdims=True))
    return e / e.sum(axis=1, keepdims=True)


def loss(theta, x, f_true, y):
    z, q, _ = forward(theta, x)
    y = np.asarray(y, dtype=np.float64)
    logp = z - z.max(axis=1, keepdims=True)
    logp = logp - np.log(np.exp(logp).sum(axis=1, keepdims=True))
    ce = -(target(f_true, z.shape[1]) * logp).sum(axis=1)
    bce = np.maximum(q, 0) - q * y + np.log1p(np.exp(-np.abs(q)))
    return float(np.mean(bce + np.where(y > 0, y * ce, 0.0)))


def loss_and_grad(theta, x, f_true, y, store=None):
    p = unpack(theta)
    z, q, cache = forward(theta, x, store)
    B, L = z.shape
    y = np.asarray(y, dtype=np.float64)
    pi = softmax(z)
    t = target(f_true, L)
    logp = np.log(np.maximum(pi, 1e-300))
    ce = -(t * logp).sum(axis=1)
    bce = np.maximum(q, 0) - q * y + np.log1p(np.exp(-np.abs(q)))
    total = float(np.mean(bce + np.where(y > 0, y * ce, 0.0)))

    g = {name: np.zeros(shp) for name, shp in SHAPES}
    dq = (1.0 / (1.0 + np.exp(-q)) - y) / B
    dz = np.where((y > 0)[:, None], y[:, None] * (pi - t), 0.0) / B
    u, pooled, h4 = cache["u"], cache["pooled"], cache["h4"]
    g["wb"] = dq @ u
    g["bb"][0] = dq.sum()
    du = dq[:, None] * p["wb"][None, :] * (u > 0)
    g["Wa"] = du.T @ pooled
    g["ba"] = du.sum(axis=0)
    dpool = du @ p["Wa"]
    g["w5"] = np.einsum("bl,bcl->c", dz, h4)
    g["b5"][0] = dz.sum()
    dh = p["w5"][None, :, None] * dz[:, None, :]
    bi = np.arange(B)[:, None]
    ci = np.arange(C)[None, :]
    dh[bi, ci, cache["amax"]] += dpool[:, :C]
    dh += dpool[:, C:, None] / L
    for l in range(4, 0, -1):
        hl, hprev = cache[f"h{l}"], cache[f"h{l - 1}"]
        da = dh * (hl > 0)
        g[f"b{l}"] = da.sum(axis=(0, 2))
        Cin = hprev.shape[1]
        hp = np.zeros((B, Cin, L + 2 * HALF))
        hp[:, :, HALF:HALF + L] = hprev
        for k in range(K):
            g[f"W{l}"][:, :, k] = np.einsum("bol,bcl->oc", da, hp[:, :, k:k + L])
        if l > 1:
            dap = np.zeros((B, C, L + 2 * HALF))
            dap[:, :, HALF:HALF + L] = da
            dprev = np.zeros_like(hprev)
            W = cache[f"W{l}"]
            for k in range(K):
                # h_prev[j] feeds a[i] with i = j - k + HALF
                dprev += np.einsum("oc,bol->bcl", W[:, :, k], dap[:, :, 2 * HALF - k:2 * HALF - k + L])
            dh = dprev
    return total, pack(g)


def predict(theta, x, store=None):
    z, q, _ = forward(theta, x, store)
    pi = softmax(z)
    B, L = z.shape
    i0 = z.argmax(axis=1)
    pos = np.zeros(B)
    for b in range(B):
        lo, hi = max(0, i0[b] - WIN), min(L, i0[b] + WIN + 1)
        w = pi[b, lo:hi]
        pos[b] = float((w * np.arange(lo, hi)).sum() / w.sum())
    return pos, 1.0 / (1.0 + np.exp(-q))
