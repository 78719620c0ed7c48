"""FP64 reference of the warm-start point-patch MLP -- TEST INFRASTRUCTURE ONLY.

Network 48 -> 128 -> 128 -> 128 -> 3 (ReLU after the hidden layers), output
v, predicted normal v/|v|, loss mean_b (1 - (v_b/|v_b|) . y_b).  The weights
the network uses are the FP32 master parameters rounded to BF16 (round to
nearest, ties to even); gradients are taken with respect to those rounded
weights.  Parameter layout (flat): W1 [128][48], b1, W2 [128][128], b2,
W3 [128][128], b3, W4 [3][128], b4.

Also the patch features of a point: the offsets of its 16 nearest neighbours
(nearest first, from the exhaustive search of oracle.knn) divided by the 16th
neighbour's distance, and the warm-start combination.

And the Adam step (Kingma & Ba, "Adam: A Method for Stochastic
Optimization", Algorithm 1, with its bias correction) that trains it.

Pins (tests/test_oracle_mlp.py): finite differences of the loss for the
gradient; worked BF16 rounding values; Adam's closed forms (first step
lr g/(|g| + eps), constant-gradient steps, a worked two-step example).
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 48, 128, 3
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(a)
    out[nan] = np.nan
    return out


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        out[name] = flat[o:o + k].reshape(shp)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in SHAPES])


def effective(master):
    """The weights the network uses: master parameters rounded to BF16."""
    return bf16_round(np.asarray(master, np.float32))


def forward(params_eff, x):
    """(v, cache) for inputs x [B][48] and effective (already rounded) parameters."""
    P = unpack(params_eff)
    x = np.asarray(x, np.float64)
    h1 = np.maximum(x @ P["W1"].T + P["b1"], 0.0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0.0)
    h3 = np.maximum(h2 @ P["W3"].T + P["b3"], 0.0)
    v = h3 @ P["W4"].T + P["b4"]
    return v, (x, h1, h2, h3)


def loss(v, y, mode=0):
    """Mean over rows of 1 - c (mode 0) or 1 - c^2 (mode 1), c = (v/|v|).y;
    a row with v = 0 counts c = 0."""
    v = np.asarray(v, np.float64)
    y = np.asarray(y, np.float64)
    nv = np.linalg.norm(v, axis=1)
    c = np.where(nv > 0, (v * y).sum(1) / np.where(nv > 0, nv, 1.0), 0.0)
    return float(np.mean(1.0 - c * c if mode else 1.0 - c))


def grad(params_eff, x, y, mode=0):
    """(loss, gradient) of the mean loss with respect to the effective parameters."""
    P = unpack(params_eff)
    v, (x, h1, h2, h3) = forward(params_eff, x)
    y = np.asarray(y, np.float64)
    B = v.shape[0]
    nv = np.linalg.norm(v, axis=1, keepdims=True)
    safe = np.where(nv > 0, nv, 1.0)
    n = v / safe
    c = (n * y).sum(1, keepdims=True)
    dc = np.where(nv > 0, (y - c * n) / safe, 0.0)      # d c / d v
    dv = (-2.0 * c * dc if mode else -dc) / B
    g = {}
    g["W4"] = dv.T @ h3
    g["b4"] = dv.sum(0)
    dz3 = (dv @ P["W4"]) * (h3 > 0)
    g["W3"] = dz3.T @ h2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ P["W3"]) * (h2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ P["W2"]) * (h1 > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return loss(v, y, mode), pack(g)


def relu_margin(params_eff, x):
    """Per sample, the smallest |pre-activation| / (sum of |terms| of that
    pre-activation) over all hidden units: where it is tiny, a lower-precision
    evaluation may take the ReLU decision the other way."""
    P = unpack(params_eff)
    h = np.asarray(x, np.float64)
    m = np.full(h.shape[0], np.inf)
    for W, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        z = h @ P[W].T + P[b]
        s = np.abs(h) @ np.abs(P[W]).T + np.abs(P[b])
        m = np.minimum(m, (np.abs(z) / np.where(s > 0, s, 1.0)).min(1))
        h = np.maximum(z, 0.0)
    return m


def grad_abs(params_eff, x, y, mode=0):
    """Per parameter, the sum over the batch of |per-sample gradient term|:
    the scale of the rounding error of any floating-point batch reduction."""
    P = unpack(params_eff)
    v, (x, h1, h2, h3) = forward(params_eff, x)
    y = np.asarray(y, np.float64)
    B = v.shape[0]
    nv = np.linalg.norm(v, axis=1, keepdims=True)
    safe = np.where(nv > 0, nv, 1.0)
    n = v / safe
    c = (n * y).sum(1, keepdims=True)
    dc = np.where(nv > 0, (y - c * n) / safe, 0.0)      # d c / d v
    dv = (-2.0 * c * dc if mode else -dc) / B
    g = {}
    g["W4"] = np.abs(dv).T @ np.abs(h3)
    g["b4"] = np.abs(dv).sum(0)
    dz3 = (dv @ P["W4"]) * (h3 > 0)
    g["W3"] = np.abs(dz3).T @ np.abs(h2)
    g["b3"] = np.abs(dz3).sum(0)
    dz2 = (dz3 @ P["W3"]) * (h2 > 0)
    g["W2"] = np.abs(dz2).T @ np.abs(h1)
    g["b2"] = np.abs(dz2).sum(0)
    dz1 = (dz2 @ P["W2"]) * (h1 > 0)
    g["W1"] = np.abs(dz1).T @ np.abs(x)
    g["b1"] = np.abs(dz1).sum(0)
    return pack(g)


def patch_features(xn, idx):
    """Features [n][48] from normalised points xn and neighbour indices idx [n][16]."""
    xn = np.asarray(xn, np.float64)
    off = xn[idx] - xn[:, None, :]                       # [n][16][3]
    d16 = np.linalg.norm(off[:, -1, :], axis=1)
    inv = np.where(d16 > 0, 1.0 / np.where(d16 > 0, d16, 1.0), 0.0)
    return (off * inv[:, None, None]).reshape(len(xn), 48)


def warm_init(direction, reference, area):
    """mu = L * d/|d| (L = area, or |reference| when area = 0), negated where d . reference < 0."""
    d = np.asarray(direction, np.float64)
    nv = np.linalg.norm(d, axis=1, keepdims=True)
    L = area if (area > 0 or reference is None) else np.linalg.norm(np.asarray(reference, np.float64), axis=1,
                                                                    keepdims=True)
    f = np.where(nv > 0, L / np.where(nv > 0, nv, 1.0), 0.0)
    if reference is not None:
        f = np.where((d * np.asarray(reference, np.float64)).sum(1, keepdims=True) < 0, -f, f)
    return d * f


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step t >= 1 (Kingma & Ba, Algorithm 1), in float64:
        m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
        m_hat = m / (1 - b1^t),  v_hat = v / (1 - b2^t),
        p <- p - lr m_hat / (sqrt(v_hat) + eps).
    Returns the new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
