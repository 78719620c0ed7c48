"""Pins of the FP64 warm-start MLP reference (finite differences, worked
BF16 values) and of its patch features."""
import numpy as np
import pytest

import oracle
from oracle import mlp as M
import synth


def test_bf16_round_worked_values():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 at 1.0
    x = np.array([1.0, 1 + 2 ** -8, 1 + 2 ** -8 + 2 ** -20, 1 + 3 * 2 ** -8, -2.5, 0.0], np.float32)
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -6, -2.5, 0.0])
    assert np.array_equal(M.bf16_round(x), want)
    r = M.bf16_round(np.random.default_rng(0).standard_normal(1000).astype(np.float32))
    u = r.astype(np.float32).view(np.uint32)
    assert np.all(u & 0xFFFF == 0)


def test_param_count_and_layout():
    assert M.N_PARAMS == 39683 == len(synth.mlp_init(0))
    p = M.unpack(np.arange(M.N_PARAMS, dtype=np.float64))
    assert p["W1"][0, 1] == 1 and p["b4"][-1] == M.N_PARAMS - 1


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_matches_finite_differences(mode):
    rng = np.random.default_rng(1)
    P = M.effective(synth.mlp_init(2))
    x = rng.standard_normal((64, 48))
    y = rng.standard_normal((64, 3))
    y /= np.linalg.norm(y, axis=1, keepdims=True)
    L, g = M.grad(P, x, y, mode)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(M.N_PARAMS)
        e[k] = h
        fd = (M.loss(M.forward(P + e, x)[0], y, mode) - M.loss(M.forward(P - e, x)[0], y, mode)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-8, (k, fd, g[k])


def test_loss_of_exact_prediction_is_zero():
    P = M.unpack(np.zeros(M.N_PARAMS))
    P["b4"][:] = [0.0, 0.0, 2.0]
    v, _ = M.forward(M.pack(P), np.zeros((5, 48)))
    assert M.loss(v, np.tile([0, 0, 1.0], (5, 1))) == 0.0
    assert M.loss(v, np.tile([0, 0, -1.0], (5, 1))) == 2.0
    # the sign-free loss: zero for either sign, one for a perpendicular label
    assert M.loss(v, np.tile([0, 0, -1.0], (5, 1)), 1) == 0.0
    assert M.loss(v, np.tile([0, 1.0, 0], (5, 1)), 1) == 1.0


def test_patch_features_are_scale_free_and_nearest_first():
    c = synth.union_cloud(800, 5)
    x = c.points.astype(np.float64)
    idx, d2 = oracle.knn(x, 16)
    f = M.patch_features(x, idx).reshape(-1, 16, 3)
    nrm = np.linalg.norm(f, axis=2)
    assert np.allclose(nrm[:, -1], 1.0)
    assert np.all(np.diff(nrm, axis=1) >= -1e-12)
    f2 = M.patch_features(3.0 * x, idx)
    assert np.allclose(f2, f.reshape(-1, 48))


def test_adam_closed_forms():
    """Adam's bias correction makes the first step lr g/(|g| + eps) and every
    step under a constant gradient g the same size; a worked two-step case:
    g1 = 1, g2 = -1 (b1 = 0.9, b2 = 0.999) gives m2 = -0.01, v2 = 0.001999,
    m_hat = -0.01/0.19, v_hat = 0.001999/0.001999 = 1, so p moves by
    +lr (0.01/0.19)/(1 + eps) in the second step."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p1, m, v = M.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=0)
    p, m, v = p1, m, v
    for t in range(2, 12):
        q, m, v = M.adam_step(p, g, m, v, t, 0.01)
        assert np.allclose(q - p, p1, rtol=1e-12, atol=1e-18)
        p = q
    p, m, v = M.adam_step(np.zeros(1), np.ones(1), np.zeros(1), np.zeros(1), 1, 0.1)
    q, m, v = M.adam_step(p, -np.ones(1), m, v, 2, 0.1)
    assert np.isclose(m[0], -0.01, rtol=1e-14) and np.isclose(v[0], 0.001999, rtol=1e-13)
    assert np.isclose(q[0] - p[0], 0.1 * (0.01 / 0.19) / (1 + 1e-8), rtol=1e-12)
