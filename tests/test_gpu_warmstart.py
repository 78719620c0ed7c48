"""The warm-start kernels (kNN, patch features, MLP forward/backward/Adam,
warm-start field) through the C ABI, against the FP64 references."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as M
import synth

pytestmark = pytest.mark.gpu


def _W():
    import paper_2405_16634_b300 as W
    return W


@pytest.mark.parametrize("n,seed", [(6000, 3), (777, 4), (40, 5)])
def test_knn16_matches_exhaustive_search(n, seed):
    W = _W()
    c = synth.union_cloud(max(n, 40), seed, n_tori=1, n_ellipsoids=2, noise=0.002)
    pts = np.ascontiguousarray(c.points[:n])
    t = W.Tree(torch.from_numpy(pts).cuda(), theta=0.5)
    idx, feat = W.knn16(t)
    idx, feat = idx.cpu().numpy(), feat.cpu().numpy()
    xn, _, _ = oracle.normalize(pts)
    oi, od2 = oracle.knn(xn, 16)
    # distances agree (neighbour order among equal distances may differ)
    gd2 = ((xn[idx] - xn[:, None, :]) ** 2).sum(-1)
    assert np.all(idx != np.arange(n)[:, None])
    assert np.all(np.diff(gd2, axis=1) >= -1e-12 * gd2.max())
    assert np.allclose(np.sqrt(gd2), np.sqrt(od2), rtol=1e-5, atol=1e-7)
    assert np.all([len(set(r)) == 16 for r in idx])
    # features are the oracle's features of the same neighbours
    assert np.allclose(feat, M.patch_features(xn, idx), atol=2e-6)


def test_knn16_with_outliers_and_density_contrast():
    """The benchmark cloud's recipe at 20,000 points: 10x density modulation
    and 1 % uniform outliers, whose neighbours lie far away."""
    W = _W()
    c = synth.config_cloud("union500k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    idx, _ = W.knn16(t)
    idx = idx.cpu().numpy()
    xn, _, _ = oracle.normalize(c.points)
    _, od2 = oracle.knn(xn, 16)
    gd2 = ((xn[idx] - xn[:, None, :]) ** 2).sum(-1)
    assert np.all(idx != np.arange(len(xn))[:, None])
    assert np.allclose(np.sqrt(gd2), np.sqrt(od2), rtol=1e-5, atol=1e-7)
    assert not c.valid.all()


def test_knn16_with_fewer_than_17_points():
    W = _W()
    pts = np.random.default_rng(0).uniform(0, 1, (9, 3)).astype(np.float32)
    t = W.Tree(torch.from_numpy(pts).cuda(), theta=0.5)
    idx, _ = W.knn16(t)
    idx = idx.cpu().numpy()
    assert np.all(idx[:, 8:] == -1)
    assert np.all(np.sort(idx[:, :8], axis=1) == np.array([[j for j in range(9) if j != i] for i in range(9)]))


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((B, 48)).astype(np.float32) * 0.5
    y = rng.standard_normal((B, 3))
    y = (y / np.linalg.norm(y, axis=1, keepdims=True)).astype(np.float32)
    return x, y


@pytest.mark.parametrize("mode", [0, 1])
def test_mlp_forward_and_gradient_match_fp64_reference(mode):
    W = _W()
    params = synth.mlp_init(7)
    m = W.Mlp(max_batch=5000, params=torch.from_numpy(params))
    m.set_loss(mode)
    P = M.effective(params)
    x, y = _batch(8, 6000)
    # keep samples whose ReLU decisions are clear in FP32: every |pre-activation|
    # above 3e-5 of the sum of its terms' magnitudes, well beyond the FP32
    # accumulation error of a 128-term dot product (a decision taken on the
    # other side of zero changes a whole per-sample term).  4097 of them span
    # several weight-gradient chunks and a ragged tail.
    keep = np.where(M.relu_margin(P, x) > 3e-5)[0][:4097]
    assert len(keep) == 4097
    x, y = np.ascontiguousarray(x[keep]), np.ascontiguousarray(y[keep])
    v = m.forward(torch.from_numpy(x)).cpu().numpy().astype(np.float64)
    vo, _ = M.forward(P, x)
    rms = np.sqrt(np.mean(vo ** 2))
    assert np.all(np.abs(v - vo) <= 1e-4 * np.maximum(np.abs(vo), rms))
    g, loss = m.grad(torch.from_numpy(x), torch.from_numpy(y))
    g = g.cpu().numpy().astype(np.float64)
    lo, go = M.grad(P, x, y, mode)
    assert abs(loss.item() - lo) <= 1e-5 * abs(lo)
    ga = M.grad_abs(P, x, y, mode)
    o, rep = 0, {}
    for name, shp in M.SHAPES:
        k = int(np.prod(shp))
        a, b, s_ = g[o:o + k], go[o:o + k], ga[o:o + k]
        rep[name] = (np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b) / (s_ + 1e-30)))
        o += k
    print("gradient errors (rel L2, max |err|/sum|term|):", rep)
    for name, (rel, scaled) in rep.items():
        assert rel <= 1e-4 or scaled <= 1e-5, (name, rel, scaled)


def test_mlp_training_reduces_the_loss():
    W = _W()
    m = W.Mlp(max_batch=2048, params=torch.from_numpy(synth.mlp_init(9)))
    x, y = _batch(10, 2048)
    X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    first = m.train_step(X, Y, 1e-3).item()
    for _ in range(200):
        last = m.train_step(X, Y, 1e-3).item()
    assert last < 0.5 * first
    # the parameters moved, and Adam's first step is about lr per weight
    p0 = synth.mlp_init(9)
    m2 = W.Mlp(max_batch=2048, params=torch.from_numpy(p0))
    m2.train_step(X, Y, 1e-3)
    dp = np.abs(m2.get_params().cpu().numpy() - p0)
    moved = dp > 0
    assert moved.mean() > 0.5
    assert np.all(dp <= 1e-3 * (1 + 1e-4))                 # |m_hat / sqrt(v_hat)| <= 1
    assert abs(np.median(dp[moved]) - 1e-3) < 1e-5         # = lr wherever |g| >> eps


def test_warm_init_matches_reference():
    W = _W()
    rng = np.random.default_rng(11)
    d = rng.standard_normal((1000, 3)).astype(np.float32)
    r = rng.standard_normal((1000, 3)).astype(np.float32)
    for area in (0.25, 0.0):
        mu = W.warm_init(torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda(), area).cpu().numpy()
        assert np.allclose(mu, M.warm_init(d, r, area), rtol=1e-6, atol=1e-7)
