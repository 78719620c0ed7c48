"""Pins of the oracle's first-order far field (far_order = 1; CPU only).

The group treecode with point-centroid representatives can add, for every far
node, the first-order Taylor terms of the kernels about the node's centroid
(the dipole-moment step toward the expansions of an FMM, which the paper
names as the way to precision control in Sec. 4.5 and as future work in
Sec. 6.3).  What pins it, none of it re-typing the oracle's formulas:

  - the order of the remaining far-field error: one far node seen from
    distance R has a relative error of order (h/R) with monopole terms and
    (h/R)^2 with the first-order terms, so doubling R halves the first and
    quarters the second -- a wrong sign or factor in any correction term
    leaves a first-order error and fails this;
  - the transpose: <A mu, s> = <mu, A^T s> exactly (A^T adds the transposed
    first-order terms through the node sums of s HPhi);
  - against the direct sums on a cloud: smaller error than the monopole
    terms at every theta, falling with theta.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import OP_A, OP_AT, OP_G


def _far_setup(op, seed=5):
    """A cluster of 12 sources (width 0.1) near (0.3, -0.2, 0.1) and two
    targets at distances 16 and 32 along a fixed direction (outside the
    normalised cube: the cluster's depth-1 octant holds only the cluster and
    is the far node of both).  nu general (not parallel)."""
    rng = np.random.default_rng(seed)
    x = np.asarray((0.3, -0.2, 0.1)) + 0.1 * (rng.random((12, 3)) - 0.5)
    direction = np.array([1.0, 0.6, -0.3]) / np.linalg.norm([1.0, 0.6, -0.3])
    c = x.mean(0)
    y = np.stack([c + 16.0 * direction, c + 32.0 * direction])
    return x, y, rng


@pytest.mark.parametrize("op", [OP_A, OP_G])
def test_far_error_order(op):
    x, y, rng = _far_setup(op)
    mu = rng.standard_normal((len(x), 3))
    xa = np.concatenate([x, y])
    nua = np.concatenate([mu, np.zeros((2, 3))])
    ex, _ = oracle.direct(op, x, mu, 0.0, y=y)
    ratio = {}
    for fo in (0, 1):
        t = oracle.Tree(xa, 0.5, leaf_size=1, far_order=fo)
        out = t.apply(op, nua, 0.0)[-2:]
        r16 = np.linalg.norm(out[0] - ex[0]) / np.linalg.norm(ex[0])
        r32 = np.linalg.norm(out[1] - ex[1]) / np.linalg.norm(ex[1])
        ratio[fo] = r16 / r32
    assert 1.6 < ratio[0] < 2.5, ratio
    assert 3.3 < ratio[1] < 4.7, ratio


def test_far_error_order_of_the_transpose():
    """A^T at the cluster points, s only at the two far targets: each
    target's contribution to a cluster point passes through the cluster's
    far node, so its error has the same order as A's."""
    x, y, rng = _far_setup(OP_AT)
    xa = np.concatenate([x, y])
    ratio = {}
    for fo in (0, 1):
        rel = []
        for k in range(2):                       # s = 1 at one target, 0 elsewhere
            s = np.zeros(len(xa))
            s[len(x) + k] = 1.0
            ex, _ = oracle.direct(OP_AT, xa, s, 0.0, y=x)
            out = oracle.Tree(xa, 0.5, leaf_size=1, far_order=fo).apply(OP_AT, s, 0.0)[:len(x)]
            rel.append(np.linalg.norm(out - ex) / np.linalg.norm(ex))
        ratio[fo] = rel[0] / rel[1]
    assert 1.6 < ratio[0] < 2.5, ratio
    assert 3.3 < ratio[1] < 4.7, ratio


@pytest.fixture(scope="module")
def cloud20k():
    c = synth.config_cloud("union50k", n=20000)
    xn, _, _ = oracle.normalize(c.points)
    mu = c.normals.astype(np.float64) * (4.0 / len(xn))
    s = np.random.default_rng(0).standard_normal(len(xn))
    return xn, mu, s


def test_first_order_operator_is_transposed_exactly(cloud20k):
    xn, mu, s = cloud20k
    rng = np.random.default_rng(1)
    mu = mu + 1e-4 * rng.standard_normal(mu.shape)
    t = oracle.Tree(xn, 0.5, far_order=1)
    A = t.apply(OP_A, mu, 0.01)
    AT = t.apply(OP_AT, s, 0.01)
    assert abs((A * s).sum() - (mu * AT).sum()) < 1e-12 * np.abs(A * s).sum()


def test_first_order_error_against_direct_sums(cloud20k):
    xn, mu, s = cloud20k
    w = 0.004
    sub = np.arange(0, len(xn), 4)
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w, y=xn[sub])
        prev = np.inf
        for theta in (1.0, 0.8, 0.5, 0.3):
            e = [np.linalg.norm(oracle.Tree(xn, theta, far_order=fo).apply(op, nu, w)[sub] - d)
                 / np.linalg.norm(d) for fo in (0, 1)]
            assert e[1] < 0.7 * e[0], (op, theta, e)
            assert e[1] < prev, (op, theta, e)
            prev = e[1]
