"""Pins of the oracle's local expansions (local_theta > 0; CPU only).

For a far node whose box gap to a target group is large next to the group's
extent, the group treecode can expand the node's far field to first order
about the centre of the group box (the target-side counterpart of the
expansions that Sec. 4.5 and Sec. 6.3 name as the way to precision control),
and the adjoint takes the exact transpose of that.  What pins it, none of it
re-typing the oracle's formulas:

  - the order of the error: with one source point the node's monopole is
    exact, so the only error left is the expansion's, of second order in
    (group extent / distance): halving the group's extent quarters it.  A
    wrong sign or factor in a first-order term leaves a first-order error,
    which only halves;
  - the same for the transposed terms, seen at the source point;
  - the transpose: <A mu, s> = <mu, A^T s> exactly;
  - the fallback: an entry is expanded only when every pair of it clears
    the cut-off, i.e. |c_g - x_B| - rho_g >= w (rho_g: the largest distance
    of the group's targets from the centre c_g); at a wider w the entry is
    summed pair by pair with the cut-off, so the result equals the one
    without expansions, bit for bit;
  - against the direct sums on a cloud: the error stays within a small
    factor of the error without expansions.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import OP_A, OP_AT, OP_G

P0 = np.array([-0.95, -0.95, -0.95])
CLUSTER_CENTRE = np.array([0.625, 0.625, 0.625])   # centre of a depth-3 cell


def _cloud(extent, seed=3):
    """P0 and a cluster of 8 points spanning `extent` around the centre of
    one depth-3 cell, so that the cluster is one target group and P0's node is
    far from it and expanded for it (gap about 2.6, extent <= 0.1)."""
    rng = np.random.default_rng(seed)
    u = rng.random((8, 3)) - 0.5
    u /= np.abs(u).max(0)                      # spans exactly [-1, 1] per axis
    x = np.concatenate([P0[None], CLUSTER_CENTRE + 0.5 * extent * u])
    return x, rng


def _structure(x, local_theta):
    t = oracle.Tree(x, 0.5, local_theta=local_theta)
    goff = t.groups()
    assert len(goff) == 3 and goff[1] == 1, goff          # {P0}, the cluster
    return t


@pytest.mark.parametrize("op", [OP_A, OP_G])
def test_local_error_order(op):
    """mu only at P0; A or G at the cluster points."""
    rel = []
    for extent in (0.1, 0.05):
        x, rng = _cloud(extent)
        mu = np.zeros((9, 3))
        mu[0] = rng.standard_normal(3)
        ex, _ = oracle.direct(op, x[:1], mu[:1], 0.0, y=x[1:])
        t0 = _structure(x, 0.0)
        t1 = _structure(x, 0.5)
        mono = t0.apply(op, mu, 0.0)[1:]
        loc = t1.apply(op, mu, 0.0)[1:]
        assert np.abs(mono - ex).max() < 1e-12 * np.abs(ex).max()     # one source: monopole exact
        rel.append(np.linalg.norm(loc - ex) / np.linalg.norm(ex))
    assert rel[0] > 0.0
    assert 3.3 < rel[0] / rel[1] < 4.7, rel


def test_local_error_order_of_the_transpose():
    """s only on the cluster; A^T at P0 gets the cluster's transposed terms."""
    rel = []
    for extent in (0.1, 0.05):
        x, rng = _cloud(extent)
        s = np.zeros(9)
        s[1:] = 1.0 + 0.3 * rng.standard_normal(8)
        ex, _ = oracle.direct(OP_AT, x, s, 0.0, y=x[:1])
        loc = _structure(x, 0.5).apply(OP_AT, s, 0.0)[:1]
        mono = _structure(x, 0.0).apply(OP_AT, s, 0.0)[:1]
        assert np.abs(mono - ex).max() < 1e-12 * np.abs(ex).max()
        rel.append(np.linalg.norm(loc - ex) / np.linalg.norm(ex))
    assert 3.3 < rel[0] / rel[1] < 4.7, rel


@pytest.fixture(scope="module")
def cloud20k():
    c = synth.config_cloud("union50k", n=20000)
    xn, _, _ = oracle.normalize(c.points)
    mu = np.nan_to_num(c.normals.astype(np.float64)) * (4.0 / len(xn))
    s = np.random.default_rng(0).standard_normal(len(xn))
    return xn, mu, s


def test_local_operator_is_transposed_exactly(cloud20k):
    xn, mu, s = cloud20k
    mu = mu + 1e-4 * np.random.default_rng(1).standard_normal(mu.shape)
    t = oracle.Tree(xn, 0.5, local_theta=0.5)
    A = t.apply(OP_A, mu, 0.004)
    AT = t.apply(OP_AT, s, 0.004)
    assert abs((A * s).sum() - (mu * AT).sum()) < 1e-12 * np.abs(A * s).sum()


def test_groups_fall_back_to_pairs_at_wide_cutoffs():
    """P0 to the cluster: |c_g - P0| = 2.713 and rho_g = 0.063, so the
    entry's bound |c_g - P0| - rho_g is 2.650; pair distances 2.697 to
    2.750.  At w = 2.71 the bound is below w: the cluster's group sums P0
    pair by pair with the cut-off (four pairs kept, four not), equal bit for
    bit to the operator without expansions.  At w = 2.5 the expansion is
    used."""
    x, rng = _cloud(0.1)
    mu = np.zeros((9, 3))
    mu[0] = rng.standard_normal(3)
    s = np.zeros(9)
    s[1:] = 1.0 + 0.3 * rng.standard_normal(8)
    t0, t1 = _structure(x, 0.0), _structure(x, 0.5)
    r = np.linalg.norm(x[1:] - x[0], axis=1)
    assert (r < 2.71).sum() == 4 and (r >= 2.71).sum() == 4
    for op, nu, rows in ((OP_A, mu, slice(1, 9)), (OP_G, mu, slice(1, 9)), (OP_AT, s, slice(0, 1))):
        wide0, wide1 = t0.apply(op, nu, 2.71)[rows], t1.apply(op, nu, 2.71)[rows]
        assert np.abs(wide0).max() > 0.0
        assert np.array_equal(wide0, wide1), op
        assert not np.array_equal(t0.apply(op, nu, 2.5)[rows], t1.apply(op, nu, 2.5)[rows]), op


def test_local_error_against_direct_sums(cloud20k):
    xn, mu, s = cloud20k
    w = 0.004
    sub = np.arange(0, len(xn), 4)
    t0 = oracle.Tree(xn, 0.5)
    t1 = oracle.Tree(xn, 0.5, local_theta=0.5)
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w, y=xn[sub])
        e0 = np.linalg.norm(t0.apply(op, nu, w)[sub] - d) / np.linalg.norm(d)
        e1 = np.linalg.norm(t1.apply(op, nu, w)[sub] - d) / np.linalg.norm(d)
        assert e1 < 1.25 * e0, (op, e0, e1)


# ---------------------------------------------------------------------------
# Clusters of consecutive groups (local_cluster = K >= 2): a far node in the
# expanded part of every member's list that is local for the cluster's box is
# expanded once about the cluster's centre.
# ---------------------------------------------------------------------------

P_LAST = np.array([0.95, 0.95, 0.95])              # last in Morton order
CLUSTER4_CENTRE = np.array([-0.625, -0.625, -0.625])


def _cluster_cloud(extent, seed=4):
    """Eight points spanning `extent` around the centre of a depth-3 cell,
    then P_LAST: with groups of 2 they form groups 0-3 (one cluster of four)
    and group 4 = {P_LAST}, whose node is far, expanded for every member and
    local for the cluster's box."""
    rng = np.random.default_rng(seed)
    u = rng.random((8, 3)) - 0.5
    u /= np.abs(u).max(0)
    x = np.concatenate([CLUSTER4_CENTRE + 0.5 * extent * u, P_LAST[None]])
    return x, rng


def _cluster_tree(x, local_theta, cluster):
    t = oracle.Tree(x, 0.5, group_size=2, local_theta=local_theta, local_cluster=cluster)
    assert np.array_equal(t.groups(), [0, 2, 4, 6, 8, 9]), t.groups()
    return t


@pytest.mark.parametrize("op", [OP_A, OP_G])
def test_cluster_error_order(op):
    """mu only at P_LAST; A or G at the eight cluster points.  The cluster's
    expansion error quarters when its extent halves, and it exceeds that of
    the four groups' own expansions (its centre lies farther from the
    targets), which shows the cluster path is the one taken."""
    rel, rel_g = [], []
    for extent in (0.1, 0.05):
        x, rng = _cluster_cloud(extent)
        mu = np.zeros((9, 3))
        mu[8] = rng.standard_normal(3)
        ex, _ = oracle.direct(op, x[8:], mu[8:], 0.0, y=x[:8])
        loc = _cluster_tree(x, 0.5, 4).apply(op, mu, 0.0)[:8]
        grp = _cluster_tree(x, 0.5, 0).apply(op, mu, 0.0)[:8]
        rel.append(np.linalg.norm(loc - ex) / np.linalg.norm(ex))
        rel_g.append(np.linalg.norm(grp - ex) / np.linalg.norm(ex))
    assert 3.3 < rel[0] / rel[1] < 4.7, rel
    assert rel[0] > 1.5 * rel_g[0], (rel, rel_g)


def test_cluster_error_order_of_the_transpose():
    """s only on the cluster; A^T at P_LAST gets the cluster's transposed
    term, built from the sums over all four member groups."""
    rel = []
    for extent in (0.1, 0.05):
        x, rng = _cluster_cloud(extent)
        s = np.zeros(9)
        s[:8] = 1.0 + 0.3 * rng.standard_normal(8)
        ex, _ = oracle.direct(OP_AT, x, s, 0.0, y=x[8:])
        loc = _cluster_tree(x, 0.5, 4).apply(OP_AT, s, 0.0)[8:]
        rel.append(np.linalg.norm(loc - ex) / np.linalg.norm(ex))
    assert 3.3 < rel[0] / rel[1] < 4.7, rel


def test_cluster_falls_back_to_pairs():
    """The cluster's bound |c_C - P_LAST| - rho_C lies below w = 2.71 while
    the pair distances straddle it: the entry is summed pair by pair, equal
    bit for bit to the operator without expansions; at w = 2.5 the cluster's
    expansion is used."""
    x, rng = _cluster_cloud(0.1)
    mu = np.zeros((9, 3))
    mu[8] = rng.standard_normal(3)
    s = np.zeros(9)
    s[:8] = 1.0 + 0.3 * rng.standard_normal(8)
    cc = 0.5 * (x[:8].min(0) + x[:8].max(0))
    bound = np.linalg.norm(cc - x[8]) - np.linalg.norm(x[:8] - cc, axis=1).max()
    r = np.linalg.norm(x[:8] - x[8], axis=1)
    assert bound < 2.71 and (r < 2.71).any() and (r >= 2.71).any() and bound > 2.5
    t0, t4 = _cluster_tree(x, 0.0, 0), _cluster_tree(x, 0.5, 4)
    for op, nu, rows in ((OP_A, mu, slice(0, 8)), (OP_G, mu, slice(0, 8)), (OP_AT, s, slice(8, 9))):
        wide0, wide4 = t0.apply(op, nu, 2.71)[rows], t4.apply(op, nu, 2.71)[rows]
        assert np.abs(wide0).max() > 0.0
        assert np.array_equal(wide0, wide4), op
        assert not np.array_equal(t0.apply(op, nu, 2.5)[rows], t4.apply(op, nu, 2.5)[rows]), op


def test_cluster_operator_is_transposed_exactly(cloud20k):
    xn, mu, s = cloud20k
    mu = mu + 1e-4 * np.random.default_rng(1).standard_normal(mu.shape)
    t = oracle.Tree(xn, 0.5, local_theta=0.5, local_cluster=4)
    A = t.apply(OP_A, mu, 0.004)
    AT = t.apply(OP_AT, s, 0.004)
    assert abs((A * s).sum() - (mu * AT).sum()) < 1e-12 * np.abs(A * s).sum()


def test_cluster_error_against_direct_sums(cloud20k):
    xn, mu, s = cloud20k
    w = 0.004
    sub = np.arange(0, len(xn), 4)
    t1 = oracle.Tree(xn, 0.5, local_theta=0.5)
    t4 = oracle.Tree(xn, 0.5, local_theta=0.5, local_cluster=4)
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w, y=xn[sub])
        e1 = np.linalg.norm(t1.apply(op, nu, w)[sub] - d) / np.linalg.norm(d)
        e4 = np.linalg.norm(t4.apply(op, nu, w)[sub] - d) / np.linalg.norm(d)
        assert e4 < 1.1 * e1, (op, e1, e4)
