"""Pins of the oracle's two treecodes against facts fixed by the paper and by
mathematics (CPU only).

* ``oracle.PaperTree``: Alg. 4 as printed -- per target, from the root, node B
  far iff |y - x_{B,nu}| > c width(B), with the nu-representatives of
  Eq. 13-14 -- over a plain geometric octree (Sec. 4.5).
* ``oracle.Tree`` in rep_mode 0: the group treecode with the paper's
  |nu|-weighted representatives and the s-representative A^T.

What pins them, none of it re-typing the oracle's formulas:
  - a far node worked by hand (exact rationals times 1/pi) for A, G and A^T;
  - the representative does not move when the sign of one source's nu flips
    (Eq. 13 weights by |nu|), so the far term stays proportional to nu_B;
  - for parallel, same-sign nu the |nu|-weighted centroid is the centre of
    the nu distribution, so the far-field error of one node falls as R^-4 with
    the target distance R (the first-order term of the Taylor series
    vanishes), where any other representative leaves an R^-3 error;
  - theta -> 0 reaches the direct sums, and the error against them falls
    with theta;
  - every node's points lie in its cube, octants partition their parent, the
    split rule holds;
  - the metrics of Eq. 16-17 on a three-point worked example.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import OP_A, OP_AT, OP_G

# ---------------------------------------------------------------------------
# A worked far node.  Two sources on the x axis,
#   x1 = (1/2, 1/2, 1/2),  x2 = (7/8, 1/2, 1/2),
# with weights of magnitude 2 and 1 and opposite signs, and one target
#   y = (-7/8, 1/2, 1/2).
# With theta = 1/2 (c = 2): the sources share the octree cell [1/2, 1]^3 of
# depth 2 (width 1/2) and split at depth 3.  Eq. 13 puts that node's
# representative at (2 x1 + 1 x2)/3 = (5/8, 1/2, 1/2), at distance 3/2 from y:
# 3/2 > c * 1/2 = 1, so the node is far, while its parent (width 1, c w = 2)
# and the root (c w = 4) are not.  Eq. 14 gives nu_B = nu1 + nu2.
#   A^T, s = (2, -1):  s_B = 1,  d = y - x_B = (-3/2, 0, 0),  |d| = 3/2
#       s_B gradPhi(x_B - y) = s_B d/(4 pi |d|^3) = -(3/2)/(4 pi 27/8) = -1/(9 pi) e_x
#   A,  mu = ((2,0,0), (-1,0,0)):  mu_B = e_x
#       gradPhi(y - x_B) . mu_B = -(d . mu_B)/(4 pi |d|^3) = (3/2)/(27 pi/2) = 1/(9 pi)
#   G:  -HPhi(d) mu_B = mu_B/(4 pi |d|^3) - 3 d (d . mu_B)/(4 pi |d|^5)
#       = (1 - 3) e_x/(4 pi 27/8) = -4/(27 pi) e_x
# A representative weighted by the signed s instead of |s| would sit at
# (2 x1 - x2)/1 = (1/8, 1/2, 1/2) (A^T = -1/pi e_x); one without the
# normalisation by sum |nu| at (15/8, 1/2, 1/2).  The group treecode in
# rep_mode 1 uses the point centroid (11/16, 1/2, 1/2) for A and G instead:
# |d| = 25/16,  A = 64/(625 pi),  G = -2048/(15625 pi) e_x.  Its A^T is the
# exact transpose of that A: the value at y collects the terms in which y is
# the source, and y's leaf is near for both other points, so it is the direct
# sum  s1 (y - x1)/(4 pi (11/8)^3) + s2 (y - x2)/(4 pi (7/4)^3)
#      = (-32/121 + 4/49)/pi e_x = -1084/(5929 pi) e_x.
# ---------------------------------------------------------------------------
X_PAIR = np.array([[0.5, 0.5, 0.5], [0.875, 0.5, 0.5]])
Y_FAR = np.array([[-0.875, 0.5, 0.5]])
S_PAIR = np.array([2.0, -1.0])
MU_PAIR = np.array([[2.0, 0.0, 0.0], [-1.0, 0.0, 0.0]])
PAPER_REP = {OP_AT: [-1 / (9 * math.pi), 0, 0], OP_A: [1 / (9 * math.pi)], OP_G: [-4 / (27 * math.pi), 0, 0]}
CENTROID_REP = {OP_AT: [-1084 / (5929 * math.pi), 0, 0], OP_A: [64 / (625 * math.pi)],
                OP_G: [-2048 / (15625 * math.pi), 0, 0]}


@pytest.mark.parametrize("op", [OP_A, OP_G, OP_AT])
def test_paper_tree_worked_far_node(op):
    P = oracle.PaperTree(X_PAIR, leaf_size=1)
    nu = S_PAIR if op == OP_AT else MU_PAIR
    out, info = P.apply(op, nu, 0.0, 0.5, y=Y_FAR)
    assert info == {"far": 1, "near": 0}
    assert np.allclose(np.ravel(out), PAPER_REP[op], rtol=1e-14, atol=0)
    # the cut-off applies to the far term too ("modified by w", Alg. 4)
    out, _ = P.apply(op, nu, 1.6, 0.5, y=Y_FAR)
    assert np.all(np.ravel(out) == 0.0)


@pytest.mark.parametrize("op", [OP_A, OP_G, OP_AT])
@pytest.mark.parametrize("rep_mode", [0, 1])
def test_group_tree_worked_far_node(op, rep_mode):
    """The same far node through the group treecode (targets are the tree's
    own points, so the target joins the cloud with nu = 0)."""
    x = np.concatenate([X_PAIR, Y_FAR])
    nu = np.concatenate([S_PAIR, [0.0]]) if op == OP_AT else np.concatenate([MU_PAIR, [[0.0, 0.0, 0.0]]])
    t = oracle.Tree(x, 0.5, leaf_size=1)
    assert t.counts()[0] >= 1
    out = t.apply(op, nu, 0.0, rep_mode=rep_mode)
    want = PAPER_REP[op] if rep_mode == 0 else CENTROID_REP[op]
    assert np.allclose(np.ravel(out[2]), want, rtol=1e-14, atol=0)


def _cluster(seed, m=12, h=0.05, centre=(0.3, -0.2, 0.1)):
    rng = np.random.default_rng(seed)
    return np.asarray(centre) + h * (rng.random((m, 3)) - 0.5), rng


@pytest.mark.parametrize("tree", ["paper", "group"])
def test_representative_ignores_the_sign_of_nu(tree):
    """Eq. 13 weights each point by |nu_i|, so flipping the sign of any s_i
    leaves x_{B,s} where it is, and the far term s_B gradPhi(x_B - y) stays
    proportional to s_B = sum s_i.  A target at distance 6 from a cluster of
    width 0.05 sees the whole cluster as one far node (also the root, whose
    c w = 4) in the paper's tree; in the group treecode the cluster's depth-1
    octant is the far node."""
    if tree == "paper":
        x, rng = _cluster(3)
        y = np.array([[6.3, -0.2, 0.1]])
    else:
        # inside the normalised cube: the cluster fills one depth-3 cell, the
        # target sits in the opposite octant (gap 2.5 > c width = 2 at depth 1)
        x, rng = _cluster(3, h=0.02, centre=(-0.7, -0.7, -0.7))
        y = np.array([[0.8, 0.8, 0.8]])
    mag = 0.5 + rng.random(len(x))
    ratios = []
    for k in range(6):
        sgn = np.where(rng.random(len(x)) < 0.5, -1.0, 1.0)
        sgn[0] = 1.0
        s = mag * sgn
        if abs(s.sum()) < 0.3:
            continue
        if tree == "paper":
            out, info = oracle.PaperTree(x, leaf_size=1).apply(OP_AT, s, 0.0, 0.5, y=y)
            assert info["far"] == 1
            v = out[0]
        else:
            xa = np.concatenate([x, y])
            v = oracle.Tree(xa, 0.5, leaf_size=1).apply(OP_AT, np.concatenate([s, [0.0]]), 0.0, rep_mode=0)[-1]
        ratios.append(v / s.sum())
    assert len(ratios) >= 3
    for r in ratios[1:]:
        assert np.allclose(r, ratios[0], rtol=1e-12, atol=0)


@pytest.mark.parametrize("op", [OP_A, OP_G, OP_AT])
def test_far_error_is_second_order_for_parallel_nu(op):
    """With nu_i = a_i e, a_i > 0 (a consistently oriented patch), the
    |nu|-weighted centroid of Eq. 13 is the first moment's centre, so the
    first-order Taylor term of the far approximation cancels and its error
    falls as R^-4 (A, A^T) or R^-5 (G) relative to the R^-2 (R^-3) size of the
    term: doubling R divides the relative error by about 4.  The point
    centroid (unequal a_i) leaves the first-order term: the relative error
    only halves."""
    x, rng = _cluster(5, h=0.1)
    a = 0.2 + rng.random(len(x))
    e = np.array([0.36, 0.48, 0.8])
    nu = a if op == OP_AT else a[:, None] * e
    direction = np.array([1.0, 0.6, -0.3]) / np.linalg.norm([1.0, 0.6, -0.3])
    centre = x.mean(0)
    rel = {}
    for R in (8.0, 16.0, 32.0):
        y = (centre + R * direction)[None, :]
        ex, _ = oracle.direct(op, x, nu, 0.0, y=y)
        out, info = oracle.PaperTree(x, leaf_size=1).apply(op, nu, 0.0, 0.5, y=y)
        assert info["far"] == 1
        rel[R] = np.linalg.norm(out - ex) / np.linalg.norm(ex)
    assert 3.3 < rel[8.0] / rel[16.0] < 4.7, rel
    assert 3.3 < rel[16.0] / rel[32.0] < 4.7, rel
    # the group treecode's point centroid: first order (A and G; its A^T is
    # the transpose of its A, which approximates the targets' side instead)
    if op == OP_AT:
        return
    xa = np.concatenate([x, (centre + 16.0 * direction)[None, :], (centre + 32.0 * direction)[None, :]])
    nua = np.concatenate([nu, np.zeros((2,) + nu.shape[1:])])
    t = oracle.Tree(xa, 0.5, leaf_size=1)
    exa, _ = oracle.direct(op, x, nu, 0.0, y=xa[-2:])
    tc = t.apply(op, nua, 0.0, rep_mode=1)[-2:]
    r16 = np.linalg.norm(tc[0] - exa[0]) / np.linalg.norm(exa[0])
    r32 = np.linalg.norm(tc[1] - exa[1]) / np.linalg.norm(exa[1])
    assert 1.6 < r16 / r32 < 2.5, (r16, r32)


@pytest.fixture(scope="module")
def cloud20k():
    c = synth.config_cloud("union50k", n=20000)
    xn, _, _ = oracle.normalize(c.points)
    mu = c.normals.astype(np.float64) * (4.0 / len(xn))
    s = np.random.default_rng(0).standard_normal(len(xn))
    return xn, mu, s


def test_paper_octree_cells(cloud20k):
    """Every node's points lie in its cube (centre c, width 2/2^depth, points
    on a face go to the upper octant); the children's ranges partition the
    parent's; inner nodes hold more than leaf_size points and are shallower
    than D; leaves hold at most leaf_size points unless at depth D."""
    xn = cloud20k[0]
    for leaf, depth in ((1, 15), (8, 15), (4, 3)):
        P = oracle.PaperTree(xn, leaf_size=leaf, max_depth=depth)
        nd = P.nodes()
        idx = nd["idx"]
        assert np.array_equal(np.sort(idx), np.arange(len(xn)))
        inner = nd["nchild"] > 0
        assert np.all(nd["count"][inner] > leaf) and np.all(nd["depth"][inner] < depth)
        assert np.all((nd["count"][~inner] <= leaf) | (nd["depth"][~inner] == depth))
        leaves = np.where(~inner)[0]
        assert nd["count"][leaves].sum() == len(xn)
        for b in range(0, len(nd["start"]), max(1, len(nd["start"]) // 3000)):
            p = xn[idx[nd["start"][b]:nd["start"][b] + nd["count"][b]]]
            half = 2.0 ** (-int(nd["depth"][b]))
            lo, hi = nd["ctr"][b] - half, nd["ctr"][b] + half
            assert np.all(p >= lo) and np.all(p < hi) or nd["depth"][b] == 0
        assert nd["count"][0] == len(xn) and nd["depth"][0] == 0


def test_paper_tree_limit_equals_direct(cloud20k):
    xn, mu, s = cloud20k
    xn, mu, s = xn[:4000], mu[:4000], s[:4000]
    w = 0.01
    P = oracle.PaperTree(xn, leaf_size=1)
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w)
        out, info = P.apply(op, nu, w, 1e-12)
        assert info["far"] == 0 and info["near"] == 4000 * 4000
        assert np.abs(out - d).max() <= 1e-12 * np.abs(d).max()


@pytest.mark.parametrize("tree", ["paper", "group_rep0", "group_rep1"])
def test_error_vs_direct_falls_with_theta(cloud20k, tree):
    xn, mu, s = cloud20k
    w = 0.01
    sub = np.arange(0, len(xn), 5)
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w, y=xn[sub])
        errs = []
        for theta in (0.8, 0.5, 0.3, 0.15):
            if tree == "paper":
                out, _ = oracle.PaperTree(xn, leaf_size=1).apply(op, nu, w, theta, y=xn[sub])
            else:
                out = oracle.Tree(xn, theta).apply(op, nu, w, rep_mode=int(tree[-1]))[sub]
            errs.append(np.linalg.norm(out - d) / np.linalg.norm(d))
        assert all(a > b for a, b in zip(errs, errs[1:])), (op, errs)
        assert errs[-1] < 2e-2, (op, errs)


def test_paper_tree_ambiguity_budget_covers_the_other_branch():
    """A far decision within amb_tol of the threshold: the budget holds the
    difference between taking the node as far and opening it, so the result
    of either decision lies within it."""
    x = X_PAIR
    # |y - x_B| = c width(B) (1 + 1e-7): far in FP64, but within a 1e-5 band
    r = 1.0 * math.sqrt(1 + 2e-7)
    y = np.array([[0.625 - r, 0.5, 0.5]])
    P = oracle.PaperTree(x, leaf_size=1)
    far, info = P.apply(OP_AT, S_PAIR, 0.0, 0.5, y=y, amb_tol=1e-5)
    assert info["far"] == 1
    opened, _ = oracle.direct(OP_AT, x, S_PAIR, 0.0, y=y)
    assert np.linalg.norm(far - opened) > 0
    assert np.linalg.norm(far - opened) <= info["amb"][0] * (1 + 1e-12)


def test_metrics_worked_example():
    """Eq. 16-17 on three points: ground truth e_x, e_y, e_z; reconstructed
    e_x, -e_y and 5 (0, 0.6, 0.8) (unnormalised).  The dot products of the unit
    normals are 1, -1, 0.8: P_co = 2/3 and AE_pcd = (0 + 1 + 0.1)/3 = 11/30."""
    gt = np.eye(3)
    rec = np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 3.0, 4.0]])
    assert oracle.p_co(gt, rec) == pytest.approx(2 / 3, abs=1e-15)
    assert oracle.ae_pcd(gt, rec) == pytest.approx(11 / 30, abs=1e-15)
    valid = np.array([True, False, True])
    assert oracle.p_co(gt, rec, valid) == 1.0
    assert oracle.ae_pcd(gt, rec, valid) == pytest.approx(0.05, abs=1e-15)
