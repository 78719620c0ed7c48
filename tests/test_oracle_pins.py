"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each compares the oracle with a
closed form, an exact identity, an invariance, a worked two-point example,
a finite-difference derivative, or an exhaustive search.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import OP_A, OP_AT, OP_G


def _sphere(n, radius=1.0):
    c = synth.fibonacci_sphere(n, radius)
    x = c.points.astype(np.float64)
    nrm = x / np.linalg.norm(x, axis=1, keepdims=True)
    return x, nrm


def _random_cloud(n, seed):
    c = synth.union_cloud(n, seed, n_tori=1, n_ellipsoids=1)
    rng = np.random.default_rng(seed + 1)
    return c.points.astype(np.float64), rng.standard_normal((n, 3)), rng.standard_normal(n)


# ---------------------------------------------------------------------------
# Direct sums: closed forms of Thm. 1 on spheres
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("radius", [0.5, 2.0])
def test_centre_value_is_exactly_one(radius):
    """F(0) with mu_j = (4 pi R^2 / N) n_j on a sphere of radius R is exactly 1
    for any placement of the points: each term is (x_j . n_j) a/(4 pi R^3) = 1/N."""
    c = synth.sphere(3001, seed=5, radius=radius)
    x = c.points.astype(np.float64)
    n = x / np.linalg.norm(x, axis=1, keepdims=True)
    x = n * radius
    mu = n * (4 * math.pi * radius ** 2 / len(x))
    out, _ = oracle.direct(OP_A, x, mu, 0.0, y=np.zeros((1, 3)))
    assert abs(out[0] - 1.0) < 1e-12


def test_two_point_worked_example_and_cutoff():
    """Source at (1,0,0) with mu = (2,0,0), target at the origin:
    gradPhi(0 - x) . mu = x.mu/(4 pi |x|^3) = 2/(4 pi); zero once w > 1."""
    x = np.array([[1.0, 0.0, 0.0]])
    mu = np.array([[2.0, 0.0, 0.0]])
    y = np.zeros((1, 3))
    a, _ = oracle.direct(OP_A, x, mu, 0.5, y=y)
    assert abs(a[0] - 2.0 / (4 * math.pi)) < 1e-15
    a, _ = oracle.direct(OP_A, x, mu, 1.5, y=y)
    assert a[0] == 0.0
    # G: -HPhi(d) mu with d = y - x = (-1,0,0): mu/(4pi) - 3 d (d.mu)/(4pi) = (2 - 6)/(4 pi) e_x
    g, _ = oracle.direct(OP_G, x, mu, 0.5, y=y)
    assert np.allclose(g[0], [-4.0 / (4 * math.pi), 0, 0], atol=1e-15)
    # A^T with s = 3 at the source: s gradPhi(x - y) = s (y - x)/(4 pi) = (-3/(4 pi), 0, 0)
    at, _ = oracle.direct(OP_AT, x, np.array([3.0]), 0.5, y=y)
    assert np.allclose(at[0], [-3.0 / (4 * math.pi), 0, 0], atol=1e-15)


@pytest.mark.parametrize("w", [0.1, 0.2])
def test_sphere_surface_closed_forms(w):
    """Continuum limits on the unit sphere with outward mu = (4 pi/N) n:
    A_w = 1/2 - w/4,  G_w = (1/(2w) - w/8) n,  (A_w^T 1)_j = (N/4pi)(1/2 - w/4) n_j."""
    N = 20000
    x, n = _sphere(N)
    a = 4 * math.pi / N
    A, _ = oracle.direct(OP_A, x, n * a, w)
    G, _ = oracle.direct(OP_G, x, n * a, w)
    AT, _ = oracle.direct(OP_AT, x, np.ones(N), w)
    assert abs(A.mean() - (0.5 - w / 4)) < 2e-3
    g_rad = (G * n).sum(1)
    assert abs(g_rad.mean() / (1 / (2 * w) - w / 8) - 1) < 1e-2
    assert np.abs(G - g_rad[:, None] * n).max() < 0.05 * abs(1 / (2 * w) - w / 8)
    at_rad = (AT * n).sum(1)
    assert abs(at_rad.mean() / (N / (4 * math.pi) * (0.5 - w / 4)) - 1) < 2e-3


def test_sphere_closed_form_error_shrinks_with_n():
    w = 0.15
    errs = []
    for N in (2000, 8000, 32000):
        x, n = _sphere(N)
        G, _ = oracle.direct(OP_G, x, n * (4 * math.pi / N), w)
        errs.append(abs((G * n).sum(1).mean() / (1 / (2 * w) - w / 8) - 1))
    assert errs[0] > errs[1] > errs[2]


def test_inside_outside_indicator():
    """F -> 1 inside, 0 outside (Thm. 1) for queries well away from the surface."""
    N = 20000
    x, n = _sphere(N)
    mu = n * (4 * math.pi / N)
    qi = synth.ball_queries(200, 3, (0, 0, 0), 0.7).astype(np.float64)
    qo = synth.ball_queries(200, 4, (0, 0, 0), 1.0).astype(np.float64)
    qo = qo / np.linalg.norm(qo, axis=1, keepdims=True) * (1.3 + np.linalg.norm(qo, axis=1, keepdims=True))
    Fi, _ = oracle.direct(OP_A, x, mu, 0.0, y=qi)
    Fo, _ = oracle.direct(OP_A, x, mu, 0.0, y=qo)
    assert np.abs(Fi - 1).max() < 1e-3
    assert np.abs(Fo).max() < 1e-3


def test_G_is_minus_gradient_of_F():
    """G(mu)(y) = -grad F(y; mu) (Eq. 8-10), checked by central differences of A."""
    x, mu, _ = _random_cloud(400, 11)
    y = synth.ball_queries(20, 12, x.mean(0), 0.5).astype(np.float64)
    # keep queries at least 0.05 away from every source
    dmin = np.sqrt(((y[:, None, :] - x[None]) ** 2).sum(-1)).min(1)
    y = y[dmin > 0.05]
    G, _ = oracle.direct(OP_G, x, mu, 0.0, y=y)
    h = 1e-5
    fd = np.zeros_like(G)
    for k in range(3):
        e = np.zeros(3); e[k] = h
        Fp, _ = oracle.direct(OP_A, x, mu, 0.0, y=y + e)
        Fm, _ = oracle.direct(OP_A, x, mu, 0.0, y=y - e)
        fd[:, k] = -(Fp - Fm) / (2 * h)
    assert np.abs(G - fd).max() < 1e-5 * np.abs(G).max()


def test_direct_adjointness_and_G_symmetry():
    """<A mu, s> = <mu, A^T s> and <nu, G mu> = <mu, G nu> (HPhi is even and symmetric)."""
    x, mu, s = _random_cloud(1500, 21)
    nu = np.random.default_rng(3).standard_normal(mu.shape)
    w = 0.02
    A, _ = oracle.direct(OP_A, x, mu, w)
    AT, _ = oracle.direct(OP_AT, x, s, w)
    lhs, rhs = (A * s).sum(), (mu * AT).sum()
    assert abs(lhs - rhs) < 1e-12 * (np.abs(A * s).sum())
    Gm, _ = oracle.direct(OP_G, x, mu, w)
    Gn, _ = oracle.direct(OP_G, x, nu, w)
    assert abs((nu * Gm).sum() - (mu * Gn).sum()) < 1e-12 * np.abs(nu * Gm).sum()


def test_scaling_invariance():
    """x -> kx, mu -> k^2 mu, w -> kw: A unchanged, G scales 1/k, A^T scales 1/k^2."""
    x, mu, s = _random_cloud(800, 31)
    w, k = 0.02, 3.0
    for op, nu, p in ((OP_A, mu, 0), (OP_G, mu, -1), (OP_AT, s, -2)):
        o1, _ = oracle.direct(op, x, nu, w)
        o2, _ = oracle.direct(op, k * x, nu * (k * k if op != OP_AT else 1.0), k * w)
        assert np.allclose(o2, o1 * k ** p, rtol=1e-10, atol=1e-10 * np.abs(o1).max())


def test_rotation_equivariance():
    x, mu, s = _random_cloud(800, 41)
    R = np.linalg.qr(np.random.default_rng(5).standard_normal((3, 3)))[0]
    w = 0.02
    A1, _ = oracle.direct(OP_A, x, mu, w)
    A2, _ = oracle.direct(OP_A, x @ R.T, mu @ R.T, w)
    assert np.allclose(A1, A2, atol=1e-10 * np.abs(A1).max())
    G1, _ = oracle.direct(OP_G, x, mu, w)
    G2, _ = oracle.direct(OP_G, x @ R.T, mu @ R.T, w)
    assert np.allclose(G1 @ R.T, G2, atol=1e-10 * np.abs(G1).max())
    T1, _ = oracle.direct(OP_AT, x, s, w)
    T2, _ = oracle.direct(OP_AT, x @ R.T, s, w)
    assert np.allclose(T1 @ R.T, T2, atol=1e-10 * np.abs(T1).max())


def test_ambiguity_budget_flags_boundary_pairs():
    """A pair at distance exactly w is flagged, and the budget is its |term|."""
    x = np.array([[0.25, 0.0, 0.0], [0.0, 0.75, 0.0]])
    mu = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    y = np.zeros((1, 3))
    out, b = oracle.direct(OP_A, x, mu, 0.25, y=y, amb_tol=1e-6)
    assert abs(b["amb"][0] - 0.25 / (4 * math.pi * 0.25 ** 3)) < 1e-12
    assert abs(b["abssum"][0] - (0.25 / (4 * math.pi * 0.25 ** 3) + 0.75 / (4 * math.pi * 0.75 ** 3))) < 1e-12
    assert abs(out[0] - (0.25 / (4 * math.pi * 0.25 ** 3) + 0.75 / (4 * math.pi * 0.75 ** 3))) < 1e-12


# ---------------------------------------------------------------------------
# Normalisation (Sec. 5.1.1)
# ---------------------------------------------------------------------------

def test_coincident_pairs_never_count():
    """Exact duplicates (the self term, repeated samples) contribute nothing,
    also at w = 0; pairs just above the 2^-20 floor do."""
    x = np.array([[0.5, 0.0, 0.0], [0.5, 0.0, 0.0], [0.5 + 2.0 ** -19, 0.0, 0.0]])
    mu = np.array([[1.0, 0, 0], [1.0, 0, 0], [1.0, 0, 0]])
    out, _ = oracle.direct(OP_A, x, mu, 0.0)
    d = 2.0 ** -19
    assert out[0] == pytest.approx(d / (4 * math.pi * d ** 3))
    assert out[2] == pytest.approx(-2 * d / (4 * math.pi * d ** 3))


def test_normalization_margin():
    c = synth.union_cloud(5000, 7)
    xn, ctr, s = oracle.normalize(c.points)
    lo, hi = xn.min(0), xn.max(0)
    assert abs(max(np.abs(lo).max(), np.abs(hi).max()) - 10.0 / 11.0) < 1e-12
    assert np.allclose(lo + hi, 0.0, atol=1e-12)     # centred bounding box


# ---------------------------------------------------------------------------
# Treecode
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cloud20k():
    c = synth.config_cloud("union50k", n=20000)
    xn, _, _ = oracle.normalize(c.points)
    rng = np.random.default_rng(0)
    mu = synth.random_unit_vectors(len(xn), 1) * 1e-4
    return xn, mu, rng.standard_normal(len(xn))


def test_tree_structure_invariants(cloud20k):
    xn = cloud20k[0]
    t = oracle.Tree(xn, 0.5, leaf_size=32, max_depth=15)
    nd = t.nodes()
    xs = xn[t.perm()]
    leaves = np.where(nd["nchild"] == 0)[0]
    # leaves partition the sorted points
    order = np.argsort(nd["start"][leaves])
    st, ct = nd["start"][leaves][order], nd["count"][leaves][order]
    assert st[0] == 0 and np.all(st[1:] == st[:-1] + ct[:-1]) and st[-1] + ct[-1] == len(xn)
    # split rule
    inner = nd["nchild"] > 0
    assert np.all(nd["count"][inner] > 32) and np.all(nd["depth"][inner] < 15)
    assert np.all((nd["count"][~inner] <= 32) | (nd["depth"][~inner] == 15))
    # every node's points lie in its dyadic cell of width 2/2^depth
    for b in range(len(nd["start"])):
        p = xs[nd["start"][b]:nd["start"][b] + nd["count"][b]]
        cell = np.floor((p + 1.0) * 2.0 ** (nd["depth"][b] - 1))
        assert np.all(cell == cell[0])
        # children cover the parent's range
        if nd["nchild"][b]:
            kids = np.where(nd["parent"] == b)[0]
            assert nd["count"][kids].sum() == nd["count"][b]


def test_tree_lists_partition_sources_and_satisfy_alg4(cloud20k):
    """For every target group, far nodes and near leaves cover each source
    exactly once, and every far use passes Alg. 4's per-target test
    |x_i - x_B| > c * width(B) (x_B the node centroid, c = 1/theta)."""
    xn = cloud20k[0]
    theta = 0.5
    t = oracle.Tree(xn, theta)
    nd = t.nodes()
    fo, fi, no, ni = t.lists()
    go = t.groups()
    xs = xn[t.perm()]
    n = len(xn)
    assert go[0] == 0 and go[-1] == n and np.all(np.diff(go) >= 1) and np.all(np.diff(go) <= 32)
    for g in range(0, len(fo) - 1, 37):
        cover = np.zeros(n, np.int32)
        for b in fi[fo[g]:fo[g + 1]]:
            cover[nd["start"][b]:nd["start"][b] + nd["count"][b]] += 1
            ti = xs[go[g]:go[g + 1]]
            dist = np.linalg.norm(ti - nd["cent"][b], axis=1)
            assert np.all(dist > (1 / theta) * 2.0 ** (1 - nd["depth"][b]))
        for b in ni[no[g]:no[g + 1]]:
            assert nd["nchild"][b] == 0
            cover[nd["start"][b]:nd["start"][b] + nd["count"][b]] += 1
        assert np.all(cover == 1)


def test_groups_never_straddle_distant_leaves(cloud20k):
    """Target groups are runs of at most 32 sorted points that end where two
    consecutive points' leaves share no ancestor within GROUP_SLACK levels of
    the deeper one or no ancestor at depth GROUP_MIN_DEPTH; with a negative
    slack they are plain runs of 32."""
    xn = cloud20k[0]
    t = oracle.Tree(xn, 0.5)
    nd = t.nodes()
    go = t.groups()
    leaves = np.where(nd["nchild"] == 0)[0]
    leaf_of = np.zeros(len(xn), np.int64)
    for b in leaves:
        leaf_of[nd["start"][b]:nd["start"][b] + nd["count"][b]] = b
    # ancestors of every node
    def ancestors(b):
        out = []
        while b >= 0:
            out.append(b)
            b = nd["parent"][b]
        return out
    # cell of depth D of each sorted point, from its 15-bit quantised coordinates
    xs = xn[t.perm()]
    q = np.clip(np.floor((xs + 1.0) * 16384.0), 0, 32767).astype(np.int64)
    cell = q >> (15 - oracle.GROUP_MIN_DEPTH)
    for g in range(len(go) - 1):
        for k in range(go[g] + 1, go[g + 1]):
            a, b = leaf_of[k - 1], leaf_of[k]
            d = max(nd["depth"][a], nd["depth"][b])
            common = set(ancestors(a)) & set(ancestors(b))
            assert max(nd["depth"][c] for c in common) >= d - oracle.GROUP_SLACK
            assert np.array_equal(cell[k - 1], cell[k])
    fixed = oracle.Tree(xn, 0.5, group_slack=-1).groups()
    assert np.array_equal(fixed, np.minimum(np.arange(len(fixed)) * 32, len(xn)))


def test_tree_limit_equals_direct(cloud20k):
    xn, mu, s = cloud20k
    xn, mu, s = xn[:4000], mu[:4000], s[:4000]
    w = 0.01
    t = oracle.Tree(xn, 1e-12)
    assert t.counts()[2] == 0          # no far interactions left
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w)
        for rm in (0, 1):
            tr = t.apply(op, nu, w, rep_mode=rm)
            assert np.abs(tr - d).max() <= 1e-12 * np.abs(d).max()


def test_tree_error_decreases_with_theta(cloud20k):
    xn, _, s = cloud20k
    # a smooth, consistently oriented field: the ground-truth-like normals of
    # a union cloud, scaled by the mean area per point
    c = synth.config_cloud("union50k", n=20000)
    mu = c.normals.astype(np.float64) * (4.0 / len(xn))
    w = 0.01
    for op, nu in ((OP_A, mu), (OP_G, mu), (OP_AT, s)):
        d, _ = oracle.direct(op, xn, nu, w)
        errs = []
        for theta in (0.8, 0.5, 0.3, 0.15):
            tr = oracle.Tree(xn, theta).apply(op, nu, w)
            errs.append(np.linalg.norm(tr - d) / np.linalg.norm(d))
        assert all(a > b for a, b in zip(errs, errs[1:])), errs
        assert errs[-1] < 2e-3


def test_tree_exact_adjoint(cloud20k):
    """rep_mode 1 makes A_tree linear; its A^T is the exact transpose."""
    xn, mu, s = cloud20k
    t = oracle.Tree(xn, 0.5)
    A = t.apply(OP_A, mu, 0.01)
    AT = t.apply(OP_AT, s, 0.01)
    assert abs((A * s).sum() - (mu * AT).sum()) < 1e-12 * np.abs(A * s).sum()


def test_tree_query_targets_match_direct_in_limit(cloud20k):
    xn, mu, _ = cloud20k
    q = synth.ball_queries(500, 9, (0, 0, 0), 0.9).astype(np.float64)
    t = oracle.Tree(xn[:5000], 1e-12)
    out, pairs, _ = t.apply_at(OP_A, mu[:5000], q, 0.0)
    d, _ = oracle.direct(OP_A, xn[:5000], mu[:5000], 0.0, y=q)
    assert pairs[0] == 0 and pairs[1] == 500 * 5000
    assert np.abs(out - d).max() <= 1e-12 * np.abs(d).max()


# ---------------------------------------------------------------------------
# Iteration (Alg. 2, Alg. 3)
# ---------------------------------------------------------------------------

def test_schedule_endpoints():
    assert oracle.schedule_width(1, 40, 0.002, 0.016) == 0.016
    assert abs(oracle.schedule_width(40, 40, 0.002, 0.016) - 0.002) < 1e-18
    assert oracle.schedule_width(1, 1, 0.002, 0.016) == 0.002
    ws = [oracle.schedule_width(i, 40, 0.002, 0.016) for i in range(1, 41)]
    assert np.allclose(np.diff(ws), -(0.016 - 0.002) / 39)


@pytest.mark.parametrize("schedule", ["linear", "cosine", "exponential"])
def test_schedule_alternatives(schedule):
    """Sec. 6.1.2's cosine and exponential decays (and the linear one of
    Alg. 3) start at w2, end at w1 and fall monotonically; each has its own
    shape: constant steps (linear), flat ends and point symmetry about the
    middle (cosine), a constant ratio with the geometric mean in the middle
    (exponential)."""
    n, w1, w2 = 41, 0.002, 0.016
    ws = np.array([oracle.schedule_width(i, n, w1, w2, schedule) for i in range(1, n + 1)])
    assert ws[0] == w2
    assert abs(ws[-1] - w1) < 1e-15
    d = np.diff(ws)
    assert np.all(d < 0)
    mid = ws[(n - 1) // 2]
    if schedule == "linear":
        assert np.allclose(d, -(w2 - w1) / (n - 1), rtol=1e-9)
        assert abs(mid - 0.5 * (w1 + w2)) < 1e-15
    elif schedule == "cosine":
        assert np.allclose(ws + ws[::-1], w1 + w2, rtol=0, atol=1e-15)
        assert abs(mid - 0.5 * (w1 + w2)) < 1e-15
        # flat at both ends, steepest in the middle: the first step is
        # (w2 - w1) sin^2(pi / (2 (n - 1))) of the whole drop
        assert abs(-d[0] - (w2 - w1) * np.sin(np.pi / (2 * (n - 1))) ** 2) < 1e-15
        assert -d[0] < -d[(n - 1) // 2 - 1]
    else:
        ratios = ws[1:] / ws[:-1]
        assert np.allclose(ratios, (w1 / w2) ** (1.0 / (n - 1)), rtol=1e-12)
        assert abs(mid - np.sqrt(w1 * w2)) < 1e-15
    assert oracle.schedule_width(1, 1, w1, w2, schedule) == w1
    it_stats = oracle.iterate(synth.fibonacci_sphere(200).points, n_iter=n, last_iter=3,
                              schedule=schedule)[1]
    assert np.array_equal(it_stats[:, 0], ws[:3])


def test_exponential_schedule_needs_positive_widths():
    with pytest.raises(ValueError):
        oracle.schedule_width(2, 10, 0.0, 0.016, "exponential")
    with pytest.raises(ValueError):
        oracle.schedule_width(2, 10, 0.002, 0.016, "quadratic")


def test_first_iteration_closed_form_on_sphere():
    """From mu = 0 on a sphere of radius R (normalised units), r = A^T b is
    radial and the exact line search gives mu = (4 pi R^2/N) n / (1 - w/(2R))
    in the continuum limit; the WNNC update keeps it radial and the rescale
    keeps its length."""
    N = 20000
    x, n = _sphere(N)
    w = 0.15
    mu, st = oracle.iterate(x.astype(np.float32), n_iter=1, w1=w, w2=w, theta=0.3)
    xn, _, s = oracle.normalize(x.astype(np.float32))
    R = np.linalg.norm(xn, axis=1).mean()          # normalised radius (10/11)
    pred = 4 * math.pi * (R / s) ** 2 / N / (1 - w / (2 * R))
    lens = np.linalg.norm(mu, axis=1)
    assert abs(lens.mean() / pred - 1) < 1e-2
    assert oracle.p_co(n, mu) == 1.0
    assert st[0, 1] == pytest.approx(N * 0.25)     # E at mu = 0 is |b|^2


def test_grad_steps_decrease_energy_and_alpha_is_line_minimum():
    """Steepest descent with the exact step of Alg. 2 never increases E, and
    the step length minimises E along r."""
    c = synth.config_cloud("union50k", n=3000)
    mu, st = oracle.iterate(c.points, n_iter=6, w1=0.02, w2=0.02, use_wnnc=False)
    E = st[:, 1]
    assert np.all(np.diff(E) < 0)
    # line minimum: E(mu_k + t r) for t = alpha (1 +- 0.2) is larger than at alpha
    xn, _, s = oracle.normalize(c.points)
    mu0, _ = oracle.iterate(c.points, n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, last_iter=3)
    mu1, _ = oracle.iterate(c.points, mu0=mu0, n_iter=6, w1=0.02, w2=0.02, use_wnnc=False,
                            first_iter=4, last_iter=4)
    step = (mu1 - mu0) * s * s

    def energy(m):
        a, _ = oracle.direct(OP_A, xn, m, 0.02)
        return ((a - 0.5) ** 2).sum()
    e0 = energy(mu1 * s * s)
    for f in (0.8, 1.2):
        assert energy(mu0 * s * s + f * step) > e0


def test_zero_init_without_grad_step_stays_zero():
    """Sec. 6.1.3: without the gradient step, mu stays at 0."""
    c = synth.config_cloud("union50k", n=2000)
    mu, _ = oracle.iterate(c.points, n_iter=5, use_grad=False)
    assert np.all(mu == 0.0)


def test_sphere_orientation_converges():
    """Dense sphere, default widths: all normals outward, small angular error,
    total |mu| close to the area (Sec. 6.1.2 reports it within a few %)."""
    c = synth.sphere(20000, 1000)
    mu, _ = oracle.iterate(c.points, n_iter=40, theta=0.3)
    assert oracle.p_co(c.normals, mu) == 1.0
    assert oracle.ae_pcd(c.normals, mu) < 0.03
    assert abs(np.linalg.norm(mu, axis=1).sum() / (4 * math.pi) - 1) < 0.05


# ---------------------------------------------------------------------------
# kNN
# ---------------------------------------------------------------------------

def test_knn_matches_sorted_distances():
    c = synth.union_cloud(600, 3)
    x = c.points.astype(np.float64)
    idx, d2 = oracle.knn(x, 16)
    D = ((x[:, None] - x[None]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    ref = np.sort(D, axis=1)[:, :16]
    assert np.allclose(d2, ref, rtol=0, atol=0)
    assert np.allclose(D[np.arange(len(x))[:, None], idx], ref)
