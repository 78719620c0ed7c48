"""Local expansions of the far field (tree parameter local_theta > 0) on the
GPU, against the oracle's independent implementation (oracle.Tree with
local_theta; pinned in tests/test_oracle_local.py).

A far node whose box gap to a target group exceeds the group box's largest
extent / local_theta is not summed per target: its terms of A and G are
expanded to first order about the group box centre (Sec. 4.5 and Sec. 6.3
name the expansions of an FMM as the way to precision control; this is their
target-side counterpart), and A^T is the exact transpose.  An entry whose
pairs may straddle the cut-off is summed pair by pair on that call.

  - the partition of every group's far list into pair-by-pair and expanded
    entries equals the one computed here from the oracle's lists and boxes
    with the same double-precision test (integer work: exact);
  - A, grad F and A^T element by element within the parity bound of
    tests/test_gpu_parity.py (the oracle's ambiguity budget covers entries
    whose cut-off decision lies within 1e-5 of its threshold);
  - the fallback path: a width at which thousands of expanded entries must
    be summed pair by pair;
  - off-surface queries, <A mu, s> = <mu, A^T s>, and the 40-iteration solve.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import OP_A, OP_AT, OP_G
from test_gpu_parity import AMB, check_close, f32
from test_iterate import _compare_fields

pytestmark = pytest.mark.gpu


def _wnnc():
    import paper_2405_16634_b300 as W
    return W


@pytest.fixture(scope="module")
def union5k():
    c = synth.union_cloud(5003, 77, n_tori=1, n_ellipsoids=2, noise=0.002)
    mu = (synth.random_unit_vectors(len(c.points), 6) * (c.area / len(c.points))).astype(np.float32)
    s = np.random.default_rng(5).standard_normal(len(c.points)).astype(np.float32)
    return c, mu, s


def _oracle_partition(points, theta, local_theta):
    """Per group: (far nodes summed pair by pair, expanded far nodes), each
    ascending, from the oracle's lists and boxes: a far node is expanded iff
    its squared box gap exceeds (extent / local_theta)^2, evaluated in double
    precision in the order the oracle writes it."""
    xn, _, _ = oracle.normalize(points)
    t = oracle.Tree(xn, theta)
    goff = t.groups()
    fo, fi, _, _ = t.lists()
    nd = t.nodes()
    y = xn[t.perm()]
    cl = 1.0 / local_theta
    out = []
    for g in range(len(goff) - 1):
        yy = y[goff[g]:goff[g + 1]]
        glo, ghi = yy.min(0), yy.max(0)
        e = ghi[0] - glo[0]
        if ghi[1] - glo[1] > e:
            e = ghi[1] - glo[1]
        if ghi[2] - glo[2] > e:
            e = ghi[2] - glo[2]
        b = fi[fo[g]:fo[g + 1]]
        a = nd["lo"][b] - ghi
        d = glo - nd["hi"][b]
        gq = np.maximum(np.maximum(a, d), 0.0)
        gap2 = (gq[:, 0] * gq[:, 0] + gq[:, 1] * gq[:, 1]) + gq[:, 2] * gq[:, 2]
        ce = cl * e
        loc = gap2 > ce * ce
        out.append((np.sort(b[~loc]), np.sort(b[loc])))
    return out


@pytest.mark.parametrize("theta,local_theta", [(0.5, 0.5), (0.5, 1.0), (0.8, 0.5)])
def test_local_partition_matches_oracle(theta, local_theta):
    W = _wnnc()
    c = synth.config_cloud("union50k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=theta, local_theta=local_theta)
    ex = t.export()
    ref = _oracle_partition(c.points, f32(theta), f32(local_theta))
    fo, fid, ls = ex["far_off"], ex["far_id"], ex["far_lsplit"]
    assert len(ref) == len(ls)
    n_local = 0
    for g, (pairs, local) in enumerate(ref):
        assert np.array_equal(fid[fo[g]:ls[g]], pairs), g
        assert np.array_equal(fid[ls[g]:fo[g + 1]], local), g
        n_local += len(local)
    entries, lpairs = t.local_stats()
    assert entries == n_local > 0
    gsize = np.diff(ex["group_off"])
    assert lpairs == int((gsize * (fo[1:] - ls)).sum())


@pytest.mark.parametrize("local_theta", [0.5, 1.0])
def test_local_operators_match_oracle(union5k, local_theta):
    W = _wnnc()
    c, mu, s = union5k
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=local_theta)
    assert t.local_stats()[0] > 0
    for w in (0.002, 0.004, 0.016):
        F = t.eval_w(torch.from_numpy(mu).cuda(), w).cpu().numpy()
        Fo, amb = oracle.eval_op(OP_A, c.points, mu, w, theta=0.5, amb_tol=AMB, local_theta=f32(local_theta))
        check_close(F, Fo, amb, what=f"A local_theta={local_theta} w={w}")
        G = t.eval_grad(torch.from_numpy(mu).cuda(), w).cpu().numpy()
        Go, amb = oracle.eval_op(OP_G, c.points, mu, w, theta=0.5, amb_tol=AMB, local_theta=f32(local_theta))
        check_close(G, Go, amb, what=f"grad local_theta={local_theta} w={w}")
        T = t.eval_adjoint(torch.from_numpy(s).cuda(), w).cpu().numpy()
        To, amb = oracle.eval_op(OP_AT, c.points, s, w, theta=0.5, amb_tol=AMB, local_theta=f32(local_theta))
        check_close(T, To, amb, what=f"AT local_theta={local_theta} w={w}")
        # the expanded operator and its transpose, on the GPU
        lhs, rhs = (F.astype(np.float64) * s).sum(), (mu.astype(np.float64) * T).sum()
        assert abs(lhs - rhs) <= 1e-5 * np.abs(F.astype(np.float64) * s).sum()


def _fallback_entries(points, theta, local_theta, w):
    """Expanded entries whose bound |c_g - x_B| - rho_g lies below w (the
    oracle's group frames and centroids)."""
    xn, _, _ = oracle.normalize(points)
    t = oracle.Tree(xn, theta)
    goff = t.groups()
    nd = t.nodes()
    y = xn[t.perm()]
    count = 0
    for g, (_, local) in enumerate(_oracle_partition(points, theta, local_theta)):
        yy = y[goff[g]:goff[g + 1]]
        cg = 0.5 * (yy.min(0) + yy.max(0))
        rho = np.linalg.norm(yy - cg, axis=1).max()
        count += int((np.linalg.norm(nd["cent"][local] - cg, axis=1) - rho < w).sum())
    return count


def test_local_fallback_matches_oracle(union5k):
    """w = 0.3 (normalised units) reaches about 2,000 of the 51,519 expanded
    entries: those are summed pair by pair with the cut-off, in the gather
    (queued per warp) and in the adjoint's node gather."""
    W = _wnnc()
    c, mu, s = union5k
    w = 0.3
    nfall = _fallback_entries(c.points, 0.5, 0.5, w)
    assert nfall > 1000, nfall
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5)
    F = t.eval_w(torch.from_numpy(mu).cuda(), w).cpu().numpy()
    Fo, amb = oracle.eval_op(OP_A, c.points, mu, w, theta=0.5, amb_tol=AMB, local_theta=0.5)
    check_close(F, Fo, amb, what=f"A fallback ({nfall} entries)")
    G = t.eval_grad(torch.from_numpy(mu).cuda(), w).cpu().numpy()
    Go, amb = oracle.eval_op(OP_G, c.points, mu, w, theta=0.5, amb_tol=AMB, local_theta=0.5)
    check_close(G, Go, amb, what="grad fallback")
    T = t.eval_adjoint(torch.from_numpy(s).cuda(), w).cpu().numpy()
    To, amb = oracle.eval_op(OP_AT, c.points, s, w, theta=0.5, amb_tol=AMB, local_theta=0.5)
    check_close(T, To, amb, what="AT fallback")


def test_local_queries_match_oracle(union5k):
    """Off-surface query points (their own groups and lists, expanded alike)."""
    W = _wnnc()
    c, mu, _ = union5k
    rng = np.random.default_rng(9)
    lo, hi = c.points.min(0), c.points.max(0)
    q = (lo + (hi - lo) * (1.3 * rng.random((4000, 3)) - 0.15)).astype(np.float32)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5)
    for grad in (False, True):
        got = t.eval_at(torch.from_numpy(mu).cuda(), torch.from_numpy(q).cuda(), 0.0, grad=grad).cpu().numpy()
        ref, b = oracle.eval_at(OP_G if grad else OP_A, c.points, mu, q, 0.0, theta=0.5, with_bounds=True,
                                local_theta=0.5)
        check_close(got, ref, b, what=f"queries local grad={grad}")


def test_local_iteration_matches_oracle():
    """40 iterations on 20,000 union points with local expansions, GPU
    against the oracle's FP64 solve with the same expansions."""
    W = _wnnc()
    c = synth.config_cloud("union50k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5)
    mg = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, n_iter=40, theta=0.5, local_theta=0.5)
    cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.995)
    pg, po = oracle.p_co(c.normals, mg), oracle.p_co(c.normals, mo)
    print(f"[local-iterate-20k] sign agreement {np.mean(cos > 0):.5f}, median cos {np.median(cos):.6f}, "
          f"median |len| diff {dlen:.2e}, P_co gpu {pg:.5f} oracle {po:.5f}")
    assert abs(pg - po) < 0.005


def test_local_solve_at_500k_agrees_with_the_pairwise_far_field():
    """The benchmark's 500k solve (tree build + 40 iterations) with the
    expansions (one level, and two with clusters of 4 groups) and without:
    the oriented fields agree point by point."""
    W = _wnnc()
    c = synth.config_cloud("union500k")
    pts = torch.from_numpy(c.points).cuda()
    fields = []
    for lt, k in ((0.0, 0), (0.5, 0), (0.5, 4)):
        t = W.Tree(pts, theta=0.5, local_theta=lt, local_cluster=k)
        fields.append(t.iterate(n_iter=40).cpu().numpy().astype(np.float64))
        t.close()
    valid = np.all(np.isfinite(c.normals), axis=1)
    p0 = oracle.p_co(c.normals[valid], fields[0][valid])
    for name, f in (("one level", fields[1]), ("clusters of 4", fields[2])):
        cos, dlen = _compare_fields(f, fields[0], min_sign=0.9999, min_cos=0.99999)
        p1 = oracle.p_co(c.normals[valid], f[valid])
        print(f"[local-500k] {name}: sign agreement {np.mean(cos > 0):.6f}, median cos {np.median(cos):.7f}, "
              f"median |len| diff {dlen:.2e}, P_co pairwise {p0:.5f} expanded {p1:.5f}")
        assert abs(p1 - p0) < 1e-3


# ---------------------------------------------------------------------------
# The second level: clusters of K consecutive groups (local_cluster = K).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("theta,k", [(0.5, 4), (0.5, 2), (0.8, 8)])
def test_cluster_partition_matches_oracle(theta, k):
    """Every group's far list in three parts, pair by pair / expanded about
    the group / about its cluster, equal as sets (each part ascending on the
    GPU) to the oracle's classes; the counts of both levels follow."""
    W = _wnnc()
    c = synth.config_cloud("union50k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=theta, local_theta=0.5, local_cluster=k)
    ex = t.export()
    xn, _, _ = oracle.normalize(c.points)
    ot = oracle.Tree(xn, f32(theta), local_theta=0.5, local_cluster=k)
    fo_o, fi_o, _, _ = ot.lists()
    cls = ot.local_classes()
    fo, fid, ls, cs = ex["far_off"], ex["far_id"], ex["far_lsplit"], ex["far_csplit"]
    gsize = np.diff(ex["group_off"])
    n_cl = n_cl_pairs = 0
    for g in range(len(ls)):
        ids, cl = fi_o[fo_o[g]:fo_o[g + 1]], cls[fo_o[g]:fo_o[g + 1]]
        for part, (a, b) in enumerate(((fo[g], ls[g]), (ls[g], cs[g]), (cs[g], fo[g + 1]))):
            assert np.array_equal(fid[a:b], np.sort(ids[cl == part])), (g, part)
        if g % k == 0:
            n_cl += fo[g + 1] - cs[g]
            n_cl_pairs += (fo[g + 1] - cs[g]) * int(gsize[g:g + k].sum())
    assert (cls == 2).sum() > 0
    assert t.cluster_stats() == (n_cl, n_cl_pairs)
    assert t.local_stats()[0] == int((cls == 1).sum())


@pytest.mark.parametrize("k", [4, 2])
def test_cluster_operators_match_oracle(union5k, k):
    """A, grad F and A^T with both levels, element by element, at three
    widths, the last (w = 0.3) reaching about 2,000 expanded entries of either
    level: their pairs are summed instead."""
    W = _wnnc()
    c, mu, s = union5k
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5, local_cluster=k)
    assert t.cluster_stats()[0] > 0
    for w in (0.002, 0.016, 0.3):
        kw = dict(theta=0.5, amb_tol=AMB, local_theta=0.5, local_cluster=k)
        F = t.eval_w(torch.from_numpy(mu).cuda(), w).cpu().numpy()
        Fo, amb = oracle.eval_op(OP_A, c.points, mu, w, **kw)
        check_close(F, Fo, amb, what=f"A cluster {k} w={w}")
        G = t.eval_grad(torch.from_numpy(mu).cuda(), w).cpu().numpy()
        Go, amb = oracle.eval_op(OP_G, c.points, mu, w, **kw)
        check_close(G, Go, amb, what=f"grad cluster {k} w={w}")
        T = t.eval_adjoint(torch.from_numpy(s).cuda(), w).cpu().numpy()
        To, amb = oracle.eval_op(OP_AT, c.points, s, w, **kw)
        check_close(T, To, amb, what=f"AT cluster {k} w={w}")
        lhs, rhs = (F.astype(np.float64) * s).sum(), (mu.astype(np.float64) * T).sum()
        assert abs(lhs - rhs) <= 1e-5 * np.abs(F.astype(np.float64) * s).sum()


def test_cluster_queries_match_oracle(union5k):
    W = _wnnc()
    c, mu, _ = union5k
    rng = np.random.default_rng(9)
    lo, hi = c.points.min(0), c.points.max(0)
    q = (lo + (hi - lo) * (1.3 * rng.random((4000, 3)) - 0.15)).astype(np.float32)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5, local_cluster=4)
    for grad in (False, True):
        got = t.eval_at(torch.from_numpy(mu).cuda(), torch.from_numpy(q).cuda(), 0.0, grad=grad).cpu().numpy()
        ref, b = oracle.eval_at(OP_G if grad else OP_A, c.points, mu, q, 0.0, theta=0.5, with_bounds=True,
                                local_theta=0.5, local_cluster=4)
        check_close(got, ref, b, what=f"queries cluster grad={grad}")


def test_cluster_iteration_matches_oracle():
    W = _wnnc()
    c = synth.config_cloud("union50k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5, local_cluster=4)
    mg = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, n_iter=40, theta=0.5, local_theta=0.5, local_cluster=4)
    cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.995)
    pg, po = oracle.p_co(c.normals, mg), oracle.p_co(c.normals, mo)
    print(f"[cluster-iterate-20k] sign agreement {np.mean(cos > 0):.5f}, median cos {np.median(cos):.6f}, "
          f"median |len| diff {dlen:.2e}, P_co gpu {pg:.5f} oracle {po:.5f}")
    assert abs(pg - po) < 0.005


def test_autograd_with_both_levels(union5k):
    """The expanded forward is linear in mu and A^T is its exact transpose, so
    the autograd backward equals central differences of the forward: with
    s = dL/dF, dL/dmu_k = <A e_k, s> = (A^T s)_k."""
    W = _wnnc()
    c, mu, s = union5k
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, local_theta=0.5, local_cluster=4)
    w = 0.004
    m = torch.from_numpy(mu).cuda().requires_grad_()
    sv = torch.from_numpy(s).cuda()
    F = W.winding_number(t, m, w)
    (F * sv).sum().backward()
    g = m.grad.double().cpu().numpy()
    assert np.array_equal(g, t.eval_adjoint(sv, w).double().cpu().numpy())
    rng = np.random.default_rng(3)
    idx = rng.choice(mu.size, 32, replace=False)
    h = 1e-3                                   # F is linear: the step costs no truncation
    fd = []
    for k in idx:
        i, j = divmod(int(k), 3)
        mp, mm = mu.copy(), mu.copy()
        mp[i, j] += h
        mm[i, j] -= h
        fp = t.eval_w(torch.from_numpy(mp).cuda(), w).double().cpu().numpy()
        fm = t.eval_w(torch.from_numpy(mm).cuda(), w).double().cpu().numpy()
        fd.append(((fp - fm) * s).sum() / (2 * h))
    ag = g.reshape(-1)[idx]
    assert np.abs(np.array(fd) - ag).max() <= 1e-3 * np.abs(ag).max()
