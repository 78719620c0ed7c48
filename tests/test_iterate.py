"""The Alg. 3 iteration: the oracle against the paper's sphere table, and the
CUDA iteration against the oracle's iteration."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sphere_area_table.txt")


def f32(x):
    return float(np.float32(x))


def _paper_table():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip() or line.startswith("stat"):
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals


def _area_stats(mu):
    a = np.linalg.norm(mu, axis=1)
    return dict(min=a.min(), max=a.max(), mean=a.mean(), total=a.sum())


@pytest.mark.slow
def test_oracle_reproduces_paper_sphere_area_table():
    """Oracle, icosphere-7 (163,842 points), 40 iterations, theta = 0.5."""
    c = synth.icosphere(7)
    mu, _ = oracle.iterate(c.points, n_iter=40, theta=0.5)
    got, ref = _area_stats(mu), _paper_table()
    for k in ("min", "max", "mean", "total"):
        assert abs(got[k] / ref[k] - 1) < 0.03, (k, got[k], ref[k])
    assert oracle.p_co(c.normals, mu) == 1.0


def _rounds_to_printed(got, printed):
    """|got - printed| <= half a unit in the last digit the paper prints
    (4 significant digits for these values): got rounds to the printed value."""
    digits = 4
    e = np.floor(np.log10(abs(printed))) - (digits - 1)
    return abs(got - printed) <= 0.5 * 10.0 ** e * (1 + 1e-9)


@pytest.mark.slow
def test_oracle_papers_treecode_reproduces_the_sphere_table_to_the_printed_digit():
    """The oracle's Alg. 3 on the paper's own treecode run as printed (Alg. 4
    per target, leaf size 1, c = 2, the |mu|-weighted representatives of
    Eq. 13) on the 163,842-point icosphere, 40 iterations from zero: the mean
    and the total of |mu| round to the values the paper's table prints
    (7.858e-5 and 12.875, Sec. 6.1.2).  The exact direct sums give a total
    2.2 % lower: the printed total carries the treecode's own approximation,
    and this oracle reproduces it.  (The table's min and max are matched to
    3 % only: 7.6255e-5 and 8.1368e-5 against 7.465e-5 and 8.330e-5.)"""
    c = synth.icosphere(7)
    mu, _ = oracle.iterate(c.points, n_iter=40, paper_theta=0.5, paper_leaf_size=1)
    got, ref = _area_stats(mu), _paper_table()
    assert _rounds_to_printed(got["mean"], ref["mean"]), (got["mean"], ref["mean"])
    assert _rounds_to_printed(got["total"], ref["total"]), (got["total"], ref["total"])
    for k in ("min", "max"):
        assert abs(got[k] / ref[k] - 1) < 0.03, (k, got[k], ref[k])
    assert oracle.p_co(c.normals, mu) == 1.0


def _gpu():
    import paper_2405_16634_b300 as W
    return W


@pytest.mark.gpu
def test_gpu_reproduces_paper_sphere_area_table():
    W = _gpu()
    c = synth.icosphere(7)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mu = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    got, ref = _area_stats(mu), _paper_table()
    for k in ("min", "max", "mean", "total"):
        assert abs(got[k] / ref[k] - 1) < 0.03, (k, got[k], ref[k])
    assert oracle.p_co(c.normals, mu) == 1.0


def _compare_fields(mu_g, mu_o, min_sign=0.995, min_cos=0.99):
    ug, uo = oracle.unit(mu_g), oracle.unit(mu_o)
    cos = (ug * uo).sum(1)
    assert np.mean(cos > 0) >= min_sign, np.mean(cos > 0)
    assert np.median(cos) >= min_cos, np.median(cos)
    lg, lo = np.linalg.norm(mu_g, axis=1), np.linalg.norm(mu_o, axis=1)
    return cos, np.median(np.abs(lg / np.maximum(lo, 1e-30) - 1))


@pytest.mark.gpu
def test_gpu_paper_exact_mode_reproduces_the_sphere_table():
    """The paper's treecode as printed on the GPU (criterion 1, leaf size 1,
    rep_mode 0), icosphere-7, 40 iterations: the mean and total of |mu| round
    to the table's printed values (as the oracle's run of the same algorithm
    does), and min, max, mean and total equal the oracle's to 1e-4."""
    W = _gpu()
    c = synth.icosphere(7)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, leaf_size=1, rep_mode=0, criterion=1)
    mu = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    got, ref = _area_stats(mu), _paper_table()
    print(f"[table] paper-exact GPU: min {got['min']:.5g} max {got['max']:.5g} mean {got['mean']:.5g} "
          f"total {got['total']:.6g} (paper: {ref['min']}, {ref['max']}, {ref['mean']}, {ref['total']})")
    assert _rounds_to_printed(got["mean"], ref["mean"]), (got["mean"], ref["mean"])
    assert _rounds_to_printed(got["total"], ref["total"]), (got["total"], ref["total"])
    mo, _ = oracle.iterate(c.points, n_iter=40, paper_theta=0.5, paper_leaf_size=1)
    go = _area_stats(mo)
    for k in ("min", "max", "mean", "total"):
        assert abs(got[k] / go[k] - 1) < 1e-4, (k, got[k], go[k])
    assert oracle.p_co(c.normals, mu) == 1.0
    t.sync_status()


@pytest.mark.gpu
@pytest.mark.parametrize("init", ["zero", "random"])
def test_gpu_iteration_sphere2k_matches_oracle(init):
    """First configuration: 2,000 sphere points, direct sums, 40 iterations."""
    W = _gpu()
    c = synth.config_cloud("sphere2k")
    n = len(c.points)
    mu0 = None if init == "zero" else synth.init_normals(n, 1001, 4 * math.pi / n)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.0)
    mg, st = t.iterate(None if mu0 is None else torch.from_numpy(mu0).cuda(), n_iter=40, stats=True)
    mg = mg.cpu().numpy().astype(np.float64)
    st = st.cpu().numpy()
    mo, so = oracle.iterate(c.points, mu0=mu0, n_iter=40)
    cos, dlen = _compare_fields(mg, mo, min_sign=1.0, min_cos=0.9999)
    assert dlen < 1e-3
    assert np.allclose(st[:, 0], so[:, 0], rtol=1e-6)
    assert np.allclose(st[:5, 1], so[:5, 1], rtol=1e-3)
    assert np.allclose(st[:5, 2], so[:5, 2], rtol=1e-3)
    if init == "zero":
        assert oracle.p_co(c.normals, mg) == 1.0


@pytest.mark.gpu
def test_orient_from_host_memory_equals_the_device_path():
    """wnnc_orient (host points in, host field out, one call) gives the field
    of the device entry points bit for bit, from zero and from a given init."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=20000)
    n = len(c.points)
    ref = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5).iterate(n_iter=10).cpu()
    h_pts = torch.from_numpy(c.points).pin_memory()
    got = W.orient(h_pts, n_iter=10, out=torch.empty(n, 3).pin_memory())
    assert torch.equal(got, ref)
    mu0 = synth.init_normals(n, 3, c.area / n)
    ref = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5).iterate(torch.from_numpy(mu0).cuda(), n_iter=10).cpu()
    got = W.orient(c.points, mu0=mu0, n_iter=10)          # pageable host memory works too
    assert torch.equal(got, ref)
    with pytest.raises(W.WnncError):
        bad = c.points.copy()
        bad[7, 1] = np.nan
        W.orient(bad, n_iter=2)


@pytest.mark.gpu
def test_gpu_first_iteration_closed_form():
    W = _gpu()
    c = synth.fibonacci_sphere(40000)
    n = len(c.points)
    w = 0.1
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.3)
    mu = t.iterate(n_iter=1, w1=w, w2=w).cpu().numpy().astype(np.float64)
    xn, _, s = oracle.normalize(c.points)
    R = np.linalg.norm(xn, axis=1).mean()
    pred = 4 * math.pi * (R / s) ** 2 / n / (1 - w / (2 * R))
    assert abs(np.linalg.norm(mu, axis=1).mean() / pred - 1) < 1e-2
    assert oracle.p_co(c.normals, mu) == 1.0


@pytest.mark.gpu
@pytest.mark.parametrize("theta,init", [(0.5, "zero"), (0.3, "random"), (0.5, "random"), (0.8, "random")])
def test_gpu_iteration_union50k_matches_oracle(theta, init):
    """Second configuration: 50,000 union points, 40 iterations at
    theta = 0.3, 0.5, 0.8, from the configuration's random unit normals (times
    the mean area) and from zero (the paper's init).  The GPU solve agrees
    with the oracle's FP64 solve on the same lists, and so does its accuracy
    against ground truth.  (Sec. 6.1.3: from a random init the method need
    not find the ground-truth orientation; the agreement is what is tested.)"""
    W = _gpu()
    c = synth.config_cloud("union50k")
    n = len(c.points)
    mu0 = None if init == "zero" else synth.init_normals(n, 2001, c.area / n)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=theta)
    mg = t.iterate(None if mu0 is None else torch.from_numpy(mu0).cuda(), n_iter=40)
    mg = mg.cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, mu0=mu0, n_iter=40, theta=f32(theta))
    cos, _ = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.995)
    pg, po = oracle.p_co(c.normals, mg), oracle.p_co(c.normals, mo)
    print(f"[iterate-50k] theta={theta} init={init}: sign agreement {np.mean(cos > 0):.5f}, "
          f"median cos {np.median(cos):.6f}, P_co gpu {pg:.5f} oracle {po:.5f}")
    # orientation accuracy against ground truth equals the oracle's
    assert abs(pg - po) < 0.005
    assert abs(oracle.ae_pcd(c.normals, mg) - oracle.ae_pcd(c.normals, mo)) < 0.005


@pytest.mark.gpu
def test_gpu_iteration_union500k_matches_oracle_at_full_size():
    """The benchmark's workload at full size (500,000 points, theta = 0.5, the
    fused iteration that bench.py times): iterations 1 and 2 of the 40-step
    schedule from zero against the oracle's FP64 iteration on the same lists.
    The step-length sums (E, |r|^2) and alpha agree to FP32 rounding, and the
    fields agree point by point."""
    W = _gpu()
    c = synth.config_cloud("union500k")
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg, sg = t.iterate(n_iter=40, last_iter=2, stats=True)
    mg = mg.cpu().numpy().astype(np.float64)
    sg = sg.cpu().numpy().astype(np.float64)
    mo, so = oracle.iterate(c.points, n_iter=40, last_iter=2, theta=f32(0.5))
    assert np.allclose(sg[:, 0], so[:, 0], rtol=1e-6)                 # widths
    assert np.allclose(sg[:, 1:], so[:, 1:], rtol=2e-4), (sg, so)      # E, alpha, |r|^2
    cos, dlen = _compare_fields(mg, mo, min_sign=0.9999, min_cos=0.99999)
    assert dlen < 1e-4, dlen


@pytest.mark.gpu
def test_gpu_full_solve_union500k_matches_oracle():
    """The benchmark solve end to end: all 40 iterations on the 500,000-point
    cloud (theta = 0.5, zero init) on the GPU against the oracle's FP64
    iteration over the same interaction lists.  Normal signs agree at
    >= 99.5 % of the points and the median cosine is >= 0.999; the orientation
    accuracy against ground truth (surface points) agrees to 0.1 %."""
    W = _gpu()
    c = synth.config_cloud("union500k")
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, n_iter=40, theta=f32(0.5))
    cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.999)
    ok = np.isfinite(c.normals).all(1)
    pg, po = oracle.p_co(c.normals[ok], mg[ok]), oracle.p_co(c.normals[ok], mo[ok])
    print(f"[iterate-500k] sign agreement {np.mean(cos > 0):.6f}, median cos {np.median(cos):.7f}, "
          f"median |len ratio - 1| {dlen:.2e}, P_co gpu {pg:.6f} oracle {po:.6f}")
    assert abs(pg - po) < 1e-3


@pytest.mark.gpu
def test_gpu_treecode_solve_matches_direct_sum_iteration():
    """Alg. 3 on the plain definitions: the GPU solve at the production
    theta = 0.5 (and theta = 0.3) against the oracle's iteration on the FP64
    direct sums (no treecode) on a 20,000-point union, 40 iterations.

    The widths follow the point spacing, as the paper sets them per data set:
    at 20,000 points this cloud is about 3x sparser than at 50,000, and the
    paper's preset for sparser, noisier scans (w1 = 0.01, w2 = 0.04,
    Sec. 5.2.6) lets the exact method converge (P_co 0.992).  There the
    treecode's ~1e-2 operator error changes no sign: agreement >= 99.5 %
    (measured 100 %).  With the default widths (w1 = 0.002 < spacing) the exact
    method itself orients only ~93 % of the points correctly and the treecode
    solve flips ~0.6 % of signs among those it cannot orient; there its
    accuracy against ground truth must equal the exact method's."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=20000)
    mo, _ = oracle.iterate(c.points, n_iter=40, w1=0.01, w2=0.04)
    for theta, min_cos in ((0.5, 0.999), (0.3, 0.999)):
        t = W.Tree(torch.from_numpy(c.points).cuda(), theta=theta)
        mg = t.iterate(n_iter=40, w1=0.01, w2=0.04).cpu().numpy().astype(np.float64)
        cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=min_cos)
        print(f"[iterate-direct] theta={theta} w=0.04->0.01: sign agreement {np.mean(cos > 0):.5f}, "
              f"median cos {np.median(cos):.6f}, median |len ratio - 1| {dlen:.2e}, "
              f"P_co gpu {oracle.p_co(c.normals, mg):.5f} direct {oracle.p_co(c.normals, mo):.5f}")
    mo, _ = oracle.iterate(c.points, n_iter=40)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg = t.iterate(n_iter=40).cpu().numpy().astype(np.float64)
    cos = (oracle.unit(mg) * oracle.unit(mo)).sum(1)
    pg, po = oracle.p_co(c.normals, mg), oracle.p_co(c.normals, mo)
    print(f"[iterate-direct] theta=0.5 w=0.016->0.002: sign agreement {np.mean(cos > 0):.5f}, "
          f"P_co gpu {pg:.5f} direct {po:.5f}")
    assert pg >= po - 0.005


@pytest.mark.gpu
def test_gpu_solve_matches_the_papers_treecode_iteration():
    """The GPU solve (group lists, theta = 0.5, leaf size 8) against the
    oracle's Alg. 3 on the paper's own treecode run as printed (Alg. 4 per
    target, leaf size 1, |nu|-weighted representatives, theta = 0.5) on a
    20,000-point union, 40 iterations with the widths of the sparser-scan
    preset (w1 = 0.01, w2 = 0.04; see the direct-sum test above): the two
    treecodes differ in every far-field decision, yet the orientations agree
    (>= 99.5 % of signs; measured 100 %)."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=20000)
    mo, _ = oracle.iterate(c.points, n_iter=40, w1=0.01, w2=0.04, paper_theta=0.5, paper_leaf_size=1)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg = t.iterate(n_iter=40, w1=0.01, w2=0.04).cpu().numpy().astype(np.float64)
    cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.999)
    print(f"[iterate-paper-tree] sign agreement {np.mean(cos > 0):.5f}, median cos {np.median(cos):.6f}, "
          f"P_co gpu {oracle.p_co(c.normals, mg):.5f} paper treecode {oracle.p_co(c.normals, mo):.5f}")
    assert oracle.p_co(c.normals, mg) >= oracle.p_co(c.normals, mo) - 0.005


@pytest.mark.gpu
def test_gpu_ablations_match_oracle():
    """The ablations of Sec. 6.1.3 against the oracle's iteration with the
    same switch: gradient steps only (no WNNC update), from zero; WNNC updates
    only (no gradient step), from a random init (Sec. 6.1.3 and Fig. 12: the
    update alone keeps whatever orientation it is given)."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    n = len(c.points)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg, sg = t.iterate(n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, stats=True)
    mo, so = oracle.iterate(c.points, n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, theta=f32(0.5))
    assert np.allclose(sg.cpu().numpy()[:, 1:], so[:, 1:], rtol=1e-3)
    _compare_fields(mg.cpu().numpy().astype(np.float64), mo, min_sign=0.999, min_cos=0.9999)
    mu0 = synth.init_normals(n, 7, c.area / n)
    mg = t.iterate(torch.from_numpy(mu0).cuda(), n_iter=10, use_grad=False).cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, mu0=mu0, n_iter=10, use_grad=False, theta=f32(0.5))
    _compare_fields(mg, mo, min_sign=0.995, min_cos=0.995)
    assert np.allclose(np.linalg.norm(mg, axis=1), np.linalg.norm(mu0, axis=1), rtol=1e-4)


@pytest.mark.gpu
def test_gpu_paper_exact_iteration_matches_oracle():
    """The paper's method as printed on the GPU -- Alg. 3 with every operator
    on the per-target treecode of Alg. 4 (criterion 1, leaf size 1, the
    |nu|-weighted representatives and the s-representative A^T) -- against
    the oracle's Alg. 3 on its own implementation of that treecode, 40
    iterations on a 10,000-point union (sparser-scan widths w1 = 0.01,
    w2 = 0.04, at which the method converges on a cloud this sparse)."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, leaf_size=1, rep_mode=0, criterion=1)
    mg, sg = t.iterate(n_iter=40, w1=0.01, w2=0.04, stats=True)
    mg = mg.cpu().numpy().astype(np.float64)
    mo, so = oracle.iterate(c.points, n_iter=40, w1=0.01, w2=0.04, paper_theta=0.5, paper_leaf_size=1)
    assert np.allclose(sg[:3, 1:].cpu().numpy(), so[:3, 1:], rtol=1e-3)
    cos, dlen = _compare_fields(mg, mo, min_sign=0.995, min_cos=0.999)
    print(f"[iterate-paper-exact] sign agreement {np.mean(cos > 0):.5f}, median cos {np.median(cos):.7f}, "
          f"P_co gpu {oracle.p_co(c.normals, mg):.5f} oracle {oracle.p_co(c.normals, mo):.5f}")
    t.sync_status()


@pytest.mark.gpu
def test_gpu_first_order_far_field_iteration_matches_oracle():
    """The fused iteration with the first-order far field (far_order 1,
    theta = 0.8) on the 50,000-point union against the oracle's iteration on
    its first-order treecode, 40 iterations; and the first two iterations of
    the unfused path (the WNNC update switched off) against the oracle's."""
    W = _gpu()
    c = synth.config_cloud("union50k")
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.8, far_order=1)
    mg, sg = t.iterate(n_iter=40, stats=True)
    mo, so = oracle.iterate(c.points, n_iter=40, theta=f32(0.8), far_order=1)
    assert np.allclose(sg.cpu().numpy()[:3, 1:], so[:3, 1:], rtol=1e-3)
    cos, dlen = _compare_fields(mg.cpu().numpy().astype(np.float64), mo, min_sign=0.995, min_cos=0.995)
    print(f"[iterate-first-order] sign agreement {np.mean(cos > 0):.5f}, median cos {np.median(cos):.6f}")
    mg, sg = t.iterate(n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, stats=True)
    mo, so = oracle.iterate(c.points, n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, theta=f32(0.8), far_order=1)
    assert np.allclose(sg.cpu().numpy()[:, 1:], so[:, 1:], rtol=1e-3)
    t.sync_status()


@pytest.mark.gpu
def test_gpu_paper_mode_iteration_matches_oracle():
    """rep_mode 0 (the paper's |nu|-weighted representatives and the
    s-representative A^T) through the whole iteration."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5, rep_mode=0)
    mg = t.iterate(n_iter=10).cpu().numpy().astype(np.float64)
    mo, _ = oracle.iterate(c.points, n_iter=10, theta=0.5, rep_mode=0)
    _compare_fields(mg, mo, min_sign=0.995, min_cos=0.995)


@pytest.mark.gpu
@pytest.mark.parametrize("schedule", ["cosine", "exponential"])
def test_gpu_width_schedules_match_oracle(schedule):
    """The cosine and exponential width decays of Sec. 6.1.2: the CUDA
    iteration takes the oracle's widths and reaches the oracle's field."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mg, sg = t.iterate(n_iter=10, schedule=schedule, stats=True)
    mo, so = oracle.iterate(c.points, n_iter=10, theta=f32(0.5), schedule=schedule)
    assert np.allclose(sg[:, 0].cpu().numpy(), so[:, 0], rtol=1e-6)
    assert np.allclose(sg[:3, 1:].cpu().numpy(), so[:3, 1:], rtol=1e-3)
    _compare_fields(mg.cpu().numpy().astype(np.float64), mo, min_sign=0.995, min_cos=0.995)


@pytest.mark.gpu
def test_gpu_schedule_argument_errors():
    W = _gpu()
    c = synth.fibonacci_sphere(500)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    with pytest.raises(W.WnncError):
        t.iterate(n_iter=3, schedule=3)
    with pytest.raises(W.WnncError):
        t.iterate(n_iter=3, w1=0.0, schedule="exponential")
    assert torch.isfinite(t.iterate(n_iter=3, w1=0.0, schedule="cosine")).all()


@pytest.mark.gpu
def test_gpu_ablations_behave_as_in_the_paper():
    """Sec. 6.1.3: without the gradient step mu stays 0; the grad step alone
    (no WNNC update) decreases the energy monotonically at fixed width."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mu = t.iterate(n_iter=5, use_grad=False)
    assert torch.count_nonzero(mu).item() == 0
    _, st = t.iterate(n_iter=6, w1=0.02, w2=0.02, use_wnnc=False, stats=True)
    E = st[:, 1].cpu().numpy()
    assert np.all(np.diff(E) < 0)


@pytest.mark.gpu
def test_gpu_fixed_area_rescale():
    """Eq. 19: with rescale = 1 every |mu_i| equals the given area."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=10000)
    n = len(c.points)
    area = np.full(n, c.area / n, np.float32)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    mu = t.iterate(n_iter=5, area=torch.from_numpy(area).cuda(), rescale=1).cpu().numpy()
    assert np.allclose(np.linalg.norm(mu, axis=1), area, rtol=1e-5)


@pytest.mark.gpu
def test_gpu_resume_equals_full_run():
    """Checkpoint/resume: iterations 1..20 then 21..40 equal one 1..40 run."""
    W = _gpu()
    c = synth.config_cloud("union50k", n=20000)
    t = W.Tree(torch.from_numpy(c.points).cuda(), theta=0.5)
    full = t.iterate(n_iter=40)
    half = t.iterate(n_iter=40, last_iter=20)
    rest = t.iterate(half, n_iter=40, first_iter=21)
    cos = (oracle.unit(full.cpu().numpy()) * oracle.unit(rest.cpu().numpy())).sum(1)
    assert np.min(cos) > 0.999
