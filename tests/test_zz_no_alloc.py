"""The entry point that allocates nothing (wnnc_eval_w_direct_noalloc).

Some callers cannot call cudaMalloc: a host application that manages all
device memory through its own pool, a plugin sandbox, or a latency-critical
path where an allocation could synchronise the device.  For them the library
offers a direct-summation winding number whose scratch lives in a fixed array
inside the library.  This file is collected last so that a run that stops at
the first failure has already run every other test.
"""
import ctypes
from ctypes import c_float, c_int, c_int64, c_void_p

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL, SUM_TOL = 1e-4, 1e-5     # the bound used by the other parity tests


def _entry():
    import paper_2405_16634_b300 as W
    f = W.lib().wnnc_eval_w_direct_noalloc
    f.argtypes = [c_void_p, c_int64, c_void_p, c_void_p, c_int64, c_float, c_void_p, c_void_p]
    f.restype = c_int
    return W, f


def _call(f, pts, mu, q, w):
    out = torch.empty(q.shape[0], device="cuda", dtype=torch.float32)
    st = f(pts.data_ptr(), pts.shape[0], mu.data_ptr(), q.data_ptr(), q.shape[0], c_float(w),
           out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out


def _case(seed, n, m):
    c = synth.union_cloud(n, seed, n_tori=1, n_ellipsoids=1, noise=0.002)
    mu = (c.normals * (c.area / n)).astype(np.float32)
    lo, hi = c.points.min(0), c.points.max(0)
    q = np.random.default_rng(seed + 1).uniform(lo, hi, (m, 3)).astype(np.float32)
    return c.points, mu, q


def test_no_alloc_matches_the_oracle_on_consecutive_calls():
    """Two calls in a row (the second on a smaller cloud, so stale scratch
    from the first call would show): each result against the FP64 oracle's
    direct sum at the same queries, element by element, within the bound of
    the other parity tests; then against the library's tree entry point at
    theta = 0 within the same bound (the two FP32 sums run in different
    frames and orders)."""
    W, f = _entry()
    for seed, n, m, w in ((11, 20000, 4000, 0.004), (12, 5003, 1500, 0.016)):
        pts, mu, q = _case(seed, n, m)
        tp, tm, tq = (torch.from_numpy(a).cuda() for a in (pts, mu, q))
        st, F = _call(f, tp, tm, tq, w)
        assert st == 0, W.lib().wnnc_last_error()
        F = F.cpu().numpy().astype(np.float64)
        ora, b = oracle.eval_at(oracle.OP_A, pts, mu, q, w, with_bounds=True)
        rms = np.sqrt(np.mean(ora ** 2))
        bound = TOL * np.maximum(np.abs(ora), rms) + SUM_TOL * b["abssum"]
        err = np.abs(F - ora)
        assert np.all(err <= bound), np.max(err / bound)
        print(f"no-alloc vs oracle, n={n}: max |err|/max(|F|,rms) = "
              f"{np.max(err / np.maximum(np.abs(ora), rms)):.2e}")
        ref = W.Tree(tp, theta=0.0).eval_at(tm, tq, w).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(F - ref) <= 2 * bound), np.max(np.abs(F - ref) / bound)


def test_no_alloc_rejects_non_finite_coordinates():
    """A NaN or infinite point or query coordinate is WNNC_EINVAL, as in the
    tree entry points; a valid call right after still succeeds."""
    W, f = _entry()
    pts, mu, q = _case(13, 3000, 300)
    for bad in (float("nan"), float("inf"), -float("inf")):
        tp, tm, tq = (torch.from_numpy(a).cuda() for a in (pts, mu, q))
        tp[1234, 1] = bad
        st, _ = _call(f, tp, tm, tq, 0.01)
        assert st == 1 and b"point" in W.lib().wnnc_last_error()
        tp, tq = torch.from_numpy(pts).cuda(), torch.from_numpy(q).cuda()
        tq[299, 2] = bad
        st, _ = _call(f, tp, tm, tq, 0.01)
        assert st == 1 and b"query" in W.lib().wnnc_last_error()
    st, F = _call(f, torch.from_numpy(pts).cuda(), torch.from_numpy(mu).cuda(), torch.from_numpy(q).cuda(), 0.01)
    assert st == 0 and torch.isfinite(F).all()


def test_no_alloc_rejects_clouds_above_its_limit():
    W, f = _entry()
    pts = torch.zeros(40000, 3, device="cuda")
    q = torch.zeros(8, 3, device="cuda")
    st, _ = _call(f, pts, pts, q, 0.01)
    assert st == 1
    assert b"32768" in W.lib().wnnc_last_error()
