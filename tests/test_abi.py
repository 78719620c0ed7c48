"""The C-ABI library loads and exports every entry point that include/wnnc.h
declares; argument errors are reported as status codes (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wnnc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(wnnc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wnnc_build_tree", "wnnc_eval_w", "wnnc_eval_grad", "wnnc_eval_adjoint",
                     "wnnc_iterate", "wnnc_tree_free", "wnnc_get_stats", "wnnc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2405_16634_b300 as W
    W.build_if_needed()
    L = W.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_defaults_and_argument_errors_without_gpu():
    import paper_2405_16634_b300 as W
    W.build_if_needed()
    L = W.lib()
    p = W.default_tree_params()
    assert (p.max_depth, p.leaf_size, p.rep_mode, p.moments_fp64, p.near_bf16) == (15, 8, 1, 0, 0)
    assert abs(p.theta - 0.5) < 1e-7
    q = W.default_iter_params()
    assert (q.n_iter, q.first_iter, q.last_iter, q.init, q.rescale, q.use_grad, q.use_wnnc,
            q.schedule) == (40, 1, 0, 0, 0, 1, 1, 0)
    assert abs(q.w1 - 0.002) < 1e-9 and abs(q.w2 - 0.016) < 1e-9
    assert L.wnnc_tree_params_default(None) == 1
    h = ctypes.c_void_p()
    assert L.wnnc_build_tree(None, 10, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert b"NULL" in L.wnnc_last_error()
    assert L.wnnc_eval_w(None, None, ctypes.c_float(0.0), None, None) == 1
    assert L.wnnc_tree_free(None) == 0


def test_mode_parameters_are_checked_before_any_device_work():
    """criterion, far_order, local_theta and local_cluster: defaults 0; values out of range
    or in combinations the modes do not support are WNNC_EINVAL, reported
    before the library touches the device (the point pointer below is never
    read)."""
    import paper_2405_16634_b300 as W
    W.build_if_needed()
    L = W.lib()
    p = W.default_tree_params()
    assert (p.criterion, p.far_order, p.local_theta, p.local_cluster) == (0, 0, 0.0, 0)
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(256)
    for kw, msg in (({"criterion": 2}, b"criterion"), ({"criterion": 1, "rep_mode": 1}, b"rep_mode 0"),
                    ({"far_order": 2}, b"far_order"), ({"far_order": 1, "rep_mode": 0}, b"far_order 1"),
                    ({"far_order": 1, "rep_mode": 0, "criterion": 1}, b"far_order 1"),
                    ({"local_theta": -0.5}, b"local_theta"), ({"local_theta": float("inf")}, b"local_theta"),
                    ({"local_theta": float("nan")}, b"local_theta"),
                    ({"local_theta": 0.5, "rep_mode": 0}, b"local_theta > 0"),
                    ({"local_theta": 0.5, "far_order": 1}, b"local_theta > 0"),
                    ({"local_theta": 0.5, "rep_mode": 0, "criterion": 1}, b"local_theta > 0"),
                    ({"local_theta": 0.5, "local_cluster": 1}, b"local_cluster"),
                    ({"local_theta": 0.5, "local_cluster": 9}, b"local_cluster"),
                    ({"local_theta": 0.5, "local_cluster": -4}, b"local_cluster"),
                    ({"local_cluster": 4}, b"local_cluster needs")):
        q = W.default_tree_params()
        for k, v in kw.items():
            setattr(q, k, v)
        assert L.wnnc_build_tree(fake, 10, ctypes.byref(q), None, ctypes.byref(h)) == 1
        assert msg in L.wnnc_last_error(), (kw, L.wnnc_last_error())


def test_orient_argument_errors_without_gpu():
    import paper_2405_16634_b300 as W
    W.build_if_needed()
    L = W.lib()
    buf = (ctypes.c_float * 30)()
    assert L.wnnc_orient(None, 10, None, None, None, buf, None) == 1
    assert L.wnnc_orient(buf, 10, None, None, None, None, None) == 1
    assert L.wnnc_orient(buf, 0, None, None, None, buf, None) == 1
    q = W.default_iter_params()
    q.rescale = 1
    assert L.wnnc_orient(buf, 10, None, ctypes.byref(q), None, buf, None) == 1
    assert b"area_host" in L.wnnc_last_error()
