"""B300-native WNNC treecode: Python binding of the C ABI in ``include/wnnc.h``.

This module only marshals arguments: every step of the computation runs in the
CUDA kernels of ``libwnnc.so`` (built in-tree by ``paper_2405_16634_b300.build``).
PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback: loading fails loudly if the library is missing, and every call
raises ``WnncError`` when the library returns a non-OK status.

Operators (Sec. 4 of the paper; w in normalised units, everything else in the
caller's units):

* ``Tree.eval_w(mu, w)``        F(x_i; mu) = A_w(mu)_i          (Eq. 5)
* ``Tree.eval_grad(mu, w)``     grad F(x_i; mu) = -G_w(mu)_i    (Eq. 8-10)
* ``Tree.eval_adjoint(s, w)``   A_w^T(s)                         (Sec. 4.5)
* ``Tree.eval_at(mu, q, w)``    F (or grad F) at query points
* ``Tree.iterate(...)``         Alg. 3 with the gradient step of Alg. 2
* ``orient(points_host)``       the whole solve from host memory to host memory
* ``winding_number(tree, mu, w)`` differentiable F(mu) whose backward is A^T.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_double, c_float, c_int, c_int64, c_void_p

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libwnnc.so")

__all__ = ["Tree", "TreeParams", "IterParams", "WnncError", "winding_number", "WindingNumber",
           "lib", "LIB_PATH", "PROF_CLASSES", "knn16", "Mlp", "MLP_PARAMS", "warm_init", "probe_fp32",
           "orient"]

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ECAPACITY",
          6: "ETIMEOUT"}
SCHEDULES = {"linear": 0, "cosine": 1, "exponential": 2}
PROF_CLASSES = ["moments", "A", "adj_far", "adj_node", "adj_near", "G", "small", "AG", "local"]


class WnncError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"wnnc status {status}: {msg}")
        self.status = status


class TreeParams(Structure):
    _fields_ = [("max_depth", c_int), ("leaf_size", c_int), ("theta", c_float),
                ("rep_mode", c_int), ("moments_fp64", c_int), ("near_bf16", c_int), ("criterion", c_int),
                ("far_order", c_int), ("local_theta", c_float), ("local_cluster", c_int)]


class IterParams(Structure):
    _fields_ = [("n_iter", c_int), ("first_iter", c_int), ("last_iter", c_int),
                ("w1", c_float), ("w2", c_float), ("init", c_int), ("rescale", c_int),
                ("use_grad", c_int), ("use_wnnc", c_int), ("schedule", c_int)]


_lib = None


def build_if_needed() -> str:
    """Compile libwnnc.so if it is missing or older than its sources (nvcc, no GPU needed)."""
    from . import build as _build
    return _build.build()


def lib():
    """Load libwnnc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2405_16634_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    L.wnnc_tree_params_default.argtypes = [POINTER(TreeParams)]
    L.wnnc_iter_params_default.argtypes = [POINTER(IterParams)]
    L.wnnc_build_tree.argtypes = [P, c_int64, POINTER(TreeParams), P, POINTER(c_void_p)]
    L.wnnc_tree_free.argtypes = [P]
    L.wnnc_eval_w.argtypes = [P, P, c_float, P, P]
    L.wnnc_eval_grad.argtypes = [P, P, c_float, P, P]
    L.wnnc_eval_adjoint.argtypes = [P, P, c_float, P, P]
    L.wnnc_eval_at.argtypes = [P, P, P, c_int64, c_float, c_int, P, P]
    L.wnnc_iterate.argtypes = [P, P, P, POINTER(IterParams), P, P]
    L.wnnc_get_stats.argtypes = [P, POINTER(c_int64), POINTER(c_int64)]
    L.wnnc_get_local_stats.argtypes = [P, POINTER(c_int64), POINTER(c_int64)]
    L.wnnc_tree_export_local.argtypes = [P, P, P]
    L.wnnc_get_cluster_stats.argtypes = [P, POINTER(c_int64), POINTER(c_int64)]
    L.wnnc_tree_info.argtypes = [P] + [POINTER(c_int64)] * 7 + [POINTER(c_int)]
    L.wnnc_tree_export.argtypes = [P] + [P] * 11
    L.wnnc_tree_walk_stats.argtypes = [P, P, P]
    L.wnnc_profile_enable.argtypes = [P, c_int]
    L.wnnc_profile_classes.argtypes = [P, ctypes.c_uint]
    L.wnnc_profile_read.argtypes = [P, P, P]
    L.wnnc_profile_reset.argtypes = [P]
    L.wnnc_sync_status.argtypes = [P, P]
    L.wnnc_knn16.argtypes = [P, P, P, P]
    L.wnnc_mlp_create.argtypes = [c_int64, POINTER(c_void_p)]
    L.wnnc_mlp_free.argtypes = [P]
    L.wnnc_mlp_set_params.argtypes = [P, P, P]
    L.wnnc_mlp_get_params.argtypes = [P, P, P]
    L.wnnc_mlp_forward.argtypes = [P, P, c_int64, P, P]
    L.wnnc_mlp_set_loss.argtypes = [P, c_int]
    L.wnnc_mlp_grad.argtypes = [P, P, P, c_int64, P, P, P]
    L.wnnc_mlp_train_step.argtypes = [P, P, P, c_int64, c_float, P, P]
    L.wnnc_warm_init.argtypes = [P, P, c_int64, c_float, P, P]
    L.wnnc_last_error.restype = ctypes.c_char_p
    L.wnnc_kernel_launches.restype = c_int64
    L.wnnc_orient.argtypes = [P, c_int64, POINTER(TreeParams), POINTER(IterParams), P, P, P]
    L.wnnc_orient.restype = c_int
    L.wnnc_debug_fail_alloc.argtypes = [c_int64]
    L.wnnc_debug_fail_alloc.restype = c_int
    L.wnnc_probe_fp32.argtypes = [P, P]
    L.wnnc_probe_fp32.restype = c_int
    L.wnnc_selftest_wait_timeout.argtypes = [P]
    L.wnnc_selftest_wait_timeout.restype = c_int
    for name in ("wnnc_tree_params_default", "wnnc_iter_params_default", "wnnc_build_tree",
                 "wnnc_tree_free", "wnnc_eval_w", "wnnc_eval_grad", "wnnc_eval_adjoint",
                 "wnnc_eval_at", "wnnc_iterate", "wnnc_get_stats", "wnnc_get_local_stats", "wnnc_tree_info",
                 "wnnc_tree_export_local", "wnnc_get_cluster_stats",
                 "wnnc_tree_export", "wnnc_tree_walk_stats", "wnnc_profile_enable", "wnnc_profile_classes", "wnnc_profile_read",
                 "wnnc_profile_reset", "wnnc_sync_status", "wnnc_knn16", "wnnc_mlp_create",
                 "wnnc_mlp_free", "wnnc_mlp_set_params", "wnnc_mlp_get_params", "wnnc_mlp_forward",
                 "wnnc_mlp_set_loss", "wnnc_mlp_grad", "wnnc_mlp_train_step", "wnnc_warm_init"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        msg = lib().wnnc_last_error().decode(errors="replace")
        raise WnncError(status, f"{STATUS.get(status, '?')}: {msg}")


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _dev_f32(t, shape, device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    t = t.to(device=device, dtype=torch.float32).contiguous()
    if tuple(t.shape) != tuple(shape):
        t = t.reshape(shape)
    return t


def orient(points_host, out=None, mu0=None, theta: float = 0.5, leaf_size: int = 8, n_iter: int = 40,
           w1: float = 0.002, w2: float = 0.016, device=None, **tree_kw):
    """The whole orientation through one C-ABI call with host buffers
    (wnnc_orient): points [n][3] float32 on the host (a numpy array or a CPU
    tensor, ideally pinned) in, the oriented field [n][3] out (into `out`, a
    float32 host tensor or array, if given).  mu0: initial field (host) or None
    for the paper's zero start.  Other tree parameters as in Tree."""
    pts = points_host if isinstance(points_host, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(
        points_host, dtype=np.float32))
    if pts.is_cuda or pts.dtype != torch.float32 or not pts.is_contiguous():
        raise ValueError("points_host must be a contiguous float32 host tensor or array")
    n = pts.shape[0]
    if out is None:
        out = torch.empty(n, 3, dtype=torch.float32)
    elif isinstance(out, np.ndarray):
        out = torch.from_numpy(out)
    if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != 3 * n:
        raise ValueError("out must be a contiguous float32 host tensor of n x 3")
    tp = default_tree_params()
    tp.theta, tp.leaf_size = float(theta), int(leaf_size)
    for k, v in tree_kw.items():
        setattr(tp, k, int(v) if not isinstance(v, float) else v)
    ip = default_iter_params()
    ip.n_iter, ip.w1, ip.w2 = int(n_iter), float(w1), float(w2)
    if mu0 is not None:
        out.copy_(torch.as_tensor(mu0, dtype=torch.float32).reshape(n, 3))
        ip.init = 1
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with torch.cuda.device(dev):
        _check(lib().wnnc_orient(pts.data_ptr(), n, ctypes.byref(tp), ctypes.byref(ip), None, out.data_ptr(),
                                 _stream_ptr(dev)))
    return out


def debug_fail_alloc(after: int) -> None:
    """Fault injection for tests: the device allocation after the next
    `after` successful ones fails with WNNC_ENOMEM (after < 0: off)."""
    _check(lib().wnnc_debug_fail_alloc(int(after)))


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().wnnc_kernel_launches())


def probe_fp32(device=None) -> float:
    """Measured FP32 FMA throughput of the device (TFLOP/s)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    v = ctypes.c_double()
    with torch.cuda.device(dev):
        _check(lib().wnnc_probe_fp32(ctypes.byref(v), _stream_ptr(dev)))
    return v.value


def selftest_wait_timeout(device=None) -> int:
    """Run one scan block whose bounded look-back wait runs out; returns the
    library status (WNNC_ETIMEOUT = 6 when the bound and its report work)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with torch.cuda.device(dev):
        return int(lib().wnnc_selftest_wait_timeout(_stream_ptr(dev)))


def default_tree_params() -> TreeParams:
    p = TreeParams()
    _check(lib().wnnc_tree_params_default(ctypes.byref(p)))
    return p


def default_iter_params() -> IterParams:
    p = IterParams()
    _check(lib().wnnc_iter_params_default(ctypes.byref(p)))
    return p


class Tree:
    """Octree, node data and interaction lists of a point cloud on one GPU."""

    def __init__(self, points, theta: float = 0.5, leaf_size: int = 8, max_depth: int = 15,
                 rep_mode: int = 1, moments_fp64: bool = False, near_bf16: bool = False,
                 criterion: int = 0, far_order: int = 0, local_theta: float = 0.0,
                 local_cluster: int = 0):
        """criterion 0: far decisions per target group on boxes, lists built once
        (default); 1: the paper's per-target test of Alg. 4 on every call
        (needs rep_mode 0; with leaf_size 1 it is Alg. 4 as printed).
        far_order 1: far nodes also carry the first-order Taylor terms of the
        kernels about their centroid (rep_mode 1, criterion 0).
        local_theta > 0: far nodes whose box gap to a target group exceeds the
        group box's extent / local_theta are expanded to first order about the
        group's centre instead of summed per target (rep_mode 1, criterion 0,
        far_order 0; A^T stays the exact transpose).  local_cluster = K (2..8)
        adds a second level: far nodes expanded for all K groups of a cluster
        of consecutive groups and local for the cluster's box are expanded once
        about the cluster's centre."""
        pts = points if isinstance(points, torch.Tensor) else torch.as_tensor(points)
        self.device = pts.device if pts.is_cuda else torch.device("cuda", torch.cuda.current_device())
        pts = _dev_f32(pts, (-1, 3), self.device)
        self.n = pts.shape[0]
        p = default_tree_params()
        p.max_depth, p.leaf_size, p.theta = int(max_depth), int(leaf_size), float(theta)
        p.rep_mode, p.moments_fp64 = int(rep_mode), int(bool(moments_fp64))
        p.near_bf16 = int(bool(near_bf16))
        p.criterion = int(criterion)
        p.far_order = int(far_order)
        p.local_theta = float(local_theta)
        p.local_cluster = int(local_cluster)
        self.params = p
        h = c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().wnnc_build_tree(pts.data_ptr(), self.n, ctypes.byref(p),
                                         _stream_ptr(self.device), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().wnnc_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- operators -----------------------------------------------------------
    def eval_w(self, mu, w: float, out: torch.Tensor | None = None) -> torch.Tensor:
        mu = _dev_f32(mu, (self.n, 3), self.device)
        out = torch.empty(self.n, device=self.device, dtype=torch.float32) if out is None else out
        _check(lib().wnnc_eval_w(self._h, mu.data_ptr(), float(w), out.data_ptr(),
                                 _stream_ptr(self.device)))
        return out

    def eval_grad(self, mu, w: float, out: torch.Tensor | None = None) -> torch.Tensor:
        mu = _dev_f32(mu, (self.n, 3), self.device)
        out = torch.empty(self.n, 3, device=self.device, dtype=torch.float32) if out is None else out
        _check(lib().wnnc_eval_grad(self._h, mu.data_ptr(), float(w), out.data_ptr(),
                                    _stream_ptr(self.device)))
        return out

    def eval_adjoint(self, s, w: float, out: torch.Tensor | None = None) -> torch.Tensor:
        s = _dev_f32(s, (self.n,), self.device)
        out = torch.empty(self.n, 3, device=self.device, dtype=torch.float32) if out is None else out
        _check(lib().wnnc_eval_adjoint(self._h, s.data_ptr(), float(w), out.data_ptr(),
                                       _stream_ptr(self.device)))
        return out

    def eval_at(self, mu, q, w: float, grad: bool = False) -> torch.Tensor:
        mu = _dev_f32(mu, (self.n, 3), self.device)
        q = _dev_f32(q, (-1, 3), self.device)
        m = q.shape[0]
        out = torch.empty((m, 3) if grad else (m,), device=self.device, dtype=torch.float32)
        _check(lib().wnnc_eval_at(self._h, mu.data_ptr(), q.data_ptr(), m, float(w), int(grad),
                                  out.data_ptr(), _stream_ptr(self.device)))
        return out

    def iterate(self, mu=None, n_iter: int = 40, w1: float = 0.002, w2: float = 0.016,
                first_iter: int = 1, last_iter: int = 0, area=None, rescale: int = 0,
                use_grad: bool = True, use_wnnc: bool = True, stats: bool = False, out=None,
                schedule="linear"):
        """Alg. 3.  mu None = zero init; returns mu (and per-iteration stats).
        schedule: width schedule "linear" (the paper's), "cosine" or "exponential"
        (or its code 0, 1, 2)."""
        p = default_iter_params()
        p.n_iter, p.first_iter, p.last_iter = int(n_iter), int(first_iter), int(last_iter)
        p.w1, p.w2 = float(w1), float(w2)
        p.init = 0 if mu is None else 1
        p.rescale, p.use_grad, p.use_wnnc = int(rescale), int(bool(use_grad)), int(bool(use_wnnc))
        p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        if out is not None:
            mu_t = out
            if mu is not None:
                mu_t.copy_(_dev_f32(mu, (self.n, 3), self.device))
        elif mu is None:
            mu_t = torch.zeros(self.n, 3, device=self.device, dtype=torch.float32)
        else:
            mu_t = _dev_f32(mu, (self.n, 3), self.device).clone()
        ar = None if area is None else _dev_f32(area, (self.n,), self.device)
        last = last_iter if last_iter > 0 else n_iter
        st = torch.zeros(max(last - first_iter + 1, 1), 4, device=self.device, dtype=torch.float32) \
            if stats else None
        _check(lib().wnnc_iterate(self._h, mu_t.data_ptr(), None if ar is None else ar.data_ptr(),
                                  ctypes.byref(p), _stream_ptr(self.device),
                                  None if st is None else st.data_ptr()))
        return (mu_t, st) if stats else mu_t

    # -- inspection ----------------------------------------------------------
    def stats(self):
        """(far pairs, near pairs) summed pair by pair in one operator evaluation
        on the points."""
        f, nn = c_int64(), c_int64()
        _check(lib().wnnc_get_stats(self._h, ctypes.byref(f), ctypes.byref(nn)))
        return f.value, nn.value

    def local_stats(self):
        """(far entries expanded about their group's centre, the pairs they stand for)."""
        e, pp = c_int64(), c_int64()
        _check(lib().wnnc_get_local_stats(self._h, ctypes.byref(e), ctypes.byref(pp)))
        return e.value, pp.value

    def cluster_stats(self):
        """((cluster, node) expansions of the second level, the pairs they stand for)."""
        e, pp = c_int64(), c_int64()
        _check(lib().wnnc_get_cluster_stats(self._h, ctypes.byref(e), ctypes.byref(pp)))
        return e.value, pp.value

    def info(self) -> dict:
        v = [c_int64() for _ in range(7)]
        d = c_int()
        _check(lib().wnnc_tree_info(self._h, *[ctypes.byref(x) for x in v], ctypes.byref(d)))
        keys = ["n", "nnodes", "nleaves", "ngroups", "far_entries", "near_ranges", "tnear_entries"]
        out = {k: x.value for k, x in zip(keys, v)}
        out["depth"] = d.value
        return out

    def walk_stats(self) -> dict:
        """How the list traversal ran: groups finished as depth-first walks,
        and whether all groups ran again with the larger buffer."""
        a, b = c_int(), c_int()
        _check(lib().wnnc_tree_walk_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"stack_walk_groups": a.value, "big_stack": bool(b.value)}

    def export(self) -> dict:
        inf = self.info()
        n, nn, ng = inf["n"], inf["nnodes"], inf["ngroups"]
        a = dict(perm=np.zeros(n, np.int64), node_start=np.zeros(nn, np.int32),
                 node_count=np.zeros(nn, np.int32), node_depth=np.zeros(nn, np.int32),
                 node_nchild=np.zeros(nn, np.int32), far_off=np.zeros(ng + 1, np.int32),
                 far_id=np.zeros(max(inf["far_entries"], 1), np.int32),
                 near_off=np.zeros(ng + 1, np.int32),
                 near_rng=np.zeros((max(inf["near_ranges"], 1), 2), np.int32),
                 group_off=np.zeros(ng + 1, np.int32), center_scale=np.zeros(4, np.float64))
        ptr = lambda x: x.ctypes.data_as(c_void_p)
        _check(lib().wnnc_tree_export(self._h, *[ptr(a[k]) for k in (
            "perm", "node_start", "node_count", "node_depth", "node_nchild", "far_off", "far_id",
            "near_off", "near_rng", "group_off", "center_scale")]))
        a["far_id"] = a["far_id"][:inf["far_entries"]]
        a["near_rng"] = a["near_rng"][:inf["near_ranges"]]
        a["far_lsplit"] = np.zeros(ng, np.int32)
        a["far_csplit"] = np.zeros(ng, np.int32)
        if ng:
            _check(lib().wnnc_tree_export_local(self._h, ptr(a["far_lsplit"]), ptr(a["far_csplit"])))
        return a

    def profile(self, enable: bool = True, classes=None):
        """Record per-class kernel times (CUDA events); `classes` (names of
        PROF_CLASSES) restricts the recording, None records every class."""
        mask = 0xFFFFFFFF if classes is None else sum(1 << PROF_CLASSES.index(c) for c in classes)
        _check(lib().wnnc_profile_classes(self._h, mask))
        _check(lib().wnnc_profile_enable(self._h, int(bool(enable))))

    def profile_read(self) -> dict:
        n = len(PROF_CLASSES)
        launches = np.zeros(n, np.int64)
        ms = np.zeros(n, np.float64)
        _check(lib().wnnc_profile_read(self._h, launches.ctypes.data_as(c_void_p),
                                       ms.ctypes.data_as(c_void_p)))
        return {k: (int(launches[i]), float(ms[i])) for i, k in enumerate(PROF_CLASSES)}

    def profile_reset(self):
        _check(lib().wnnc_profile_reset(self._h))

    def sync_status(self) -> None:
        _check(lib().wnnc_sync_status(self._h, _stream_ptr(self.device)))


def knn16(tree: Tree):
    """(idx [n][16] int32 input indices, feat [n][48] float32) of the tree's points."""
    idx = torch.empty(tree.n, 16, device=tree.device, dtype=torch.int32)
    feat = torch.empty(tree.n, 48, device=tree.device, dtype=torch.float32)
    _check(lib().wnnc_knn16(tree._h, idx.data_ptr(), feat.data_ptr(), _stream_ptr(tree.device)))
    return idx, feat


MLP_PARAMS = 39683


class Mlp:
    """The warm-start point-patch MLP (48 -> 128 -> 128 -> 128 -> 3, BF16 weights)."""

    def __init__(self, max_batch: int = 65536, params=None, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.max_batch = int(max_batch)
        h = c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().wnnc_mlp_create(self.max_batch, ctypes.byref(h)))
        self._h = h
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().wnnc_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        p = _dev_f32(params, (MLP_PARAMS,), self.device)
        _check(lib().wnnc_mlp_set_params(self._h, p.data_ptr(), _stream_ptr(self.device)))
        torch.cuda.current_stream(self.device).synchronize()

    def get_params(self) -> torch.Tensor:
        p = torch.empty(MLP_PARAMS, device=self.device, dtype=torch.float32)
        _check(lib().wnnc_mlp_get_params(self._h, p.data_ptr(), _stream_ptr(self.device)))
        return p

    def forward(self, x) -> torch.Tensor:
        x = _dev_f32(x, (-1, 48), self.device)
        y = torch.empty(x.shape[0], 3, device=self.device, dtype=torch.float32)
        _check(lib().wnnc_mlp_forward(self._h, x.data_ptr(), x.shape[0], y.data_ptr(), _stream_ptr(self.device)))
        return y

    def set_loss(self, mode: int):
        """0: 1 - c (signed, default); 1: 1 - c^2 (sign-free); c = (y/|y|).label."""
        _check(lib().wnnc_mlp_set_loss(self._h, int(mode)))

    def grad(self, x, label):
        x = _dev_f32(x, (-1, 48), self.device)
        label = _dev_f32(label, (x.shape[0], 3), self.device)
        g = torch.empty(MLP_PARAMS, device=self.device, dtype=torch.float32)
        loss = torch.empty(1, device=self.device, dtype=torch.float32)
        _check(lib().wnnc_mlp_grad(self._h, x.data_ptr(), label.data_ptr(), x.shape[0], g.data_ptr(),
                                   loss.data_ptr(), _stream_ptr(self.device)))
        return g, loss

    def train_step(self, x, label, lr: float) -> torch.Tensor:
        loss = torch.empty(1, device=self.device, dtype=torch.float32)
        _check(lib().wnnc_mlp_train_step(self._h, x.data_ptr(), label.data_ptr(), x.shape[0], float(lr),
                                         loss.data_ptr(), _stream_ptr(self.device)))
        return loss


def warm_init(direction, reference, area: float) -> torch.Tensor:
    """mu = area * dir/|dir|, flipped where dir . reference < 0 (reference may be None)."""
    d = direction.contiguous()
    n = d.shape[0]
    mu = torch.empty_like(d)
    ref = None if reference is None else reference.contiguous()
    _check(lib().wnnc_warm_init(d.data_ptr(), None if ref is None else ref.data_ptr(), n, float(area),
                                mu.data_ptr(), _stream_ptr(d.device)))
    return mu


class WindingNumber(torch.autograd.Function):
    """F(mu) = A_w(mu) at the tree's points; backward = A_w^T (Sec. 4.5).

    The backward is the exact transpose of the forward tree operator only for
    a tree with point-centroid representatives (rep_mode 1) and float
    near-field coordinates: then gradients agree with finite differences of
    the forward.  With the paper's |nu|-weighted representatives (rep_mode 0)
    the forward is not even linear in mu (the representatives move with mu)
    and A^T is the paper's separate s-representative treecode; with bfloat16
    near-field coordinates the forward rounds coordinates that the adjoint
    does not.  forward() refuses such trees rather than return a gradient
    that is not the forward's."""

    @staticmethod
    def forward(ctx, mu, tree: Tree, w: float):
        if tree.params.rep_mode != 1 or tree.params.near_bf16:
            raise ValueError("winding_number needs a tree with rep_mode=1 and near_bf16=False: "
                             "only then is the backward (A^T) the exact transpose of the forward")
        ctx.tree, ctx.w = tree, w
        return tree.eval_w(mu.detach(), w)

    @staticmethod
    def backward(ctx, g):
        return ctx.tree.eval_adjoint(g.contiguous(), ctx.w), None, None


def winding_number(tree: Tree, mu: torch.Tensor, w: float) -> torch.Tensor:
    return WindingNumber.apply(mu, tree, w)
