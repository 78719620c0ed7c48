"""FP64 CPU oracle for the WNNC hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is written from the paper alone and
shares no code with the CUDA path; it loads a small C library
(``wnnc_oracle.c``, built into ``oracle/_build/``) that holds the O(N^2) sums,
the treecode and the iteration, all in double precision.

Units.  ``direct`` works on whatever coordinates it is given.  The ``eval_*``
and ``iterate`` functions mirror the library's boundary: points and normals in
the caller's units, the smoothing width ``w`` in the normalised units of
Sec. 5.1.1 (the cloud scaled into [-1,1]^3 with a 1/11 margin, by s), and
results converted back (mu scales like area, s^2; the gradient of F like 1/length, s;
A^T s like s^2 so that <A mu, v> = <mu, A^T v> holds in caller units).

Parity status of each function (pins live in tests/test_oracle_pins.py):
  direct A, G, A^T   pinned (closed forms on spheres, F(centre)=1, FD of A = -G,
                     adjointness, symmetry, scaling and rotation invariance)
  paper treecode     pinned (Alg. 4 per target with the Eq. 13-14 representatives:
  (PaperTree)        theta->0 equals direct, a hand-worked far node for A, G and
                     A^T, representatives invariant under sign flips of nu and
                     inside the node's convex hull, second-order far error for
                     parallel nu, error vs direct falls with theta, octree cells)
  tree A, G, A^T     pinned (theta->0 limit equals direct, error decreases with
  (group treecode)   theta in both representative modes, exact adjointness of
                     the rep_mode-1 pair, Alg. 4 per-target criterion holds for
                     every far use, the hand-worked far node in rep_mode 0)
  iterate            pinned (first-iteration closed form on a sphere, energy
                     decrease of the exact line search, P_co = 100% on a sphere,
                     the zero-init / no-grad-step behaviour of Sec. 6.1.3)
  knn                pinned (against sorting all distances)
  mlp                pinned (finite differences)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from ctypes import POINTER, c_double, c_int, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wnnc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

OP_A, OP_G, OP_AT = 0, 1, 2
GROUP_SIZE = 32
GROUP_SLACK = 3     # target groups never straddle leaves without a common ancestor 3 levels up
GROUP_MIN_DEPTH = 3  # ... and stay inside one cell of depth 3


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp -ffp-contract=off: a C file of the oracle into a shared library."""
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-std=c11", src, "-o", out, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load(build())
    return _lib


def load(path: str):
    """Load a build of wnnc_oracle.c and declare its C signatures."""
    L = ctypes.CDLL(path)
    d, i64, P = c_double, c_int64, POINTER
    L.or_num_threads.restype = c_int
    L.or_normalize.argtypes = [c_void_p, i64, c_void_p, c_void_p, c_void_p]
    L.or_direct.argtypes = [c_int, c_void_p, i64, c_void_p, c_void_p, i64, d, d, c_void_p, c_void_p,
                            c_void_p]
    L.or_tree_build.argtypes = [c_void_p, i64, c_int, c_int, c_int, d, c_int, c_int]
    L.or_tree_ngroups.argtypes = [c_void_p]
    L.or_tree_ngroups.restype = i64
    L.or_tree_groups.argtypes = [c_void_p, c_void_p]
    L.or_tree_build.restype = c_void_p
    L.or_tree_set_far_order.argtypes = [c_void_p, c_int]
    L.or_tree_set_local.argtypes = [c_void_p, d, c_int]
    L.or_tree_local_classes.argtypes = [c_void_p, c_void_p]
    L.or_tree_free.argtypes = [c_void_p]
    L.or_tree_nnodes.argtypes = [c_void_p]
    L.or_tree_nnodes.restype = i64
    L.or_tree_nodes.argtypes = [c_void_p] + [c_void_p] * 5
    L.or_tree_perm.argtypes = [c_void_p, c_void_p]
    L.or_tree_boxes.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.or_tree_counts.argtypes = [c_void_p, c_void_p]
    L.or_tree_lists.argtypes = [c_void_p] + [c_void_p] * 4
    L.or_tree_apply.argtypes = [c_void_p, c_int, c_int, d, c_void_p, c_void_p, d, c_void_p, c_void_p]
    L.or_tree_apply_at.argtypes = [c_void_p, c_int, c_int, d, c_void_p, c_void_p, i64, c_void_p,
                                   c_void_p, c_void_p]
    L.or_schedule_width.argtypes = [c_int, c_int, d, d]
    L.or_schedule_width.restype = d
    L.or_schedule_width2.argtypes = [c_int, c_int, d, d, c_int]
    L.or_schedule_width2.restype = d
    L.or_iterate.argtypes = [c_void_p, c_void_p, d, c_void_p, i64, c_void_p, c_int, c_int, c_int, d, d,
                             c_int, c_int, c_void_p, c_int, c_int, c_int, c_void_p]
    L.or_ptree_build.argtypes = [c_void_p, i64, c_int, c_int]
    L.or_ptree_build.restype = c_void_p
    L.or_ptree_free.argtypes = [c_void_p]
    L.or_ptree_nnodes.argtypes = [c_void_p]
    L.or_ptree_nnodes.restype = i64
    L.or_ptree_nodes.argtypes = [c_void_p] + [c_void_p] * 6
    L.or_ptree_apply.argtypes = [c_void_p, c_int, d, d, c_void_p, c_void_p, i64, c_void_p, d, c_void_p,
                                 c_void_p, c_void_p]
    L.or_knn.argtypes = [c_void_p, i64, c_int, c_void_p, c_void_p]
    return L


def _p(a):
    return a.ctypes.data_as(c_void_p) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def num_threads() -> int:
    return lib().or_num_threads()


# ---------------------------------------------------------------------------
# Normalisation (Sec. 5.1.1)
# ---------------------------------------------------------------------------

def normalize(points):
    """(xn, center, scale): xn = (x - center) * scale, in float64."""
    pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    n = pts.shape[0]
    xn = np.empty((n, 3))
    c = np.empty(3)
    s = np.empty(1)
    lib().or_normalize(_p(pts), n, _p(xn), _p(c), _p(s))
    return xn, c, float(s[0])


def apply_normalization(q, center, scale):
    """Map caller-unit query points into normalised units (same formula)."""
    q = np.asarray(q, dtype=np.float32).astype(np.float64).reshape(-1, 3)
    return (q - center) * scale


# ---------------------------------------------------------------------------
# Direct O(N*M) sums (the plain definitions of A, G, A^T)
# ---------------------------------------------------------------------------

def direct(op: int, x, nu, w: float, y=None, amb_tol: float = 0.0):
    """Direct sum of operator ``op`` with sources x, attribute nu, targets y
    (default: the sources).  Returns (out, bounds); bounds is None unless
    amb_tol > 0, else a dict of per-target arrays:
      amb    sum of |term| over pairs whose r^2 is within amb_tol*w^2 of w^2
             (a lower-precision cut-off test may decide them either way)
      abssum sum of |term| over the counted pairs (the scale of the rounding
             error of any floating-point evaluation of the sum)."""
    x = _f64(x, (-1, 3))
    y = x if y is None else _f64(y, (-1, 3))
    ns, nt = x.shape[0], y.shape[0]
    nu = _f64(nu, (ns, 3) if op != OP_AT else (ns,))
    out = np.zeros(nt) if op == OP_A else np.zeros((nt, 3))
    amb = np.zeros(nt) if amb_tol > 0 else None
    abssum = np.zeros(nt) if amb_tol > 0 else None
    lib().or_direct(op, _p(x), ns, _p(nu), _p(y), nt, float(w), float(amb_tol), _p(out), _p(amb),
                    _p(abssum))
    return out, (None if amb is None else {"amb": amb, "abssum": abssum})


# ---------------------------------------------------------------------------
# Treecode
# ---------------------------------------------------------------------------

class Tree:
    """Source octree + on-surface target groups over normalised points xn."""

    def __init__(self, xn, theta: float, leaf_size: int = 8, max_depth: int = 15,
                 group_size: int = GROUP_SIZE, group_slack: int = GROUP_SLACK,
                 group_min_depth: int = GROUP_MIN_DEPTH, far_order: int = 0,
                 local_theta: float = 0.0, local_cluster: int = 0):
        """far_order 1 adds the first-order Taylor terms of the kernels about
        each far node's point centroid (rep_mode 1; A, G and the exact A^T).
        local_theta > 0 (far_order 0, rep_mode 1) expands the far field of
        every far node whose box gap to a target group exceeds the group
        box's largest extent / local_theta to first order about the group box
        centre (A, G and the exact A^T); an entry falls back to pair terms at
        widths w that may reach one of its pairs.  local_cluster >= 2 also
        expands, once per cluster of that many consecutive groups, the far
        nodes in the expanded part of every member's list that are local for
        the cluster's box, about the cluster's centre."""
        self.xn = _f64(xn, (-1, 3))
        self.n = self.xn.shape[0]
        self.theta = float(theta)
        self._h = lib().or_tree_build(_p(self.xn), self.n, leaf_size, group_size, max_depth, self.theta,
                                      int(group_slack), int(group_min_depth))
        lib().or_tree_set_far_order(self._h, int(far_order))
        lib().or_tree_set_local(self._h, float(local_theta), int(local_cluster))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tree_free(self._h)
            self._h = None

    def apply(self, op: int, nu, w: float, rep_mode: int = 1, amb_tol: float = 0.0):
        """Tree operator on the points; with amb_tol > 0 returns (out, bounds)
        (bounds as in ``direct``)."""
        nu = _f64(nu, (self.n, 3) if op != OP_AT else (self.n,))
        out = np.zeros(self.n) if op == OP_A else np.zeros((self.n, 3))
        amb = np.zeros(self.n) if amb_tol > 0 else None
        abssum = np.zeros(self.n) if amb_tol > 0 else None
        lib().or_tree_apply(self._h, op, rep_mode, float(w), _p(nu), _p(out), float(amb_tol), _p(amb),
                            _p(abssum))
        return (out, {"amb": amb, "abssum": abssum}) if amb_tol > 0 else out

    def apply_at(self, op: int, nu, qn, w: float, rep_mode: int = 1):
        """(out, pairs, abssum) at off-surface targets qn."""
        nu = _f64(nu, (self.n, 3))
        qn = _f64(qn, (-1, 3))
        m = qn.shape[0]
        out = np.zeros(m) if op == OP_A else np.zeros((m, 3))
        pairs = np.zeros(2, np.int64)
        abssum = np.zeros(m)
        lib().or_tree_apply_at(self._h, op, rep_mode, float(w), _p(nu), _p(qn), m, _p(out), _p(pairs),
                               _p(abssum))
        return out, pairs, abssum

    def counts(self):
        """(far list entries, near list entries, far pairs, near pairs)."""
        c = np.zeros(4, np.int64)
        lib().or_tree_counts(self._h, _p(c))
        return tuple(int(v) for v in c)

    def nodes(self):
        m = lib().or_tree_nnodes(self._h)
        start = np.zeros(m, np.int64); count = np.zeros(m, np.int64)
        depth = np.zeros(m, np.int32); nchild = np.zeros(m, np.int32); parent = np.zeros(m, np.int64)
        lib().or_tree_nodes(self._h, _p(start), _p(count), _p(depth), _p(nchild), _p(parent))
        lo = np.zeros((m, 3)); hi = np.zeros((m, 3)); cent = np.zeros((m, 3))
        lib().or_tree_boxes(self._h, _p(lo), _p(hi), _p(cent))
        return dict(start=start, count=count, depth=depth, nchild=nchild, parent=parent,
                    lo=lo, hi=hi, cent=cent)

    def perm(self):
        p = np.zeros(self.n, np.int64)
        lib().or_tree_perm(self._h, _p(p))
        return p

    def groups(self):
        """Group offsets: group g = sorted points goff[g] .. goff[g+1]-1."""
        ng = lib().or_tree_ngroups(self._h)
        g = np.zeros(ng + 1, np.int64)
        lib().or_tree_groups(self._h, _p(g))
        return g

    def local_classes(self):
        """Per far entry (in the order of ``lists``): 0 summed pair by pair, 1
        expanded about its group's centre, 2 about its cluster's."""
        c = np.zeros(max(self.counts()[0], 1), np.int8)
        lib().or_tree_local_classes(self._h, _p(c))
        return c[:self.counts()[0]]

    def lists(self):
        ng = lib().or_tree_ngroups(self._h)
        c = self.counts()
        fo = np.zeros(ng + 1, np.int64); no = np.zeros(ng + 1, np.int64)
        fi = np.zeros(max(c[0], 1), np.int64); ni = np.zeros(max(c[1], 1), np.int64)
        lib().or_tree_lists(self._h, _p(fo), _p(fi), _p(no), _p(ni))
        return fo, fi[:c[0]], no, ni[:c[1]]


# ---------------------------------------------------------------------------
# The paper's treecode (Sec. 4.5, Eq. 13-14, Alg. 4)
# ---------------------------------------------------------------------------

class PaperTree:
    """Alg. 4 as printed: a geometric octree of the sources (cubes of
    [-1,1]^3 split into octants while they hold more than leaf_size points and
    are shallower than max_depth; leaf_size 1 is the paper's), the
    nu-representatives of Eq. 13-14 recomputed per call, and for each target
    a recursion from the root taking node B as far iff
    |y - x_{B,nu}| > width(B)/theta.  Coordinates are used as given (call
    ``normalize`` first for the paper's frame)."""

    def __init__(self, x, leaf_size: int = 1, max_depth: int = 15):
        self.x = _f64(x, (-1, 3))          # kept alive: the C side points into it
        self.n = self.x.shape[0]
        self._h = lib().or_ptree_build(_p(self.x), self.n, int(leaf_size), int(max_depth))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_ptree_free(self._h)
            self._h = None

    def apply(self, op: int, nu, w: float, theta: float, y=None, amb_tol: float = 0.0):
        """(out, info): op at targets y (default: the sources).  info holds
        'far' and 'near' term counts and, with amb_tol > 0, per-target 'amb'
        (sum |term| of cut-off-ambiguous pairs plus the branch difference of
        far decisions within amb_tol of the threshold) and 'abssum'."""
        y = self.x if y is None else _f64(y, (-1, 3))
        nt = y.shape[0]
        nu = _f64(nu, (self.n, 3) if op != OP_AT else (self.n,))
        out = np.zeros(nt) if op == OP_A else np.zeros((nt, 3))
        amb = np.zeros(nt) if amb_tol > 0 else None
        abssum = np.zeros(nt) if amb_tol > 0 else None
        cnt = np.zeros(2, np.int64)
        lib().or_ptree_apply(self._h, op, float(theta), float(w), _p(nu), _p(y), nt, _p(out), float(amb_tol),
                             _p(amb), _p(abssum), _p(cnt))
        info = {"far": int(cnt[0]), "near": int(cnt[1])}
        if amb_tol > 0:
            info.update(amb=amb, abssum=abssum)
        return out, info

    def nodes(self):
        m = lib().or_ptree_nnodes(self._h)
        start = np.zeros(m, np.int64); count = np.zeros(m, np.int64)
        depth = np.zeros(m, np.int32); nchild = np.zeros(m, np.int32)
        ctr = np.zeros((m, 3)); idx = np.zeros(self.n, np.int64)
        lib().or_ptree_nodes(self._h, _p(start), _p(count), _p(depth), _p(nchild), _p(ctr), _p(idx))
        return dict(start=start, count=count, depth=depth, nchild=nchild, ctr=ctr, idx=idx)


def eval_paper(op: int, points, nu, w: float, theta: float, targets=None, leaf_size: int = 1,
               max_depth: int = 15, amb_tol: float = 0.0):
    """The paper's treecode (Alg. 4) in caller units, like ``eval_op``:
    op A: nu = mu -> F;  op G: nu = mu -> grad F = -G;  op AT: nu = s -> A^T s.
    targets: indices of the points to evaluate at (default all).  Returns
    (out, info) with info as in ``PaperTree.apply`` (bounds scaled to caller
    units)."""
    xn, c, s = normalize(points)
    y = xn if targets is None else xn[np.asarray(targets)]
    nu = np.asarray(nu, dtype=np.float64)
    nun = nu * (s * s) if op != OP_AT else nu
    out, info = PaperTree(xn, leaf_size, max_depth).apply(op, nun, w, theta, y=y, amb_tol=amb_tol)
    f = 1.0
    if op == OP_G:
        out, f = -out * s, s
    elif op == OP_AT:
        out, f = out * (s * s), s * s
    for k in ("amb", "abssum"):
        if k in info:
            info[k] = info[k] * f
    return out, info


def eval_direct_at(op: int, points, nu, w: float, targets=None, amb_tol: float = 1e-5):
    """The direct sums in caller units at a subset of the points (indices
    ``targets``, default all), over all points as sources: (out, bounds)."""
    xn, c, s = normalize(points)
    y = xn if targets is None else xn[np.asarray(targets)]
    nu = np.asarray(nu, dtype=np.float64)
    nun = nu * (s * s) if op != OP_AT else nu
    out, b = direct(op, xn, nun, w, y=y, amb_tol=amb_tol)
    f = 1.0
    if op == OP_G:
        out, f = -out * s, s
    elif op == OP_AT:
        out, f = out * (s * s), s * s
    if b is not None:
        b = {k: v * f for k, v in b.items()}
    return out, b


# ---------------------------------------------------------------------------
# Boundary-shaped entry points (caller units, like the library's C ABI)
# ---------------------------------------------------------------------------

def _setup(points, theta, leaf_size, max_depth, far_order=0, local_theta=0.0, local_cluster=0):
    xn, c, s = normalize(points)
    tree = (Tree(xn, theta, leaf_size, max_depth, far_order=far_order, local_theta=local_theta,
                 local_cluster=local_cluster)
            if theta > 0 else None)
    return xn, c, s, tree


def eval_op(op: int, points, nu, w: float, theta: float = 0.0, leaf_size: int = 8,
            max_depth: int = 15, rep_mode: int = 1, amb_tol: float = 0.0, far_order: int = 0,
            local_theta: float = 0.0, local_cluster: int = 0):
    """One operator at the input points, caller units in and out.

    op A: nu = mu (N,3) -> F (N,);  op G: nu = mu -> grad F = -G (N,3);
    op AT: nu = s (N,) -> A^T s (N,3).  theta = 0 uses the direct sums."""
    xn, c, s, tree = _setup(points, theta, leaf_size, max_depth, far_order, local_theta, local_cluster)
    nu = np.asarray(nu, dtype=np.float64)
    nun = nu * (s * s) if op != OP_AT else nu
    bounds = None
    if tree is None:
        out, bounds = direct(op, xn, nun, w, amb_tol=amb_tol)
    elif amb_tol > 0:
        out, bounds = tree.apply(op, nun, w, rep_mode, amb_tol=amb_tol)
    else:
        out = tree.apply(op, nun, w, rep_mode)
    f = 1.0
    if op == OP_G:
        out, f = -out * s, s          # grad F in caller units
    elif op == OP_AT:
        out, f = out * (s * s), s * s
    if bounds is not None:
        bounds = {k: v * f for k, v in bounds.items()}
    return out, bounds


def eval_at(op: int, points, mu, queries, w: float, theta: float = 0.0, leaf_size: int = 8,
            max_depth: int = 15, rep_mode: int = 1, with_bounds: bool = False, far_order: int = 0,
            local_theta: float = 0.0, local_cluster: int = 0):
    """A (F) or grad F at off-surface query points (caller units); with
    with_bounds also the per-target bounds (amb is zero here: w applies only
    through the cut-off, and off-surface tests use w = 0)."""
    xn, c, s, tree = _setup(points, theta, leaf_size, max_depth, far_order, local_theta, local_cluster)
    qn = apply_normalization(queries, c, s)
    mun = np.asarray(mu, dtype=np.float64) * (s * s)
    if tree is None:
        out, b = direct(op, xn, mun, w, y=qn, amb_tol=1e-5)
        abssum = b["abssum"]
    else:
        out, _, abssum = tree.apply_at(op, mun, qn, w, rep_mode)
    f = s if op == OP_G else 1.0
    out = -out * s if op == OP_G else out
    if with_bounds:
        return out, {"amb": np.zeros(len(out)), "abssum": abssum * f}
    return out


def iterate(points, mu0=None, n_iter: int = 40, w1: float = 0.002, w2: float = 0.016,
            theta: float = 0.0, leaf_size: int = 8, max_depth: int = 15, rep_mode: int = 1,
            first_iter: int = 1, last_iter: int | None = None, rescale: int = 0, area=None,
            use_grad: bool = True, use_wnnc: bool = True, schedule="linear", paper_theta: float = 0.0,
            paper_leaf_size: int = 1, far_order: int = 0, local_theta: float = 0.0,
            local_cluster: int = 0):
    """Alg. 3 on the cloud; returns (mu in caller units, stats[iter] = (w, E, alpha, |r|^2)).
    Operators: theta > 0 the group treecode (leaf_size, rep_mode); else
    paper_theta > 0 the paper's treecode (Alg. 4, per target, paper_leaf_size);
    else the direct sums.
    schedule: the width schedule, "linear" (Alg. 3), "cosine" or "exponential"
    (the alternatives of Sec. 6.1.2; see schedule_width)."""
    xn, c, s, tree = _setup(points, theta, leaf_size, max_depth, far_order, local_theta, local_cluster)
    ptree = PaperTree(xn, paper_leaf_size, max_depth) if (tree is None and paper_theta > 0) else None
    n = xn.shape[0]
    mu = np.zeros((n, 3)) if mu0 is None else np.array(mu0, dtype=np.float64).reshape(n, 3) * (s * s)
    last = n_iter if last_iter is None else last_iter
    stats = np.zeros((max(last - first_iter + 1, 0), 4))
    ar = None if area is None else np.ascontiguousarray(np.asarray(area, np.float64) * (s * s))
    lib().or_iterate(tree._h if tree is not None else None, ptree._h if ptree is not None else None,
                     float(paper_theta), _p(xn), n, _p(mu), n_iter, first_iter,
                     last, float(w1), float(w2), rep_mode, rescale, _p(ar), int(use_grad),
                     int(use_wnnc), _schedule_code(schedule, w1, w2), _p(stats))
    return mu / (s * s), stats


SCHEDULES = {"linear": 0, "cosine": 1, "exponential": 2}


def _schedule_code(schedule, w1, w2) -> int:
    code = SCHEDULES.get(schedule, -1) if isinstance(schedule, str) else int(schedule)
    if code not in (0, 1, 2):
        raise ValueError(f"unknown width schedule {schedule!r}")
    if code == 2 and not (w1 > 0 and w2 > 0):
        raise ValueError("the exponential width schedule needs w1 > 0 and w2 > 0")
    return code


def schedule_width(i: int, n_iter: int, w1: float, w2: float, schedule="linear") -> float:
    """Width of iteration i of n_iter: linear w2 (1-t) + w1 t (Alg. 3), cosine
    w1 + (w2-w1)(1 + cos(pi t))/2 or exponential w2 (w1/w2)^t, t = (i-1)/(n-1)."""
    return lib().or_schedule_width2(i, n_iter, w1, w2, _schedule_code(schedule, w1, w2))


def knn(x, k: int = 16):
    """Exhaustive k nearest neighbours (excluding the point itself)."""
    x = _f64(x, (-1, 3))
    n = x.shape[0]
    idx = np.zeros((n, k), np.int64)
    d2 = np.zeros((n, k))
    lib().or_knn(_p(x), n, k, _p(idx), _p(d2))
    return idx, d2


# ---------------------------------------------------------------------------
# Metrics (Sec. 5.1.4)
# ---------------------------------------------------------------------------

def unit(v):
    v = np.asarray(v, dtype=np.float64)
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    return np.divide(v, nrm, out=np.zeros_like(v), where=nrm > 0)


def ae_pcd(n_gt, n_rec, valid=None):
    """AE_pcd = mean (1 - n_gt . n_rec) / 2 over valid points."""
    d = (unit(n_gt) * unit(n_rec)).sum(1)
    if valid is not None:
        d = d[valid]
    return float(np.mean((1.0 - d) / 2.0))


def p_co(n_gt, n_rec, valid=None):
    """P_co = fraction of points with n_gt . n_rec > 0."""
    d = (np.asarray(n_gt, np.float64) * np.asarray(n_rec, np.float64)).sum(1)
    if valid is not None:
        d = d[valid]
    return float(np.mean(d > 0))
