"""Seeded synthetic point clouds shaped like the paper's workloads.

This module is shared by the FP64 oracle tests and the CUDA path's tests and
benchmark.  It only draws inputs (points, ground-truth normals, initial normal
fields, network weights); it holds none of the method's arithmetic.

The paper evaluates on scanned/CAD models (Sec. 5) that are not available
here, so every workload is a seeded union of analytic primitives sampled
area-uniformly, with optional positional noise, density modulation and
outliers:

* ``sphere``            -- uniform points on a sphere (normalised Gaussians).
* ``fibonacci_sphere``  -- deterministic near-uniform sphere points.
* ``icosphere``         -- vertices of a subdivided icosahedron (the unit-sphere
                           model of the area-convergence table, Sec. 6.1.2).
* ``union_cloud``       -- union of tori and ellipsoids; samples inside another
                           primitive are dropped, so the cloud samples the
                           boundary of the union (a closed surface) and the
                           ground-truth normal is the owning primitive's
                           outward normal.

All generators use ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Cloud", "sphere", "fibonacci_sphere", "icosphere", "random_unit_vectors",
    "union_cloud", "config_cloud", "ball_queries", "CONFIGS",
]


@dataclass
class Cloud:
    """A synthetic point cloud.

    points   (N,3) float32  positions in the generator's units (unit cube)
    normals  (N,3) float32  ground-truth outward unit normals (NaN rows for outliers)
    valid    (N,)  bool     False for outliers (no ground truth)
    area     float          estimated total surface area of the sampled surface
    """
    points: np.ndarray
    normals: np.ndarray
    valid: np.ndarray
    area: float


def random_unit_vectors(n: int, seed: int) -> np.ndarray:
    """n unit vectors uniform on S^2 (normalised Gaussians), float64."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def sphere(n: int, seed: int, radius: float = 1.0) -> Cloud:
    """n uniform points on a sphere of the given radius centred at 0."""
    u = random_unit_vectors(n, seed)
    pts = (radius * u).astype(np.float32)
    return Cloud(pts, u.astype(np.float32), np.ones(n, bool), 4.0 * math.pi * radius ** 2)


def fibonacci_sphere(n: int, radius: float = 1.0) -> Cloud:
    """Deterministic golden-angle spiral points on a sphere (near-uniform)."""
    k = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * k / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * math.pi * (3.0 - math.sqrt(5.0))
    u = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)
    pts = (radius * u).astype(np.float32)
    return Cloud(pts, u.astype(np.float32), np.ones(n, bool), 4.0 * math.pi * radius ** 2)


def icosphere(level: int) -> Cloud:
    """Vertices of an icosahedron subdivided ``level`` times, projected to the unit sphere.

    Each subdivision splits every triangle into four; level 7 gives 163,842
    vertices, the unit-sphere model of the paper's area-convergence table.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = np.array(verts, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(faces, dtype=np.int64)
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        ekey = e[:, 0] * (nv + 1) + e[:, 1]
        uniq, inv = np.unique(ekey, return_inverse=True)
        a = uniq // (nv + 1)
        b = uniq % (nv + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = inv.reshape(3, -1) + nv          # midpoints of edges (01, 12, 20) per face
        m01, m12, m20 = m[0], m[1], m[2]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
        v = np.concatenate([v, mid], axis=0)
    return Cloud(v.astype(np.float32), v.astype(np.float32), np.ones(v.shape[0], bool), 4.0 * math.pi)


# ----------------------------------------------------------------------------
# Unions of tori and ellipsoids
# ----------------------------------------------------------------------------

def _rand_rotation(rng) -> np.ndarray:
    """Uniform random rotation from a uniform unit quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


class _Torus:
    def __init__(self, R, r, rot, c):
        self.R, self.r, self.rot, self.c = R, r, rot, c

    def bound(self):
        return self.R + self.r

    def area(self):
        return 4.0 * math.pi ** 2 * self.R * self.r

    def sample(self, rng, m):
        out_p, out_n, need = [], [], m
        while need > 0:
            k = max(2 * need, 64)
            u = rng.uniform(0, 2 * math.pi, k)
            v = rng.uniform(0, 2 * math.pi, k)
            keep = rng.uniform(0, 1, k) < (self.R + self.r * np.cos(v)) / (self.R + self.r)
            u, v = u[keep][:need], v[keep][:need]
            rho = self.R + self.r * np.cos(v)
            p = np.stack([rho * np.cos(u), rho * np.sin(u), self.r * np.sin(v)], 1)
            n = np.stack([np.cos(v) * np.cos(u), np.cos(v) * np.sin(u), np.sin(v)], 1)
            out_p.append(p)
            out_n.append(n)
            need -= p.shape[0]
        p = np.concatenate(out_p) @ self.rot.T + self.c
        n = np.concatenate(out_n) @ self.rot.T
        return p, n

    def inside(self, x):
        y = (x - self.c) @ self.rot
        q = np.sqrt(y[:, 0] ** 2 + y[:, 1] ** 2) - self.R
        return q * q + y[:, 2] ** 2 < self.r * self.r


class _Ellipsoid:
    def __init__(self, abc, rot, c):
        self.abc, self.rot, self.c = np.asarray(abc, float), rot, c

    def bound(self):
        return float(self.abc.max())

    def area(self):
        a, b, c = self.abc
        p = 1.6075  # Knud Thomsen's approximation
        return 4 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)

    def sample(self, rng, m):
        a, b, c = self.abc
        gmax = max(b * c, a * c, a * b)
        out_p, out_n, need = [], [], m
        while need > 0:
            k = max(2 * need, 64)
            u = rng.standard_normal((k, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            g = a * b * c * np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2 + (u[:, 2] / c) ** 2)
            u = u[rng.uniform(0, 1, k) < g / gmax][:need]
            p = u * self.abc
            n = p / self.abc ** 2
            n /= np.linalg.norm(n, axis=1, keepdims=True)
            out_p.append(p)
            out_n.append(n)
            need -= p.shape[0]
        p = np.concatenate(out_p) @ self.rot.T + self.c
        n = np.concatenate(out_n) @ self.rot.T
        return p, n

    def inside(self, x):
        y = (x - self.c) @ self.rot
        return ((y / self.abc) ** 2).sum(1) < 1.0

    def extent_along(self, d):
        """Distance from the centre to the surface along unit direction d (world frame)."""
        y = self.rot.T @ d
        return 1.0 / math.sqrt(float(((y / self.abc) ** 2).sum()))


def _center(rng, bound):
    lo, hi = min(bound, 0.5), max(1.0 - bound, 0.5)
    return rng.uniform(lo, hi, 3)


def _density_field(rng, n_modes=8, kmax=4 * math.pi):
    """Seeded sum of random Fourier modes, min-max normalised on the unit cube."""
    ks = []
    while len(ks) < n_modes:
        k = rng.uniform(-kmax, kmax, 3)
        if np.linalg.norm(k) <= kmax:
            ks.append(k)
    ks = np.array(ks)
    ph = rng.uniform(0, 2 * math.pi, n_modes)
    amp = rng.uniform(0.5, 1.0, n_modes)
    grid = rng.uniform(0, 1, (20000, 3))
    raw = np.cos(grid @ ks.T + ph) @ amp
    lo, hi = raw.min(), raw.max()

    def f(x):
        return np.clip((np.cos(x @ ks.T + ph) @ amp - lo) / (hi - lo), 0.0, 1.0)
    return f


def union_cloud(n: int, seed: int, n_tori: int = 2, n_ellipsoids: int = 2,
                noise: float = 0.0, density_mod: bool = False,
                outlier_frac: float = 0.0, torus_R=(0.3, 0.5), torus_r=(0.08, 0.15),
                semi_axes=(0.2, 0.5), thin_torus_r: float | None = None,
                touching_pairs: int = 0, pair_gap: float = 0.005) -> Cloud:
    """Area-uniform samples of the boundary of a union of seeded tori and ellipsoids.

    Samples that fall inside another primitive are dropped and drawing repeats
    until exactly ``n - n_outliers`` surface points remain.  ``density_mod``
    thins samples with acceptance 10**f(x)/10 for a seeded low-frequency field
    f in [0,1] (a 10x density contrast).  ``outlier_frac`` adds uniform points
    in the bounding box (valid=False).  ``thin_torus_r`` makes half of the tori
    thin (minor radius fixed); ``touching_pairs`` adds ellipsoid pairs whose
    surfaces are ``pair_gap`` apart along the line of centres.
    """
    rng = np.random.default_rng(seed)
    prims = []
    for t in range(n_tori):
        R = rng.uniform(*torus_R)
        r = rng.uniform(*torus_r)
        if thin_torus_r is not None and t % 2 == 0:
            r = thin_torus_r
        prims.append(_Torus(R, r, _rand_rotation(rng), None))
        prims[-1].c = _center(rng, prims[-1].bound())
    for _ in range(n_ellipsoids):
        e = _Ellipsoid(rng.uniform(*semi_axes, 3), _rand_rotation(rng), None)
        e.c = _center(rng, e.bound())
        prims.append(e)
    for _ in range(touching_pairs):
        e1 = _Ellipsoid(rng.uniform(semi_axes[0], 0.5 * (semi_axes[0] + semi_axes[1]), 3),
                        _rand_rotation(rng), None)
        e1.c = _center(rng, 2 * e1.bound())
        e2 = _Ellipsoid(rng.uniform(semi_axes[0], 0.5 * (semi_axes[0] + semi_axes[1]), 3),
                        _rand_rotation(rng), None)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        # bisection on the centre offset so that the surfaces are pair_gap apart
        # along the line of centres
        lo, hi = 0.0, 4.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            gap = mid - e1.extent_along(d) - e2.extent_along(-d)
            lo, hi = (mid, hi) if gap < pair_gap else (lo, mid)
        e2.c = e1.c + d * 0.5 * (lo + hi)
        prims += [e1, e2]

    n_out = int(round(outlier_frac * n))
    n_surf = n - n_out
    areas = np.array([p.area() for p in prims])
    dens = _density_field(rng) if density_mod else None

    kept_p, kept_n, total, drawn, kept_cnt = [], [], 0, 0, 0
    while total < n_surf:
        need = n_surf - total
        draw = max(int(need * 1.3), 256)
        counts = rng.multinomial(draw, areas / areas.sum())
        for pi, (prim, m) in enumerate(zip(prims, counts)):
            if m == 0:
                continue
            p, nn = prim.sample(rng, m)
            keep = np.ones(m, bool)
            for qi, other in enumerate(prims):
                if qi != pi:
                    keep &= ~other.inside(p)
            drawn += m
            kept_cnt += int(keep.sum())
            if dens is not None:
                keep &= rng.uniform(0, 1, m) < 10.0 ** dens(p) / 10.0
            kept_p.append(p[keep])
            kept_n.append(nn[keep])
            total += int(keep.sum())
    P = np.concatenate(kept_p)
    Nn = np.concatenate(kept_n)
    sel = rng.permutation(P.shape[0])[:n_surf]
    P, Nn = P[sel], Nn[sel]
    if noise > 0:
        P = P + rng.normal(0.0, noise, P.shape)
    area = float(areas.sum() * kept_cnt / max(drawn, 1))
    valid = np.ones(n, bool)
    if n_out > 0:
        lo, hi = P.min(0), P.max(0)
        O = rng.uniform(lo, hi, (n_out, 3))
        P = np.concatenate([P, O])
        Nn = np.concatenate([Nn, np.full((n_out, 3), np.nan)])
        valid[n_surf:] = False
        perm = rng.permutation(n)
        P, Nn, valid = P[perm], Nn[perm], valid[perm]
    return Cloud(P.astype(np.float32), Nn.astype(np.float32), valid, area)


def ball_queries(m: int, seed: int, center, radius: float) -> np.ndarray:
    """m query points uniform in a ball (for off-surface winding-number checks)."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    rad = radius * rng.uniform(0, 1, m) ** (1.0 / 3.0)
    return (np.asarray(center, float) + u * rad[:, None]).astype(np.float32)


# The workloads (sizes and structure) of the five benchmark/parity configurations.
CONFIGS = {
    "sphere2k": dict(kind="sphere", n=2000, seed=1000),
    "union50k": dict(kind="union", n=50_000, seed=2000, n_tori=2, n_ellipsoids=2, noise=0.002),
    "union500k": dict(kind="union", n=500_000, seed=3000, n_tori=6, n_ellipsoids=6,
                      density_mod=True, outlier_frac=0.01),
    "union2m": dict(kind="union", n=2_000_000, seed=5000, n_tori=10, n_ellipsoids=10,
                    thin_torus_r=0.01, touching_pairs=2, noise=0.001),
}


def config_cloud(name: str, n: int | None = None, seed: int | None = None) -> Cloud:
    """Cloud of a named configuration (optionally resized / reseeded)."""
    cfg = dict(CONFIGS[name])
    kind = cfg.pop("kind")
    if n is not None:
        cfg["n"] = n
    if seed is not None:
        cfg["seed"] = seed
    if kind == "sphere":
        return sphere(cfg["n"], cfg["seed"])
    return union_cloud(**cfg)


def random_cloud_spec(seed: int) -> dict:
    """Parameters of one warm-start training/held-out cloud: 3-10 primitives,
    20k-200k points (log-uniform)."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(3, 11))
    nt = int(rng.integers(1, k))
    n = int(round(math.exp(rng.uniform(math.log(20_000), math.log(200_000)))))
    return dict(n=n, seed=seed, n_tori=nt, n_ellipsoids=k - nt, noise=0.002)


def init_normals(n: int, seed: int, area_per_point: float) -> np.ndarray:
    """Random unit normals (unoriented) times an equal area weight, float32 (N,3)."""
    return (random_unit_vectors(n, seed) * area_per_point).astype(np.float32)


def mlp_init(seed: int) -> np.ndarray:
    """Initial parameters of the 48-128-128-128-3 warm-start MLP (He-uniform
    weights, zero biases), flat float32 in the layout W1, b1, W2, b2, W3, b3,
    W4, b4."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((128, 48), (128, 128), (128, 128), (3, 128)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)
