"""The winding-number field on a regular grid.

Once the iteration has oriented the points, the discretised winding number
F(y; mu) = sum_j grad Phi(y - x_j) . mu_j (Eq. 5, the discretisation of the
Gauss formula, Thm. 1) is an indicator of the enclosed volume: about 1 inside,
0 outside and 1/2 on the surface.  Surface reconstruction evaluates it in
space and contours it; this module evaluates it at the nodes of a grid around
the cloud with the library's query treecode (``Tree.eval_at``, the same far /
near decisions of Alg. 4 for groups of query points).  Contouring is not done
here.

    python -m paper_2405_16634_b300.wnf [--res 128] [--workload union500k]

times a res^3 grid on the oriented benchmark cloud and prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import torch

from . import Tree

N_ITER, THETA, W1, W2 = 40, 0.5, 0.002, 0.016


def grid_box(points: torch.Tensor, pad: float = 0.05):
    """Lower corner and side of the cube grid around the points: the bounding
    box's largest side plus `pad` of it on each side, centred on the box."""
    lo = points.min(dim=0).values
    hi = points.max(dim=0).values
    side = float((hi - lo).max()) * (1.0 + 2.0 * pad)
    centre = 0.5 * (lo + hi)
    return centre - 0.5 * side, side


def grid_points(lo: torch.Tensor, side: float, res: int, k0: int = 0, k1: int | None = None):
    """Nodes k0 .. k1-1 of a res^3 grid (x slowest, z fastest) as float32 [m][3]."""
    k1 = res ** 3 if k1 is None else k1
    k = torch.arange(k0, k1, device=lo.device, dtype=torch.int64)
    h = side / (res - 1)
    ijk = torch.stack([k // (res * res), (k // res) % res, k % res], dim=1).to(torch.float32)
    return (lo.to(torch.float32) + h * ijk).contiguous()


def grid_field(tree: Tree, mu: torch.Tensor, lo: torch.Tensor, side: float, res: int, w: float = W1,
               chunk: int = 1 << 21) -> torch.Tensor:
    """F(y; mu) at the res^3 nodes of the cube [lo, lo + side]^3, as a
    [res, res, res] float32 tensor indexed (x, y, z).  Queries go to the
    treecode `chunk` at a time, which bounds the memory of their lists.  The
    treecode groups the queries of one call (32 in Morton order), so the far /
    near decisions, and the values within the treecode's theta-dependent
    error, depend on the chunking."""
    m = res ** 3
    out = torch.empty(m, device=mu.device, dtype=torch.float32)
    for k0 in range(0, m, chunk):
        k1 = min(m, k0 + chunk)
        out[k0:k1] = tree.eval_at(mu, grid_points(lo, side, res, k0, k1), w)
    return out.view(res, res, res)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--res", type=int, default=128)
    ap.add_argument("--workload", default="union500k")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if here not in sys.path:
        sys.path.insert(0, here)
    import synth
    c = synth.config_cloud(a.workload, seed=3000)
    pts = torch.from_numpy(c.points).cuda()
    tree = Tree(pts, theta=THETA)
    mu = tree.iterate(n_iter=N_ITER, w1=W1, w2=W2)
    lo, side = grid_box(pts)
    F = grid_field(tree, mu, lo, side, a.res)       # warm-up (pool, lists)
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(a.reps):
        t0 = time.perf_counter()
        F = grid_field(tree, mu, lo, side, a.res)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    m = a.res ** 3
    print(json.dumps({"workload": a.workload, "n_points": len(c.points), "res": a.res, "queries": m,
                      "seconds": best, "queries_per_s": m / best,
                      "inside_frac": float((F > 0.5).float().mean()),
                      "f_min": float(F.min()), "f_max": float(F.max())}))


if __name__ == "__main__":
    main()
