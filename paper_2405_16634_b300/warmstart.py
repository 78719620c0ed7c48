"""Learned warm start of the WNNC iteration (not in the paper).

A point-patch MLP maps each point's 16-NN patch (nearest first, offsets
divided by the 16th neighbour distance) to a normal direction.  It is trained
on the normals the method itself produces after its full 40 iterations on
seeded synthetic clouds.  At solve time:

1. build the tree, compute the patch features (``knn16``) and run the network;
2. run the first s iterations of the schedule from zero: the paper reports
   an overall correct orientation within the method's first few iterations
   (Sec. 5.3); this field gives the sign and the per-point lengths (areas);
3. start from the network's direction, with the sign and length of that
   field (``warm_init``);
4. run only the last k iterations of the width schedule.

The network is trained with the sign-free loss 1 - c^2 by default: a local
patch cannot tell inside from outside.

The plain 40-iteration solve stays the reference for accuracy.  Every numerical
step runs in the library's kernels; this module only drives them (batch
shuffling uses torch indexing).

    python -m paper_2405_16634_b300.warmstart [--train 200] [--heldout 20] [--out file.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

from . import Mlp, Tree, knn16, warm_init

N_ITER, THETA = 40, 0.5
# The training and held-out clouds carry sigma = 0.002 positional noise; the
# paper's widths for noisy scans (Sec. 5.2.6) are used for them.
W1, W2 = 0.01, 0.04


def _synth():
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if here not in sys.path:
        sys.path.insert(0, here)
    import synth
    return synth


def labelled_patches(points: torch.Tensor, keep: int | None, seed: int):
    """(features [m][48], unit labels [m][3]) of one cloud: the method's own
    converged normals as labels, a random subset of `keep` points."""
    t = Tree(points, theta=THETA)
    mu = t.iterate(n_iter=N_ITER, w1=W1, w2=W2)
    _, feat = knn16(t)
    lab = warm_init(mu, None, 1.0)                 # unit normals
    n = points.shape[0]
    if keep is not None and keep < n:
        g = torch.Generator(device="cpu").manual_seed(seed)
        sel = torch.randperm(n, generator=g)[:keep].to(points.device)
        feat, lab = feat[sel], lab[sel]
    t.close()
    return feat, lab


def make_dataset(seeds, keep: int = 20000, device="cuda"):
    synth = _synth()
    X, Y = [], []
    for s in seeds:
        spec = synth.random_cloud_spec(s)
        c = synth.union_cloud(**spec)
        f, l = labelled_patches(torch.from_numpy(c.points).to(device), keep, s)
        X.append(f)
        Y.append(l)
    return torch.cat(X), torch.cat(Y)


def train(mlp: Mlp, X: torch.Tensor, Y: torch.Tensor, epochs: int = 4, batch: int = 32768,
          lr: float = 1e-3, seed: int = 0):
    """Adam on shuffled mini-batches, learning rate on a per-epoch cosine
    decay from lr to lr/20; returns the mean loss per epoch."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    n = X.shape[0]
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        lr_e = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * ep / max(epochs, 1))))
        losses = []
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            losses.append(mlp.train_step(X[idx].contiguous(), Y[idx].contiguous(), lr_e))
        hist.append(float(torch.stack(losses).mean().item()))
    return hist


def plain_solve(points: torch.Tensor, n_iter: int = N_ITER, widths=(W1, W2)):
    t = Tree(points, theta=THETA)
    mu = t.iterate(n_iter=n_iter, w1=widths[0], w2=widths[1])
    t.close()
    return mu


def warm_solve(points: torch.Tensor, mlp: Mlp, k: int, s: int = 1, signed: bool = True, widths=(W1, W2)):
    """Iterations 1..s of the schedule from zero (sign and length reference),
    the network's directions with that sign and length, then the last k
    iterations of the schedule.  signed=False keeps the network's own sign."""
    w1, w2 = widths
    t = Tree(points, theta=THETA)
    _, feat = knn16(t)
    d = mlp.forward(feat)
    mu_s = t.iterate(n_iter=N_ITER, last_iter=s, w1=w1, w2=w2)
    mu0 = warm_init(d, mu_s, 0.0) if signed else warm_init(d, None, float(mu_s.norm(dim=1).mean()))
    first = max(s + 1, N_ITER - k + 1)
    mu = t.iterate(mu0, n_iter=N_ITER, first_iter=first, w1=w1, w2=w2) if k > 0 else mu0
    t.close()
    return mu


def _metrics(n_gt, mu, valid):
    ng = np.asarray(n_gt, np.float64)
    m = np.asarray(mu, np.float64)
    nm = np.linalg.norm(m, axis=1, keepdims=True)
    u = np.divide(m, nm, out=np.zeros_like(m), where=nm > 0)
    d = (ng * u).sum(1)[valid]
    return float(np.mean(d > 0)), float(np.mean((1 - d) / 2))


def _timed(fn, reps: int = 3):
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(reps):
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return out, best


def evaluate(mlp: Mlp, heldout_seeds, plain_iters=(2, 3, 5, 10, 20, 40),
             warm=((1, 0), (1, 1), (1, 2), (1, 4), (1, 9), (2, 1), (2, 3), (3, 2), (3, 7)),
             signed_net: bool = False):
    synth = _synth()
    rows = []
    for s in heldout_seeds:
        c = synth.union_cloud(**synth.random_cloud_spec(s))
        pts = torch.from_numpy(c.points).cuda()
        r = {"seed": s, "n": len(c.points)}
        for n in plain_iters:
            mu, dt = _timed(lambda: plain_solve(pts, n))
            r[f"plain{n}"] = _metrics(c.normals, mu.cpu().numpy(), c.valid) + (dt,)
        for s_, k in warm:
            mu, dt = _timed(lambda: warm_solve(pts, mlp, k, s_))
            r[f"warm_s{s_}_k{k}"] = _metrics(c.normals, mu.cpu().numpy(), c.valid) + (dt,)
        # stage times of the warm start: tree build, kNN + features, network
        t = Tree(pts, theta=THETA)
        _, r["t_tree_s"] = _timed(lambda: Tree(pts, theta=THETA).close())
        (_, feat), r["t_knn_s"] = _timed(lambda: knn16(t))
        _, r["t_mlp_s"] = _timed(lambda: mlp.forward(feat))
        t.close()
        if signed_net:      # the network's own sign, lengths from iteration 1
            mu, dt = _timed(lambda: warm_solve(pts, mlp, 9, 1, signed=False))
            r["warm_netsign_k9"] = _metrics(c.normals, mu.cpu().numpy(), c.valid) + (dt,)
        rows.append(r)
    keys = [k for k in rows[0] if k not in ("seed", "n") and not k.startswith("t_")]
    summary = {k: {"p_co": float(np.mean([r[k][0] for r in rows])),
                   "ae_pcd": float(np.mean([r[k][1] for r in rows])),
                   "time_s": float(np.mean([r[k][2] for r in rows]))} for k in keys}
    for k in ("n", "t_tree_s", "t_knn_s", "t_mlp_s"):
        summary[k] = float(np.mean([r[k] for r in rows]))
    return summary, rows


def evaluate_workload(mlp: Mlp, name: str = "union500k", seed: int = 3000, widths=(0.002, 0.016),
                      plain_iters=(5, 10, 20, 40), warm=((1, 4), (1, 9), (3, 2), (3, 7), (3, 17))):
    """Plain and warm solves of one benchmark workload (the 500,000-point
    union by default, with its widths), timed whole including the tree build;
    orientation accuracy against the primitives' normals (outliers excluded)."""
    synth = _synth()
    c = synth.config_cloud(name, seed=seed)
    pts = torch.from_numpy(c.points).cuda()
    out = {"workload": name, "n": len(c.points), "widths": list(widths)}
    for n in plain_iters:
        mu, dt = _timed(lambda: plain_solve(pts, n, widths))
        p_co, ae = _metrics(c.normals, mu.cpu().numpy(), c.valid)
        out[f"plain{n}"] = {"p_co": p_co, "ae_pcd": ae, "time_s": dt}
    for s_, k in warm:
        mu, dt = _timed(lambda: warm_solve(pts, mlp, k, s_, widths=widths))
        p_co, ae = _metrics(c.normals, mu.cpu().numpy(), c.valid)
        out[f"warm_s{s_}_k{k}"] = {"p_co": p_co, "ae_pcd": ae, "time_s": dt}
    t = Tree(pts, theta=THETA)
    (_, feat), out["t_knn_s"] = _timed(lambda: knn16(t))
    _, out["t_mlp_s"] = _timed(lambda: mlp.forward(feat))
    t.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--heldout", type=int, default=20)
    ap.add_argument("--keep", type=int, default=20000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--loss", type=int, default=1, help="0: 1 - c, 1: 1 - c^2 (sign-free)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--workload", default=None,
                    help="also compare plain and warm solves on this benchmark cloud (e.g. union500k)")
    a = ap.parse_args(argv)
    synth = _synth()
    t0 = time.perf_counter()
    X, Y = make_dataset([4000 + k for k in range(a.train)], keep=a.keep)
    t_data = time.perf_counter() - t0
    mlp = Mlp(max_batch=32768, params=torch.from_numpy(synth.mlp_init(1)))
    mlp.set_loss(a.loss)
    t0 = time.perf_counter()
    hist = train(mlp, X, Y, epochs=a.epochs)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    summary, rows = evaluate(mlp, [4500 + k for k in range(a.heldout)], signed_net=a.loss == 0)
    res = {"loss_mode": a.loss, "train_clouds": a.train, "train_samples": int(X.shape[0]), "epochs": a.epochs,
           "loss_per_epoch": hist, "t_data_s": t_data, "t_train_s": t_train,
           "heldout": a.heldout, "summary": summary, "per_cloud": rows}
    if a.workload:
        res["workload"] = evaluate_workload(mlp, a.workload)
        print(json.dumps({"workload": res["workload"]}, indent=1))
    txt = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    print(json.dumps({"summary": summary, "loss_per_epoch": hist, "t_data_s": t_data,
                      "t_train_s": t_train, "train_samples": int(X.shape[0])}, indent=1))
    return mlp


if __name__ == "__main__":
    main()
