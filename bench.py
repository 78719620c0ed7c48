"""Benchmark: the WNNC normal-orientation solve on the 500,000-point workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wnnc|reference]

A step is one pass of the whole hot path on one synthetic cloud: tree build
(normalisation, Morton sort, octree, node data, interaction lists) and the 40
iterations of Alg. 3 (moments, A, A^T, grad step, G + rescale).  Inputs are
resident in HBM when the timed region starts; L2 is flushed (a 256 MiB write)
before every step.  `value` is whole-job WNNC iterations/s.  The JSON line also
reports interactions/s, the fraction of FP32 peak, the roofline of the
dominant kernel (the fused A+G treecode gather, timed live with the library's
CUDA-event profiler on its launch stream), an end-to-end number through one C-ABI call
with host buffers (`wnnc_orient`: pinned host points in, host field out, copies inside),
the CPU oracle as a baseline, and SM clocks sampled during the timed region.

After the timed region the line adds `variants`: one or two whole solves of the paper's own
treecode as printed (per-target Alg. 4, leaf size 1) and of the first-order far field on the
same cloud, for comparison (not part of `value`; `--no-variants` skips them).

`--impl reference` times the FP64 CPU oracle on the same workload: each step
is one full iteration of Alg. 3 on the whole cloud (the oracle builds its own
tree inside the call).  With N > 1 (torchrun) every rank solves its own cloud
(replicas: the problems are independent and there is no exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ITER = 40
W1, W2 = 0.002, 0.016
THETA = 0.5
WORKLOADS = {
    "union500k": ("union500k: 500,000 points on a union of 6 tori + 6 ellipsoids, 10x density "
                  "modulation, 1% outliers; theta=0.5 (c=2), leaf_size=8, group slack 3, depth 15; 40 iterations "
                  "w2=0.016 -> w1=0.002"),
    "union50k": ("union50k: 50,000 points on a union of 2 tori + 2 ellipsoids, noise 0.002; "
                 "theta=0.5, leaf_size=8, group slack 3, depth 15; 40 iterations w2=0.016 -> w1=0.002 "
                 "(small case for profiling)"),
    "union2m": ("union2m: 2,000,000 points on 24 primitives incl. thin tori (r=0.01) and "
                "near-touching ellipsoid pairs (gap 0.005), noise 0.001; theta=0.5; 40 iterations"),
}
CONFIG_NAME = "union500k"
WORKLOAD = WORKLOADS[CONFIG_NAME]
# algorithmic FP32 flops per pair term (FMA = 2, rsqrt = 1; the cut-off select is not counted):
# A 18, A^T 18, G 31; A and G together 33 (they share d, r^2, rsqrt, r^-3 and d.mu: 16)
FLOPS_A, FLOPS_AT, FLOPS_G, FLOPS_AG = 18, 18, 31, 33
FLOPS_ITER = 2 * FLOPS_AG + FLOPS_AT               # A+G(mu), A^T(s), A+G(r) per iteration
# per far entry expanded about its group's centre (local_theta > 0): the value
# of A and G and the Jacobian of G at the centre (A+G), the transposed
# expansion from the group's sums (A^T); an FMA counts two
FLOPS_LOCAL_AG, FLOPS_LOCAL_AT = 88, 41
FLOPS_LOCAL_ITER = 2 * FLOPS_LOCAL_AG + FLOPS_LOCAL_AT
LOCAL_THETA = 0.5    # local expansions of far nodes about target groups (0 = off)
LOCAL_CLUSTER = 4    # second expansion level: clusters of that many groups (0 = none)
PAPER_RTX3090_ITER_PER_S_500K = 40 / 31.63          # context only (different model and GPU)
# Variants solved once each after the timed region (name, tree parameters, timed solves):
# the paper's own treecode as printed (Alg. 4 per target and per call, leaf size 1,
# |nu|-weighted representatives), and the first-order far field at two opening angles.
# Also the default method at theta = 0.8, where its errors against the direct sums (A 2.2e-2,
# grad F 5.8e-3, A^T 3.6e-2 at 500k) are still below those of the paper's own treecode at the
# paper's theta = 0.5 (2.4e-2, 4.6e-2, 1.5e-1): the speed at the paper's accuracy.
VARIANTS = [
    ("paper_alg4_per_target_leaf1_theta0.5", dict(theta=0.5, leaf_size=1, rep_mode=0, criterion=1), 1),
    ("pairwise_far_field_theta0.5", dict(theta=0.5, local_theta=0.0), 3),
    ("group_lists_theta0.8", dict(theta=0.8), 3),
    ("local_expansions_one_level_theta0.5", dict(theta=0.5, local_theta=0.5), 3),
    ("local_expansions_theta0.8", dict(theta=0.8, local_theta=0.5, local_cluster=4), 3),
    ("first_order_far_field_theta0.5", dict(theta=0.5, far_order=1), 2),
    ("first_order_far_field_theta0.8", dict(theta=0.8, far_order=1), 2),
]
# DRAM bytes (read + write) of one launch of the fused A+G kernel on union500k, from ncu
# (one ncu capture of that kernel on this workload), with and without the local
# expansions (their far lists differ, and with them the gather leaves its sums to a
# separate pass); None once the kernel has changed.
AG_TRAFFIC_BYTES = {0.5: 49.012224e6 + 0.121344e6, 0.0: 107.725568e6 + 4.595968e6}


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: power above the midpoint of the observed range
        thr = 0.5 * (min(power) + max(power))
        loaded = [s for s, p in zip(sm, power) if p >= thr] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "samples": len(sm),
                "samples_under_load": len(loaded), "power_w_max": max(power),
                "reasons": sorted(reasons)}


def dist_setup(backend: str | None = None):
    """(dist or None, world size, rank, local rank) from the launcher's
    environment; the process group uses NCCL where CUDA is present, else gloo."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, world, rank, local
    return None, 1, 0, 0


def max_over_ranks(dist, x: float) -> float:
    """The largest x over all ranks (the job ends with its slowest rank)."""
    if dist is None:
        return x
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, iters_per_step: int, steps: int, ms: float) -> float:
    """Iterations/s of the whole job: every rank solves its own cloud in the
    same (slowest-rank) time."""
    return world * iters_per_step * steps / (ms / 1e3)


def make_cloud(rank: int):
    import synth
    return synth.config_cloud(CONFIG_NAME, seed=3000 + rank)


def cpu_baseline_oracle(points) -> dict:
    """The FP64 oracle (as it stands) on one full iteration of the same cloud."""
    import oracle
    t0 = time.perf_counter()
    oracle.iterate(points, n_iter=N_ITER, first_iter=1, last_iter=1, w1=W1, w2=W2, theta=THETA)
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": "iter/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"iteration 1 of 40 (w = w2) on the full {len(points)}-point cloud, "
                      f"FP64 direct/treecode oracle incl. its own tree build; {dt:.1f} s"}


def run_reference(args):
    dist, world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    c = make_cloud(0)
    oracle.build()
    for _ in range(args.warmup):
        oracle.iterate(c.points, n_iter=N_ITER, first_iter=1, last_iter=1, w1=W1, w2=W2, theta=THETA)
    t0 = time.perf_counter()
    for k in range(args.steps):
        it = 1 + (k % N_ITER)
        oracle.iterate(c.points, n_iter=N_ITER, first_iter=it, last_iter=it, w1=W1, w2=W2, theta=THETA)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": "WNNC iterations/s (500k points)", "value": value,
        "unit": "iter/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "each step = one full iteration of Alg. 3 on the whole cloud "
                                   "(FP64 oracle, its own tree build included)"},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    import paper_2405_16634_b300 as W

    dist, world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W.build_if_needed()
    W.lib()
    c = make_cloud(rank)
    n = len(c.points)
    pts = torch.from_numpy(c.points).to(dev)
    mu = torch.empty(n, 3, device=dev, dtype=torch.float32)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream(dev)

    def step(prof: dict | None, classes=None):
        flush.zero_()
        t = W.Tree(pts, theta=THETA, local_theta=LOCAL_THETA, local_cluster=LOCAL_CLUSTER)
        if prof is not None:
            t.profile(True, classes=classes)
        t.iterate(n_iter=N_ITER, w1=W1, w2=W2, out=mu)
        if prof is not None:
            for k, (cnt, ms) in t.profile_read().items():
                a, b = prof.get(k, (0, 0.0))
                prof[k] = (a + cnt, b + ms)
        stats = t.stats() + tuple(a + b for a, b in zip(t.local_stats(), t.cluster_stats()))
        t.close()
        return stats

    for _ in range(args.warmup):
        step(None)
    torch.cuda.synchronize(dev)

    # T_pre / T_main split on one untimed step (CUDA events)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    t = W.Tree(pts, theta=THETA, local_theta=LOCAL_THETA, local_cluster=LOCAL_CLUSTER)
    e1.record(stream)
    t.iterate(n_iter=N_ITER, w1=W1, w2=W2, out=mu)
    e2.record(stream)
    torch.cuda.synchronize(dev)
    t_pre_ms, t_main_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    info = t.info()
    t.close()
    # kernel-time shares of all classes, from one untimed step (every class
    # recorded: two events per launch group)
    share_prof: dict = {}
    step(share_prof)
    torch.cuda.synchronize(dev)

    # ---- timed region (events only around the fused A+G launches, whose
    # live average duration gives the roofline) ----
    prof: dict = {}
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    launches0 = W.kernel_launches()
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev_a.record(stream)
    for _ in range(args.steps):
        far_pairs, near_pairs, local_entries, local_pairs = step(prof, classes=["AG"])
    ev_b.record(stream)
    torch.cuda.synchronize(dev)
    launches = W.kernel_launches() - launches0
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(dist, ev_a.elapsed_time(ev_b))
    ms_per_step = ms / args.steps
    value = whole_job_rate(world, N_ITER, args.steps, ms)

    # ---- end to end through one C-ABI call with host buffers (wnnc_orient:
    # host points in, host field out; the copies, the tree build and the 40
    # iterations inside the call), pinned host memory ----
    e2e = None
    if not args.no_e2e:
        h_pts = torch.from_numpy(c.points).pin_memory()
        h_mu = torch.empty(n, 3, dtype=torch.float32).pin_memory()
        W.orient(h_pts, out=h_mu, theta=THETA, n_iter=N_ITER, w1=W1, w2=W2, local_theta=LOCAL_THETA,
                 local_cluster=LOCAL_CLUSTER)  # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            W.orient(h_pts, out=h_mu, theta=THETA, n_iter=N_ITER, w1=W1, w2=W2, local_theta=LOCAL_THETA,
                     local_cluster=LOCAL_CLUSTER)
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(dist, time.perf_counter() - t0)
        e2e = {"value": whole_job_rate(world, N_ITER, args.steps, 1e3 * dt), "unit": "iter/s",
               "h2d_bytes_per_step": int(h_pts.numel() * 4),
               "d2h_bytes_per_step": int(h_mu.numel() * 4),
               "call": "wnnc_orient (C ABI, host buffers in and out)"}

    # ---- variants of the method on the same cloud (after the timed region;
    # not part of `value`): the paper's own treecode as printed, and the
    # first-order far field ----
    variants = None
    if not args.no_variants and rank == 0:
        variants = {}
        for name, kw, steps in VARIANTS:
            vt = []
            for k in range(1 + steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                tv = W.Tree(pts, **kw)
                tv.iterate(n_iter=N_ITER, w1=W1, w2=W2, out=mu)
                b.record(stream)
                torch.cuda.synchronize(dev)
                if k > 0:
                    vt.append(a.elapsed_time(b))
                vf, vn = tv.stats()
                tv.close()
            ms_v = sum(vt) / len(vt)
            variants[name] = {"tree": kw, "iter_per_s": N_ITER / (ms_v / 1e3), "ms_per_solve": ms_v,
                              "steps": steps, "far_pairs_group_lists": vf, "near_pairs_group_lists": vn}

    if rank != 0:
        return 0

    inter_per_op = far_pairs + near_pairs
    inter_per_iter = 4 * inter_per_op
    props = torch.cuda.get_device_properties(dev)
    fp32_measured = W.probe_fp32(dev)
    peaks = read_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    peak = fp32_peak_tflops(props.multi_processor_count, max_mhz)
    flops_iter = FLOPS_ITER * inter_per_op + FLOPS_LOCAL_ITER * local_entries
    flops_per_s = flops_iter * N_ITER * args.steps * world / (ms / 1e3)
    g_launch, g_ms = prof.get("AG", (0, 0.0))
    g_avg_ms = g_ms / max(g_launch, 1)
    flops_ag = FLOPS_AG * inter_per_op        # the gather's pair terms (the expanded entries run apart)
    g_achieved = flops_ag / (g_avg_ms / 1e3) / 1e12
    shares = {k: round(v[1] / max(sum(x[1] for x in share_prof.values()), 1e-9), 4)
              for k, v in share_prof.items()}
    line = {
        "metric": "WNNC iterations/s (500k points)" if CONFIG_NAME == "union500k"
                  else f"WNNC iterations/s ({CONFIG_NAME})",
        "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_points": n, "iterations_per_step": N_ITER,
                   "theta": THETA, "local_theta": LOCAL_THETA, "local_cluster": LOCAL_CLUSTER,
                   "l2": "flushed before every step (256 MiB write, inside the timed region)",
                   "step": "tree build + 40 iterations"},
        "interactions_per_s": inter_per_iter * N_ITER * args.steps * world / (ms / 1e3),
        "interactions_per_iteration": inter_per_iter,
        "local_entries_per_operator": local_entries,
        "local_pairs_per_operator": local_pairs,
        "fp32_tflops": flops_per_s / 1e12,
        "fp32_peak_frac": flops_per_s / 1e12 / peak,
        "t_pre_ms": t_pre_ms, "t_main_ms": t_main_ms,
        "iter_per_s_main_only": N_ITER / (t_main_ms / 1e3),
        "tree": info,
        "roofline": {"kernel": "k_gather<AG, ...> (fused treecode sums of A and G on one field)",
                     "bound": "alu", "achieved": g_achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": g_achieved / peak,
                     # dram__bytes_read.sum + dram__bytes_write.sum of one launch of this
                     # kernel (one ncu capture on this workload); only valid for
                     # the default workload and the kernel version that was profiled
                     "traffic": AG_TRAFFIC_BYTES.get(LOCAL_THETA) if CONFIG_NAME == "union500k" else None,
                     "traffic_unit": "bytes",
                     "peak_source": f"FP32 FMA: {props.multi_processor_count} SMs x 128 lanes x 2 "
                                    f"x {max_mhz:.0f} MHz (max SM clock of MEASURED_PEAKS.json)",
                     "peak_measured_fma_stream": fp32_measured,
                     "frac_of_measured": g_achieved / fp32_measured,
                     "avg_launch_ms": g_avg_ms, "launches": g_launch,
                     "flops_per_launch": flops_ag},
        "kernel_time_share": shares,
        "gpu_launches": launches,
        "clocks": clocks,
        "paper_context": {"rtx3090_iter_per_s_500k": PAPER_RTX3090_ITER_PER_S_500K},
    }
    if e2e:
        line["e2e"] = e2e
    if variants:
        line["variants"] = variants
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_oracle(c.points)
    print(json.dumps(line), flush=True)
    return 0


def main():
    global CONFIG_NAME, WORKLOAD, LOCAL_THETA, LOCAL_CLUSTER
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wnnc", choices=["wnnc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the solves of the method's variants after the timed region")
    ap.add_argument("--config", default="union500k", choices=sorted(WORKLOADS),
                    help="workload (the default is the one the metric is quoted on)")
    ap.add_argument("--local-theta", type=float, default=LOCAL_THETA,
                    help="local expansions of far nodes about target groups (0 = off)")
    ap.add_argument("--local-cluster", type=int, default=LOCAL_CLUSTER,
                    help="second expansion level: clusters of that many groups (0 = none)")
    args = ap.parse_args()
    CONFIG_NAME, WORKLOAD = args.config, WORKLOADS[args.config]
    LOCAL_THETA = args.local_theta
    LOCAL_CLUSTER = args.local_cluster
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
