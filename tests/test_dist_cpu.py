"""The multi-process path of bench.py on CPU: two ranks over gloo.

Every rank solves its own cloud (replicas, no exchange on the data path);
the host logic that joins the ranks is the rendezvous, the max of the timed
region over ranks, and the whole-job rate.  Nothing here uses a GPU.
"""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, w, r, local = bench.dist_setup(backend="gloo")
    ms = 100.0 + 50.0 * r                      # rank 1 is the slower one
    mx = bench.max_over_ranks(dist, ms)
    q.put((r, w, local, mx, bench.whole_job_rate(w, bench.N_ITER, 3, mx)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert [r[2] for r in res] == [0, 1]
    assert all(r[3] == 150.0 for r in res)
    # two replicas of 3 steps x 40 iterations in the slowest rank's 150 ms
    assert all(abs(r[4] - 2 * 40 * 3 / 0.150) < 1e-9 for r in res)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    saved = {k: os.environ.pop(k, None) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    try:
        dist, w, r, local = bench.dist_setup()
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v
    assert (dist, w, r, local) == (None, 1, 0, 0)
    assert bench.max_over_ranks(None, 12.5) == 12.5
    assert bench.whole_job_rate(1, 40, 10, 1000.0) == 400.0
