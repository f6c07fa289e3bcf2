"""The N > 1 path on the CPU: two gloo ranks take disjoint parameter bands
(weak scaling, no collective on the data path) and the bench's whole-job
reduction gives the sum of steps over the maximum time."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench
import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.rank_band(W.duffing_rkck(8, 4, 0, 1), rank)
    steps = 1000.0 * (rank + 1)
    ms = 10.0 + rank
    e2e_steps, e2e_s = 500.0 * (rank + 1), 2.0 + rank
    tot, mx, e2e = bench.reduce_over_ranks(steps, ms, e2e_steps, e2e_s, world, "cpu")
    q.put((rank, float(w["p"][1].min()), float(w["p"][1].max()), tot, mx, e2e))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, lo0, hi0, tot0, mx0, e0), (r1, lo1, hi1, tot1, mx1, e1) = out
    assert hi0 < lo1  # disjoint bands of B
    assert tot0 == tot1 == 3000.0 and mx0 == mx1 == 11.0
    assert np.isclose(e0, 1500.0 / 3.0) and np.isclose(e1, e0)


def test_single_rank_reduction_is_identity():
    assert bench.reduce_over_ranks(10.0, 2.0, 4.0, 2.0, 1, "cpu") == (10.0, 2.0, 2.0)
