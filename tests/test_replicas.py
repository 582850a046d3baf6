"""Multi-replica path of bench.py on CPU (gloo, world size 2): the whole-job
figures are the slowest rank's time and the summed samples; each rank draws
its own population; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, q):
    sys.path.insert(0, root)
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    import bench

    dist.barrier()
    t, n = bench.reduce_over_ranks(1.5 + rank, 1000 * (rank + 1), dist, "cpu")
    q.put((rank, t, n))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ROOT, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for _, t, n in got:
        assert t == 2.5          # max over ranks
        assert n == 3000.0       # sum over ranks


def test_reduce_over_ranks_single_process_is_identity():
    import bench

    assert bench.reduce_over_ranks(0.25, 7, None, "cpu") == (0.25, 7.0)


def test_replicas_draw_independent_populations():
    import bench

    a = bench.workload("sphere16", 0)["coords"]
    b = bench.workload("sphere16", 1)["coords"]
    assert a.shape == b.shape and not np.array_equal(a, b)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench

    class A:
        workload, gpus, steps, warmup = "sphere16", 2, 1, 3

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(A()) == 0
