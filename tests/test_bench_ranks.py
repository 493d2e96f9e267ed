"""Replicas on several ranks (no GPU): the bench's whole-job figure over world_size 2
gloo processes on the CPU is the slowest rank's time and the sum of the ranks' work,
and the replicas draw different seeded inputs."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1102_3137_gb300 import inputs as I
    total_ms = [100.0, 150.0][rank]
    ms, value = bench.aggregate_ranks(total_ms, 1000, 5, world, "cpu")
    w = I.WORKLOADS["square128_K64_p4_k32"]
    _, _, sigma, _ = I.make_inputs(w, K=2, seed=w.seed + rank)
    q.put((rank, ms, value, float(np.abs(sigma).sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for _, ms, value, _ in got:
        assert ms == pytest.approx(30.0)                      # max(100, 150) ms / 5 steps
        assert value == pytest.approx(2 * 1000 / 0.030)       # both ranks' units over that time
    assert got[0][3] != got[1][3]                              # each replica its own inputs


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_ranks(80.0, 500, 4, 1)
    assert ms == 20.0 and value == pytest.approx(500 / 0.020)
