"""The multi-rank path of the benchmark on CPU ranks (gloo, world size 2).

Each rank evaluates its own proposals (weak scaling, no data-path
collective); the only exchange is the MAX of the ranks' timed intervals, and
the job's rate is all ranks' units over that slowest time.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2003_03508_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, "cpu")
        rate = bench.job_rate(256 * 20, world, t)
        d = synth.batched_inputs(K=4, T=200, n_prop=3, seed=bench.rank_seed(3, rank))
        q.put((rank, t, rate, d["params"].P.copy()))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    times = [812.5, 1311.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda r: r[0])
    for rank, t, rate, _ in res:
        assert t == max(times)
        assert rate == pytest.approx(2 * 256 * 20 / (max(times) / 1e3))
    # the ranks evaluate different proposals
    assert not np.array_equal(res[0][3], res[1][3])


def test_single_rank_is_the_identity():
    assert bench.max_over_ranks(5.0, 1, "cpu") == 5.0
    assert bench.job_rate(100, 1, 1000.0) == pytest.approx(100.0)
