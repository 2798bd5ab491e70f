"""The benchmark's multi-rank path on CPU: two gloo ranks, each an independent
replica; the job's time is the slowest rank's and its residuals are summed."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]
    res = [1.0e6, 3.0e6][rank]
    t, u = bench.reduce_over_ranks(ms, res, world)
    dist.barrier()
    results[rank] = (t, u)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_units():
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, u = results[r]
        assert t == 20.0 and u == 4.0e6


def test_single_rank_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.0, 5.0, 1) == (7.0, 5.0)
