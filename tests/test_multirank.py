"""The replica (N > 1) path of bench.py on CPU: world_size-2 gloo ranks, each with
its own timing and unit count; the whole-job time is the slowest rank's and the
units are summed (no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist)
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (150.0, 3000.0)


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(12.5, 7.0, None) == (12.5, 7.0)
