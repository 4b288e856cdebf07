"""The N > 1 path of bench.py: independent replicas, whole-job value = units of all ranks over the
slowest rank's time (max-reduce over ranks; no data-path collective).  Run as two gloo ranks on
the CPU."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = 1.0 + rank            # rank 1 is the slow one
    value, tmax = bench.aggregate_over_ranks(local, 1000.0, world, "cpu")
    out[rank] = (value, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        value, tmax = out[r]
        assert tmax == pytest.approx(2.0)
        assert value == pytest.approx(world * 1000.0 / 2.0)


def test_single_rank_aggregation_is_local():
    sys.path.insert(0, ROOT)
    import bench
    value, tmax = bench.aggregate_over_ranks(0.5, 100.0, 1)
    assert tmax == 0.5 and value == pytest.approx(200.0)
