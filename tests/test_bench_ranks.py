"""The bench's multi-rank timing (replicas, weak scaling) on CPU with gloo:
every rank reports its own time, the job takes the slowest rank's, and the
whole-job rate counts every rank's units."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [100.0 + 50.0 * rank, 300.0 - 10.0 * rank]  # this rank's (device ms, end-to-end ms)
    agg = bench.max_over_ranks(local, torch.device("cpu"), world)
    out[rank] = (agg, bench.job_rate(1e9, world, agg[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        agg, rate = out[r]
        assert agg == [150.0, 300.0]  # the slowest rank's device time and end-to-end time
        assert rate == pytest.approx(2e9 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.5], None, 1) == [1.5, 2.5]
    assert bench.job_rate(10.0, 1, 1000.0) == pytest.approx(10.0)
