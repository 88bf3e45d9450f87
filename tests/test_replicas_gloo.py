"""The multi-GPU path is independent replicas: the only collective is the max over ranks of the
timed region. Two gloo ranks on CPU check the aggregation (weak scaling, slowest rank's time)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.job_throughput(times[rank], 1000, 5, world, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_over_ranks():
    world, times = 2, [100.0, 250.0]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 250.0
        assert abs(value - world * 1000 * 5 / 0.25) < 1e-6


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_throughput(200.0, 1000, 5, 1, None, "cpu") == (200.0, 25000.0)


def _rank_served(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ratings, secs = [(3000, 2.0), (5000, 4.0)][rank]
    out[rank] = bench.job_rate(ratings, secs, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_served_replicas_sum_ratings_over_slowest_rank():
    """Served replicas: the job's rate is every rank's ratings over the slowest rank's wall time."""
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_served, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == pytest.approx((3000 + 5000) / 4.0)
