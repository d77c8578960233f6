"""The replicas path of bench.py on the CPU: two gloo ranks time different
amounts, every rank ends with the slowest rank's time, and the whole-job
throughput counts the cells of both replicas over that time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 1.5 + rank  # seconds: rank 1 is the slow one
        t = bench.max_over_ranks(mine, dist, "cpu")
        out[rank] = (t, bench.job_mlups(world, 1_000_000, 100, t))
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(2.5)
    # 2 replicas x 1e6 cells x 100 steps in 2.5 s
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1e6 * 100 / 2.5 / 1e6)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.job_mlups(1, 10, 10, 1.0) == pytest.approx(1e-4)
