"""Multi-process host logic of the benchmark (CPU, gloo, two ranks): the
timed region's clock is the slowest rank's, and the whole-job value counts
every rank's units over it (the multi-GPU path runs one replica per GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 3.5 * rank, dist, "cpu")
        out[rank] = (t, bench.job_value(world, 1000, 4, t))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_times_the_job():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == pytest.approx(13.5)
        assert v == pytest.approx(world * 1000 * 4 / 13.5e-3)


def test_single_rank_is_its_own_time():
    assert bench.max_over_ranks(7.25, None, "cpu") == 7.25
    assert bench.job_value(1, 10, 2, 4.0) == pytest.approx(10 * 2 / 4e-3)
