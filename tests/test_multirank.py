"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timings
are reduced with a maximum over ranks and the whole-job throughput counts
every replica's node updates in the slowest rank's time."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [0.5 + rank, 2.0 - rank]   # rank 0 is faster on the first entry, slower on the second
        got = bench.max_over_ranks(local, world, "cpu")
        out[rank] = got + [bench.job_mlups(1000, 10, world, got[0])]
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t0, t1, value = out[rank]
        assert t0 == 1.5 and t1 == 2.0
        assert value == pytest.approx(world * 1000 * 10 / 1.5 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.0, 2.0], 1, "cpu") == [1.0, 2.0]
    assert bench.job_mlups(16777216, 500, 1, 0.5) == pytest.approx(16777216 * 500 / 0.5 / 1e6)
