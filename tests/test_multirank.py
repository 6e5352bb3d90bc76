"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, no data-path collective)
agree on the slowest rank's step time and report the whole-job sweeps per second."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    out[rank] = bench.aggregate(times[rank], world)
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    import torch.multiprocessing as mp
    world, times = 2, [80.0, 100.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in range(world):
        step_max, value = res[r]
        assert step_max == 100.0                       # the slowest rank
        assert value == pytest.approx(world * 1000.0 / 100.0)  # both replicas' sweeps per second


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(50.0, 1) == (50.0, 20.0)
