"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks agree on
the slowest rank's time, and the whole-job value counts both replicas."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.5, 20.0][rank]          # rank 1 is the slower one
    got = bench.slowest_rank_ms(ms, world, "cpu")
    out[rank] = got
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == 20.0 and out[1] == 20.0


def test_whole_job_value_counts_every_replica():
    import bench
    # 4 M nodes per rank, 2 ranks, 0.25 ms per step -> 33,554 MLUPS
    assert bench.whole_job_mlups(4 * 1024 * 1024, 2, 0.25) == pytest.approx(2 * 4194304 / 0.25e-3 / 1e6)
    assert bench.slowest_rank_ms(3.0, 1, "cpu") == 3.0
