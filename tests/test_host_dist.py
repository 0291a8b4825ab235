"""The multi-GPU bench path on CPU (gloo, world size 2): every rank runs an independent
replica, the job's time is the maximum over ranks, and the job's throughput counts the
units of all ranks.  The distributed setup reads the launcher's environment."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, loc = bench.dist_setup(None)
    ms = bench.job_time_ms(10.0 + 5.0 * rank, w)          # rank 1 is the slow one
    rate = bench.job_rate(20, ms, w)
    out[rank] = (r, w, loc, ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_over_two_gloo_ranks():
    world = 2
    # a spawned manager: the test process may already run the oracle's OpenMP threads,
    # and a fork of a multi-threaded process can deadlock
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        r, w, loc, ms, rate = out[rank]
        assert (r, w, loc) == (rank, world, rank)
        assert ms == 15.0                                  # the maximum over ranks
        assert abs(rate - 2 * 20 / 15e-3) < 1e-9           # units of both ranks / job time


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(7.5, 1) == 7.5
    assert bench.job_rate(3, 7.5, 1) == 3 / 7.5e-3
