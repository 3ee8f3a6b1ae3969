"""Host logic of the benchmark's multi-rank (replica) path on two gloo ranks
on the CPU: the job's step time is the slowest rank's, None stays None on
every rank, and the throughput counts the units of all ranks."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(1.0 + 0.5 * rank, world, "cpu")
    none = bench.max_over_ranks(None, world, "cpu")
    val = bench.job_throughput(1000.0, world, ms)
    out[rank] = (ms, none, val)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, none, val = res[rank]
        assert ms == 1.5 and none is None
        assert abs(val - 1000.0 * 2 / 1.5e-3) < 1e-6


def test_single_rank_is_untouched():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_throughput(10.0, 1, 2.0) == 5000.0
