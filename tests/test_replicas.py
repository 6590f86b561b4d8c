"""The multi-GPU path of the benchmark is replicas only (no exchange step: one patch's transform fits
one GPU): each rank times its own replica and the job's figure is all ranks' points over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]  # rank 1 is the slowest replica
    slow = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (slow, bench.replica_throughput(1_000_000, world, 10, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        slow, value = out[r]
        assert slow == 150.0
        assert value == pytest.approx(2 * 1_000_000 * 10 / 0.150 / 1e6)


def test_single_rank_is_unchanged():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.replica_throughput(2_000_000, 1, 5, 100.0) == pytest.approx(100.0)
