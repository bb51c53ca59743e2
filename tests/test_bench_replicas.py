"""The replica timing of bench.py over several ranks (gloo on CPU, world
size 2): the job's time is the slowest replica's, its throughput counts every
replica's frames."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        my_ms = 2.0 + 3.0 * rank           # rank 1 is the slower replica
        ms = bench.max_over_ranks(my_ms, dist, torch, "cpu")
        dist.barrier()
        out[rank] = (ms, bench.job_frames_per_s(ms, world))
    finally:
        dist.destroy_process_group()


def test_slowest_replica_sets_the_job_time():
    world = 2
    port = _free_port()
    mgr = tmp.get_context("spawn").Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == (5.0, world * 1000.0 / 5.0)
