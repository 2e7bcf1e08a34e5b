"""The N-replica path of bench.py on CPU: two gloo ranks, each with its own
time; the job's time is the slowest rank's, and the job's throughput counts
every rank's cells (weak scaling, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 95.5][rank]
        m = bench.reduce_max(elapsed, dist, device="cpu")
        out[rank] = (m, bench.job_throughput(1000, 10, world, m))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (120.0, 1000 * 10 * 2 / 0.12)


def test_single_process_needs_no_collective():
    import bench
    assert bench.reduce_max(7.5, None) == 7.5
    assert bench.job_throughput(100, 4, 1, 2.0) == pytest.approx(100 * 4 / 2e-3)
