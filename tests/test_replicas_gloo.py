"""bench.py's N > 1 path runs one independent replica per rank (the solver does not shard across
GPUs): the job's time is the slowest rank's, and the value counts every rank's solves.  Checked
with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [2.0, 3.5][rank]          # seconds this rank took for its steps
        m = bench.replica_max(local, dist)
        out[rank] = (m, bench.replica_throughput(5, world, m))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_all_solves():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 3.5
        assert v == pytest.approx(5 * 2 / 3.5)


def test_single_process_has_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_max(1.25, None) == 1.25
    assert bench.replica_throughput(3, 1, 1.5) == pytest.approx(2.0)
