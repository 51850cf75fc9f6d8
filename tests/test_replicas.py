"""The N > 1 path of bench.py: independent replicas whose throughput is the
work summed over ranks over the slowest rank's time, checked with two gloo
ranks on the CPU (no GPU, no collective on the data path)."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    secs = 1.0 + rank            # rank 1 is the slower replica
    work = 100.0 * (rank + 1)
    t, w = bench.aggregate_replicas(secs, work, world, torch.device("cpu"))
    dist.barrier()
    out[rank] = (t, w)
    dist.destroy_process_group()


def test_two_replicas_aggregate_on_gloo():
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (2.0, 300.0)


def test_single_replica_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(3.0, 7.0, 1, None) == (3.0, 7.0)
