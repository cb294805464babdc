"""The replicas path of bench.py on CPU: two gloo ranks aggregate their timings (max) and arc scans (sum)
the way `bench.py --gpus N` does under torchrun."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, scans = bench.aggregate_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1), "cpu")
        out[rank] = (ms, scans)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of a process that already runs threads
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (150.0, 3000.0)
