"""The replica aggregation of bench.py over torch.distributed (gloo, two CPU
ranks): the whole-job value is the points of all ranks over the slowest
rank's time, and every rank gets the same answer."""
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


def _rank(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    pts = [1.0e9, 3.0e9][rank]
    ms = [200.0, 500.0][rank]
    value, t_max = bench.combine_ranks(pts, ms, dist, "cpu")
    out[rank] = (value, t_max)
    dist.destroy_process_group()


def test_two_rank_aggregation():
    pytest.importorskip("torch.distributed")
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(_free_port(), out), nprocs=2, join=True)
    for r in range(2):
        value, t_max = out[r]
        assert t_max == 500.0
        assert abs(value - 4.0e9 / 0.5) < 1e-6 * value


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    value, t_max = bench.combine_ranks(2.0e9, 250.0)
    assert t_max == 250.0 and abs(value - 8.0e9) < 1e-3
