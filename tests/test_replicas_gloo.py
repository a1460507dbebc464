"""Multi-GPU mode is replicas only: every rank runs the whole query on its own
GPU and the reported time is the slowest rank's.  The max-over-ranks
reduction bench.py uses is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    got = bench.reduce_max(1.5 + rank, world, "cpu")
    ws, r, _ = bench.dist_env()
    out[rank] = (got, ws, r)
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a process that has torch threads
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (2.5, 2, 0) and out[1] == (2.5, 2, 1)
