"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2): each rank times its
own lattice (weak scaling, no data-path collective); the job's time is the slowest
rank's and the throughput counts the work of every rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]                # rank 1 is slower
    ms_max, gbs = bench.reduce_over_ranks(ms, 100, world, 10 ** 9, dist, torch.device("cpu"))
    out[rank] = (ms_max, gbs)
    dist.destroy_process_group()


def test_reduce_over_ranks_two_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of this threaded process
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms_max, gbs = res[r]
        assert ms_max == 150.0
        assert abs(gbs - 2 * 1e9 * 100 / 0.150 / 1e9) < 1e-9


def test_reduce_over_ranks_single():
    import bench
    ms_max, gbs = bench.reduce_over_ranks(200.0, 50, 1, 2 * 10 ** 9)
    assert ms_max == 200.0 and abs(gbs - 500.0) < 1e-9
