"""bench.py's multi-rank path on the CPU: two gloo ranks time different amounts of work; the
reported time is the slowest rank's and the throughput counts every rank's replica."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, ws, torch.device("cpu"))
    out[rank] = (ms, bench.replica_throughput(ws, 1000, 4, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
    assert out[0][0] == out[1][0] == pytest.approx(150.0)
    assert out[0][1] == pytest.approx(2 * 1000 * 4 / 0.150)
