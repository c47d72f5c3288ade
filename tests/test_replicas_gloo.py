"""The multi-GPU form is independent replicas (one laminate solve per rank, no
collective on the data path): the benchmark combines the ranks as the slowest
rank's time and the sum of their work.  Exercised here with two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]
    units = [1_000_000, 3_000_000][rank]
    t, u = bench.aggregate_ranks(ms, units, world, torch.device("cpu"))
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        t, u = out[r]
        assert t == 150.0 and u == 4_000_000


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_ranks(12.5, 7, 1, None) == (12.5, 7)
