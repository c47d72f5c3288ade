"""The multi-GPU form is independent replicas (one laminate solve per rank, no
collective on the data path): the benchmark combines the ranks as the slowest
rank's time and the sum of their work, and the batch of independent laminates
is split across the ranks by DOF.  Exercised here with two gloo ranks on the
CPU."""
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


def _shard_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1707_04228_gb300 import inputs
    lams = inputs.batch_plates(count=96, nev=8)
    costs = [l.n_dof for l in lams]
    mine = bench.shard_worklist(costs, world)[rank]
    seen = torch.zeros(len(lams), dtype=torch.int64)
    seen[mine] = 1
    dist.all_reduce(seen)                         # each laminate on exactly one rank
    dof = sum(costs[i] for i in mine)
    t, u = bench.aggregate_ranks(dof * 1e-6, dof, world, torch.device("cpu"))
    out[rank] = (list(mine), seen.tolist(), dof, t, u, sum(costs))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_batch_split():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_shard_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    m0, seen, d0, t, u, total = out[0]
    m1, _, d1, _, _, _ = out[1]
    assert seen == [1] * 96 and not set(m0) & set(m1)
    assert u == total == d0 + d1                  # whole-job work is every laminate once
    assert t == max(d0, d1) * 1e-6                # slowest rank's time
    assert max(d0, d1) <= 1.02 * total / 2        # the split by DOF is balanced


def test_shard_worklist_small_cases():
    import bench
    assert bench.shard_worklist([5, 3, 2], 1) == [[0, 1, 2]]
    assert bench.shard_worklist([5, 3, 2], 2) == [[0], [1, 2]]
    assert bench.shard_worklist([1, 1], 4) == [[0], [1], [], []]
