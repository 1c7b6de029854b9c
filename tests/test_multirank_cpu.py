"""Multi-rank host logic on CPU (gloo, world size 2).

The batched workload shards independent problems over ranks with no exchange
on the data path; only the timing is reduced (max over ranks).  Here two gloo
processes check that the shards partition the batch, are balanced, and that
the reduction returns the slowest rank's time.
"""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import workloads


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    kinds, lengths, steps = workloads.batch_problems()
    work = [float(n) * float(s) for n, s in zip(lengths, steps)]
    shards = bench.shard_problems(work, world)
    mine = shards[rank]
    t = 1.0 + rank                      # rank 1 is the slow one
    tmax = bench.max_over_ranks(t, world, device="cpu")
    q.put((rank, mine, sum(work[i] for i in mine), tmax))
    dist.destroy_process_group()


def test_batch_sharding_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    all_idx = sorted(res[0][1] + res[1][1])
    assert all_idx == list(range(4096))                       # a partition
    loads = [r[2] for r in res]
    assert max(loads) / min(loads) < 1.01                      # balanced
    assert res[0][3] == res[1][3] == 2.0                       # max over ranks


def test_shard_single_rank_identity():
    import bench
    assert bench.shard_problems([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
