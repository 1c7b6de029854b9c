"""One periodic problem sharded over 2 and 3 ranks (gloo on CPU), through the product exchange layer.

``paper_1504_01380_gb300.shard`` assigns each rank a contiguous slice of whole tiles,
runs the stages of Section 3 on it and exchanges one leading-edge half per stage
with one neighbour, alternating left and right, plus one final message of the
points a straddling window stored past the slice's end.  Here each rank's stages
run on a CPU stand-in (tests/shard_standin.py, the library's edge layout in FP64
with the oracle's point update) and the messages go through torch.distributed
(gloo).  The assembled field must equal the oracle's per-step stepping bit for bit
at every step count shape (q odd and even, with and without a remainder, below one
tile height); a message delivered late still gives the exact field, and a lost one
ends the waiting ranks with SWEPT_ETIMEOUT within their budget instead of hanging.
"""
from __future__ import annotations

import os
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import workloads
from paper_1504_01380_gb300 import shard

HEAT, KS = 0, 1
PRM = {HEAT: [0.25], KS: [workloads.KS_DT, workloads.KS_DX]}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial(stencil, N):
    return workloads.uniform(N, 91) if stencil == HEAT else workloads.ks_smoothed(N, 92) * 10.0


def _cases(B, h):
    # q odd / even with rem 0, q odd / even with rem > 0, below one tile height, one triangle
    return [3 * h, 4 * h, 3 * h + 5, 2 * h + h // 2, h // 2 + 1, h, 1]


class FaultyTransport(shard.TorchDistTransport):
    """Host-side fault injection: the send of ``tag`` on rank ``rank`` is dropped (lost) or
    posted ``delay`` seconds late."""

    def __init__(self, rank, fault_rank, fault_tag, delay=None):
        super().__init__()
        self.rank, self.fault_rank, self.fault_tag, self.delay = rank, fault_rank, fault_tag, delay

    def post(self, send_buf, dst, recv_buf, src, tag):
        import torch.distributed as dist
        if self.rank == self.fault_rank and tag == self.fault_tag:
            if self.delay is None:                                    # lost: only the receive
                return shard._TorchHandle([dist.irecv(recv_buf, src, tag=tag)])
            time.sleep(self.delay)                                    # late
        return super().post(send_buf, dst, recv_buf, src, tag)


def _worker(rank, world, port, q, mode):
    import torch.distributed as dist

    from tests.shard_standin import StandinRunner
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    try:
        if mode == "exact":
            runs = [(st, B, n) for st, B in ((HEAT, 32), (KS, 64)) for n in _cases(B, B // (2 if st == HEAT else 4))]
            for i, (st, B, nsteps) in enumerate(runs):
                r = 1 if st == HEAT else 2
                N = world * 2 * B
                sl = shard.Slice(N, B, world, rank)
                u0 = _initial(st, N)
                run = StandinRunner(st, PRM[st], u0[sl.start:sl.start + sl.n_local], B)
                adv = shard.ShardedAdvance(run, shard.TorchDistTransport(), sl, B // (2 * r), r, nsteps,
                                           timeout_s=60, tag_base=1000 * i)
                status = adv.run()
                out.append((st, B, nsteps, status, run.u, adv.messages))
            q.put((rank, out))
            dist.destroy_process_group()
            return
        # fault injection: heat, B = 32, 5h + 3 steps; the message after stage 2 from rank 1
        B, h, nsteps = 32, 16, 5 * 16 + 3
        N = world * 2 * B
        sl = shard.Slice(N, B, world, rank)
        run = StandinRunner(HEAT, PRM[HEAT], _initial(HEAT, N)[sl.start:sl.start + sl.n_local], B)
        delay = 1.0 if mode == "late" else None
        tr = FaultyTransport(rank, 1, 2 * 2, delay)
        adv = shard.ShardedAdvance(run, tr, sl, h, 1, nsteps, timeout_s=3.0 if mode == "late" else 1.0)
        t0 = time.monotonic()
        status = adv.run()
        q.put((rank, [(HEAT, B, nsteps, status, run.u, time.monotonic() - t0)]))
    finally:
        if mode == "lost":
            # unmatched operations stay posted after a timeout: leave without tearing the group down
            q.close()
            q.join_thread()
            os._exit(0)


def _reduce_worker(rank, world, port, q):
    """Each rank's partials (exactly rounded sums of its slice, the stand-in for the slice's
    swept_reduce), combined over the ranks by the product reducer."""
    import math

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N = world * 1000
    u, v = workloads.uniform(N, 93), workloads.uniform(N, 94)
    lo, hi = rank * 1000, (rank + 1) * 1000
    red = shard.TorchDistReducer()
    parts = [math.fsum(u[lo:hi]), 0.5 * math.fsum(u[lo:hi] ** 2), math.fsum(u[lo:hi] * v[lo:hi])]
    got = [red.allreduce(torch.tensor([p], dtype=torch.float64)) for p in parts]
    q.put((rank, got))
    dist.destroy_process_group()


def _spawn(world, mode, timeout=300):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    target, args = (_reduce_worker, ()) if mode == "reduce" else (_worker, (mode,))
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=timeout) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_advance_bit_exact(world):
    res = _spawn(world, "exact")
    nruns = len(res[0])
    for i in range(nruns):
        st, B, nsteps = res[0][i][:3]
        N = world * 2 * B
        got = np.concatenate([res[r][i][4] for r in range(world)])
        want = oracle.advance_f64(st, PRM[st], _initial(st, N), nsteps)
        assert all(res[r][i][3] == shard.SWEPT_OK for r in range(world))
        assert np.array_equal(got, want), (world, st, nsteps, np.flatnonzero(got != want)[:8])
        # one edge half per stage boundary, plus the final head message when a straddler wrapped
        r_ = 1 if st == HEAT else 2
        stages = shard.schedule(nsteps, B // (2 * r_))
        extra = 1 if shard.wrapped_head(nsteps, B // (2 * r_), B, r_) else 0
        assert res[0][i][5] == len(stages) - 1 + extra


def test_late_message_still_exact():
    world = 3
    res = _spawn(world, "late")
    got = np.concatenate([res[r][0][4] for r in range(world)])
    st, B, nsteps = res[0][0][:3]
    want = oracle.advance_f64(st, PRM[st], _initial(st, world * 2 * B), nsteps)
    assert all(res[r][0][3] == shard.SWEPT_OK for r in range(world))
    assert np.array_equal(got, want)


def test_lost_message_times_out():
    world = 3
    res = _spawn(world, "lost")
    statuses = {r: res[r][0][3] for r in range(world)}
    # rank 1's message after stage 2 goes left (stage 2 is unshifted) to rank 0, which gives up
    assert statuses[0] == shard.SWEPT_ETIMEOUT
    assert all(s in (shard.SWEPT_OK, shard.SWEPT_ETIMEOUT) for s in statuses.values())
    assert all(res[r][0][5] < 30 for r in range(world))      # every rank ended within its budgets


def test_schedule_and_wrapped_head():
    """The stage list is swept_advance's; the wrapped head is where an odd stage's straddler
    stores past the slice end (checked against a direct count of the stored positions)."""
    assert shard.schedule(0, 16) == []
    assert shard.schedule(5, 16) == [(0, 0, 5), (1, 5, 0)]
    assert shard.schedule(48, 16) == [(0, 0, 16), (1, 16, 16), (2, 16, 16), (3, 16, 0)]
    assert shard.schedule(35, 16) == [(0, 0, 16), (1, 16, 16), (2, 16, 3), (3, 3, 0)]
    for B, r in ((32, 1), (64, 2)):
        h = B // (2 * r)
        for levels in range(1, 5 * h):
            wrapped = set()
            for k, hv, ht in shard.schedule(levels, h):
                if k % 2 == 0:
                    continue
                if ht == 0 and hv == h:
                    xs = range(B)
                elif ht == 0:
                    xs = range(B // 2 - r * hv, B // 2 + r * hv)
                elif ht < h:
                    xs = range(r * ht, B - r * ht)
                else:
                    xs = []
                wrapped |= {x - B // 2 for x in xs if x >= B // 2}
            assert wrapped == set(range(shard.wrapped_head(levels, h, B, r))), (B, levels)


def test_slice_rejects_partial_tiles():
    with pytest.raises(ValueError):
        shard.Slice(1000, 64, 3, 0)
    s = shard.Slice(3 * 4 * 64, 64, 3, 2)
    assert (s.n_local, s.nwin, s.start, s.left, s.right) == (256, 4, 512, 1, 0)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reduction_same_bits_on_every_rank(world):
    """The FP64 reductions of a sharded field: every rank holds the same bits, within one
    rounding per rank of the exact sum (each partial rounded once, their sum rounded once)."""
    import math
    res = _spawn(world, "reduce")
    N = world * 1000
    u, v = workloads.uniform(N, 93), workloads.uniform(N, 94)
    exact = [math.fsum(u), 0.5 * math.fsum(u ** 2), math.fsum(u * v)]
    scale = [np.sum(np.abs(u)), 0.5 * np.sum(u ** 2), np.sum(np.abs(u * v))]
    for r in range(world):
        assert res[r] == res[0]
    for g, e, sc in zip(res[0], exact, scale):
        assert abs(g - e) <= (world + 1) * 2.0 ** -53 * sc


def test_combine_partials_is_order_free():
    rng = np.random.default_rng(5)
    parts = list(rng.standard_normal(7) * 10.0 ** rng.integers(-8, 8, 7))
    want = shard.combine_partials(parts)
    for _ in range(5):
        rng.shuffle(parts)
        assert shard.combine_partials(parts) == want
