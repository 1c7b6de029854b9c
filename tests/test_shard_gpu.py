"""The sharded advance's GPU side on one GPU: several slices, each its own plan, in one process.

``paper_1504_01380_gb300.shard`` runs each slice's stages through the C ABI
(swept_stage on a plan over the slice, swept_edge_copy for the edge halves it
sends and receives).  Here G slices of one periodic problem share this GPU and
their messages go through an in-process loopback (device copies), driven
round-robin by ``shard.drive_in_process``: each slice's stage kernels finish
before its messages are read, so no kernel waits on another.  The assembled
field must equal the oracle bit for bit, for FP64 and the compensated state,
with per-window and ring kernels, over every step-count shape.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from paper_1504_01380_gb300 import shard
from tests.test_parity_gpu import params_of

pytestmark = pytest.mark.gpu


class _LoopHandle:
    def __init__(self, box, key, recv_buf):
        self.box, self.key, self.recv_buf, self.got = box, key, recv_buf, False

    def done(self):
        if not self.got and self.key in self.box:
            self.recv_buf.copy_(self.box.pop(self.key))
            self.got = True
        return self.got

    def wait(self, timeout_s):
        return self.done()


class LoopbackTransport:
    """Messages between slices of one process: a send is a device copy into a mailbox."""

    def __init__(self, rank, box):
        self.rank, self.box = rank, box

    def post(self, send_buf, dst, recv_buf, src, tag):
        self.box[(self.rank, dst, tag)] = send_buf.clone()
        return _LoopHandle(self.box, (src, self.rank, tag), recv_buf)


def _run(sw, stencil, dtype, B, world, nloc_tiles, nsteps, u0, ring):
    import torch
    r = 1 if stencil == 0 else 2
    N = u0.size
    box, progs, runners = {}, [], []
    for rank in range(world):
        sl = shard.Slice(N, B, world, rank)
        plan = sw.swept_plan(sl.n_local, r, stencil, params_of(stencil), dtype, B)
        if ring:                       # full diamonds on the ring kernel (two warps per slice)
            sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
            sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 2)
        t = torch.tensor(u0[sl.start:sl.start + sl.n_local], dtype=torch.float64, device="cuda")
        u = t if dtype == sw.SWEPT_F64 else sw.swept_f32c_split(t)
        run = shard.PlanRunner(plan, u)
        runners.append((plan, run))
        progs.append(shard.ShardedAdvance(run, LoopbackTransport(rank, box), sl, plan.h, r, nsteps).program())
    assert shard.drive_in_process(progs, timeout_s=10) == shard.SWEPT_OK
    torch.cuda.synchronize()
    if dtype == sw.SWEPT_F64:
        return np.concatenate([run.u.cpu().numpy() for _, run in runners])
    hi = np.concatenate([run.u[:run.plan.N].cpu().numpy() for _, run in runners])
    lo = np.concatenate([run.u[run.plan.N:].cpu().numpy() for _, run in runners])
    return hi, lo


@pytest.mark.parametrize("stencil,dtype,B", [(0, 0, 64), (0, 1, 128), (1, 0, 128), (1, 1, 256)])
@pytest.mark.parametrize("world,nloc_tiles,ring", [(2, 3, False), (3, 9, True)])
def test_sharded_slices_on_one_gpu_bit_exact(cuda_lib, stencil, dtype, B, world, nloc_tiles, ring):
    sw = cuda_lib
    r = 1 if stencil == 0 else 2
    h = B // (2 * r)
    N = world * nloc_tiles * B
    u0 = workloads.uniform(N, 93) if stencil == 0 else workloads.ks_smoothed(N, 94) * 10.0
    for nsteps in (3 * h, 4 * h, 3 * h + 5, 2 * h + h // 2, h // 2 + 1, 1):
        got = _run(sw, stencil, dtype, B, world, nloc_tiles, nsteps, u0, ring)
        if dtype == sw.SWEPT_F64:
            want = oracle.advance_f64(stencil, params_of(stencil), u0, nsteps)
            assert np.array_equal(got, want), (nsteps, np.flatnonzero(got != want)[:8])
        else:
            hi, lo = oracle.split_f32c(u0)
            whi, wlo = oracle.advance_f32c(stencil, params_of(stencil), hi, lo, nsteps)
            assert np.array_equal(got[0], whi) and np.array_equal(got[1], wlo), nsteps


def test_stage_and_edge_copy_arguments(cuda_lib):
    """swept_stage and swept_edge_copy refuse out-of-range stages, windows and sides."""
    import torch
    sw = cuda_lib
    plan = sw.swept_plan(4 * 64, 1, 0, [0.25], sw.SWEPT_F64, 64)
    u = torch.zeros(4 * 64, dtype=torch.float64, device="cuda")
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    for k, hv, ht in ((0, 0, 0), (-1, 0, 5), (0, 33, 0), (0, 0, 33)):
        with pytest.raises(sw.SweptError):
            sw.swept_stage(plan, u, k, hv, ht)
    for w, side in ((4, 0), (-1, 0), (0, 2)):
        with pytest.raises(sw.SweptError):
            sw.swept_edge_copy(plan, 1, w, side, buf, False)
    plan.destroy()


def test_sharded_runge_kutta_and_euler(cuda_lib):
    """The sharded path for the schemes with several sub-timesteps per time step and wider
    point states: KS by the Runge-Kutta rule (levels = 2 x steps; (u, m) edge pairs) and the
    Euler equations in compensated FP32 (levels = 4 x steps; the state's six blocks of N/G
    floats per slice; 48-byte edge elements), three slices on this GPU against the oracle."""
    import torch
    from tests.test_euler_gpu import state as euler_state
    sw = cuda_lib
    # Runge-Kutta KS, FP64
    B, world = 128, 3
    N = world * 4 * B
    prm = params_of(1)
    u0 = workloads.ks_smoothed(N, 95) * 10.0
    for nsteps in (3 * (B // 8) + 2, 5 * (B // 8)):       # h = B/4 levels = B/8 steps
        box, progs, runs = {}, [], []
        for rank in range(world):
            sl = shard.Slice(N, B, world, rank)
            plan = sw.swept_plan(sl.n_local, 2, sw.SWEPT_KS_RK2, prm, sw.SWEPT_F64, B)
            u = torch.tensor(u0[sl.start:sl.start + sl.n_local], device="cuda")
            run = shard.PlanRunner(plan, u)
            runs.append(run)
            progs.append(shard.ShardedAdvance(run, LoopbackTransport(rank, box), sl, plan.h, 2,
                                              2 * nsteps).program())
        assert shard.drive_in_process(progs, timeout_s=10) == shard.SWEPT_OK
        torch.cuda.synchronize()
        got = np.concatenate([r.u.cpu().numpy() for r in runs])
        assert np.array_equal(got, oracle.advance_rk2_f64(3, prm, u0, nsteps)), nsteps
    # Euler equations, compensated FP32
    B, world = 64, 2
    N = world * 5 * B
    q, prm_e = euler_state(N, 96)                       # (N, 3) rows
    for nsteps in (3 * (B // 8) + 1, 4 * (B // 8)):     # h = B/2 levels = B/8 steps
        box, progs, runs = {}, [], []
        for rank in range(world):
            sl = shard.Slice(N, B, world, rank)
            part = q[sl.start:sl.start + sl.n_local]
            planar = np.concatenate([part[:, 0], part[:, 1], part[:, 2]])
            plan = sw.swept_plan(sl.n_local, 1, sw.SWEPT_EULER, prm_e, sw.SWEPT_F32C, B)
            u = sw.swept_f32c_split(torch.tensor(planar, device="cuda"))
            run = shard.PlanRunner(plan, u)
            runs.append(run)
            progs.append(shard.ShardedAdvance(run, LoopbackTransport(rank, box), sl, plan.h, 1,
                                              4 * nsteps).program())
        assert shard.drive_in_process(progs, timeout_s=10) == shard.SWEPT_OK
        torch.cuda.synchronize()
        hi, lo = oracle.split_f32c(np.ascontiguousarray(q).reshape(-1))
        whi, wlo = oracle.euler_advance_f32c(prm_e, hi.reshape(-1, 3), lo.reshape(-1, 3), nsteps)
        n = N // world
        for rank, run in enumerate(runs):
            a = run.u.cpu().numpy()
            ghi = a[:3 * n].reshape(3, n).T
            glo = a[3 * n:].reshape(3, n).T
            assert np.array_equal(ghi, whi[rank * n:(rank + 1) * n]), (nsteps, rank)
            assert np.array_equal(glo, wlo[rank * n:(rank + 1) * n]), (nsteps, rank)


class _LocalReducer:
    """The all-gather of a sharded reduction, for slices of one process: the partials are
    collected, then combined as the product reducer combines them."""

    def __init__(self):
        self.parts = []

    def allreduce(self, partial):
        self.parts.append(partial.item())
        return shard.combine_partials(self.parts)


@pytest.mark.parametrize("dtype", [0, 1])
def test_sharded_reduction_matches_whole_field(cuda_lib, dtype):
    """sharded_reduce over 4 slices of one field (each slice's swept_reduce, combined once)
    against the oracle's exactly rounded sums: within the single-field bound plus one
    rounding per slice."""
    import torch
    from oracle import reductions as ored
    sw = cuda_lib
    world, B, N = 4, 256, 4 * 256 * 64
    u0, v = workloads.heat_noise_modes(N, 16, 4), workloads.uniform(N, 6)
    vals = u0 if dtype == 0 else oracle.merge_f32c(*oracle.split_f32c(u0))
    got = {}
    for what in (sw.SWEPT_SUM, sw.SWEPT_HALF_SUMSQ, sw.SWEPT_DOT):
        red = _LocalReducer()
        for rank in range(world):
            sl = shard.Slice(N, B, world, rank)
            plan = sw.swept_plan(sl.n_local, 1, 0, [0.25], dtype, B)
            seg = u0[sl.start:sl.start + sl.n_local]
            if dtype == 0:
                u = torch.tensor(seg, device="cuda")
            else:
                hi, lo = oracle.split_f32c(seg)
                u = torch.tensor(np.concatenate([hi, lo]), device="cuda")
            vv = torch.tensor(v[sl.start:sl.start + sl.n_local], device="cuda")
            got[what] = shard.sharded_reduce(plan, u, what, red, v=vv if what == sw.SWEPT_DOT else None)
            plan.destroy()
    eps = np.finfo(np.float64).eps
    for what, ex, scale in ((sw.SWEPT_SUM, ored.total(vals), np.sum(np.abs(vals))),
                            (sw.SWEPT_HALF_SUMSQ, ored.half_sumsq(vals), ored.half_sumsq(vals)),
                            (sw.SWEPT_DOT, ored.dot(vals, v), np.sum(np.abs(vals * v)))):
        assert abs(got[what] - ex) <= 4 * eps * abs(ex) + (world + N * eps) * eps * scale, (what, got[what], ex)
