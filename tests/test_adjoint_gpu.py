"""Swept adjoint: against the oracle's discrete adjoint, closed forms and finite differences."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

KS_PRM = [workloads.KS_DT, workloads.KS_DX]


def dev(x):
    import torch
    return torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("B,K_cycles", [(64, 1), (64, 2), (128, 3), (64, 64)])
def test_ks_adjoint_matches_oracle(cuda_lib, B, K_cycles):
    """N = 256, 500 steps: bit-exact against the oracle's discrete adjoint (J = 1/2 sum u^2)."""
    sw = cuda_lib
    n, nsteps = 256, 500
    u0 = workloads.ks_smoothed(n, 47) * 10
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, B)
    uT = oracle.advance_f64(1, KS_PRM, u0, nsteps)
    want = oracle.adjoint_f64(1, KS_PRM, u0, uT, nsteps)
    got = sw.swept_adjoint(plan, dev(u0), dev(uT), nsteps, K_cycles).cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    assert np.array_equal(got, want)


def test_ks_adjoint_segmentation_invariant(cuda_lib):
    sw = cuda_lib
    n, nsteps = 4096, 777
    u0 = workloads.ks_smoothed(n, 5) * 10
    lam = workloads.uniform(n, 6)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    outs = [sw.swept_adjoint(plan, dev(u0), dev(lam), nsteps, k).cpu().numpy() for k in (1, 2, 5, 64)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    assert np.array_equal(outs[0], oracle.adjoint_f64(1, KS_PRM, u0, lam, nsteps))


@pytest.mark.parametrize("B,warps", [(128, 1), (128, 3), (128, 0), (256, 2)])
def test_ks_adjoint_ring_sweep_matches_oracle(cuda_lib, B, warps):
    """The transposed sweep on the ring kernel (forced, with several run lengths): each slot
    reads the forward state of the window and level it computes; bit-exact against the oracle."""
    sw = cuda_lib
    n = 32 * B
    u0 = workloads.ks_smoothed(n, 9) * 10
    lam = workloads.uniform(n, 10)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
    for nsteps, K in ((4 * plan.h + 3, 1), (7 * plan.h, 2), (5 * plan.h + 11, 64)):
        got = sw.swept_adjoint(plan, dev(u0), dev(lam), nsteps, K).cpu().numpy()
        assert np.array_equal(got, oracle.adjoint_f64(1, KS_PRM, u0, lam, nsteps)), (nsteps, K)


@pytest.mark.parametrize("stream", [1, 0])
def test_ks_adjoint_checkpoint_dumps_every_kernel(cuda_lib, stream):
    """The forward pass's flat checkpoints are stored by whichever kernel runs the stage: the
    streamed ring (stream = 1), one ring launch per stage (stream = 0), and the per-window
    kernel (few windows).  Checkpoint intervals of 1 to 4 stages and step counts around the
    stage boundaries, bit-exact against the oracle's discrete adjoint."""
    sw = cuda_lib
    B = 128
    for nwin, ring in ((24, True), (4, False)):
        n = nwin * B
        u0 = workloads.ks_smoothed(n, 21) * 10
        lam = workloads.uniform(n, 22)
        plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, B)
        if ring:
            sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
            sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 4)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_STREAM, stream)
        h = plan.h
        for nsteps, K in ((9 * h, 1), (9 * h + 5, 2), (13 * h + h - 1, 1), (2 * h + 1, 64), (h - 3, 1)):
            got = sw.swept_adjoint(plan, dev(u0), dev(lam), nsteps, K).cpu().numpy()
            assert np.array_equal(got, oracle.adjoint_f64(1, KS_PRM, u0, lam, nsteps)), (nwin, nsteps, K)
        plan.destroy()


def test_adjoint_scratch_is_bounded(cuda_lib):
    """The scratch is 8N * ([rem > 0] + ceil(q/m) + (m + 1) h) bytes with m the minimiser: for the
    adjoint workload (N = 2^20, 20000 steps, B = 256, at most 64 cycles between checkpoints) 349
    states, under 4 GiB; none for heat."""
    sw = cuda_lib
    n = 1 << 20
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    b = sw.swept_adjoint_scratch(plan, 20000, 64)
    assert b == 349 * 8 * n and b < 4 * 2 ** 30
    assert sw.swept_adjoint_scratch(plan, 0, 64) == 0
    assert sw.swept_adjoint_scratch(plan, 20, 64) == (1 + 2 * 64) * 8 * n       # q = 0: rem levels only
    heat = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F64, 256)
    assert sw.swept_adjoint_scratch(heat, 20000, 64) == 0
    plan.destroy()
    heat.destroy()


def test_ks_adjoint_2p22_runs_and_matches_fd(cuda_lib):
    """N = 2^22 (four times the adjoint workload's field), 2000 steps: the gradient fits and
    agrees with central differences along two directions within 1e-6."""
    import torch
    sw = cuda_lib
    n, nsteps = 1 << 22, 2000
    u0 = workloads.ks_smoothed(n, 23)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    J = _J_factory(sw, plan, nsteps)
    _, uT = J(u0)
    g = sw.swept_adjoint(plan, dev(u0), uT, nsteps, 64)
    torch.cuda.synchronize()
    assert sw.swept_adjoint_scratch(plan, nsteps, 64) < 6 * 2 ** 30
    g = g.cpu().numpy()
    for d in range(2):
        v = workloads.fd_direction(n, d)
        eps = 1e-6
        fd = (J(u0 + eps * v)[0] - J(u0 - eps * v)[0]) / (2 * eps)
        ad = math.fsum(g * v)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (d, fd, ad)
    plan.destroy()


def test_heat_adjoint_is_forward_2n(cuda_lib):
    """Heat: grad of 1/2 sum u(T)^2 = A^(2n) u0 (A symmetric), bit for bit."""
    sw = cuda_lib
    n, nsteps = 8192, 300
    u0 = workloads.uniform(n, 8)
    plan = sw.swept_plan(n, 1, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F64, 256)
    uT = oracle.advance_f64(0, [0.25], u0, nsteps)
    got = sw.swept_adjoint(plan, dev(u0), dev(uT), nsteps).cpu().numpy()
    assert np.array_equal(got, oracle.advance_f64(0, [0.25], u0, 2 * nsteps))


def test_adjoint_rejects_compensated_plan(cuda_lib):
    sw = cuda_lib
    plan = sw.swept_plan(1024, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F32C, 256)
    import torch
    z = torch.zeros(1024, dtype=torch.float64, device="cuda")
    with pytest.raises(sw.SweptError) as ei:
        sw.swept_adjoint(plan, z, z, 10)
    assert ei.value.code == sw.SWEPT_ENOTSUP


def test_autograd_function(cuda_lib):
    import torch
    sw = cuda_lib
    n, nsteps = 2048, 400
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    u0 = dev(workloads.ks_smoothed(n, 11) * 10).requires_grad_(True)
    uT = sw.SweptAdvance.apply(u0, plan, nsteps)
    J = 0.5 * (uT * uT).sum()
    (g,) = torch.autograd.grad(J, u0)
    want = oracle.adjoint_f64(1, KS_PRM, u0.detach().cpu().numpy(), uT.detach().cpu().numpy(), nsteps)
    assert np.array_equal(g.cpu().numpy(), want)


def _J_factory(sw, plan, nsteps):
    import torch

    def J(u):
        t = dev(u)
        sw.swept_advance(plan, t, nsteps)
        return sw.swept_reduce(plan, t, sw.SWEPT_HALF_SUMSQ).item(), t
    return J


def test_ks_adjoint_full_size_short_horizon_fd(cuda_lib):
    """N = 2^20, 2000 steps, 8 checkpoint segments: <grad J, v> within 1e-6 of central differences."""
    sw = cuda_lib
    n, nsteps = 1 << 20, 2000
    u0 = workloads.ks_adjoint_state(n)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    J = _J_factory(sw, plan, nsteps)
    _, uT = J(u0)
    g = sw.swept_adjoint(plan, dev(u0), uT, nsteps, 2).cpu().numpy()
    for d in range(8):
        v = workloads.fd_direction(n, d)
        eps = 1e-6
        fd = (J(u0 + eps * v)[0] - J(u0 - eps * v)[0]) / (2 * eps)
        ad = math.fsum(g * v)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (d, fd, ad)


def test_ks_adjoint_full_size_fd_converges(cuda_lib):
    """N = 2^20, 20000 steps, checkpoints every 64 cycles (the adjoint workload).

    Over 40 time units the chaotic dynamics amplify the O(eps^2) truncation of the
    central difference D(eps): halving eps must shrink |D - AD| about fourfold
    (quadratic), and the Richardson combination (4 D(eps/2) - D(eps)) / 3, which
    cancels the eps^2 term, must agree with the adjoint within 1e-6.
    """
    sw = cuda_lib
    n, nsteps = 1 << 20, 20000
    u0 = workloads.ks_adjoint_state(n)
    plan = sw.swept_plan(n, 2, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 256)
    J = _J_factory(sw, plan, nsteps)
    _, uT = J(u0)
    g = sw.swept_adjoint(plan, dev(u0), uT, nsteps, 64).cpu().numpy()
    for d in range(4):
        v = workloads.fd_direction(n, d)
        ad = math.fsum(g * v)
        errs, fds = [], []
        for eps in (1e-6, 5e-7, 2.5e-7):
            fd = (J(u0 + eps * v)[0] - J(u0 - eps * v)[0]) / (2 * eps)
            fds.append(fd)
            errs.append(abs(fd - ad) / abs(ad))
        rich = (4 * fds[2] - fds[1]) / 3
        assert abs(rich - ad) <= 1e-6 * abs(ad), (d, rich, ad, errs)
        assert errs[0] <= 1e-2, (d, errs)
        if errs[0] > 1e-4:           # truncation-dominated: must converge quadratically
            assert errs[1] <= errs[0] / 2.5 and errs[2] <= errs[1] / 2.5, (d, errs)
        else:                        # already at the rounding floor of J's differences
            assert max(errs) <= 1e-3, (d, errs)
