"""GPU parity of the Euler-equations path (Section 7's scheme) against the oracle.

Swept stages (per-window and ring kernels) and the naive stepper must equal the
oracle's per-step stepping bit for bit, in FP64 and on the compensated FP32
state: both sides evaluate the same expressions in the same precision, the
swept rule only reorders independent point updates.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import reductions as ored

pytestmark = pytest.mark.gpu

EULER, F64, F32C = 4, 0, 1
GAMMA = 1.4
BMAX = {F64: 128, F32C: 256}


def state(n, seed=0, cfl=0.2):
    """Periodic Sod-like state (Section 7's left/right states) plus a seeded smooth
    velocity and density perturbation, so that every minmod branch and both wave
    directions occur.  Returns (q of shape (n, 3), params)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    rho = np.where(left, 0.125, 1.0) * (1.0 + 0.05 * np.sin(2 * np.pi * (x + rng.uniform())))
    p = np.where(left, 0.1, 1.0)
    u = 0.2 * np.cos(2 * np.pi * (3 * x + rng.uniform()))
    q = np.stack([rho, rho * u, p / (GAMMA - 1.0) + 0.5 * rho * u * u], axis=1)
    dx = 1.0 / n
    return q, [cfl * dx, dx, GAMMA]


def to_device(q, dtype=F64):
    """(N, 3) FP64 state -> planar device layout (FP64: rho, m, E; F32C: hi of the three, then lo)."""
    import torch
    planar = np.ascontiguousarray(q.T).reshape(-1)
    if dtype == F64:
        return torch.tensor(planar, dtype=torch.float64, device="cuda")
    hi, lo = oracle.split_f32c(planar)
    return torch.tensor(np.concatenate([hi, lo]), dtype=torch.float32, device="cuda")


def from_device(t, n, dtype=F64):
    """Device state -> (N, 3) FP64 array, or (hi, lo) pair of (N, 3) float32 arrays."""
    a = t.cpu().numpy()
    if dtype == F64:
        return a.reshape(3, n).T
    return np.ascontiguousarray(a[:3 * n].reshape(3, n).T), np.ascontiguousarray(a[3 * n:].reshape(3, n).T)


def oracle_run(prm, q, nsteps, dtype=F64):
    if dtype == F64:
        return oracle.euler_advance(prm, q, nsteps)
    hi, lo = oracle.split_f32c(np.ascontiguousarray(q).reshape(-1))
    return oracle.euler_advance_f32c(prm, hi.reshape(-1, 3), lo.reshape(-1, 3), nsteps)


def run(sw, plan, q, nsteps, naive=False):
    import torch
    u = to_device(q, plan.dtype)
    (sw.swept_naive_advance if naive else sw.swept_advance)(plan, u, nsteps)
    torch.cuda.synchronize()
    return from_device(u, len(q), plan.dtype)


def assert_same(got, want):
    if isinstance(got, tuple):
        for g, w in zip(got, want):
            assert_same(g, w)
        return
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} values differ, first at {bad[:4].tolist()}"


def merged(x):
    return x if not isinstance(x, tuple) else x[0].astype(np.float64) + x[1].astype(np.float64)


CASES = [(d, B) for d in (F64, F32C) for B in (32, 64, 128, 256) if B <= BMAX[d]]


@pytest.mark.parametrize("dtype,B", CASES)
@pytest.mark.parametrize("diamond", [1, 2])      # per-window kernel, ring kernel
def test_swept_bit_exact_vs_oracle(cuda_lib, dtype, B, diamond):
    sw = cuda_lib
    N = 16 * B
    q, prm = state(N, B + diamond)
    plan = sw.swept_plan(N, 1, EULER, prm, dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, diamond)
    per_stage = plan.h // 4                     # time steps per stage (h levels)
    for nsteps in sorted({1, 2, per_stage - 1, per_stage, per_stage + 1, 3 * per_stage + 2}):
        if nsteps >= 1:
            assert_same(run(sw, plan, q, nsteps), oracle_run(prm, q, nsteps, dtype))


@pytest.mark.parametrize("dtype", [F64, F32C])
def test_naive_bit_exact_vs_oracle_ragged(cuda_lib, dtype):
    """N = 32*37 is not a multiple of the naive kernel's 127-point block."""
    sw = cuda_lib
    N = 32 * 37
    q, prm = state(N, 7)
    plan = sw.swept_plan(N, 1, EULER, prm, dtype, 32)
    for nsteps in (1, 2, 9):
        assert_same(run(sw, plan, q, nsteps, naive=True), oracle_run(prm, q, nsteps, dtype))


@pytest.mark.parametrize("dtype,B", [(F64, 32), (F64, 128), (F32C, 32), (F32C, 256)])
def test_single_window_is_its_own_neighbour(cuda_lib, dtype, B):
    sw = cuda_lib
    q, prm = state(B, 3)
    plan = sw.swept_plan(B, 1, EULER, prm, dtype, B)
    for nsteps in (1, B // 8, B // 4 + 3):
        assert_same(run(sw, plan, q, nsteps), oracle_run(prm, q, nsteps, dtype))


@pytest.mark.parametrize("dtype", [F64, F32C])
def test_zero_steps_and_uniform_state(cuda_lib, dtype):
    sw = cuda_lib
    N = 256
    q, prm = state(N, 1)
    plan = sw.swept_plan(N, 1, EULER, prm, dtype, 64)
    assert_same(run(sw, plan, q, 0), oracle_run(prm, q, 0, dtype))
    uni = np.tile([0.7, 0.35, 2.5], (N, 1))
    want = oracle_run(prm, uni, 0, dtype)
    assert_same(run(sw, plan, uni, 40), want)
    assert_same(run(sw, plan, uni, 40, naive=True), want)


@pytest.mark.parametrize("dtype,B", [(F64, 64), (F32C, 128)])
def test_full_size_swept_equals_naive_and_oracle_samples(cuda_lib, dtype, B):
    """N = 2^20 cells, 200 time steps (800 sub-timesteps), ring launch: swept == naive bit for
    bit; oracle values at sampled cells from their dependence cone; the three conserved totals
    kept to rounding; the compensated state within the FP32-flux bound of the FP64 oracle."""
    sw = cuda_lib
    N, nsteps = 1 << 20, 200
    q, prm = state(N, 11)
    plan = sw.swept_plan(N, 1, EULER, prm, dtype, B)
    got = run(sw, plan, q, nsteps)
    assert_same(got, run(sw, plan, q, nsteps, naive=True))
    half = 4 * nsteps + 4                      # 4 sub-timesteps of radius 1 per step
    rng = np.random.default_rng(0)
    for x in [0, N - 1, 31, 32, B - 1, B] + [int(v) for v in rng.integers(0, N, 3)]:
        idx = (x + np.arange(-half, half + 1)) % N
        want = oracle_run(prm, q[idx], nsteps, dtype)
        if dtype == F64:
            assert np.array_equal(got[x], want[half]), (x, got[x], want[half])
        else:
            assert np.array_equal(got[0][x], want[0][half]) and np.array_equal(got[1][x], want[1][half]), x
            ref = oracle.euler_advance(prm, q[idx], nsteps)[half]
            assert np.all(np.abs(merged(got)[x] - ref) <= 2e-4 * (np.abs(ref) + 1.0)), x
    vals = merged(got)
    for c in range(3):
        scale = math.fsum(np.abs(q[:, c])) + 1.0
        tol = 1e-12 if dtype == F64 else 1e-8
        assert abs(ored.total(vals[:, c]) - ored.total(q[:, c])) <= tol * scale


def test_reduce_on_a_component_block(cuda_lib):
    """swept_reduce over the momentum block (u + N) of an Euler state."""
    import torch
    sw = cuda_lib
    N = 4096
    q, prm = state(N, 5)
    plan = sw.swept_plan(N, 1, EULER, prm, F64, 64)
    u = to_device(q)
    got = sw.swept_reduce(plan, u[N:], sw.SWEPT_SUM).item()
    want = ored.total(q[:, 1])
    assert abs(got - want) <= 4 * np.finfo(float).eps * np.sum(np.abs(q[:, 1]))
    del torch


def test_adjoint_not_supported(cuda_lib):
    import torch
    sw = cuda_lib
    q, prm = state(256, 2)
    plan = sw.swept_plan(256, 1, EULER, prm, F64, 64)
    u = to_device(q)
    with pytest.raises(sw.SweptError) as e:
        sw.swept_adjoint(plan, u, u, 3)
    assert e.value.code == sw.SWEPT_ENOTSUP


@pytest.mark.parametrize("dtype,B", [(F64, 64), (F32C, 128)])
def test_streamed_ring(cuda_lib, dtype, B):
    """Streamed ring stages for the Euler equations (four sub-timesteps per step; the
    ring's two windows are at the same sub-timestep in every slot): 19 windows on 6 warps,
    up to 6 streamed stages, bit-exact against the oracle."""
    sw = cuda_lib
    N = 19 * B
    q, prm = state(N, 7 + B)
    plan = sw.swept_plan(N, 1, EULER, prm, dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, 2)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 6)
    per_stage = plan.h // 4
    for nsteps in (3 * per_stage, 7 * per_stage + 3):
        assert_same(run(sw, plan, q, nsteps), oracle_run(prm, q, nsteps, dtype))
