"""GPU parity of the Euler-equations path (Section 7's scheme) against the oracle.

Swept stages (per-window and ring kernels) and the naive stepper must equal the
oracle's per-step stepping bit for bit: both evaluate the same expressions in
FP64, the swept rule only reorders independent point updates.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from oracle import reductions as ored

pytestmark = pytest.mark.gpu

EULER, F64 = 4, 0
GAMMA = 1.4


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


def to_device(q):
    import torch
    return torch.tensor(np.ascontiguousarray(q.T).reshape(-1), dtype=torch.float64, device="cuda")


def from_device(t, n):
    return t.cpu().numpy().reshape(3, n).T


def run(sw, plan, q, nsteps, naive=False):
    import torch
    u = to_device(q)
    (sw.swept_naive_advance if naive else sw.swept_advance)(plan, u, nsteps)
    torch.cuda.synchronize()
    return from_device(u, len(q))


def assert_same(got, want):
    bad = np.argwhere(got != want)
    assert bad.size == 0, f"{len(bad)} values differ, first at {bad[:4].tolist()}"


@pytest.mark.parametrize("B", [32, 64, 128])
@pytest.mark.parametrize("diamond", [1, 2])      # per-window kernel, ring kernel
def test_swept_bit_exact_vs_oracle(cuda_lib, B, diamond):
    sw = cuda_lib
    N = 16 * B
    q, prm = state(N, B + diamond)
    plan = sw.swept_plan(N, 1, EULER, prm, F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, diamond)
    per_stage = plan.h // 4                     # time steps per stage (h levels)
    for nsteps in sorted({1, 2, per_stage - 1, per_stage, per_stage + 1, 3 * per_stage + 2}):
        if nsteps >= 1:
            assert_same(run(sw, plan, q, nsteps), oracle.euler_advance(prm, q, nsteps))


def test_naive_bit_exact_vs_oracle_ragged(cuda_lib):
    """N = 32*37 is not a multiple of the naive kernel's 128-point block."""
    sw = cuda_lib
    N = 32 * 37
    q, prm = state(N, 7)
    plan = sw.swept_plan(N, 1, EULER, prm, F64, 32)
    for nsteps in (1, 2, 9):
        assert_same(run(sw, plan, q, nsteps, naive=True), oracle.euler_advance(prm, q, nsteps))


@pytest.mark.parametrize("B", [32, 128])
def test_single_window_is_its_own_neighbour(cuda_lib, B):
    sw = cuda_lib
    q, prm = state(B, 3)
    plan = sw.swept_plan(B, 1, EULER, prm, F64, B)
    for nsteps in (1, B // 8, B // 4 + 3):
        assert_same(run(sw, plan, q, nsteps), oracle.euler_advance(prm, q, nsteps))


def test_zero_steps_and_uniform_state(cuda_lib):
    sw = cuda_lib
    N = 256
    q, prm = state(N, 1)
    plan = sw.swept_plan(N, 1, EULER, prm, F64, 64)
    assert_same(run(sw, plan, q, 0), q)
    uni = np.tile([0.7, 0.35, 2.5], (N, 1))
    assert_same(run(sw, plan, uni, 40), uni)
    assert_same(run(sw, plan, uni, 40, naive=True), uni)


def test_full_size_swept_equals_naive_and_oracle_samples(cuda_lib):
    """N = 2^20 cells, 200 time steps (800 sub-timesteps), B = 64 ring launch: swept ==
    naive bit for bit; oracle values at sampled cells from their dependence cone; the
    three conserved totals kept to rounding."""
    import torch
    sw = cuda_lib
    N, nsteps = 1 << 20, 200
    q, prm = state(N, 11)
    plan = sw.swept_plan(N, 1, EULER, prm, F64, 64)
    got = run(sw, plan, q, nsteps)
    assert_same(got, run(sw, plan, q, nsteps, naive=True))
    half = 4 * nsteps + 4                      # 4 sub-timesteps of radius 1 per step
    rng = np.random.default_rng(0)
    for x in [0, N - 1, 31, 32, 63, 64] + [int(v) for v in rng.integers(0, N, 3)]:
        idx = (x + np.arange(-half, half + 1)) % N
        want = oracle.euler_advance(prm, q[idx], nsteps)[half]
        assert np.array_equal(got[x], want), (x, got[x], want)
    for c in range(3):
        scale = math.fsum(np.abs(q[:, c])) + 1.0
        assert abs(ored.total(got[:, c]) - ored.total(q[:, c])) <= 1e-12 * scale
    del torch


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
