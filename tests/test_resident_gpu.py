"""The cluster-resident advance: every stage of a swept advance in one launch of one thread block
cluster (one warp per window, the edges in shared memory, read by the neighbouring windows through
distributed shared memory, a cluster barrier between stages), and the naive stepper's steps in one
cluster.  Bit-exact against the oracle; the per-stage launches give the same bits; plans that do
not fit one cluster fall back to the per-stage launches."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from tests.test_parity_gpu import HEAT, KS, F64, F32C, F32, params_of, initial, oracle_run, run_gpu, assert_same

pytestmark = pytest.mark.gpu

CASES = [(st, dt, B, nwin) for st in (HEAT, KS) for dt in (F64, F32C, F32) for B in (32, 64, 128)
         if (B // 32) % (1 if st == HEAT else 2) == 0 for nwin in (1, 3, 12, 32, 64)]


@pytest.mark.parametrize("stencil,dtype,B,nwin", CASES)
def test_resident_bit_exact(cuda_lib, stencil, dtype, B, nwin):
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    N = nwin * B
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    h = plan.h
    u0 = initial(stencil, N, 11000 + N + B)
    for nsteps in sorted({1, h - 1, h, h + 1, 2 * h, 3 * h + h // 2 + 1, 12 * h + 7}):
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))
        assert sw.swept_plan_last_advance(plan) == (1, 0, -1.0)


@pytest.mark.parametrize("stencil,dtype", [(HEAT, F64), (KS, F32C), (HEAT, F32)])
def test_resident_equals_stage_launches(cuda_lib, stencil, dtype):
    """SWEPT_OPT_RESIDENT = 0 runs the per-stage launches: the same bits, more launches."""
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    B, N = 64, 64 * 48
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    u0 = initial(stencil, N, 12000 + N)
    nsteps = 40 * plan.h + 3
    a = run_gpu(sw, plan, u0, nsteps)
    assert sw.swept_plan_last_advance(plan)[0] == 1
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RESIDENT, 0)
    b = run_gpu(sw, plan, u0, nsteps)
    assert sw.swept_plan_last_advance(plan)[0] > 1
    assert_same(plan, a, b)


def test_resident_runge_kutta(cuda_lib):
    from tests.test_rk2_gpu import prm, initial as rk2_initial, run as rk2_run
    sw = cuda_lib
    for st, B, N in ((2, 32, 32 * 32), (2, 64, 64 * 5), (3, 64, 64 * 32)):
        r = 1 if st == 2 else 2
        plan = sw.swept_plan(N, r, st, prm(st), F64, B)
        per = plan.h // 2
        u0 = rk2_initial(st, N, 12500 + N)
        for nsteps in (1, per, per + 1, 7 * per + 3):
            assert np.array_equal(rk2_run(sw, plan, u0, nsteps), oracle.advance_rk2_f64(st, prm(st), u0, nsteps))
            assert sw.swept_plan_last_advance(plan)[0] == 1


def test_resident_falls_back(cuda_lib):
    """33 and 65 windows (no cluster shape), a forced kernel choice, uneven tiles: the per-stage
    launches, same bits."""
    sw = cuda_lib
    for N, B, force in ((33 * 32, 32, False), (65 * 32, 32, False), (16 * 64, 64, True), (10 * 64 + 5, 64, False)):
        plan = sw.swept_plan(N, 1, HEAT, params_of(HEAT), F64, B)
        if force:
            sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_WINDOW)
        u0 = initial(HEAT, N, 13000 + N)
        nsteps = 5 * plan.h + 2
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(HEAT, F64, u0, nsteps))
        assert sw.swept_plan_last_advance(plan)[0] > 1


def test_resident_under_graph_capture(cuda_lib):
    import torch
    sw = cuda_lib
    N, B = 1024, 32
    plan = sw.swept_plan(N, 1, HEAT, params_of(HEAT), F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
    u0 = initial(HEAT, N, 14000)
    want = oracle_run(HEAT, F64, u0, 2000)
    src = torch.tensor(u0, device="cuda")
    u = src.clone()
    for _ in range(2):
        u.copy_(src)
        sw.swept_advance(plan, u, 2000)
        torch.cuda.synchronize()
        assert np.array_equal(u.cpu().numpy(), want)
    assert sw.swept_plan_last_advance(plan)[0] == 1


@pytest.mark.parametrize("stencil,dtype", [(st, dt) for st in (HEAT, KS) for dt in (F64, F32C, F32)])
def test_naive_resident_bit_exact(cuda_lib, stencil, dtype):
    """SWEPT_OPT_NAIVE_RESIDENT: the naive steps in one cluster (N = 64, 1000, 4096, 4100: split
    over at most 16 blocks; 1000 into 10 of 100, 4100 into 10 of 410), and N = 4099 (prime, more
    than one block's 4094 points) on the per-step launches; every case bit-exact against the
    oracle."""
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    for N in (64, 1000, 4096, 4100, 4099):
        plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, 0)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_NAIVE_RESIDENT, 1)
        u0 = initial(stencil, N, 15000 + N)
        for nsteps in (1, 2, 333):
            assert_same(plan, run_gpu(sw, plan, u0, nsteps, naive=True), oracle_run(stencil, dtype, u0, nsteps))
