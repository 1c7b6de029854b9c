"""Persistent advance (SWEPT_OPT_PERSISTENT): every stage in one launch, windows synchronised by
device flags.  Bit-exact against the oracle for every schedule shape (a lone trapezoid and its
fill, full diamonds, a remainder), both stencils and the three precisions; plans it does not
apply to take the per-stage path with the same result."""
from __future__ import annotations

import numpy as np
import pytest

from tests.test_parity_gpu import HEAT, KS, F64, F32C, F32, params_of, initial, oracle_run, run_gpu, assert_same

pytestmark = pytest.mark.gpu

CASES = [(st, dt, B) for st in (HEAT, KS) for dt in (F64, F32C, F32) for B in (32, 64, 128, 256)
         if (B // 32) % (1 if st == HEAT else 2) == 0]


@pytest.mark.parametrize("stencil,dtype,B", CASES)
def test_persistent_bit_exact(cuda_lib, stencil, dtype, B):
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    N = 16 * B
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_PERSISTENT, 1)
    h = plan.h
    u0 = initial(stencil, N, 2000 + B)
    for nsteps in sorted({1, h - 1, h, h + 1, 2 * h, 5 * h + h // 2 + 1, 40 * h + 3}):
        got = run_gpu(sw, plan, u0, nsteps)
        assert sw.swept_plan_status(plan) == 0
        assert_same(plan, got, oracle_run(stencil, dtype, u0, nsteps))


def test_persistent_single_window_and_graph(cuda_lib):
    """One window (its own neighbour), and the persistent launch replayed from a CUDA graph."""
    sw = cuda_lib
    plan = sw.swept_plan(64, 1, HEAT, [0.25], F64, 64)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_PERSISTENT, 1)
    u0 = initial(HEAT, 64, 7)
    assert_same(plan, run_gpu(sw, plan, u0, 333), oracle_run(HEAT, F64, u0, 333))
    plan = sw.swept_plan(32 * 64, 1, HEAT, [0.25], F64, 64)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_PERSISTENT, 1)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
    u0 = initial(HEAT, 32 * 64, 8)
    want = oracle_run(HEAT, F64, u0, 1000)
    for _ in range(2):
        assert_same(plan, run_gpu(sw, plan, u0, 1000), want)
    assert sw.swept_plan_status(plan) == 0


def test_persistent_not_applicable_takes_stage_path(cuda_lib):
    """K = 16 (B = 512) is outside the persistent instantiations: the per-stage path runs."""
    sw = cuda_lib
    N = 8 * 512
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F32C, 512)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_PERSISTENT, 1)
    u0 = initial(HEAT, N, 9)
    assert_same(plan, run_gpu(sw, plan, u0, 1000), oracle_run(HEAT, F32C, u0, 1000))


def test_persistent_lost_message_times_out_and_gpu_stays_usable(cuda_lib):
    """A window whose publishes are dropped (a lost message): its neighbours' bounded waits run
    out, the status reads SWEPT_ETIMEOUT, and the next advance on the same context is exact."""
    import torch
    sw = cuda_lib
    N, B = 16 * 64, 64
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_PERSISTENT, 1)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIMEOUT_MS, 200)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, 5)
    u0 = initial(HEAT, N, 11)
    run_gpu(sw, plan, u0, 10 * plan.h + 3)
    assert sw.swept_plan_status(plan) == sw.SWEPT_ETIMEOUT
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, -1)
    got = run_gpu(sw, plan, u0, 10 * plan.h + 3)
    assert sw.swept_plan_status(plan) == 0
    assert_same(plan, got, oracle_run(HEAT, F64, u0, 10 * plan.h + 3))
    del torch
