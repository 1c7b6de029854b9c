"""Ring-pipelined diamond kernel: bit-exact against the oracle for every split of windows.

The ring kernel streams a run of windows per warp; these tests force it on
small problems with 1 warp (one run over every window), 2 and 3 warps
(uneven runs) and one warp per window, for both stencils and precisions.
"""
from __future__ import annotations

import pytest

import oracle
from tests.test_parity_gpu import (CASES, assert_same, initial, oracle_run, params_of,
                                   run_gpu)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("stencil,dtype,B", CASES)
@pytest.mark.parametrize("warps", [1, 2, 3, 0])
def test_ring_bit_exact_vs_oracle(cuda_lib, stencil, dtype, B, warps):
    sw = cuda_lib
    r = 1 if stencil == 0 else 2
    h = B // (2 * r)
    nwin = 7                      # odd: uneven runs for 2 and 3 warps
    N = nwin * B
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps if warps else nwin)
    u0 = initial(stencil, N, 4000 + B)
    for nsteps in (3 * h, 4 * h + 1):       # 2 and 3 full diamond stages
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))


@pytest.mark.parametrize("stencil,dtype", [(0, 0), (1, 1)])
def test_window_and_ring_agree(cuda_lib, stencil, dtype):
    sw = cuda_lib
    r = 1 if stencil == 0 else 2
    B = 256
    N = 64 * B
    u0 = initial(stencil, N, 99)
    out = []
    for mode in (sw.SWEPT_DIAMOND_WINDOW, sw.SWEPT_DIAMOND_RING):
        plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, mode)
        out.append(run_gpu(sw, plan, u0, 10 * plan.h + 7))
    assert_same(plan, out[1], out[0])


# The last three are the streamed kernels the benchmark times: heat compensated at B = 1024
# (the headline) and KS compensated at B = 512 and 1024 (the KS report's tile sweep).
STREAM_CASES = [(0, 0, 64), (0, 1, 128), (0, 2, 32), (1, 0, 128), (1, 1, 256), (1, 2, 64),
                (0, 1, 1024), (1, 1, 512), (1, 1, 1024)]


@pytest.mark.parametrize("stencil,dtype,B", STREAM_CASES)
@pytest.mark.parametrize("warps", [1, 4, 10])
def test_streamed_ring_many_stages(cuda_lib, stencil, dtype, B, warps):
    """Streamed ring (every full diamond of the advance in one launch; a warp's last slot of a
    stage fills its first window of the next, and the run drifts one window right every
    second stage): 31 windows over 1, 4 and 10 warps (runs of 31, 7-8 and 3-4 windows),
    2 to 9 streamed stages, bit-exact against the oracle and against one ring launch per
    stage (SWEPT_OPT_STREAM = 0)."""
    sw = cuda_lib
    r = 1 if stencil == 0 else 2
    h = B // (2 * r)
    nwin = 31
    N = nwin * B
    u0 = initial(stencil, N, 5000 + B + warps)
    plans = []
    for stream in (1, 0):
        plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_STREAM, stream)
        plans.append(plan)
    for nsteps in (3 * h, 5 * h + 3, 10 * h + h // 2):
        got = run_gpu(sw, plans[0], u0, nsteps)
        assert_same(plans[0], got, oracle_run(stencil, dtype, u0, nsteps))
        assert_same(plans[0], got, run_gpu(sw, plans[1], u0, nsteps))
        assert sw.swept_plan_status(plans[0]) == 0


def test_streamed_ring_automatic_choice(cuda_lib):
    """With the automatic kernel choice, an advance over more windows than four per SM
    streams its diamonds; the bits equal the per-stage ring launches and the naive stepper."""
    import torch
    sw = cuda_lib
    B = 256
    nwin = 4 * torch.cuda.get_device_properties(0).multi_processor_count + 37
    N = nwin * B
    u0 = initial(0, N, 77)
    outs = []
    for stream in (1, 0):
        plan = sw.swept_plan(N, 1, 0, params_of(0), 1, B)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_STREAM, stream)
        outs.append(run_gpu(sw, plan, u0, 6 * plan.h + 11))
        assert sw.swept_plan_status(plan) == 0
    assert_same(plan, outs[0], outs[1])
    assert_same(plan, outs[0], run_gpu(sw, plan, u0, 6 * plan.h + 11, naive=True))


def test_last_advance_counts_and_ring_time(cuda_lib):
    """swept_plan_last_advance: an advance of q*h + rem levels enqueues the first triangle,
    one streamed ring launch for the q - 1 diamonds, the last fill and the remainder stage
    (q + 1 launches, q - 1 ring launches, without streaming); SWEPT_OPT_TIME_RING gives the
    ring launches' device time, -1 without it."""
    import torch
    sw = cuda_lib
    B = 256
    nwin = 4 * torch.cuda.get_device_properties(0).multi_processor_count + 5
    N = nwin * B
    u0 = initial(0, N, 3)
    plan = sw.swept_plan(N, 1, 0, params_of(0), 1, B)
    h = plan.h
    nsteps = 7 * h + 9                     # q = 7, rem = 9
    run_gpu(sw, plan, u0, nsteps)
    assert sw.swept_plan_last_advance(plan) == (4, 1, -1.0)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIME_RING, 1)
    run_gpu(sw, plan, u0, nsteps)
    n, nr, ms = sw.swept_plan_last_advance(plan)
    assert (n, nr) == (4, 1) and ms > 0.0
    sw.swept_plan_set(plan, sw.SWEPT_OPT_STREAM, 0)
    run_gpu(sw, plan, u0, nsteps)
    n, nr, ms = sw.swept_plan_last_advance(plan)
    assert (n, nr) == (9, 6) and ms > 0.0
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIME_RING, 0)
    run_gpu(sw, plan, u0, 2 * h)           # q = 2: one diamond stage, timing off
    assert sw.swept_plan_last_advance(plan)[2] == -1.0
    plan.destroy()


@pytest.mark.parametrize("dtype", [0, 1])
def test_streamed_lost_progress_times_out_and_gpu_stays_usable(cuda_lib, dtype):
    """A warp of a streamed ring launch whose slot counter is never published (a lost
    message, SWEPT_OPT_DROP_WINDOW): its left neighbour's bounded wait runs out, the
    status reads SWEPT_ETIMEOUT, and the next advance on the same context is exact."""
    sw = cuda_lib
    B = 128
    N = 24 * B
    plan = sw.swept_plan(N, 1, 0, params_of(0), dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 4)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIMEOUT_MS, 100)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, 2)
    u0 = initial(0, N, 13)
    nsteps = 8 * plan.h + 3
    run_gpu(sw, plan, u0, nsteps)
    assert sw.swept_plan_status(plan) == sw.SWEPT_ETIMEOUT
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, -1)
    got = run_gpu(sw, plan, u0, nsteps)
    assert sw.swept_plan_status(plan) == 0
    assert_same(plan, got, oracle_run(0, dtype, u0, nsteps))
