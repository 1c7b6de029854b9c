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
