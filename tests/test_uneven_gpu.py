"""Uneven tiles (N not a multiple of the tile width): the last windows are B + 32r wide.  Swept
advances bit-exact against the oracle for both stencils, the three single-step precisions,
several tile widths and mixes of regular and wide windows (none regular, one wide, several
wide), for step counts around every stage boundary."""
from __future__ import annotations

import pytest

from tests.test_parity_gpu import HEAT, KS, F64, F32C, F32, params_of, initial, oracle_run, run_gpu, assert_same

pytestmark = pytest.mark.gpu


def layouts(B, r):
    """(nreg, nwide) mixes -> N = nreg*B + nwide*(B + 32r)."""
    return [(n, w) for n, w in ((0, 1), (1, 1), (5, 1), (3, 2), (9, 4)) if w * 32 * r < B or w == 1 and n == 0]


CASES = [(st, dt, B, nreg, nwide) for st in (HEAT, KS) for dt in (F64, F32C, F32) for B in (32, 64, 128, 512)
         if (B // 32) % (1 if st == HEAT else 2) == 0
         for nreg, nwide in layouts(B, 1 if st == HEAT else 2)]


@pytest.mark.parametrize("stencil,dtype,B,nreg,nwide", CASES)
def test_uneven_bit_exact(cuda_lib, stencil, dtype, B, nreg, nwide):
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    N = nreg * B + nwide * (B + 32 * r)
    if N % B and (N % B) // (32 * r) != nwide:
        pytest.skip("layout not produced by this N")
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    h = plan.h
    u0 = initial(stencil, N, 3000 + N)
    for nsteps in sorted({1, h - 1, h, h + 1, 2 * h, 3 * h + h // 2 + 1}):
        if nsteps >= 1:
            assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))


def test_uneven_default_tile_for_a_prime_multiple(cuda_lib):
    """N = 32 * 1009: the default tile is 512 points with one 544-point window; 3000 steps."""
    sw = cuda_lib
    N = 32 * 1009
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F32C, 0)
    assert plan.B == 512
    u0 = initial(HEAT, N, 77)
    assert_same(plan, run_gpu(sw, plan, u0, 3000), oracle_run(HEAT, F32C, u0, 3000))
    assert_same(plan, run_gpu(sw, plan, u0, 3000, naive=True), oracle_run(HEAT, F32C, u0, 3000))


def test_uneven_adjoint_not_supported(cuda_lib):
    import torch
    sw = cuda_lib
    N = 128 + 192                         # one 128-point and one 192-point window
    plan = sw.swept_plan(N, 2, KS, params_of(KS), F64, 128)
    z = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(sw.SweptError) as e:
        sw.swept_adjoint(plan, z, z, 5)
    assert e.value.code == sw.SWEPT_ENOTSUP


@pytest.mark.parametrize("stencil,dtype,B,warps", [(HEAT, F32C, 128, 3), (HEAT, F64, 64, 0), (KS, F32C, 256, 2),
                                                   (KS, F64, 128, 0)])
def test_uneven_with_ring_for_the_regular_windows(cuda_lib, stencil, dtype, B, warps):
    """The regular windows' full diamonds on the ring kernel (forced; several run lengths), the
    wide windows alongside."""
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    nwide = max(1, (B // (32 * r)) - 1)
    N = 20 * B + nwide * (B + 32 * r)
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
    u0 = initial(stencil, N, 4000 + B)
    for nsteps in (4 * plan.h + 3, 6 * plan.h):
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))
