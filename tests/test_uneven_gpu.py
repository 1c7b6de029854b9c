"""Uneven tiles (N not a multiple of the tile width): the last windows are B + 32r wide.  Swept
advances bit-exact against the oracle for heat and KS in the three single-step precisions, the
Runge-Kutta stencils and the Euler equations, several tile widths and mixes of regular and wide
windows (none regular, one wide, several wide), for step counts around every stage boundary."""
from __future__ import annotations

import numpy as np
import pytest

from tests.test_parity_gpu import HEAT, KS, F64, F32C, F32, params_of, initial, oracle_run, run_gpu, assert_same

pytestmark = pytest.mark.gpu


def layouts(B, r):
    """(nreg, nwide) mixes -> N = nreg*B + nwide*(B + 32r)."""
    return [(n, w) for n, w in ((0, 1), (1, 1), (5, 1), (3, 2), (9, 4)) if w * 32 * r < B or w == 1 and n == 0]


CASES = [(st, dt, B, nreg, nwide) for st in (HEAT, KS) for dt in (F64, F32C, F32) for B in (32, 64, 128, 512, 1024)
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


# Any N: the last wide window takes what is left (B + 1 .. B + 32r points), so N need not be
# a multiple of 32r.  Primes, N just above one tile, several wide windows with an odd last one.
ANY_N = [(HEAT, F64, 32, 1009), (HEAT, F32C, 64, 357), (HEAT, F32, 128, 4099), (HEAT, F64, 512, 512 * 3 + 7),
         (KS, F64, 128, 1009), (KS, F32C, 64, 100), (KS, F32C, 256, 3001), (KS, F32, 64, 65),
         (HEAT, F32C, 1024 // 2, 32 * 1009 + 7)]


@pytest.mark.parametrize("stencil,dtype,B,N", ANY_N)
def test_any_n_bit_exact(cuda_lib, stencil, dtype, B, N):
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    h = plan.h
    u0 = initial(stencil, N, 7000 + N)
    for nsteps in sorted({1, h - 1, h, h + 1, 2 * h, 3 * h + h // 2 + 1}):
        if nsteps >= 1:
            assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))


@pytest.mark.parametrize("stencil,N,B", [(HEAT, 1009, 128), (HEAT, 50, 32), (KS, 1009, 128), (KS, 100, 64),
                                         (HEAT, 32 * 1009 + 7, 512)])
def test_any_n_default_tile(cuda_lib, stencil, N, B):
    """B = 0 picks the widest tile that fits N (a prime N, N below twice the smallest tile):
    swept == oracle and naive == oracle."""
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), F32C, 0)
    assert plan.B == B
    u0 = initial(stencil, N, 8000 + N)
    nsteps = 3 * plan.h + 5
    want = oracle_run(stencil, F32C, u0, nsteps)
    assert_same(plan, run_gpu(sw, plan, u0, nsteps), want)
    assert_same(plan, run_gpu(sw, plan, u0, nsteps, naive=True), want)


def test_any_n_runge_kutta_and_euler(cuda_lib):
    """The last window of any width for the Runge-Kutta pairs and the Euler point states."""
    import oracle
    from tests.test_rk2_gpu import prm, initial as rk2_initial, run as rk2_run
    from tests.test_euler_gpu import state, run as euler_run, oracle_run as euler_oracle, assert_same as euler_same
    sw = cuda_lib
    for st, B, N in ((2, 64, 64 * 4 + 33), (3, 128, 128 * 3 + 71)):
        r = 1 if st == 2 else 2
        plan = sw.swept_plan(N, r, st, prm(st), F64, B)
        u0 = rk2_initial(st, N, 9000 + N)
        for nsteps in (1, plan.h // 2, 3 * (plan.h // 2) + 2):
            assert np.array_equal(rk2_run(sw, plan, u0, nsteps), oracle.advance_rk2_f64(st, prm(st), u0, nsteps))
    for dtype, B, N in ((F64, 64, 64 * 3 + 45), (F32C, 128, 128 * 4 + 101)):
        q, prm_e = state(N, 9100 + N)
        plan = sw.swept_plan(N, 1, 4, prm_e, dtype, B)
        per_stage = plan.h // 4
        for nsteps in (1, per_stage, 3 * per_stage + 1):
            euler_same(euler_run(sw, plan, q, nsteps), euler_oracle(prm_e, q, nsteps, dtype))


@pytest.mark.parametrize("N,B,ring", [(128 + 192, 128, False), (1009, 128, False), (20 * 128 + 3 * 192 + 77, 128, True),
                                      (13 * 256 + 101, 256, True), (64 * 40 + 31, 64, False),
                                      (9 * 1024 + 130, 1024, True)])
def test_uneven_adjoint_matches_oracle(cuda_lib, N, B, ring):
    """The KS adjoint on uneven tiles of any N: the forward pass's checkpoints come from the
    regular windows' kernels and from the wide windows' trapezoid loads, the transposed sweep
    runs the regular windows (per window or on the ring) and then the wide ones; bit-exact
    against the oracle's discrete adjoint, for step counts around the stage boundaries."""
    import oracle
    import torch
    sw = cuda_lib
    u0 = initial(KS, N, 9500 + N)
    lam = initial(HEAT, N, 9600 + N)
    plan = sw.swept_plan(N, 2, KS, params_of(KS), F64, B)
    if ring:
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 3)
    h = plan.h
    for nsteps, K in ((3 * h + 5, 1), (6 * h, 2), (h - 1, 64), (9 * h + h // 2, 1)):
        got = sw.swept_adjoint(plan, torch.tensor(u0, device="cuda"), torch.tensor(lam, device="cuda"),
                               nsteps, K).cpu().numpy()
        want = oracle.adjoint_f64(KS, params_of(KS), u0, lam, nsteps)
        assert np.array_equal(got, want), (N, B, nsteps, K, np.flatnonzero(got != want)[:8])


# Full diamond stages of an uneven tiling on the ring: with SWEPT_OPT_STREAM every one of them in
# one streamed launch (the regular windows' runs and one warp per wide window, per-window stage
# counters), without it one launch per stage running the ring over the regular windows and the wide
# windows together.  Forced at small N (the ring kernel with a few warps, or with its automatic
# warp count), automatic where the regular windows outnumber four per SM.  (stencil, dtype, B, N,
# ring warps: None = automatic choice of kernel, 0 = ring with automatic warps)
JOINT = [(HEAT, F64, 128, 128 * 25 + 100, 3), (HEAT, F32C, 128, 128 * 12 + 33, 0), (HEAT, F32, 64, 64 * 15 + 7, 2),
         (KS, F64, 128, 128 * 20 + 100, 4), (KS, F32C, 512, 512 * 12 + 300, 3), (KS, F32, 256, 256 * 10 + 130, 0),
         (HEAT, F32C, 32, 32 * 700 + 7, None), (KS, F32C, 64, 64 * 700 + 50, None),
         (HEAT, F32C, 1024, 1024 * 12 + 100, 3), (KS, F64, 1024, 1024 * 10 + 200, 0)]


@pytest.mark.parametrize("stream", [1, 0])
@pytest.mark.parametrize("stencil,dtype,B,N,warps", JOINT)
def test_uneven_ring_and_wide_windows(cuda_lib, stencil, dtype, B, N, warps, stream):
    sw = cuda_lib
    r = 1 if stencil == HEAT else 2
    plan = sw.swept_plan(N, r, stencil, params_of(stencil), dtype, B)
    if warps is not None:
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_STREAM, stream)
    h = plan.h
    u0 = initial(stencil, N, 9700 + N)
    for nsteps in (h + 1, 4 * h, 5 * h + h // 2 + 1):
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(stencil, dtype, u0, nsteps))
        assert sw.swept_plan_status(plan) == 0
    # 5h + h/2 + 1 steps: the triangle, 4 diamonds, the last V-fill with the remainder's
    # trapezoid and the remainder's V-fill (two launches for each of those three); the
    # diamonds in one streamed launch, or one launch each
    assert sw.swept_plan_last_advance(plan)[:2] == ((1 + 3 * 2, 1) if stream else (4 + 3 * 2, 4))


def test_uneven_joint_launch_runge_kutta(cuda_lib):
    """The joint launch for the Runge-Kutta pairs (forced ring, two and three warps)."""
    import oracle
    from tests.test_rk2_gpu import prm, initial as rk2_initial, run as rk2_run
    sw = cuda_lib
    for st, B, N, warps in ((2, 64, 64 * 30 + 20, 2), (3, 128, 128 * 20 + 70, 3)):
        r = 1 if st == 2 else 2
        plan = sw.swept_plan(N, r, st, prm(st), F64, B)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
        per = plan.h // 2
        u0 = rk2_initial(st, N, 9800 + N)
        for nsteps in (per + 1, 4 * per + 3):
            assert np.array_equal(rk2_run(sw, plan, u0, nsteps), oracle.advance_rk2_f64(st, prm(st), u0, nsteps))


def test_uneven_streamed_lost_window_times_out(cuda_lib):
    """A window of the streamed uneven launch that never publishes (SWEPT_OPT_DROP_WINDOW, here
    a wide one and a regular one) makes its readers' bounded waits run out: the advance reports
    SWEPT_ETIMEOUT, and the next advance on the same plan, without the fault, is bit-exact."""
    sw = cuda_lib
    N, B = 128 * 20 + 100, 128
    plan = sw.swept_plan(N, 1, HEAT, params_of(HEAT), F32C, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 3)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_TIMEOUT_MS, 100)
    u0 = initial(HEAT, N, 9900)
    nsteps = 6 * plan.h + 3
    nwin = N // B
    for drop in (nwin - 1, 5):
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, drop)
        run_gpu(sw, plan, u0, nsteps)
        assert sw.swept_plan_status(plan) == sw.SWEPT_ETIMEOUT
        sw.swept_plan_set(plan, sw.SWEPT_OPT_DROP_WINDOW, -1)
        assert_same(plan, run_gpu(sw, plan, u0, nsteps), oracle_run(HEAT, F32C, u0, nsteps))
        assert sw.swept_plan_status(plan) == 0
