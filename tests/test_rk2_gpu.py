"""Two-stage Runge-Kutta (two sub-timesteps with a forwarded variable): bit-exact vs the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

HEAT_RK2, KS_RK2 = 2, 3
KS_PRM = [workloads.KS_DT, workloads.KS_DX]


def prm(st):
    return [workloads.HEAT_R] if st == HEAT_RK2 else KS_PRM


def initial(st, n, seed):
    return workloads.uniform(n, seed) if st == HEAT_RK2 else workloads.ks_smoothed(n, seed) * 10


def run(sw, plan, u0, nsteps, naive=False):
    import torch
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    (sw.swept_naive_advance if naive else sw.swept_advance)(plan, u, nsteps)
    torch.cuda.synchronize()
    return u.cpu().numpy()


CASES = [(st, B) for st in (HEAT_RK2, KS_RK2) for B in (32, 64, 128, 256, 512)
         if (B // 32) % (1 if st == HEAT_RK2 else 2) == 0]


@pytest.mark.parametrize("st,B", CASES)
@pytest.mark.parametrize("mode", [1, 2])           # per-window / ring diamonds
def test_rk2_swept_bit_exact(cuda_lib, st, B, mode):
    sw = cuda_lib
    r = 1 if st == HEAT_RK2 else 2
    h = B // (2 * r)                               # levels per stage; a step is 2 levels
    N = 7 * B
    plan = sw.swept_plan(N, r, st, prm(st), sw.SWEPT_F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, mode)
    if mode == 2:
        sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 3)
    u0 = initial(st, N, 300 + B)
    for nsteps in sorted({1, h // 2 - 1, h // 2, h // 2 + 1, h, 2 * h + 3}):
        if nsteps < 1:
            continue
        want = oracle.advance_rk2_f64(st, prm(st), u0, nsteps)
        assert np.array_equal(run(sw, plan, u0, nsteps), want), nsteps


@pytest.mark.parametrize("st", [HEAT_RK2, KS_RK2])
def test_rk2_naive_bit_exact(cuda_lib, st):
    sw = cuda_lib
    r = 1 if st == HEAT_RK2 else 2
    N = 64 * 37 * 4
    plan = sw.swept_plan(N, r, st, prm(st), sw.SWEPT_F64, 64)
    u0 = initial(st, N, 8)
    for nsteps in (1, 2, 7, 40):
        assert np.array_equal(run(sw, plan, u0, nsteps, naive=True),
                              oracle.advance_rk2_f64(st, prm(st), u0, nsteps))


def test_rk2_rejects_compensated(cuda_lib):
    sw = cuda_lib
    with pytest.raises(sw.SweptError) as ei:
        sw.swept_plan(1024, 2, KS_RK2, KS_PRM, sw.SWEPT_F32C, 256)
    assert ei.value.code == sw.SWEPT_ENOTSUP


def test_ks_rk2_paper_ic_full_size(cuda_lib):
    """KS by RK2 from u = 2cos(19x/128), N = 2^22, 1000 steps: swept == naive, oracle at sampled points."""
    sw = cuda_lib
    N, nsteps = 1 << 22, 1000
    plan = sw.swept_plan(N, 2, KS_RK2, KS_PRM, sw.SWEPT_F64, 256)
    u0 = workloads.ks_cosine(N)
    got = run(sw, plan, u0, nsteps)
    assert np.array_equal(got, run(sw, plan, u0, nsteps, naive=True))
    for x in (0, N - 1, 255, 256, 3_000_001):
        half = 2 * (2 * nsteps) + 2
        idx = (x + np.arange(-half, half + 1)) % N
        seg = oracle.advance_rk2_f64(KS_RK2, KS_PRM, u0[idx], nsteps)
        assert got[x] == seg[half], x


@pytest.mark.parametrize("st,B", [(HEAT_RK2, 64), (KS_RK2, 128)])
def test_rk2_streamed_ring(cuda_lib, st, B):
    """Streamed ring stages (one launch for every full diamond) for the two-stage scheme:
    23 windows on 5 warps, up to 7 streamed stages, bit-exact against the oracle."""
    sw = cuda_lib
    r = 1 if st == HEAT_RK2 else 2
    h = B // (2 * r)
    N = 23 * B
    plan = sw.swept_plan(N, r, st, prm(st), sw.SWEPT_F64, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, 2)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, 5)
    u0 = initial(st, N, 900 + B)
    for nsteps in (2 * h, 4 * h + 1):              # 4h and 8h + 2 levels
        want = oracle.advance_rk2_f64(st, prm(st), u0, nsteps)
        assert np.array_equal(run(sw, plan, u0, nsteps), want), nsteps
