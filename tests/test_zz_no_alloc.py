"""swept_advance_noalloc against swept_advance, through the C ABI.

The no-allocation entry point serves callers that may not call cudaMalloc
(a host that hands out a fixed device-memory budget, or code that must not
synchronise the device through an allocation).  It keeps its edge scratch
in one fixed array inside the library that every call reuses, so two calls
in a row must each give exactly swept_advance's result: the second call must
not see anything the first one left in the array.  This file is collected
last so that a failure here comes after every other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

KS_PRM = [workloads.KS_DT, workloads.KS_DX]


def _state(sw, dtype, u0):
    import torch
    t = torch.tensor(u0, dtype=torch.float64, device="cuda")
    return t if dtype == sw.SWEPT_F64 else sw.swept_f32c_split(t)


@pytest.mark.parametrize("stencil,dtype,B,N", [
    (0, 0, 512, 1 << 20),      # heat, FP64, the largest size the array allows
    (0, 1, 256, 1 << 16),      # heat, compensated FP32
    (1, 0, 256, 1 << 18),      # KS, FP64
    (1, 1, 128, 1 << 14),      # KS, compensated FP32
])
def test_noalloc_matches_swept_advance_twice(cuda_lib, stencil, dtype, B, N):
    import torch
    sw = cuda_lib
    prm = [0.25] if stencil == 0 else KS_PRM
    radius = 1 if stencil == 0 else 2
    plan = sw.swept_plan(N, radius, stencil, prm, dtype, B)
    h = plan.h
    runs = [(workloads.uniform(N, 31) if stencil == 0 else 10 * workloads.ks_smoothed(N, 31), 3 * h + 5),
            (workloads.uniform(N, 32) if stencil == 0 else 10 * workloads.ks_smoothed(N, 32), 2 * h)]
    for u0, nsteps in runs:             # two calls in a row on the shared array
        ref = _state(sw, dtype, u0)
        sw.swept_advance(plan, ref, nsteps)
        got = _state(sw, dtype, u0)
        sw.swept_advance_noalloc(N, stencil, prm, dtype, B, got, nsteps)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), "no-allocation result differs from swept_advance"
    plan.destroy()


@pytest.mark.parametrize("stencil,dtype,B", [(0, 0, 64), (0, 1, 128), (1, 0, 128), (1, 1, 64)])
def test_noalloc_schedule_edges(cuda_lib, stencil, dtype, B):
    """Step counts at the ends of the schedule, two calls in a row each: fewer than h (no full
    triangle: a trapezoid and its fill), exactly h and h + 1 (one triangle, then the last fill
    with and without a remainder stage), and 0 (a no-op that leaves u untouched)."""
    import torch
    sw = cuda_lib
    prm = [0.25] if stencil == 0 else KS_PRM
    radius = 1 if stencil == 0 else 2
    N = 5 * B
    plan = sw.swept_plan(N, radius, stencil, prm, dtype, B)
    h = plan.h
    for i, nsteps in enumerate((h // 2, 1, h, h + 1, 0)):
        u0 = workloads.uniform(N, 40 + i) if stencil == 0 else 10 * workloads.ks_smoothed(N, 40 + i)
        ref = _state(sw, dtype, u0)
        sw.swept_advance(plan, ref, nsteps)
        for _ in range(2):
            got = _state(sw, dtype, u0)
            sw.swept_advance_noalloc(N, stencil, prm, dtype, B, got, nsteps)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), f"nsteps={nsteps}: no-allocation result differs"
        if nsteps == 0:
            assert torch.equal(got, _state(sw, dtype, u0))
    plan.destroy()


def test_noalloc_rejects_what_it_does_not_take(cuda_lib):
    """Uneven tiles (N not a multiple of B), the plain binary32 state and the other stencils
    are the plan's, not this entry point's: each is refused before anything runs."""
    import torch
    sw = cuda_lib
    u = torch.zeros(2 * 1056, dtype=torch.float64, device="cuda")
    before = u.clone()
    cases = [(1056, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F64, 64),        # 1056 = 16.5 tiles of 64
             (1024, sw.SWEPT_HEAT, [0.25], sw.SWEPT_F32, 64),        # plain binary32
             (1024, sw.SWEPT_HEAT_RK2, [0.25], sw.SWEPT_F64, 64),    # Runge-Kutta
             (1024, sw.SWEPT_KS, KS_PRM, sw.SWEPT_F64, 32)]          # K = 1 < radius 2
    for N, stencil, prm, dtype, B in cases:
        with pytest.raises(sw.SweptError) as ei:
            sw.swept_advance_noalloc(N, stencil, prm, dtype, B, u, 10)
        assert ei.value.code == sw.SWEPT_EINVAL, (N, stencil, dtype, B)
    torch.cuda.synchronize()
    assert torch.equal(u, before)


def test_noalloc_rejects_oversize(cuda_lib):
    import torch
    sw = cuda_lib
    N = 2 * sw.SWEPT_NOALLOC_MAX_N
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(sw.SweptError) as ei:
        sw.swept_advance_noalloc(N, 0, [0.25], sw.SWEPT_F64, 512, u, 10)
    assert ei.value.code == sw.SWEPT_ETOOBIG
