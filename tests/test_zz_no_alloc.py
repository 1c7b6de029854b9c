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


def test_noalloc_rejects_oversize(cuda_lib):
    import torch
    sw = cuda_lib
    N = 2 * sw.SWEPT_NOALLOC_MAX_N
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    with pytest.raises(sw.SweptError) as ei:
        sw.swept_advance_noalloc(N, 0, [0.25], sw.SWEPT_F64, 512, u, 10)
    assert ei.value.code == sw.SWEPT_ETOOBIG
