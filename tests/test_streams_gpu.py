"""The library on the caller's streams: captured into the caller's CUDA graph, two plans
advancing concurrently on two streams, and argument checks that reject a call before any
launch (misaligned state, a state tensor too small)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

HEAT, KS = 0, 1
F64, F32C = 0, 1
KS_PRM = [workloads.KS_DT, workloads.KS_DX]


def test_advance_captured_in_a_user_graph(cuda_lib):
    """torch.cuda.graph capture of swept_advance (its programmatic dependent launches
    included), replayed twice from a restored input: the oracle's bits both times."""
    import torch
    sw = cuda_lib
    N, B = 64 * 128, 128
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F64, B)
    nsteps = 3 * plan.h + 5
    u0 = workloads.uniform(N, 61)
    want = oracle.advance_f64(HEAT, [0.25], u0, nsteps)
    src = torch.tensor(u0, device="cuda")
    u = src.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sw.swept_advance(plan, u, nsteps)          # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sw.swept_advance(plan, u, nsteps)
    for _ in range(2):
        u.copy_(src)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(u.cpu().numpy(), want)


def test_two_plans_on_two_streams(cuda_lib):
    """A heat plan and a KS plan advanced at the same time on two streams."""
    import torch
    sw = cuda_lib
    N = 32 * 256
    ph = sw.swept_plan(N, 1, HEAT, [0.25], F64, 256)
    pk = sw.swept_plan(N, 2, KS, KS_PRM, F32C, 256)
    uh0 = workloads.uniform(N, 62)
    uk0 = workloads.ks_smoothed(N, 63) * 10
    hi, lo = oracle.split_f32c(uk0)
    uh = torch.tensor(uh0, device="cuda")
    uk = torch.tensor(np.concatenate([hi, lo]), device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s1):
        sw.swept_advance(ph, uh, 700, stream=s1)
    with torch.cuda.stream(s2):
        sw.swept_advance(pk, uk, 450, stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(uh.cpu().numpy(), oracle.advance_f64(HEAT, [0.25], uh0, 700))
    wh, wl = oracle.advance_f32c(KS, KS_PRM, hi, lo, 450)
    assert np.array_equal(uk.cpu().numpy(), np.concatenate([wh, wl]))


def test_misaligned_or_short_state_is_rejected(cuda_lib):
    import torch
    sw = cuda_lib
    N = 1024
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F64, 64)
    buf = torch.zeros(N + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(sw.SweptError) as e:
        sw.swept_advance(plan, buf[1:], 10)            # 8-byte offset: not 16-byte aligned
    assert e.value.code == sw.SWEPT_EINVAL
    with pytest.raises(ValueError):
        sw.swept_advance(plan, torch.zeros(N - 1, dtype=torch.float64, device="cuda"), 10)
    # the plan is still usable afterwards
    u0 = workloads.uniform(N, 64)
    u = torch.tensor(u0, device="cuda")
    sw.swept_advance(plan, u, 33)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), oracle.advance_f64(HEAT, [0.25], u0, 33))
