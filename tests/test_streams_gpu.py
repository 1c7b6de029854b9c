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


def _streamed_plan(sw, N, radius, stencil, prm, dtype, B, warps):
    """A plan whose advances stream their diamond stages (ring forced, explicit warps)."""
    plan = sw.swept_plan(N, radius, stencil, prm, dtype, B)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_DIAMOND, sw.SWEPT_DIAMOND_RING)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_RING_WARPS, warps)
    return plan


def test_streamed_advance_in_graphs(cuda_lib):
    """The streamed ring launch is cooperative: captured by SWEPT_OPT_GRAPH and by the
    caller's torch.cuda.graph, replayed twice each, the oracle's bits every time."""
    import torch
    sw = cuda_lib
    N, B = 40 * 256, 256
    u0 = workloads.uniform(N, 64)
    nsteps = 6 * (B // 2) + 7
    want = oracle.advance_f64(HEAT, [0.25], u0, nsteps)
    src = torch.tensor(u0, device="cuda")
    plan = _streamed_plan(sw, N, 1, HEAT, [0.25], F64, B, 9)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
    u = src.clone()
    for _ in range(2):
        u.copy_(src)
        sw.swept_advance(plan, u, nsteps)
        torch.cuda.synchronize()
        assert np.array_equal(u.cpu().numpy(), want)
    assert sw.swept_plan_status(plan) == 0
    plan2 = _streamed_plan(sw, N, 1, HEAT, [0.25], F64, B, 9)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        sw.swept_advance(plan2, u, nsteps)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sw.swept_advance(plan2, u, nsteps)
    for _ in range(2):
        u.copy_(src)
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(u.cpu().numpy(), want)
    assert sw.swept_plan_status(plan2) == 0


def test_two_streamed_advances_at_once(cuda_lib):
    """Two plans whose automatic choice streams, each over every resident warp slot (at
    least 3 windows for each of 64 warps per SM), advanced at the same time on two streams:
    a cooperative launch is all co-resident or waits, so neither times out, and both give
    the naive stepper's bits."""
    import torch
    sw = cuda_lib
    B = 256
    nwin = 3 * 64 * torch.cuda.get_device_properties(0).multi_processor_count
    N = nwin * B
    ph = sw.swept_plan(N, 1, HEAT, [0.25], F32C, B)
    pk = sw.swept_plan(N, 2, KS, KS_PRM, F32C, B)
    uh0 = workloads.uniform(N, 65)
    uk0 = workloads.ks_smoothed(N, 66) * 10
    states = []
    for u0 in (uh0, uk0):
        hi, lo = oracle.split_f32c(u0)
        states.append(torch.tensor(np.concatenate([hi, lo]), device="cuda"))
    want = []
    for plan, st, n in ((ph, states[0], 9 * 128 + 3), (pk, states[1], 9 * 64 + 5)):
        ref = st.clone()
        sw.swept_naive_advance(plan, ref, n)
        want.append(ref)
    uh, uk = states[0].clone(), states[1].clone()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    for _ in range(3):
        with torch.cuda.stream(s1):
            uh.copy_(states[0])
            sw.swept_advance(ph, uh, 9 * 128 + 3, stream=s1)
        with torch.cuda.stream(s2):
            uk.copy_(states[1])
            sw.swept_advance(pk, uk, 9 * 64 + 5, stream=s2)
        torch.cuda.synchronize()
        assert sw.swept_plan_status(ph) == 0 and sw.swept_plan_status(pk) == 0
        assert torch.equal(uh, want[0]) and torch.equal(uk, want[1])
    assert sw.swept_plan_last_advance(ph)[1] == 1 and sw.swept_plan_last_advance(pk)[1] == 1


def test_automatic_stream_choice_under_graph_capture(cuda_lib):
    """With the automatic kernel choice the streamed launch is decided (an occupancy query)
    while SWEPT_OPT_GRAPH captures the advance: the replayed graph streams its diamonds
    and gives the naive stepper's bits, twice."""
    import torch
    sw = cuda_lib
    B = 256
    nwin = 4 * torch.cuda.get_device_properties(0).multi_processor_count + 24
    N = nwin * B
    u0 = workloads.uniform(N, 67)
    hi, lo = oracle.split_f32c(u0)
    src = torch.tensor(np.concatenate([hi, lo]), device="cuda")
    plan = sw.swept_plan(N, 1, HEAT, [0.25], F32C, B)
    nsteps = 7 * plan.h + 3
    ref = src.clone()
    sw.swept_naive_advance(plan, ref, nsteps)
    sw.swept_plan_set(plan, sw.SWEPT_OPT_GRAPH, 1)
    u = src.clone()
    for _ in range(2):
        u.copy_(src)
        sw.swept_advance(plan, u, nsteps)
        torch.cuda.synchronize()
        assert torch.equal(u, ref)
        assert sw.swept_plan_status(plan) == 0
    assert sw.swept_plan_last_advance(plan)[1] == 1      # counts of the captured advance
