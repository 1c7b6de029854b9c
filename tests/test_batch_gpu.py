"""Batched persistent launch: every problem bit-exact against the oracle.

Also: the queue with a single thread block (every dependency waited on),
a message lost on the host side (one item never publishes) ending in
SWEPT_ETIMEOUT with the GPU still usable, the 4096-problem workload
checked on sampled problems, and the naive batched stepper (one launch per
step over the active problems) bit-exact against the oracle and the swept
launch.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads
from tests.test_parity_gpu import oracle_point

pytestmark = pytest.mark.gpu

KS_PRM = (workloads.KS_DT, workloads.KS_DX)


def prm(stencil):
    return (workloads.HEAT_R, 0.0) if stencil == 0 else KS_PRM


def build_pool(batch, states, dtype):
    """Host bytes of the pool with every problem's initial state at its offset."""
    buf = np.zeros(batch.pool_bytes, dtype=np.uint8)
    for off, u0 in zip(batch.offsets, states):
        n = len(u0)
        if dtype == 0:
            buf[off:off + 8 * n] = np.frombuffer(np.ascontiguousarray(u0, np.float64).tobytes(), np.uint8)
        else:
            hi, lo = oracle.split_f32c(u0)
            buf[off:off + 8 * n] = np.frombuffer(np.concatenate([hi, lo]).tobytes(), np.uint8)
    return buf


def read_state(buf, off, n, dtype):
    raw = buf[off:off + 8 * n].tobytes()
    if dtype == 0:
        return np.frombuffer(raw, np.float64)
    a = np.frombuffer(raw, np.float32)
    return a[:n], a[n:]


def run_batch(sw, problems, states, dtype, B_heat=512, B_ks=512, grid=None):
    import torch
    batch = sw.swept_batch_plan([(st, n, ns, prm(st)) for st, n, ns in problems], dtype, B_heat, B_ks)
    if grid:
        sw.swept_batch_set(batch, sw.SWEPT_BOPT_GRID, grid)
    pool = torch.tensor(build_pool(batch, states, dtype), device="cuda")
    sw.swept_advance_batch(batch, pool)
    status = sw.swept_batch_status(batch)
    return batch, pool.cpu().numpy(), status


def expect(stencil, dtype, u0, nsteps):
    if dtype == 0:
        return oracle.advance_f64(stencil, prm(stencil)[: 1 if stencil == 0 else 2], u0, nsteps)
    hi, lo = oracle.split_f32c(u0)
    return oracle.advance_f32c(stencil, prm(stencil)[: 1 if stencil == 0 else 2], hi, lo, nsteps)


def same(got, want, dtype):
    if dtype == 0:
        return np.array_equal(got, want)
    return np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


SMALL = [(0, 512, 1), (1, 1024, 300), (0, 2048, 255), (1, 512, 128), (0, 1536, 700),
         (1, 2560, 129), (0, 512, 0), (1, 3072, 1000), (0, 4096, 257), (1, 1024, 64),
         (0, 1024, 511), (1, 512, 7),
         (0, 36864, 1100), (1, 18432, 777)]     # several runs of windows per stage


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("bh,bk", [(512, 512), (256, 256), (512, 256)])
def test_batch_bit_exact(cuda_lib, dtype, bh, bk):
    sw = cuda_lib
    states = [workloads.uniform(n, 10 + i) if st == 0 else 10 * workloads.ks_smoothed(n, 10 + i)
              for i, (st, n, ns) in enumerate(SMALL)]
    batch, out, status = run_batch(sw, SMALL, states, dtype, bh, bk)
    assert status == 0
    for (st, n, ns), off, u0 in zip(SMALL, batch.offsets, states):
        assert same(read_state(out, off, n, dtype), expect(st, dtype, u0, ns), dtype), (st, n, ns)


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("run_len", [1, 3, 32])
def test_batch_run_lengths(cuda_lib, dtype, run_len):
    """SWEPT_BOPT_RUN_LEN: items of 1 window (every ring run a single window), 3 (runs cut
    mid-problem) and 32 (longer than most problems): bit-exact against the oracle; the
    default run length is one of 32, 16, 8."""
    import torch
    sw = cuda_lib
    states = [workloads.uniform(n, 60 + i) if st == 0 else 10 * workloads.ks_smoothed(n, 60 + i)
              for i, (st, n, ns) in enumerate(SMALL)]
    batch = sw.swept_batch_plan([(st, n, ns, prm(st)) for st, n, ns in SMALL], dtype, 256, 512)
    assert batch.info()["run_len"] in (8, 16, 32)
    sw.swept_batch_set(batch, sw.SWEPT_BOPT_RUN_LEN, run_len)
    assert batch.info()["run_len"] == run_len
    pool = torch.tensor(build_pool(batch, states, dtype), device="cuda")
    sw.swept_advance_batch(batch, pool)
    assert sw.swept_batch_status(batch) == 0
    out = pool.cpu().numpy()
    for (st, n, ns), off, u0 in zip(SMALL, batch.offsets, states):
        assert same(read_state(out, off, n, dtype), expect(st, dtype, u0, ns), dtype), (st, n, ns)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_naive_bit_exact(cuda_lib, dtype):
    """Per-step stepping over the ragged batch (odd and even step counts, a problem with none)."""
    import torch
    sw = cuda_lib
    states = [workloads.uniform(n, 30 + i) if st == 0 else 10 * workloads.ks_smoothed(n, 30 + i)
              for i, (st, n, ns) in enumerate(SMALL)]
    batch = sw.swept_batch_plan([(st, n, ns, prm(st)) for st, n, ns in SMALL], dtype, 256, 512)
    pool = torch.tensor(build_pool(batch, states, dtype), device="cuda")
    sw.swept_batch_naive_advance(batch, pool)
    out = pool.cpu().numpy()
    for (st, n, ns), off, u0 in zip(SMALL, batch.offsets, states):
        assert same(read_state(out, off, n, dtype), expect(st, dtype, u0, ns), dtype), (st, n, ns)
    # the same pool through the swept launch: identical bytes
    pool2 = torch.tensor(build_pool(batch, states, dtype), device="cuda")
    sw.swept_advance_batch(batch, pool2)
    assert sw.swept_batch_status(batch) == 0
    assert np.array_equal(pool2.cpu().numpy(), out)


@pytest.mark.parametrize("dtype", [0, 1])
def test_batch_single_block(cuda_lib, dtype):
    """One block of 4 warps: most items wait on their neighbours."""
    sw = cuda_lib
    probs = [(0, 4096, 600), (1, 2048, 400), (0, 512, 300), (0, 20480, 900)]
    states = [workloads.uniform(n, 50 + i) if st == 0 else 10 * workloads.ks_smoothed(n, 50 + i)
              for i, (st, n, ns) in enumerate(probs)]
    batch, out, status = run_batch(sw, probs, states, dtype, grid=1)
    assert status == 0
    for (st, n, ns), off, u0 in zip(probs, batch.offsets, states):
        assert same(read_state(out, off, n, dtype), expect(st, dtype, u0, ns), dtype)


def test_batch_lost_message_times_out_and_gpu_stays_usable(cuda_lib):
    import torch
    sw = cuda_lib
    probs = [(0, 8192, 2000), (1, 4096, 1000)]
    states = [workloads.uniform(8192, 1), 10 * workloads.ks_smoothed(4096, 2)]
    batch = sw.swept_batch_plan([(st, n, ns, prm(st)) for st, n, ns in probs], 1)
    info = batch.info()
    sw.swept_batch_set(batch, sw.SWEPT_BOPT_TIMEOUT_S, 0.05)
    assert info["stages"] >= 2
    sw.swept_batch_set(batch, sw.SWEPT_BOPT_DROP_ITEM, 0)   # a stage-0 item: stage 1 waits on it
    pool = torch.tensor(build_pool(batch, states, 1), device="cuda")
    sw.swept_advance_batch(batch, pool)
    assert sw.swept_batch_status(batch) == sw.SWEPT_ETIMEOUT
    # the context is intact: the same batch without the drop gives the right answer
    sw.swept_batch_set(batch, sw.SWEPT_BOPT_DROP_ITEM, -1)
    pool = torch.tensor(build_pool(batch, states, 1), device="cuda")
    sw.swept_advance_batch(batch, pool)
    assert sw.swept_batch_status(batch) == 0
    out = pool.cpu().numpy()
    for (st, n, ns), off, u0 in zip(probs, batch.offsets, states):
        assert same(read_state(out, off, n, 1), expect(st, 1, u0, ns), 1)


def test_batch_4096_problems_sampled(cuda_lib):
    """The ragged 4096-problem workload: sampled problems and points against the oracle."""
    import torch
    sw = cuda_lib
    kinds, lengths, steps = workloads.batch_problems()
    rng = np.random.default_rng(7)
    problems = [(int(k), int(n), int(s)) for k, n, s in zip(kinds, lengths, steps)]
    batch = sw.swept_batch_plan([(st, n, ns, prm(st)) for st, n, ns in problems], 1)
    pick = sorted(set(rng.choice(len(problems), 6, replace=False).tolist()
                      + [int(np.argmin(lengths)), int(np.argmax(lengths))]))
    # full-pool initial state is large; only sampled problems get real data, the rest seeded noise
    buf = np.zeros(batch.pool_bytes, dtype=np.uint8)
    states = {}
    for i in pick:
        st, n, ns = problems[i]
        u0 = workloads.heat_noise_modes(n, 16, 9000 + i) if st == 0 else workloads.ks_smoothed(n, 9000 + i)
        states[i] = u0
        hi, lo = oracle.split_f32c(u0)
        off = batch.offsets[i]
        buf[off:off + 8 * n] = np.frombuffer(np.concatenate([hi, lo]).tobytes(), np.uint8)
    pool = torch.tensor(buf, device="cuda")
    sw.swept_advance_batch(batch, pool)
    assert sw.swept_batch_status(batch) == 0
    assert batch.info()["run_len"] in (8, 16, 32)
    out = pool.cpu().numpy()
    for i in pick:
        st, n, ns = problems[i]
        got = read_state(out, batch.offsets[i], n, 1)
        u0 = states[i]
        if n * ns <= 2e8:
            assert same(got, expect(st, 1, u0, ns), 1), (i, st, n, ns)
        else:
            for x in (0, n - 1, int(rng.integers(0, n))):
                want = oracle_point(st, 1, u0, x, ns)
                assert got[0][x] == want[0] and got[1][x] == want[1], (i, x)


def test_batch_graph_and_direct_launch_agree(cuda_lib):
    """A mid-size ragged batch (256 problems of the 4096-problem recipe, fewer steps), launched
    directly and through the captured graph: identical results, both complete."""
    import torch
    sw = cuda_lib
    kinds, lengths, steps = workloads.batch_problems(256, 512, 65536, 500, 3000)
    problems = [(int(k), int(n), int(s), prm(int(k))) for k, n, s in zip(kinds, lengths, steps)]
    out = []
    for graph in (0, 1):
        batch = sw.swept_batch_plan(problems, 1, 256, 512)
        sw.swept_batch_set(batch, sw.SWEPT_BOPT_GRAPH, graph)
        buf = np.zeros(batch.pool_bytes, dtype=np.uint8)
        rng = np.random.default_rng(3)
        for off, (st, n, ns, _) in zip(batch.offsets, problems):
            hi, lo = oracle.split_f32c(rng.uniform(-1, 1, n))
            buf[off:off + 8 * n] = np.frombuffer(np.concatenate([hi, lo]).tobytes(), np.uint8)
        pool = torch.tensor(buf, device="cuda")
        sw.swept_advance_batch(batch, pool)
        assert sw.swept_batch_status(batch) == 0
        out.append(pool.cpu().numpy())
    assert np.array_equal(out[0], out[1])
