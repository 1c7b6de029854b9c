"""Seeded synthetic inputs for the swept-rule workloads.

This module is the one place both the CPU oracle side and the GPU side take
their inputs from.  It draws random numbers and builds initial conditions;
it holds none of the stepping arithmetic (no stencil, no update rule).

Every generator is deterministic given its seed (NumPy PCG64 via
``numpy.random.default_rng``).  Arrays are FP64 on the host.

Workloads (sizes as run by the tests and the benchmark):

* heat_modes_1024   -- N = 1024, sum of sin/cos modes k = 1..8 with N(0,1)
                       amplitudes (heat, r = 0.25, 2000 steps, B = 32).
* heat_noise_modes  -- N = 2**24, uniform[-1, 1] white noise plus 16 low
                       modes with N(0,1) amplitudes (heat, r = 0.25, 20000 steps).
* ks_smoothed       -- N = 2**22, 0.1 * N(0,1) noise smoothed by ten
                       3-point averages (Kuramoto-Sivashinsky, dx = 0.5,
                       dt = 0.002, 50000 steps).
* batch_problems    -- 4096 problems, lengths log-uniform in [512, 262144]
                       rounded to a multiple of 512, step counts uniform in
                       [1000, 20000], half heat and half KS.
* ks_adjoint        -- N = 2**20 KS state for the adjoint, plus i.i.d. N(0,1)
                       finite-difference directions.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1504_01380

HEAT_R = 0.25
KS_DX = 0.5
KS_DT = 0.002


def seed_for(workload_index: int) -> int:
    """Seed of workload ``workload_index`` (0 = N=1024 heat, ... 4 = adjoint)."""
    return SEED_BASE + int(workload_index)


def _modes(n: int, kmax: int, rng: np.random.Generator) -> np.ndarray:
    """sum_{k=1..kmax} a_k sin(2 pi k i / n) + b_k cos(2 pi k i / n).

    Amplitudes are drawn as a_1, b_1, a_2, b_2, ... from N(0, 1).
    """
    amp = rng.standard_normal(2 * kmax)
    i = np.arange(n, dtype=np.float64)
    u = np.zeros(n, dtype=np.float64)
    for k in range(1, kmax + 1):
        ang = (2.0 * np.pi * k / n) * i
        u += amp[2 * (k - 1)] * np.sin(ang) + amp[2 * (k - 1) + 1] * np.cos(ang)
    return u


def mode_amplitudes(kmax: int, seed: int) -> np.ndarray:
    """The (a_1, b_1, ..., a_kmax, b_kmax) amplitudes ``heat_modes`` draws."""
    return np.random.default_rng(seed).standard_normal(2 * kmax)


def heat_modes(n: int = 1024, kmax: int = 8, seed: int | None = None) -> np.ndarray:
    """Initial condition made only of low Fourier modes k = 1..kmax."""
    rng = np.random.default_rng(seed_for(0) if seed is None else seed)
    return _modes(n, kmax, rng)


def heat_noise_modes(n: int = 1 << 24, kmax: int = 16, seed: int | None = None) -> np.ndarray:
    """uniform[-1, 1] white noise plus kmax low modes with N(0,1) amplitudes."""
    rng = np.random.default_rng(seed_for(1) if seed is None else seed)
    noise = rng.uniform(-1.0, 1.0, n)
    return noise + _modes(n, kmax, rng)


def smooth3(v: np.ndarray, times: int) -> np.ndarray:
    """``times`` periodic 3-point averages v_i <- ((v_{i-1} + v_i) + v_{i+1}) / 3."""
    v = np.array(v, dtype=np.float64, copy=True)
    for _ in range(times):
        v = ((np.roll(v, 1) + v) + np.roll(v, -1)) / 3.0
    return v


def ks_smoothed(n: int = 1 << 22, seed: int | None = None) -> np.ndarray:
    """0.1 * N(0,1) white noise smoothed by ten 3-point averages."""
    rng = np.random.default_rng(seed_for(2) if seed is None else seed)
    return 0.1 * smooth3(rng.standard_normal(n), 10)


def batch_problems(count: int = 4096, nmin: int = 512, nmax: int = 262144,
                   smin: int = 1000, smax: int = 20000, quantum: int = 512,
                   seed: int | None = None):
    """Ragged batch description: (kinds, lengths, steps) as int64 arrays.

    kinds: 0 = heat, 1 = KS; exactly half of the problems (a seeded
    permutation) are heat.  lengths are exp(U[ln nmin, ln nmax]) rounded to
    the nearest multiple of ``quantum`` (and clamped to [nmin, nmax]); steps
    are integers uniform in [smin, smax].
    """
    rng = np.random.default_rng(seed_for(3) if seed is None else seed)
    logn = rng.uniform(np.log(nmin), np.log(nmax), count)
    lengths = np.rint(np.exp(logn) / quantum).astype(np.int64) * quantum
    lengths = np.clip(lengths, nmin, nmax)
    steps = rng.integers(smin, smax + 1, count, dtype=np.int64)
    kinds = np.ones(count, dtype=np.int64)
    kinds[rng.permutation(count)[: count // 2]] = 0
    return kinds, lengths, steps


def batch_initial(kinds: np.ndarray, lengths: np.ndarray, seed: int | None = None,
                  seed_offsets=None) -> list:
    """One initial condition per batch problem (heat: noise + modes, KS: smoothed).

    Problem p of the full batch draws from seed base + 10000 + p; ``seed_offsets``
    gives the full-batch index of each listed problem when a subset is passed.
    """
    base = seed_for(3) if seed is None else seed
    idx = list(range(len(kinds))) if seed_offsets is None else list(seed_offsets)
    out = []
    for p, kind, n in zip(idx, kinds.tolist(), lengths.tolist()):
        s = base + 10_000 + p
        out.append(heat_noise_modes(n, 16, s) if kind == 0 else ks_smoothed(n, s))
    return out


def ks_cosine(n: int = 1 << 22, dx: float = KS_DX) -> np.ndarray:
    """The KS initial condition of the paper's Section 6 run: u(x, 0) = 2 cos(19 x / 128),
    sampled at x_i = i * dx.  (On a periodic grid of N*dx this leaves a small jump at the
    wrap, which the fourth-order dissipation smooths in the first steps.)"""
    x = np.arange(n, dtype=np.float64) * dx
    return 2.0 * np.cos(19.0 * x / 128.0)


def ks_adjoint_state(n: int = 1 << 20, seed: int | None = None) -> np.ndarray:
    """KS initial state for the adjoint workload (same recipe as ks_smoothed)."""
    return ks_smoothed(n, seed_for(4) if seed is None else seed)


def fd_direction(n: int, d: int, seed: int | None = None) -> np.ndarray:
    """Finite-difference direction number ``d``: i.i.d. N(0,1), not normalised."""
    base = seed_for(4) if seed is None else seed
    return np.random.default_rng(base + 1000 + d).standard_normal(n)


def uniform(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Plain uniform noise for small parity cases."""
    return np.random.default_rng(seed).uniform(lo, hi, n)
