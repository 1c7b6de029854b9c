"""Pins of the CPU oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed-form
Fourier decay/growth factors, invariants of the schemes (conservation,
maximum principle, translation and reflection symmetry), the PDE's
textbook difference formulas evaluated in exact rational arithmetic, IEEE
rounding emulated on rationals, and a literal simulation of the swept stages.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle.swept_bruteforce import swept_simulate
from tests import exact_arith as X

EPS = np.finfo(np.float64).eps
HEAT, KS = oracle.HEAT, oracle.KS
KS_PRM = (workloads.KS_DT, workloads.KS_DX)


def ks_consts64(dt, dx):
    dx2 = dx * dx
    return -(dt / (4.0 * dx)), -(dt / dx2), -(dt / (dx2 * dx2))


# --------------------------------------------------------------------------
# Heat: closed forms (the step is diagonal in the Fourier basis)
# --------------------------------------------------------------------------

def heat_gain(k, n, r):
    """Per-step factor of Fourier mode k: g_k = 1 - 4 r sin^2(pi k / n)."""
    return 1.0 - 4.0 * r * np.sin(np.pi * k / n) ** 2


@pytest.mark.parametrize("k", [1, 3, 17, 100, 256])
def test_heat_single_mode_decay(k):
    n, r, nsteps = 512, 0.25, 300
    i = np.arange(n)
    u0 = np.cos(2 * np.pi * k * i / n)
    got = oracle.advance_f64(HEAT, [r], u0, nsteps)
    want = heat_gain(k, n, r) ** nsteps * u0
    # FP64 rounding: a few ulps per step of a quantity bounded by max|u0|
    assert np.max(np.abs(got - want)) <= 8 * nsteps * EPS * np.max(np.abs(u0)) + 1e-300


def test_heat_r025_gain_is_cos_squared():
    n = 64
    k = np.arange(n)
    assert np.allclose(heat_gain(k, n, 0.25), np.cos(np.pi * k / n) ** 2, atol=1e-15)


@pytest.mark.parametrize("r", [0.25, 0.1, 0.5])
def test_heat_spectral_propagation(r):
    """The 1024-point modes workload against exact Fourier propagation of the same u0."""
    n, nsteps = 1024, 2000
    u0 = workloads.heat_modes(n, 8)
    got = oracle.advance_f64(HEAT, [r], u0, nsteps)
    k = np.arange(n // 2 + 1)
    want = np.fft.irfft(np.fft.rfft(u0) * heat_gain(k, n, r) ** nsteps, n)
    assert np.max(np.abs(got - want)) <= 8 * nsteps * EPS * np.max(np.abs(u0))


def test_heat_modes_workload_closed_form():
    """u^n = sum_k g_k^n (a_k sin + b_k cos), the amplitudes drawn by the generator."""
    n, r, nsteps = 1024, 0.25, 2000
    u0 = workloads.heat_modes(n, 8)
    amp = workloads.mode_amplitudes(8, workloads.seed_for(0))
    i = np.arange(n)
    want = np.zeros(n)
    for k in range(1, 9):
        g = heat_gain(k, n, r) ** nsteps
        ang = 2 * np.pi * k * i / n
        want += g * (amp[2 * k - 2] * np.sin(ang) + amp[2 * k - 1] * np.cos(ang))
    got = oracle.advance_f64(HEAT, [r], u0, nsteps)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(u0))


def test_heat_linearity():
    n, r = 300, 0.25
    a = workloads.uniform(n, 11)
    b = workloads.uniform(n, 12)
    alpha, beta = 0.75, -1.5
    lhs = oracle.advance_f64(HEAT, [r], alpha * a + beta * b, 50)
    rhs = alpha * oracle.advance_f64(HEAT, [r], a, 50) + beta * oracle.advance_f64(HEAT, [r], b, 50)
    assert np.max(np.abs(lhs - rhs)) <= 1e-14 * 200


@pytest.mark.parametrize("r", [0.25, 0.5, 0.37])
def test_heat_maximum_principle(r):
    u0 = workloads.uniform(777, 5)
    u = oracle.advance_f64(HEAT, [r], u0, 400)
    d = 4 * EPS * np.max(np.abs(u0))
    assert u.min() >= u0.min() - d and u.max() <= u0.max() + d


def test_heat_unstable_beyond_half():
    """r > 1/2 amplifies the k = N/2 mode (|g| > 1): the bound r <= 1/2 is sharp."""
    n = 64
    u0 = np.cos(np.pi * np.arange(n))        # k = n/2
    u = oracle.advance_f64(HEAT, [0.6], u0, 10)
    assert np.max(np.abs(u)) > 2.0


# --------------------------------------------------------------------------
# Invariants shared by both schemes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("stencil,prm,u0", [
    (HEAT, [0.25], workloads.uniform(1000, 1)),
    (KS, KS_PRM, workloads.ks_smoothed(1024, 7)),
])
def test_conservation(stencil, prm, u0):
    """The discrete sum is conserved: every difference term telescopes."""
    nsteps = 500
    u = oracle.advance_f64(stencil, prm, u0, nsteps)
    scale = math.fsum(np.abs(u0)) + math.fsum(np.abs(u))
    assert abs(math.fsum(u) - math.fsum(u0)) <= 4 * nsteps * EPS * scale


@pytest.mark.parametrize("stencil,prm", [(HEAT, [0.25]), (KS, KS_PRM)])
@pytest.mark.parametrize("shift", [1, 5, 33, 250])
def test_translation_equivariance(stencil, prm, shift):
    u0 = workloads.ks_smoothed(256, 3) if stencil == KS else workloads.uniform(256, 3)
    a = oracle.advance_f64(stencil, prm, np.roll(u0, shift), 37)
    b = np.roll(oracle.advance_f64(stencil, prm, u0, 37), shift)
    assert np.array_equal(a, b)


def test_heat_reflection_symmetry():
    u0 = workloads.uniform(200, 9)
    a = oracle.advance_f64(HEAT, [0.3], u0[::-1], 41)
    b = oracle.advance_f64(HEAT, [0.3], u0, 41)[::-1]
    assert np.array_equal(a, b)


def test_ks_odd_reflection_symmetry():
    """u(x) -> -u(-x) maps KS solutions to KS solutions; the scheme keeps it bit for bit."""
    u0 = workloads.ks_smoothed(256, 4) * 10
    a = oracle.advance_f64(KS, KS_PRM, -u0[::-1], 80)
    b = -oracle.advance_f64(KS, KS_PRM, u0, 80)[::-1]
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# KS against the PDE
# --------------------------------------------------------------------------

def ks_textbook_exact(u, i, dt, dx):
    """u_i + dt*(-(u^2/2)_x - u_xx - u_xxxx) with the textbook central differences, exact."""
    n = len(u)
    q = [Fraction(u[(i + k) % n]) for k in range(-2, 3)]
    dt, dx = Fraction(dt), Fraction(dx)
    flux_x = (q[3] ** 2 / 2 - q[1] ** 2 / 2) / (2 * dx)
    u_xx = (q[1] - 2 * q[2] + q[3]) / dx ** 2
    u_xxxx = (q[0] - 4 * q[1] + 6 * q[2] - 4 * q[3] + q[4]) / dx ** 4
    return q[2] + dt * (-flux_x - u_xx - u_xxxx)


@pytest.mark.parametrize("dx,dt", [(0.5, 0.002), (0.3, 0.0005), (1.0, 0.01)])
def test_ks_step_matches_pde_differences(dx, dt):
    u = workloads.ks_smoothed(64, 21) * 20.0
    got = oracle.step_f64(KS, [dt, dx], u)
    for i in range(len(u)):
        want = float(ks_textbook_exact(u, i, dt, dx))
        # a few roundings of terms bounded by |u| + dt*(|u u_x| + |u_xx| + |u_xxxx|)
        scale = abs(u[i]) + dt * (4 * max(abs(u)) ** 2 / dx + 4 * max(abs(u)) / dx ** 2
                                  + 16 * max(abs(u)) / dx ** 4)
        assert abs(got[i] - want) <= 16 * EPS * scale


def test_heat_step_matches_pde_differences():
    u = workloads.uniform(50, 2)
    r = 0.3
    got = oracle.step_f64(HEAT, [r], u)
    for i in range(50):
        q = [Fraction(u[(i + k) % 50]) for k in (-1, 0, 1)]
        want = float(q[1] + Fraction(r) * (q[0] - 2 * q[1] + q[2]))
        assert abs(got[i] - want) <= 8 * EPS * 3


@pytest.mark.parametrize("k", [1, 40, 128, 200, 255])
def test_ks_linear_mode_growth(k):
    """Small amplitude: mode k is scaled by 1 + dt*(4s/dx^2 - 16 s^2/dx^4), s = sin^2(pi k/N)."""
    n = 512
    dt, dx = KS_PRM
    A = 1e-10
    u0 = A * np.cos(2 * np.pi * k * np.arange(n) / n)
    u1 = oracle.step_f64(KS, KS_PRM, u0)
    s = np.sin(np.pi * k / n) ** 2
    g = 1 + dt * (4 * s / dx ** 2 - 16 * s ** 2 / dx ** 4)
    assert np.max(np.abs(u1 - g * u0)) <= 1e-9 * A


def test_ks_nonlinear_term_closed_form():
    """u = A sin(th j): the flux difference adds a dt/(4dx) A^2 sin(2th) sin(2 th j) (negated)."""
    n, k = 256, 5
    dt, dx = KS_PRM
    A = 3.0
    th = 2 * np.pi * k / n
    j = np.arange(n)
    u0 = A * np.sin(th * j)
    u1 = oracle.step_f64(KS, KS_PRM, u0)
    s = np.sin(th / 2) ** 2
    lin = 1 + dt * (4 * s / dx ** 2 - 16 * s ** 2 / dx ** 4)
    want = lin * u0 - dt / (4 * dx) * A ** 2 * np.sin(2 * th) * np.sin(2 * th * j)
    assert np.max(np.abs(u1 - want)) <= 1e-13 * A


# --------------------------------------------------------------------------
# IEEE rounding of every operation (rational emulation)
# --------------------------------------------------------------------------

def exact_step64(stencil, prm, u):
    n = len(u)
    out = []
    if stencil == HEAT:
        r = prm[0]
        for i in range(n):
            um, u0, up = u[i - 1], u[i], u[(i + 1) % n]
            s = X.add64(um, up)
            w = X.sub64(s, X.mul64(2.0, u0))
            out.append(X.fma64(r, w, u0))
    else:
        a, b, e = ks_consts64(*prm)
        for i in range(n):
            v = [u[(i + k) % n] for k in range(-2, 3)]
            Gm, Gp = X.mul64(v[1], v[1]), X.mul64(v[3], v[3])
            wm = X.sub64(X.add64(v[0], v[2]), X.mul64(2.0, v[1]))
            w0 = X.sub64(X.add64(v[1], v[3]), X.mul64(2.0, v[2]))
            wp = X.sub64(X.add64(v[2], v[4]), X.mul64(2.0, v[3]))
            D = X.sub64(X.add64(wm, wp), X.mul64(2.0, w0))
            t = X.sub64(Gp, Gm)
            out.append(X.fma64(e, D, X.fma64(b, w0, X.fma64(a, t, v[2]))))
    return np.array(out)


def exact_step32c(stencil, prm, hi, lo):
    n = len(hi)
    ho, lout = [], []
    if stencil == HEAT:
        r32 = X.r32(Fraction(prm[0]))
    else:
        a, b, e = (X.r32(Fraction(c)) for c in ks_consts64(*prm))
    for i in range(n):
        if stencil == HEAT:
            hm, h0, hp = float(hi[i - 1]), float(hi[i]), float(hi[(i + 1) % n])
            w = X.add32(X.sub32(hm, h0), X.sub32(hp, h0))
            y = X.fma32(r32, w, float(lo[i]))
        else:
            v = [float(hi[(i + k) % n]) for k in range(-2, 3)]
            wm = X.add32(X.sub32(v[0], v[1]), X.sub32(v[2], v[1]))
            w0 = X.add32(X.sub32(v[1], v[2]), X.sub32(v[3], v[2]))
            wp = X.add32(X.sub32(v[2], v[3]), X.sub32(v[4], v[3]))
            D = X.add32(X.sub32(wm, w0), X.sub32(wp, w0))
            t = X.mul32(X.sub32(v[3], v[1]), X.add32(v[3], v[1]))
            y = X.fma32(e, D, X.fma32(b, w0, X.fma32(a, t, float(lo[i]))))
        h, l = X.two_sum32(float(hi[i]), y)
        ho.append(h)
        lout.append(l)
    return np.array(ho, dtype=np.float32), np.array(lout, dtype=np.float32)


@pytest.mark.parametrize("stencil,prm,scale", [
    (HEAT, [0.25], 1.0), (HEAT, [0.1], 1.0), (KS, KS_PRM, 5.0), (KS, (0.0013, 0.7), 5.0)])
@pytest.mark.parametrize("n", [8, 13, 32])
def test_single_step_f64_ieee_exact(stencil, prm, scale, n):
    u = workloads.uniform(n, 100 + n) * scale
    assert np.array_equal(oracle.step_f64(stencil, prm, u), exact_step64(stencil, prm, u))


@pytest.mark.parametrize("stencil,prm,scale", [
    (HEAT, [0.25], 1.0), (HEAT, [0.1], 1.0), (KS, KS_PRM, 5.0), (KS, (0.0013, 0.7), 5.0)])
@pytest.mark.parametrize("n", [8, 21, 32])
def test_single_step_f32c_ieee_exact(stencil, prm, scale, n):
    u = workloads.uniform(n, 200 + n) * scale
    hi, lo = oracle.split_f32c(u)
    ho, lout = oracle.step_f32c(stencil, prm, hi, lo)
    eh, el = exact_step32c(stencil, prm, hi, lo)
    assert np.array_equal(ho, eh) and np.array_equal(lout, el)


def exact_step32(stencil, prm, u):
    """The FP64 expressions with every operation rounded to binary32 (rational emulation)."""
    n = len(u)
    u = [float(x) for x in u]
    out = []
    if stencil == HEAT:
        r = X.r32(Fraction(prm[0]))
        for i in range(n):
            s = X.add32(u[i - 1], u[(i + 1) % n])
            w = X.sub32(s, X.mul32(2.0, u[i]))
            out.append(X.fma32(r, w, u[i]))
    else:
        a, b, e = (X.r32(Fraction(c)) for c in ks_consts64(*prm))
        for i in range(n):
            v = [u[(i + k) % n] for k in range(-2, 3)]
            Gm, Gp = X.mul32(v[1], v[1]), X.mul32(v[3], v[3])
            wm = X.sub32(X.add32(v[0], v[2]), X.mul32(2.0, v[1]))
            w0 = X.sub32(X.add32(v[1], v[3]), X.mul32(2.0, v[2]))
            wp = X.sub32(X.add32(v[2], v[4]), X.mul32(2.0, v[3]))
            D = X.sub32(X.add32(wm, wp), X.mul32(2.0, w0))
            t = X.sub32(Gp, Gm)
            out.append(X.fma32(e, D, X.fma32(b, w0, X.fma32(a, t, v[2]))))
    return np.array(out, dtype=np.float32)


@pytest.mark.parametrize("stencil,prm,scale", [
    (HEAT, [0.25], 1.0), (HEAT, [0.1], 1.0), (KS, KS_PRM, 5.0), (KS, (0.0013, 0.7), 5.0)])
@pytest.mark.parametrize("n", [8, 19, 32])
def test_single_step_f32_ieee_exact(stencil, prm, scale, n):
    u = (workloads.uniform(n, 300 + n) * scale).astype(np.float32)
    assert np.array_equal(oracle.step_f32(stencil, prm, u), exact_step32(stencil, prm, u))


def test_plain_f32_error_and_compensation_gain():
    """Heat, 3000 steps: the plain binary32 scheme stays within its rounding-growth bound of FP64
    (3000 steps x a few 2^-24 relative), and the compensated state is more than 10x closer."""
    n, r, nsteps = 4096, 0.25, 3000
    u0 = workloads.heat_noise_modes(n, 16, 77)
    ref = oracle.advance_f64(HEAT, [r], u0, nsteps)
    v = oracle.advance_f32(HEAT, [r], u0.astype(np.float32), nsteps)
    err_p = np.max(np.abs(v.astype(np.float64) - ref)) / np.max(np.abs(u0))
    hi, lo = oracle.split_f32c(u0)
    hi, lo = oracle.advance_f32c(HEAT, [r], hi, lo, nsteps)
    err_c = np.max(np.abs(oracle.merge_f32c(hi, lo) - ref)) / np.max(np.abs(u0))
    assert 1e-8 < err_p <= 4 * nsteps * 2.0 ** -24
    assert err_p > 10 * err_c


def test_split_merge_exact():
    u = workloads.uniform(1000, 8) * 1e3
    hi, lo = oracle.split_f32c(u)
    for x, h, l in zip(u[:200], hi[:200], lo[:200]):
        assert float(h) == X.r32(Fraction(x))
        assert float(l) == X.r32(Fraction(x) - Fraction(float(h)))
    m = oracle.merge_f32c(hi, lo)
    # hi + lo carries 48 bits: |u - merge| <= 2^-48 |u|
    assert np.max(np.abs(m - u) / np.abs(u)) <= 2.0 ** -47


def test_two_sum_pair_is_exact_sum():
    """After a step, hi' + lo' equals hi + y exactly (TwoSum is error-free)."""
    u = workloads.uniform(64, 31)
    hi, lo = oracle.split_f32c(u)
    ho, lout = oracle.step_f32c(HEAT, [0.25], hi, lo)
    for i in range(64):
        hm, h0, hp = float(hi[i - 1]), float(hi[i]), float(hi[(i + 1) % 64])
        w = X.add32(X.sub32(hm, h0), X.sub32(hp, h0))
        y = X.fma32(0.25, w, float(lo[i]))
        assert Fraction(float(ho[i])) + Fraction(float(lout[i])) == Fraction(float(hi[i])) + Fraction(y)


# --------------------------------------------------------------------------
# Compensated FP32 against FP64
# --------------------------------------------------------------------------

def test_f32c_heat_error_bound_and_compensation_gain():
    """Heat, N=4096, 3000 steps: compensated FP32 stays within 1e-6 of FP64; plain FP32 does not."""
    n, r, nsteps = 4096, 0.25, 3000
    u0 = workloads.heat_noise_modes(n, 16, 77)
    ref = oracle.advance_f64(HEAT, [r], u0, nsteps)
    hi, lo = oracle.split_f32c(u0)
    hi, lo = oracle.advance_f32c(HEAT, [r], hi, lo, nsteps)
    err_c = np.max(np.abs(oracle.merge_f32c(hi, lo) - ref)) / np.max(np.abs(u0))
    # plain FP32 with r = 1/4: r*w is exact, so fl(u + r w) equals the fused form
    v = u0.astype(np.float32)
    for _ in range(nsteps):
        s = np.roll(v, 1) + np.roll(v, -1)
        w = s - np.float32(2) * v
        v = v + np.float32(r) * w
    err_p = np.max(np.abs(v.astype(np.float64) - ref)) / np.max(np.abs(u0))
    assert err_c <= 1e-6
    assert err_p > 10 * err_c


def test_f32c_smooth_field_no_drift():
    """Smooth data, 20000 steps: the compensated state tracks the exact solution to ~1e-6.

    This is the case where cancellation in a sum-form second difference
    (fl(h[i-1] + h[i+1]) - 2h[i]) drifts by |u| 2^-24 per step; the difference form does not.
    """
    n, r, nsteps = 2048, 0.25, 20000
    i = np.arange(n)
    u0 = 2.5 + 10.0 * np.sin(2 * np.pi * 3 * i / n) + 0.3 * np.cos(2 * np.pi * 40 * i / n)
    k = np.arange(n // 2 + 1)
    exact = np.fft.irfft(np.fft.rfft(u0) * heat_gain(k, n, r) ** nsteps, n)
    hi, lo = oracle.split_f32c(u0)
    hi, lo = oracle.advance_f32c(HEAT, [r], hi, lo, nsteps)
    err = np.max(np.abs(oracle.merge_f32c(hi, lo) - exact)) / np.max(np.abs(u0))
    assert err <= 1e-6


def test_f32c_ks_error_first_steps():
    n, nsteps = 2048, 2000
    u0 = workloads.ks_smoothed(n, 55)
    ref = oracle.advance_f64(KS, KS_PRM, u0, nsteps)
    hi, lo = oracle.split_f32c(u0)
    hi, lo = oracle.advance_f32c(KS, KS_PRM, hi, lo, nsteps)
    err = np.max(np.abs(oracle.merge_f32c(hi, lo) - ref)) / np.max(np.abs(ref))
    assert err <= 1e-5


# --------------------------------------------------------------------------
# The swept stages (Section 3) reproduce per-step stepping exactly
# --------------------------------------------------------------------------

@pytest.mark.parametrize("stencil,prm", [(HEAT, [0.25]), (KS, KS_PRM)])
@pytest.mark.parametrize("B", [4, 8, 16])
@pytest.mark.parametrize("nsteps", [0, 1, 3, 4, 7, 8, 9, 16, 23, 40])
def test_swept_bruteforce_matches_per_step(stencil, prm, B, nsteps):
    n = 16
    rad = oracle.radius(stencil)
    if B % (2 * rad):
        pytest.skip("B must be a multiple of 2r")
    u0 = workloads.ks_smoothed(n, 90) * 10 if stencil == KS else workloads.uniform(n, 90)
    tr = swept_simulate(stencil, prm, u0, n // B, nsteps)
    want = oracle.advance_f64(stencil, prm, u0, nsteps)
    assert np.array_equal(np.array(tr.u_final), want)
    # every space-time value computed exactly once: no redundant work
    assert all(c == 1 for c in tr.compute_count.values())
    assert len(tr.compute_count) == n * nsteps


@pytest.mark.parametrize("stencil,prm,B", [(HEAT, [0.25], 8), (HEAT, [0.25], 16), (KS, KS_PRM, 16)])
def test_swept_bruteforce_stage_geometry(stencil, prm, B):
    """Stage work and message sizes: triangle B*h/2-ish, diamonds B*h, edges 2r per level."""
    n = 48
    rad = oracle.radius(stencil)
    h = B // (2 * rad)
    nsteps = 5 * h
    u0 = workloads.uniform(n, 3)
    tr = swept_simulate(stencil, prm, u0, n // B, nsteps)
    # first stage: shrinking triangle, level m on B - 2 r m points, m = 1..h-1
    tri = sum(B - 2 * rad * m for m in range(1, h))
    assert tr.computed[0] == [tri] * (n // B)
    # middle stages: diamonds of B*h updates (the n^2/2 per stage of Section 4)
    for k in range(1, 4):
        assert tr.computed[k] == [B * h] * (n // B)
    # the neighbour's data a node reads in a diamond stage: 2r values on each of h levels
    for k in range(1, 4):
        for node_reads in tr.reads[k]:
            assert len(node_reads) == h
            assert all(len(xs) == 2 * rad for xs in node_reads.values())


def test_swept_single_node_is_its_own_neighbour():
    u0 = workloads.uniform(16, 4)
    tr = swept_simulate(HEAT, [0.25], u0, 1, 12)
    assert np.array_equal(np.array(tr.u_final), oracle.advance_f64(HEAT, [0.25], u0, 12))


# --------------------------------------------------------------------------
# Discrete adjoint
# --------------------------------------------------------------------------

def test_adjoint_step_dot_product_ks():
    """<J v, w> = <v, J^T w>; the KS step is quadratic, so central differences give J v."""
    n = 128
    u = workloads.ks_smoothed(n, 41) * 20
    v = workloads.uniform(n, 42)
    w = workloads.uniform(n, 43)
    eps = 1e-3
    Jv = (oracle.step_f64(KS, KS_PRM, u + eps * v) - oracle.step_f64(KS, KS_PRM, u - eps * v)) / (2 * eps)
    JTw = oracle.adjoint_step_f64(KS, KS_PRM, u, w)
    lhs, rhs = math.fsum(Jv * w), math.fsum(v * JTw)
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + 1)


def test_adjoint_step_dot_product_heat():
    n = 100
    v = workloads.uniform(n, 44)
    w = workloads.uniform(n, 45)
    u = np.zeros(n)
    Jv = oracle.step_f64(HEAT, [0.3], v)          # linear: J v = step(v)
    JTw = oracle.adjoint_step_f64(HEAT, [0.3], u, w)
    assert abs(math.fsum(Jv * w) - math.fsum(v * JTw)) <= 1e-13 * n


def test_heat_adjoint_equals_forward_2n():
    """J = 1/2 sum u(T)^2, heat: grad = A^(2n) u0 since A is symmetric."""
    n, nsteps = 256, 60
    u0 = workloads.uniform(n, 46)
    uT = oracle.advance_f64(HEAT, [0.25], u0, nsteps)
    g = oracle.adjoint_f64(HEAT, [0.25], u0, uT, nsteps)
    assert np.array_equal(g, oracle.advance_f64(HEAT, [0.25], u0, 2 * nsteps))


def test_ks_adjoint_vs_finite_differences():
    n, nsteps = 256, 500
    u0 = workloads.ks_smoothed(n, 47)

    def J(u):
        uT = oracle.advance_f64(KS, KS_PRM, u, nsteps)
        return 0.5 * math.fsum(uT * uT)

    uT = oracle.advance_f64(KS, KS_PRM, u0, nsteps)
    g = oracle.adjoint_f64(KS, KS_PRM, u0, uT, nsteps)
    for d in range(4):
        v = workloads.fd_direction(n, d, 12345)
        eps = 1e-6
        fd = (J(u0 + eps * v) - J(u0 - eps * v)) / (2 * eps)
        ad = math.fsum(g * v)
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 1e-9


# --------------------------------------------------------------------------
# Workload generators
# --------------------------------------------------------------------------

def test_batch_recipe():
    kinds, lengths, steps = workloads.batch_problems()
    assert len(kinds) == 4096 and (kinds == 0).sum() == 2048
    assert np.all(lengths % 512 == 0) and lengths.min() >= 512 and lengths.max() <= 262144
    assert steps.min() >= 1000 and steps.max() <= 20000
    k2, l2, s2 = workloads.batch_problems()
    assert np.array_equal(lengths, l2) and np.array_equal(steps, s2) and np.array_equal(kinds, k2)


def test_generators_deterministic():
    assert np.array_equal(workloads.heat_modes(1024, 8), workloads.heat_modes(1024, 8))
    assert np.array_equal(workloads.ks_smoothed(4096), workloads.ks_smoothed(4096))


# --------------------------------------------------------------------------
# Reductions: exactly rounded against exact rational sums
# --------------------------------------------------------------------------

def test_reductions_exact():
    from oracle import reductions as R
    u = workloads.uniform(500, 60) * np.logspace(-8, 8, 500)
    v = workloads.uniform(500, 61)
    assert R.total(u) == float(sum(Fraction(x) for x in u))
    assert R.dot(u, v) == float(sum(Fraction(x) * Fraction(y) for x, y in zip(u, v)))
    assert R.half_sumsq(u) == float(sum(Fraction(x) ** 2 for x in u) / 2)


# --------------------------------------------------------------------------
# Two-stage Runge-Kutta (midpoint) as two sub-timesteps (Section 2)
# --------------------------------------------------------------------------

HEAT_RK2, KS_RK2 = oracle.HEAT_RK2, oracle.KS_RK2


@pytest.mark.parametrize("k", [1, 7, 64, 100])
def test_heat_rk2_mode_gain(k):
    """Mode k is scaled by 1 + z + z^2/2 per step, z = -4 r sin^2(pi k/N)."""
    n, r, nsteps = 256, 0.25, 150
    u0 = np.cos(2 * np.pi * k * np.arange(n) / n)
    z = -4 * r * np.sin(np.pi * k / n) ** 2
    got = oracle.advance_rk2_f64(HEAT_RK2, [r], u0, nsteps)
    assert np.max(np.abs(got - (1 + z + z * z / 2) ** nsteps * u0)) <= 16 * nsteps * EPS


@pytest.mark.parametrize("k", [1, 40, 128, 255])
def test_ks_rk2_linear_mode_gain(k):
    n = 512
    dt, dx = KS_PRM
    A = 1e-10
    u0 = A * np.cos(2 * np.pi * k * np.arange(n) / n)
    s = np.sin(np.pi * k / n) ** 2
    z = dt * (4 * s / dx ** 2 - 16 * s ** 2 / dx ** 4)
    u1 = oracle.advance_rk2_f64(KS_RK2, KS_PRM, u0, 1)
    assert np.max(np.abs(u1 - (1 + z + z * z / 2) * u0)) <= 1e-9 * A


def test_ks_rk2_second_order_in_time():
    """Halving dt (twice the steps) moves the result by ~1/4 as much: the scheme is second order."""
    n, dx = 256, 0.5
    u0 = workloads.ks_smoothed(n, 3) * 10
    T = 0.2
    ref = oracle.advance_rk2_f64(KS_RK2, [T / 800, dx], u0, 800)
    errs = [np.max(np.abs(oracle.advance_rk2_f64(KS_RK2, [T / m, dx], u0, m) - ref)) for m in (50, 100)]
    assert 3.2 < errs[0] / errs[1] < 4.8


@pytest.mark.parametrize("stencil,prm", [(HEAT_RK2, [0.25]), (KS_RK2, KS_PRM)])
def test_rk2_conservation_and_symmetry(stencil, prm):
    u0 = workloads.ks_smoothed(300, 8) * 10 if stencil == KS_RK2 else workloads.uniform(300, 8)
    u = oracle.advance_rk2_f64(stencil, prm, u0, 200)
    scale = math.fsum(np.abs(u0)) + math.fsum(np.abs(u))
    assert abs(math.fsum(u) - math.fsum(u0)) <= 8 * 200 * EPS * scale
    a = oracle.advance_rk2_f64(stencil, prm, np.roll(u0, 17), 50)
    assert np.array_equal(a, np.roll(oracle.advance_rk2_f64(stencil, prm, u0, 50), 17))


def exact_rk2_step(stencil, prm, u):
    """One RK2 step with every operation's rounding emulated on rationals."""
    n = len(u)
    if stencil == HEAT_RK2:
        r = prm[0]

        def sub(v, base, scale):
            return [X.fma64(X.mul64(scale, r), X.sub64(X.add64(v[i - 1], v[(i + 1) % n]), X.mul64(2.0, v[i])),
                            base[i]) for i in range(n)]
    else:
        a, b, e = ks_consts64(*prm)

        def sub(v, base, scale):
            out = []
            for i in range(n):
                x = [v[(i + k) % n] for k in range(-2, 3)]
                Gm, Gp = X.mul64(x[1], x[1]), X.mul64(x[3], x[3])
                wm = X.sub64(X.add64(x[0], x[2]), X.mul64(2.0, x[1]))
                w0 = X.sub64(X.add64(x[1], x[3]), X.mul64(2.0, x[2]))
                wp = X.sub64(X.add64(x[2], x[4]), X.mul64(2.0, x[3]))
                D = X.sub64(X.add64(wm, wp), X.mul64(2.0, w0))
                t = X.sub64(Gp, Gm)
                out.append(X.fma64(X.mul64(scale, e), D, X.fma64(X.mul64(scale, b), w0,
                                                                  X.fma64(X.mul64(scale, a), t, base[i]))))
            return out
    m = sub(list(u), list(u), 0.5)
    return np.array(sub(m, list(u), 1.0))


@pytest.mark.parametrize("stencil,prm,scale", [(HEAT_RK2, [0.3], 1.0), (KS_RK2, KS_PRM, 5.0)])
def test_rk2_step_ieee_exact(stencil, prm, scale):
    u = workloads.uniform(16, 5) * scale
    assert np.array_equal(oracle.advance_rk2_f64(stencil, prm, u, 1), exact_rk2_step(stencil, prm, u))


@pytest.mark.parametrize("stencil,prm", [(HEAT_RK2, [0.25]), (KS_RK2, KS_PRM)])
@pytest.mark.parametrize("B", [4, 8, 16])
@pytest.mark.parametrize("nsteps", [1, 3, 4, 9, 20])
def test_rk2_swept_bruteforce_matches_per_step(stencil, prm, B, nsteps):
    """The swept stages with the forwarded pair (u, m) equal per-step RK2 (levels = 2 x steps)."""
    n = 16
    if B % (2 * oracle.radius(stencil)):
        pytest.skip("B must be a multiple of 2r")
    u0 = workloads.ks_smoothed(n, 91) * 10 if stencil == KS_RK2 else workloads.uniform(n, 91)
    tr = swept_simulate(stencil, prm, u0, n // B, 2 * nsteps)
    assert np.array_equal(np.array(tr.u_final), oracle.advance_rk2_f64(stencil, prm, u0, nsteps))
    assert all(c == 1 for c in tr.compute_count.values())
