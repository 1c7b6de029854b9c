"""Single-point sub-timestep in Python (FP64), for the swept brute force.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

The evaluation order is the canonical one stated in ``oracle.c``.  Python
floats are IEEE binary64 with round-to-nearest-even for + - *; the fused
multiply-add is evaluated exactly on rationals and rounded once
(``float(Fraction)`` is correctly rounded), so this is a correctly rounded
fma independent of the C library.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def fma(a: float, b: float, c: float) -> float:
    """Correctly rounded a*b + c in binary64."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def ks_constants(dt: float, dx: float):
    """(a, b, e) of the KS update: -(dt/(4dx)), -(dt/dx^2), -(dt/dx^4), FP64."""
    dx2 = dx * dx
    return -(dt / (4.0 * dx)), -(dt / dx2), -(dt / (dx2 * dx2))


def heat_point(um: float, u0: float, up: float, r: float) -> float:
    """u' = fma(r, (um + up) - 2 u0, u0)."""
    s = um + up
    w = s - 2.0 * u0
    return fma(r, w, u0)


def ks_point(v, a: float, b: float, e: float) -> float:
    """KS update at the centre of v = (u[i-2], ..., u[i+2])."""
    Gm = v[1] * v[1]
    Gp = v[3] * v[3]
    wm = (v[0] + v[2]) - 2.0 * v[1]
    w0 = (v[1] + v[3]) - 2.0 * v[2]
    wp = (v[2] + v[4]) - 2.0 * v[3]
    D = (wm + wp) - 2.0 * w0
    t = Gp - Gm
    return fma(e, D, fma(b, w0, fma(a, t, v[2])))


EULER = 4


def _minmod(a: float, b: float) -> float:
    if a > 0.0 and b > 0.0:
        return min(a, b)
    if a < 0.0 and b < 0.0:
        return max(a, b)
    return 0.0


def euler_face_flux(qL, qR, g1: float):
    """Interface flux with Roe-spectral-radius dissipation (order as in oracle.c)."""
    uL, uR = qL[1] / qL[0], qR[1] / qR[0]
    pL = g1 * (qL[2] - 0.5 * (qL[1] * uL))
    pR = g1 * (qR[2] - 0.5 * (qR[1] * uR))
    HL, HR = (qL[2] + pL) / qL[0], (qR[2] + pR) / qR[0]
    fL = (qL[1], fma(qL[1], uL, pL), (qL[2] + pL) * uL)
    fR = (qR[1], fma(qR[1], uR, pR), (qR[2] + pR) * uR)
    sl, sr = math.sqrt(qL[0]), math.sqrt(qR[0])
    d = sl + sr
    ut = (sl * uL + sr * uR) / d
    Ht = (sl * HL + sr * HR) / d
    c2 = g1 * (Ht - 0.5 * (ut * ut))
    lam = abs(ut) + math.sqrt(max(c2, 0.0))
    return tuple(0.5 * ((fL[k] + fR[k]) - lam * (qR[k] - qL[k])) for k in range(3))


EULER_F32C = 5

_F32 = np.float32


def round_f32(x: Fraction) -> np.float32:
    """The binary32 value nearest to the rational x (ties to even), subnormals included."""
    if x == 0:
        return _F32(0.0)
    sign = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if x < Fraction(2) ** e:
        e -= 1                                   # now 2^e <= x < 2^(e+1)
    q = max(e - 23, -149)                        # quantum of the binade (or of subnormals)
    m = x / Fraction(2) ** q
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return _F32(sign * float(n * Fraction(2) ** q))


def fma32(a, b, c) -> np.float32:
    """Correctly rounded a*b + c in binary32 (exact rational arithmetic, one rounding)."""
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    if exact == 0:
        return _F32(a) * _F32(b) + _F32(c)       # IEEE sign of an exact zero sum
    return round_f32(exact)


def two_sum32(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def euler_face_flux_f32(qL, qR, g1):
    """Binary32 interface flux, the same expression order as the FP64 one."""
    half = _F32(0.5)
    uL, uR = qL[1] / qL[0], qR[1] / qR[0]
    pL = g1 * (qL[2] - half * (qL[1] * uL))
    pR = g1 * (qR[2] - half * (qR[1] * uR))
    eL, eR = qL[2] + pL, qR[2] + pR
    HL, HR = eL / qL[0], eR / qR[0]
    fL = (qL[1], fma32(qL[1], uL, pL), eL * uL)
    fR = (qR[1], fma32(qR[1], uR, pR), eR * uR)
    sl, sr = np.sqrt(qL[0]), np.sqrt(qR[0])
    d = sl + sr
    ut = (sl * uL + sr * uR) / d
    Ht = (sl * HL + sr * HR) / d
    c2 = g1 * (Ht - half * (ut * ut))
    lam = abs(ut) + np.sqrt(max(c2, _F32(0.0)))
    return tuple(half * ((fL[k] + fR[k]) - lam * (qR[k] - qL[k])) for k in range(3))


def _minmod32(a, b):
    z = _F32(0.0)
    if a > z and b > z:
        return min(a, b)
    if a < z and b < z:
        return max(a, b)
    return z


def make_point_update(stencil: int, params):
    """Return (radius, f) with f(values at i-r..i+r of level t, t) -> value at i of level t+1.

    Forward Euler (stencils 0, 1): values are floats.  Two-stage Runge-Kutta
    (stencils 2 heat, 3 KS; Section 2's two sub-timesteps with a forwarded
    variable): values are pairs (u, m); even levels take sub-timestep A,
    (u, m) -> (u, u + dt/2 f(u)), odd levels sub-timestep B,
    (u, m) -> (u + dt f(m), m).  The second component after B is carried
    along unchanged and never read.  Euler equations (stencil 4, Section 7):
    values are 9-tuples (q, q_mid, slopes) of conserved variables; level t
    takes sub-timestep t mod 4 (slopes of q, half-step flux update into
    q_mid, slopes of q_mid, full-step flux update of q from q_mid's fluxes).
    Euler equations on the compensated FP32 state (stencil 5): 12-tuples of
    numpy float32 (hi, lo, q_mid, slopes), every operation in binary32.
    """
    if stencil == 0:
        r = float(params[0])
        return 1, (lambda v, t: heat_point(v[0], v[1], v[2], r))
    if stencil == 1:
        a, b, e = ks_constants(float(params[0]), float(params[1]))
        return 2, (lambda v, t: ks_point(v, a, b, e))
    if stencil == 2:
        r = float(params[0])

        def heat_rk2(v, t):
            u0 = v[1][0]
            if t % 2 == 0:
                s = v[0][0] + v[2][0]
                w = s - 2.0 * u0
                return (u0, fma(0.5 * r, w, u0))
            s = v[0][1] + v[2][1]
            w = s - 2.0 * v[1][1]
            return (fma(r, w, u0), v[1][1])
        return 1, heat_rk2
    if stencil == 3:
        a, b, e = ks_constants(float(params[0]), float(params[1]))

        def ks_rk2(v, t):
            u0 = v[2][0]
            if t % 2 == 0:
                return (u0, ks_point([x[0] for x in v], 0.5 * a, 0.5 * b, 0.5 * e))
            x = [y[1] for y in v]
            Gm, Gp = x[1] * x[1], x[3] * x[3]
            wm = (x[0] + x[2]) - 2.0 * x[1]
            w0 = (x[1] + x[3]) - 2.0 * x[2]
            wp = (x[2] + x[4]) - 2.0 * x[3]
            D = (wm + wp) - 2.0 * w0
            tt = Gp - Gm
            return (fma(e, D, fma(b, w0, fma(a, tt, u0))), x[2])
        return 2, ks_rk2
    if stencil == EULER:
        dtdx, g1 = params[0] / params[1], params[2] - 1.0

        def euler(v, t):
            # state per point: (q0, q1, q2, qm0, qm1, qm2, s0, s1, s2)
            sub = t % 4
            c = v[1]
            if sub in (0, 2):                      # slopes of q (0) or of the midpoint (2)
                o = 0 if sub == 0 else 3
                sl = tuple(_minmod(c[o + k] - v[0][o + k], v[2][o + k] - c[o + k]) for k in range(3))
                return c[:6] + sl
            o = 0 if sub == 1 else 3                 # fluxes from q (1) or the midpoint (3)
            def face(a, b):
                qL = tuple(fma(0.5, a[6 + k], a[o + k]) for k in range(3))
                qR = tuple(fma(-0.5, b[6 + k], b[o + k]) for k in range(3))
                return euler_face_flux(qL, qR, g1)
            Fl, Fr = face(v[0], c), face(c, v[2])
            ca = (0.5 if sub == 1 else 1.0) * dtdx
            new = tuple(fma(-ca, Fr[k] - Fl[k], c[k]) for k in range(3))
            if sub == 1:
                return c[:3] + new + c[6:]
            return new + c[3:]
        return 1, euler
    if stencil == EULER_F32C:
        cf = _F32(params[0] / params[1])
        ch = _F32(0.5) * cf
        g1 = _F32(params[2] - 1.0)

        def euler_f32c(v, t):
            # state per point: (hi0..2, lo0..2, qm0..2, s0..2), binary32
            sub = t % 4
            c = v[1]
            if sub in (0, 2):                      # slopes of hi (0) or of the midpoint (2)
                o = 0 if sub == 0 else 6
                sl = tuple(_minmod32(c[o + k] - v[0][o + k], v[2][o + k] - c[o + k]) for k in range(3))
                return c[:9] + sl
            o = 0 if sub == 1 else 6

            def face(a, b):
                qL = tuple(fma32(_F32(0.5), a[9 + k], a[o + k]) for k in range(3))
                qR = tuple(fma32(_F32(-0.5), b[9 + k], b[o + k]) for k in range(3))
                return euler_face_flux_f32(qL, qR, g1)
            Fl, Fr = face(v[0], c), face(c, v[2])
            if sub == 1:
                qm = tuple(c[k] + fma32(-ch, Fr[k] - Fl[k], c[3 + k]) for k in range(3))
                return c[:6] + qm + c[9:]
            hl = [two_sum32(c[k], fma32(-cf, Fr[k] - Fl[k], c[3 + k])) for k in range(3)]
            return tuple(h for h, _ in hl) + tuple(l for _, l in hl) + c[6:]
        return 1, euler_f32c
    raise ValueError(f"unknown stencil {stencil}")
