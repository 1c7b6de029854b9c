"""Single-point sub-timestep in Python (FP64), for the swept brute force.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

The evaluation order is the canonical one stated in ``oracle.c``.  Python
floats are IEEE binary64 with round-to-nearest-even for + - *; the fused
multiply-add is evaluated exactly on rationals and rounded once
(``float(Fraction)`` is correctly rounded), so this is a correctly rounded
fma independent of the C library.
"""
from __future__ import annotations

from fractions import Fraction


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


def make_point_update(stencil: int, params):
    """Return (radius, f) with f(values u[i-r..i+r]) -> u'[i]."""
    if stencil == 0:
        r = float(params[0])
        return 1, (lambda v: heat_point(v[0], v[1], v[2], r))
    if stencil == 1:
        a, b, e = ks_constants(float(params[0]), float(params[1]))
        return 2, (lambda v: ks_point(v, a, b, e))
    raise ValueError(f"unknown stencil {stencil}")
