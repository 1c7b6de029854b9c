"""Exactly rounded FP64 reductions: conserved sum, objective, directional derivative.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

* ``total(u)``       = sum_i u_i, correctly rounded (``math.fsum``).
* ``half_sumsq(u)``  = 1/2 sum_i u_i^2, the objective J of the adjoint; the
  squares are split exactly (Dekker's two-product with Veltkamp splitting)
  so the sum is of exact terms, then correctly rounded.
* ``dot(u, v)``      = sum_i u_i v_i, the directional derivative <grad J, v>.

The FP32-compensated state enters as its merged FP64 values fl64(hi + lo).
"""
from __future__ import annotations

import math

import numpy as np

_SPLIT = 134217729.0          # 2^27 + 1


def _split(a: np.ndarray):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_product(a: np.ndarray, b: np.ndarray):
    """p = fl(a*b), e with p + e = a*b exactly (no overflow or underflow assumed)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def total(u) -> float:
    return math.fsum(np.asarray(u, dtype=np.float64))


def dot(u, v) -> float:
    p, e = two_product(u, v)
    return math.fsum(np.concatenate([p, e]))


def half_sumsq(u) -> float:
    return 0.5 * dot(u, u)
