"""IEEE round-to-nearest-even arithmetic evaluated exactly on rationals.

Each operation is computed exactly (``fractions.Fraction``) and rounded once
to binary64 or binary32.  This reproduces what an IEEE-conforming machine
must return for + - * and fused multiply-add, independently of any C
library, compiler flag or hardware.  Binary32 values are carried as Python
floats (every binary32 value is exactly a binary64 value).
"""
from __future__ import annotations

from fractions import Fraction

F32_MAX = Fraction((2 ** 24 - 1) * 2 ** 104)
F32_OVERFLOW = Fraction(2 ** 128 - 2 ** 103)   # RN overflows at or above this


def r64(q: Fraction) -> float:
    """Round an exact rational to binary64 (float(Fraction) is correctly rounded)."""
    return float(q)


def r32(q: Fraction) -> float:
    """Round an exact rational to binary32, ties to even, with subnormals."""
    q = Fraction(q)
    if q == 0:
        return 0.0
    neg = q < 0
    a = -q if neg else q
    if a >= F32_OVERFLOW:
        return float("-inf") if neg else float("inf")
    # exponent e with 2^23 <= a / 2^e < 2^24
    e = a.numerator.bit_length() - a.denominator.bit_length() - 24
    while a / Fraction(2) ** e >= 2 ** 24:
        e += 1
    while a / Fraction(2) ** e < 2 ** 23:
        e -= 1
    e = max(e, -149)
    m = round(a / Fraction(2) ** e)           # Fraction.__round__: ties to even
    v = float(Fraction(m) * Fraction(2) ** e)
    return -v if neg else v


def F(x) -> Fraction:
    return Fraction(x)


# binary64
def add64(a, b): return r64(F(a) + F(b))
def sub64(a, b): return r64(F(a) - F(b))
def mul64(a, b): return r64(F(a) * F(b))
def fma64(a, b, c): return r64(F(a) * F(b) + F(c))


# binary32
def add32(a, b): return r32(F(a) + F(b))
def sub32(a, b): return r32(F(a) - F(b))
def mul32(a, b): return r32(F(a) * F(b))
def fma32(a, b, c): return r32(F(a) * F(b) + F(c))


def two_sum32(a, b):
    """Knuth TwoSum in binary32, every operation rounded."""
    s = add32(a, b)
    bb = sub32(s, a)
    ea = sub32(a, sub32(s, bb))
    eb = sub32(b, bb)
    return s, add32(ea, eb)
