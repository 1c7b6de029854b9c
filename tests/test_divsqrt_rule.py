"""The acceptance rule of the Euler kernels' straight-line division and square root, in exact
arithmetic on the CPU.

The compensated Euler kernels take a candidate quotient q1 (square root s1) from an
approximate reciprocal and one correction, and keep it only where a test on the rounded
remainder accepts it; elsewhere they recompute with the correctly rounded library
operation.  The GPU test compares the kernel with CUDA's results; this one checks the rule
itself, with every rounding done exactly on rationals: over random operands, quotients and
roots next to rounding midpoints, and powers of two (where the neighbour towards zero is
half an ulp away), the rule must accept a candidate only if it is the correctly rounded
result, whatever the candidate (the correct one or either neighbour), and must accept the
correct one nearly always.  The rule, as the kernel states it:

  division:    |b| in [2^-30, 2^31), e' = exponent of the binary32 number just below |q1|
               in [-72, 120], and |RN(RN(a - b q1) * 2^(24 - e'))| < |b|  (or a = +-0)
  square root: x in [2^-100, 2^101) and |RN(RN(x - s1^2) * 2^(23 - e'))| < s1  (or x = +-0)
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

M32 = 0xFFFFFFFF


def bits(x) -> int:
    return int(np.array(x, dtype=np.float32).view(np.uint32))


def from_bits(u: int) -> np.float32:
    return np.array(u & M32, dtype=np.uint32).view(np.float32)[()]


def rn32(x: Fraction) -> np.float32:
    """Round a rational to the nearest binary32 number, ties to even (subnormals
    included; magnitudes from 2^128 on give infinity)."""
    if x == 0:
        return np.float32(0.0)
    sgn = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    quantum = Fraction(2) ** (max(e, -126) - 23)
    m = x / quantum
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = n * quantum
    if v >= Fraction(2) ** 128:
        return np.float32(sgn * np.inf)
    return np.float32(sgn * float(v))          # exact: v has at most 24 significant bits


def F(x) -> Fraction:
    return Fraction(float(x))


def nextup(x):
    return np.nextafter(np.float32(x), np.float32(np.inf))


def nextdown(x):
    return np.nextafter(np.float32(x), np.float32(-np.inf))


def accept_div(a, b, q1) -> bool:
    mb = bits(b) & 0x7FFFFFFF
    b_ok = ((mb - (97 << 23)) & M32) < (61 << 23)
    if F(a) == 0:
        return b_ok
    r1 = rn32(F(a) - F(b) * F(q1))
    t = ((bits(q1) - 1) & M32) & 0x7F800000
    sc = from_bits((278 << 23) - t)
    in_range = ((t - (55 << 23)) & M32) < (193 << 23)
    if not (b_ok and in_range):
        return False
    return abs(F(rn32(F(r1) * F(sc)))) < abs(F(b))


def accept_sqrt(x, s1) -> bool:
    xb = bits(x)
    if xb & 0x7FFFFFFF == 0:
        return True
    in_range = ((xb - (27 << 23)) & M32) < (201 << 23)
    if not in_range:
        return False
    r1 = rn32(F(x) - F(s1) * F(s1))
    sc = from_bits((277 << 23) - (((bits(s1) - 1) & M32) & 0x7F800000))
    return abs(F(rn32(F(r1) * F(sc)))) < F(s1)


def rn_sqrt(x) -> np.float32:
    """The correctly rounded binary32 square root of a positive binary32 number: the
    candidate from floor(sqrt) of the scaled integer, then the nearer of it and its
    successor by comparing squares (no square root of a binary32 number is a midpoint)."""
    fx = F(x)
    e = (fx.numerator.bit_length() - fx.denominator.bit_length()) // 2
    scale = Fraction(2) ** (2 * (23 - e) + 2)
    v = fx * scale                              # sqrt(v) = sqrt(x) 2^(24 - e)
    n = math.isqrt(v.numerator // v.denominator)
    lo = rn32(Fraction(n) / Fraction(2) ** (24 - e))
    best = None
    for c in (nextdown(lo), lo, nextup(lo), nextup(nextup(lo))):
        if best is None or _closer(c, best, fx):
            best = c
    return best


def _closer(c, d, fx) -> bool:
    """|c - sqrt(fx)| < |d - sqrt(fx)| for positive c != d, exactly: the midpoint test
    ((c + d) / 2)^2 against fx."""
    m = (F(c) + F(d)) / 2
    return (m * m < fx) == (F(c) > F(d))


def _log_uniform(rng, lo, hi, n):
    return [np.float32(v) for v in np.exp2(rng.uniform(np.log2(lo), np.log2(hi), n))]


def _ulp(x) -> Fraction:
    return F(nextup(abs(np.float32(x)))) - F(abs(np.float32(x)))


def _check_div_case(a, b):
    q = rn32(F(a) / F(b))
    accepted = {}
    for c in (nextdown(q), q, nextup(q)):
        acc = accept_div(a, b, c)
        assert not acc or c == q, (a, b, c, q)
        accepted[float(c)] = acc
    return accepted[float(q)]


def _check_sqrt_case(x):
    s = rn_sqrt(x)
    acc_s = None
    for c in (nextdown(s), s, nextup(s)):
        acc = accept_sqrt(x, c)
        assert not acc or c == s, (x, c, s)
        if c == s:
            acc_s = acc
    return acc_s


def test_rn32_and_rn_sqrt_helpers():
    assert rn32(Fraction(1, 3)) == np.float32(1.0) / np.float32(3.0)
    assert rn32(Fraction(1) + Fraction(1, 2 ** 24)) == np.float32(1.0)           # tie to even
    assert rn32(Fraction(1) + Fraction(3, 2 ** 25)) == nextup(np.float32(1.0))
    for x in (2.0, 3.0, 0.5, 1e-20, 7e30):
        assert rn_sqrt(np.float32(x)) == np.float32(math.sqrt(float(np.float32(x))))


def test_division_rule_random_operands():
    rng = np.random.default_rng(1)
    a = _log_uniform(rng, 2.0 ** -40, 2.0 ** 60, 600)        # quotients inside the range
    b = _log_uniform(rng, 2.0 ** -29, 2.0 ** 30, 600)
    acc = [_check_div_case(x * (1 if i % 2 else -1), y) for i, (x, y) in enumerate(zip(a, b))]
    assert np.mean(acc) > 0.99


def test_division_rule_near_midpoints():
    rng = np.random.default_rng(2)
    acc = []
    for b, q in zip(_log_uniform(rng, 2.0 ** -20, 2.0 ** 20, 300), _log_uniform(rng, 2.0 ** -20, 2.0 ** 20, 300)):
        m = F(q) + _ulp(q) / 2
        a = rn32(F(b) * m)
        for aa in (nextdown(a), a, nextup(a)):
            acc.append(_check_div_case(aa, b))
    assert np.mean(acc) > 0.98


def test_division_rule_at_powers_of_two():
    """Quotients just below and above 2^e: towards zero the neighbour is half an ulp
    away, so the rounding boundary is a quarter ulp below 2^e."""
    rng = np.random.default_rng(3)
    acc = []
    for b in _log_uniform(rng, 1.0, 2.0 ** 10, 200):
        e = int(rng.integers(-40, 40))
        p = Fraction(2) ** e
        up_ulp = Fraction(2) ** (e - 23)
        for off in (-up_ulp / 4, -up_ulp / 8, up_ulp / 4, up_ulp / 2, -up_ulp * 3 / 8, Fraction(0)):
            a = rn32(F(b) * (p + off))
            for aa in (nextdown(a), a, nextup(a)):
                acc.append(_check_div_case(aa, b))
    # the bound at a power of two is half the usual one (conservative): many of these
    # deliberately borderline cases go to the library form, but not all
    assert np.mean(acc) > 0.2


def test_division_rule_range_edges():
    one = np.float32(1.0)
    # quotient range: e' in [-72, 120]
    assert accept_div(nextup(np.float32(2.0 ** -72)), one, nextup(np.float32(2.0 ** -72)))
    assert not accept_div(np.float32(2.0 ** -72), one, np.float32(2.0 ** -72))
    assert accept_div(np.float32(2.0 ** 91), np.float32(2.0 ** -30), np.float32(2.0 ** 121))
    # divisor range
    assert not accept_div(one, nextdown(np.float32(2.0 ** -30)), rn32(1 / F(nextdown(np.float32(2.0 ** -30)))))
    assert not accept_div(one, np.float32(2.0 ** 31), np.float32(2.0 ** -31))
    # zero numerators pass for any divisor in range
    assert accept_div(np.float32(-0.0), np.float32(3.0), np.float32(-0.0))


def test_square_root_rule():
    rng = np.random.default_rng(4)
    acc = [_check_sqrt_case(x) for x in _log_uniform(rng, 2.0 ** -99, 2.0 ** 100, 600)]
    assert np.mean(acc) > 0.99
    # next to midpoints: x = RN((s + u/2)^2) and its neighbours
    acc = []
    for s in _log_uniform(rng, 2.0 ** -40, 2.0 ** 40, 300):
        m = F(s) + _ulp(s) / 2
        x = rn32(m * m)
        for xx in (nextdown(x), x, nextup(x)):
            acc.append(_check_sqrt_case(xx))
    assert np.mean(acc) > 0.98
    # powers of two and just below them (the lower neighbour half an ulp away)
    for e in range(-40, 41, 3):
        p = np.float32(2.0 ** e)
        for x in (p * p, nextdown(p * p), nextup(p * p), rn32(F(p) * F(p) * (1 - Fraction(1, 2 ** 24)))):
            _check_sqrt_case(np.float32(x))
    # range edges and non-positive inputs
    assert accept_sqrt(np.float32(2.0 ** -100), np.float32(2.0 ** -50))
    assert not accept_sqrt(nextdown(np.float32(2.0 ** -100)), rn_sqrt(nextdown(np.float32(2.0 ** -100))))
    assert not accept_sqrt(np.float32(2.0 ** 101), np.float32(2.0 ** 50.5))
    assert accept_sqrt(np.float32(-0.0), np.float32(-0.0))
    assert not accept_sqrt(np.float32(-1.0), np.float32(1.0))


@pytest.mark.parametrize("wrong_shift", [23, 24, 25])
def test_a_wrong_bound_is_caught(wrong_shift):
    """Planted mistake: scaling the remainder by 2^(wrong - e') instead of 2^(24 - e') (a
    bound twice too large, or half) must either accept a wrong candidate somewhere on the
    near-midpoint cases or reject far more correct ones; the kernel's shift (24) does
    neither."""
    def accept_wrong(a, b, q1):
        mb = bits(b) & 0x7FFFFFFF
        if F(a) == 0:
            return True
        r1 = rn32(F(a) - F(b) * F(q1))
        t = ((bits(q1) - 1) & M32) & 0x7F800000
        sc = from_bits(((127 + wrong_shift + 127) << 23) - t)
        return ((mb - (97 << 23)) & M32) < (61 << 23) and abs(F(rn32(F(r1) * F(sc)))) < abs(F(b))

    rng = np.random.default_rng(5)
    wrong, right = 0, 0
    for b, q in zip(_log_uniform(rng, 2.0 ** -10, 2.0 ** 10, 200), _log_uniform(rng, 2.0 ** -10, 2.0 ** 10, 200)):
        a = rn32(F(b) * (F(q) + _ulp(q) / 2))
        qq = rn32(F(a) / F(b))
        for c in (nextdown(qq), qq, nextup(qq)):
            if accept_wrong(a, b, c):
                if c == qq:
                    right += 1
                else:
                    wrong += 1
    if wrong_shift == 24:
        assert wrong == 0 and right > 190
    else:
        assert wrong > 0 or right < 150
