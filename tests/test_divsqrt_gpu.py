"""The Euler kernels' straight-line binary32 division and square root against CUDA's.

The compensated Euler kernels divide and take square roots without branches and accept a
result only where an exact remainder test proves it correctly rounded; elsewhere they
recompute it with the correctly rounded library operation.  So wherever the straight-line
form reports a result as proven it must equal __fdiv_rn / __fsqrt_rn bit for bit; inside
its operand range it must prove nearly every result (or the kernels would run the slow
form); outside that range it must decline.

Inputs: random bit patterns over every sign and exponent; operands spread over the range;
quotients and roots built next to rounding midpoints (the cases a wrong acceptance test
gets wrong) and their neighbours; exact quotients and roots, powers of two; signed zeros;
the range edges on both sides; subnormals, infinities and NaN; values like the Euler
states (densities, momenta down to tiny magnitudes, energies).
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

B_LO, B_HI = 2.0 ** -30, 2.0 ** 31          # divisor range of the straight-line division
X_LO, X_HI = 2.0 ** -100, 2.0 ** 101        # square-root range (or x = +-0)
# quotient range: the binary32 number just below |a / b| has an exponent in [-72, 120]
Q_BIASED_LO, Q_BIASED_HI = 127 - 72, 127 + 120


def _div_in_range(a, b, qref):
    """Where the straight-line division applies: b in range, and a = +-0 or the exponent
    of the number just below the correctly rounded |a / b| in range (NaN and infinite
    quotients are out)."""
    with np.errstate(invalid="ignore"):
        inb = (np.abs(b) >= B_LO) & (np.abs(b) < B_HI)
        t = ((qref.view(np.uint32) - np.uint32(1)) >> np.uint32(23)) & np.uint32(0xff)
        inq = (t >= Q_BIASED_LO) & (t <= Q_BIASED_HI) & np.isfinite(qref)
    return inb & ((a == 0) | inq)


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _log_uniform(rng, lo, hi, n, signed=True):
    e = rng.uniform(np.log2(lo), np.log2(hi), n)
    v = _f32(np.exp2(e))
    v = v[(v >= lo) & (v < hi)]
    if signed:
        v = v * np.where(rng.random(v.size) < 0.5, -1, 1).astype(np.float32)
    return v


def _ulp(x):
    x = np.abs(x.astype(np.float32))
    return (np.nextafter(x, np.float32(np.inf)) - x).astype(np.float64)


def _run(sw, a, b):
    import torch
    ta = torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")
    tb = torch.tensor(np.ascontiguousarray(b, dtype=np.float32), device="cuda")
    out, ok = sw.swept_check_div_sqrt(ta, tb)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ok.cpu().numpy().astype(bool)


def _check_proven_equal(out, ok):
    bits = out.view(np.uint32)
    for k, (t, r) in enumerate(((0, 1), (2, 3))):
        bad = ok[k] & (bits[t] != bits[r])
        assert not bad.any(), (k, np.flatnonzero(bad)[:8])


def _midpoint_cases(rng, n):
    """a, b with a / b next to the midpoint of two binary32 numbers, and x with sqrt(x)
    next to one: b * m and m * m are exact in binary64 (24 + 25 and 25 + 25 bits)."""
    b = _log_uniform(rng, 2.0 ** -20, 2.0 ** 20, n)
    q = _log_uniform(rng, 2.0 ** -20, 2.0 ** 20, b.size)
    m = np.abs(q.astype(np.float64)) + _ulp(q) / 2
    a = _f32(b.astype(np.float64) * m * np.sign(q))
    s = _log_uniform(rng, 2.0 ** -40, 2.0 ** 40, n, signed=False)
    ms = s.astype(np.float64) + _ulp(s) / 2
    x = _f32(ms * ms)
    # neighbours one ulp either side: the remainder changes sign around the midpoint
    a = np.concatenate([a, np.nextafter(a, np.float32(np.inf)), np.nextafter(a, np.float32(-np.inf))])
    b = np.concatenate([b, b, b])
    x = np.concatenate([x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))])
    return a, b, x


def test_random_bit_patterns(cuda_lib):
    rng = np.random.default_rng(20260101)
    n = 1 << 20
    a = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
    b = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32).view(np.float32)
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    ind = _div_in_range(a, b, out[1])
    with np.errstate(invalid="ignore"):
        inx = (a >= X_LO) & (a < X_HI)
    # outside the range nothing is accepted; inside it nearly everything is
    assert not (ok[0] & ~ind).any()
    assert not (ok[1] & ~inx).any()
    assert ind.sum() > n // 8 and ok[0][ind].mean() > 0.999
    assert ok[1][inx].mean() > 0.999


def test_operands_across_the_range(cuda_lib):
    rng = np.random.default_rng(7)
    n = 1 << 19
    a = _log_uniform(rng, 2.0 ** -100, 2.0 ** 127, n)
    b = _log_uniform(rng, B_LO, B_HI, n)
    k = min(a.size, b.size)
    a, b = a[:k], b[:k]
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    ind = _div_in_range(a, b, out[1])
    assert not (ok[0] & ~ind).any()
    assert ind.mean() > 0.5 and ok[0][ind].mean() > 0.9999
    x = np.abs(a)
    x = x[(x >= X_LO) & (x < X_HI)]
    b = b[: x.size]
    out, ok = _run(cuda_lib, x, b)
    _check_proven_equal(out, ok)
    assert ok[1].mean() > 0.9999


def test_near_midpoints(cuda_lib):
    rng = np.random.default_rng(11)
    a, b, x = _midpoint_cases(rng, 1 << 18)
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    assert ok[0].mean() > 0.99
    out, ok = _run(cuda_lib, x, np.ones_like(x))
    _check_proven_equal(out, ok)
    assert ok[1].mean() > 0.99


def test_exact_results_powers_of_two_and_zeros(cuda_lib):
    rng = np.random.default_rng(3)
    n = 1 << 16
    # products of short integers scaled by powers of two: exact quotients
    bi = rng.integers(1, 1 << 12, n).astype(np.float64) * np.exp2(rng.integers(-25, 19, n))
    qi = rng.integers(1, 1 << 12, n).astype(np.float64) * np.exp2(rng.integers(-25, 25, n))
    qi[: n // 8] = np.exp2(rng.integers(-40, 40, n // 8))          # powers of two
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    b, a = _f32(bi * sgn), _f32(bi * qi)
    zeros = np.array([0.0, -0.0, 0.0, -0.0], dtype=np.float32)
    zb = np.array([1.5, 1.5, -3.0, -3.0], dtype=np.float32)
    a, b = np.concatenate([a, zeros]), np.concatenate([b, zb])
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    assert ok[0].all()                         # exact quotients (r = 0) and signed zeros
    assert np.array_equal(out[0][-4:].view(np.uint32), (zeros / zb).view(np.uint32))
    # exact roots (squares of short integers times even powers of two) and signed zeros
    r = rng.integers(1, 1 << 12, n).astype(np.float64) * np.exp2(rng.integers(-20, 20, n))
    x = np.concatenate([_f32(r * r), zeros])
    out, ok = _run(cuda_lib, x, np.ones_like(x))
    _check_proven_equal(out, ok)
    assert ok[1].all()
    assert np.array_equal(out[2][-4:].view(np.uint32), zeros.view(np.uint32))


def test_range_edges_and_specials(cuda_lib):
    f = np.float32
    up = lambda v: np.nextafter(f(v), f(np.inf))
    dn = lambda v: np.nextafter(f(v), f(-np.inf))
    # divisors: the edges of their range, with a quotient well inside
    b_in = [B_LO, dn(B_HI), -B_LO, -dn(B_HI), 1.0]
    b_out = [dn(B_LO), B_HI, -B_HI, 1e-40, np.inf, -np.inf, np.nan, 0.0, -0.0]
    # quotients at the edges of theirs, from exact products with powers of two
    q_in = [up(2.0 ** -72), f(3 * 2.0 ** -73), 2.0 ** 100, dn(2.0 ** 121), -up(2.0 ** -72)]
    q_out = [2.0 ** -72, dn(2.0 ** -72), 2.0 ** -100, up(2.0 ** 121), -(2.0 ** -72)]
    scale = [1.0, -1.0, 2.0 ** -6, 2.0 ** 6]
    a, b, want = [], [], []
    for bb in b_in:
        a.append(0.75 * bb); b.append(bb); want.append(True)
    for bb in b_out:
        a.append(0.75); b.append(bb); want.append(False)
    for q, w in [(q, True) for q in q_in] + [(q, False) for q in q_out]:
        for c in scale:
            a.append(float(q) * c); b.append(c); want.append(w)
    for x in (1e-42, np.inf, -np.inf, np.nan):       # subnormal, infinite and NaN numerators
        a.append(x); b.append(1.0); want.append(False)
    a, b, want = np.array(a, dtype=np.float32), np.array(b, dtype=np.float32), np.array(want)
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    assert np.array_equal(ok[0], want), np.flatnonzero(ok[0] != want)
    x = np.array([X_LO, dn(X_HI), 1.0, dn(X_LO), X_HI, -1.0, -X_LO, 1e-42, np.inf, np.nan], dtype=np.float32)
    out, ok = _run(cuda_lib, x, np.ones_like(x))
    _check_proven_equal(out, ok)
    assert ok[1][:3].all() and not ok[1][3:].any()


def test_euler_like_operands(cuda_lib):
    rng = np.random.default_rng(5)
    n = 1 << 18
    rho = _f32(rng.uniform(0.1, 1.1, n))
    mom = _f32(rng.uniform(-0.3, 0.3, n) * np.exp2(-rng.integers(0, 60, n) * (rng.random(n) < 0.2)))
    en = _f32(rng.uniform(0.2, 3.0, n))
    a = np.concatenate([mom, en, en])
    b = np.concatenate([rho, rho, _f32(np.sqrt(rho.astype(np.float64)) * 2)])
    out, ok = _run(cuda_lib, a, b)
    _check_proven_equal(out, ok)
    assert ok[0].mean() > 0.9999
    out, ok = _run(cuda_lib, np.concatenate([rho, en]), np.ones(2 * n, dtype=np.float32))
    _check_proven_equal(out, ok)
    assert ok[1].mean() > 0.9999


def test_rejects_bad_arguments(cuda_lib):
    import torch
    sw = cuda_lib
    a = torch.ones(4, device="cuda")
    with pytest.raises(ValueError):
        sw.swept_check_div_sqrt(a, torch.ones(5, device="cuda"))
    with pytest.raises(ValueError):
        sw.swept_check_div_sqrt(a.double(), a.double())
    out, ok = sw.swept_check_div_sqrt(torch.empty(0, device="cuda"), torch.empty(0, device="cuda"))
    assert out.shape == (4, 0) and ok.shape == (2, 0)
