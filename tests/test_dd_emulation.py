"""CPU emulation of the double-float helpers of the CUDA path (fe_dd.cuh).

The element tensors of the FE_PREC_F32X2 kernels are computed in pairs of FP32 numbers, and FP64
values cross into and out of that format through integer bit manipulation.  This file restates
each helper step by step (Python integers for the bit work, numpy float32 for the correctly
rounded FP32 operations, exact rationals for the fused multiply-add) and checks the properties
the kernels rely on:

* f2_from_f64: hi + lo is within 2^-47 |x| of x for 2^-74 <= |x| < 2^128, and hi alone is x
  truncated to 24 bits;
* f2_to_f64: within one FP64 ulp of the exact hi + lo of a normalised pair (|lo| <= ulp(hi)/2,
  what every pair operation returns);
* two_sum and fast_two_sum are error-free (s + e == a + b exactly);
* the pair product and the same-sign pair sum stay within a few units of 2^-48 relative.
"""
import math
import struct
from fractions import Fraction as Fr

import numpy as np
import pytest

f32 = np.float32


def u2f(u):
    return f32(struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0])


def f2u(x):
    return struct.unpack("<I", struct.pack("<f", f32(x)))[0]


def f2i(x):
    return struct.unpack("<i", struct.pack("<f", f32(x)))[0]


def d2u(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def u2d(u):
    return struct.unpack("<d", struct.pack("<Q", u & 0xFFFFFFFFFFFFFFFF))[0]


def round_f32(q: Fr):
    """Exact rational -> nearest FP32 (ties to even), the rounding of one fused FP32 operation."""
    if q == 0:
        return f32(0.0)
    s = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    while Fr(2) ** e > q:
        e -= 1
    while Fr(2) ** (e + 1) <= q:
        e += 1
    e = max(e, -126)
    ulp = Fr(2) ** (e - 23)
    m = q / ulp
    n = m.numerator // m.denominator
    r = m - n
    if r > Fr(1, 2) or (r == Fr(1, 2) and n % 2 == 1):
        n += 1
    return f32(float(s * n * ulp))


def fmaf(a, b, c):
    return round_f32(Fr(float(a)) * Fr(float(b)) + Fr(float(c)))


def fadd(a, b):
    return f32(f32(a) + f32(b))


def fsub(a, b):
    return f32(f32(a) - f32(b))


def fmul(a, b):
    return f32(f32(a) * f32(b))


# ----------------------------------------------------------------- the helpers, step by step
def two_sum(a, b):
    s = fadd(a, b)
    bb = fsub(s, a)
    err = fadd(fsub(a, fsub(s, bb)), fsub(b, bb))
    return s, err


def fast_two_sum(a, b):
    s = fadd(a, b)
    return s, fsub(b, fsub(s, a))


def f2_from_f64(x):
    b = d2u(x)
    sign = (b >> 63) << 31
    e = (b >> 52) & 0x7FF
    m = b & 0xFFFFFFFFFFFFF
    if e < 1023 - 126:
        return u2f(sign), f32(0.0)
    if e > 1023 + 127:
        return u2f(sign | 0x7F800000), f32(0.0)
    hi = u2f(sign | ((e - 1023 + 127) << 23) | (m >> 29))
    rem = m & 0x1FFFFFFF
    lo = f32(0.0)
    le = e - 1023 - 52 + 127
    if rem != 0 and le >= 1:
        fa = fsub(u2f(0x4B000000 | (rem >> 14)), 8388608.0)
        fb = fsub(u2f(0x4B000000 | (rem & 0x3FFF)), 8388608.0)
        lo = fmul(fmaf(fa, 16384.0, fb), u2f(le << 23))
        if sign:
            lo = -lo
    return hi, lo


def f2_to_f64(hi, lo):
    hb = f2u(hi)
    eh = (hb >> 23) & 0xFF
    sign = (hb >> 31) << 63
    if eh == 0:
        return u2d(sign)
    if eh == 0xFF:
        return u2d(sign | 0x7FF0000000000000 | ((hb & 0x7FFFFF) << 29))
    S = ((hb & 0x7FFFFF) | 0x800000) << 29
    if eh >= 52:
        sc1 = u2f((300 - eh) << 23)
        r1 = fmaf(lo, sc1, 12582912.0)
        t1 = f2i(r1) - 0x4B400000
        rem = fmaf(-f32(t1), u2f((eh - 46) << 23), lo)
        r2 = fmaf(rem, u2f((306 - eh) << 23), 12582912.0)
        t2 = f2i(r2) - 0x4B400000
        t = t1 * 64 + t2
        S += -t if (hb >> 31) else t
    ed = eh - 127 + 1023
    if S < (1 << 52):
        S <<= 1
        ed -= 1
    elif S >= (1 << 53):
        S >>= 1
        ed += 1
    return u2d(sign | (ed << 52) | (S & ((1 << 52) - 1)))


def dd_add(a, b):
    s, e0 = two_sum(a[0], b[0])
    e = fadd(e0, fadd(a[1], b[1]))
    return fast_two_sum(s, e)


def dd_mul(a, b):
    p = fmul(a[0], b[0])
    e = fmaf(a[0], b[0], -p)
    e = fmaf(a[0], b[1], e)
    e = fmaf(a[1], b[0], e)
    return fast_two_sum(p, e)


def exact(pair):
    return Fr(float(pair[0])) + Fr(float(pair[1]))


def _doubles(rng, n, lo_exp, hi_exp):
    mant = rng.uniform(1.0, 2.0, n)
    exps = rng.integers(lo_exp, hi_exp, n)
    sign = rng.choice([-1.0, 1.0], n)
    return [float(s * math.ldexp(m, int(k))) for s, m, k in zip(sign, mant, exps)]


# ----------------------------------------------------------------- checks
def test_round_f32_matches_numpy_on_doubles():
    """The exact-rational rounding agrees with numpy's float64 -> float32 rounding on doubles."""
    rng = np.random.default_rng(0)
    for x in _doubles(rng, 2000, -120, 120):
        assert round_f32(Fr(x)) == f32(x)


def test_from_f64_precision():
    rng = np.random.default_rng(1)
    for x in _doubles(rng, 3000, -74, 127) + [1.0, -1.0, 0.1, -1 / 3, 2.0 ** -74, 1.5 * 2.0 ** 127]:
        hi, lo = f2_from_f64(x)
        assert abs(exact((hi, lo)) - Fr(x)) <= Fr(2) ** -47 * abs(Fr(x)), x
        # hi is x truncated to FP32's 24 significant bits
        assert abs(Fr(float(hi))) <= abs(Fr(x)) and abs(Fr(x) - Fr(float(hi))) < Fr(2) ** -23 * abs(Fr(x))


def test_from_f64_edges():
    assert f2_from_f64(0.0) == (0.0, 0.0)
    assert f2_from_f64(1e-300)[0] == 0.0 and f2_from_f64(1e-300)[1] == 0.0  # below FP32's range: zero
    hi, lo = f2_from_f64(1e300)
    assert np.isinf(hi) and hi > 0 and lo == 0.0
    hi, lo = f2_from_f64(-1e300)
    assert np.isinf(hi) and hi < 0
    # FP32 values convert exactly (lo == 0)
    for x in (1.0, -0.75, 3.0 * 2.0 ** -20, 2.0 ** 100):
        assert f2_from_f64(x) == (f32(x), 0.0)


def test_to_f64_within_one_ulp():
    rng = np.random.default_rng(2)
    for x in _doubles(rng, 3000, -70, 120):
        hi = f32(x)
        lo = f32(x - float(hi))  # a normalised pair: |lo| <= ulp(hi) / 2
        r = f2_to_f64(hi, lo)
        assert abs(Fr(r) - exact((hi, lo))) <= Fr(math.ulp(r)), (x, r)


def test_roundtrip_through_a_normalised_pair():
    """f2_from_f64 truncates hi, so its lo can reach one ulp of hi; every pair operation returns a
    normalised pair (fast_two_sum), and that is what f2_to_f64 is given in the kernels."""
    rng = np.random.default_rng(3)
    for x in _doubles(rng, 2000, -70, 120):
        r = f2_to_f64(*fast_two_sum(*f2_from_f64(x)))
        assert abs(Fr(r) - Fr(x)) <= Fr(2) ** -47 * abs(Fr(x)) + Fr(math.ulp(x)), x


def test_to_f64_needs_a_normalised_pair():
    """The precondition is real: a pair with |lo| beyond ulp(hi)/2 can leave the rounding-constant
    range of f2_to_f64 (documented beside the helper)."""
    x = 198514904.83191335
    hi, lo = f2_from_f64(x)
    assert abs(Fr(float(lo))) > Fr(math.ulp(float(hi))) / 2
    assert abs(Fr(f2_to_f64(hi, lo)) - Fr(x)) > Fr(2) ** -40 * Fr(x)


def test_error_free_transformations():
    rng = np.random.default_rng(4)
    a = rng.standard_normal(3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-30, 30, 3000).astype(np.float32)
    b = rng.standard_normal(3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-30, 30, 3000).astype(np.float32)
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        assert Fr(float(s)) + Fr(float(e)) == Fr(float(x)) + Fr(float(y))
        big, small = (x, y) if abs(x) >= abs(y) else (y, x)
        s, e = fast_two_sum(big, small)
        assert Fr(float(s)) + Fr(float(e)) == Fr(float(x)) + Fr(float(y))


@pytest.mark.parametrize("op", ["mul", "add"])
def test_pair_arithmetic_relative_error(op):
    rng = np.random.default_rng(5)
    xs = _doubles(rng, 2000, -20, 20)
    ys = _doubles(rng, 2000, -20, 20)
    worst = Fr(0)
    for x, y in zip(xs, ys):
        if op == "add":
            y = math.copysign(y, x)  # same signs: no cancellation
        a, b = f2_from_f64(x), f2_from_f64(y)
        want = exact(a) * exact(b) if op == "mul" else exact(a) + exact(b)
        got = exact(dd_mul(a, b) if op == "mul" else dd_add(a, b))
        worst = max(worst, abs(got - want) / abs(want))
    assert worst <= Fr(2) ** -45, float(worst)
