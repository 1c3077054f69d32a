"""The binary32-pair arithmetic of the library's binary64-accuracy parts (estimator forms, mixed
refinement), restated in numpy binary32 and checked against exact rational arithmetic: the bounds its
comments state hold for the scheme itself.  (The CUDA kernels are checked on the GPU against the
binary64 forms and the oracle.)

* split: hi = x cut to 24 significand bits, lo = the next 24 bits: |x - hi - lo| < 2^-47 |x|;
* TwoSum: s + e = a + b exactly;
* a running sum of pair products (exact product by fma, errors accumulated in lo, al*bl dropped):
  within 2^-44 of the exact sum relative to the sum of the magnitudes of the terms.
"""

import struct
from fractions import Fraction

import numpy as np

f32 = np.float32


def split(x: float):
    """hi: x with its significand cut to 24 bits; lo: the next 24 bits of the rest (truncated)."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    sign = -1.0 if b >> 63 else 1.0
    e = (b >> 52) & 0x7FF
    mant = b & ((1 << 52) - 1)
    hi = sign * (1 + (mant >> 29) / 2.0**23) * 2.0 ** (e - 1023)
    r = mant & ((1 << 29) - 1)
    if r == 0:
        return f32(hi), f32(0.0)
    p = r.bit_length() - 1
    m24 = r >> (p - 23) if p >= 23 else r << (23 - p)
    lo = sign * m24 * 2.0 ** (p - 23) * 2.0 ** (e - 1023 - 52)
    return f32(hi), f32(lo)


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fma32(a, b, c):
    """binary32 fma: the exact a*b + c rounded once."""
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def acc_products(pairs):
    hi, lo = f32(0), f32(0)
    for (ah, al), (bh, bl) in pairs:
        p = f32(ah * bh)
        e = fma32(ah, bh, -p)
        e = fma32(ah, bl, e)
        e = fma32(al, bh, e)
        hi, t = two_sum(hi, p)
        lo = f32(lo + f32(t + e))
    s = f32(hi + lo)
    return s, f32(lo - f32(s - hi))


def test_split_keeps_48_bits():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000),
                         [1.0, -1.0, 1.0 + 2.0**-52, 3.0, 2.0**-100, -(2.0**100)]])
    for x in xs:
        h, l = split(float(x))
        err = abs(Fraction(float(x)) - Fraction(float(h)) - Fraction(float(l)))
        assert err < Fraction(2) ** -47 * abs(Fraction(float(x))), x
        # hi is x truncated toward zero to 24 significand bits
        assert abs(float(h)) <= abs(float(x)) and abs(float(x) - float(h)) < 2.0**-23 * abs(float(x))


def test_two_sum_is_exact():
    rng = np.random.default_rng(1)
    a = (rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000)).astype(np.float32)
    b = (rng.standard_normal(5000) * 10.0 ** rng.integers(-8, 8, 5000)).astype(np.float32)
    for x, y in zip(a, b):
        s, e = two_sum(x, y)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(x)) + Fraction(float(y))


def test_pair_product_sums_keep_44_bits():
    """Eight pair products, as one node of the estimator's form or of the residual: the running
    (hi, lo) sum is within 2^-44 of the exact sum of the binary64 products, relative to the sum of
    the terms' magnitudes (cancellation is measured against that, as for any floating-point sum)."""
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(400):
        s = rng.standard_normal(8) * 10.0 ** rng.integers(-3, 3)
        x = rng.standard_normal(8) * 10.0 ** rng.integers(-6, 1)
        pairs = [(split(float(a)), split(float(b))) for a, b in zip(s, x)]
        h, l = acc_products(pairs)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(s, x))
        mag = sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(s, x))
        err = abs(Fraction(float(h)) + Fraction(float(l)) - exact) / mag
        worst = max(worst, float(err))
    assert worst < 2.0**-44, worst
