"""Error bound of the float64 reciprocal used in the secular pole sums
(rcp_nr in csrc/secular.cu), checked on the CPU by replaying its steps
exactly: the float32 seed of x's leading 24 bits (truncated), its correctly
rounded float32 reciprocal (the IEEE operation the kernel's rcp.rn.f32 is),
the exact widening to float64, then two Newton-Raphson steps
y <- y + y (1 - x y) with fused multiply-adds (each rounded once, emulated
with exact rationals).  The result must lie within 2 ulp of 1/x across the
exponent range the kernel sends down this path."""
import struct
from fractions import Fraction

import numpy as np


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def seed(x):
    bits = struct.unpack("<Q", struct.pack("<d", x))[0]
    hi, lo = bits >> 32, bits & 0xFFFFFFFF
    e = (hi >> 20) & 0x7FF
    fb = (hi & 0x80000000) | ((e - 896) << 23) | ((hi & 0xFFFFF) << 3) | (lo >> 29)
    f = np.frombuffer(struct.pack("<I", fb), dtype=np.float32)[0]
    return float(np.float32(1.0) / f)   # correctly rounded float32 reciprocal, widened exactly


def rcp_nr(x):
    e = (struct.unpack("<Q", struct.pack("<d", x))[0] >> 52) & 0x7FF
    if e < 1023 - 120 or e > 1023 + 120:
        return 1.0 / x
    y = seed(x)
    r = fma(-x, y, 1.0)
    y = fma(y, r, y)
    r = fma(-x, y, 1.0)
    return fma(y, r, y)


def ulp_err(y, x):
    exact = 1 / Fraction(x)
    return abs(Fraction(y) - exact) / Fraction(np.spacing(abs(float(exact))))


def test_rcp_within_two_ulp():
    rng = np.random.default_rng(7)
    xs = np.concatenate([
        rng.uniform(1.0, 2.0, 2000) * 2.0 ** rng.integers(-119, 120, 2000),
        -rng.uniform(1.0, 2.0, 500) * 2.0 ** rng.integers(-60, 60, 500),
        [1.0, 2.0, 3.0, 0.1, 1 - 2 ** -53, 1 + 2 ** -52, 2.0 ** 119.9, 2.0 ** -119.5],
    ])
    worst = max(ulp_err(rcp_nr(float(x)), float(x)) for x in xs)
    assert worst <= 2, float(worst)


def test_seed_is_float32_accurate():
    """The seed alone is within 2^-22 relative (truncation of x to 24 bits,
    then a correctly rounded float32 reciprocal)."""
    rng = np.random.default_rng(8)
    for x in rng.uniform(1.0, 2.0, 500) * 2.0 ** rng.integers(-100, 100, 500):
        assert abs(seed(float(x)) * float(x) - 1.0) < 2.0 ** -22


def test_out_of_range_takes_division():
    for x in (2.0 ** -125, 2.0 ** 125, 1e-300, 1e300, -3e-200):
        assert rcp_nr(x) == 1.0 / x
