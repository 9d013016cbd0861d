"""The acceptance test of the library's fast FP64 division, checked in exact
rational arithmetic on the CPU.

The GPU division (used for the edge weights c_ij, Sec. 3.1) returns a
candidate quotient q only when the exact residual a - b q satisfies
|a - b q| < |b| h(q), where h(q) is the half-gap from q to its nearer
neighbour: half an ulp of q, a quarter of one when |q| is a power of two
(the gap below it is half the gap above).  This file restates that
criterion with Python fractions and checks the property it rests on: a
candidate passes only if it is the correctly rounded quotient, and the
correctly rounded quotient passes except when a / b lies in the outer half
of the wider side of a power of two (where the GPU falls back to the
compiler's division).  The GPU side is held to IEEE quotients by
tests/test_gpu_divide.py.  The last test does the same for the edge
weights' exact doubling 2 a on integer bits (normal, subnormal, overflowing
and infinite a), against the IEEE product.
"""
import math
from fractions import Fraction

import numpy as np


def half_gap(q: float) -> Fraction:
    """The smaller half-gap around a normal, nonzero q, as the GPU code takes
    it: 2^(e-53) for |q| in [2^e, 2^(e+1)), 2^(e-54) at |q| = 2^e."""
    m, e = math.frexp(abs(q))  # |q| = m 2^e, m in [1/2, 1)
    eq = e - 1
    return Fraction(2) ** (eq - 54) if m == 0.5 else Fraction(2) ** (eq - 53)


def accepted(a: float, b: float, q: float) -> bool:
    r = Fraction(a) - Fraction(b) * Fraction(q)
    return abs(r) < abs(Fraction(b)) * half_gap(q)


def rn(a: float, b: float) -> float:
    return float(np.float64(a) / np.float64(b))


def _cases(rng, n):
    a = rng.uniform(1, 2, n) * np.exp2(rng.integers(-60, 60, n)) * rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * np.exp2(rng.integers(-60, 60, n))
    # small-integer divisors, powers of two, quotients near powers of two and near midpoints
    b2 = rng.choice([3.0, 5.0, 7.0, 0.75, 1.5, 1.0, 2.0, 0.5], n)
    q2 = np.exp2(rng.integers(-20, 20, n)) * np.where(rng.random(n) < 0.5, 1.0, 1.0 + rng.integers(-3, 4, n) * 2.0 ** -52)
    a2 = q2 * b2
    return np.concatenate([a, a2]), np.concatenate([b, b2])


def test_only_the_correctly_rounded_quotient_passes():
    rng = np.random.default_rng(2)
    A, B = _cases(rng, 4000)
    for a, b in zip(A.tolist(), B.tolist()):
        q = rn(a, b)
        for cand in (q, math.nextafter(q, math.inf), math.nextafter(q, -math.inf)):
            if accepted(a, b, cand):
                assert cand == q, (a, b, cand, q)


def test_the_correctly_rounded_quotient_passes_unless_beside_a_power_of_two():
    rng = np.random.default_rng(3)
    A, B = _cases(rng, 4000)
    rejected = 0
    for a, b in zip(A.tolist(), B.tolist()):
        q = rn(a, b)
        if not accepted(a, b, q):
            rejected += 1
            # only where q is a power of two and a / b lies above it by at least
            # a quarter ulp (the half-gap on the wider side is not used)
            assert math.frexp(abs(q))[0] == 0.5, (a, b, q)
            exact = Fraction(a) / Fraction(b)
            assert abs(exact) > abs(Fraction(q)), (a, b, q)
    assert rejected < 0.05 * len(A)


def _bits(x: float) -> int:
    import struct
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _from_bits(u: int) -> float:
    import struct
    return struct.unpack("<d", struct.pack("<Q", u & 0xFFFFFFFFFFFFFFFF))[0]


def twice_bits(x: float) -> float:
    """The edge weights' exact doubling on integer bits, as the GPU code
    takes it: exponent + 1 for normal x below the top binade, the
    significand shifted for a subnormal (a carry makes it normal), infinity
    from the top binade, infinity kept."""
    u = _bits(x)
    sign, mag = u & 0x8000000000000000, u & 0x7FFFFFFFFFFFFFFF
    e = mag >> 52
    if e == 0:
        return _from_bits(sign | (mag << 1))
    if e < 2046:
        return _from_bits(u + (1 << 52))
    if e == 2046:
        return _from_bits(sign | 0x7FF0000000000000)
    return x


def test_doubling_on_the_bits_equals_the_product():
    rng = np.random.default_rng(4)
    xs = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072009e-308, 2.2250738585072014e-308, 1.1125369292536007e-308,
          1.7976931348623157e308, -1.7976931348623157e308, 8.98846567431158e307, math.inf, -math.inf, 1.0, -3.5]
    xs += (rng.standard_normal(2000) * np.exp2(rng.integers(-1074, 1024, 2000))).tolist()
    with np.errstate(over="ignore"):
        for x in xs:
            want = float(np.float64(2.0) * np.float64(x))
            got = twice_bits(x)
            assert _bits(got) == _bits(want), (x, got, want)
