"""Exact IEEE binary32 arithmetic on Python Fractions, for deciding test cases
that sit within rounding of a threshold.  fmaf(a, b, c) is the exact a*b + c
rounded once to binary32 (round half to even), as IEEE 754 defines it."""
from fractions import Fraction

import numpy as np


def round_f32(q) -> np.float32:
    q = Fraction(q)
    if q == 0:
        return np.float32(0.0)
    neg = q < 0
    a = -q if neg else q
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    if Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)  # subnormal range keeps the -149 quantum
    quantum = Fraction(2) ** (e - 23)
    m = a / quantum
    f = m.numerator // m.denominator
    rem = m - f
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and f % 2 == 1):
        f += 1
    r = float(f * quantum)
    return np.float32(-r if neg else r)


def F(x) -> Fraction:
    return Fraction(float(np.float32(x)))


def fmaf(a, b, c) -> np.float32:
    return round_f32(F(a) * F(b) + F(c))


def mulf(a, b) -> np.float32:
    return round_f32(F(a) * F(b))


def subf(a, b) -> np.float32:
    return round_f32(F(a) - F(b))
