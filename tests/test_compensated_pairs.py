"""The compensated-pair arithmetic that SF_MIXED_FF uses for its {6j} contractions, checked on the
host in IEEE binary32 (numpy float32): a value is a (hi, lo) pair of floats, products are formed
exactly (Dekker's TwoProduct; with float32 operands the product is exact in float64, which plays
the role of the FMA), high parts are summed with Knuth's TwoSum and all rounding errors go to a
second float sum (Ogita, Rump and Oishi, Dot2). The claim behind the design: the result, kept as
a pair, is within a few units of 2^-48 of the sum of |terms| even when the terms cancel, i.e.
far below the 6e-8 relative error of the FP32 booster contractions. No device work."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def two_prod(a, b):
    p = f32(a * b)
    e = f32(np.float64(a) * np.float64(b) - np.float64(p))   # exact: a*b has at most 48 bits
    return p, e


def split(d):
    hi = f32(d)
    return hi, f32(d - np.float64(hi))


def dot2_pairs(xs, ys):
    """sum_k x_k y_k with x_k, y_k given as float64, split into (hi, lo) float pairs."""
    sh, sl = f32(0.0), f32(0.0)
    for x, y in zip(xs, ys):
        ah, al = split(x)
        bh, bl = split(y)
        p, e = two_prod(ah, bh)
        e = f32(e + f32(ah * bl))
        e = f32(e + f32(al * bh))
        s, t = two_sum(sh, p)
        sh = s
        sl = f32(sl + f32(t + e))
    return two_sum(sh, sl)



@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n", [8, 27])
def test_dot2_pairs_error_bound(seed, n):
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(200):
        # alternating signs and a near-cancelling last term, like a {6j} sum over x
        xs = rng.standard_normal(n) * np.where(np.arange(n) % 2, -1.0, 1.0) * 1e-2
        ys = rng.standard_normal(n)
        ys[-1] = -float(np.dot(xs[:-1], ys[:-1]) / xs[-1]) * (1 + 1e-9 * rng.standard_normal())
        h, l = dot2_pairs(xs, ys)
        got = Fraction(float(h)) + Fraction(float(l))
        # the reference is the exact dot product of the split operands' full values
        ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(xs, ys))
        scale = sum(abs(float(x) * float(y)) for x, y in zip(xs, ys))
        worst = max(worst, float(abs(got - ref)) / scale)
    # splitting the operands costs 2^-48 each; the compensated sum adds a few units more
    assert worst <= 16 * n * 2.0 ** -48, worst


def test_plain_float32_would_not_do():
    # the same cancelling sums in plain float32 lose almost all digits: the pairs are needed
    rng = np.random.default_rng(1)
    n = 27
    xs = rng.standard_normal(n) * 1e-2
    ys = rng.standard_normal(n)
    ys[-1] = -float(np.dot(xs[:-1], ys[:-1]) / xs[-1]) * (1 + 1e-9)
    plain = f32(0.0)
    for x, y in zip(xs, ys):
        plain = f32(plain + f32(f32(x) * f32(y)))
    ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(xs, ys))
    h, l = dot2_pairs(xs, ys)
    err_plain = abs(Fraction(float(plain)) - ref)
    err_pair = abs(Fraction(float(h)) + Fraction(float(l)) - ref)
    assert err_pair * 1000 < err_plain
