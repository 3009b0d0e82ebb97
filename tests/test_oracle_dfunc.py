"""Pins of the oracle's SL(2,C) boost matrix elements (Sec. 3, eq. francois) against the
defining integral, a textbook closed form, unitarity, the boost generator, the large-r
exponential structure the paper prints, and the reflection symmetry m -> -m."""
import math

import mpmath
import pytest

from oracle import dfunc


@pytest.fixture(autouse=True)
def _prec():
    with mpmath.workdps(30):
        yield


@pytest.mark.parametrize("tk,tl,tm,g,r", [
    (2, 2, 0, 1.2, 0.7), (2, 6, -2, 1.2, 0.05), (1, 5, 1, 5.0, 1.3),
    (3, 7, -1, 0.1, 2.5), (4, 8, 4, 1.2, 4.0), (2, 4, 2, 1.2, 9.0)])
def test_closed_form_equals_definition(tk, tl, tm, g, r):
    rho = g * (tk / 2 + 1)
    a = dfunc.d_definition(tk, rho, tl, tm, r, dps=25)
    b = dfunc.DClosed(tk, rho, tl, tm).eval(r, dps=25)
    assert abs(a - b) <= 1e-20 * max(abs(a), 1e-3)


@pytest.mark.parametrize("g", [0.1, 1.2, 5.0])
def test_k0_is_elementary_spherical_function(g):
    # (rho, k) = (gamma, 0): d_{000}(r) = sin(rho r) / (rho sinh r)
    dc = dfunc.DClosed(0, g, 0, 0)
    for r in (0.01, 0.5, 2.0, 7.0, 30.0):
        gm = mpmath.mpf(g)
        ref = mpmath.sin(gm * r) / (gm * mpmath.sinh(r))
        v = dc.eval(r, dps=25)
        assert abs(v - ref) <= 1e-22 * max(abs(ref), 1e-30)


def test_identity_at_r0():
    for tk, tl, tm in [(2, 2, 0), (2, 4, 2), (3, 3, -1), (3, 9, 3)]:
        v = dfunc.DClosed(tk, 1.2 * (tk / 2 + 1), tl, tm).eval(1e-9, dps=20)
        ref = 1 if tl == tk else 0
        assert abs(v - ref) < 1e-8


@pytest.mark.parametrize("tk,tm", [(2, 0), (2, 2), (3, -1)])
def test_unitarity_row(tk, tm):
    # sum_l |d_{k l m}(r)|^2 = 1 (first row of a unitary matrix); l truncated at k + 24
    rho = 1.2 * (tk / 2 + 1)
    for r in (0.3, 0.8):
        s = mpmath.fsum(abs(dfunc.DClosed(tk, rho, tk + 2 * n, tm).eval(r, dps=20)) ** 2 for n in range(25))
        assert abs(s - 1) < 1e-12


@pytest.mark.parametrize("tk,tm,g", [(2, 2, 1.2), (2, -2, 1.2), (3, 1, 5.0), (4, 0, 0.1)])
def test_boost_generator(tk, tm, g):
    # d'_{kkm}(0) = -i <k m| K |k m> = -i rho m / (k+1) = -i gamma m
    rho = g * (tk / 2 + 1)
    h = mpmath.mpf("1e-10")
    dc = dfunc.DClosed(tk, rho, tk, tm)
    der = (dc.eval(h, dps=30) - 1) / h
    assert abs(der.imag + g * tm / 2) < 1e-8
    assert abs(der.real) < 1e-8


@pytest.mark.parametrize("tk,tl,tm", [(2, 6, 2), (2, 6, -2), (3, 5, 1), (4, 4, 0)])
def test_large_r_exponential_structure(tk, tl, tm):
    # d(r) ~ C exp(-r(1 + k - |m|)) exp(-+ i rho r): the leading terms of eq. francois
    g = 1.2
    rho = g * (tk / 2 + 1)
    dc = dfunc.DClosed(tk, rho, tl, tm)
    rho = mpmath.mpf(rho)
    k, m = tk / 2, tm / 2
    r1, r2 = 30, 31
    ratio = dc.eval(r2, dps=25) / dc.eval(r1, dps=25)
    sgn = -1 if m > 0 else 1
    if m == 0:
        # both families decay alike: d e^{r(1+k)} = C+ e^{i rho r} + C- e^{-i rho r} + O(e^{-2r});
        # fit C+- at r = 30, 31 and predict r = 32
        f = [dc.eval(r, dps=25) * mpmath.exp(r * (1 + k)) for r in (30, 31, 32)]
        M = mpmath.matrix([[mpmath.expj(rho * 30), mpmath.expj(-rho * 30)],
                           [mpmath.expj(rho * 31), mpmath.expj(-rho * 31)]])
        c = mpmath.lu_solve(M, mpmath.matrix([f[0], f[1]]))
        pred = c[0] * mpmath.expj(rho * 32) + c[1] * mpmath.expj(-rho * 32)
        assert abs(pred - f[2]) < 1e-20 * abs(f[2]) + 1e-20
    else:
        ref = mpmath.exp(-(1 + k - abs(m))) * mpmath.expj(sgn * rho)
        assert abs(ratio - ref) < 1e-10


@pytest.mark.parametrize("tk,tl,tm", [(2, 4, 2), (3, 7, 1), (2, 6, 0)])
def test_reflection_symmetry(tk, tl, tm):
    # conj(d_{k l m}) = (-1)^(k-l) d_{k l -m} with the basis phases used here
    rho = 1.2 * (tk / 2 + 1)
    a = dfunc.DClosed(tk, rho, tl, tm)
    b = dfunc.DClosed(tk, rho, tl, -tm)
    sg = (-1) ** ((tl - tk) // 2)
    for r in (0.2, 1.5, 6.0):
        va, vb = a.eval(r, dps=25), b.eval(r, dps=25)
        assert abs(mpmath.conj(va) - sg * vb) < 1e-20
