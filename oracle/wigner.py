"""Exact SU(2) recoupling symbols for the oracle.

Test infrastructure only: nothing in the product package may import this module.

Every spin is passed DOUBLED (``tj = 2*j``) so that half-integers are exact integers.
Values are computed exactly with Python integers and ``fractions.Fraction``; a symbol is
returned as ``(S, R)`` meaning ``value = S * sqrt(R)`` with ``S`` an integer or Fraction and
``R`` a non-negative Fraction, and rounded to float or mpmath only at the very end.

Formulas (standard textbook forms, the ones the paper's Wigner library evaluates exactly,
Sec. 3 "Internals", reference [Johansson-Forssen 2015]):

* {6j}: Racah's single-sum formula (Edmonds, Angular Momentum in QM, eq. 6.3.7).
* (3j): Racah's formula (Edmonds eq. 3.7.3).
* 4jm: two 3j symbols coupled through the intertwiner spin, the normalisation that makes the
  factors sqrt(2i+1) and (2k+1) of the vertex amplitude (Sec. 2, eq. vertex-ampl) orthonormalise
  the intertwiner basis.
* {15j}: the auxiliary-spin sum of five {6j} printed in Sec. 2, eq. 15j.
"""
from fractions import Fraction
from functools import lru_cache
import math

import mpmath


def tri(ta, tb, tc):
    """Triangle condition for doubled spins: |a-b| <= c <= a+b and a+b+c integer."""
    return abs(ta - tb) <= tc <= ta + tb and (ta + tb + tc) % 2 == 0


def pair_range(ta, tb, tc, td):
    """Doubled values of x with tri(a,b,x) and tri(c,d,x), in steps of 1 (2 when doubled).

    This is the range of an intertwiner that couples the pair (a,b) to the pair (c,d).
    Empty list when no such x exists (including a parity clash between a+b and c+d).
    """
    if (ta + tb + tc + td) % 2:
        return []
    lo = max(abs(ta - tb), abs(tc - td))
    hi = min(ta + tb, tc + td)
    return list(range(lo, hi + 1, 2)) if lo <= hi else []


@lru_cache(maxsize=None)
def _fact(n):
    return math.factorial(n)


def _delta2(ta, tb, tc):
    """Triangle coefficient squared, Delta(abc)^2 = (a+b-c)!(a-b+c)!(-a+b+c)!/(a+b+c+1)!."""
    return Fraction(_fact((ta + tb - tc) // 2) * _fact((ta - tb + tc) // 2) * _fact((-ta + tb + tc) // 2),
                    _fact((ta + tb + tc) // 2 + 1))


@lru_cache(maxsize=None)
def sixj_exact(ta, tb, tc, td, te, tf):
    """{a b c; d e f} = S * sqrt(R) exactly (Edmonds eq. 6.3.7). Returns (0, 0) if a triad fails."""
    if not (tri(ta, tb, tc) and tri(ta, te, tf) and tri(td, tb, tf) and tri(td, te, tc)):
        return 0, Fraction(0)
    a1 = (ta + tb + tc) // 2
    a2 = (ta + te + tf) // 2
    a3 = (td + tb + tf) // 2
    a4 = (td + te + tc) // 2
    b1 = (ta + tb + td + te) // 2
    b2 = (ta + tc + td + tf) // 2
    b3 = (tb + tc + te + tf) // 2
    zmin = max(a1, a2, a3, a4)
    zmax = min(b1, b2, b3)
    S = 0
    for z in range(zmin, zmax + 1):
        num = _fact(z + 1)
        den = (_fact(z - a1) * _fact(z - a2) * _fact(z - a3) * _fact(z - a4)
               * _fact(b1 - z) * _fact(b2 - z) * _fact(b3 - z))
        assert num % den == 0  # each Racah term is an integer (multinomial times z+1)
        S += (-1) ** z * (num // den)
    R = _delta2(ta, tb, tc) * _delta2(ta, te, tf) * _delta2(td, tb, tf) * _delta2(td, te, tc)
    return S, R


@lru_cache(maxsize=None)
def threej_exact(t1, t2, t3, tm1, tm2, tm3):
    """(j1 j2 j3; m1 m2 m3) = S * sqrt(R) exactly (Edmonds eq. 3.7.3)."""
    if tm1 + tm2 + tm3 != 0 or not tri(t1, t2, t3):
        return 0, Fraction(0)
    for tj, tm in ((t1, tm1), (t2, tm2), (t3, tm3)):
        if abs(tm) > tj or (tj + tm) % 2:
            return 0, Fraction(0)
    j1m1p, j1m1m = (t1 + tm1) // 2, (t1 - tm1) // 2
    j2m2p, j2m2m = (t2 + tm2) // 2, (t2 - tm2) // 2
    j3m3p, j3m3m = (t3 + tm3) // 2, (t3 - tm3) // 2
    # t ranges so that all six factorial arguments below are >= 0
    k1 = (t3 - t2 + tm1) // 2          # j3 - j2 + m1
    k2 = (t3 - t1 - tm2) // 2          # j3 - j1 - m2
    k3 = (t1 + t2 - t3) // 2           # j1 + j2 - j3
    k4 = j1m1m                          # j1 - m1
    k5 = j2m2p                          # j2 + m2
    tmin = max(0, -k1, -k2)
    tmax = min(k3, k4, k5)
    S = Fraction(0)
    for t in range(tmin, tmax + 1):
        S += Fraction((-1) ** t, _fact(t) * _fact(k1 + t) * _fact(k2 + t) * _fact(k3 - t)
                      * _fact(k4 - t) * _fact(k5 - t))
    e = (t1 - t2 - tm3) // 2           # j1 - j2 - m3, an integer (possibly negative)
    if e % 2:
        S = -S
    R = _delta2(t1, t2, t3) * (_fact(j1m1p) * _fact(j1m1m) * _fact(j2m2p) * _fact(j2m2m)
                               * _fact(j3m3p) * _fact(j3m3m))
    return S, R


def to_mpf(SR, dps=50):
    """Value S*sqrt(R) as an mpmath number at ``dps`` digits."""
    S, R = SR
    if S == 0 or R == 0:
        return mpmath.mpf(0)
    with mpmath.workdps(dps + 10):
        v = mpmath.mpf(S.numerator if isinstance(S, Fraction) else S)
        if isinstance(S, Fraction):
            v /= S.denominator
        v *= mpmath.sqrt(mpmath.mpf(R.numerator) / R.denominator)
    return +v


def to_float(SR):
    """Correctly rounded double (barring a tie at 200 bits) of S*sqrt(R)."""
    with mpmath.workprec(200):
        return float(to_mpf(SR, 60))


def sixj(ta, tb, tc, td, te, tf):
    """{6j} as a double (rounded once from the exact value)."""
    return to_float(sixj_exact(ta, tb, tc, td, te, tf))


def sixj_mp(ta, tb, tc, td, te, tf, dps=50):
    return to_mpf(sixj_exact(ta, tb, tc, td, te, tf), dps)


def threej(t1, t2, t3, tm1, tm2, tm3):
    return to_float(threej_exact(t1, t2, t3, tm1, tm2, tm3))


def threej_mp(t1, t2, t3, tm1, tm2, tm3, dps=50):
    return to_mpf(threej_exact(t1, t2, t3, tm1, tm2, tm3), dps)


def fourjm_mp(tj, tm, ti, dps=50):
    """4jm symbol (j1 j2 j3 j4; m1 m2 m3 m4)^(i), the intertwiner of Sec. 2, eq. booster.

    Couples (j1 j2) to i and i to (j3 j4):
        sum_m (-1)^(i-m) (j1 j2 i; m1 m2 m) (i j3 j4; -m m3 m4).
    Only m = -(m1+m2) contributes. Normalisation: sum over all m of 4jm^(i) 4jm^(i') equals
    delta_{ii'}/(2i+1).
    """
    t1, t2, t3, t4 = tj
    m1, m2, m3, m4 = tm
    if m1 + m2 + m3 + m4 != 0:
        return mpmath.mpf(0)
    tmi = -(m1 + m2)
    if abs(tmi) > ti or (ti + tmi) % 2:
        return mpmath.mpf(0)
    ph = -1 if ((ti - tmi) // 2) % 2 else 1
    a = threej_mp(t1, t2, ti, m1, m2, tmi, dps)
    if a == 0:
        return mpmath.mpf(0)
    b = threej_mp(ti, t3, t4, -tmi, m3, m4, dps)
    return ph * a * b


def fifteenj_phase_exponent(ti1, tk2, tk3, tk4, tk5, tj12, tj13, tj14, tj15,
                            tl23, tl24, tl25, tl34, tl35, tl45):
    """Doubled exponent of the {15j} sign: twice the sum of all fifteen entries (Sec. 2, eq. 15j)."""
    return (ti1 + tk2 + tk3 + tk4 + tk5 + tj12 + tj13 + tj14 + tj15
            + tl23 + tl24 + tl25 + tl34 + tl35 + tl45)


def fifteenj_mp(tj, tl, ti1, tk, dps=40):
    """{15j} of the first kind as the auxiliary-spin sum of five {6j} (Sec. 2, eq. 15j).

    tj: the ten doubled boundary spins (j12, j13, j14, j15, j23, j24, j25, j34, j35, j45);
    tl: the six doubled virtual spins (l23, l24, l25, l34, l35, l45);
    ti1: doubled i1; tk: doubled (k2, k3, k4, k5).

        {15j} = (-1)^E sum_x (2x+1) {i1 l25 x; k5 j14 j15} {j14 k5 x; l35 k4 l45}
                 {k4 l35 x; k3 l24 l34} {l24 k3 x; j13 k2 l23} {k2 j13 x; i1 l25 j12}

    with E the sum of the fifteen entries of the 3x5 array (the reading of the elided exponent).
    Raises ValueError if E is not an integer.
    """
    j12, j13, j14, j15, j23, j24, j25, j34, j35, j45 = tj
    l23, l24, l25, l34, l35, l45 = tl
    k2, k3, k4, k5 = tk
    i1 = ti1
    E2 = fifteenj_phase_exponent(i1, k2, k3, k4, k5, j12, j13, j14, j15, l23, l24, l25, l34, l35, l45)
    if E2 % 2:
        raise ValueError("non-integer 15j phase exponent")
    sgn = -1 if (E2 // 2) % 2 else 1
    tot = mpmath.mpf(0)
    with mpmath.workdps(dps):
        lo = abs(i1 - l25)
        hi = i1 + l25
        for x in range(lo, hi + 1, 2):
            s1 = sixj_mp(i1, l25, x, k5, j14, j15, dps)
            if s1 == 0:
                continue
            s2 = sixj_mp(j14, k5, x, l35, k4, l45, dps)
            if s2 == 0:
                continue
            s3 = sixj_mp(k4, l35, x, k3, l24, l34, dps)
            if s3 == 0:
                continue
            s4 = sixj_mp(l24, k3, x, j13, k2, l23, dps)
            if s4 == 0:
                continue
            s5 = sixj_mp(k2, j13, x, i1, l25, j12, dps)
            tot += (x + 1) * s1 * s2 * s3 * s4 * s5
    return sgn * tot
