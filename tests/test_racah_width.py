"""Host-side check of the integer widths the exact {6j} kernel relies on (no device work).

The kernel carries the Racah terms t_z = (z+1)! / [prod_i (z - a_i)! prod_j (b_j - z)!] exactly in
32-bit limbs and picks 8, 16 or 24 limbs per symbol from the bound t_z <= (z+1) 7^z (the seven
factorial arguments sum to z, so t_z is (z+1) times a multinomial coefficient of z into seven
parts) plus 32 bits of headroom for its multiply-then-divide steps. This test checks the bound
and the headroom with exact integers on random admissible symbols up to the largest spins the
table kernel admits."""
import math

import numpy as np
import pytest

LOG2_7 = 2.8074   # the constant the kernel uses (slightly above log2 7 = 2.80735...)


def tri(a, b, c):
    return abs(a - b) <= c <= a + b and (a + b + c) % 2 == 0


def racah_terms(ta, tb, tc, td, te, tf):
    a = [(ta + tb + tc) // 2, (ta + te + tf) // 2, (td + tb + tf) // 2, (td + te + tc) // 2]
    b = [(ta + tb + td + te) // 2, (ta + tc + td + tf) // 2, (tb + tc + te + tf) // 2]
    assert sum(b) == sum(a)          # the seven factorial arguments of each term sum to z
    out = []
    for z in range(max(a), min(b) + 1):
        den = 1
        for n in [z - ai for ai in a] + [bj - z for bj in b]:
            den *= math.factorial(n)
        num = math.factorial(z + 1)
        assert num % den == 0
        out.append((z, num // den))
    return out


def limbs_chosen(zmax):
    bits = math.log2(zmax + 2) + LOG2_7 * zmax + 34.0
    return 8 if bits <= 256 else (16 if bits <= 512 else 24)


def test_log2_7_constant_is_an_upper_bound():
    assert LOG2_7 >= math.log2(7)


@pytest.mark.parametrize("seed", range(4))
def test_terms_fit_the_chosen_width(seed):
    rng = np.random.default_rng(seed)
    checked = 0
    while checked < 150:
        t = [int(v) for v in rng.integers(0, 113, size=6)]   # doubled spins up to 56
        ta, tb, tc, td, te, tf = t
        if not (tri(ta, tb, tc) and tri(ta, te, tf) and tri(td, tb, tf) and tri(td, te, tc)):
            continue
        terms = racah_terms(*t)
        if not terms:
            continue
        zmax = terms[-1][0]
        nl = limbs_chosen(zmax)
        for z, tz in terms:
            assert tz <= (z + 1) * 7 ** z
            # the largest intermediate: a term times a 32-bit numerator, and the sum of all terms
            assert tz.bit_length() + 32 <= 32 * nl
        assert sum(tz for _, tz in terms).bit_length() <= 32 * nl
        checked += 1


def test_width_thresholds():
    # 8 limbs up to zmax = 76, 16 up to 167 (the figures quoted in the kernel's comment)
    assert limbs_chosen(76) == 8 and limbs_chosen(77) == 16
    assert limbs_chosen(167) == 16 and limbs_chosen(168) == 24
