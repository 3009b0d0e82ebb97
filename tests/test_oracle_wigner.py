"""Pins of the oracle's exact Wigner symbols against closed forms, symmetries, orthogonality,
the Biedenharn-Elliott identity, a brute-force magnetic-number network and a library routine."""
import itertools
import math
import random

import mpmath
import pytest

from oracle import wigner

W = wigner


@pytest.fixture(autouse=True)
def _high_precision():
    with mpmath.workdps(50):
        yield


def spins(maxtwo):
    return range(0, maxtwo + 1)


def test_sixj_special_value():
    # {a b c; 0 c b} = (-1)^(a+b+c) / sqrt((2b+1)(2c+1))   (Edmonds eq. 6.3.2)
    n = 0
    for ta, tb, tc in itertools.product(spins(8), repeat=3):
        if not W.tri(ta, tb, tc):
            continue
        v = W.sixj(ta, tb, tc, 0, tc, tb)
        ref = (-1) ** ((ta + tb + tc) // 2) / math.sqrt((tb + 1) * (tc + 1))
        assert v == pytest.approx(ref, rel=1e-15, abs=0)
        n += 1
    assert n > 100


def test_sixj_zero_on_failed_triad():
    assert W.sixj(2, 2, 6, 2, 2, 2) == 0.0      # (1,1,3) fails
    assert W.sixj(1, 2, 2, 2, 2, 2) == 0.0      # parity of (1/2,1,1) fails


def test_sixj_tetrahedral_symmetry():
    rnd = random.Random(5)
    checked = 0
    while checked < 60:
        a = [rnd.randint(0, 10) for _ in range(6)]
        ta, tb, tc, td, te, tf = a
        v = W.sixj_exact(ta, tb, tc, td, te, tf)
        if v[0] == 0:
            continue
        checked += 1
        # column permutations
        for p in itertools.permutations(range(3)):
            top = [a[i] for i in p]
            bot = [a[3 + i] for i in p]
            assert W.sixj_exact(*top, *bot) == v
        # exchange upper and lower in two columns
        assert W.sixj_exact(td, te, tc, ta, tb, tf) == v
        assert W.sixj_exact(ta, te, tf, td, tb, tc) == v


def test_sixj_orthogonality():
    # sum_x (2x+1)(2g+1) {a b x; c d g}{a b x; c d g'} = delta_{g g'}
    for ta, tb, tc, td in [(2, 3, 3, 2), (4, 4, 4, 4), (3, 5, 4, 2), (6, 5, 3, 4)]:
        gs = [g for g in range(0, 20) if W.tri(ta, td, g) and W.tri(tc, tb, g)]
        xs = [x for x in range(0, 20) if W.tri(ta, tb, x) and W.tri(tc, td, x)]
        for g, gp in itertools.product(gs, gs):
            s = mpmath.fsum((x + 1) * (g + 1) * W.sixj_mp(ta, tb, x, tc, td, g)
                            * W.sixj_mp(ta, tb, x, tc, td, gp) for x in xs)
            assert abs(s - (1 if g == gp else 0)) < 1e-30


def test_sixj_biedenharn_elliott():
    # sum_x (-1)^(S+x) (2x+1) {a b x; c d p}{c d x; e f q}{e f x; b a r} = {p q r; e a d}{p q r; f b c}
    rnd = random.Random(11)
    hits = 0
    for _ in range(4000):
        ta, tb, tc, td, te, tf, tp, tq, tr = [rnd.randint(0, 6) for _ in range(9)]
        rhs = W.sixj_mp(tp, tq, tr, te, ta, td) * W.sixj_mp(tp, tq, tr, tf, tb, tc)
        S2 = ta + tb + tc + td + te + tf + tp + tq + tr
        lhs = mpmath.mpf(0)
        nz = False
        for tx in range(0, 30):
            t1 = W.sixj_mp(ta, tb, tx, tc, td, tp)
            if t1 == 0:
                continue
            t2 = W.sixj_mp(tc, td, tx, te, tf, tq)
            t3 = W.sixj_mp(te, tf, tx, tb, ta, tr)
            if t2 == 0 or t3 == 0:
                continue
            nz = True
            e2 = S2 + tx
            assert e2 % 2 == 0
            lhs += (-1) ** (e2 // 2) * (tx + 1) * t1 * t2 * t3
        if nz or rhs != 0:
            hits += 1
            assert abs(lhs - rhs) < 1e-30
        if hits >= 40:
            break
    assert hits >= 12


def test_sixj_matches_library_routine():
    sw = pytest.importorskip("sympy.physics.wigner")
    from sympy import Rational
    rnd = random.Random(2)
    n = 0
    while n < 40:
        a = [rnd.randint(0, 14) for _ in range(6)]
        if W.sixj_exact(*a)[0] == 0:
            continue
        ref = float(sw.wigner_6j(*[Rational(x, 2) for x in a]))
        assert W.sixj(*a) == pytest.approx(ref, rel=1e-14)
        n += 1


def test_threej_closed_form_and_orthogonality():
    # (j j 0; m -m 0) = (-1)^(j-m)/sqrt(2j+1)
    for tj in range(0, 9):
        for tm in range(-tj, tj + 1, 2):
            ref = (-1) ** ((tj - tm) // 2) / math.sqrt(tj + 1)
            assert W.threej(tj, tj, 0, tm, -tm, 0) == pytest.approx(ref, rel=1e-15)
    # sum_{m1 m2} (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3) = delta_{j3 j3'}/(2j3+1)
    t1, t2 = 3, 4
    for t3, t3p in itertools.product(range(1, 8, 2), repeat=2):
        for tm3 in range(-min(t3, t3p), min(t3, t3p) + 1, 2):
            s = mpmath.fsum(W.threej_mp(t1, t2, t3, m1, -m1 - tm3, tm3) * W.threej_mp(t1, t2, t3p, m1, -m1 - tm3, tm3)
                            for m1 in range(-t1, t1 + 1, 2) if abs(-m1 - tm3) <= t2)
            ref = mpmath.mpf(1) / (t3 + 1) if t3 == t3p else 0
            assert abs(s - ref) < 1e-30


def test_threej_matches_library_routine():
    sw = pytest.importorskip("sympy.physics.wigner")
    from sympy import Rational
    rnd = random.Random(3)
    n = 0
    while n < 40:
        t1, t2, t3 = [rnd.randint(0, 10) for _ in range(3)]
        m1 = rnd.randrange(-t1, t1 + 1, 2) if t1 else 0
        m2 = rnd.randrange(-t2, t2 + 1, 2) if t2 else 0
        m3 = -m1 - m2
        if W.threej_exact(t1, t2, t3, m1, m2, m3)[0] == 0:
            continue
        ref = float(sw.wigner_3j(*[Rational(x, 2) for x in (t1, t2, t3, m1, m2, m3)]))
        assert W.threej(t1, t2, t3, m1, m2, m3) == pytest.approx(ref, rel=1e-14)
        n += 1


def _mvals(t):
    return range(-t, t + 1, 2)


@pytest.mark.parametrize("tj", [(2, 2, 2, 2), (1, 3, 2, 2), (3, 3, 1, 1)])
def test_fourjm_orthonormality_and_reflection(tj):
    irng = W.pair_range(*tj)
    for ti, tip in itertools.product(irng, irng):
        s = mpmath.mpf(0)
        for m in itertools.product(*[_mvals(t) for t in tj[:3]]):
            m4 = -sum(m)
            if abs(m4) > tj[3]:
                continue
            mm = (*m, m4)
            s += W.fourjm_mp(tj, mm, ti) * W.fourjm_mp(tj, mm, tip)
        ref = mpmath.mpf(1) / (ti + 1) if ti == tip else 0
        assert abs(s - ref) < 1e-30
    # m -> -m gives (-1)^(j1+j2+j3+j4)
    sg = (-1) ** (sum(tj) // 2)
    for ti in irng:
        for m in itertools.product(*[_mvals(t) for t in tj[:3]]):
            m4 = -sum(m)
            if abs(m4) > tj[3]:
                continue
            mm = (*m, m4)
            assert abs(W.fourjm_mp(tj, tuple(-x for x in mm), ti) - sg * W.fourjm_mp(tj, mm, ti)) < 1e-30


# --- {15j}: brute-force SU(2) BF pentagon network and cyclic relabelling -----------------

FACES = ("12", "13", "14", "15", "23", "24", "25", "34", "35", "45")
NODE_ORDER = {1: ("12", "13", "14", "15"), 2: ("23", "24", "25", "12"), 3: ("34", "35", "13", "23"),
              4: ("45", "14", "24", "34"), 5: ("15", "25", "35", "45")}


def _network(tj, ti):
    """Sum over all magnetic numbers of prod_nodes 4jm^(i_a), links paired by (-1)^(j-m) delta_{m,-m'}.

    A face ab (a < b) carries m at node a and -m at node b.
    """
    j = dict(zip(FACES, tj))
    tot = mpmath.mpf(0)
    for ms in itertools.product(*[_mvals(j[f]) for f in FACES]):
        m = dict(zip(FACES, ms))
        v = mpmath.mpf(1)
        for a in range(1, 6):
            args = NODE_ORDER[a]
            mm = tuple(m[f] if int(f[0]) == a else -m[f] for f in args)
            v *= W.fourjm_mp(tuple(j[f] for f in args), mm, ti[a - 1])
            if v == 0:
                break
        if v == 0:
            continue
        ph = sum((j[f] - m[f]) // 2 for f in FACES)
        tot += (-1) ** ph * v
    return tot


def _ranges(tj):
    j = dict(zip(FACES, tj))
    return [W.pair_range(*[j[f] for f in NODE_ORDER[a]]) for a in range(1, 6)]


@pytest.mark.parametrize("tj", [(1,) * 10, (1, 2, 1, 2, 2, 1, 2, 2, 2, 2), (2, 1, 1, 2, 1, 1, 2, 1, 1, 1)])
def test_fifteenj_equals_bf_network(tj):
    """The printed x-sum {15j} equals the BF network built from the booster 4jm orderings,
    up to one sign that does not depend on the intertwiners (pins the 15j phase reading and
    the 4jm convention together)."""
    rngs = _ranges(tj)
    assert all(rngs)
    ratios = set()
    n = 0
    for ti in itertools.product(*rngs):
        a = W.fifteenj_mp(tj, tj[4:], ti[0], ti[1:])
        b = _network(tj, ti)
        if abs(a) < 1e-25 and abs(b) < 1e-25:
            continue
        n += 1
        assert abs(a) > 1e-25
        ratios.add(round(float(b / a), 12))
    assert n > 0
    assert len(ratios) == 1 and abs(abs(ratios.pop()) - 1) < 1e-12


def _cyc(tj):
    """Relabel nodes a -> a+1 (mod 5): face ab of the new boundary carries the old face (a-1)(b-1)."""
    j = dict(zip(FACES, tj))
    out = []
    for f in FACES:
        a, b = int(f[0]) - 1, int(f[1]) - 1
        a = 5 if a == 0 else a
        b = 5 if b == 0 else b
        key = "%d%d" % (min(a, b), max(a, b))
        out.append(j[key])
    return tuple(out)


def test_fifteenj_cyclic_invariance():
    rnd = random.Random(7)
    done = 0
    while done < 6:
        tj = tuple(rnd.randint(1, 4) for _ in range(10))
        rngs = _ranges(tj)
        if not all(rngs):
            continue
        done += 1
        tjc = _cyc(tj)
        for _ in range(6):
            ti = [rnd.choice(r) for r in rngs]
            a = W.fifteenj_mp(tj, tj[4:], ti[0], ti[1:])
            # intertwiner of old node a sits at new node a+1
            tic = [ti[4], ti[0], ti[1], ti[2], ti[3]]
            b = W.fifteenj_mp(tjc, tjc[4:], tic[0], tic[1:])
            assert abs(a - b) <= 1e-28 * max(1, abs(a))
