"""Pins of the oracle's booster quadrature, shell-sum vertex amplitude and boundary contraction."""
import itertools
import math

import mpmath
import numpy as np
import pytest

from oracle import booster, contract, quadrature, vertex, wigner
from paper_2107_13952_gb300 import inputs


@pytest.fixture(autouse=True)
def _prec():
    with mpmath.workdps(40):
        yield


def test_rule_integrates_polynomials():
    xs, ws = quadrature.rule_nodes(40, 7, 6)
    x0 = mpmath.exp(-40)
    for p in range(0, 12):
        s = mpmath.fsum(w * x ** p for x, w in zip(xs, ws))
        ref = (1 - x0 ** (p + 1)) / (p + 1)
        assert abs(s - ref) < 1e-30


@pytest.mark.parametrize("r_max,n,order", [(40, 7, 6), (40, 40, 50), (12, 3, 4)])
def test_rule_panel_geometry(r_max, n, order):
    """Panel layout of Sec. 3 "Booster coefficients": the x-range is cut into n panels with
    |I_k| = k |I_1|, the first (shortest) one at the x -> 0 end, so |I_1| = 2/(n(n+1)) of the
    range. Written here from the paper's statement, not from the oracle: sorted by x, the k-th
    run of `order` nodes must lie inside [x0 + |I_1| k(k-1)/2, x0 + |I_1| k(k+1)/2] and its
    weights must add up to the panel length k |I_1| (a reversed or uniform partition fails)."""
    xs, ws = quadrature.rule_nodes(r_max, n, order)
    pairs = sorted(zip(xs, ws), key=lambda p: p[0])
    x0 = mpmath.exp(-mpmath.mpf(r_max))
    width = (1 - x0) * mpmath.mpf(2) / (n * (n + 1))
    assert len(pairs) == n * order
    for k in range(1, n + 1):
        run = pairs[(k - 1) * order:k * order]
        lo = x0 + width * k * (k - 1) / 2
        hi = x0 + width * k * (k + 1) / 2
        assert all(lo < x < hi for x, _ in run), k
        assert abs(mpmath.fsum(w for _, w in run) - k * width) < mpmath.mpf(10) ** -35 * k * width
    assert abs(x0 + width * n * (n + 1) / 2 - 1) < mpmath.mpf(10) ** -35


@pytest.mark.parametrize("g", [0.5, 1.2])
def test_booster_spin_zero_closed_form(g):
    """All spins 0: d_{000} = sin(g r)/(g sinh r), 4jm = 1, so
    B4 = (1/(4 pi g^4)) int sin^4(g r)/sinh^2 r dr = (F(g) - F(2g)/4)/(4 pi g^4),
    with F(a) = int sin^2(a r)/sinh^2 r dr = (pi a coth(pi a) - 1)/2."""
    xs, ws = quadrature.rule_nodes(40, 40, 30)
    wm = booster.node_weights(xs, ws)
    tabs = [booster.DTable(0, g, [0], xs) for _ in range(4)]
    B, _, _, _ = booster.booster((0, 0, 0, 0), (0, 0, 0, 0), tabs, wm)

    def F(a):
        return (math.pi * a / math.tanh(math.pi * a) - 1) / 2
    ref = (F(g) - F(2 * g) / 4) / (4 * math.pi * g ** 4)
    assert B.shape == (1, 1)
    # the panelled rule resolves the ln(x) oscillation of the first panel to ~1e-11
    assert B[0, 0] == pytest.approx(ref, rel=1e-9)


def test_booster_real_and_symmetric_at_l_equal_j():
    xs, ws = quadrature.rule_nodes(40, 6, 12)
    wm = booster.node_weights(xs, ws)
    for tj in [(2, 2, 2, 2), (1, 3, 2, 2)]:
        tabs = [booster.DTable(t, 1.2, [t], xs) for t in tj]
        B, ir, kr, im = booster.booster(tj, tj, tabs, wm)
        assert im <= 1e-14 * np.abs(B).max()
        np.testing.assert_allclose(B, B.T, rtol=0, atol=1e-15 * np.abs(B).max())
    # odd sum of (l - j): still real with the i^(k-l) phase convention
    tj, tl = (2, 2, 2, 2), (2, 4, 2, 2)
    tabs = [booster.DTable(a, 1.2, [b], xs) for a, b in zip(tj, tl)]
    B, _, _, im = booster.booster(tj, tl, tabs, wm)
    assert im <= 1e-14 * np.abs(B).max()


def test_booster_strand_exchange_phases():
    """The booster couples its strands as (a1 a2)(a3 a4) in both 4jm symbols and integrates a
    product symmetric in the strands, so exchanging strands changes it by the 3j phases alone
    (eq. booster with the 4jm of the framed algorithm): a1 <-> a2 by (-1)^(j1+j2+i+l1+l2+k),
    a3 <-> a4 by (-1)^(j3+j4+i+l3+l4+k), and the pairs (a1 a2) <-> (a3 a4) by (-1)^(2i+2k).
    A booster that coupled (a1 a3)(a2 a4), or a 4jm without its (-1)^(i-m), fails these."""
    xs, ws = quadrature.rule_nodes(40, 6, 12)
    wm = booster.node_weights(xs, ws)
    tj, tl = (2, 1, 3, 2), (4, 3, 5, 2)
    tabs = [booster.DTable(a, 1.2, [b], xs) for a, b in zip(tj, tl)]
    B, ir, kr, _ = booster.booster(tj, tl, tabs, wm)
    assert np.abs(B).max() > 0
    cases = [((1, 0, 2, 3), lambda ti, tk: (tj[0] + tj[1] + ti + tl[0] + tl[1] + tk) // 2),
             ((0, 1, 3, 2), lambda ti, tk: (tj[2] + tj[3] + ti + tl[2] + tl[3] + tk) // 2),
             ((2, 3, 0, 1), lambda ti, tk: ti + tk)]
    for perm, phase in cases:
        Bp, irp, krp, _ = booster.booster(tuple(tj[q] for q in perm), tuple(tl[q] for q in perm),
                                          [tabs[q] for q in perm], wm)
        assert list(irp) == list(ir) and list(krp) == list(kr)
        sign = np.array([[(-1) ** (phase(ti, tk) % 2) for tk in kr] for ti in ir], dtype=float)
        np.testing.assert_allclose(Bp, sign * B, rtol=0, atol=1e-13 * np.abs(B).max())
        assert np.abs(Bp - B).max() > 1e-3 * np.abs(B).max() or np.all(sign == 1)


def test_booster_quadrature_converges():
    tj, tl = (2, 2, 2, 2), (2, 4, 4, 2)
    out = []
    for npan, order in [(20, 20), (40, 25)]:
        xs, ws = quadrature.rule_nodes(40, npan, order)
        wm = booster.node_weights(xs, ws)
        tabs = [booster.DTable(a, 1.2, [b], xs) for a, b in zip(tj, tl)]
        out.append(booster.booster(tj, tl, tabs, wm)[0])
    assert np.abs(out[0] - out[1]).max() <= 1e-9 * np.abs(out[1]).max()


# --- vertex ----------------------------------------------------------------------------

def _fifteenj_tensor(tj):
    I = vertex.intertwiner_ranges(tj)
    T = np.zeros([len(r) for r in I])
    for idx in itertools.product(*[range(len(r)) for r in I]):
        ti = [I[e][idx[e]] for e in range(5)]
        T[idx] = float(wigner.fifteenj_mp(tj, tj[4:], ti[0], ti[1:]))
    return T, I


@pytest.mark.parametrize("tj", [(2,) * 10, (1, 2, 1, 2, 2, 1, 2, 2, 2, 2), (4, 3, 3, 4, 4, 5, 1, 3, 2, 5)])
def test_bf_limit_engine(tj):
    """(2k+1) B = delta_ik at dl = 0 turns the EPRL shell sum into prod sqrt(2i+1) {15j}."""
    assert inputs.boundary_is_valid(tj)
    A = vertex.vertex_amplitude(tj, 0, booster.identity_boosters(tj))
    T, I = _fifteenj_tensor(tj)
    fac = np.ones(1)
    fac = np.sqrt(np.array(I[0]) + 1.0)
    for r in I[1:]:
        fac = np.multiply.outer(fac, np.sqrt(np.array(r) + 1.0))
    np.testing.assert_allclose(A, fac * T, rtol=1e-13, atol=1e-15)


def _random_boosters(tj, dl, seed):
    rng = np.random.default_rng(seed)
    out = {}
    for e in (2, 3, 4, 5):
        n3 = (dl + 1) ** 3
        klo = np.zeros(n3, dtype=np.int64)
        dks = []
        for t in range(n3):
            d = (t // ((dl + 1) ** 2), (t // (dl + 1)) % (dl + 1), t % (dl + 1))
            tl6 = dict(zip(vertex.FREE, [tj[vertex.FACES.index(f)] for f in vertex.FREE]))
            for f, df in zip(vertex.EDGE_TRIPLES[e], d):
                tl6[f] += 2 * df
            bj, bl = vertex.edge_spins(tj, tuple(tl6[f] for f in vertex.FREE))[e]
            kr = wigner.pair_range(*bl)
            klo[t] = kr[0] if kr else 0
            dks.append(len(kr))
        di = len(wigner.pair_range(*vertex.edge_spins(tj, tuple(tj[4:]))[e][0]))
        out[e] = {"B": rng.standard_normal((n3, di, max(dks))), "klo": klo}
    return out


def test_shell_contraction_brute_force():
    """The einsum contraction of one shell equals explicit loops over all indices."""
    tj, dl = (5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 1
    assert inputs.boundary_is_valid(tj)
    bs = _random_boosters(tj, dl, 3)
    six = vertex.SixJCache()
    done = 0
    for s in range(vertex.n_shells(dl)):
        C = vertex.shell_contribution(tj, dl, s, bs, six)
        if C is None:
            continue
        tl = vertex.shell_spins(tj, dl, s)
        I = vertex.intertwiner_ranges(tj)
        K = vertex.k_ranges(tj, tl)
        ref = np.zeros_like(C)
        for i in itertools.product(*[range(len(r)) for r in I]):
            acc = 0.0
            for k in itertools.product(*[range(len(r)) for r in K]):
                w = float(wigner.fifteenj_mp(tj, tl, I[0][i[0]], [K[e][k[e]] for e in range(4)]))
                prod = w
                for e in range(4):
                    b = bs[e + 2]
                    t = vertex.triple_index(tj, dl, e + 2, tl)
                    kk = (K[e][k[e]] - b["klo"][t]) // 2
                    prod *= (K[e][k[e]] + 1) * b["B"][t][i[e + 1], kk]
                acc += prod
            ref[i] = acc
        np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())
        done += 1
        if done == 3:
            break
    assert done == 3


def test_shell_additivity_and_single_shell():
    tj, dl = (2,) * 10, 2
    bs = _random_boosters(tj, dl, 5)
    six = vertex.SixJCache()
    N = vertex.n_shells(dl)
    full = vertex.vertex_amplitude(tj, dl, bs, sixj=six)
    a = vertex.vertex_amplitude(tj, dl, bs, shells=range(0, 300), sixj=six)
    b = vertex.vertex_amplitude(tj, dl, bs, shells=range(300, N), sixj=six)
    np.testing.assert_allclose(a + b, full, rtol=1e-12, atol=1e-14 * np.abs(full).max())
    # dl = 0 is a single shell
    assert vertex.n_shells(0) == 1


def test_contraction_paths_agree_and_gradients():
    tj, dl = (2,) * 10, 1
    bs = _random_boosters(tj, dl, 9)
    I = vertex.intertwiner_ranges(tj)
    psis = inputs.boundary_vectors([len(r) for r in I], seed=1)
    A = vertex.vertex_amplitude(tj, dl, bs)
    a_full = contract.contract_full(A, psis)
    g_full = contract.grad_psi_full(A, psis)
    a, gpsi, gB = contract.contract_by_shell(tj, dl, bs, psis)
    assert abs(a - a_full) <= 1e-13 * abs(a_full)
    for e in range(5):
        np.testing.assert_allclose(gpsi[e], g_full[e], rtol=1e-12, atol=1e-14 * abs(a_full))
    # a is linear in each booster entry: the derivative equals a one-sided difference quotient
    rng = np.random.default_rng(0)
    for e in (2, 5):
        for _ in range(3):
            t = int(rng.integers(0, (dl + 1) ** 3))
            i = int(rng.integers(0, bs[e]["B"].shape[1]))
            k = int(rng.integers(0, bs[e]["B"].shape[2]))
            h = 1e-3
            bs2 = {f: {"B": bs[f]["B"].copy(), "klo": bs[f]["klo"]} for f in bs}
            bs2[e]["B"][t, i, k] += h
            a2 = contract.contract_full(vertex.vertex_amplitude(tj, dl, bs2), psis)
            assert abs((a2 - a_full) / h - gB[e][t, i, k]) <= 1e-9 * max(1.0, abs(gB[e][t, i, k]))
