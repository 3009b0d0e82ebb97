"""Parity of the CUDA path with the oracle, stage by stage, through the C ABI.

* {6j} tables: every entry within 1 ulp of the exactly computed symbol (correct rounding).
* rapidity rule nodes: relative 1e-14.
* d-tables: max |difference| <= 1e-12 * max|d| per face.
* boosters: max |difference| <= 1e-11 * max|B| per edge (same rule, each side its own nodes).
* vertex tensor: normwise relative error <= 1e-10 (FP64 target), with uploaded (oracle or random)
  boosters <= 1e-12; shell-range additivity and shell lists.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import quadrature as oq
from oracle import vertex as ov
from oracle import wigner as ow
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu

SMALL_RULE = (40.0, 4, 10)
F = ov.FACES


def _tables(two_j, dl, gamma=1.2):
    return sf.sf_6j_table([sf.vertex(two_j, gamma, dl)])


def _sixj_args(table, slot, D, tj, a, b, x):
    j = dict(zip(F, tj))
    if table == 1:
        l25 = j["25"] + 2 * slot
        return (a, l25, x, b, j["14"], j["15"])
    if table == 2:
        l35, l45 = j["35"] + 2 * (slot // D), j["45"] + 2 * (slot % D)
        return (j["14"], a, x, l35, b, l45)
    if table == 3:
        l24, l34, l35 = j["24"] + 2 * (slot // (D * D)), j["34"] + 2 * ((slot // D) % D), j["35"] + 2 * (slot % D)
        return (a, l35, x, b, l24, l34)
    if table == 4:
        l23, l24 = j["23"] + 2 * (slot // D), j["24"] + 2 * (slot % D)
        return (l24, a, x, j["13"], b, l23)
    l25 = j["25"] + 2 * slot
    return (a, j["13"], x, b, l25, j["12"])


def _check_6j(t, tj, dl, max_per_table=None, seed=0):
    D = dl + 1
    rng = np.random.default_rng(seed)
    checked = 0
    for k in range(1, 6):
        vals = sf.table_copy(t, 0, sf.SF_TAB_6J, k).numpy()
        slots = sf.table_copy(t, 0, sf.SF_TAB_6J_SLOTS, k).numpy()
        entries = []
        for si, (off, alo, blo, xlo, na, nb, nx, _) in enumerate(slots):
            for ia in range(na):
                for ib in range(nb):
                    for ix in range(nx):
                        entries.append((si, off + (ia * nb + ib) * nx + ix, alo + 2 * ia, blo + 2 * ib, xlo + 2 * ix))
        if max_per_table and len(entries) > max_per_table:
            pick = rng.choice(len(entries), size=max_per_table, replace=False)
            entries = [entries[i] for i in pick]
        for si, e, a, b, x in entries:
            ref = ow.sixj(*_sixj_args(k, si, D, tj, a, b, x))
            got = vals[e]
            assert abs(got - ref) <= np.spacing(abs(ref)), (k, si, a, b, x, got, ref)
            checked += 1
    return checked


@pytest.mark.parametrize("tj,dl", [((2,) * 10, 2), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2), ((1,) * 10, 3)])
def test_6j_tables_exact_full(lib, tj, dl):
    t = _tables(tj, dl)
    assert _check_6j(t, tj, dl) > 100


@pytest.mark.parametrize("tj,dl", [((16,) * 10, 10), ((8,) * 10, 20), ((12,) * 10, 12)])
def test_6j_tables_exact_sampled_large(lib, tj, dl):
    t = _tables(tj, dl)
    assert _check_6j(t, tj, dl, max_per_table=400, seed=dl) == 2000


def _racah_zmax(ta, tb, tc, td, te, tf):
    return min((ta + tb + td + te) // 2, (ta + tc + td + tf) // 2, (tb + tc + te + tf) // 2)


def test_6j_tables_exact_wide_limbs(lib):
    """Spins 28 at dl 0, the largest the table kernel admits: the top S3 entries have Racah sums up
    to z = 140, beyond the 8-limb width (z <= 76), so both limb widths that can occur (8 and 16;
    the 24-limb path needs z > 167) are compared against the exact symbol."""
    tj, dl = (56,) * 10, 0
    t = _tables(tj, dl)
    vals = sf.table_copy(t, 0, sf.SF_TAB_6J, 3).numpy()
    (off, alo, blo, xlo, na, nb, nx, _), = sf.table_copy(t, 0, sf.SF_TAB_6J_SLOTS, 3).numpy()
    widths = {8: 0, 16: 0}
    rng = np.random.default_rng(5)
    for it in range(4000):
        # every other draw near the top of the box, where z is largest
        if it % 2:
            ia, ib = na - 1 - int(rng.integers(0, 1 + na // 6)), nb - 1 - int(rng.integers(0, 1 + nb // 6))
        else:
            ia, ib = int(rng.integers(0, na)), int(rng.integers(0, nb))
        ix = int(rng.integers(0, nx))
        args = _sixj_args(3, 0, dl + 1, tj, alo + 2 * ia, blo + 2 * ib, xlo + 2 * ix)
        ref = ow.sixj(*args)
        if ref == 0.0:
            continue
        z = _racah_zmax(*args)
        w = 8 if z <= 76 else 16
        if widths[w] >= 40:
            continue
        got = vals[off + (ia * nb + ib) * nx + ix]
        assert abs(got - ref) <= np.spacing(abs(ref)), (args, got, ref)
        widths[w] += 1
    assert min(widths.values()) > 0, widths


def test_rule_nodes(lib):
    t = _tables((2,) * 10, 0)
    sf.sf_boosters(t, (40.0, 40, 50))
    x = sf.table_copy(t, 0, sf.SF_TAB_NODES, 0).numpy()
    w = sf.table_copy(t, 0, sf.SF_TAB_NODES, 1).numpy()
    r = sf.table_copy(t, 0, sf.SF_TAB_NODES, 2).numpy()
    X, Wt = oq.rule_nodes(40.0, 40, 50)
    X = np.array([float(v) for v in X])
    Wt = np.array([float(v) for v in Wt])
    pg, po = np.argsort(x), np.argsort(X)      # node order inside a panel is not part of the rule
    np.testing.assert_allclose(x[pg], X[po], rtol=1e-14, atol=0)
    np.testing.assert_allclose(w[pg], Wt[po], rtol=1e-12, atol=0)
    np.testing.assert_allclose(r[pg], -np.log(X[po]), rtol=1e-13, atol=1e-16)


def _oracle_dtable(tk, gamma, nl, rule):
    xs, _ = oq.rule_nodes(*rule)
    tab = ob.DTable(tk, gamma, [tk + 2 * p for p in range(nl)], xs)
    out = np.array([[tab.get(tk + 2 * p, tm) for tm in range(-tk, tk + 1, 2)] for p in range(nl)])
    return out[..., np.argsort(np.array([float(x) for x in xs]))]


def _gpu_order(t):
    return np.argsort(sf.table_copy(t, 0, sf.SF_TAB_NODES, 0).numpy())


@pytest.mark.parametrize("tj,dl,gamma", [((2,) * 10, 1, 1.2), ((1, 2, 1, 2, 2, 1, 2, 2, 2, 2), 2, 5.0)])
def test_dtables(lib, tj, dl, gamma):
    t = _tables(tj, dl, gamma)
    sf.sf_boosters(t, SMALL_RULE)
    nn = SMALL_RULE[1] * SMALL_RULE[2]
    for f in range(10):
        nl = 1 if f < 4 else dl + 1
        got = sf.table_copy(t, 0, sf.SF_TAB_D, f).numpy().reshape(nl, tj[f] + 1, nn)[..., _gpu_order(t)]
        ref = _oracle_dtable(tj[f], gamma, nl, SMALL_RULE)
        err = np.abs(got - ref).max()
        assert err <= 1e-12 * np.abs(ref).max(), (f, err, np.abs(ref).max())


def test_dtables_large_spin_sampled(lib):
    # j = 4, l up to 4 + 12, gamma = 5 (rho = 25): a few (l, m) rows against the oracle
    tj, dl, gamma = (8,) * 10, 12, 5.0
    t = _tables(tj, dl, gamma)
    sf.sf_boosters(t, SMALL_RULE)
    nn = SMALL_RULE[1] * SMALL_RULE[2]
    got = sf.table_copy(t, 0, sf.SF_TAB_D, 9).numpy().reshape(dl + 1, 9, nn)[..., _gpu_order(t)]
    xs, _ = oq.rule_nodes(*SMALL_RULE)
    xs = sorted(xs)
    rho = gamma * (4 + 1)
    from oracle import dfunc
    import mpmath
    worst = 0.0
    for p, tm in [(0, 8), (6, 0), (12, -8), (12, 4), (3, -2)]:
        dc = dfunc.DClosed(8, rho, 8 + 2 * p, tm)
        ref = np.array([complex(dc.eval(-mpmath.log(x), 20)) for x in xs])
        worst = max(worst, np.abs(got[p, (tm + 8) // 2] - ref).max())
    assert worst <= 1e-12


def _oracle_boosters(tj, dl, gamma, rule):
    return ob.vertex_boosters(tj, dl, gamma, *rule)


@pytest.mark.parametrize("tj,dl,gamma", [((2,) * 10, 1, 1.2), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 1, 0.1)])
def test_boosters(lib, tj, dl, gamma):
    t = _tables(tj, dl, gamma)
    sf.sf_boosters(t, SMALL_RULE)
    ref = _oracle_boosters(tj, dl, gamma, SMALL_RULE)
    for e in (2, 3, 4, 5):
        got = sf.sf_boosters_download(t, 0, e).cpu().numpy()
        assert got.shape == ref[e]["B"].shape
        err = np.abs(got - ref[e]["B"]).max()
        assert err <= 1e-11 * np.abs(ref[e]["B"]).max(), (e, err)


def _random_boosters(tj, dl, seed):
    rng = np.random.default_rng(seed)
    t = _tables(tj, dl)
    out = {}
    for e in (2, 3, 4, 5):
        shape = sf.booster_shape(t, 0, e)
        B = rng.standard_normal(shape)
        klo = np.zeros(shape[0], dtype=np.int64)
        D = dl + 1
        for tt in range(shape[0]):
            d = (tt // (D * D), (tt // D) % D, tt % D)
            tl6 = dict(zip(ov.FREE, [tj[F.index(f)] for f in ov.FREE]))
            for f, df in zip(ov.EDGE_TRIPLES[e], d):
                tl6[f] += 2 * df
            bj, bl = ov.edge_spins(tj, tuple(tl6[f] for f in ov.FREE))[e]
            kr = ow.pair_range(*bl)
            klo[tt] = kr[0] if kr else 0
            B[tt, :, len(kr):] = 0.0
        out[e] = {"B": B, "klo": klo}
    return t, out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("tj,dl", [((2,) * 10, 2), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2), ((6,) * 10, 1),
                                   ((1, 2, 1, 4, 5, 5, 5, 2, 1, 2), 1)])
def test_amplitude_random_boosters(lib, tj, dl):
    """Contraction engine with non-symmetric random boosters: every index mapping is exercised."""
    assert inputs.boundary_is_valid(tj)
    t, bs = _random_boosters(tj, dl, seed=dl + sum(tj))
    for e in (2, 3, 4, 5):
        sf.sf_boosters_upload(t, 0, e, bs[e]["B"])
    A = sf.sf_vertex_amplitude(t)[0].cpu().numpy()
    ref = ov.vertex_amplitude(tj, dl, bs)
    assert _rel(A, ref) <= 1e-12


def test_bf_limit(lib):
    tj = (4, 3, 3, 4, 4, 5, 1, 3, 2, 5)
    t = _tables(tj, 0)
    bs = ob.identity_boosters(tj)
    for e in (2, 3, 4, 5):
        sf.sf_boosters_upload(t, 0, e, bs[e]["B"])
    A = sf.sf_vertex_amplitude(t)[0].cpu().numpy()
    I = ov.intertwiner_ranges(tj)
    ref = np.zeros([len(r) for r in I])
    import itertools
    for idx in itertools.product(*[range(len(r)) for r in I]):
        ti = [I[e][idx[e]] for e in range(5)]
        ref[idx] = float(ow.fifteenj_mp(tj, tj[4:], ti[0], ti[1:])) * np.prod([np.sqrt(x + 1.0) for x in ti])
    np.testing.assert_allclose(A, ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())


@pytest.mark.parametrize("tj,dl,gamma", [((2,) * 10, 2, 1.2), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 1, 5.0)])
def test_amplitude_end_to_end(lib, tj, dl, gamma):
    t = _tables(tj, dl, gamma)
    sf.sf_boosters(t, SMALL_RULE)
    A = sf.sf_vertex_amplitude(t)[0].cpu().numpy()
    ref = ov.vertex_amplitude(tj, dl, _oracle_boosters(tj, dl, gamma, SMALL_RULE))
    assert _rel(A, ref) <= 1e-10


def test_shell_ranges_and_lists(lib):
    tj, dl = (2,) * 10, 2
    t, bs = _random_boosters(tj, dl, seed=4)
    for e in (2, 3, 4, 5):
        sf.sf_boosters_upload(t, 0, e, bs[e]["B"])
    N = ov.n_shells(dl)
    full = sf.sf_vertex_amplitude(t)[0]
    a = sf.sf_vertex_amplitude(t, shell_begin=0, shell_end=311)[0]
    b = sf.sf_vertex_amplitude(t, shell_begin=311, shell_end=N)[0]
    assert float((a + b - full).norm() / full.norm()) <= 1e-13
    sub = inputs.shell_subset(N, 57, seed=3)
    got = sf.sf_vertex_amplitude(t, shell_list=sub)[0].cpu().numpy()
    ref = ov.vertex_amplitude(tj, dl, bs, shells=sub)
    assert _rel(got, ref) <= 1e-12
    # deterministic: bitwise identical on repeat
    again = sf.sf_vertex_amplitude(t)[0]
    assert torch.equal(again, full)
