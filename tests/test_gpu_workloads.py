"""Parity on the benchmarked workloads at their full sizes, in the launch configuration of the
benchmark, on outputs the oracle can compute; plus the small workload whole.

* all spins 8, dl 10 (largest vertex of the homogeneous sweep) and all spins 4, dl 20 (85,766,121
  shells): partial sums over seeded 10^4-shell subsets of the non-empty shells, through the
  shell-list entry point, against the oracle's sums stored by ``tests/golden/make_subsets.py``;
  FP64 path within 1e-10 and mixed path within its stated 1e-6 (normwise relative);
* d-table entries of the spin-8 vertex on the full 2000-node rule against the closed form;
* all spins 1, dl 0..3: boosters on the full 2000-node rule and the whole tensor, end to end;
* 256 irregular vertices in one batched launch: small vertices against the oracle, sampled ones
  against single-vertex launches, both precisions.

Where the oracle's arbitrary-precision d-tables on the 2000-node rule would take hours (large
spins), seeded random boosters are injected; the quadrature itself is checked on the full rule
for spin 1 here and on shorter rules for larger spins in test_gpu_parity.py.
"""
import os

import mpmath
import numpy as np
import pytest

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import dfunc
from oracle import quadrature as oq
from oracle import vertex as ov
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FULL_RULE = inputs.RULE_DEFAULT
FP64_BOUND = 1e-10
MIXED_BOUND = 1e-6


def _upload(t, vtx, bs):
    for e in (2, 3, 4, 5):
        assert tuple(sf.booster_shape(t, vtx, e)) == bs[e]["B"].shape
        sf.sf_boosters_upload(t, vtx, e, bs[e]["B"])


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("name", ["sweep_j8_dl10_subset", "large_shell_j4_dl20_subset"])
def test_full_size_shell_subsets(lib, name):
    g = np.load(os.path.join(GOLDEN, name + ".npz"))
    tj, dl, gamma = tuple(int(v) for v in g["two_j"]), int(g["dl"]), float(g["gamma"])
    t = sf.sf_6j_table([sf.vertex(tj, gamma, dl)])
    bs = ob.random_boosters(tj, dl, int(g["booster_seed"]))
    _upload(t, 0, bs)
    shells = g["shells"]
    outs, kap = sf.sf_vertex_amplitude(t, shell_list=shells, kappa=True)
    a64 = outs[0].cpu().numpy()
    # sum over the subset of the shells' contribution norms (the numerator of kappa)
    assert abs(kap[0] - float(g["kappa"])) <= 1e-10 * float(g["kappa"]), (kap[0], float(g["kappa"]))
    amx = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED, shell_list=shells)[0].cpu().numpy()
    aff = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_FF, shell_list=shells)[0].cpu().numpy()
    atc = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_TC, shell_list=shells)[0].cpu().numpy()
    atf = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_PX, shell_list=shells)[0].cpu().numpy()
    ref = g["A"]
    for a, bound in ((a64, FP64_BOUND), (amx, MIXED_BOUND), (aff, MIXED_BOUND), (atc, MIXED_BOUND),
                     (atf, MIXED_BOUND)):
        if "idx" in g:      # large tensor: a seeded sample of entries plus the norm of the whole
            assert abs(np.linalg.norm(a) - float(g["A_norm"])) <= bound * float(g["A_norm"])
            got = a.reshape(-1)[g["idx"]]
        else:
            got = a
        assert _rel(got, ref) <= bound
        # elementwise form of the same comparison: relative error on every (sampled) entry, with
        # an absolute floor at the scale of the largest entry, because rounding errors follow the
        # size of the shell contributions, not of the entry they cancel into: 1e-13 of the largest
        # entry for FP64 (a few units of 1e-16 times the sum of the 10^4 contributions' sizes) and
        # the stated bound of the largest entry for the mixed paths (FP32 rounding of the same)
        amax = np.abs(ref).max()
        floor = 1e-3 * bound * amax if bound == FP64_BOUND else bound * amax
        big = np.abs(ref) >= 1e-8 * amax
        dev = np.abs(got - ref)
        assert np.all(dev <= bound * np.abs(ref) + floor), (bound, float(dev.max() / amax))
        rel_el = float((dev[big] / np.abs(ref[big])).max())
        print("%s bound %g: normwise %.2e, elementwise max rel (entries >= 1e-8 max) %.2e"
              % (name, bound, _rel(got, ref), rel_el))
        if bound == FP64_BOUND:
            assert rel_el <= 1e-6


def test_dtable_entries_full_rule(lib):
    tj, dl, gamma = (16,) * 10, 10, 1.2
    t = sf.sf_6j_table([sf.vertex(tj, gamma, dl)])
    sf.sf_boosters(t, FULL_RULE)
    x = sf.table_copy(t, 0, sf.SF_TAB_NODES, 0).numpy()
    nn = len(x)
    assert nn == FULL_RULE[1] * FULL_RULE[2]
    rho = gamma * (8 + 1)
    rng = np.random.default_rng(5)
    for f in (4, 8, 9):
        tab = sf.table_copy(t, 0, sf.SF_TAB_D, f).numpy().reshape(dl + 1, 17, nn)
        scale = np.abs(tab).max()
        for _ in range(12):
            p, im, n = int(rng.integers(0, dl + 1)), int(rng.integers(0, 17)), int(rng.integers(0, nn))
            ref = complex(dfunc.DClosed(16, rho, 16 + 2 * p, -16 + 2 * im).eval(-mpmath.log(mpmath.mpf(x[n])), 20))
            assert abs(tab[p, im, n] - ref) <= 1e-12 * scale, (f, p, im, n)


BOOSTER_CASES = ["j8_dl10_short", "j8_dl10_full", "j6_dl12_g5_short", "j6_dl12_g5_full", "zero_edge_full"]


@pytest.mark.parametrize("name", BOOSTER_CASES)
def test_boosters_sampled_against_oracle(lib, name):
    """k_booster on sampled triples of the benchmarked vertices (spin 8, dl 10; the 256-vertex
    batch's extreme faces spin 6, gamma 5, dl 12) and on every triple of a vertex whose edge 5
    couples four spin-0 faces, against ``tests/golden/make_boosters.py``: the node sums of these
    cases run in chunks of 16 (spin 8) up to 1024 nodes (spin 0, one full and one partial chunk of
    the 2000-node rule); bound 1e-11 of the largest entry per edge."""
    g = np.load(os.path.join(GOLDEN, "boosters_" + name + ".npz"))
    tj, dl, gamma = tuple(int(v) for v in g["two_j"]), int(g["dl"]), float(g["gamma"])
    rule = (float(g["rule"][0]), int(g["rule"][1]), int(g["rule"][2]))
    t = sf.sf_6j_table([sf.vertex(tj, gamma, dl)])
    sf.sf_boosters(t, rule)
    got = {e: sf.sf_boosters_download(t, 0, e).cpu().numpy() for e in (2, 3, 4, 5)}
    for e in (2, 3, 4, 5):
        sel = np.nonzero(g["edge"] == e)[0]
        assert len(sel) > 0
        scale = max(np.abs(g["B"][q]).max() for q in sel)
        for q in sel:
            tt, nk = int(g["t"][q]), int(g["nk"][q])
            di = got[e].shape[1]
            ref = g["B"][q][:di, :nk]
            assert np.abs(got[e][tt, :, :nk] - ref).max() <= 1e-11 * scale, (e, tt)
            assert np.all(got[e][tt, :, nk:] == 0.0)


def test_dtables_composite_rule(lib):
    """rho = 70 (spin 6, gamma 10): on the 2000-node rule the nodes of largest r ask for more
    Gauss-Legendre points than the largest library rule, so the d-table kernel integrates them
    with a composite rule; entries against the closed form, 1e-12 of the face maximum everywhere
    (the nodes of largest r, one in the middle and the smallest r, where l > k entries vanish
    like r^(l-k)), and relative 1e-10 at the composite-rule nodes where |m| = k (no cancellation
    in the integral there: the entry decays only as e^-r)."""
    tj, dl, gamma = (12,) * 10, 2, 10.0
    t = sf.sf_6j_table([sf.vertex(tj, gamma, dl)])
    sf.sf_boosters(t, FULL_RULE)
    x = sf.table_copy(t, 0, sf.SF_TAB_NODES, 0).numpy()
    r = sf.table_copy(t, 0, sf.SF_TAB_NODES, 2).numpy()
    nn = len(x)
    rho = gamma * (6 + 1)
    band = rho + 0.25 * (12 + 12 + 2 * dl) + 1.0
    far = np.argsort(-r)[:6]
    assert 48 + r[far[0]] * band > 1024          # these nodes take the composite rule
    for f in (4, 9):
        tab = sf.table_copy(t, 0, sf.SF_TAB_D, f).numpy().reshape(dl + 1, 13, nn)
        scale = np.abs(tab).max()
        for p in (0, dl):
            for im in (0, 6, 12):
                for n in list(far) + [int(np.argsort(-r)[200]), int(np.argmin(r))]:
                    ref = complex(dfunc.DClosed(12, rho, 12 + 2 * p, -12 + 2 * im).eval(
                        -mpmath.log(mpmath.mpf(x[n])), 25))
                    err = abs(tab[p, im, n] - ref)
                    assert err <= 1e-12 * scale, (f, p, im, n, err)
                    if im in (0, 12) and n in far:
                        assert err <= 1e-10 * abs(ref), (f, p, im, n, err, abs(ref))


@pytest.fixture(scope="module")
def spin1_full_rule():
    xs, ws = oq.rule_nodes(*FULL_RULE)
    return xs, ws, ob.face_tables((2,) * 10, 3, 1.2, xs)


def test_simplex_j1_full_rule_end_to_end(lib, spin1_full_rule):
    # all spins 1: the oracle's boosters on the 2000-node rule for dl = 3 contain those of dl < 3
    xs, ws, tabs = spin1_full_rule
    tj, gamma = (2,) * 10, 1.2
    ref_b = ob.vertex_boosters(tj, 3, gamma, *FULL_RULE, tables=tabs)
    t3 = sf.sf_6j_table([sf.vertex(tj, gamma, 3)])
    sf.sf_boosters(t3, FULL_RULE)
    for e in (2, 3, 4, 5):
        got = sf.sf_boosters_download(t3, 0, e).cpu().numpy()
        ref = ref_b[e]["B"]
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), e
    for dl in range(4):
        spec = inputs.simplex_j1(dl)
        t = sf.sf_6j_table([sf.vertex(spec["two_j"], spec["gamma"], dl)])
        sf.sf_boosters(t, FULL_RULE)
        A = sf.sf_vertex_amplitude(t)[0].cpu().numpy()
        ref = ov.vertex_amplitude(tj, dl, ob.vertex_boosters(tj, dl, gamma, *FULL_RULE, tables=tabs))
        assert _rel(A, ref) <= FP64_BOUND, dl


BATCH_SHELL_END = 729     # per vertex: the first 729 group-major shells (all of them for dl <= 2)


@pytest.fixture(scope="module")
def batch256(lib):
    batch = inputs.random_batch(256, seed=0)
    verts = [sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in batch]
    t = sf.sf_6j_table(verts)
    bss = [ob.random_boosters(b["two_j"], b["dl"], 1000 + i) for i, b in enumerate(batch)]
    for i in range(len(batch)):
        _upload(t, i, bss[i])
    return batch, verts, t, bss


def test_random_batch_256_against_oracle(lib, batch256):
    batch, verts, t, bss = batch256
    out64 = sf.sf_vertex_amplitude(t, shell_end=BATCH_SHELL_END)
    outmx = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED, shell_end=BATCH_SHELL_END)
    outff = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_FF, shell_end=BATCH_SHELL_END)
    outtc = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_TC, shell_end=BATCH_SHELL_END)
    outtf = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_PX, shell_end=BATCH_SHELL_END)
    small = [i for i, b in enumerate(batch) if b["dl"] <= 2]
    assert small
    rng = np.random.default_rng(7)
    for i in rng.choice(small, size=min(8, len(small)), replace=False):
        b = batch[int(i)]
        ref = ov.vertex_amplitude(b["two_j"], b["dl"], bss[int(i)])
        assert _rel(out64[int(i)].cpu().numpy(), ref) <= FP64_BOUND
        assert _rel(outmx[int(i)].cpu().numpy(), ref) <= MIXED_BOUND
        assert _rel(outff[int(i)].cpu().numpy(), ref) <= MIXED_BOUND
        assert _rel(outtc[int(i)].cpu().numpy(), ref) <= MIXED_BOUND
        assert _rel(outtf[int(i)].cpu().numpy(), ref) <= MIXED_BOUND


def test_random_batch_256_against_single_launches(lib, batch256):
    batch, verts, t, bss = batch256
    out64 = sf.sf_vertex_amplitude(t, shell_end=BATCH_SHELL_END)
    outmx = sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED, shell_end=BATCH_SHELL_END)
    rng = np.random.default_rng(8)
    for i in (int(v) for v in rng.choice(len(batch), size=8, replace=False)):
        t1 = sf.sf_6j_table([verts[i]])
        _upload(t1, 0, bss[i])
        s64 = sf.sf_vertex_amplitude(t1, shell_end=BATCH_SHELL_END)[0]
        smx = sf.sf_vertex_amplitude(t1, precision=sf.SF_MIXED, shell_end=BATCH_SHELL_END)[0]
        n = float(s64.norm())
        if n == 0.0:
            assert float(out64[i].abs().max()) == 0.0
            continue
        assert float((out64[i] - s64).norm()) <= 1e-13 * n
        assert float((outmx[i] - smx).norm()) <= 1e-6 * n


def test_random_batch_boosters_match_single(lib):
    # batched quadrature (16 irregular vertices, short rule) equals per-vertex launches
    batch = inputs.random_batch(16, seed=3)
    verts = [sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in batch]
    t = sf.sf_6j_table(verts)
    rule = (40.0, 4, 10)
    sf.sf_boosters(t, rule)
    for i in (0, 5, 11):
        t1 = sf.sf_6j_table([verts[i]])
        sf.sf_boosters(t1, rule)
        for e in (2, 3, 4, 5):
            a = sf.sf_boosters_download(t, i, e)
            b = sf.sf_boosters_download(t1, 0, e)
            assert float((a - b).abs().max()) <= 1e-14 * max(float(b.abs().max()), 1e-300)


SWEEP_SMALL_RULE = (40.0, 40, 50)


@pytest.mark.parametrize("lam", [1, 2])
def test_sweep_small_vertices_full_size(lib, lam):
    """The two smallest vertices of the homogeneous sweep (all spins 1/2 and all spins 1, gamma 1.2,
    dl 10: 11^6 shells each) in full: boosters by quadrature on the 2000-node rule and the whole
    shell sum, every precision, against the oracle's tensors and cancellation sums written by
    ``tests/golden/make_sweep_small.py``."""
    g = np.load(os.path.join(GOLDEN, "sweep_small_dl10.npz"))
    ref, kref = g["A_%d" % lam], float(g["kappa_%d" % lam])
    t = sf.sf_6j_table([sf.vertex((lam,) * 10, 1.2, 10)])
    sf.sf_boosters(t, SWEEP_SMALL_RULE)
    outs, kap = sf.sf_vertex_amplitude(t, kappa=True)
    assert abs(kap[0] - kref) <= 1e-10 * kref, (kap[0], kref)
    amax = float(np.abs(ref).max())
    for prec, bound in ((sf.SF_FP64, FP64_BOUND), (sf.SF_MIXED, MIXED_BOUND), (sf.SF_MIXED_FF, MIXED_BOUND),
                        (sf.SF_MIXED_TC, MIXED_BOUND), (sf.SF_MIXED_PX, MIXED_BOUND)):
        a = outs[0] if prec == sf.SF_FP64 else sf.sf_vertex_amplitude(t, precision=prec)[0]
        a = a.cpu().numpy()
        assert a.shape == ref.shape
        assert _rel(a, ref) <= bound, (prec, _rel(a, ref))
        assert np.all(np.abs(a - ref) <= bound * np.abs(ref) + bound * amax), prec


@pytest.mark.parametrize("prec", [sf.SF_FP64, sf.SF_MIXED_TC])
def test_mixed_size_batch_matches_single_vertex_calls(lib, prec):
    """A batch whose largest vertex (all spins 8) needs one CTA per SM and whose smaller vertices
    fit two: the library runs the two classes as separate launches; every vertex's tensor equals
    its single-vertex call up to the summation order of the x chunks."""
    specs = [((16,) * 10, 1.2, 2), ((4,) * 10, 1.2, 3), ((5, 3, 4, 4, 6, 3, 4, 3, 4, 4), 5.0, 2), ((2,) * 10, 0.1, 4)]
    verts = [sf.vertex(*s) for s in specs]
    t = sf.sf_6j_table(verts)
    sf.sf_boosters(t, (40.0, 4, 10))
    outs = sf.sf_vertex_amplitude(t, precision=prec)
    for i, s in enumerate(specs):
        ti = sf.sf_6j_table([sf.vertex(*s)])
        sf.sf_boosters(ti, (40.0, 4, 10))
        ref = sf.sf_vertex_amplitude(ti, precision=prec)[0]
        assert _rel(outs[i].cpu().numpy(), ref.cpu().numpy()) <= 1e-12, (i, prec)
