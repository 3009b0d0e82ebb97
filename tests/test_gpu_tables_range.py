"""Tables built for part of the shell range (``sf_6j_table_range``): the shell sum over any range
inside it is bitwise the sum on whole tables (same slots, same boosters where read), in every
precision and through plans; the boosters of the groups outside are zero; calls that reach
outside are refused, and so is the adjoint."""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu

RULE = (40.0, 4, 10)


@pytest.mark.parametrize("lam,dl,frac", [(8, 4, (3, 7)), (16, 10, (5, 6)), (5, 6, (0, 1))])
def test_restricted_tables_give_the_same_bits(lib, lam, dl, frac):
    D = dl + 1
    verts = [sf.vertex((lam,) * 10, 1.2, dl), sf.vertex((lam - 1,) * 10, 1.2, dl)]
    G = D ** 3
    g0, g1 = G * frac[0] // 8, G * frac[1] // 8
    b, e = g0 * D ** 3, g1 * D ** 3
    full = sf.sf_6j_table(verts)
    sf.sf_boosters(full, RULE)
    part = sf.sf_6j_table(verts, shell_range=(b, e))
    sf.sf_boosters(part, RULE)
    for prec in (sf.SF_FP64, sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX):
        a = sf.sf_vertex_amplitude(full, prec, b, e)
        c = sf.sf_vertex_amplitude(part, prec, b, e)
        for x, y in zip(a, c):
            assert torch.equal(x, y), prec
    # a sub-range of the restriction and a plan over it
    bm = b + (e - b) // 3 // D ** 3 * D ** 3
    a = sf.sf_vertex_amplitude(full, sf.SF_MIXED_TC, bm, e)
    plan = sf.Plan(part, sf.SF_MIXED_TC, bm, e)
    plan.run()
    plan.sync()
    for x, y in zip(a, plan.outputs):
        assert torch.equal(x, y)


def test_unneeded_boosters_are_zero(lib):
    lam, dl = 6, 3
    D = dl + 1
    g0, g1 = 20, 23                  # groups (d25, d35, d45) = (1, 1, 0) .. (1, 1, 2)
    part = sf.sf_6j_table([sf.vertex((lam,) * 10, 1.2, dl)], shell_range=(g0 * D ** 3, g1 * D ** 3))
    full = sf.sf_6j_table([sf.vertex((lam,) * 10, 1.2, dl)])
    sf.sf_boosters(part, RULE)
    sf.sf_boosters(full, RULE)
    groups = [(g // (D * D), (g // D) % D, g % D) for g in range(g0, g1)]
    n25 = {g[0] for g in groups}
    n35 = {g[1] for g in groups}
    n45 = {g[2] for g in groups}
    sel = {2: lambda a, b, c: c in n25, 3: lambda a, b, c: b in n35, 4: lambda a, b, c: a in n45,
           5: lambda a, b, c: (a, b, c) in groups}
    # the offsets of the edge's pair of free strands within a triple (equal spins here, so the
    # library computes the triple with the smaller offset first and fills the other by exchange)
    pair = {2: (0, 1), 3: (0, 1), 4: (1, 2), 5: (1, 2)}
    for e in (2, 3, 4, 5):
        Bp = sf.sf_boosters_download(part, 0, e).cpu().numpy()
        Bf = sf.sf_boosters_download(full, 0, e).cpu().numpy()
        sa, sb = pair[e]
        for t in range(D ** 3):
            abc = [t // (D * D), (t // D) % D, t % D]
            sw = list(abc)
            sw[sa], sw[sb] = sw[sb], sw[sa]
            if sel[e](*abc):
                assert np.array_equal(Bp[t], Bf[t]), (e, t)
            elif abc[sa] < abc[sb] and sel[e](*sw):   # the exchange source of a selected triple
                assert np.array_equal(Bp[t], Bf[t]), (e, t)
            else:
                assert not Bp[t].any(), (e, t)


def test_calls_outside_are_refused(lib):
    lam, dl = 4, 3
    D = dl + 1
    b, e = 10 * D ** 3, 30 * D ** 3
    t = sf.sf_6j_table([sf.vertex((lam,) * 10, 1.2, dl)], shell_range=(b, e))
    sf.sf_boosters(t, RULE)
    for (bb, ee) in ((0, e), (b, e + D ** 3), (0, 2 ** 62)):
        with pytest.raises(sf.SfError) as err:
            sf.sf_vertex_amplitude(t, sf.SF_FP64, bb, ee)
        assert err.value.code == sf.SF_ERR_ARG
    with pytest.raises(sf.SfError):
        sf.sf_vertex_amplitude(t, shell_list=np.array([0, b], dtype=np.int64))
    with pytest.raises(sf.SfError):
        sf.Plan(t, sf.SF_FP64, 0, e)
    _, dims = sf.intertwiner_ranges((lam,) * 10, 1.2, dl)
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims)]
    with pytest.raises(sf.SfError):
        sf.sf_vertex_adjoint(t, psis)
    sf.sf_vertex_amplitude(t, sf.SF_FP64, b, e)      # inside: fine
