"""Boundary-contracted amplitude and its adjoint through the C ABI (sf_vertex_adjoint).

* against the oracle's per-shell direct summation (value, d a/d psi_e, d a/d B_e), 1e-12;
* at the full boundary-contraction workload (all spins 3, gamma 1.2, dl 8, 531,441 shells):
  the value against the contraction of the FP64 vertex tensor, gradients against central finite
  differences (h = 1e-6, FP64);
* torch.autograd.gradcheck through the autograd Function on a small vertex.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import contract as oc
from oracle import vertex as ov
from oracle import wigner as ow
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu


def _setup(tj, dl, seed):
    t = sf.sf_6j_table([sf.vertex(tj, 1.2, dl)])
    rng = np.random.default_rng(seed)
    bs = {}
    D = dl + 1
    for e in (2, 3, 4, 5):
        shape = sf.booster_shape(t, 0, e)
        B = rng.standard_normal(shape)
        klo = np.zeros(shape[0], dtype=np.int64)
        for tt in range(shape[0]):
            d = (tt // (D * D), (tt // D) % D, tt % D)
            tl6 = dict(zip(ov.FREE, [tj[ov.FACES.index(f)] for f in ov.FREE]))
            for f, df in zip(ov.EDGE_TRIPLES[e], d):
                tl6[f] += 2 * df
            kr = ow.pair_range(*ov.edge_spins(tj, tuple(tl6[f] for f in ov.FREE))[e][1])
            klo[tt] = kr[0] if kr else 0
            B[tt, :, len(kr):] = 0.0
        bs[e] = {"B": B, "klo": klo}
        sf.sf_boosters_upload(t, 0, e, B)
    _, dim = sf.intertwiner_ranges(tj, 1.2, dl)
    psis = inputs.boundary_vectors(dim, seed=seed)
    return t, bs, psis


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.mark.parametrize("tj,dl", [((2,) * 10, 1), ((6,) * 10, 1), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2)])
def test_adjoint_matches_oracle(lib, tj, dl):
    t, bs, psis = _setup(tj, dl, seed=11)
    a, gpsi, gB = sf.sf_vertex_adjoint(t, [torch.tensor(p) for p in psis])
    ra, rpsi, rB = oc.contract_by_shell(tj, dl, bs, psis)
    assert abs(complex(a) - ra) <= 1e-12 * abs(ra)
    for e in range(5):
        assert _rel(gpsi[e].cpu().numpy(), rpsi[e]) <= 1e-12
    for k, e in enumerate((2, 3, 4, 5)):
        assert _rel(gB[k].cpu().numpy(), rB[e]) <= 1e-12


def test_adjoint_full_workload_value_and_finite_differences(lib):
    spec = inputs.boundary_contraction_vertex()
    tj, dl = spec["two_j"], spec["dl"]
    t, bs, psis = _setup(tj, dl, seed=13952)
    tp = [torch.tensor(p, device="cuda") for p in psis]
    a, gpsi, gB = sf.sf_vertex_adjoint(t, tp)
    A = sf.sf_vertex_amplitude(t)[0].to(torch.complex128)
    ref = torch.einsum("abcde,a,b,c,d,e->", A, *tp)
    assert abs(complex(a) - complex(ref)) <= 1e-11 * abs(complex(ref))
    h = 1e-6
    rng = np.random.default_rng(1)
    # psi: a is holomorphic, so a(psi + h) - a(psi - h) over 2h gives d a / d psi exactly up to rounding
    for e in (0, 2, 4):
        i = int(rng.integers(0, len(psis[e])))
        for step in (h, 1j * h):
            p_plus = [p.clone() for p in tp]
            p_minus = [p.clone() for p in tp]
            p_plus[e][i] += step
            p_minus[e][i] -= step
            ap = complex(sf.sf_vertex_adjoint(t, p_plus, want_grads=False)[0])
            am = complex(sf.sf_vertex_adjoint(t, p_minus, want_grads=False)[0])
            fd = (ap - am) / (2 * step)
            assert abs(fd - complex(gpsi[e][i])) <= 1e-6 * (abs(complex(gpsi[e][i])) + abs(complex(a)))
    # one booster entry per edge
    for k, e in enumerate((2, 3, 4, 5)):
        B = bs[e]["B"]
        nz = np.argwhere(np.abs(B) > 0)
        tt, i, c = (int(v) for v in nz[int(rng.integers(0, len(nz)))])
        vals = []
        for sgn in (1, -1):
            B2 = B.copy()
            B2[tt, i, c] += sgn * h
            sf.sf_boosters_upload(t, 0, e, B2)
            vals.append(complex(sf.sf_vertex_adjoint(t, tp, want_grads=False)[0]))
        sf.sf_boosters_upload(t, 0, e, B)
        fd = (vals[0] - vals[1]) / (2 * h)
        g = complex(gB[k][tt, i, c])
        assert abs(fd - g) <= 1e-6 * (abs(g) + abs(complex(a)))


def test_gradcheck_through_autograd_function(lib):
    tj, dl = (1,) * 10, 1
    t, bs, psis = _setup(tj, dl, seed=3)
    tp = [torch.tensor(p, device="cuda", requires_grad=True) for p in psis]
    tB = [torch.tensor(bs[e]["B"], device="cuda") for e in (2, 3, 4, 5)]

    def f_psi(*ps):
        return sf.eprl_contraction(t, list(ps), tB)
    assert torch.autograd.gradcheck(f_psi, tuple(tp), eps=1e-6, atol=1e-9, rtol=1e-6)

    tB2 = [b.clone().requires_grad_(True) for b in tB]
    fixed = [p.detach() for p in tp]

    def f_B(b2, b3, b4, b5):
        return sf.eprl_contraction(t, fixed, [b2, b3, b4, b5])
    assert torch.autograd.gradcheck(f_B, tuple(tB2), eps=1e-6, atol=1e-9, rtol=1e-6)
