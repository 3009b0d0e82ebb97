"""Boundary items of the C ABI through ctypes: a reduced set of boundary intertwiners (the paper's
restricted intertwiner range, Sec. 3 after the framed algorithm and Sec. 4), the adjoint's
precision argument and its amplitude-only mode.

* sub-range: the tensor computed for a block of the intertwiner ranges equals that block of the
  whole tensor, to 1e-13 for the FP64 path (the work is split differently, so the summation order
  differs) and within 1e-6 for the mixed paths (every precision, plain calls, plans and the
  allocation-free call);
* the adjoint accepts SF_FP64 only and refuses tables with a sub-range;
* the amplitude-only adjoint (no gradient outputs) equals the amplitude of the full adjoint;
* kappa_out: the sum over shells of the contributions' norms equals the oracle's, on whole
  vertices, sub-ranges (where it is the norms of the block) and shell ranges.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import vertex as ov
from paper_2107_13952_gb300 import inputs

pytestmark = pytest.mark.gpu


def _upload(t, vtx, bs):
    for e in (2, 3, 4, 5):
        sf.sf_boosters_upload(t, vtx, e, bs[e]["B"])


CASES = [((6,) * 10, 2, [(1, 3), (0, 2), (2, 0), (1, 4), (0, 1)]),
         ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2, [(0, 1), (1, 0), (0, 0), (1, 1), (0, 0)]),
         ((12,) * 10, 1, [(3, 5), (6, 7), (0, 13), (12, 1), (4, 6)])]


@pytest.mark.parametrize("tj,dl,sub", CASES)
@pytest.mark.parametrize("prec", [sf.SF_FP64, sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX])
def test_sub_range_is_block_of_whole_tensor(lib, tj, dl, sub, prec):
    bs = ob.random_boosters(tj, dl, 77)
    tw = sf.sf_6j_table([sf.vertex(tj, 1.2, dl)])
    ts = sf.sf_6j_table([sf.vertex(tj, 1.2, dl, sub=sub)])
    _upload(tw, 0, bs)
    _upload(ts, 0, bs)
    whole = sf.sf_vertex_amplitude(tw, precision=prec)[0]
    part = sf.sf_vertex_amplitude(ts, precision=prec)[0]
    lo, dim = sf.output_ranges(sf.vertex(tj, 1.2, dl, sub=sub))
    _, full = sf.intertwiner_ranges(tj, 1.2, dl)
    assert list(part.shape) == dim
    sl = tuple(slice(f, f + (c if c else full[e] - f)) for e, (f, c) in enumerate(sub))
    ref = whole[sl]
    n = float(ref.norm())
    bound = 1e-13 if prec == sf.SF_FP64 else 1e-6
    assert float((part - ref).norm()) <= bound * max(n, 1e-300)
    # plan and (FP64) allocation-free call over the same sub-range
    plan = sf.Plan(ts, prec)
    plan.run()
    plan.sync()
    assert float((plan.outputs[0] - ref).norm()) <= bound * max(n, 1e-300)
    if prec == sf.SF_FP64:
        out = [torch.empty(dim, dtype=torch.float64, device="cuda")]
        sf.sf_vertex_amplitude_noalloc(ts, out)
        assert float((out[0] - ref).norm()) <= 1e-13 * max(n, 1e-300)


def test_sub_range_in_a_batch(lib):
    batch = inputs.random_batch(6, seed=11)
    subs = []
    for b in batch:
        _, d = sf.intertwiner_ranges(b["two_j"], b["gamma"], b["dl"])
        subs.append([(di // 2, (di + 1) // 2) if di > 1 else (0, 0) for di in d])
    bss = [ob.random_boosters(b["two_j"], b["dl"], 500 + i) for i, b in enumerate(batch)]
    tw = sf.sf_6j_table([sf.vertex(b["two_j"], b["gamma"], b["dl"]) for b in batch])
    ts = sf.sf_6j_table([sf.vertex(b["two_j"], b["gamma"], b["dl"], sub=s) for b, s in zip(batch, subs)])
    for i in range(len(batch)):
        _upload(tw, i, bss[i])
        _upload(ts, i, bss[i])
    whole = sf.sf_vertex_amplitude(tw, shell_end=4096)
    part = sf.sf_vertex_amplitude(ts, shell_end=4096)
    for w, p, s in zip(whole, part, subs):
        sl = tuple(slice(f, f + c) if c else slice(0, None) for f, c in s)
        ref = w[sl]
        assert float((p - ref).norm()) <= 1e-13 * max(float(ref.norm()), 1e-300)


def test_bad_sub_range_is_refused(lib):
    for sub in ([(0, 9), (0, 0), (0, 0), (0, 0), (0, 0)], [(-1, 0)] + [(0, 0)] * 4, [(7, 0)] + [(0, 0)] * 4):
        with pytest.raises(sf.SfError) as e:
            sf.sf_6j_table([sf.vertex((6,) * 10, 1.2, 1, sub=sub)])
        assert e.value.code == sf.SF_ERR_ARG


def _adjoint_tables(tj, dl, sub=None):
    t = sf.sf_6j_table([sf.vertex(tj, 1.2, dl, sub=sub)])
    _upload(t, 0, ob.random_boosters(tj, dl, 31))
    return t


def test_adjoint_precision_and_sub_range_checks(lib):
    tj, dl = (4,) * 10, 1
    t = _adjoint_tables(tj, dl)
    _, dims = sf.intertwiner_ranges(tj, 1.2, dl)
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims)]
    for p in (sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX, 7):
        with pytest.raises(sf.SfError) as e:
            sf.sf_vertex_adjoint(t, psis, precision=p)
        assert e.value.code == sf.SF_ERR_ARG
    ts = _adjoint_tables(tj, dl, sub=[(1, 2), (0, 0), (0, 0), (0, 0), (0, 0)])
    with pytest.raises(sf.SfError) as e:
        sf.sf_vertex_adjoint(ts, psis)
    assert e.value.code == sf.SF_ERR_ARG


@pytest.mark.parametrize("tj,dl", [((4,) * 10, 2), ((6,) * 10, 3), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2)])
def test_amplitude_only_adjoint_matches_full(lib, tj, dl):
    t = _adjoint_tables(tj, dl)
    _, dims = sf.intertwiner_ranges(tj, 1.2, dl)
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims, seed=3)]
    a_full, g, gb = sf.sf_vertex_adjoint(t, psis, want_grads=True)
    a_only, g0, gb0 = sf.sf_vertex_adjoint(t, psis, want_grads=False)
    assert g0 == [] and gb0 == []
    a_full, a_only = complex(a_full), complex(a_only)
    assert abs(a_full - a_only) <= 1e-13 * abs(a_full)
    # and both equal the contraction of the FP64 tensor
    A = sf.sf_vertex_amplitude(t)[0].to(torch.complex128)
    ref = torch.einsum("abcde,a,b,c,d,e->", A, *psis)
    assert abs(a_only - complex(ref)) <= 1e-12 * abs(complex(ref))


def test_autograd_forward_without_grads_skips_them(lib):
    tj, dl = (4,) * 10, 1
    t = _adjoint_tables(tj, dl)
    _, dims = sf.intertwiner_ranges(tj, 1.2, dl)
    psis = [torch.tensor(v, dtype=torch.complex128, device="cuda") for v in inputs.boundary_vectors(dims)]
    Bs = [sf.sf_boosters_download(t, 0, e) for e in (2, 3, 4, 5)]
    with torch.no_grad():
        n0 = sf.kernel_launches()
        a = sf.eprl_contraction(t, psis, Bs)
        n_plain = sf.kernel_launches() - n0
    psis_g = [p.clone().requires_grad_(True) for p in psis]
    n0 = sf.kernel_launches()
    a_g = sf.eprl_contraction(t, psis_g, Bs)
    n_grad = sf.kernel_launches() - n0
    assert abs(complex(a) - complex(a_g.detach())) <= 1e-13 * abs(complex(a))
    assert n_plain < n_grad     # the gradient kernels were not launched without a need for them


@pytest.mark.parametrize("tj,dl", [((2,) * 10, 2), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2), ((6,) * 10, 1)])
def test_kappa_matches_oracle(lib, tj, dl):
    bs = ob.random_boosters(tj, dl, 5)
    t = sf.sf_6j_table([sf.vertex(tj, 1.2, dl)])
    _upload(t, 0, bs)
    ref_A, ref_k = ov.vertex_amplitude(tj, dl, bs, return_kappa=True)
    for prec in (sf.SF_FP64, sf.SF_MIXED_FF):
        outs, kap = sf.sf_vertex_amplitude(t, precision=prec, kappa=True)
        assert abs(kap[0] - ref_k) <= 1e-11 * ref_k
    # a shell range: the oracle over the same shells
    n = ov.n_shells(dl)
    b, e = n // 5, (3 * n) // 4
    _, kap = sf.sf_vertex_amplitude(t, shell_begin=b, shell_end=e, kappa=True)
    _, ref_k2 = ov.vertex_amplitude(tj, dl, bs, shells=range(b, e), return_kappa=True)
    assert abs(kap[0] - ref_k2) <= 1e-11 * max(ref_k2, 1e-300)
    # a sub-range: the norms of the block of every contribution
    _, full = sf.intertwiner_ranges(tj, 1.2, dl)
    sub = [(d // 2, 0) for d in full]
    ts = sf.sf_6j_table([sf.vertex(tj, 1.2, dl, sub=sub)])
    _upload(ts, 0, bs)
    _, kap = sf.sf_vertex_amplitude(ts, kappa=True)
    sl = tuple(slice(d // 2, None) for d in full)
    ref_k3 = 0.0
    cache = ov.SixJCache()
    for s_ in range(n):
        C = ov.vertex_amplitude(tj, dl, bs, shells=[s_], sixj=cache)
        ref_k3 += float(np.linalg.norm(C[sl]))
    assert abs(kap[0] - ref_k3) <= 1e-11 * max(ref_k3, 1e-300)
