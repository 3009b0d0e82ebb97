"""The allocation-free entry point gives the same vertex tensor as sf_vertex_amplitude.

sf_vertex_amplitude_noalloc is for callers that must not allocate device memory while they run
(a framework that owns a fixed memory pool, a host that forbids allocation after start-up). It
takes its scratch from one fixed device array, so two calls in a row must both match the
allocating entry point, and a request larger than the array must be refused with SF_ERR_LIMIT.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf

pytestmark = pytest.mark.gpu


def _tables(tj, dl, seed):
    t = sf.sf_6j_table([sf.vertex(tj, 1.2, dl)])
    rng = np.random.default_rng(seed)
    for e in (2, 3, 4, 5):
        sf.sf_boosters_upload(t, 0, e, rng.standard_normal(sf.booster_shape(t, 0, e)))
    return t


@pytest.mark.parametrize("tj,dl", [((2,) * 10, 2), ((6,) * 10, 2)])
def test_noalloc_matches_allocating_entry_point(lib, tj, dl):
    t = _tables(tj, dl, seed=7)
    ref = sf.sf_vertex_amplitude(t)[0]
    for _ in range(2):
        out = [torch.full_like(ref, float("nan"))]
        sf.sf_vertex_amplitude_noalloc(t, out)
        rel = float((out[0] - ref).norm() / ref.norm())
        assert rel <= 1e-12
    # a shell range behaves like the allocating entry point's range
    n = sf.num_shells(tj, 1.2, dl)
    ref_r = sf.sf_vertex_amplitude(t, shell_begin=0, shell_end=n // 2)[0]
    out = [torch.empty_like(ref)]
    sf.sf_vertex_amplitude_noalloc(t, out, shell_begin=0, shell_end=n // 2)
    assert float((out[0] - ref_r).norm() / ref_r.norm()) <= 1e-12


def test_noalloc_rejects_oversized_requests(lib):
    # sixteen vertices with all spins lambda/2, dl = 10: the partial tiles exceed the fixed array
    verts = [sf.vertex((lam,) * 10, 1.2, 10) for lam in range(1, 17)]
    t = sf.sf_6j_table(verts)
    rng = np.random.default_rng(0)
    for v in range(16):
        for e in (2, 3, 4, 5):
            sf.sf_boosters_upload(t, v, e, rng.standard_normal(sf.booster_shape(t, v, e)))
    outs = [torch.empty(sf.intertwiner_ranges((lam,) * 10, 1.2, 10)[1], dtype=torch.float64, device="cuda")
            for lam in range(1, 17)]
    with pytest.raises(sf.SfError) as e:
        sf.sf_vertex_amplitude_noalloc(t, outs)
    assert e.value.code == sf.SF_ERR_LIMIT
