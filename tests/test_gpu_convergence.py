"""The shell-convergence driver (Sec. 5 "Lorentzian 4-simplex asymptotics", fig. lorasym-conv)
through the C ABI: the tensors A(dl) of one boundary for dl = 0..dl_max in one batched launch.

* small cutoffs against the oracle (spin 1, dl = 0..2, quadrature boosters on a short rule,
  whole tensors, 1e-10);
* nesting: A(dl) equals the FP64 sum over the shells of the dl_max grid whose six offsets are at
  most dl (shell list on the dl_max tables), so the study's differences are those of the shell sum;
* the study's record: one row per (lambda, gamma) with dl_max relative changes.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import vertex as ov
from paper_2107_13952_gb300 import network as net

pytestmark = pytest.mark.gpu

RULE = (40.0, 4, 10)


def _psis(dims, seed):
    rng = np.random.default_rng(seed)
    return [v / np.linalg.norm(v) for v in (rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in dims)]


def test_small_cutoffs_against_oracle(lib):
    tj, gamma, dl_max = (2,) * 10, 1.2, 2
    _, dims = sf.intertwiner_ranges(tj, gamma, dl_max)
    tensors, amps = net.shell_convergence(tj, gamma, dl_max, _psis(dims, 1), rule=RULE)
    for dl, A in enumerate(tensors):
        ref = ov.vertex_amplitude(tj, dl, ob.vertex_boosters(tj, dl, gamma, *RULE))
        assert float(np.linalg.norm(A.cpu().numpy() - ref)) <= 1e-10 * float(np.linalg.norm(ref)), dl


@pytest.mark.parametrize("lam,gamma", [(4, 1.2), (6, 5.0)])
def test_cutoffs_nest_in_the_largest_grid(lib, lam, gamma):
    tj, dl_max = (lam,) * 10, 4
    _, dims = sf.intertwiner_ranges(tj, gamma, dl_max)
    tensors, _ = net.shell_convergence(tj, gamma, dl_max, _psis(dims, 2), rule=RULE)
    t = sf.sf_6j_table([sf.vertex(tj, gamma, dl_max)])
    sf.sf_boosters(t, RULE)
    D = dl_max + 1
    offs = np.indices((D,) * 6).reshape(6, -1)          # axes (d25, d35, d45, d24, d34, d23): group-major
    for dl in range(dl_max):
        sel = np.nonzero(offs.max(axis=0) <= dl)[0].astype(np.int64)
        A = sf.sf_vertex_amplitude(t, shell_list=sel)[0]
        n = float(tensors[dl].norm())
        assert float((A - tensors[dl]).norm()) <= 1e-12 * n, dl


def test_study_record(lib):
    res = net.convergence_study(lams=(2,), gammas=(0.1, 1.2), dl_max=3, rule=RULE)
    assert len(res["rows"]) == 2
    for row in res["rows"]:
        assert len(row["rel_change_amplitude"]) == 3 and len(row["rel_change_tensor"]) == 3
        assert all(np.isfinite(row["rel_change_tensor"]))
