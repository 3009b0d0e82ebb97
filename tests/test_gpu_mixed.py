"""Mixed-precision shell sums. SF_MIXED: the booster contractions over k2, k3 and k4 take FP32
inputs with FP32 accumulation inside one (l24, l34) 5-tuple; the {6j} contractions, the x-sum and
every cross-shell sum stay FP64. SF_MIXED_FF: the same booster contractions, with the {6j}
contractions and the x-sum in compensated FP32 pairs (Dot2). SF_MIXED_TC: the k4 contraction on the
tensor cores (split BF16, FP32 accumulation), the k2, l23 and k3 contractions in FP32, the x-sum
and the cross-shell sums in FP64. SF_MIXED_PX: the booster and S3 contractions in FP32 on the
CUDA cores, the x-sum in compensated FP32 pairs. Stated bound for all four: normwise
relative error <= 1e-6 against the FP64 results, reported beside the cancellation factor
kappa = sum_s ||C_s|| / ||sum_s C_s||."""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import vertex as ov

pytestmark = pytest.mark.gpu

SMALL_RULE = (40.0, 4, 10)


def _rel(a, b):
    return float((a - b).norm() / b.norm())


MIXED_PATHS = [sf.SF_MIXED, sf.SF_MIXED_FF, sf.SF_MIXED_TC, sf.SF_MIXED_PX]


@pytest.mark.parametrize("prec", MIXED_PATHS)
@pytest.mark.parametrize("tj,dl", [((2,) * 10, 3), ((5, 1, 3, 1, 2, 2, 5, 4, 5, 1), 2)])
def test_mixed_matches_oracle(lib, tj, dl, prec):
    t = sf.sf_6j_table([sf.vertex(tj, 1.2, dl)])
    sf.sf_boosters(t, SMALL_RULE)
    A = sf.sf_vertex_amplitude(t, precision=prec)[0].cpu().numpy()
    ref, norm_sum = ov.vertex_amplitude(tj, dl, ob.vertex_boosters(tj, dl, 1.2, *SMALL_RULE), return_kappa=True)
    kappa = norm_sum / np.linalg.norm(ref)
    err = float(np.linalg.norm(A - ref) / np.linalg.norm(ref))
    print("precision %d vs oracle: rel err %.3e, kappa %.2f" % (prec, err, kappa))
    assert err <= 1e-6


@pytest.mark.parametrize("prec", MIXED_PATHS)
@pytest.mark.parametrize("lam,dl,frac", [(4, 10, 1.0), (8, 10, 1.0 / 16), (16, 10, 1.0 / 128), (12, 12, 1.0 / 64)])
def test_mixed_vs_fp64_homogeneous(lib, lam, dl, frac, prec):
    t = sf.sf_6j_table([sf.vertex((lam,) * 10, 1.2, dl)])
    sf.sf_boosters(t, (40.0, 40, 50))
    D = dl + 1
    end = int(D ** 3 * frac) * D ** 3 if frac < 1 else D ** 6
    a64 = sf.sf_vertex_amplitude(t, precision=sf.SF_FP64, shell_end=end)[0]
    amx = sf.sf_vertex_amplitude(t, precision=prec, shell_end=end)[0]
    err = _rel(amx, a64)
    print("lambda=%d dl=%d: precision %d vs FP64 rel err %.3e" % (lam, dl, prec, err))
    assert err <= 1e-6


def test_fp64_path_unchanged_by_mixed_instantiation(lib):
    # determinism of the FP64 path across repeated calls with the mixed path in between
    t = sf.sf_6j_table([sf.vertex((6,) * 10, 1.2, 3)])
    sf.sf_boosters(t, SMALL_RULE)
    a = sf.sf_vertex_amplitude(t)[0].clone()
    sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED)
    sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_FF)
    sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_TC)
    sf.sf_vertex_amplitude(t, precision=sf.SF_MIXED_PX)
    b = sf.sf_vertex_amplitude(t)[0]
    assert torch.equal(a, b)
