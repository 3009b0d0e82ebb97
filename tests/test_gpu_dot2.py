"""The compensated-pair dot products of SF_MIXED_FF on the device, through ``sf_check_dot2``, which
runs the shell kernel's own pair steps (Dot2 of Ogita, Rump and Oishi with Dekker's FMA
TwoProduct). Cancelling sums like a {6j} x-sum; the reference is the exact rational dot product of
the operands' pair values. Bound: 16 n 2^-48 of the sum of |terms| (the dropped lo x lo term and
the compensated sum), the bound that the host restatement in test_compensated_pairs.py meets;
plain float32 accumulation of the same sums fails it by orders of magnitude."""
from fractions import Fraction

import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf

pytestmark = pytest.mark.gpu


def _split(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _cases(n, n_dots, seed):
    rng = np.random.default_rng(seed)
    xs = rng.standard_normal((n_dots, n)) * np.where(np.arange(n) % 2, -1.0, 1.0) * 1e-2
    ys = rng.standard_normal((n_dots, n))
    ys[:, -1] = -np.einsum("ij,ij->i", xs[:, :-1], ys[:, :-1]) / xs[:, -1] * (1 + 1e-9 * rng.standard_normal(n_dots))
    return xs, ys


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("n", [8, 27])
def test_device_dot2_error_bound(lib, kind, n):
    n_dots = 256
    xs, ys = _cases(n, n_dots, 100 + n + kind)
    ah, al = _split(xs)
    a = np.stack([ah, al], axis=-1)
    if kind == 0:
        yv = ys.astype(np.float32)
        b = yv
        yval = yv.astype(np.float64)
    else:
        bh, bl = _split(ys)
        b = np.stack([bh, bl], axis=-1)
        yval = bh.astype(np.float64) + bl.astype(np.float64)   # exact: the pair's value
    xval = ah.astype(np.float64) + al.astype(np.float64)
    out = sf.check_dot2(kind, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    worst = 0.0
    for q in range(n_dots):
        ref = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(xval[q], yval[q]))
        got = Fraction(float(out[q, 0])) + Fraction(float(out[q, 1]))
        scale = float(sum(abs(Fraction(float(x)) * Fraction(float(y))) for x, y in zip(xval[q], yval[q])))
        worst = max(worst, float(abs(got - ref)) / scale)
        # normalised pair: |lo| <= ulp(hi) / 2
        assert abs(float(out[q, 1])) <= np.spacing(np.float32(abs(out[q, 0]))) / 2 + 1e-45
    assert worst <= 16 * n * 2.0 ** -48, worst
    plain = np.zeros(n_dots, dtype=np.float32)
    for k in range(n):
        plain = (plain + (xval[:, k].astype(np.float32) * yval[:, k].astype(np.float32))).astype(np.float32)
    ref0 = np.einsum("ij,ij->i", xval, yval)
    scale0 = np.einsum("ij,ij->i", np.abs(xval), np.abs(yval))
    assert np.max(np.abs(plain - ref0) / scale0) > 1000 * worst


def test_device_dot2_rejects_bad_kind(lib):
    a = torch.zeros((1, 2, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(sf.SfError):
        sf.check_dot2(2, a, a)
