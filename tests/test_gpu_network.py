"""Vertex-tensor contractions and the Delta_3 network on the GPU, through the C ABI, against the
oracle (oracle/network.py).

* vector contractions (3, 4 or 5 trailing indices) on seeded random tensors, the paper's
  homogeneous shapes (2J+1)^5 for J = 2, 4, 12 and irregular ones: error within 1e-13 of the
  sum of |terms| (the oracle's own rounding is of that order);
* at the largest size of the paper's GPU benchmark (J = 24, 49^5 entries, 2.3 GB): rank-1
  tensors against the product of dot products (the factorised closed form), and the two-vertex
  contraction of seeded random tensors against the oracle on the host copy;
* Delta_3: synthetic blocks against the oracle per x and summed; and end to end for J = 1,
  dl = 1 with the vertex tensors of the shell sum (quadrature boosters on a short rule) against
  the oracle's tensors and network.
"""
import numpy as np
import pytest
import torch

import paper_2107_13952_gb300 as sf
from oracle import booster as ob
from oracle import network as on
from oracle import vertex as ov
from paper_2107_13952_gb300 import network as net

pytestmark = pytest.mark.gpu


def _vecs(dims, rng):
    return [rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in dims]


@pytest.mark.parametrize("dims", [(5,) * 5, (9,) * 5, (25,) * 5, (3, 7, 2, 11, 4), (1, 1, 1, 1, 1), (13, 1, 5, 1, 33)])
@pytest.mark.parametrize("nv", [3, 4, 5])
def test_contract_vectors_against_oracle(lib, dims, nv):
    rng = np.random.default_rng(sum(dims) * 7 + nv)
    A = rng.standard_normal(dims)
    psis = _vecs(dims[5 - nv:], rng)
    got = sf.contract_vectors(torch.from_numpy(A).cuda(), psis).cpu().numpy()
    ref = on.contract_vectors(A, psis)
    scale = on.contract_vectors(np.abs(A), [np.abs(p) for p in psis]).real
    assert got.shape == ref.shape
    assert np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300)
    # the same call twice gives the same bits (fixed-order sums)
    again = sf.contract_vectors(torch.from_numpy(A).cuda(), psis).cpu().numpy()
    assert np.array_equal(got, again)


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 1001, 9 ** 5, 25 ** 5 + 3])
def test_contract_vertices_against_oracle(lib, n):
    rng = np.random.default_rng(n)
    A, B = rng.standard_normal(n), rng.standard_normal(n)
    got = float(sf.contract_vertices(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()))
    ref = on.contract_vertices(A, B)
    assert abs(got - ref) <= 1e-13 * float(np.abs(A * B).sum())


def test_full_size_j24(lib):
    D = 49
    rng = np.random.default_rng(24)
    us = [rng.standard_normal(D) for _ in range(5)]
    ut = [torch.from_numpy(u).cuda() for u in us]
    A = torch.einsum("a,b,c,d,e->abcde", *ut).contiguous()      # rank-1 input, built on the device
    psis = _vecs([D] * 5, rng)
    dots = [complex(np.dot(u, p)) for u, p in zip(us, psis)]
    a = complex(sf.contract_vectors(A, psis))
    ref = np.prod(dots)
    assert abs(a - ref) <= 1e-12 * np.prod([np.abs(u).dot(np.abs(p)) for u, p in zip(us, psis)])
    P = sf.contract_vectors(A, psis[2:]).cpu().numpy()
    refP = np.multiply.outer(us[0], us[1]) * np.prod(dots[2:])
    assert np.abs(P - refP).max() <= 1e-12 * np.abs(refP).max()
    sq = float(sf.contract_vertices(A, A))
    ref2 = np.prod([np.dot(u, u) for u in us])
    assert abs(sq - ref2) <= 1e-12 * ref2
    del A
    X = torch.randn(D ** 5, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    Y = torch.randn(D ** 5, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    got = float(sf.contract_vertices(X, Y))
    Xh, Yh = X.cpu().numpy(), Y.cpu().numpy()
    ref = on.contract_vertices(Xh, Yh)
    assert abs(got - ref) <= 1e-13 * float(np.abs(Xh).dot(np.abs(Yh)))


def test_delta3_synthetic_blocks(lib):
    rng = np.random.default_rng(31)
    nb = 5
    nks = [3, 5, 5, 3]
    tensors = [rng.standard_normal((n, n, nb, nb, nb)) for n in nks]
    two_x = [0, 2, 4, 6]
    two_klo = [4, 0, 0, 2]
    psis = _vecs([nb] * 9, rng)
    amps, tot = sf.delta3_amplitudes([torch.from_numpy(T).cuda() for T in tensors], two_x, two_klo, psis)
    ref_amps, ref_tot = on.delta3_total(tensors, two_x, two_klo, psis)
    np.testing.assert_allclose(amps.cpu().numpy(), ref_amps, rtol=1e-12, atol=1e-12 * np.abs(ref_amps).max())
    assert abs(complex(tot) - ref_tot) <= 1e-12 * np.abs(ref_amps).sum()


def test_delta3_end_to_end_j1(lib):
    two_J, dl, gamma, rule = 2, 1, 1.2, (40.0, 4, 10)
    rng = np.random.default_rng(1)
    psis = [v / np.linalg.norm(v) for v in _vecs([3] * 9, rng)]
    xs, amps, tot, tensors = net.delta3(two_J, dl, gamma, psis, rule=rule)
    assert xs == [0, 2, 4, 6]
    ref_tensors, klo = [], []
    for tx in xs:
        tj = (tx,) + (two_J,) * 9
        ref_tensors.append(ov.vertex_amplitude(tj, dl, ob.vertex_boosters(tj, dl, gamma, *rule)))
        klo.append(ov.intertwiner_ranges(tj)[0][0])
    for A, R in zip(tensors, ref_tensors):
        assert float(np.linalg.norm(A.cpu().numpy() - R)) <= 1e-10 * float(np.linalg.norm(R))
    ref_amps, ref_tot = on.delta3_total(ref_tensors, xs, klo, psis)
    np.testing.assert_allclose(amps.cpu().numpy(), ref_amps, rtol=1e-9, atol=1e-10 * np.abs(ref_amps).max())
    assert abs(complex(tot) - ref_tot) <= 1e-9 * np.abs(ref_amps).sum()


def test_contraction_argument_errors(lib):
    A = torch.zeros((2, 2, 2, 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(sf.SfError):
        sf.contract_vectors(A, [np.ones(2)] * 2)
    with pytest.raises(sf.SfError):
        sf.delta3_amplitudes([torch.zeros((2, 3, 2, 2, 2), dtype=torch.float64, device="cuda")], [0], [0],
                             [np.ones(2)] * 9)
