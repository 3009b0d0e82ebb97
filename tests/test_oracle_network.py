"""Pins of the oracle's vertex-tensor contractions and Delta_3 amplitude (no device work).

* rank-1 tensors A = u1 x u2 x u3 x u4 x u5: every contraction with boundary vectors factorises
  into dot products u_e . psi_e (a transposed or mis-paired index fails it);
* the complete two-vertex contraction of A with itself is ||A||^2, of two rank-1 tensors the
  product of the factors' dot products;
* Delta_3: with diagonal internal blocks the amplitude reduces to (-1)^x (2x+1) sum_k (-1)^k d_k^3
  times the boundary factors; relabelling the three vertices cyclically leaves it unchanged.
"""
import numpy as np
import pytest

from oracle import network


def _rank1(dims, rng):
    us = [rng.standard_normal(d) for d in dims]
    A = us[0]
    for u in us[1:]:
        A = np.multiply.outer(A, u)
    return A, us


def _vecs(dims, rng):
    return [rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in dims]


@pytest.mark.parametrize("dims", [(3, 4, 2, 5, 3), (1, 1, 1, 1, 1), (5, 5, 5, 5, 5), (2, 3, 7, 1, 4)])
@pytest.mark.parametrize("nv", [3, 4, 5])
def test_rank_one_contraction_factorises(dims, nv):
    rng = np.random.default_rng(sum(dims) + nv)
    A, us = _rank1(dims, rng)
    psis = _vecs(dims[5 - nv:], rng)
    got = network.contract_vectors(A, psis)
    scal = np.prod([np.dot(u, p) for u, p in zip(us[5 - nv:], psis)])
    lead = us[0] if nv == 4 else (np.multiply.outer(us[0], us[1]) if nv == 3 else np.array(1.0))
    np.testing.assert_allclose(got, lead * scal, rtol=1e-12, atol=1e-12 * np.abs(lead * scal).max())


def test_vertex_contractions():
    rng = np.random.default_rng(4)
    dims = (4, 3, 5, 2, 6)
    A = rng.standard_normal(dims)
    assert abs(network.contract_vertices(A, A) - np.linalg.norm(A) ** 2) <= 1e-12 * np.linalg.norm(A) ** 2
    R1, u = _rank1(dims, rng)
    R2, v = _rank1(dims, rng)
    ref = np.prod([np.dot(a, b) for a, b in zip(u, v)])
    assert abs(network.contract_vertices(R1, R2) - ref) <= 1e-12 * abs(ref)


def _delta3_case(nk, nb, two_x, rng):
    d = rng.standard_normal(nk)
    u = [rng.standard_normal(nb) for _ in range(3)]
    A = np.zeros((nk, nk, nb, nb, nb))
    for k in range(nk):
        A[k, k] = d[k] * np.multiply.outer(np.multiply.outer(u[0], u[1]), u[2])
    psis = _vecs([nb] * 9, rng)
    return A, d, u, psis


@pytest.mark.parametrize("two_klo,nk", [(0, 3), (2, 4), (4, 5)])
def test_delta3_diagonal_blocks_closed_form(two_klo, nk):
    rng = np.random.default_rng(nk)
    two_x = 4
    A, d, u, psis = _delta3_case(nk, 3, two_x, rng)
    boundary = np.prod([np.dot(u[e % 3], psis[e]) for e in range(9)])
    ks = [(two_klo + 2 * n) // 2 for n in range(nk)]
    ref = (-1) ** (two_x // 2) * (two_x + 1) * sum((-1) ** k * d[n] ** 3 for n, k in enumerate(ks)) * boundary
    got = network.delta3_amplitude(A, two_x, two_klo, psis)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_delta3_cyclic_relabelling_invariance():
    rng = np.random.default_rng(9)
    nk, nb = 4, 3
    A = rng.standard_normal((nk, nk, nb, nb, nb))
    psis = _vecs([nb] * 9, rng)
    a0 = network.delta3_amplitude(A, 2, 0, psis)
    # roles (0, 1, 2) -> (2, 0, 1): vertex 0 takes vertex 2's states, 1 takes 0's, 2 takes 1's
    shifted = psis[6:9] + psis[0:3] + psis[3:6]
    a1 = network.delta3_amplitude(A, 2, 0, shifted)
    assert abs(a0 - a1) <= 1e-12 * abs(a0)
    # a non-cyclic exchange of two vertices is a different network (the pin has teeth)
    swapped = psis[3:6] + psis[0:3] + psis[6:9]
    assert abs(network.delta3_amplitude(A, 2, 0, swapped) - a0) > 1e-6 * abs(a0)


def test_delta3_total_sums_over_x():
    rng = np.random.default_rng(2)
    As = [rng.standard_normal((n, n, 3, 3, 3)) for n in (2, 3, 4)]
    psis = _vecs([3] * 9, rng)
    amps, tot = network.delta3_total(As, [0, 2, 4], [2, 0, 0], psis)
    assert abs(tot - sum(network.delta3_amplitude(A, tx, tk, psis)
                         for A, tx, tk in zip(As, [0, 2, 4], [2, 0, 0]))) <= 1e-12 * abs(tot)
