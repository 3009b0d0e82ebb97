"""Contractions of vertex tensors and the Delta_3 spin foam, for the oracle.

Test infrastructure only: nothing in the product package may import this module.

Sec. 3 "Tensor contractions" (eq. vertex-contraction): a spin foam amplitude is the contraction
of its vertex tensors A[i1][i2][i3][i4][i5] over the intertwiner indices that the 2-complex
connects, and with boundary states on the boundary edges. The paper's GPU examples
(Sec. 4 "Tensor contractions on CPU and GPU", fig. contractions) are the complete contraction of
two vertex tensors and of one vertex tensor with five boundary states.

Sec. 5 "The Delta_3 graph": three vertices pairwise joined by internal edges (intertwiners
k1, k2, k3) that share one internal face of spin x; with all boundary spins J and the internal
face x, the three vertex tensors are equal (boundary spins (x, J, ..., J)) and each is contracted
with three boundary states on its indices (i3, i4, i5), leaving a matrix over its two internal
edges: T_A over (k1, k2), T_B over (k3, k1), T_C over (k2, k3) in the order the paper's listing
reads them. The amplitude at fixed x is

    (-1)^x (2x+1) sum_{k1 k2 k3} (-1)^(k1+k2+k3) T_A[k2, k1] T_B[k1, k3] T_C[k3, k2]

with the paper's column-major T_A[k2, k1] equal to the row-major partial contraction
P_A[k1][k2] of A[i1][i2][...] (i1 the first internal edge, i2 the second); the graph's amplitude
is the sum over x. Plain numpy in float64/complex128; each step as stated.
"""
import numpy as np


def contract_vectors(A, psis):
    """sum over the trailing len(psis) indices of A[i1..i5] prod psi_e[i_e]; psis[0] pairs with
    index 5 - len(psis) + 1 (one-based). Returns the complex array over the leading indices."""
    A = np.asarray(A, dtype=np.float64)
    T = A.astype(np.complex128)
    for psi in reversed(psis):          # contract the last index with the last vector, and so on
        T = T @ np.asarray(psi, dtype=np.complex128)
    return T


def contract_vertices(A, B):
    """Complete contraction sum_i A[i] B[i] of two vertex tensors of the same shape."""
    return float(np.dot(np.asarray(A, dtype=np.float64).ravel(), np.asarray(B, dtype=np.float64).ravel()))


def delta3_amplitude(A, two_x, two_klo, psis):
    """Delta_3 amplitude at one internal spin x (doubled: two_x) from the vertex tensor A of
    boundary spins (x, J, ..., J); two_klo is the doubled lowest internal intertwiner (the first
    value of i1 and of i2); psis: nine boundary vectors, three per vertex on (i3, i4, i5)."""
    PA = contract_vectors(A, psis[0:3])     # P_A[k1][k2]
    PB = contract_vectors(A, psis[3:6])     # P_B[k3][k1]
    PC = contract_vectors(A, psis[6:9])     # P_C[k2][k3]
    nk = PA.shape[0]
    ks = [(two_klo + 2 * n) // 2 for n in range(nk)]
    amx = 0.0 + 0.0j
    for n1 in range(nk):
        for n2 in range(nk):
            for n3 in range(nk):
                sign = (-1) ** (ks[n1] + ks[n2] + ks[n3])
                # the listing's tA[k2, k1] tB[k1, k3] tC[k3, k2] in row-major form
                amx += sign * PA[n1, n2] * PB[n3, n1] * PC[n2, n3]
    x = two_x // 2
    return (-1) ** x * (two_x + 1) * amx


def delta3_total(tensors, two_x, two_klo, psis):
    """Per-x amplitudes and their sum over the internal face's spin."""
    amps = [delta3_amplitude(A, tx, tk, psis) for A, tx, tk in zip(tensors, two_x, two_klo)]
    return np.array(amps), complex(sum(amps))
