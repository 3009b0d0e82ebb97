"""Drivers over the C ABI for networks of vertices (argument marshalling only).

* ``delta3``: the Delta_3 spin foam of Sec. 5 "The Delta_3 graph" (three vertices, one internal
  face of spin x, three internal edges): for every admissible x the vertex tensor of boundary
  spins (x, J, ..., J) from the shell sum (all x in one batched tables object and one persistent
  launch), then the three partial contractions with the nine boundary vectors and the internal
  sum, per x and summed over x (``sf_delta3_amplitudes``).
* ``shell_convergence``: the amplitude at shell cutoffs dl = 0..dl_max (Sec. 5 "Lorentzian
  4-simplex asymptotics", fig. lorasym-conv) as one batched launch over the dl_max + 1 vertices
  of the same boundary, each contracted with the same boundary vectors.

Every arithmetic step runs in the library's kernels; these functions only build the argument
lists. The boundary vectors are the caller's (the paper's coherent states are not part of this
library: any unit vectors over the intertwiner ranges may be passed).
"""
from . import (SF_FP64, SfError, contract_vectors, delta3_amplitudes, intertwiner_ranges, sf_6j_table, sf_boosters,
               sf_vertex_amplitude, vertex)


def delta3_spins(two_J):
    """Doubled internal spins x of the Delta_3 graph with all boundary spins J (integers): every x
    for which the boundary (x, J, ..., J) has non-empty intertwiner ranges."""
    assert two_J % 2 == 0, "integer boundary spins"
    xs = []
    for two_x in range(0, 3 * two_J + 1, 2):
        tj = (two_x,) + (two_J,) * 9
        try:
            intertwiner_ranges(tj)
        except SfError:
            continue
        xs.append(two_x)
    return xs


def delta3(two_J, dl, gamma, psis, rule=(40.0, 40, 50), precision=SF_FP64, boosters=None):
    """Delta_3 amplitudes per internal spin and their sum, with boundary spins J (doubled two_J),
    shell cutoff dl and Immirzi gamma. psis: nine boundary vectors of length 2J+1 (three per
    vertex, on its boundary intertwiners i3, i4, i5). boosters: optional callable (tables, index,
    two_j) that uploads boosters instead of computing them by quadrature (e.g. the BF limit).
    Returns (two_x list, amps [n_x] complex, total complex, vertex tensors)."""
    xs = delta3_spins(two_J)
    verts = [vertex((tx,) + (two_J,) * 9, gamma, dl) for tx in xs]
    t = sf_6j_table(verts)
    if boosters is None:
        sf_boosters(t, rule)
    else:
        for i, tx in enumerate(xs):
            boosters(t, i, (tx,) + (two_J,) * 9)
    tensors = sf_vertex_amplitude(t, precision)
    klo = [intertwiner_ranges((tx,) + (two_J,) * 9, gamma, dl)[0][0] for tx in xs]
    amps, total = delta3_amplitudes(tensors, xs, klo, psis)
    return xs, amps, total, tensors


def shell_convergence(two_j, gamma, dl_max, psis, rule=(40.0, 40, 50), precision=SF_FP64):
    """Vertex tensors A(dl) of one boundary for dl = 0..dl_max (one tables object, one batched
    shell sum) and their contractions a(dl) with the five boundary vectors psis.
    Returns (tensors, amplitudes)."""
    verts = [vertex(two_j, gamma, d) for d in range(dl_max + 1)]
    t = sf_6j_table(verts)
    sf_boosters(t, rule)
    tensors = sf_vertex_amplitude(t, precision)
    amps = [contract_vectors(A, psis) for A in tensors]
    return tensors, amps
