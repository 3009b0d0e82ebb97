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


def convergence_study(lams=(2, 10), gammas=(0.1, 1.2, 5.0, 10.0), dl_max=12, rule=(40.0, 40, 50), seed=13952,
                      precision=SF_FP64):
    """The shell-convergence study of Sec. 5 (fig. lorasym-conv) on homogeneous boundaries: for all
    spins j = lambda/2 and each gamma, the relative change of the vertex amplitude between shell
    cutoff dl and dl_max, for dl = 0..dl_max - 1, both for the boundary-contracted amplitude (seeded
    unit vectors) and for the whole tensor (2-norm). Returns a JSON-ready dict."""
    import numpy as np
    out = {"rule": list(rule), "dl_max": dl_max, "precision": int(precision), "rows": []}
    for lam in lams:
        tj = (lam,) * 10
        _, dims = intertwiner_ranges(tj, 1.0, dl_max)
        rng = np.random.default_rng(seed + lam)
        psis = [v / np.linalg.norm(v) for v in
                (rng.standard_normal(d) + 1j * rng.standard_normal(d) for d in dims)]
        for g in gammas:
            tensors, amps = shell_convergence(tj, g, dl_max, psis, rule=rule, precision=precision)
            ref_a = complex(amps[-1])
            ref_A = tensors[-1]
            nA = float(ref_A.norm())
            row = {"lambda": lam, "gamma": g, "amplitude": [ref_a.real, ref_a.imag], "tensor_norm": nA,
                   "rel_change_amplitude": [abs(complex(a) - ref_a) / abs(ref_a) for a in amps[:-1]],
                   "rel_change_tensor": [float((A - ref_A).norm()) / nA for A in tensors[:-1]]}
            out["rows"].append(row)
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="shell-convergence study (relative change of the amplitude vs dl)")
    ap.add_argument("--lams", default="2,10")
    ap.add_argument("--gammas", default="0.1,1.2,5.0,10.0")
    ap.add_argument("--dl-max", type=int, default=12)
    ap.add_argument("--rule", default="40,40,50", help="r_max,n_panels,order")
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    r = a.rule.split(",")
    res = convergence_study(tuple(int(v) for v in a.lams.split(",")), tuple(float(v) for v in a.gammas.split(",")),
                            a.dl_max, (float(r[0]), int(r[1]), int(r[2])))
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)
