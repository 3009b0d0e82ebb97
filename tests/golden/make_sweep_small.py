"""Write the oracle's whole vertex tensors of the two smallest vertices of the homogeneous sweep
at full size, with boosters by quadrature on the full rule.

    python tests/golden/make_sweep_small.py [--workers N]

Calls only ``oracle/``. Vertices: all spins 1/2 and all spins 1 (lambda = 1, 2), gamma 1.2,
dl 10 (11^6 = 1,771,561 shells each), rule r_max 40, 40 panels x 50 Gauss-Legendre nodes; the
booster tensors from ``oracle.booster.vertex_boosters`` (d-functions by the closed form in
arbitrary precision) and the shell sum from ``oracle.vertex.vertex_amplitude`` over all shells, in
64 fixed chunks of the shell range (each chunk in shell order, chunks added in order). Saves, per
vertex, ``A`` (the whole tensor, prod sqrt(2 i_e + 1) applied) and ``kappa`` (sum of the shells'
contribution norms) in ``sweep_small_dl10.npz`` under the keys ``A_<lambda>``, ``kappa_<lambda>``.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import booster as ob      # noqa: E402
from oracle import quadrature as oq   # noqa: E402
from oracle import vertex as ov       # noqa: E402

RULE = (40.0, 40, 50)
DL = 10
GAMMA = 1.2
LAMS = (1, 2)
N_CHUNKS = 64


def _dtable(args):
    tk, tl = args
    xs, _ = oq.rule_nodes(*RULE)
    return (tk, tl), ob.DTable(tk, GAMMA, [tl], xs)


_B = {}


def _chunk(args):
    lam, lo, hi, path = args
    if lam not in _B:
        _B[lam] = dict(np.load(path, allow_pickle=True)["b"].item())
    A, kap = ov.vertex_amplitude((lam,) * 10, DL, _B[lam], shells=range(lo, hi), return_kappa=True)
    return A, kap


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    a = ap.parse_args()
    ctx = mp.get_context("spawn")
    out = {}
    for lam in LAMS:
        t0 = time.time()
        tj = (lam,) * 10
        faces = {}
        with ctx.Pool(a.workers) as pool:
            need = sorted({(lam, lam + 2 * d) for d in range(DL + 1)})
            tabs = dict(pool.map(_dtable, need, chunksize=1))
        xs, ws = oq.rule_nodes(*RULE)

        class Face:
            def __init__(self, tk):
                self.tk = tk

            def get(self, tl, tm):
                return tabs[(self.tk, tl)].get(tl, tm)
        for f in ov.FACES:
            faces[f] = Face(lam)
        b = ob.vertex_boosters(tj, DL, GAMMA, *RULE, tables=faces)
        path = os.path.join(HERE, "_boosters_tmp_%d.npz" % lam)
        np.savez(path, b=np.array(b, dtype=object))
        n = ov.n_shells(DL)
        bounds = [n * c // N_CHUNKS for c in range(N_CHUNKS + 1)]
        with ctx.Pool(a.workers) as pool:
            parts = pool.map(_chunk, [(lam, bounds[c], bounds[c + 1], path) for c in range(N_CHUNKS)], chunksize=1)
        os.remove(path)
        A = parts[0][0].copy()
        for p in parts[1:]:
            A += p[0]
        out["A_%d" % lam] = A
        out["kappa_%d" % lam] = float(sum(p[1] for p in parts))
        print("lambda %d: |A| = %.6e, kappa sum %.6e, %.0f s" % (lam, np.linalg.norm(A), out["kappa_%d" % lam],
                                                              time.time() - t0), flush=True)
    np.savez_compressed(os.path.join(HERE, "sweep_small_dl10.npz"), **out)


if __name__ == "__main__":
    main()
