"""Write the oracle's booster matrices on sampled virtual-spin triples of the benchmarked vertices.

    python tests/golden/make_boosters.py [--workers N] [--only NAME]

Calls only ``oracle/`` (booster quadrature of eq. booster on the rule of Sec. 3 "Booster
coefficients", d-functions by the exact-coefficient closed form). Cases:

* ``j8_dl10_short`` / ``j8_dl10_full``: all spins 8, gamma 1.2, dl 10 (the largest vertex of the
  homogeneous sweep), on the rule (r_max 40, 4 panels x 10 nodes) and on the full rule
  (40 panels x 50 nodes); 17 x 17 matrices whose node sums run in chunks of 16 nodes;
* ``j6_dl12_g5_short`` / ``j6_dl12_g5_full``: all spins 6, gamma 5.0, dl 12 (the extreme faces of
  the 256-vertex batch: largest spin, largest gamma, largest dl);
* ``zero_edge_full``: spins (1, 1, 1, 0, 1, 1, 0, 1, 0, 0), gamma 1.2, dl 2, every triple of every
  edge on the full rule: edge 5 couples four spin-0 faces, whose node sums run in chunks of 1024
  (one full chunk and one partial chunk of the 2000 nodes).

Triples are mixed-radix indices t = (a D + b) D + c of the edge's three free-face offsets (the
booster layout of include/sf_eprl.h); each case stores, for its sampled (edge, t) pairs:
    edge, t   int64 [n]
    B         float64 [n, D_i, D_kmax_case] (zero beyond each triple's k range)
    nk        int64 [n]   k-range length of each triple
    two_j, gamma, dl, rule
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
from oracle import wigner as ow       # noqa: E402

SHORT = (40.0, 4, 10)
FULL = (40.0, 40, 50)
CASES = {
    "j8_dl10_short": dict(two_j=(16,) * 10, gamma=1.2, dl=10, rule=SHORT, per_edge=4, seed=1),
    "j8_dl10_full": dict(two_j=(16,) * 10, gamma=1.2, dl=10, rule=FULL, per_edge=1, seed=2, offsets=(0, 10)),
    "j6_dl12_g5_short": dict(two_j=(12,) * 10, gamma=5.0, dl=12, rule=SHORT, per_edge=3, seed=3),
    "j6_dl12_g5_full": dict(two_j=(12,) * 10, gamma=5.0, dl=12, rule=FULL, per_edge=1, seed=4, offsets=(0, 12)),
    "zero_edge_full": dict(two_j=(2, 2, 2, 0, 2, 2, 0, 2, 0, 0), gamma=1.2, dl=2, rule=FULL, per_edge=None, seed=5),
}


def edge_triple_spins(tj, dl, e, t):
    """(boundary spins, virtual spins) of edge e at triple t, in the edge's coupling order."""
    D = dl + 1
    d = (t // (D * D), (t // D) % D, t % D)
    tl6 = dict(zip(ov.FREE, [tj[ov.FACES.index(f)] for f in ov.FREE]))
    for f, df in zip(ov.EDGE_TRIPLES[e], d):
        tl6[f] += 2 * df
    return ov.edge_spins(tj, tuple(tl6[f] for f in ov.FREE))[e]


def sample_triples(spec):
    tj, dl = spec["two_j"], spec["dl"]
    D = dl + 1
    rng = np.random.default_rng(spec["seed"])
    out = []
    for e in (2, 3, 4, 5):
        if spec["per_edge"] is None:
            ts = list(range(D ** 3))
        else:
            if "offsets" in spec:
                vals = spec["offsets"]
                ts = [int((a * D + b) * D + c) for a, b, c in [tuple(rng.choice(vals, 3)) for _ in range(spec["per_edge"])]]
            else:
                ts = [0, D ** 3 - 1] + [int(v) for v in rng.integers(0, D ** 3, spec["per_edge"] - 2)]
        for t in ts:
            if ow.pair_range(*edge_triple_spins(tj, dl, e, t)[1]):
                out.append((e, t))
    return out


def _dtable(args):
    tk, gamma, tl, rule = args
    xs, _ = oq.rule_nodes(*rule)
    return (tk, tl), ob.DTable(tk, gamma, [tl], xs)


def make(name, spec, workers):
    t0 = time.time()
    tj, dl, gamma, rule = spec["two_j"], spec["dl"], spec["gamma"], spec["rule"]
    pairs = sample_triples(spec)
    faces = {2: ("23", "24", "25", "12"), 3: ("34", "35", "13", "23"), 4: ("45", "14", "24", "34"),
             5: ("15", "25", "35", "45")}
    need = set()
    for e, t in pairs:
        bj, bl = edge_triple_spins(tj, dl, e, t)
        for a in range(4):
            need.add((bj[a], bl[a]))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        tabs = dict(pool.map(_dtable, [(tk, gamma, tl, rule) for tk, tl in sorted(need)], chunksize=1))
    xs, ws = oq.rule_nodes(*rule)
    wm = ob.node_weights(xs, ws)
    mats, nks = [], []
    for e, t in pairs:
        bj, bl = edge_triple_spins(tj, dl, e, t)
        B, _, _, _ = ob.booster(bj, bl, [tabs[(bj[a], bl[a])] for a in range(4)], wm)
        mats.append(B)
        nks.append(B.shape[1])
    di = max(m.shape[0] for m in mats)
    dk = max(nks)
    arr = np.zeros((len(mats), di, dk))
    for q, m in enumerate(mats):
        arr[q, :m.shape[0], :m.shape[1]] = m
    np.savez_compressed(os.path.join(HERE, "boosters_" + name + ".npz"), edge=np.array([p[0] for p in pairs]),
                        t=np.array([p[1] for p in pairs]), B=arr, nk=np.array(nks), two_j=np.array(tj),
                        gamma=gamma, dl=dl, rule=np.array(rule))
    print("%s: %d boosters, %d d-tables, %.0f s" % (name, len(pairs), len(need), time.time() - t0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    for name, spec in CASES.items():
        if a.only in (None, name):
            make(name, spec, a.workers)


if __name__ == "__main__":
    main()
