"""Write the oracle's partial shell sums over seeded 10^4-shell subsets of the two largest workloads.

    python tests/golden/make_subsets.py [--workers N] [--only NAME]

Calls only ``oracle/`` (and the seeded input generators). For each workload it draws 10^4 shells
uniformly from the non-empty ones (rejection on the k ranges, ``default_rng(seed)``), takes
seeded random boosters (``oracle.booster.random_boosters``, zero outside the k ranges), sums the
shell contributions in 64 fixed chunks (each chunk in shell order, chunks added in order, so the
result does not depend on the worker count) and saves:

    shells  int64 [10^4], sorted linear shell indices (group-major order)
    A       float64 vertex tensor of the subset, prod sqrt(2 i_e + 1) applied; for tensors of more
            than 65,536 entries only a seeded sample: ``idx`` (flat indices, sorted) and ``A``
            (those entries), with ``A_norm`` the 2-norm of the whole tensor
    kappa   sum over the subset of |C_s|_2 (the cancellation scale of the sum)
    two_j, gamma, dl, booster_seed, shapes (per edge 2..5 the booster tensor shape)

Workloads: all spins 8 (j = 8) with dl = 10, the largest vertex of the homogeneous sweep; and all
spins 4 (j = 4) with dl = 20, 21^6 = 85,766,121 shells.
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
from oracle import vertex as ov       # noqa: E402

N_SUBSET = 10_000
N_CHUNKS = 64
MAX_FULL = 65536
N_SAMPLE = 8192
WORKLOADS = {
    "sweep_j8_dl10_subset": dict(two_j=(16,) * 10, gamma=1.2, dl=10, shell_seed=2107, booster_seed=13952),
    "large_shell_j4_dl20_subset": dict(two_j=(8,) * 10, gamma=1.2, dl=20, shell_seed=2108, booster_seed=13953),
}


def pick_shells(tj, dl, n, seed):
    rng = np.random.default_rng(seed)
    N = ov.n_shells(dl)
    seen = set()
    while len(seen) < n:
        s = int(rng.integers(0, N))
        if s not in seen and all(ov.k_ranges(tj, ov.shell_spins(tj, dl, s))):
            seen.add(s)
    return np.array(sorted(seen), dtype=np.int64)


_BOOSTERS = {}


def _chunk(args):
    tj, dl, seed, shells = args
    key = (tj, dl, seed)
    if key not in _BOOSTERS:
        _BOOSTERS[key] = ob.random_boosters(tj, dl, seed)
    A, kappa = ov.vertex_amplitude(tj, dl, _BOOSTERS[key], shells=shells, return_kappa=True)
    return A, kappa


def make(name, spec, workers):
    tj, dl = spec["two_j"], spec["dl"]
    t0 = time.time()
    shells = pick_shells(tj, dl, N_SUBSET, spec["shell_seed"])
    chunks = np.array_split(shells, N_CHUNKS)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        parts = pool.map(_chunk, [(tj, dl, spec["booster_seed"], c) for c in chunks], chunksize=1)
    A = parts[0][0].copy()
    for p in parts[1:]:
        A += p[0]
    kappa = float(sum(p[1] for p in parts))
    bs = ob.random_boosters(tj, dl, spec["booster_seed"])
    shapes = np.array([bs[e]["B"].shape for e in (2, 3, 4, 5)], dtype=np.int64)
    out = os.path.join(HERE, name + ".npz")
    extra = {}
    if A.size > MAX_FULL:
        rng = np.random.default_rng(spec["shell_seed"] + 1)
        idx = np.sort(rng.choice(A.size, size=N_SAMPLE, replace=False)).astype(np.int64)
        extra = dict(idx=idx, A_norm=float(np.linalg.norm(A)), shape=np.array(A.shape, dtype=np.int64))
        A = A.reshape(-1)[idx]
    np.savez_compressed(out, shells=shells, A=A, kappa=kappa, two_j=np.array(tj, dtype=np.int64),
                        gamma=spec["gamma"], dl=dl, booster_seed=spec["booster_seed"], shapes=shapes, **extra)
    print("%s: %d shells, kappa = %.6e, %.0f s" % (name, len(shells), kappa, time.time() - t0))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    ap.add_argument("--only", default=None)
    a = ap.parse_args()
    for name, spec in WORKLOADS.items():
        if a.only in (None, name):
            make(name, spec, a.workers)


if __name__ == "__main__":
    main()
