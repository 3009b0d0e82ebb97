"""Seeded synthetic inputs for the EPRL vertex workloads (no amplitude arithmetic lives here).

Shared by the tests, the benchmark and the oracle checks; it computes nothing of the method
itself (no symbols, boosters or contractions), only the workload descriptions and random draws.

Workloads (spins are doubled integers, order j12 j13 j14 j15 j23 j24 j25 j34 j35 j45):
* ``simplex_j1``: all spins 1, gamma 1.2, dl in 0..3, rule (r_max 40, 40 panels, 50 nodes);
* ``homogeneous_sweep``: all spins lambda/2 for lambda = 1..16, gamma 1.2, dl 10;
* ``random_batch``: 256 boundaries, spins uniform in {1/2..6}, rejected until all five
  intertwiner ranges are non-empty, dl uniform in 0..12, gamma from {0.1, 1.2, 5.0};
* ``large_shell``: all spins 4, gamma 1.2, dl 20;
* ``boundary_contraction``: all spins 3, gamma 1.2, dl 8, five complex unit boundary vectors.
"""
import numpy as np

DEFAULT_SEED = 13952
RULE_DEFAULT = (40.0, 40, 50)      # r_max, n_panels, GL order per panel: 2000 nodes


def simplex_j1(dl):
    return dict(two_j=(2,) * 10, gamma=1.2, dl=int(dl))


def homogeneous(two_j, dl, gamma=1.2):
    return dict(two_j=(int(two_j),) * 10, gamma=float(gamma), dl=int(dl))


def homogeneous_sweep():
    return [homogeneous(lam, 10) for lam in range(1, 17)]


def large_shell():
    return homogeneous(8, 20)


def boundary_contraction_vertex():
    return homogeneous(6, 8)


def _nonempty(ta, tb, tc, td):
    # an intertwiner coupling (a,b) to (c,d) exists: parity match and overlapping triangles
    if (ta + tb + tc + td) % 2:
        return False
    return max(abs(ta - tb), abs(tc - td)) <= min(ta + tb, tc + td)


def boundary_is_valid(tj):
    """All five intertwiner ranges non-empty (the input's admissibility, used for rejection)."""
    j12, j13, j14, j15, j23, j24, j25, j34, j35, j45 = tj
    return (_nonempty(j12, j13, j14, j15) and _nonempty(j23, j24, j25, j12)
            and _nonempty(j34, j35, j13, j23) and _nonempty(j45, j14, j24, j34)
            and _nonempty(j15, j25, j35, j45))


def random_batch(n=256, seed=0, max_two_j=12, max_dl=12, gammas=(0.1, 1.2, 5.0)):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        tj = tuple(int(v) for v in rng.integers(1, max_two_j + 1, size=10))
        if not boundary_is_valid(tj):
            continue
        dl = int(rng.integers(0, max_dl + 1))
        g = float(gammas[int(rng.integers(0, len(gammas)))])
        out.append(dict(two_j=tj, gamma=g, dl=dl))
    return out


def boundary_vectors(dims, seed=DEFAULT_SEED):
    """Five complex vectors, N(0,1) real and imaginary parts, each normalised to unit 2-norm."""
    rng = np.random.default_rng(seed)
    out = []
    for d in dims:
        v = rng.standard_normal(d) + 1j * rng.standard_normal(d)
        out.append(v / np.linalg.norm(v))
    return out


def shell_subset(n_total, n_pick, seed=DEFAULT_SEED):
    """Seeded sorted subset of linear shell indices (uniform without replacement)."""
    rng = np.random.default_rng(seed)
    n_pick = min(int(n_pick), int(n_total))
    return np.sort(rng.choice(int(n_total), size=n_pick, replace=False)).astype(np.int64)


def random_boosters_like(shapes, seed=DEFAULT_SEED):
    """Random real booster-shaped arrays (for contraction-engine tests that bypass quadrature)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(s) for s in shapes]
