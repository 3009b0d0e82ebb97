"""Lorentzian EPRL vertex amplitude by the shell sum, for the oracle (Sec. 2, eq. vertex-ampl;
Sec. 3 "Tensor contractions", the framed vertex algorithm).

Test infrastructure only: nothing in the product package may import this module.

    A_v(j_f; i_e) = prod_{e=1..5} sqrt(2 i_e + 1)
                    * sum_{shells l} sum_{k_2..k_5} {15j}(j, l; i_1, k_2..k_5) prod_{e=2..5} (2k_e+1) B4_e(i_e, k_e)

Conventions (doubled spins throughout):
* boundary order  (j12, j13, j14, j15, j23, j24, j25, j34, j35, j45);
* free faces      (l23, l24, l25, l34, l35, l45), l_f = j_f + d_f with d_f in [0, dl];
  gauge faces l_1b = j_1b (Sec. 2 below eq. vertex-ampl);
* linear shell index s = ((((d25*(dl+1) + d35)*(dl+1) + d45)*(dl+1) + d24)*(dl+1) + d34)*(dl+1) + d23
  (an enumeration convention only; the paper does not order its shells);
* edge couplings (the argument orders of the booster tensors in the framed algorithm):
    edge 1: (j12 j13 | j14 j15) -> i1           (no booster)
    edge 2: (j23 j24 | j25 j12) -> i2, (l23 l24 | l25 j12) -> k2
    edge 3: (j34 j35 | j13 j23) -> i3, (l34 l35 | j13 l23) -> k3
    edge 4: (j45 j14 | j24 j34) -> i4, (l45 j14 | l24 l34) -> k4
    edge 5: (j15 j25 | j35 j45) -> i5, (j15 l25 | l35 l45) -> k5
* booster of edge e for the shell is selected by its three free faces, in argument order:
    edge 2 (l23, l24, l25), edge 3 (l34, l35, l23), edge 4 (l45, l24, l34), edge 5 (l25, l35, l45);
  stored as B[e][t][i - i_lo][k - k_lo(t)], t the mixed-radix index of the three d_f.
* output A[i1][i2][i3][i4][i5], i5 fastest (the paper's column-major A^{i5 i4 i3 i2 i1}).
"""
import numpy as np

from . import wigner

FACES = ("12", "13", "14", "15", "23", "24", "25", "34", "35", "45")
FREE = ("23", "24", "25", "34", "35", "45")
EDGE_TRIPLES = {2: ("23", "24", "25"), 3: ("34", "35", "23"), 4: ("45", "24", "34"), 5: ("25", "35", "45")}


def boundary_dict(tj):
    return dict(zip(FACES, tj))


def intertwiner_ranges(tj):
    """Doubled ranges of i1..i5 (Sec. 3, framed algorithm step 2)."""
    j = boundary_dict(tj)
    return [wigner.pair_range(j["12"], j["13"], j["14"], j["15"]),
            wigner.pair_range(j["23"], j["24"], j["25"], j["12"]),
            wigner.pair_range(j["34"], j["35"], j["13"], j["23"]),
            wigner.pair_range(j["45"], j["14"], j["24"], j["34"]),
            wigner.pair_range(j["15"], j["25"], j["35"], j["45"])]


def edge_spins(tj, tl):
    """Per edge 2..5: (boundary 4-tuple, virtual 4-tuple) in coupling order."""
    j = boundary_dict(tj)
    l = dict(j)
    l.update(dict(zip(FREE, tl)))
    return {2: ((j["23"], j["24"], j["25"], j["12"]), (l["23"], l["24"], l["25"], j["12"])),
            3: ((j["34"], j["35"], j["13"], j["23"]), (l["34"], l["35"], j["13"], l["23"])),
            4: ((j["45"], j["14"], j["24"], j["34"]), (l["45"], j["14"], l["24"], l["34"])),
            5: ((j["15"], j["25"], j["35"], j["45"]), (j["15"], l["25"], l["35"], l["45"]))}


def n_shells(dl):
    return (dl + 1) ** 6


def shell_offsets(s, dl):
    """Linear shell index -> (d23, d24, d25, d34, d35, d45)."""
    D = dl + 1
    d23 = s % D
    s //= D
    d34 = s % D
    s //= D
    d24 = s % D
    s //= D
    d45 = s % D
    s //= D
    d35 = s % D
    d25 = s // D
    return (d23, d24, d25, d34, d35, d45)


def shell_spins(tj, dl, s):
    j = boundary_dict(tj)
    d = shell_offsets(s, dl)
    return tuple(j[f] + 2 * df for f, df in zip(FREE, d))


def triple_index(tj, dl, e, tl):
    """Index t of the booster triple of edge e for virtual spins tl (six doubled free l)."""
    j = boundary_dict(tj)
    l = dict(zip(FREE, tl))
    a, b, c = ((l[f] - j[f]) // 2 for f in EDGE_TRIPLES[e])
    return (a * (dl + 1) + b) * (dl + 1) + c


def k_ranges(tj, tl):
    es = edge_spins(tj, tl)
    return [wigner.pair_range(*es[e][1]) for e in (2, 3, 4, 5)]


class SixJCache:
    """Exact {6j} rounded once to float64, memoised on the six doubled arguments."""

    def __init__(self):
        self.c = {}

    def __call__(self, *a):
        v = self.c.get(a)
        if v is None:
            v = wigner.sixj(*a)
            self.c[a] = v
        return v


def shell_W(tj, tl, sixj, i1s=None):
    """W[i1, k2, k3, k4, k5] of one shell: the {15j} block (Sec. 2 eq. 15j; algorithm step 6(i)).

    Returns (W, i1 range, [k2..k5 ranges]) or None when a k range is empty.
    """
    j = boundary_dict(tj)
    l23, l24, l25, l34, l35, l45 = tl
    j12, j13, j14, j15 = j["12"], j["13"], j["14"], j["15"]
    I1 = intertwiner_ranges(tj)[0] if i1s is None else i1s
    K2, K3, K4, K5 = k_ranges(tj, tl)
    if not (K2 and K3 and K4 and K5 and I1):
        return None
    xpar = (I1[0] + l25) % 2
    xmax = max(I1) + l25
    X = list(range(xpar, xmax + 1, 2))
    S1 = np.array([[[sixj(i1, l25, x, k5, j14, j15) for x in X] for k5 in K5] for i1 in I1])
    S2 = np.array([[[sixj(j14, k5, x, l35, k4, l45) for x in X] for k4 in K4] for k5 in K5])
    S3 = np.array([[[sixj(k4, l35, x, k3, l24, l34) for x in X] for k3 in K3] for k4 in K4])
    S4 = np.array([[[sixj(l24, k3, x, j13, k2, l23) for x in X] for k2 in K2] for k3 in K3])
    S5 = np.array([[[sixj(k2, j13, x, i1, l25, j12) for x in X] for i1 in I1] for k2 in K2])
    dim = np.array([x + 1 for x in X], dtype=float)
    # W[a,b,c,d,e] = sum_x (2x+1) S1[a,e,x] S2[e,d,x] S3[d,c,x] S4[c,b,x] S5[b,a,x]
    W = np.einsum("x,aex,edx,dcx,cbx,bax->abcde", dim, S1, S2, S3, S4, S5, optimize=True)
    # sign (-1)^E with E the sum of the 15 entries; E's parity depends on (i1, k2..k5)
    base = j12 + j13 + j14 + j15 + sum(tl)
    E2 = (np.array(I1)[:, None, None, None, None] + np.array(K2)[None, :, None, None, None]
          + np.array(K3)[None, None, :, None, None] + np.array(K4)[None, None, None, :, None]
          + np.array(K5)[None, None, None, None, :] + base)
    if np.any(E2 % 2):
        raise ArithmeticError("non-integer 15j phase exponent")
    W = W * np.where((E2 // 2) % 2 == 1, -1.0, 1.0)
    return W, I1, [K2, K3, K4, K5]


def shell_contribution(tj, dl, s, boosters, sixj):
    """Contribution C_s[i1..i5] of shell s (algorithm steps 6(i)-(iii)); None if the shell is empty.

    boosters: dict e -> dict with 'B' [(dl+1)^3, D_i, D_kmax], 'klo' [(dl+1)^3] (doubled k_lo).
    """
    tl = shell_spins(tj, dl, s)
    res = shell_W(tj, tl, sixj)
    if res is None:
        return None
    W, I1, Ks = res
    mats = []
    for e, K in zip((2, 3, 4, 5), Ks):
        t = triple_index(tj, dl, e, tl)
        b = boosters[e]
        k0 = (K[0] - b["klo"][t]) // 2
        Bsub = b["B"][t][:, k0:k0 + len(K)]
        mats.append(Bsub * np.array([k + 1 for k in K], dtype=float)[None, :])
    # step 6(iii): contract over k2..k5 with the four (2k+1)-weighted booster sub-matrices
    T = np.einsum("abcde,pb,qc,rd,se->apqrs", W, *mats, optimize=True)
    return T


def vertex_amplitude(tj, dl, boosters, shells=None, sixj=None, return_kappa=False):
    """A_v[i1][i2][i3][i4][i5] over a shell range/list (default: all (dl+1)^6 shells).

    Partial sums over disjoint shell sets add up (shell-range additivity).
    """
    sixj = sixj or SixJCache()
    I = intertwiner_ranges(tj)
    A = np.zeros([len(r) for r in I])
    fac = np.sqrt(np.array(I[0], dtype=float) + 1)
    for r in I[1:]:
        fac = np.multiply.outer(fac, np.sqrt(np.array(r, dtype=float) + 1))
    norm_sum = 0.0
    for s in (range(n_shells(dl)) if shells is None else shells):
        C = shell_contribution(tj, dl, int(s), boosters, sixj)
        if C is None:
            continue
        A += C
        norm_sum += float(np.linalg.norm(C * fac))
    A = A * fac
    if return_kappa:
        return A, norm_sum
    return A
