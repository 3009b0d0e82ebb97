"""Booster functions B4^gamma for the oracle (Sec. 2, eq. booster; Sec. 3 "Booster coefficients").

Test infrastructure only: nothing in the product package may import this module.

    B4(j_1..j_4, i; l_1..l_4, k) = sum_{m_a} 4jm(j; m)^(i) 4jm(l; m)^(k)
                                   * int_0^inf dr sinh^2(r)/(4 pi) prod_a d^{gamma(j_a+1), j_a}_{j_a l_a m_a}(r)

The r-integral is the rule of ``quadrature.rule_nodes`` (same panels and node count as the GPU
path), with every d value taken from the arbitrary-precision closed form (``dfunc.DClosed``)
and rounded once to complex128; the node sums and the m-sum are plain float64/complex128.
The imaginary part is checked to vanish (the phase convention of ``dfunc`` makes B4 real).
"""
import itertools

import mpmath
import numpy as np

from . import dfunc, quadrature, wigner


class DTable:
    """d^{gamma(k+1),k}_{k l m}(r_n) for one face: all l in ``tls``, all m, all rule nodes."""

    def __init__(self, tk, gamma, tls, xs, dps=20):
        self.tk = tk
        self.rho = mpmath.mpf(gamma) * (mpmath.mpf(tk) / 2 + 1)
        self.tls = list(tls)
        self.tms = list(range(-tk, tk + 1, 2))
        self.vals = {}
        rs = [-mpmath.log(x) for x in xs]
        for tl in self.tls:
            for tm in self.tms:
                dc = dfunc.DClosed(tk, self.rho, tl, tm)
                self.vals[(tl, tm)] = np.array([complex(dc.eval(r, dps)) for r in rs])

    def get(self, tl, tm):
        return self.vals[(tl, tm)]


def node_weights(xs, ws):
    """w_n * (1-x_n^2)^2/(16 pi x_n^3) as float64."""
    return np.array([float(w * quadrature.measure_weight(x)) for x, w in zip(xs, ws)])


def booster(tj, tl, dtabs, wmeas, check_real=1e-12):
    """Booster matrix B[i, k] (float64) for one edge and one virtual-spin tuple.

    tj, tl: four doubled spins each, in the coupling order (a1 a2 | a3 a4) of the edge;
    dtabs: four ``DTable`` objects (faces of the four strands); wmeas: ``node_weights``.
    Returns (B, irange, krange, max|Im B|).
    """
    irng = wigner.pair_range(*tj)
    krng = wigner.pair_range(*tl)
    B = np.zeros((len(irng), len(krng)), dtype=complex)
    T = np.zeros((len(irng), len(krng)))      # sum over m of |term|: the scale of the rounding in B
    ms = [range(-t, t + 1, 2) for t in tj]
    for m1, m2, m3 in itertools.product(*ms[:3]):
        m4 = -(m1 + m2 + m3)
        if abs(m4) > tj[3] or (tj[3] - m4) % 2:
            continue
        mm = (m1, m2, m3, m4)
        integ = np.sum(wmeas * dtabs[0].get(tl[0], m1) * dtabs[1].get(tl[1], m2)
                       * dtabs[2].get(tl[2], m3) * dtabs[3].get(tl[3], m4))
        wj = [float(wigner.fourjm_mp(tj, mm, ti)) for ti in irng]
        wl = [float(wigner.fourjm_mp(tl, mm, tk)) for tk in krng]
        B += np.outer(wj, wl) * integ
        T += np.abs(np.outer(wj, wl)) * abs(integ)
    im = float(np.max(np.abs(B.imag))) if B.size else 0.0
    if check_real is not None and B.size:
        # the imaginary parts of the m and -m terms cancel exactly, so only rounding of the
        # m-sum remains: measured against the sum of |terms| (B itself vanishes identically when
        # the sum of l - j over the four strands is odd, and then only rounding is left in it)
        scale = max(float(np.max(T)), 1e-300)
        if im > check_real * scale:
            raise ArithmeticError("booster is not real: max|Im| / (sum of |terms|) = %g" % (im / scale))
    return B.real.copy(), irng, krng, im


def face_tables(tj, dl, gamma, xs):
    """One ``DTable`` per boundary face: free faces carry l = j..j+dl, gauge faces l = j."""
    from . import vertex
    tabs = {}
    for f, t in zip(vertex.FACES, tj):
        tls = [t] if f in ("12", "13", "14", "15") else [t + 2 * d for d in range(dl + 1)]
        tabs[f] = DTable(t, gamma, tls, xs)
    return tabs


def _edge_faces():
    # the four strands of each edge in coupling order (gauge faces first-index only)
    return {2: ("23", "24", "25", "12"), 3: ("34", "35", "13", "23"),
            4: ("45", "14", "24", "34"), 5: ("15", "25", "35", "45")}


def vertex_boosters(tj, dl, gamma, r_max, n_panels, order, tables=None):
    """All booster matrices of a vertex, in the layout B[e][t][i - i_lo][k - k_lo(t)].

    Returns {e: {'B': float64 [(dl+1)^3, D_i, D_kmax], 'klo': int [(dl+1)^3], 'maxim': float}}.
    """
    from . import vertex
    xs, ws = quadrature.rule_nodes(r_max, n_panels, order)
    wm = node_weights(xs, ws)
    tabs = tables or face_tables(tj, dl, gamma, xs)
    out = {}
    n3 = (dl + 1) ** 3
    for e in (2, 3, 4, 5):
        mats, klos = [], []
        maxim = 0.0
        for t in range(n3):
            d = (t // ((dl + 1) ** 2), (t // (dl + 1)) % (dl + 1), t % (dl + 1))
            tl6 = dict(zip(vertex.FREE, [tj[vertex.FACES.index(f)] for f in vertex.FREE]))
            for f, df in zip(vertex.EDGE_TRIPLES[e], d):
                tl6[f] += 2 * df
            tl = tuple(tl6[f] for f in vertex.FREE)
            bj, bl = vertex.edge_spins(tj, tl)[e]
            krng = wigner.pair_range(*bl)
            if not krng:
                mats.append(None)
                klos.append(0)
                continue
            faces = _edge_faces()[e]
            B, _, _, im = booster(bj, bl, [tabs[f] for f in faces], wm)
            maxim = max(maxim, im)
            mats.append(B)
            klos.append(krng[0])
        di = len(wigner.pair_range(*vertex.edge_spins(tj, tuple(tj[4:]))[e][0]))
        dk = max([m.shape[1] for m in mats if m is not None] + [1])
        arr = np.zeros((n3, di, dk))
        for t, m in enumerate(mats):
            if m is not None:
                arr[t, :, :m.shape[1]] = m
        out[e] = {"B": arr, "klo": np.array(klos, dtype=np.int64), "maxim": maxim}
    return out


def random_boosters(tj, dl, seed):
    """Seeded N(0,1) booster tensors in the layout of ``vertex_boosters``, for contraction tests
    that bypass the quadrature. Entries outside each triple's k range are zero. One generator
    ``default_rng(seed)`` draws the edges in the order 2, 3, 4, 5, each as one block
    [(dl+1)^3, D_i, D_kmax].
    """
    from . import vertex
    rng = np.random.default_rng(seed)
    n3 = (dl + 1) ** 3
    out = {}
    for e in (2, 3, 4, 5):
        kr = []
        for t in range(n3):
            d = (t // ((dl + 1) ** 2), (t // (dl + 1)) % (dl + 1), t % (dl + 1))
            tl6 = dict(zip(vertex.FREE, [tj[vertex.FACES.index(f)] for f in vertex.FREE]))
            for f, df in zip(vertex.EDGE_TRIPLES[e], d):
                tl6[f] += 2 * df
            kr.append(wigner.pair_range(*vertex.edge_spins(tj, tuple(tl6[f] for f in vertex.FREE))[e][1]))
        di = len(wigner.pair_range(*vertex.edge_spins(tj, tuple(tj[4:]))[e][0]))
        dk = max([len(k) for k in kr] + [1])
        B = rng.standard_normal((n3, di, dk))
        for t, k in enumerate(kr):
            B[t, :, len(k):] = 0.0
        out[e] = {"B": B, "klo": np.array([k[0] if k else 0 for k in kr], dtype=np.int64), "maxim": 0.0}
    return out


def identity_boosters(tj):
    """SU(2) BF limit at dl = 0: (2k+1) B_e[i, k] = delta_ik, so A_v = prod sqrt(2i+1) {15j}."""
    from . import vertex
    out = {}
    for e in (2, 3, 4, 5):
        bj, bl = vertex.edge_spins(tj, tuple(tj[4:]))[e]
        rng = wigner.pair_range(*bj)
        B = np.diag([1.0 / (i + 1) for i in rng])[None, :, :]
        out[e] = {"B": B, "klo": np.array([rng[0] if rng else 0], dtype=np.int64), "maxim": 0.0}
    return out
