"""Host-side bookkeeping of the shell grid (numpy; no arithmetic of the amplitude itself).

* ``nonempty_shells``: which shells of the (dl+1)^6 grid have all four virtual-intertwiner ranges
  non-empty (the others contribute nothing, Sec. 3 framed algorithm);
* ``canonical_flops``: per shell, the FP64 flop count of the framed algorithm (the {15j} block W by
  its x-sum, then the four booster mode products), the cost model of the shell sum;
* ``group_costs``: the same summed over each (l25, l35, l45) group, the unit of work the shell
  kernel schedules and the unit in which a shell range is split across processes.

Arrays are indexed by the library's group-major linear shell index
s = ((((d25 D + d35) D + d45) D + d24) D + d34) D + d23, D = dl + 1.
"""
import numpy as np

from . import intertwiner_ranges

GAMMA_ANY = 1.0   # the ranges and counts do not depend on gamma


def _pair(a, b, c, d):
    a, b, c, d = np.broadcast_arrays(a, b, c, d)
    lo = np.maximum(np.abs(a - b), np.abs(c - d))
    hi = np.minimum(a + b, c + d)
    n = np.where(((a + b + c + d) % 2 == 0) & (hi >= lo), (hi - lo) // 2 + 1, 0)
    return lo, n


def _shell_axes(tj, dl):
    """The six free-face spins on a broadcast grid, axes (d25, d35, d45, d24, d34, d23): the
    group-major linear shell order of the library, so the flattened grid is indexed by s."""
    D = dl + 1
    d = np.arange(D)
    sh = [1] * 6

    def ax(i):
        s = list(sh)
        s[i] = D
        return d.reshape(s)
    j12, j13, j14, j15, j23, j24, j25, j34, j35, j45 = tj
    return (j25 + 2 * ax(0), j35 + 2 * ax(1), j45 + 2 * ax(2), j24 + 2 * ax(3), j34 + 2 * ax(4), j23 + 2 * ax(5))


def nonempty_shells(tj, dl):
    """Boolean array over the linear shell index: all four k ranges of the shell non-empty."""
    j12, j13, j14, j15 = tj[:4]
    l25, l35, l45, l24, l34, l23 = _shell_axes(tj, dl)
    ok = ((_pair(j15, l25, l35, l45)[1] > 0) & (_pair(l45, j14, l24, l34)[1] > 0)
          & (_pair(l23, l24, l25, j12)[1] > 0) & (_pair(l34, l35, j13, l23)[1] > 0))
    return np.broadcast_to(ok, (dl + 1,) * 6).reshape(-1)


def canonical_flops(tj, dl):
    """Per-shell FP64 flop count of the framed algorithm (W by the x-sum, then four mode products,
    FMA = 2 flops) over the linear shell index; zero for empty shells."""
    lo, dim = intertwiner_ranges(tj, GAMMA_ANY, dl)
    j12, j13, j14, j15 = tj[:4]
    l25, l35, l45, l24, l34, l23 = _shell_axes(tj, dl)
    k5lo, n5 = _pair(j15, l25, l35, l45)
    k4lo, n4 = _pair(l45, j14, l24, l34)
    k2lo, n2 = _pair(l23, l24, l25, j12)
    k3lo, n3 = _pair(l34, l35, j13, l23)
    shape = (dl + 1,) * 6
    i1 = lo[0] + 2 * np.arange(dim[0])

    def count_tri(lo_, n_, a, x):
        # labels k = lo_ + 2c, c < n_, with |k - a| <= x <= k + a and k + a + x even
        c = np.arange(int(np.max(n_)) + 1 if np.size(n_) else 1)
        kk = np.asarray(lo_)[..., None] + 2 * c
        valid = c < np.asarray(n_)[..., None]
        okt = (np.abs(kk - np.asarray(a)[..., None]) <= x) & (x <= kk + np.asarray(a)[..., None]) & \
              ((kk + np.asarray(a)[..., None] + x) % 2 == 0)
        return (valid & okt).sum(axis=-1)
    # the parity of x is that of i1 + l25 (fixed per shell), so only every other x contributes; each
    # count is formed on the small grid of the faces it depends on and broadcast in the product
    xmax = int(2 * max(tj) + 4 * dl + 2)
    w = np.zeros(shape)
    for x in range(0, xmax + 1):
        m1 = ((np.abs(i1[None, :] - np.asarray(l25).reshape(-1, 1)) <= x)
              & (x <= i1[None, :] + np.asarray(l25).reshape(-1, 1))
              & ((i1[None, :] + np.asarray(l25).reshape(-1, 1) + x) % 2 == 0)).sum(axis=1).reshape(np.shape(l25))
        if not m1.any():
            continue
        w += m1 * count_tri(k5lo, n5, j14, x) * count_tri(k4lo, n4, l35, x) * count_tri(k3lo, n3, l24, x) \
            * count_tri(k2lo, n2, j13, x)
    n2, n3, n4, n5 = (np.broadcast_to(v, shape) for v in (n2, n3, n4, n5))
    d1, d2, d3, d4, d5 = dim
    contr = (d1 * d2 * n2 * n3 * n4 * n5 + d1 * d2 * d3 * n3 * n4 * n5 + d1 * d2 * d3 * d4 * n4 * n5
             + d1 * d2 * d3 * d4 * d5 * n5)
    live = (n2 > 0) & (n3 > 0) & (n4 > 0) & (n5 > 0)
    return np.where(live, 2.0 * w + 2.0 * contr, 0.0).reshape(-1)


def group_costs(tj, dl):
    """Canonical flops of each (l25, l35, l45) group: [D^3] in group order g = (d25 D + d35) D + d45."""
    D = dl + 1
    return canonical_flops(tj, dl).reshape(D ** 3, D ** 3).sum(axis=1)
