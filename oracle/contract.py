"""Boundary-contracted vertex amplitude and its gradients, for the oracle.

Test infrastructure only: nothing in the product package may import this module.

The paper contracts vertex tensors with boundary intertwiner vectors (Sec. 3 "Usage",
``contract(v, cs...)``; Sec. 3 GPU contraction benchmark):

    a = sum_{i1..i5} A[i1,i2,i3,i4,i5] psi_1[i1] psi_2[i2] psi_3[i3] psi_4[i4] psi_5[i5]

a is multilinear in the psi_e and in each booster matrix, so its holomorphic derivatives are
plain partial contractions (no conjugates). The gradient with respect to a booster entry
B_e[t][i, k] sums, over every shell whose edge-e triple is t, the shell's {15j} block
contracted with every other factor.
"""
import numpy as np

from . import vertex


def contract_full(A, psis):
    """a from the full tensor."""
    return np.einsum("abcde,a,b,c,d,e->", A, *psis)


def grad_psi_full(A, psis):
    """d a / d psi_e from the full tensor (holomorphic derivatives)."""
    subs = "abcde"
    out = []
    for e in range(5):
        ops = [psis[f] for f in range(5) if f != e]
        spec = ",".join(subs[f] for f in range(5) if f != e)
        out.append(np.einsum("abcde," + spec + "->" + subs[e], A, *ops))
    return out


def contract_by_shell(tj, dl, boosters, psis, shells=None, sixj=None):
    """(a, [d a/d psi_e], {e: d a/d B_e}) by direct per-shell summation.

    d a/d B_e has the booster layout [(dl+1)^3, D_i, D_kmax] (entries of padded k are zero).
    """
    sixj = sixj or vertex.SixJCache()
    I = vertex.intertwiner_ranges(tj)
    sq = [np.sqrt(np.array(r, dtype=float) + 1) for r in I]
    ph = [psis[e] * sq[e] for e in range(5)]          # sqrt(2i+1) psi_e[i]
    a = 0j
    gpsi = [np.zeros(len(r), dtype=complex) for r in I]
    gB = {e: np.zeros(boosters[e]["B"].shape, dtype=complex) for e in (2, 3, 4, 5)}
    for s in (range(vertex.n_shells(dl)) if shells is None else shells):
        tl = vertex.shell_spins(tj, dl, int(s))
        res = vertex.shell_W(tj, tl, sixj)
        if res is None:
            continue
        W, I1, Ks = res
        Bw, ts, k0s = [], [], []
        for e, K in zip((2, 3, 4, 5), Ks):
            t = vertex.triple_index(tj, dl, e, tl)
            b = boosters[e]
            k0 = (K[0] - b["klo"][t]) // 2
            Bw.append(b["B"][t][:, k0:k0 + len(K)] * np.array([k + 1 for k in K], dtype=float)[None, :])
            ts.append(t)
            k0s.append(k0)
        # phi_e[k] = sum_i sqrt(2i+1) psi_e[i] (2k+1) B_e[i,k]
        phi = [ph[0]] + [ph[e + 1] @ Bw[e] for e in range(4)]
        a += np.einsum("abcde,a,b,c,d,e->", W, *phi)
        subs = "abcde"
        for e in range(5):
            ops = [phi[f] for f in range(5) if f != e]
            spec = ",".join(subs[f] for f in range(5) if f != e)
            G = np.einsum("abcde," + spec + "->" + subs[e], W, *ops)   # d a_s / d phi_e
            if e == 0:
                gpsi[0] += sq[0] * G
            else:
                be = Bw[e - 1]
                gpsi[e] += sq[e] * (be @ G)
                K = Ks[e - 1]
                kw = np.array([k + 1 for k in K], dtype=float)
                gB[e + 1][ts[e - 1]][:, k0s[e - 1]:k0s[e - 1] + len(K)] += np.outer(ph[e], kw * G)
    return a, gpsi, gB
