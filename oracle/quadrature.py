"""Rapidity quadrature rule for the booster integral (Sec. 3 "Booster coefficients").

Test infrastructure only: nothing in the product package may import this module.

The paper maps r to x = e^-r, splits the x-range into n panels whose lengths grow linearly
away from x = 0 (|I_k| = k |I_1|, so |I_1| = 2/(n(n+1)) of the range), and integrates each
panel with a Gauss-type rule. Reading used here (the paper gives neither r_max nor the node
count): the panels cover x in [e^-r_max, 1], each panel carries ``order`` Gauss-Legendre
nodes, and the booster integrand in x is

    sinh(r)^2/(4 pi) dr  ->  (1 - x^2)^2 / (16 pi x^3) dx.

Nodes are computed here in mpmath (Newton iteration on the Legendre three-term recurrence) and
are independent of any other implementation.
"""
import mpmath


def legendre_nodes(n, dps=40):
    """Gauss-Legendre nodes and weights on [-1, 1] to ``dps`` digits (Newton on P_n)."""
    xs, ws = [], []
    with mpmath.workdps(dps + 10):
        for i in range(1, n + 1):
            x = mpmath.cos(mpmath.pi * (i - mpmath.mpf(1) / 4) / (n + mpmath.mpf(1) / 2))
            for _ in range(100):
                p0, p1 = mpmath.mpf(1), x
                for kk in range(2, n + 1):
                    p0, p1 = p1, ((2 * kk - 1) * x * p1 - (kk - 1) * p0) / kk
                dp = n * (x * p1 - p0) / (x * x - 1)
                dx = p1 / dp
                x -= dx
                if abs(dx) < mpmath.mpf(10) ** (-(dps + 8)):
                    break
            p0, p1 = mpmath.mpf(1), x
            for kk in range(2, n + 1):
                p0, p1 = p1, ((2 * kk - 1) * x * p1 - (kk - 1) * p0) / kk
            dp = n * (x * p1 - p0) / (x * x - 1)
            xs.append(x)
            ws.append(2 / ((1 - x * x) * dp * dp))
    return xs, ws


def rule_nodes(r_max, n_panels, order, dps=40):
    """Nodes x_n (ascending panels) and weights of the booster rule on [e^-r_max, 1].

    Panel k (k = 1..n_panels) spans [x0 + D k(k-1)/2, x0 + D k(k+1)/2] with
    D = 2 (1 - x0) / (n_panels (n_panels + 1)) and x0 = e^-r_max.
    Returns mpmath lists (x, w) of length n_panels * order.
    """
    gx, gw = legendre_nodes(order, dps)
    X, W = [], []
    with mpmath.workdps(dps + 10):
        x0 = mpmath.exp(-mpmath.mpf(r_max))
        D = 2 * (1 - x0) / (n_panels * (n_panels + 1))
        for k in range(1, n_panels + 1):
            a = x0 + D * k * (k - 1) / 2
            b = x0 + D * k * (k + 1) / 2
            h = (b - a) / 2
            for xi, wi in zip(gx, gw):
                X.append(a + h * (xi + 1))
                W.append(h * wi)
    return X, W


def measure_weight(x):
    """(1 - x^2)^2 / (16 pi x^3): the booster measure sinh^2(r)/(4 pi) dr written in x = e^-r."""
    return (1 - x * x) ** 2 / (16 * mpmath.pi * x ** 3)
