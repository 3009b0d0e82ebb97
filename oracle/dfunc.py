"""SL(2,C) boost matrix elements d^{rho,k}_{j l m}(r) for the oracle (Sec. 3, eq. francois).

Test infrastructure only: nothing in the product package may import this module.

The paper prints only the structure of these functions (a finite sum of complex exponentials
over a power of (e^r - e^-r)); the coefficients are in a cited work that is not reproduced.
The oracle therefore DEFINES them by the compact-picture integral of the principal-series
representation (rho, k), with the first spin fixed to j = k (Y-map, Sec. 2 below eq. booster):

    d(r) = i^(k-l) * Phi_l * sqrt((2k+1)(2l+1))
           * int_0^1 dt  d^k_{m k}(beta) d^l_{m k}(beta_r) u^(-1+i rho)

    t = sin^2(beta/2),  u = e^-r (1-t) + e^r t,  tan(beta_r/2) = e^r tan(beta/2),
    Phi_l = prod_{n=k+1}^{l} (n - i rho)/|n - i rho|,
    d^j_{m'm}(beta): the textbook Wigner small-d (Edmonds eq. 4.1.23).

The phase Phi_l * i^(k-l) makes the boosters real; every other admissible choice changes A_v
only by per-face factors that appear squared (each free face enters two boosters).

Two evaluations are provided:

* ``d_definition``: the integral above by adaptive mpmath quadrature (slow; the definition).
* ``DClosed``: the same function as the finite exponential sum that eq. francois describes,
  obtained by expanding the integrand in powers of u. With x = e^-r and q = x^2:

      d(r) = K (1-q)^-(k+l+1) [ e^{+i rho r} x^(k+1+m) Q+(q) + e^{-i rho r} x^(k+1-m) Q-(q) ]

  Its coefficients are computed from exact rationals; evaluation is in mpmath at a working
  precision raised with the cancellation factor (1-q)^-(k+l+1), mirroring the paper's use of
  arbitrary precision for this formula. The denominator power is k+l+1 (the printed "j+l+m" is
  read as a typo: with m it would grow at large r for m<0).

Spins are doubled integers throughout: tk = 2k, tl = 2l, tm = 2m.
"""
from fractions import Fraction
from functools import lru_cache
import math

import mpmath


def _f(n):
    return math.factorial(n)


def wigner_small_d_mp(tj, tmp, tm, beta):
    """Textbook Wigner small-d d^j_{m'm}(beta) (Edmonds eq. 4.1.23), doubled spins, mpmath."""
    j_mp = (tj + tmp) // 2
    j_mm = (tj - tmp) // 2
    j_p = (tj + tm) // 2
    j_m = (tj - tm) // 2
    c = mpmath.cos(beta / 2)
    s = mpmath.sin(beta / 2)
    pref = mpmath.sqrt(mpmath.mpf(_f(j_mp) * _f(j_mm) * _f(j_p) * _f(j_m)))
    tot = mpmath.mpf(0)
    dmm = (tmp - tm) // 2                  # m' - m
    for sgm in range(max(0, -dmm), min(j_p, j_mm) + 1):
        den = _f(j_p - sgm) * _f(sgm) * _f(dmm + sgm) * _f(j_mm - sgm)
        term = mpmath.mpf((-1) ** (dmm + sgm)) / den
        pc = j_p + j_mm - 2 * sgm         # 2j + m - m' - 2sigma = (j+m) + (j-m') - 2 sigma
        ps = dmm + 2 * sgm                # m' - m + 2 sigma
        tot += term * c ** pc * s ** ps
    return pref * tot


def phase_phi(tk, tl, rho):
    """Phi_l = prod_{n=k+1}^{l} (n - i rho)/|n - i rho| (spins doubled)."""
    ph = mpmath.mpc(1)
    for tn in range(tk + 2, tl + 1, 2):
        z = mpmath.mpc(mpmath.mpf(tn) / 2, -rho)
        ph *= z / abs(z)
    return ph


def i_power(e):
    """i**e for an integer e."""
    return [mpmath.mpc(1), mpmath.mpc(0, 1), mpmath.mpc(-1), mpmath.mpc(0, -1)][e % 4]


def d_definition(tk, rho, tl, tm, r, dps=30):
    """d^{rho,k}_{k l m}(r) by adaptive quadrature of the defining compact integral (slow)."""
    assert abs(tm) <= tk and (tk - tm) % 2 == 0 and tl >= tk and (tl - tk) % 2 == 0
    with mpmath.workdps(dps + 15):
        rho = mpmath.mpf(rho)
        r = mpmath.mpf(r)
        er, emr = mpmath.exp(r), mpmath.exp(-r)

        def integrand(beta):
            t = mpmath.sin(beta / 2) ** 2
            u = emr * (1 - t) + er * t
            br = 2 * mpmath.atan(er * mpmath.tan(beta / 2)) if beta < mpmath.pi else mpmath.pi
            return (mpmath.sin(beta) / 2 * wigner_small_d_mp(tk, tm, tk, beta)
                    * wigner_small_d_mp(tl, tm, tk, br) * mpmath.power(u, mpmath.mpc(-1, rho)))

        val = mpmath.quad(integrand, mpmath.linspace(0, mpmath.pi, 9))
        pref = i_power((tk - tl) // 2) * phase_phi(tk, tl, rho) * mpmath.sqrt((tk + 1) * (tl + 1))
        return +(pref * val)


class DClosed:
    """Exponential-sum closed form of d^{rho,k}_{k l m}(r) with exactly derived coefficients.

    Derivation (written out so that it can be checked against the definition above):
      d^k_{mk}(beta) d^l_{mk}(beta_r) = sqrt(C(2k,k+m)) sum_s w_s (1-t)^(k+l-s) t^s e^{r(m-k-l+2s)} u^-l
      with w_s the Wigner-d sum coefficients of d^l_{mk}. Substituting 1-t = (e^r-u)/(2 sinh r),
      t = (u-e^-r)/(2 sinh r), dt = du/(2 sinh r), expanding both binomials and integrating
      u^(n-1+i rho) with n = alpha+beta-l gives exponentials e^{r(m+2beta-l+i rho)} (from the upper
      limit) and e^{r(m+l-2alpha-i rho)} (from the lower limit).
    """

    def __init__(self, tk, rho, tl, tm, dps=60):
        assert abs(tm) <= tk and (tk - tm) % 2 == 0 and tl >= tk and (tl - tk) % 2 == 0
        self.tk, self.tl, self.tm = tk, tl, tm
        k2, l2, m2 = tk, tl, tm
        # integer-valued combinations (spins are half-integers but these are integers)
        kpm = (k2 + m2) // 2        # k+m
        kmm = (k2 - m2) // 2        # k-m
        lpm = (l2 + m2) // 2        # l+m
        lmm = (l2 - m2) // 2        # l-m
        lpk = (l2 + k2) // 2        # l+k
        lmk = (l2 - k2) // 2        # l-k
        self.n_plus = lmm           # Q+ has degree l-m in q
        self.n_minus = lpm          # Q- has degree l+m in q
        self.kl1 = lpk + 1          # power of (1-q)
        # rational Wigner-d coefficients w'_s (common sqrt factor pulled into K)
        svals = range(max(0, kmm), min(lpk, lmm) + 1)
        # exact rational coefficient sums, grouped by the 1/sigma denominator n = alpha+beta-l
        # plus family indexed by beta (exponent m+2beta-l), minus family by alpha (exp m+l-2alpha)
        plus = {}   # beta -> {n: Fraction}
        minus = {}  # alpha -> {n: Fraction}
        # the l appearing in n = alpha + beta - l is the (possibly half-integer) spin l; keep 2n
        for s in svals:
            ws = Fraction((-1) ** ((-kmm + s) % 2), _f(lpk - s) * _f(s) * _f(s - kmm) * _f(lmm - s))
            A = lpk - s
            for alpha in range(A + 1):
                ca = math.comb(A, alpha)
                for beta in range(s + 1):
                    c = ws * ca * math.comb(s, beta) * (-1) ** ((alpha + s - beta) % 2)
                    tn = 2 * (alpha + beta) - l2          # 2n
                    plus.setdefault(beta, {}).setdefault(tn, Fraction(0))
                    plus[beta][tn] += c
                    minus.setdefault(alpha, {}).setdefault(tn, Fraction(0))
                    minus[alpha][tn] -= c
        self.plus_rat = plus
        self.minus_rat = minus
        self.rho = rho
        self.lpk, self.lmk, self.lpm, self.lmm, self.kpm, self.kmm = lpk, lmk, lpm, lmm, kpm, kmm
        self._coef_dps = None
        self._build_coeffs(dps)

    def _build_coeffs(self, dps):
        with mpmath.workdps(dps):
            rho = mpmath.mpf(self.rho)
            self.P = {b: mpmath.fsum(mpmath.mpf(v.numerator) / v.denominator / mpmath.mpc(mpmath.mpf(tn) / 2, rho)
                                     for tn, v in d.items() if v != 0)
                      for b, d in self.plus_rat.items()}
            self.M = {a: mpmath.fsum(mpmath.mpf(v.numerator) / v.denominator / mpmath.mpc(mpmath.mpf(tn) / 2, rho)
                                     for tn, v in d.items() if v != 0)
                      for a, d in self.minus_rat.items()}
            common = mpmath.sqrt(mpmath.mpf(_f(self.lpm) * _f(self.lmm) * _f(self.lpk) * _f(self.lmk)))
            ck = mpmath.sqrt(mpmath.mpf(math.comb(self.tk, self.kpm)))
            self.K = (i_power((self.tk - self.tl) // 2) * phase_phi(self.tk, self.tl, rho)
                      * mpmath.sqrt((self.tk + 1) * (self.tl + 1)) * common * ck)
        self._coef_dps = dps

    def raw_terms(self):
        """(exponent in r, sign of i rho in the exponent, coefficient) of the bracketed sum."""
        out = []
        m = mpmath.mpf(self.tm) / 2
        l = mpmath.mpf(self.tl) / 2
        for b, c in self.P.items():
            out.append((m + 2 * b - l, +1, c))
        for a, c in self.M.items():
            out.append((m + l - 2 * a, -1, c))
        return out

    def eval(self, r, dps=30):
        """d(r) to about ``dps`` digits; precision grows with the cancellation at small r."""
        r = mpmath.mpf(r)
        # bits lost to cancellation ~ (k+l+1) log2(1/(2 sinh r)) when 2 sinh r < 1, plus margin
        with mpmath.workdps(20):
            loss = 0
            sh = 2 * mpmath.sinh(r) if r > 0 else mpmath.mpf(0)
            if r == 0:
                loss = 10 ** 6
            elif sh < 1:
                loss = float(self.kl1 * mpmath.log10(1 / sh))
        if r == 0:
            return mpmath.mpc(1 if self.tl == self.tk else 0)
        need = int(dps + loss + 20 + 0.3 * (self.tl + self.tk))
        if self._coef_dps is None or self._coef_dps < need:
            self._build_coeffs(need)
        with mpmath.workdps(need):
            m = mpmath.mpf(self.tm) / 2
            l = mpmath.mpf(self.tl) / 2
            k = mpmath.mpf(self.tk) / 2
            rho = mpmath.mpf(self.rho)
            tot = mpmath.mpc(0)
            eip = mpmath.expj(rho * r)
            eim = mpmath.expj(-rho * r)
            for b, c in self.P.items():
                tot += c * mpmath.exp(r * (m + 2 * b - l)) * eip
            for a, c in self.M.items():
                tot += c * mpmath.exp(r * (m + l - 2 * a)) * eim
            val = self.K * tot / (2 * mpmath.sinh(r)) ** (k + l + 1)
        with mpmath.workdps(dps):
            return +val
