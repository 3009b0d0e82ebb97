// Exact Wigner symbols on the device.
//
// The paper evaluates {6j} and 3j symbols exactly (Sec. 3, the Wigner-symbol library of
// Johansson and Forssen): integer Racah sums, then one rounding. Here each Racah term is an
// integer that is carried from one term to the next by an exact multiply/divide with small
// integers (hypergeometric term ratio), the alternating sum is formed exactly in BigU, and the
// square root of the factorial prefactor is taken in double-double; the result is rounded once.
#pragma once
#include "sf_internal.cuh"

// n! as a double-double from the table F (F[n], n <= SF_FACT_MAX)
__device__ inline dd sf_fact(const dd* F, int n) { return F[n]; }

// sqrt((x+y-z)!(x-y+z)!(-x+y+z)! / (x+y+z+1)!) for doubled x, y, z
__device__ inline dd sf_delta(const dd* F, int x, int y, int z) {
    dd num = dd_mul(dd_mul(F[(x + y - z) / 2], F[(x - y + z) / 2]), F[(-x + y + z) / 2]);
    return dd_sqrt(dd_div(num, F[(x + y + z) / 2 + 1]));
}

// Triangle coefficients sf_delta(x, y, z) of every triad of doubled spins up to m, tabulated once
// (x, y, z in [0, m]; zero where the triad fails): each {6j} takes four of them.
struct TriTable {
    const dd* d;
    int m1;   // m + 1
    __device__ dd at(int x, int y, int z) const { return d[((int64_t)x * m1 + y) * m1 + z]; }
};

// flush an accumulated numerator/denominator pair into t (exact: t*num/den is an integer)
template <int NL> __device__ inline void sf_muldiv(BigUT<NL>& t, uint32_t num, uint32_t den, uint32_t& ovf) {
    ovf |= bi_mul(t, num);
    if (den > 1u) bi_divexact(t, den);
}

// The exact alternating Racah sum of {a b c; d e f} for z in [zmin, zmax], times the four
// triangle coefficients, rounded once; NL limbs hold every term (see sf_sixj).
template <int NL>
__device__ inline double sf_sixj_sum(int ta, int tb, int tc, int td, int te, int tf, int zmin, int zmax, const int a[4],
                                     const int b[3], const TriTable& tt, int* status) {
    uint32_t ovf = 0;
    // first term (zmin+1)! / prod of seven factorials whose arguments sum to zmin:
    // (zmin+1) times a multinomial, built one exact factor at a time
    BigUT<NL> t;
    bi_set(t, 1u);
    {
        const int n7[7] = {zmin - a[0], zmin - a[1], zmin - a[2], zmin - a[3], b[0] - zmin, b[1] - zmin, b[2] - zmin};
        uint32_t num = 1u, den = 1u;
        int m = 0;
        for (int i = 0; i < 7; i++) {
            for (int k = 1; k <= n7[i]; k++) {
                m++;
                if ((uint64_t)num * (uint64_t)m > 0xFFFFFFFFull || (uint64_t)den * (uint64_t)k > 0xFFFFFFFFull) {
                    sf_muldiv(t, num, den, ovf);
                    num = 1u;
                    den = 1u;
                }
                num *= (uint32_t)m;
                den *= (uint32_t)k;
            }
        }
        sf_muldiv(t, num, den, ovf);
        ovf |= bi_mul(t, (uint32_t)(zmin + 1));
    }
    BigUT<NL> pos, neg;
    bi_zero(pos);
    bi_zero(neg);
    for (int z = zmin; z <= zmax; z++) {
        if (z & 1) ovf |= bi_add(neg, t); else ovf |= bi_add(pos, t);
        if (z == zmax) break;
        // term ratio t_{z+1}/t_z = (z+2)(b1-z)(b2-z)(b3-z) / ((z+1-a1)(z+1-a2)(z+1-a3)(z+1-a4))
        uint32_t num = (uint32_t)(z + 2) * (uint32_t)(b[0] - z) * (uint32_t)(b[1] - z) * (uint32_t)(b[2] - z);
        uint32_t den = (uint32_t)(z + 1 - a[0]) * (uint32_t)(z + 1 - a[1]) * (uint32_t)(z + 1 - a[2]) * (uint32_t)(z + 1 - a[3]);
        sf_muldiv(t, num, den, ovf);
    }
    if (ovf && status) atomicCAS(status, SF_DEV_OK, SF_DEV_BIGINT_OVERFLOW);
    int c = bi_cmp(pos, neg);
    if (c == 0) return 0.0;
    dd S;
    if (c > 0) { bi_sub(pos, neg); S = bi_to_dd(pos); }
    else { bi_sub(neg, pos); S = dd_neg(bi_to_dd(neg)); }
    S = dd_mul(S, tt.at(ta, tb, tc));
    S = dd_mul(S, tt.at(ta, te, tf));
    S = dd_mul(S, tt.at(td, tb, tf));
    S = dd_mul(S, tt.at(td, te, tc));
    return dd_to_d(S);
}

// {a b c; d e f}, doubled spins. Racah's single sum (Edmonds eq. 6.3.7). The term of index z is
// (z+1) times a multinomial coefficient of z into seven parts, so it is below (z+1) 7^z; with
// 32 bits of headroom for the exact multiply-then-divide steps, 8, 16 or 24 limbs are chosen
// from that bound at zmax (8 limbs up to zmax = 76, 16 up to 167).
__device__ inline double sf_sixj(int ta, int tb, int tc, int td, int te, int tf, const TriTable& tt, int* status) {
    if (!(sf_tri(ta, tb, tc) && sf_tri(ta, te, tf) && sf_tri(td, tb, tf) && sf_tri(td, te, tc))) return 0.0;
    const int a[4] = {(ta + tb + tc) / 2, (ta + te + tf) / 2, (td + tb + tf) / 2, (td + te + tc) / 2};
    const int b[3] = {(ta + tb + td + te) / 2, (ta + tc + td + tf) / 2, (tb + tc + te + tf) / 2};
    const int zmin = imax_(imax_(a[0], a[1]), imax_(a[2], a[3]));
    const int zmax = imin_(imin_(b[0], b[1]), b[2]);
    if (zmin > zmax) return 0.0;
    const float bits = log2f((float)(zmax + 2)) + 2.8074f * (float)zmax + 34.0f;   // log2 7 = 2.8074
    if (bits <= 256.0f) return sf_sixj_sum<8>(ta, tb, tc, td, te, tf, zmin, zmax, a, b, tt, status);
    if (bits <= 512.0f) return sf_sixj_sum<16>(ta, tb, tc, td, te, tf, zmin, zmax, a, b, tt, status);
    return sf_sixj_sum<SF_BI_LIMBS>(ta, tb, tc, td, te, tf, zmin, zmax, a, b, tt, status);
}

// C(n, k) multiplied into t exactly (k steps of *(n-k+i)/i, batched)
__device__ inline void sf_mul_binom(BigU& t, int n, int k, uint32_t& ovf) {
    uint32_t num = 1u, den = 1u;
    for (int i = 1; i <= k; i++) {
        uint32_t f = (uint32_t)(n - k + i);
        if ((uint64_t)num * f > 0xFFFFFFFFull || (uint64_t)den * (uint64_t)i > 0xFFFFFFFFull) {
            sf_muldiv(t, num, den, ovf);
            num = 1u;
            den = 1u;
        }
        num *= f;
        den *= (uint32_t)i;
    }
    sf_muldiv(t, num, den, ovf);
}

// (j1 j2 j3; m1 m2 m3) as double-double, doubled arguments. Racah's formula (Edmonds eq. 3.7.3)
// rewritten as an alternating sum of products of three binomials:
//   3j = (-1)^(j1-j2-m3) sqrt( prod (j+-m)! / (J! P! Q! (j1+j2+j3+1)!) ) sum_t (-1)^t C(J,t) C(P,A-t) C(Q,B-t)
//   J = j1+j2-j3, P = j1-j2+j3, Q = -j1+j2+j3, A = j1-m1, B = j2+m2.
__device__ inline dd sf_threej_dd(int t1, int t2, int t3, int tm1, int tm2, int tm3, const dd* F, int* status) {
    dd zero{0.0, 0.0};
    if (tm1 + tm2 + tm3 != 0) return zero;
    if (!sf_tri(t1, t2, t3)) return zero;
    if (iabs_(tm1) > t1 || iabs_(tm2) > t2 || iabs_(tm3) > t3) return zero;
    if (((t1 + tm1) & 1) || ((t2 + tm2) & 1) || ((t3 + tm3) & 1)) return zero;
    const int J = (t1 + t2 - t3) / 2, P = (t1 - t2 + t3) / 2, Q = (-t1 + t2 + t3) / 2;
    const int A = (t1 - tm1) / 2, B = (t2 + tm2) / 2;
    const int k1 = (t3 - t2 + tm1) / 2, k2 = (t3 - t1 - tm2) / 2;
    const int tmin = imax_(0, imax_(-k1, -k2));
    const int tmax = imin_(J, imin_(A, B));
    if (tmin > tmax) return zero;
    uint32_t ovf = 0;
    BigU t;
    bi_set(t, 1u);
    sf_mul_binom(t, J, tmin, ovf);
    sf_mul_binom(t, P, A - tmin, ovf);
    sf_mul_binom(t, Q, B - tmin, ovf);
    BigU pos, neg;
    bi_zero(pos);
    bi_zero(neg);
    for (int s = tmin; s <= tmax; s++) {
        if (s & 1) ovf |= bi_add(neg, t); else ovf |= bi_add(pos, t);
        if (s == tmax) break;
        uint32_t num = (uint32_t)(J - s) * (uint32_t)(A - s) * (uint32_t)(B - s);
        uint32_t den = (uint32_t)(s + 1) * (uint32_t)(k1 + s + 1) * (uint32_t)(k2 + s + 1);
        sf_muldiv(t, num, den, ovf);
    }
    if (ovf && status) atomicCAS(status, SF_DEV_OK, SF_DEV_BIGINT_OVERFLOW);
    int c = bi_cmp(pos, neg);
    if (c == 0) return zero;
    dd S;
    if (c > 0) { bi_sub(pos, neg); S = bi_to_dd(pos); }
    else { bi_sub(neg, pos); S = dd_neg(bi_to_dd(neg)); }
    dd num = dd_mul(dd_mul(F[(t1 + tm1) / 2], F[(t1 - tm1) / 2]), dd_mul(F[(t2 + tm2) / 2], F[(t2 - tm2) / 2]));
    num = dd_mul(num, dd_mul(F[(t3 + tm3) / 2], F[(t3 - tm3) / 2]));
    dd den = dd_mul(dd_mul(F[J], F[P]), dd_mul(F[Q], F[(t1 + t2 + t3) / 2 + 1]));
    S = dd_mul(S, dd_sqrt(dd_div(num, den)));
    if (((t1 - t2 - tm3) / 2) & 1) S = dd_neg(S);
    return S;
}
