// Boundary-contracted vertex amplitude and its adjoint, recomputing every shell's {15j} ring.
//
//   a = sum_i A[i1..i5] psi_1[i1] ... psi_5[i5]
//     = sum_shells sigma_s sum_x (2x+1) tr(W1 S1 W5 S2 W4 S3 W3 S4 W2 S5)
//
// with the ring of the five {6j} of eq. 15j read as matrices S1[i1,k5], S2[k5,k4], S3[k4,k3],
// S4[k3,k2], S5[k2,i1] at fixed x, and diagonal weights on its nodes:
//   W1[i1] = (-1)^(i1-i1lo) sqrt(2 i1 + 1) psi_1[i1],
//   We[k]  = (-1)^(k-klo) sum_i sqrt(2i+1) psi_e[i] (2k+1) B_e[t_e(shell)][i][k]   (e = 2..5).
// The derivative of the trace with respect to one node's weight is the diagonal of the ring
// product with that weight removed, from prefix and suffix products. Per shell the kernel
// stores a_s and the five node derivatives; fixed-order reductions then give a, d a/d psi_e and
// d a/d B_e (the {15j} block is never stored).
#include "sf_internal.cuh"

#define SF_ADJ_DMAX 12          // largest node dimension handled by one warp
#define SF_ADJ_WARPS 4

struct cplx { double x, y; };
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return cplx{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cplx cfma(cplx a, cplx b, cplx c) {
    return cplx{fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}

__device__ __forceinline__ double s6a(const double* __restrict__ S, const SlotDesc* sp, int a, int b, int x) {
    const SlotDesc sd = *sp;
    const int da = a - sd.alo, db = b - sd.blo, dx = x - sd.xlo;
    if (((da | db | dx) & 1) != 0) return 0.0;
    const int ia = da >> 1, ib = db >> 1, ix = dx >> 1;
    if ((unsigned)ia >= (unsigned)sd.na || (unsigned)ib >= (unsigned)sd.nb || (unsigned)ix >= (unsigned)sd.nx) return 0.0;
    return __ldg(S + sd.off + ((int64_t)ia * sd.nb + ib) * sd.nx + ix);
}

// C[r][c] = sum_m A[r][m] B[m][c] for dims (nr x nm) (nm x nc), all row-major with stride DM
__device__ __forceinline__ void wmat(int DM, int nr, int nm, int nc, const cplx* A, const cplx* B, cplx* C, int lane) {
    for (int q = lane; q < nr * nc; q += 32) {
        const int r = q / nc, c = q % nc;
        cplx acc{0.0, 0.0};
        for (int m = 0; m < nm; m++) acc = cfma(A[r * DM + m], B[m * DM + c], acc);
        C[r * DM + c] = acc;
    }
    __syncwarp();
}

// per shell: out[0] = a_s; then derivatives w.r.t. the node weights in the order
// i1 (n1), k5 (n5), k4 (n4), k3 (n3), k2 (n2), each padded to `stride_node` entries
// shared memory per warp: 14 matrices DM x DM, node weights [5][DM], derivative sums [5][DM]
__global__ void __launch_bounds__(32 * SF_ADJ_WARPS) k_adjoint_shell(const VtxDev* __restrict__ vp, const cplx* __restrict__ phi1,
                                                                       const cplx* __restrict__ psi_all, int64_t nshell,
                                                                       int stride_node, int DM, int want_nodes,
                                                                       cplx* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char adj_smem[];
    const VtxDev& v = *vp;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int D = v.D;
    const int j12 = v.tj[F12], j13 = v.tj[F13], j14 = v.tj[F14], j15 = v.tj[F15];
    cplx* wbase = reinterpret_cast<cplx*>(adj_smem) + (size_t)warp * (14 * DM * DM + 10 * DM);
    cplx* M[14];
    for (int q = 0; q < 14; q++) M[q] = wbase + q * DM * DM;
    cplx* swp = wbase + 14 * DM * DM;          // node weights [5][DM]
    cplx* sdp = swp + 5 * DM;                  // derivative accumulators [5][DM]
    const int64_t gw = (int64_t)blockIdx.x * SF_ADJ_WARPS + warp, nw = (int64_t)gridDim.x * SF_ADJ_WARPS;
    const int n1 = v.di[0], i1lo = v.ilo[0];
    for (int64_t s = gw; s < nshell; s += nw) {
        const int d23 = (int)(s % D), d34 = (int)((s / D) % D), d24 = (int)((s / (D * D)) % D);
        const int d45 = (int)((s / ((int64_t)D * D * D)) % D), d35 = (int)((s / ((int64_t)D * D * D * D)) % D);
        const int d25 = (int)(s / ((int64_t)D * D * D * D * D));
        const int l23 = v.tj[F23] + 2 * d23, l24 = v.tj[F24] + 2 * d24, l25 = v.tj[F25] + 2 * d25;
        const int l34 = v.tj[F34] + 2 * d34, l35 = v.tj[F35] + 2 * d35, l45 = v.tj[F45] + 2 * d45;
        int k2lo, nk2, k3lo, nk3, k4lo, nk4, k5lo, nk5;
        sf_pair_range(l23, l24, l25, j12, &k2lo, &nk2);
        sf_pair_range(l34, l35, j13, l23, &k3lo, &nk3);
        sf_pair_range(l45, j14, l24, l34, &k4lo, &nk4);
        sf_pair_range(j15, l25, l35, l45, &k5lo, &nk5);
        cplx* o = out + s * (1 + 5 * (int64_t)stride_node);
        if (nk2 == 0 || nk3 == 0 || nk4 == 0 || nk5 == 0) {
            for (int q = lane; q < 1 + 5 * stride_node; q += 32) o[q] = cplx{0.0, 0.0};
            __syncwarp();
            continue;
        }
        const int t2 = (d23 * D + d24) * D + d25, t3 = (d34 * D + d35) * D + d23;
        const int t4 = (d45 * D + d24) * D + d34, t5 = (d25 * D + d35) * D + d45;
        const int tt[4] = {t2, t3, t4, t5};
        const int klo_e[4] = {k2lo, k3lo, k4lo, k5lo}, nk_e[4] = {nk2, nk3, nk4, nk5};
        // node weights: sw[0] = W1 (i1); sw[1..4] = W5, W4, W3, W2 (ring order k5, k4, k3, k2)
        for (int q = lane; q < n1; q += 32) swp[q] = phi1[q];
        for (int e = 0; e < 4; e++) {
            const int node = 4 - e;   // e=0 (edge 2, k2) -> node 4; e=3 (edge 5, k5) -> node 1
            const int di = v.di[e + 1], ilo = v.ilo[e + 1];
            const double* B = v.B[e] + (int64_t)tt[e] * di * v.dkmax[e];
            const cplx* ps = psi_all + 32 * (e + 1);
            for (int c = lane; c < nk_e[e]; c += 32) {
                cplx acc{0.0, 0.0};
                for (int i = 0; i < di; i++) {
                    const double f = sqrt((double)(ilo + 2 * i + 1)) * B[i * v.dkmax[e] + c];
                    acc.x = fma(f, ps[i].x, acc.x);
                    acc.y = fma(f, ps[i].y, acc.y);
                }
                const double g = (double)(klo_e[e] + 2 * c + 1) * ((c & 1) ? -1.0 : 1.0);
                swp[node * DM + c] = cplx{g * acc.x, g * acc.y};
            }
        }
        for (int q = lane; q < 5 * DM; q += 32) sdp[q] = cplx{0.0, 0.0};
        __syncwarp();
        // node dims in ring order: n1 (i1), nk5, nk4, nk3, nk2; node labels' lows
        const int nd[5] = {n1, nk5, nk4, nk3, nk2};
        const int E2 = j12 + j13 + j14 + j15 + i1lo + k2lo + k3lo + k4lo + k5lo + l23 + l24 + l25 + l34 + l35 + l45;
        const double sig = ((E2 >> 1) & 1) ? -1.0 : 1.0;
        // x range from i1 with l25 and k2 with j13
        const int i1hi = i1lo + 2 * (n1 - 1), k2hi = k2lo + 2 * (nk2 - 1);
        int xlo = imax_(i1lo > l25 ? i1lo - l25 : (l25 > i1hi ? l25 - i1hi : ((l25 + i1lo) & 1)),
                        k2lo > j13 ? k2lo - j13 : (j13 > k2hi ? j13 - k2hi : ((j13 + k2lo) & 1)));
        const int xhi = imin_(i1hi + l25, k2hi + j13);
        if (((xlo + i1lo + l25) & 1) != 0) xlo++;
        const SlotDesc* sp1 = v.slot[0] + d25;
        const SlotDesc* sp2 = v.slot[1] + d35 * D + d45;
        const SlotDesc* sp3 = v.slot[2] + (d24 * D + d34) * D + d35;
        const SlotDesc* sp4 = v.slot[3] + d23 * D + d24;
        const SlotDesc* sp5 = v.slot[4] + d25;
        cplx aval{0.0, 0.0};
        for (int x = xlo; x <= xhi; x += 2) {
            // links L1..L5 (stored in M[5..9]) and M_n = W_n L_n (stored in M[0..4])
            for (int q = lane; q < n1 * nk5; q += 32) {
                const int r = q / nk5, c = q % nk5;
                M[5][r * DM + c] = cplx{s6a(v.S[0], sp1, i1lo + 2 * r, k5lo + 2 * c, x), 0.0};
            }
            for (int q = lane; q < nk5 * nk4; q += 32) {
                const int r = q / nk4, c = q % nk4;
                M[6][r * DM + c] = cplx{s6a(v.S[1], sp2, k5lo + 2 * r, k4lo + 2 * c, x), 0.0};
            }
            for (int q = lane; q < nk4 * nk3; q += 32) {
                const int r = q / nk3, c = q % nk3;
                M[7][r * DM + c] = cplx{s6a(v.S[2], sp3, k4lo + 2 * r, k3lo + 2 * c, x), 0.0};
            }
            for (int q = lane; q < nk3 * nk2; q += 32) {
                const int r = q / nk2, c = q % nk2;
                M[8][r * DM + c] = cplx{s6a(v.S[3], sp4, k3lo + 2 * r, k2lo + 2 * c, x), 0.0};
            }
            for (int q = lane; q < nk2 * n1; q += 32) {
                const int r = q / n1, c = q % n1;
                M[9][r * DM + c] = cplx{s6a(v.S[4], sp5, k2lo + 2 * r, i1lo + 2 * c, x), 0.0};
            }
            __syncwarp();
            for (int n = 0; n < 5; n++) {
                const int nr = nd[n], nc = nd[(n + 1) % 5];
                for (int q = lane; q < nr * nc; q += 32) {
                    const int r = q / nc, c = q % nc;
                    M[n][r * DM + c] = cmul(swp[n * DM + r], M[5 + n][r * DM + c]);
                }
            }
            __syncwarp();
            // prefixes P1 = M0, P2 = P1 M1, P3 = P2 M2, P4 = P3 M3  -> M[10], M[11], M[12] (P2..P4)
            wmat(DM, nd[0], nd[1], nd[2], M[0], M[1], M[10], lane);
            wmat(DM, nd[0], nd[2], nd[3], M[10], M[2], M[11], lane);
            wmat(DM, nd[0], nd[3], nd[4], M[11], M[3], M[12], lane);
            if (!want_nodes) {
                // the amplitude alone: a_x = tr(P4 M4) = sum_c sum_r P4[c][r] M4[r][c]
                const double wx = sig * (double)(x + 1);
                cplx part{0.0, 0.0};
                for (int c = lane; c < nd[0]; c += 32) {
                    cplx acc{0.0, 0.0};
                    for (int r = 0; r < nd[4]; r++) acc = cfma(M[12][c * DM + r], M[4][r * DM + c], acc);
                    part.x += wx * acc.x;
                    part.y += wx * acc.y;
                }
                for (int off = 16; off > 0; off >>= 1) {
                    part.x += __shfl_xor_sync(0xffffffffu, part.x, off);
                    part.y += __shfl_xor_sync(0xffffffffu, part.y, off);
                }
                aval.x += part.x;
                aval.y += part.y;
                __syncwarp();
                continue;
            }
            // suffixes without the starting node's weight: R4 = L4 (node 4 -> node 0);
            // R3 = L3 M4, R2 = L2 M3 M4, R1 = L1 M2 M3 M4, R0 = L0 M1 M2 M3 M4. Q = M_n R_{n} reused.
            // R4 in M[9]; Q4 = M[4] (= W4 L4). R3 = L3 Q4 -> M[13]
            wmat(DM, nd[3], nd[4], nd[0], M[8], M[4], M[13], lane);
            const double wx = sig * (double)(x + 1);
            // node 4 (k2): d[c] = sum_r R4[c][r] P4[r][c];  node 3 (k3): R3 and P3
            for (int c = lane; c < nd[4]; c += 32) {
                cplx acc{0.0, 0.0};
                for (int r = 0; r < nd[0]; r++) acc = cfma(M[9][c * DM + r], M[12][r * DM + c], acc);
                sdp[4 * DM + c].x += wx * acc.x;
                sdp[4 * DM + c].y += wx * acc.y;
            }
            for (int c = lane; c < nd[3]; c += 32) {
                cplx acc{0.0, 0.0};
                for (int r = 0; r < nd[0]; r++) acc = cfma(M[13][c * DM + r], M[11][r * DM + c], acc);
                sdp[3 * DM + c].x += wx * acc.x;
                sdp[3 * DM + c].y += wx * acc.y;
            }
            __syncwarp();
            // Q3 = W3 R3 (rows node 3) -> reuse M[12] (P4 no longer needed); R2 = L2 Q3 -> M[9]
            for (int q = lane; q < nd[3] * nd[0]; q += 32) {
                const int r = q / nd[0], c = q % nd[0];
                M[12][r * DM + c] = cmul(swp[3 * DM + r], M[13][r * DM + c]);
            }
            __syncwarp();
            wmat(DM, nd[2], nd[3], nd[0], M[7], M[12], M[9], lane);
            for (int c = lane; c < nd[2]; c += 32) {
                cplx acc{0.0, 0.0};
                for (int r = 0; r < nd[0]; r++) acc = cfma(M[9][c * DM + r], M[10][r * DM + c], acc);
                sdp[2 * DM + c].x += wx * acc.x;
                sdp[2 * DM + c].y += wx * acc.y;
            }
            __syncwarp();
            // Q2 = W2 R2 -> M[13]; R1 = L1 Q2 -> M[12]
            for (int q = lane; q < nd[2] * nd[0]; q += 32) {
                const int r = q / nd[0], c = q % nd[0];
                M[13][r * DM + c] = cmul(swp[2 * DM + r], M[9][r * DM + c]);
            }
            __syncwarp();
            wmat(DM, nd[1], nd[2], nd[0], M[6], M[13], M[12], lane);
            for (int c = lane; c < nd[1]; c += 32) {
                cplx acc{0.0, 0.0};
                for (int r = 0; r < nd[0]; r++) acc = cfma(M[12][c * DM + r], M[0][r * DM + c], acc);
                sdp[1 * DM + c].x += wx * acc.x;
                sdp[1 * DM + c].y += wx * acc.y;
            }
            __syncwarp();
            // Q1 = W1 R1 -> M[9]; R0 = L0 Q1 -> M[13]; node 0 derivative = diag(R0); a_x = sum_c W0[c] R0[c][c]
            for (int q = lane; q < nd[1] * nd[0]; q += 32) {
                const int r = q / nd[0], c = q % nd[0];
                M[9][r * DM + c] = cmul(swp[DM + r], M[12][r * DM + c]);
            }
            __syncwarp();
            wmat(DM, nd[0], nd[1], nd[0], M[5], M[9], M[13], lane);
            cplx part{0.0, 0.0};
            for (int c = lane; c < nd[0]; c += 32) {
                const cplx dg = M[13][c * DM + c];
                sdp[c].x += wx * dg.x;
                sdp[c].y += wx * dg.y;
                const cplx t = cmul(swp[c], dg);
                part.x += wx * t.x;
                part.y += wx * t.y;
            }
            for (int off = 16; off > 0; off >>= 1) {
                part.x += __shfl_xor_sync(0xffffffffu, part.x, off);
                part.y += __shfl_xor_sync(0xffffffffu, part.y, off);
            }
            aval.x += part.x;
            aval.y += part.y;
            __syncwarp();
        }
        if (lane == 0) o[0] = aval;
        if (want_nodes)
            for (int n = 0; n < 5; n++)
            for (int c = lane; c < stride_node; c += 32)
                o[1 + n * stride_node + c] = (c < nd[n]) ? sdp[n * DM + c] : cplx{0.0, 0.0};
        __syncwarp();
    }
}

// per (edge, triple): G[c] = sum over the triple's shells of the node derivative; then
// gB[t][i][c] = sqrt(2i+1) psi[i] (2k+1) (-1)^c G[c] and P[t][i] = sum_c sqrt(2i+1)(2k+1) B[t][i][c] (-1)^c G[c]
__global__ void k_adjoint_triples(const VtxDev* __restrict__ vp, int edge, const cplx* __restrict__ psi_all,
                                  const cplx* __restrict__ shell_out, int stride_node, cplx* __restrict__ gB,
                                  cplx* __restrict__ Ppsi) {
    const VtxDev& v = *vp;
    const int e = edge - 2;
    const int D = v.D;
    const int t = blockIdx.x;
    const int a = t / (D * D), b = (t / D) % D, c3 = t % D;   // triple offsets in the edge's argument order
    const int node = 4 - e;                                   // derivative slot of this edge's k
    const int di = v.di[e + 1], ilo = v.ilo[e + 1], dk = v.dkmax[e];
    int klo, nk;
    {
        // virtual spins of this edge's triple (same as the booster tables)
        const int F[4][3] = {{F23, F24, F25}, {F34, F35, F23}, {F45, F24, F34}, {F25, F35, F45}};
        const int la = v.tj[F[e][0]] + 2 * a, lb = v.tj[F[e][1]] + 2 * b, lc = v.tj[F[e][2]] + 2 * c3;
        if (e == 0) sf_pair_range(la, lb, lc, v.tj[F12], &klo, &nk);
        else if (e == 1) sf_pair_range(la, lb, v.tj[F13], lc, &klo, &nk);
        else if (e == 2) sf_pair_range(la, v.tj[F14], lb, lc, &klo, &nk);
        else sf_pair_range(v.tj[F15], la, lb, lc, &klo, &nk);
    }
    __shared__ cplx G[64];
    for (int q = threadIdx.x; q < dk; q += blockDim.x) {
        cplx acc{0.0, 0.0};
        if (q < nk) {
            // shells containing the triple: loop over the three other free offsets in a fixed order
            for (int u = 0; u < D; u++)
                for (int w = 0; w < D; w++)
                    for (int z = 0; z < D; z++) {
                        int d23, d24, d25, d34, d35, d45;
                        if (e == 0) { d23 = a; d24 = b; d25 = c3; d34 = u; d35 = w; d45 = z; }
                        else if (e == 1) { d34 = a; d35 = b; d23 = c3; d24 = u; d25 = w; d45 = z; }
                        else if (e == 2) { d45 = a; d24 = b; d34 = c3; d23 = u; d25 = w; d35 = z; }
                        else { d25 = a; d35 = b; d45 = c3; d23 = u; d24 = w; d34 = z; }
                        const int64_t s = (((((int64_t)d25 * D + d35) * D + d45) * D + d24) * D + d34) * D + d23;
                        const cplx g = shell_out[s * (1 + 5 * (int64_t)stride_node) + 1 + node * stride_node + q];
                        acc.x += g.x;
                        acc.y += g.y;
                    }
            if (q & 1) { acc.x = -acc.x; acc.y = -acc.y; }
        }
        G[q] = acc;
    }
    __syncthreads();
    const cplx* ps = psi_all + 32 * (e + 1);
    const double* B = v.B[e] + (int64_t)t * di * dk;
    for (int q = threadIdx.x; q < di * dk; q += blockDim.x) {
        const int i = q / dk, cc = q % dk;
        const double f = sqrt((double)(ilo + 2 * i + 1)) * (double)(klo + 2 * cc + 1);
        const cplx g = G[cc];
        const cplx pg = cmul(ps[i], g);
        if (gB) gB[(int64_t)t * di * dk + q] = (cc < nk) ? cplx{f * pg.x, f * pg.y} : cplx{0.0, 0.0};
    }
    for (int i = threadIdx.x; i < di; i += blockDim.x) {
        cplx acc{0.0, 0.0};
        for (int cc = 0; cc < nk; cc++) {
            const double f = sqrt((double)(ilo + 2 * i + 1)) * (double)(klo + 2 * cc + 1) * B[i * dk + cc];
            acc.x = fma(f, G[cc].x, acc.x);
            acc.y = fma(f, G[cc].y, acc.y);
        }
        Ppsi[(int64_t)t * 32 + i] = acc;
    }
}

// fixed-order sums: a = sum_s a_s, g1[i] = sqrt(2i+1)(-1)^i sum_s d1_s[i], g_e[i] = sum_t P_e[t][i]
__global__ void k_adjoint_final(const VtxDev* __restrict__ vp, const cplx* __restrict__ shell_out, int stride_node,
                                int64_t nshell, const cplx* __restrict__ P, int64_t ntrip, cplx* a_out,
                                cplx* g1, cplx* g2, cplx* g3, cplx* g4, cplx* g5) {
    const VtxDev& v = *vp;
    const int which = blockIdx.x;   // 0: a, 1: g1, 2..5: g_e
    __shared__ double rx[256], ry[256];
    const int n = which == 0 ? 1 : v.di[which - 1];
    for (int i = 0; i < n; i++) {
        double sx = 0.0, sy = 0.0;
        if (which <= 1) {
            for (int64_t s = threadIdx.x; s < nshell; s += blockDim.x) {
                const cplx z = shell_out[s * (1 + 5 * (int64_t)stride_node) + (which == 0 ? 0 : 1 + i)];
                sx += z.x;
                sy += z.y;
            }
        } else {
            const cplx* Pe = P + (int64_t)(which - 2) * ntrip * 32;
            for (int64_t t = threadIdx.x; t < ntrip; t += blockDim.x) {
                sx += Pe[t * 32 + i].x;
                sy += Pe[t * 32 + i].y;
            }
        }
        rx[threadIdx.x] = sx;
        ry[threadIdx.x] = sy;
        __syncthreads();
        for (int off = 128; off > 0; off >>= 1) {
            if (threadIdx.x < off) { rx[threadIdx.x] += rx[threadIdx.x + off]; ry[threadIdx.x] += ry[threadIdx.x + off]; }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            cplx z{rx[0], ry[0]};
            if (which == 0) *a_out = z;
            else if (which == 1) {
                const double f = sqrt((double)(v.ilo[0] + 2 * i + 1)) * ((i & 1) ? -1.0 : 1.0);
                g1[i] = cplx{f * z.x, f * z.y};
            } else {
                cplx* g = which == 2 ? g2 : which == 3 ? g3 : which == 4 ? g4 : g5;
                g[i] = z;
            }
        }
        __syncthreads();
    }
}

// W1 = (-1)^(i - ilo) sqrt(2i+1) psi_1, and psi_1..5 gathered into one padded array
__global__ void k_adjoint_prep(const VtxDev* __restrict__ vp, const cplx* p1, const cplx* p2, const cplx* p3,
                               const cplx* p4, const cplx* p5, cplx* phi1, cplx* psi_all) {
    const VtxDev& v = *vp;
    const cplx* ps[5] = {p1, p2, p3, p4, p5};
    for (int q = threadIdx.x; q < 5 * 32; q += blockDim.x) {
        const int e = q / 32, i = q % 32;
        psi_all[q] = (i < v.di[e]) ? ps[e][i] : cplx{0.0, 0.0};
    }
    for (int i = threadIdx.x; i < v.di[0]; i += blockDim.x) {
        const double f = sqrt((double)(v.ilo[0] + 2 * i + 1)) * ((i & 1) ? -1.0 : 1.0);
        phi1[i] = cplx{f * p1[i].x, f * p1[i].y};
    }
}

int sf_adjoint_launch(const VtxDev* d_v, const VtxDev& h, const double* const psi[5], double* a_out,
                      double* const grad_psi[5], double* const grad_B[4], void* scratch, size_t scratch_bytes,
                      int num_sms, cudaStream_t s) {
    const int stride_node = SF_ADJ_DMAX;
    int mx = 0;
    for (int e = 0; e < 5; e++) mx = imax_(mx, h.di[e]);
    for (int e = 0; e < 4; e++) mx = imax_(mx, h.dkmax[e]);
    if (mx > SF_ADJ_DMAX || h.di[0] > 32) return sf_set_error(SF_ERR_LIMIT, "adjoint supports dimensions up to %d", SF_ADJ_DMAX);
    const int64_t per_shell = 1 + 5 * (int64_t)stride_node;
    char* b = (char*)scratch;
    cplx* psi_all = (cplx*)b;                b += 5 * 32 * sizeof(cplx);
    cplx* phi1 = (cplx*)b;                   b += 32 * sizeof(cplx);
    cplx* P = (cplx*)b;                      b += 4 * h.ntrip * 32 * sizeof(cplx);
    cplx* shell_out = (cplx*)b;              b += (size_t)h.nshell * per_shell * sizeof(cplx);
    if ((size_t)(b - (char*)scratch) > scratch_bytes) return sf_set_error(SF_ERR_OOM, "adjoint scratch too small");
    k_adjoint_prep<<<1, 160, 0, s>>>(d_v, (const cplx*)psi[0], (const cplx*)psi[1], (const cplx*)psi[2],
                                     (const cplx*)psi[3], (const cplx*)psi[4], phi1, psi_all);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    int64_t blocks = (h.nshell + SF_ADJ_WARPS - 1) / SF_ADJ_WARPS;
    if (blocks > (int64_t)num_sms * 64) blocks = (int64_t)num_sms * 64;
    const size_t smem = (size_t)SF_ADJ_WARPS * (14 * mx * mx + 10 * mx) * sizeof(cplx);
    SF_CUDA_TRY(cudaFuncSetAttribute(k_adjoint_shell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int want_nodes = (grad_psi || grad_B) ? 1 : 0;
    k_adjoint_shell<<<(unsigned)blocks, 32 * SF_ADJ_WARPS, smem, s>>>(d_v, phi1, psi_all, h.nshell, stride_node, mx,
                                                                       want_nodes, shell_out);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    for (int e = 0; e < 4 && want_nodes; e++) {
        cplx* gB = grad_B ? (cplx*)grad_B[e] : nullptr;   // optional: the psi gradients only need P
        k_adjoint_triples<<<(unsigned)h.ntrip, 64, 0, s>>>(d_v, e + 2, psi_all, shell_out, stride_node, gB,
                                                           P + (int64_t)e * h.ntrip * 32);
        sf_note_launch(1);
        SF_CUDA_TRY(cudaGetLastError());
    }
    cplx* g[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int e = 0; e < 5; e++) g[e] = grad_psi ? (cplx*)grad_psi[e] : nullptr;
    k_adjoint_final<<<(grad_psi ? 6 : 1), 256, 0, s>>>(d_v, shell_out, stride_node, h.nshell, P, h.ntrip, (cplx*)a_out,
                                                       g[0], g[1], g[2], g[3], g[4]);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

size_t sf_adjoint_scratch_bytes(const VtxDev& h) {
    const int64_t per_shell = 1 + 5 * (int64_t)SF_ADJ_DMAX;
    return (5 * 32 + 32) * sizeof(cplx) + 4 * (size_t)h.ntrip * 32 * sizeof(cplx) +
           (size_t)h.nshell * per_shell * sizeof(cplx) + 1024;
}
