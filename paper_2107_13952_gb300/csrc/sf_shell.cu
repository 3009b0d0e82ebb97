// Shell sum of the vertex amplitude (Sec. 3 framed algorithm, steps 5-7), FP64 path.
//
// Per shell the framed algorithm builds W[i1,k2..k5] = (-1)^E sum_x (2x+1) S1 S2 S3 S4 S5 and
// contracts it with the four booster matrices. The same sum is evaluated here in an order that
// never materialises W and that hoists every factor out of the shells it does not depend on:
// S3 and B4 do not depend on l23, S1, S2 and B5 depend on neither l23, l24 nor l34. For one
// output tile (i1, i2) and one group (l25, l35, l45):
//
//   for (l24, l34):                                       K4 and the S3 slot fixed
//     for x in chunks:
//       U[k3, x, i3] = sum_{l23} R_{l23}[k3, x] B3_{l23}[i3, k3]     (k3 over the union of K3)
//          R_{l23}[k3, x] = (2k3+1)(-1)^(k3-k3lo) sigma_s sum_{k2} S4[k3,k2,x] S5[k2,i1,x] B2'[i2,k2]
//       P[k4, x, i3] = sum_{k3} S3[k4,k3,x] U[k3, x, i3]
//       V[k4, k5, i3] += sum_x (2x+1) S1[i1,k5,x] S2[k5,k4,x] P[k4, x, i3]
//     Y[i4, k5, i3] += sum_{k4} V[k4,k5,i3] B4'[i4,k4]
//   T[i4, i5, i3] += sum_{k5} Y[i4,k5,i3] B5'[i5,k5]
//
// with B' = (2k+1) (-1)^(k - k_lo) B and sigma_s = (-1)^(E_lo/2) the shell's {15j} sign at the
// lowest intertwiners; the remaining (-1)^(i1 - i1_lo) and prod_e sqrt(2 i_e + 1) are applied
// by the reduction. Each CTA owns whole work items (tile, range of groups), so the partial sums
// and their fixed-order reduction are deterministic.
#include "sf_internal.cuh"

// {6j} table read with box and parity checks (zero outside: the symbol vanishes there)
__device__ __forceinline__ double s6(const double* __restrict__ S, const SlotDesc& sd, int a, int b, int x) {
    const int da = a - sd.alo, db = b - sd.blo, dx = x - sd.xlo;
    if (((da | db | dx) & 1) != 0) return 0.0;
    const int ia = da >> 1, ib = db >> 1, ix = dx >> 1;
    if ((unsigned)ia >= (unsigned)sd.na || (unsigned)ib >= (unsigned)sd.nb || (unsigned)ix >= (unsigned)sd.nx)
        return 0.0;
    return __ldg(S + sd.off + ((int64_t)ia * sd.nb + ib) * sd.nx + ix);
}

__device__ __forceinline__ SlotDesc load_slot(const SlotDesc* p) {
    SlotDesc s;
    s.off = p->off; s.alo = p->alo; s.blo = p->blo; s.xlo = p->xlo; s.na = p->na; s.nb = p->nb; s.nx = p->nx;
    return s;
}

__device__ __forceinline__ bool shell_selected(const ShellFilter& f, int64_t s) {
    if (f.bitmap) return (__ldg(f.bitmap + (s >> 5)) >> (s & 31)) & 1u;
    return s >= f.begin && s < f.end;
}

struct ShellSmem {
    double *T, *Y, *V, *U, *P, *Q, *R, *SB, *B4, *B5;
};

__device__ inline ShellSmem carve(double* base, int mdi, int mdk, int mk3u, int xc, int D) {
    ShellSmem s;
    double* p = base;
    s.T = p;  p += mdi * mdi * mdi;
    s.Y = p;  p += mdi * mdi * mdk;
    s.V = p;  p += mdk * mdk * mdi;
    s.U = p;  p += mk3u * xc * mdi;
    s.P = p;  p += mdk * xc * mdi;
    s.Q = p;  p += mdk * mdk * xc;
    s.R = p;  p += D * mdk * xc;
    s.SB = p; p += D * mdk * xc;
    s.B4 = p; p += mdi * mdk;
    s.B5 = p; p += mdi * mdk;
    return s;
}

size_t sf_shell_smem_doubles(int mdi, int mdk, int mk3u, int xc, int D) {
    return (size_t)mdi * mdi * mdi + (size_t)mdi * mdi * mdk + (size_t)mdk * mdk * mdi + (size_t)mk3u * xc * mdi +
           (size_t)mdk * xc * mdi + (size_t)mdk * mdk * xc + 2ull * D * mdk * xc + 2ull * mdi * mdk;
}

__global__ void __launch_bounds__(256) k_shell_fp64(const VtxDev* __restrict__ V, int mdi, int mdk, int mk3u, int XC,
                                                    int Dmax, const WorkItem* __restrict__ items, int n_items,
                                                    int* counter, double* __restrict__ part, ShellFilter filt) {
    extern __shared__ double smem[];
    __shared__ int s_item;
    __shared__ int s_k2lo[SF_MAX_DL + 1], s_nk2[SF_MAX_DL + 1], s_k3lo[SF_MAX_DL + 1], s_nk3[SF_MAX_DL + 1];
    __shared__ double s_sig[SF_MAX_DL + 1];
    __shared__ SlotDesc s_sd4[SF_MAX_DL + 1];
    const ShellSmem sm = carve(smem, mdi, mdk, mk3u, XC, Dmax);
    const int tid = threadIdx.x, nth = blockDim.x;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        const VtxDev& v = V[w.vtx];
        const int D = v.D;
        const int j12 = v.tj[F12], j13 = v.tj[F13], j14 = v.tj[F14], j15 = v.tj[F15];
        const int i1 = v.ilo[0] + 2 * w.i1;
        const int ci2 = w.i2;
        const int di3 = v.di[2], di4 = v.di[3], di5 = v.di[4];
        const int dk1 = v.dkmax[1];
        const int jsum = j12 + j13 + j14 + j15 + v.ilo[0];
        for (int q = tid; q < di3 * di4 * di5; q += nth) sm.T[q] = 0.0;
        for (int g = w.g0; g < w.g1; g++) {
            const int d25 = g / (D * D), d35 = (g / D) % D, d45 = g % D;
            const int l25 = v.tj[F25] + 2 * d25, l35 = v.tj[F35] + 2 * d35, l45 = v.tj[F45] + 2 * d45;
            int k5lo, nk5;
            sf_pair_range(j15, l25, l35, l45, &k5lo, &nk5);
            if (nk5 == 0) continue;
            __syncthreads();
            const int t5 = (d25 * D + d35) * D + d45;
            {
                const double* B5 = v.B[3] + (int64_t)t5 * di5 * v.dkmax[3];
                for (int q = tid; q < di5 * nk5; q += nth) {
                    int i5 = q / nk5, c5 = q % nk5;
                    double f = (double)(k5lo + 2 * c5 + 1) * ((c5 & 1) ? -1.0 : 1.0);
                    sm.B5[q] = f * B5[i5 * v.dkmax[3] + c5];
                }
            }
            for (int q = tid; q < di4 * nk5 * di3; q += nth) sm.Y[q] = 0.0;
            const SlotDesc sd1 = load_slot(v.slot[0] + d25);
            const SlotDesc sd5 = load_slot(v.slot[4] + d25);
            const SlotDesc sd2 = load_slot(v.slot[1] + d35 * D + d45);
            // x bounds from i1 (with l25) and the k5 range (with j14)
            const int k5hi = k5lo + 2 * (nk5 - 1);
            const int x_lo_a = iabs_(i1 - l25), x_hi_a = i1 + l25;
            const int x_lo_b = (j14 < k5lo) ? (k5lo - j14) : (j14 > k5hi ? j14 - k5hi : ((j14 + k5lo) & 1));
            const int x_hi_b = k5hi + j14;
            for (int p = 0; p < D * D; p++) {
                const int d24 = p / D, d34 = p % D;
                const int l24 = v.tj[F24] + 2 * d24, l34 = v.tj[F34] + 2 * d34;
                int k4lo, nk4;
                sf_pair_range(l45, j14, l24, l34, &k4lo, &nk4);
                if (nk4 == 0) continue;
                const int k4hi = k4lo + 2 * (nk4 - 1);
                const int x_lo_c = (l35 < k4lo) ? (k4lo - l35) : (l35 > k4hi ? l35 - k4hi : ((l35 + k4lo) & 1));
                const int x_hi_c = k4hi + l35;
                int xlo = imax_(x_lo_a, imax_(x_lo_b, x_lo_c));
                const int xhi = imin_(x_hi_a, imin_(x_hi_b, x_hi_c));
                if (((xlo - x_lo_a) & 1) != 0) xlo++;   // parity of i1 + l25
                if (xlo > xhi) continue;
                // per-l23 shell data (uniform across the block) and the union of the k3 ranges
                __syncthreads();
                int k3ulo = 1 << 30, k3uhi = -1;
                bool any = false;
                for (int d = 0; d < D; d++) {
                    const int l23 = v.tj[F23] + 2 * d;
                    int k2lo, nk2, k3lo, nk3;
                    sf_pair_range(l23, l24, l25, j12, &k2lo, &nk2);
                    sf_pair_range(l34, l35, j13, l23, &k3lo, &nk3);
                    const int64_t s = (((int64_t)g * D + d24) * D + d34) * D + d;   // group-major order
                    if (nk2 == 0 || nk3 == 0 || !shell_selected(filt, s)) { nk2 = 0; nk3 = 0; }
                    if (nk3 > 0) {
                        any = true;
                        k3ulo = imin_(k3ulo, k3lo);
                        k3uhi = imax_(k3uhi, k3lo + 2 * (nk3 - 1));
                    }
                    if (tid == 0) {
                        s_k2lo[d] = k2lo; s_nk2[d] = nk2; s_k3lo[d] = k3lo; s_nk3[d] = nk3;
                        const int E2 = jsum + k2lo + k3lo + k4lo + k5lo + l23 + l24 + l25 + l34 + l35 + l45;
                        s_sig[d] = ((E2 >> 1) & 1) ? -1.0 : 1.0;
                        s_sd4[d] = load_slot(v.slot[3] + d * D + d24);
                    }
                }
                if (!any) continue;
                const int nk3u = (k3uhi - k3ulo) / 2 + 1;
                const int t4 = (d45 * D + d24) * D + d34;
                {
                    const double* B4 = v.B[2] + (int64_t)t4 * di4 * v.dkmax[2];
                    for (int q = tid; q < di4 * nk4; q += nth) {
                        int i4 = q / nk4, c4 = q % nk4;
                        double f = (double)(k4lo + 2 * c4 + 1) * ((c4 & 1) ? -1.0 : 1.0);
                        sm.B4[q] = f * B4[i4 * v.dkmax[2] + c4];
                    }
                }
                for (int q = tid; q < nk4 * nk5 * di3; q += nth) sm.V[q] = 0.0;
                const SlotDesc sd3 = load_slot(v.slot[2] + (d24 * D + d34) * D + d35);
                for (int xc0 = xlo; xc0 <= xhi; xc0 += 2 * XC) {
                    const int nxc = imin_(XC, (xhi - xc0) / 2 + 1);
                    __syncthreads();
                    // A: SB[d][k2][x] = sigma_d (2k2+1)(-1)^(k2-k2lo) B2[t2][i2][k2] S5[k2,i1,x]
                    for (int q = tid; q < D * mdk * nxc; q += nth) {
                        const int xc = q % nxc, r = q / nxc, c2 = r % mdk, d = r / mdk;
                        if (c2 >= s_nk2[d]) continue;
                        const int k2 = s_k2lo[d] + 2 * c2, x = xc0 + 2 * xc;
                        const int t2 = (d * D + d24) * D + d25;
                        const double b2 = v.B[0][((int64_t)t2 * v.di[1] + ci2) * v.dkmax[0] + c2];
                        const double f = (double)(k2 + 1) * ((c2 & 1) ? -s_sig[d] : s_sig[d]);
                        sm.SB[(d * mdk + c2) * XC + xc] = f * b2 * s6(v.S[4], sd5, k2, i1, x);
                    }
                    __syncthreads();
                    // B: R[d][k3][x] = (2k3+1)(-1)^(k3-k3lo) sum_k2 S4_d[k3,k2,x] SB[d][k2][x]
                    for (int q = tid; q < D * mdk * nxc; q += nth) {
                        const int xc = q % nxc, r = q / nxc, c3 = r % mdk, d = r / mdk;
                        if (c3 >= s_nk3[d]) continue;
                        const int k3 = s_k3lo[d] + 2 * c3, x = xc0 + 2 * xc;
                        const SlotDesc sd4 = s_sd4[d];
                        const int k2lo = s_k2lo[d], nk2 = s_nk2[d];
                        double acc = 0.0;
                        for (int c2 = 0; c2 < nk2; c2++)
                            acc = fma(s6(v.S[3], sd4, k3, k2lo + 2 * c2, x), sm.SB[(d * mdk + c2) * XC + xc], acc);
                        sm.R[(d * mdk + c3) * XC + xc] = acc * (double)(k3 + 1) * ((c3 & 1) ? -1.0 : 1.0);
                    }
                    __syncthreads();
                    // C: U[k3u][x][i3] = sum_d R[d][k3][x] B3_d[i3][k3]
                    for (int q = tid; q < nk3u * nxc * di3; q += nth) {
                        const int i3 = q % di3, r = q / di3, xc = r % nxc, ku = r / nxc;
                        const int k3 = k3ulo + 2 * ku;
                        double acc = 0.0;
                        for (int d = 0; d < D; d++) {
                            const int c3 = (k3 - s_k3lo[d]) >> 1;
                            if (k3 < s_k3lo[d] || c3 >= s_nk3[d]) continue;
                            const int t3 = (d34 * D + d35) * D + d;
                            acc = fma(sm.R[(d * mdk + c3) * XC + xc], __ldg(v.B[1] + ((int64_t)t3 * di3 + i3) * dk1 + c3), acc);
                        }
                        sm.U[q] = acc;
                    }
                    __syncthreads();
                    // D: P[k4][x][i3] = sum_k3 S3[k4,k3,x] U[k3][x][i3]
                    for (int q = tid; q < nk4 * nxc * di3; q += nth) {
                        const int i3 = q % di3, r = q / di3, xc = r % nxc, c4 = r / nxc;
                        const int k4 = k4lo + 2 * c4, x = xc0 + 2 * xc;
                        double acc = 0.0;
                        for (int ku = 0; ku < nk3u; ku++)
                            acc = fma(s6(v.S[2], sd3, k4, k3ulo + 2 * ku, x), sm.U[(ku * nxc + xc) * di3 + i3], acc);
                        sm.P[q] = acc;
                    }
                    // E: Q[k5][k4][x] = (2x+1) S1[i1,k5,x] S2[k5,k4,x]
                    for (int q = tid; q < nk5 * nk4 * nxc; q += nth) {
                        const int xc = q % nxc, r = q / nxc, c4 = r % nk4, c5 = r / nk4;
                        const int k5 = k5lo + 2 * c5, k4 = k4lo + 2 * c4, x = xc0 + 2 * xc;
                        sm.Q[q] = (double)(x + 1) * s6(v.S[0], sd1, i1, k5, x) * s6(v.S[1], sd2, k5, k4, x);
                    }
                    __syncthreads();
                    // F: V[k4][k5][i3] += sum_x Q[k5][k4][x] P[k4][x][i3]
                    for (int q = tid; q < nk4 * nk5 * di3; q += nth) {
                        const int i3 = q % di3, r = q / di3, c5 = r % nk5, c4 = r / nk5;
                        double acc = sm.V[q];
                        for (int xc = 0; xc < nxc; xc++)
                            acc = fma(sm.Q[(c5 * nk4 + c4) * nxc + xc], sm.P[(c4 * nxc + xc) * di3 + i3], acc);
                        sm.V[q] = acc;
                    }
                }
                __syncthreads();
                // G: Y[i4][k5][i3] += sum_k4 V[k4][k5][i3] B4'[i4][k4]
                for (int q = tid; q < di4 * nk5 * di3; q += nth) {
                    const int i3 = q % di3, r = q / di3, c5 = r % nk5, i4 = r / nk5;
                    double acc = sm.Y[q];
                    for (int c4 = 0; c4 < nk4; c4++)
                        acc = fma(sm.V[(c4 * nk5 + c5) * di3 + i3], sm.B4[i4 * nk4 + c4], acc);
                    sm.Y[q] = acc;
                }
            }
            __syncthreads();
            // H: T[i4][i5][i3] += sum_k5 Y[i4][k5][i3] B5'[i5][k5]
            for (int q = tid; q < di4 * di5 * di3; q += nth) {
                const int i3 = q % di3, r = q / di3, i5 = r % di5, i4 = r / di5;
                double acc = sm.T[q];
                for (int c5 = 0; c5 < nk5; c5++)
                    acc = fma(sm.Y[(i4 * nk5 + c5) * di3 + i3], sm.B5[i5 * nk5 + c5], acc);
                sm.T[q] = acc;
            }
        }
        __syncthreads();
        // partial tile in [i3][i4][i5] order
        double* out = part + w.part_off;
        for (int q = tid; q < di3 * di4 * di5; q += nth) {
            const int i5 = q % di5, r = q / di5, i4 = r % di4, i3 = r / di4;
            out[q] = sm.T[(i4 * di5 + i5) * di3 + i3];
        }
    }
}

int sf_shell_fp64_launch(const VtxDev* d_v, int mdi, int mdk, int mk3u, int xc, int Dmax, const WorkItem* d_items,
                         int n_items, int* d_counter, double* d_part, ShellFilter filt, int num_sms, cudaStream_t s) {
    size_t smem = sf_shell_smem_doubles(mdi, mdk, mk3u, xc, Dmax) * sizeof(double);
    if (smem > 200 * 1024) return sf_set_error(SF_ERR_LIMIT, "shell kernel needs %zu bytes of shared memory", smem);
    SF_CUDA_TRY(cudaFuncSetAttribute(k_shell_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    SF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_shell_fp64, 256, smem));
    if (per_sm < 1) per_sm = 1;
    int grid = num_sms * per_sm;
    if (grid > n_items) grid = n_items;
    SF_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), s));
    k_shell_fp64<<<grid, 256, smem, s>>>(d_v, mdi, mdk, mk3u, xc, Dmax, d_items, n_items, d_counter, d_part, filt);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// A[i1][i2][i3][i4][i5] = (-1)^(n_i1) prod_e sqrt(2 i_e + 1) * sum_{chunks} part[tile, chunk][i3][i4][i5]
// items of one vertex are laid out tile-major with `nchunk` consecutive items per tile
__global__ void k_reduce(const VtxDev* __restrict__ V, int vtx, const WorkItem* __restrict__ items, int item0,
                         int nchunk, const double* __restrict__ part, double* __restrict__ A) {
    const VtxDev& v = V[vtx];
    const int tile = blockIdx.x;
    const int ci1 = tile / v.di[1], ci2 = tile % v.di[1];
    const int n3 = v.di[2] * v.di[3] * v.di[4];
    const double s12 = sqrt((double)(v.ilo[0] + 2 * ci1 + 1)) * sqrt((double)(v.ilo[1] + 2 * ci2 + 1)) *
                       ((ci1 & 1) ? -1.0 : 1.0);
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunk; c++) acc += part[items[item0 + tile * nchunk + c].part_off + q];
        const int c5 = q % v.di[4], c4 = (q / v.di[4]) % v.di[3], c3 = q / (v.di[4] * v.di[3]);
        const double s = s12 * sqrt((double)(v.ilo[2] + 2 * c3 + 1)) * sqrt((double)(v.ilo[3] + 2 * c4 + 1)) *
                         sqrt((double)(v.ilo[4] + 2 * c5 + 1));
        A[(int64_t)tile * n3 + q] = s * acc;
    }
}

int sf_reduce_launch(const VtxDev* d_v, int vtx, int ntiles, const WorkItem* d_items, int item0, int nchunk,
                     const double* d_part, double* A, cudaStream_t s) {
    k_reduce<<<ntiles, 256, 0, s>>>(d_v, vtx, d_items, item0, nchunk, d_part, A);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// membership bitmap of a shell list
__global__ void k_bitmap(const int64_t* __restrict__ list, int64_t n, int64_t nshell, uint32_t* bm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = list[i];
    if (s < 0 || s >= nshell) return;
    atomicOr(bm + (s >> 5), 1u << (s & 31));
}

int sf_bitmap_launch(const int64_t* d_list, int64_t n, int64_t nshell, uint32_t* d_bm, cudaStream_t s) {
    SF_CUDA_TRY(cudaMemsetAsync(d_bm, 0, ((nshell + 31) / 32) * sizeof(uint32_t), s));
    if (n > 0) {
        k_bitmap<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d_list, n, nshell, d_bm);
        sf_note_launch(1);
        SF_CUDA_TRY(cudaGetLastError());
    }
    return SF_OK;
}
