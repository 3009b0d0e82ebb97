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
#include <type_traits>
#include <cuda_bf16.h>

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

// C[bt][m][n] (+)= sum_k A[bt][m][k] B[bt][k][n] for a batch of small matrices in shared memory,
// each thread computing 4 consecutive outputs of the flattened [bt][m][n] index space (no padded
// lanes for odd sizes; every output sums over k in increasing order). T: element type of A and B,
// accumulation in T, result added to (ACC) or stored into the double C.
template <typename T, bool ACC>
__device__ __forceinline__ void flat_gemm(int nbatch, int M, int N, int K, const T* A, int a_bs, int am, int ak,
                                          const T* B, int b_bs, int bk, int bn, double* C, int c_bs, int cm, int cn,
                                          int tid, int nth) {
    const int MN = M * N, L = nbatch * MN;
    for (int o0 = 4 * tid; o0 < L; o0 += 4 * nth) {
        int aoff[4], boff[4], coff[4];
        T acc[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int o = o0 + j < L ? o0 + j : L - 1;
            const int bt = o / MN, r = o - bt * MN, m = r / N, n = r - m * N;
            aoff[j] = bt * a_bs + m * am;
            boff[j] = bt * b_bs + n * bn;
            coff[j] = bt * c_bs + m * cm + n * cn;
            acc[j] = T(0);
        }
        for (int k = 0; k < K; k++) {
#pragma unroll
            for (int j = 0; j < 4; j++) acc[j] = fma(A[aoff[j] + k * ak], B[boff[j] + k * bk], acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (o0 + j < L) {
                if (ACC) C[coff[j]] += (double)acc[j];
                else C[coff[j]] = (double)acc[j];
            }
        }
    }
}

// ----------------------------------------------------------------------------------------------
// Compensated FP32 pairs (SF_MIXED_FF). A value is held as (hi, lo) with |lo| <= ulp(hi)/2.
// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, the FMA form of Dekker's
// TwoProduct) as published; the intrinsics keep the compiler from contracting them into FMAs.
// Dot products follow Ogita, Rump and Oishi's Dot2 (SIAM J. Sci. Comput. 26, 2005): the exact
// products' high parts are summed with TwoSum, every rounding error goes to a second FP32 sum, and
// the pair is normalised at the end, so the result is as accurate as a dot product in twice the
// working precision (about 2^-48 relative to the sum of |terms|).
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b| or a == 0
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// one Dot2 step: (sh, sl) += (ah + al) * b, with b a single float
__device__ __forceinline__ void ff_dot_step(float ah, float al, float b, float& sh, float& sl) {
    const float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    float s, t;
    ff_two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}
// one Dot2 step with a pair on both sides (the lo * lo term, below 2^-48 relative, is dropped)
__device__ __forceinline__ void ff_dot_step2(float ah, float al, float bh, float bl, float& sh, float& sl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    float s, t;
    ff_two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}
// normalised product of two pairs
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    float h, l;
    ff_fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}
// normalised product of a pair and a float
__device__ __forceinline__ float2 ff_mul_f(float2 a, float b) {
    const float p = __fmul_rn(a.x, b);
    float e = __fmaf_rn(a.x, b, -p);
    e = __fmaf_rn(a.y, b, e);
    float h, l;
    ff_fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}
// normalised pair from an unnormalised Dot2 accumulator (TwoSum: |sl| may exceed |sh| after cancellation)
__device__ __forceinline__ float2 ff_norm(float sh, float sl) {
    float h, l;
    ff_two_sum(sh, sl, h, l);
    return make_float2(h, l);
}
// pair + pair (both normalised), normalised
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    float s, t;
    ff_two_sum(a.x, b.x, s, t);
    t = __fadd_rn(t, __fadd_rn(a.y, b.y));
    float h, l;
    ff_fast_two_sum(s, t, h, l);
    return make_float2(h, l);
}

// Verification of the pair steps above on the device: n_dots dot products of length len with the
// same step order as the kernel's contractions (k increasing, Dot2 accumulator, normalised at the
// end). kind 0: pair x float (ff_dot_step, the S3 contraction); kind 1: pair x pair (ff_dot_step2,
// the x-sum).
__global__ void k_check_dot2(int kind, int n_dots, int len, const float2* __restrict__ a, const float* __restrict__ bf,
                             const float2* __restrict__ bp, float2* __restrict__ out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_dots) return;
    float sh = 0.0f, sl = 0.0f;
    for (int k = 0; k < len; k++) {
        const float2 x = a[(int64_t)q * len + k];
        if (kind == 0) {
            ff_dot_step(x.x, x.y, bf[(int64_t)q * len + k], sh, sl);
        } else {
            const float2 y = bp[(int64_t)q * len + k];
            ff_dot_step2(x.x, x.y, y.x, y.y, sh, sl);
        }
    }
    out[q] = ff_norm(sh, sl);
}

extern "C" int sf_check_dot2(int32_t kind, int32_t n_dots, int32_t len, const float* a, const float* b, float* out,
                             cudaStream_t stream) {
    if (kind != 0 && kind != 1) return sf_set_error(SF_ERR_ARG, "kind must be 0 (pair x float) or 1 (pair x pair)");
    if (n_dots < 0 || len < 0 || (n_dots > 0 && (!a || !b || !out))) return sf_set_error(SF_ERR_ARG, "bad arguments");
    if (n_dots == 0) return SF_OK;
    k_check_dot2<<<(n_dots + 127) / 128, 128, 0, stream>>>(kind, n_dots, len, reinterpret_cast<const float2*>(a), b,
                                                           reinterpret_cast<const float2*>(b),
                                                           reinterpret_cast<float2*>(out));
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    SF_CUDA_TRY(cudaStreamSynchronize(stream));
    return SF_OK;
}

// floor(o / d) for 0 <= o < 2^31, 1 <= d: multiply by m = floor((2^32 - 1) / d), which
// underestimates by at most one, then correct once
struct FDiv { unsigned m; int d; };
__device__ __forceinline__ FDiv fdiv_make(int d) { return FDiv{0xFFFFFFFFu / (unsigned)d, d}; }
__device__ __forceinline__ int fdiv_q(int o, FDiv f) {
    int q = (int)__umulhi((unsigned)o, f.m);
    if (o - q * f.d >= f.d) q++;
    return q;
}

// Staging loop over q in [0, L) with U elements per thread in flight: all U loads of a round are
// issued before any result is stored, so a thread waits for one L2 round trip per round instead
// of one per element. ld(q) gathers an element, st(q, value) stores it.
template <int U, typename LoadF, typename StoreF>
__device__ __forceinline__ void gather_loop(int L, int tid, int nth, LoadF ld, StoreF st) {
    for (int q0 = tid; q0 < L; q0 += U * nth) {
        decltype(ld(0)) val[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int q = q0 + u * nth;
            if (q < L) val[u] = ld(q);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int q = q0 + u * nth;
            if (q < L) st(q, val[u]);
        }
    }
}

// Small batched GEMMs of the mixed paths, C[bt][m][n] (+)= sum_k A[bt][m][k] B[bt][k][n] with A
// contiguous in k and B, C contiguous in n. Each thread computes RM rows of one column n;
// consecutive threads take consecutive n, so B loads are contiguous and A loads are broadcasts;
// every output sums over k in increasing order. KIND selects the arithmetic:
//   GEMM_FF_D: A (hi, lo) pairs, B floats, Dot2 accumulation, C = the normalised pair;
//   GEMM_FF_F: A and B pairs, Dot2 accumulation, C += the pair (pair addition);
//   GEMM_F32:  A and B floats, FP32 FMA accumulation, C (double) += the float result.
//   GEMM_F32_FF: as GEMM_F32, with C a pair (C += the float result, pair addition);
//   GEMM_F32_SET: as GEMM_F32, C (double) = the float result;
//   GEMM_F32_SETF: as GEMM_F32, C (float) = the result;
//   GEMM_FF_DA: as GEMM_FF_D, C += the pair (pair addition).
enum { GEMM_FF_D = 0, GEMM_FF_F = 1, GEMM_F32 = 2, GEMM_F32_FF = 3, GEMM_F32_SET = 4, GEMM_F32_SETF = 5, GEMM_FF_DA = 6 };
template <int KIND, int RM>
__device__ __forceinline__ void rows_gemm(int nbatch, int M, int N, int K, const void* Av, int a_bs, int am,
                                          const void* Bv, int b_bs, int bk, void* Cv, int c_bs, int cm, int tid,
                                          int nth) {
    constexpr bool F32 = KIND == GEMM_F32 || KIND == GEMM_F32_FF || KIND == GEMM_F32_SET || KIND == GEMM_F32_SETF;
    using TA = typename std::conditional<F32, float, float2>::type;
    using TB = typename std::conditional<KIND == GEMM_FF_F, float2, float>::type;
    const TA* A = reinterpret_cast<const TA*>(Av);
    const TB* B = reinterpret_cast<const TB*>(Bv);
    const int MB = (M + RM - 1) / RM, L = nbatch * MB * N;
    const FDiv dN = fdiv_make(N), dMB = fdiv_make(MB);
    for (int o = tid; o < L; o += nth) {
        const int r = fdiv_q(o, dN), n = o - r * N;
        const int bt = fdiv_q(r, dMB), mb = r - bt * MB;
        const TA* ap[RM];
#pragma unroll
        for (int i = 0; i < RM; i++) ap[i] = A + bt * a_bs + imin_(mb * RM + i, M - 1) * am;
        const TB* bp = B + bt * b_bs + n;
        float sh[RM], sl[RM];
#pragma unroll
        for (int i = 0; i < RM; i++) { sh[i] = 0.0f; sl[i] = 0.0f; }
#pragma unroll 4
        for (int k = 0; k < K; k++) {
            const TB b = *bp;
            bp += bk;
#pragma unroll
            for (int i = 0; i < RM; i++) {
                const TA a = ap[i][k];
                if constexpr (F32) sh[i] = fmaf(a, b, sh[i]);
                else if constexpr (KIND == GEMM_FF_D || KIND == GEMM_FF_DA) ff_dot_step(a.x, a.y, b, sh[i], sl[i]);
                else ff_dot_step2(a.x, a.y, b.x, b.y, sh[i], sl[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < RM; i++) {
            const int m = mb * RM + i;
            if (m < M) {
                const int co = bt * c_bs + m * cm + n;
                if constexpr (KIND == GEMM_F32) {
                    reinterpret_cast<double*>(Cv)[co] += (double)sh[i];
                } else if constexpr (KIND == GEMM_F32_SET) {
                    reinterpret_cast<double*>(Cv)[co] = (double)sh[i];
                } else if constexpr (KIND == GEMM_F32_SETF) {
                    reinterpret_cast<float*>(Cv)[co] = sh[i];
                } else if constexpr (KIND == GEMM_F32_FF) {
                    float2* cp = reinterpret_cast<float2*>(Cv) + co;
                    *cp = ff_add(*cp, make_float2(sh[i], 0.0f));
                } else {
                    float2* cp = reinterpret_cast<float2*>(Cv) + co;
                    const float2 v = ff_norm(sh[i], sl[i]);
                    if constexpr (KIND == GEMM_FF_F || KIND == GEMM_FF_DA) *cp = ff_add(*cp, v);
                    else *cp = v;
                }
            }
        }
    }
}

// {6j} lookups with box and parity checks for the FP32 copies (zero outside)
__device__ __forceinline__ int s6_index(const SlotDesc& sd, int a, int b, int x) {
    const int da = a - sd.alo, db = b - sd.blo, dx = x - sd.xlo;
    if (((da | db | dx) & 1) != 0) return -1;
    const int ia = da >> 1, ib = db >> 1, ix = dx >> 1;
    if ((unsigned)ia >= (unsigned)sd.na || (unsigned)ib >= (unsigned)sd.nb || (unsigned)ix >= (unsigned)sd.nx) return -1;
    return (ia * sd.nb + ib) * sd.nx + ix;
}
__device__ __forceinline__ float2 s6ff(const float2* __restrict__ S, const SlotDesc& sd, int a, int b, int x) {
    const int i = s6_index(sd, a, b, x);
    return i < 0 ? make_float2(0.0f, 0.0f) : __ldg(S + sd.off + i);
}
__device__ __forceinline__ float s6f(const float* __restrict__ S, const SlotDesc& sd, int a, int b, int x) {
    const int i = s6_index(sd, a, b, x);
    return i < 0 ? 0.0f : __ldg(S + sd.off + i);
}

// Asynchronous global-to-shared copies of 4 or 8 bytes (cp.async, cached at all levels): the
// bytes beyond src_bytes are zero-filled, and with src_bytes 0 nothing is read. A thread issues
// any number of them without holding registers for the values; cp_async_wait_all waits for all
// of the thread's copies (a barrier then publishes them to the block).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ----------------------------------------------------------------------------------------------
// Tensor-core booster contraction (SF_MIXED_TC). An FP32 value v is split into three BF16 pieces,
// h0 = bf16(v), h1 = bf16(v - h0), h2 = bf16(v - h0 - h1) (each difference exact in FP32), which
// hold its 24 significant bits; a product a b is formed from the six piece products of order
// <= 2 (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1, a2 b0; the dropped ones are below 2^-23 |a b|),
// accumulated in FP32 by mma.sync m16n8k16 (BF16 inputs, FP32 accumulators): FP32-class accuracy
// on the tensor pipe. BF16 keeps the FP32 exponent range, so no scaling is needed.
// Operand planes in shared memory: piece-major, rows of ks = Kp + 8 BF16 (the 8-element pad puts
// the eight rows that one fragment load touches on distinct banks).
// ----------------------------------------------------------------------------------------------
__host__ __device__ inline int tc_ks(int mdk) { return ((mdk + 15) / 16) * 16 + 8; }
__host__ __device__ inline size_t tc_ap_doubles(int mdk, int mni3) {   // V^T planes, 3 x Mp x ks BF16
    const size_t mp = (((size_t)mdk * mni3 + 15) / 16) * 16;
    return (3 * mp * tc_ks(mdk) * 2 + 7) / 8;
}
__host__ __device__ inline size_t tc_bp_doubles(int mdi, int mdk) {    // B4' planes, 3 x Np x ks BF16
    const size_t np = (((size_t)mdi + 7) / 8) * 8;
    return (3 * np * tc_ks(mdk) * 2 + 7) / 8;
}
__device__ __forceinline__ void split3_bf16(float v, unsigned short& h0, unsigned short& h1, unsigned short& h2) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = __fsub_rn(v, __bfloat162float(b0));
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(b1));
    const __nv_bfloat16 b2 = __float2bfloat16_rn(r2);
    h0 = __bfloat16_as_ushort(b0);
    h1 = __bfloat16_as_ushort(b1);
    h2 = __bfloat16_as_ushort(b2);
}
__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// Y[n][m] += sum_k A[m][k] B[n][k] for m < M, n < N, k < K from the planes Ap (Mp x ks per piece)
// and Bp (Np x ks per piece); each warp takes 16 x 8 output tiles in turn.
__device__ __forceinline__ void tc_gemm_acc(const unsigned short* __restrict__ Ap, const unsigned short* __restrict__ Bp,
                                            int M, int N, int K, int ks, double* __restrict__ Y, int tid, int nth) {
    const int Mp = (M + 15) & ~15, Np = (N + 7) & ~7, Kp = (K + 15) & ~15;
    const int planeA = Mp * ks, planeB = Np * ks;
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const int nmt = Mp >> 4, nnt = Np >> 3;
    for (int job = warp; job < nmt * nnt; job += nth >> 5) {
        const int mt = job % nmt, nt = job / nmt;
        float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int k0 = 0; k0 < Kp; k0 += 16) {
            uint32_t a[3][4], b[3][2];
#pragma unroll
            for (int pc = 0; pc < 3; pc++) {
                const unsigned short* ab = Ap + pc * planeA + (mt * 16 + g) * ks + k0 + 2 * t;
                a[pc][0] = *reinterpret_cast<const uint32_t*>(ab);
                a[pc][1] = *reinterpret_cast<const uint32_t*>(ab + 8 * ks);
                a[pc][2] = *reinterpret_cast<const uint32_t*>(ab + 8);
                a[pc][3] = *reinterpret_cast<const uint32_t*>(ab + 8 * ks + 8);
                const unsigned short* bb = Bp + pc * planeB + (nt * 8 + g) * ks + k0 + 2 * t;
                b[pc][0] = *reinterpret_cast<const uint32_t*>(bb);
                b[pc][1] = *reinterpret_cast<const uint32_t*>(bb + 8);
            }
            // smallest products first
            mma_bf16_16816(c, a[2], b[0]);
            mma_bf16_16816(c, a[1], b[1]);
            mma_bf16_16816(c, a[0], b[2]);
            mma_bf16_16816(c, a[1], b[0]);
            mma_bf16_16816(c, a[0], b[1]);
            mma_bf16_16816(c, a[0], b[0]);
        }
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const int m = mt * 16 + g + 8 * h, n = nt * 8 + 2 * t + j;
                if (m < M && n < N) Y[n * M + m] += (double)c[2 * h + j];
            }
    }
}

#define SF_TRT 2   // output-tile register blocks per thread (2 x 4 doubles each); one at 1024 threads

struct ShellSmem {
    double *Y, *V, *B3s, *B4, *B5, *S3s, *Q, *R, *P, *SB, *U;
    float *Vf, *B4f;   // mixed path: FP32 copies for the k4 booster contraction
    unsigned short *Ap, *Bp;   // tensor-core path: BF16 planes of V^T and of B4'
    float* B2s;                // asynchronous staging: the scaled B2 entries of the 5-tuple, [d][c2] (FP32 or FP64)
    double* S1s;               // asynchronous staging: the S1 entries of the x chunk, [c5][x] (pairs or FP64)
};

// Shared-memory layout of one CTA. mni3: largest i3 extent of a work item. Buffers whose
// lifetimes within an x chunk do not overlap share space: R (written in B, read in C) with P
// (written in D, read in F), SB (A -> B) with U (C -> D); the FP32 copy Vf of V (used after the
// x loop) lies over the chunk buffers.
__host__ __device__ inline size_t shell_chunk_doubles(int mdk, int mk3u, int xc, int D, int mni3) {
    const size_t rp = (size_t)D * mdk * xc > (size_t)mdk * xc * mni3 ? (size_t)D * mdk * xc : (size_t)mdk * xc * mni3;
    const size_t su = (size_t)D * mdk * xc > (size_t)mk3u * xc * mni3 ? (size_t)D * mdk * xc : (size_t)mk3u * xc * mni3;
    return (size_t)xc * mdk * mk3u + (size_t)mdk * mdk * xc + rp + su;
}
// extra space of the asynchronously staged paths: B2s (D x mdk floats, or doubles in the FP64
// path) and S1s (mdk x xc pairs or doubles)
__host__ __device__ inline size_t shell_b2s_doubles(int mdk, int D, bool d64) {
    return d64 ? (size_t)D * mdk : ((size_t)D * mdk + 1) / 2;
}
__host__ __device__ inline size_t shell_px_doubles(int mdk, int xc, int D, bool d64) {
    return shell_b2s_doubles(mdk, D, d64) + (size_t)mdk * xc;
}

__device__ inline ShellSmem carve(double* base, int mdi, int mdk, int mk3u, int xc, int D, int mni3, bool tc, bool px,
                                  bool d64) {
    ShellSmem s;
    double* p = base;
    s.Y = p;   p += mdi * mdk * mni3;
    s.V = p;   p += mdk * mdk * mni3;
    s.B3s = p; p += D * mdk * mni3;
    s.B4 = p;  p += mdi * mdk;
    s.B5 = p;  p += mdi * mdk;
    s.B4f = reinterpret_cast<float*>(p);
    p += (mdi * mdk + 1) / 2;
    s.Bp = reinterpret_cast<unsigned short*>(p);
    if (tc) p += tc_bp_doubles(mdi, mdk);
    s.B2s = reinterpret_cast<float*>(p);
    s.S1s = p + shell_b2s_doubles(mdk, D, d64);
    if (px) p += shell_px_doubles(mdk, xc, D, d64);
    double* chunk = p;
    s.Ap = reinterpret_cast<unsigned short*>(chunk);   // after the x loop, over the chunk buffers
    s.S3s = p; p += xc * mdk * mk3u;
    s.Q = p;   p += mdk * mdk * xc;
    s.R = p;
    s.P = p;
    p += (D * mdk * xc > mdk * xc * mni3) ? D * mdk * xc : mdk * xc * mni3;
    s.SB = p;
    s.U = p;
    s.Vf = reinterpret_cast<float*>(chunk);
    return s;
}

size_t sf_shell_smem_doubles(int mdi, int mdk, int mk3u, int xc, int D, int mni3, int mode) {
    const bool mix = mode >= 1, tc = mode == 3, px = mode != 1;   // px: asynchronous staging
    const size_t chunk = shell_chunk_doubles(mdk, mk3u, xc, D, mni3);
    size_t over = mix ? ((size_t)mdk * mdk * mni3 + 1) / 2 : 0;   // Vf, or the V^T planes
    if (tc) over = tc_ap_doubles(mdk, mni3);
    return (size_t)mdi * mdk * mni3 + (size_t)mdk * mdk * mni3 + (size_t)D * mdk * mni3 + 2ull * mdi * mdk +
           ((size_t)mdi * mdk + 1) / 2 + (tc ? tc_bp_doubles(mdi, mdk) : 0) + (px ? shell_px_doubles(mdk, xc, D, mode == 0) : 0) +
           (chunk > over ? chunk : over);
}

// MODE 0: every phase in FP64 (the FP64 path). MODE 1 (the mixed path): the booster
// contractions over k2 (B2, with S4 S5), over k3 (B3, summed over l23) and over k4 (B4) take FP32
// inputs and accumulate in FP32 within one (l24, l34) 5-tuple; the {6j} contractions (S3, and the
// x-sum with S1 S2), every sum across 5-tuples and groups, and the k5 contraction stay FP64.
// MODE 2: as MODE 1, but the {6j} contractions (phases D and F, and the products Q) run on
// compensated FP32 pairs with Dot2 accumulation, from (hi, lo) copies of S1, S2, S3; V is kept as
// a pair across the x chunks of a 5-tuple and Y across the 5-tuples of a group (converted to FP64
// for the k5 contraction); the booster operands come from FP32 copies of the boosters. GB300's FP64 pipe issues 2 FMAs per clock per SM
// against 128 FP32 FMAs, so a pair step of about 11 FP32 instructions is several times cheaper.
// MODE 3: as MODE 1, with the k4 contraction on the tensor cores (split BF16, below) and the S3
// contraction in FP32. MODE 4: the booster contractions and the S3 contraction in FP32 on the
// CUDA cores, the x-sum (phase F) on compensated FP32 pairs: Q from the (hi, lo) copies of S1 and
// S2, P in FP32, V a pair accumulated by Dot2 steps (pair times float); the remaining FP64 work
// is the k5 contraction and the sums across 5-tuples and groups.
// NT threads per CTA: 512 (one CTA per SM) or 256 (two CTAs per SM, whose phases interleave);
// MODE 4 also 1024 (one CTA per SM, 64 registers a thread: its staging holds no values in
// registers, so twice the warps hide the shared-memory and L2 latencies of its phases).
// A work item covers the i3 sub-range [i3b, i3b + ni3) of its output tile.
template <int MODE, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 512 / NT) k_shell(const VtxDev* __restrict__ V, int mdi, int mdk, int mk3u, int XC,
                                                        int Dmax, int mni3, const WorkItem* __restrict__ items,
                                                        int n_items, int* counter, double* __restrict__ part,
                                                        ShellFilter filt) {
    constexpr bool MIX = MODE >= 1;
    constexpr bool FF = MODE == 2;
    constexpr bool TC = MODE == 3;   // k4 contraction on the tensor cores, S3 contraction FP32, x-sum FP64
    constexpr bool PX = MODE == 4;   // S3 contraction FP32, x-sum on compensated pairs
    constexpr bool F32IN = FF || TC || PX;   // booster operands from the FP32 copies
    constexpr bool AS = MODE != 1;               // operands staged by asynchronous copies
    constexpr bool PQ = FF || PX;                // Q and S1 as compensated pairs
    constexpr bool D64 = MODE == 0;              // ... as FP64 values (B2s, SB, S3s, B3 rows)
    constexpr int TRT = NT >= 1024 ? 1 : SF_TRT;   // output-tile blocks per thread
    constexpr int GU = FF ? 4 : 2;   // staging elements in flight per thread (FP64 values: register budget)
    extern __shared__ double smem[];
    __shared__ int s_item;
    __shared__ int s_k2lo[SF_MAX_DL + 1], s_nk2[SF_MAX_DL + 1], s_k3lo[SF_MAX_DL + 1], s_nk3[SF_MAX_DL + 1];
    __shared__ int2 s_c3n[SF_MAX_DL + 1];   // per l23: (offset of the k3 union start in its k3 range, range size)
    __shared__ double s_sig[SF_MAX_DL + 1];
    __shared__ float s_sigf[SF_MAX_DL + 1];
    __shared__ SlotDesc s_sd4[SF_MAX_DL + 1];
    __shared__ SlotDesc s_sdx[4];   // slots of S1, S5, S2 (per group) and S3 (per 5-tuple), read in place
    __shared__ VtxDev s_v;          // the current work item's vertex record
    __shared__ int s_vtx;
    if (threadIdx.x == 0) s_vtx = -1;
    const ShellSmem sm = carve(smem, mdi, mdk, mk3u, XC, Dmax, mni3, TC, AS, D64);
    const int tid = threadIdx.x, nth = NT;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        // the vertex record in shared memory: its fields are read throughout the item, and from
        // global memory they would be evicted from L1 by the streamed {6j} slabs
        if (w.vtx != s_vtx) {
            const int* src = reinterpret_cast<const int*>(V + w.vtx);
            int* dst = reinterpret_cast<int*>(&s_v);
            for (int q = tid; q < (int)(sizeof(VtxDev) / sizeof(int)); q += nth) dst[q] = src[q];
            __syncthreads();
            if (tid == 0) s_vtx = w.vtx;
        }
        const VtxDev& v = s_v;
        const int D = v.D;
        const int j12 = v.tj[F12], j13 = v.tj[F13], j14 = v.tj[F14], j15 = v.tj[F15];
        const int i1 = v.ilo[0] + 2 * w.i1;
        const int ci2 = w.i2;
        // output block: i3 in [i3b, i3b + ni3) of the whole range, i4 and i5 from the vertex's
        // sub-range (rows o4.., o5.. of the edge-4 and edge-5 boosters)
        const int di3 = w.ni3, i3b = w.i3b, di3f = v.di[2], di4 = v.od[3], di5 = v.od[4];
        const int o4 = v.olo[3], o5 = v.olo[4];
        const int dk1 = v.dkmax[1];
        const int jsum = j12 + j13 + j14 + j15 + v.ilo[0];
        // output tile T[i4][i5][i3] in registers: blocks (i4, 2 i5, 4 i3), block b = tid + r * nth
        const int tb5 = (di5 + 1) / 2, tb3 = (di3 + 3) / 4, tper = tb5 * tb3;
        double T[TRT][2][4];
#pragma unroll
        for (int r = 0; r < TRT; r++)
#pragma unroll
            for (int i = 0; i < 2; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) T[r][i][j] = 0.0;
        for (int g = w.g0; g < w.g1; g++) {
            const int d25 = g / (D * D), d35 = (g / D) % D, d45 = g % D;
            const int l25 = v.tj[F25] + 2 * d25, l35 = v.tj[F35] + 2 * d35, l45 = v.tj[F45] + 2 * d45;
            int k5lo, nk5;
            sf_pair_range(j15, l25, l35, l45, &k5lo, &nk5);
            if (nk5 == 0) continue;
            __syncthreads();
            const int t5 = (d25 * D + d35) * D + d45;
            {
                const double* B5 = v.B[3] + (int64_t)t5 * v.di[4] * v.dkmax[3];
                for (int q = tid; q < di5 * nk5; q += nth) {
                    const int i5 = q / nk5, c5 = q % nk5;
                    const double f = (double)(k5lo + 2 * c5 + 1) * ((c5 & 1) ? -1.0 : 1.0);
                    sm.B5[q] = f * B5[(i5 + o5) * v.dkmax[3] + c5];
                }
            }
            for (int q = tid; q < di4 * nk5 * di3; q += nth) sm.Y[q] = 0.0;
            if (tid == 0) {
                s_sdx[0] = load_slot(v.slot[0] + d25);
                s_sdx[1] = load_slot(v.slot[4] + d25);
                s_sdx[2] = load_slot(v.slot[1] + d35 * D + d45);
            }
            const SlotDesc& sd1 = s_sdx[0];
            const SlotDesc& sd5 = s_sdx[1];
            const SlotDesc& sd2 = s_sdx[2];
            const int k5hi = k5lo + 2 * (nk5 - 1);
            const int x_lo_a = iabs_(i1 - l25), x_hi_a = i1 + l25;
            const int x_lo_b = (j14 < k5lo) ? (k5lo - j14) : (j14 > k5hi ? j14 - k5hi : ((j14 + k5lo) & 1));
            const int x_hi_b = k5hi + j14;
            bool gany = false;
            const int p_lo = w.single ? ((w.single - 1) >> 6) : 0, p_hi = w.single ? p_lo + 1 : D * D;
            const int d_one = w.single ? ((w.single - 1) & 63) : -1;
            for (int p = p_lo; p < p_hi; p++) {
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
                __syncthreads();   // the previous 5-tuple is done with the per-l23 arrays and the buffers
                // per-l23 shell data, one thread per l23
                for (int d = tid; d < D; d += nth) {
                    const int l23 = v.tj[F23] + 2 * d;
                    int k2lo, nk2, k3lo, nk3;
                    sf_pair_range(l23, l24, l25, j12, &k2lo, &nk2);
                    sf_pair_range(l34, l35, j13, l23, &k3lo, &nk3);
                    const int64_t s = (((int64_t)g * D + d24) * D + d34) * D + d;   // group-major order
                    if (nk2 == 0 || nk3 == 0 || !shell_selected(filt, s) || (d_one >= 0 && d != d_one)) { nk2 = 0; nk3 = 0; }
                    s_k2lo[d] = k2lo; s_nk2[d] = nk2; s_k3lo[d] = k3lo; s_nk3[d] = nk3;
                    const int E2 = jsum + k2lo + k3lo + k4lo + k5lo + l23 + l24 + l25 + l34 + l35 + l45;
                    s_sig[d] = ((E2 >> 1) & 1) ? -1.0 : 1.0;
                    s_sigf[d] = ((E2 >> 1) & 1) ? -1.0f : 1.0f;
                    s_sd4[d] = load_slot(v.slot[3] + d * D + d24);
                }
                __syncthreads();
                // the union of the k3 ranges (every thread, from the shared arrays)
                int k3ulo = 1 << 30, k3uhi = -1;
                for (int d = 0; d < D; d++) {
                    const int nk3 = s_nk3[d], k3lo = s_k3lo[d];
                    if (nk3 > 0) {
                        k3ulo = imin_(k3ulo, k3lo);
                        k3uhi = imax_(k3uhi, k3lo + 2 * (nk3 - 1));
                    }
                }
                if (k3uhi < 0) continue;   // no selected shell in this 5-tuple
                gany = true;
                for (int d = tid; d < D; d += nth) s_c3n[d] = make_int2((k3ulo - s_k3lo[d]) / 2, s_nk3[d]);
                const int nk3u = (k3uhi - k3ulo) / 2 + 1;
                const FDiv f_nk3u = fdiv_make(nk3u), f_di3 = fdiv_make(di3), f_mdk5 = fdiv_make(mdk);
                const int t4 = (d45 * D + d24) * D + d34;
                if constexpr (TC) {
                    // B4'[i4][c4] as BF16 planes [piece][i4][c4] (zero-padded to whole tiles)
                    const float* B4 = v.Bf[2] + (int64_t)t4 * v.di[3] * v.dkmax[2];
                    const int ks = tc_ks(mdk), Np = (di4 + 7) & ~7, Kp2 = ((nk4 + 15) & ~15) / 2;
                    for (int q = tid; q < Np * Kp2; q += nth) {
                        const int n = q / Kp2, k0 = 2 * (q - n * Kp2);
                        float w0 = 0.0f, w1 = 0.0f;
                        if (n < di4) {
                            const float* row = B4 + (int64_t)(n + o4) * v.dkmax[2];
                            if (k0 < nk4) w0 = (float)(k4lo + 2 * k0 + 1) * ((k0 & 1) ? -1.0f : 1.0f) * row[k0];
                            if (k0 + 1 < nk4) w1 = (float)(k4lo + 2 * k0 + 3) * ((k0 & 1) ? 1.0f : -1.0f) * row[k0 + 1];
                        }
                        unsigned short a0, a1, a2, b0, b1, b2;
                        split3_bf16(w0, a0, a1, a2);
                        split3_bf16(w1, b0, b1, b2);
                        uint32_t* dst = reinterpret_cast<uint32_t*>(sm.Bp + n * ks + k0);
                        const int pl = (Np * ks) / 2;   // one plane, in 32-bit words
                        dst[0] = (uint32_t)a0 | ((uint32_t)b0 << 16);
                        dst[pl] = (uint32_t)a1 | ((uint32_t)b1 << 16);
                        dst[2 * pl] = (uint32_t)a2 | ((uint32_t)b2 << 16);
                    }
                } else if constexpr (FF || PX) {
                    const float* B4 = v.Bf[2] + (int64_t)t4 * v.di[3] * v.dkmax[2];
                    for (int q = tid; q < di4 * nk4; q += nth) {
                        const int i4 = q / nk4, c4 = q % nk4;
                        const float f = (float)(k4lo + 2 * c4 + 1) * ((c4 & 1) ? -1.0f : 1.0f);
                        sm.B4f[q] = f * B4[(i4 + o4) * v.dkmax[2] + c4];
                    }
                } else {
                    const double* B4 = v.B[2] + (int64_t)t4 * v.di[3] * v.dkmax[2];
                    for (int q = tid; q < di4 * nk4; q += nth) {
                        const int i4 = q / nk4, c4 = q % nk4;
                        const double f = (double)(k4lo + 2 * c4 + 1) * ((c4 & 1) ? -1.0 : 1.0);
                        sm.B4[q] = f * B4[(i4 + o4) * v.dkmax[2] + c4];
                    }
                }
                // raw B3 rows of every l23, transposed to [d][c3][i3] (read along c3: coalesced)
                {
                    const int t30 = (d34 * D + d35) * D;
                    auto b3_at = [&](int q, int& d, int& i3, int& c3) {
                        const int r = fdiv_q(q, f_mdk5);
                        c3 = q - r * mdk;
                        d = fdiv_q(r, f_di3);
                        i3 = r - d * di3;
                    };
                    if constexpr (AS) {
                        // asynchronous copies (zero past the row's dk1 entries), and the scaled
                        // B2 entries of the 5-tuple: B2s[d][c2] = sigma_d (2k2+1)(-1)^c2 B2[t2][i2][k2]
                        float* b3f = reinterpret_cast<float*>(sm.B3s);
                        for (int q = tid; q < D * mdk * di3; q += nth) {
                            int d, i3, c3;
                            b3_at(q, d, i3, c3);
                            const int64_t o = ((int64_t)(t30 + d) * di3f + i3b + i3) * dk1 + c3;
                            const int e = (d * mdk + c3) * di3 + i3;
                            if constexpr (D64) cp_async8(sm.B3s + e, c3 < dk1 ? v.B[1] + o : v.B[1], c3 < dk1 ? 8 : 0);
                            else cp_async4(b3f + e, c3 < dk1 ? v.Bf[1] + o : v.Bf[1], c3 < dk1 ? 4 : 0);
                        }
                        double* b2d = reinterpret_cast<double*>(sm.B2s);
                        for (int q = tid; q < D * mdk; q += nth) {
                            const int d = q / mdk, c2 = q - d * mdk;
                            const int k2 = s_k2lo[d] + 2 * c2;
                            const int64_t bi = ((int64_t)((d * D + d24) * D + d25) * v.di[1] + ci2) * v.dkmax[0] + c2;
                            if constexpr (D64) {
                                double b = 0.0;
                                if (c2 < s_nk2[d]) {
                                    const double f = (double)(k2 + 1) * ((c2 & 1) ? -s_sig[d] : s_sig[d]);
                                    b = f * __ldg(v.B[0] + bi);
                                }
                                b2d[q] = b;
                            } else {
                                float b = 0.0f;
                                if (c2 < s_nk2[d]) {
                                    const float f = (float)(k2 + 1) * ((c2 & 1) ? -s_sigf[d] : s_sigf[d]);
                                    b = f * __ldg(v.Bf[0] + bi);
                                }
                                sm.B2s[q] = b;
                            }
                        }
                    } else if constexpr (F32IN) {
                        gather_loop<4>(D * mdk * di3, tid, nth, [&](int q) {
                            int d, i3, c3;
                            b3_at(q, d, i3, c3);
                            return (c3 < dk1) ? __ldg(v.Bf[1] + ((int64_t)(t30 + d) * di3f + i3b + i3) * dk1 + c3) : 0.0f;
                        }, [&](int q, float val) {
                            int d, i3, c3;
                            b3_at(q, d, i3, c3);
                            reinterpret_cast<float*>(sm.B3s)[(d * mdk + c3) * di3 + i3] = val;
                        });
                    } else {
                        gather_loop<4>(D * mdk * di3, tid, nth, [&](int q) {
                            int d, i3, c3;
                            b3_at(q, d, i3, c3);
                            return (c3 < dk1) ? __ldg(v.B[1] + ((int64_t)(t30 + d) * di3f + i3b + i3) * dk1 + c3) : 0.0;
                        }, [&](int q, double val) {
                            int d, i3, c3;
                            b3_at(q, d, i3, c3);
                            if constexpr (MIX) reinterpret_cast<float*>(sm.B3s)[(d * mdk + c3) * di3 + i3] = (float)val;
                            else sm.B3s[(d * mdk + c3) * di3 + i3] = val;
                        });
                    }
                }
                for (int q = tid; q < nk4 * nk5 * di3; q += nth) sm.V[q] = 0.0;
                if (tid == 0) s_sdx[3] = load_slot(v.slot[2] + (d24 * D + d34) * D + d35);
                const SlotDesc& sd3 = s_sdx[3];
                for (int xc0 = xlo; xc0 <= xhi; xc0 += 2 * XC) {
                    const int nxc = imin_(XC, (xhi - xc0) / 2 + 1);
                    __syncthreads();
                    // A: SB[d][k2][x] = sigma_d (2k2+1)(-1)^(k2-k2lo) B2[t2][i2][k2] S5[k2,i1,x];
                    //    S3s[x][k4][k3u] staged from the S3 slot (zero outside its box)
                    const FDiv f_nxc = fdiv_make(nxc), f_mdk = fdiv_make(mdk), f_nk4 = fdiv_make(nk4);
                    if constexpr (AS) {
                        // every operand by asynchronous copies (zero outside the slot boxes), then
                        // the products in place: SB = B2s S5 (FP32, or FP64 in MODE 0), and
                        // Q = ((S1 S2) (2x+1)) as pairs (MODES 2 and 4) or Q = ((2x+1) S1) S2 in FP64
                        // from the prescaled S1x (MODES 0 and 3), with the roundings of forming
                        // them from loaded values
                        float* sbf = reinterpret_cast<float*>(sm.SB);
                        float* s3f = reinterpret_cast<float*>(sm.S3s);
                        float2* qf = reinterpret_cast<float2*>(sm.Q);
                        float2* s1f = reinterpret_cast<float2*>(sm.S1s);
                        for (int q = tid; q < D * mdk * nxc; q += nth) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, d = fdiv_q(r, f_mdk), c2 = r - d * mdk;
                            if (c2 >= s_nk2[d]) continue;
                            const int i = s6_index(sd5, s_k2lo[d] + 2 * c2, i1, xc0 + 2 * xc);
                            const int e = (d * mdk + c2) * XC + xc;
                            if constexpr (D64) cp_async8(sm.SB + e, v.S[4] + (i < 0 ? 0 : sd5.off + i), i < 0 ? 0 : 8);
                            else cp_async4(sbf + e, i < 0 ? v.S5f : v.S5f + sd5.off + i, i < 0 ? 0 : 4);
                        }
                        for (int q = tid; q < nxc * nk4 * nk3u; q += nth) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, c4 = fdiv_q(r, f_nk3u), ku = r - c4 * nk3u;
                            const int i = s6_index(sd3, k4lo + 2 * c4, k3ulo + 2 * ku, xc0 + 2 * xc);
                            const int e = (xc * nk4 + c4) * nk3u + ku;
                            if constexpr (D64) {
                                cp_async8(sm.S3s + e, v.S[2] + (i < 0 ? 0 : sd3.off + i), i < 0 ? 0 : 8);
                            } else if constexpr (FF) {   // the (hi, lo) pair
                                cp_async8(reinterpret_cast<float2*>(sm.S3s) + e, v.Sff[2] + (i < 0 ? 0 : sd3.off + i),
                                          i < 0 ? 0 : 8);
                            } else {
                                const float* src = reinterpret_cast<const float*>(v.Sff[2] + (i < 0 ? 0 : sd3.off + i));
                                cp_async4(s3f + e, src, i < 0 ? 0 : 4);   // the high part
                            }
                        }
                        for (int q = tid; q < nk5 * nk4 * nxc; q += nth) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, c5 = fdiv_q(r, f_nk4), c4 = r - c5 * nk4;
                            const int i = s6_index(sd2, k5lo + 2 * c5, k4lo + 2 * c4, xc0 + 2 * xc);
                            if constexpr (PQ) cp_async8(qf + q, v.Sff[1] + (i < 0 ? 0 : sd2.off + i), i < 0 ? 0 : 8);
                            else cp_async8(sm.Q + q, v.S[1] + (i < 0 ? 0 : sd2.off + i), i < 0 ? 0 : 8);
                        }
                        for (int q = tid; q < nk5 * nxc; q += nth) {
                            const int c5 = fdiv_q(q, f_nxc), xc = q - c5 * nxc;
                            const int i = s6_index(sd1, i1, k5lo + 2 * c5, xc0 + 2 * xc);
                            if constexpr (PQ) cp_async8(s1f + q, v.Sff[0] + (i < 0 ? 0 : sd1.off + i), i < 0 ? 0 : 8);
                            else cp_async8(sm.S1s + q, v.S1x + (i < 0 ? 0 : sd1.off + i), i < 0 ? 0 : 8);
                        }
                        cp_async_wait_all();
                        __syncthreads();
                        for (int q = tid; q < D * mdk * nxc; q += nth) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, d = fdiv_q(r, f_mdk), c2 = r - d * mdk;
                            if (c2 >= s_nk2[d]) continue;
                            if constexpr (D64) {
                                double* e = sm.SB + (d * mdk + c2) * XC + xc;
                                *e = reinterpret_cast<const double*>(sm.B2s)[d * mdk + c2] * *e;
                            } else {
                                float* e = sbf + (d * mdk + c2) * XC + xc;
                                *e = sm.B2s[d * mdk + c2] * *e;
                            }
                        }
                        for (int q = tid; q < nk5 * nk4 * nxc; q += nth) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, c5 = fdiv_q(r, f_nk4);
                            if constexpr (PQ) qf[q] = ff_mul_f(ff_mul(s1f[c5 * nxc + xc], qf[q]), (float)(xc0 + 2 * xc + 1));
                            else sm.Q[q] = sm.S1s[c5 * nxc + xc] * sm.Q[q];
                        }
                    } else {
                    {
                        // SB: gather (B2 entry, S5 entry) pairs, then scale and store
                        auto sb_at = [&](int q, int& d, int& c2, int& xc) {
                            const int r = fdiv_q(q, f_nxc);
                            xc = q - r * nxc;
                            d = fdiv_q(r, f_mdk);
                            c2 = r - d * mdk;
                        };
                        using T2 = typename std::conditional<F32IN, float2, double2>::type;
                        gather_loop<GU>(D * mdk * nxc, tid, nth, [&](int q) {
                            int d, c2, xc;
                            sb_at(q, d, c2, xc);
                            T2 val;
                            val.x = 0; val.y = 0;
                            if (c2 < s_nk2[d]) {
                                const int k2 = s_k2lo[d] + 2 * c2, x = xc0 + 2 * xc;
                                const int64_t bi = ((int64_t)((d * D + d24) * D + d25) * v.di[1] + ci2) * v.dkmax[0] + c2;
                                if constexpr (F32IN) {
                                    val.x = __ldg(v.Bf[0] + bi);
                                    val.y = s6f(v.S5f, sd5, k2, i1, x);
                                } else {
                                    val.x = __ldg(v.B[0] + bi);
                                    val.y = s6(v.S[4], sd5, k2, i1, x);
                                }
                            }
                            return val;
                        }, [&](int q, T2 val) {
                            int d, c2, xc;
                            sb_at(q, d, c2, xc);
                            if (c2 >= s_nk2[d]) return;
                            const int k2 = s_k2lo[d] + 2 * c2;
                            if constexpr (F32IN) {
                                const float f = (float)(k2 + 1) * ((c2 & 1) ? -s_sigf[d] : s_sigf[d]);
                                reinterpret_cast<float*>(sm.SB)[(d * mdk + c2) * XC + xc] = (f * val.x) * val.y;
                            } else {
                                const double f = (double)(k2 + 1) * ((c2 & 1) ? -s_sig[d] : s_sig[d]);
                                const double sb = f * val.x * val.y;
                                if constexpr (MIX) reinterpret_cast<float*>(sm.SB)[(d * mdk + c2) * XC + xc] = (float)sb;
                                else sm.SB[(d * mdk + c2) * XC + xc] = sb;
                            }
                        });
                    }
                    // S3s[x][k4][k3u] from the S3 slot, read along x (contiguous in the table) and
                    // stored transposed
                    {
                        auto s3_at = [&](int q, int& xc, int& c4, int& ku) {
                            const int r = fdiv_q(q, f_nxc);
                            xc = q - r * nxc;
                            c4 = fdiv_q(r, f_nk3u);
                            ku = r - c4 * nk3u;
                        };
                        if constexpr (TC || PX) {
                            gather_loop<4>(nxc * nk4 * nk3u, tid, nth, [&](int q) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                return s6ff(v.Sff[2], sd3, k4lo + 2 * c4, k3ulo + 2 * ku, xc0 + 2 * xc).x;
                            }, [&](int q, float val) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                reinterpret_cast<float*>(sm.S3s)[(xc * nk4 + c4) * nk3u + ku] = val;
                            });
                        } else if constexpr (FF) {
                            gather_loop<4>(nxc * nk4 * nk3u, tid, nth, [&](int q) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                return s6ff(v.Sff[2], sd3, k4lo + 2 * c4, k3ulo + 2 * ku, xc0 + 2 * xc);
                            }, [&](int q, float2 val) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                reinterpret_cast<float2*>(sm.S3s)[(xc * nk4 + c4) * nk3u + ku] = val;
                            });
                        } else {
                            gather_loop<GU>(nxc * nk4 * nk3u, tid, nth, [&](int q) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                return s6(v.S[2], sd3, k4lo + 2 * c4, k3ulo + 2 * ku, xc0 + 2 * xc);
                            }, [&](int q, double val) {
                                int xc, c4, ku;
                                s3_at(q, xc, c4, ku);
                                sm.S3s[(xc * nk4 + c4) * nk3u + ku] = val;
                            });
                        }
                    }
                    // E: Q[k5][k4][x] = (2x+1) S1[i1,k5,x] S2[k5,k4,x]
                    if constexpr (FF || PX) {
                        gather_loop<4>(nk5 * nk4 * nxc, tid, nth, [&](int q) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, c5 = fdiv_q(r, f_nk4), c4 = r - c5 * nk4;
                            const int k5 = k5lo + 2 * c5, k4 = k4lo + 2 * c4, x = xc0 + 2 * xc;
                            const float2 a = s6ff(v.Sff[0], sd1, i1, k5, x), b = s6ff(v.Sff[1], sd2, k5, k4, x);
                            return make_float4(a.x, a.y, b.x, b.y);
                        }, [&](int q, float4 val) {
                            const int x = xc0 + 2 * (q - fdiv_q(q, f_nxc) * nxc);
                            reinterpret_cast<float2*>(sm.Q)[q] =
                                ff_mul_f(ff_mul(make_float2(val.x, val.y), make_float2(val.z, val.w)), (float)(x + 1));
                        });
                    } else {
                        // (2x+1) S1 comes from the prescaled copy S1x: the same rounding as forming
                        // (x+1) * S1 here, so Q is bitwise the product ((x+1) S1) S2
                        gather_loop<GU>(nk5 * nk4 * nxc, tid, nth, [&](int q) {
                            const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, c5 = fdiv_q(r, f_nk4), c4 = r - c5 * nk4;
                            const int k5 = k5lo + 2 * c5, k4 = k4lo + 2 * c4, x = xc0 + 2 * xc;
                            return make_double2(s6(v.S1x, sd1, i1, k5, x), s6(v.S[1], sd2, k5, k4, x));
                        }, [&](int q, double2 val) {
                            sm.Q[q] = val.x * val.y;
                        });
                    }
                    }
                    __syncthreads();
                    // B: R[d][k3][x] = (2k3+1)(-1)^(k3-k3lo) sum_k2 S4_d[k3,k2,x] SB[d][k2][x]
                    for (int q = tid; q < D * mdk * nxc; q += nth) {
                        const int r = fdiv_q(q, f_nxc), xc = q - r * nxc, d = fdiv_q(r, f_mdk), c3 = r - d * mdk;
                        const int nk3 = s_nk3[d];
                        if (c3 >= nk3) continue;
                        const int k3 = s_k3lo[d] + 2 * c3, x = xc0 + 2 * xc;
                        const SlotDesc sd4 = s_sd4[d];
                        const int k2lo = s_k2lo[d], nk2 = s_nk2[d];
                        // the k3 and k2 ranges lie inside the slot box; only x can fall outside it
                        const int ia = (k3 - sd4.alo) >> 1, ix = (x - sd4.xlo) >> 1, ib0 = (k2lo - sd4.blo) >> 1;
                        const bool inbox = (unsigned)ix < (unsigned)sd4.nx && ((x - sd4.xlo) & 1) == 0;
                        const double* s4p = v.S[3] + sd4.off + ((int64_t)ia * sd4.nb + ib0) * sd4.nx + ix;
                        if constexpr (MIX) {
                            const float sgn3 = (float)(k3 + 1) * ((c3 & 1) ? -1.0f : 1.0f);
                            const float* sbp = reinterpret_cast<const float*>(sm.SB) + (d * mdk) * XC + xc;
                            // the FP32 copy of S4 holds the same roundings as converting each entry here
                            const float* s4f = v.S4f + sd4.off + ((int64_t)ia * sd4.nb + ib0) * sd4.nx + ix;
                            float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
                            if (inbox) {
                                const int nx = sd4.nx;
                                int c2 = 0;
                                for (; c2 + 3 < nk2; c2 += 4) {   // four loads in flight
                                    const float s0 = __ldg(s4f + c2 * nx), s1 = __ldg(s4f + (c2 + 1) * nx);
                                    const float s2 = __ldg(s4f + (c2 + 2) * nx), s3 = __ldg(s4f + (c2 + 3) * nx);
                                    acc0 = fmaf(s0, sbp[c2 * XC], acc0);
                                    acc1 = fmaf(s1, sbp[(c2 + 1) * XC], acc1);
                                    acc2 = fmaf(s2, sbp[(c2 + 2) * XC], acc2);
                                    acc3 = fmaf(s3, sbp[(c2 + 3) * XC], acc3);
                                }
                                for (; c2 < nk2; c2++) acc0 = fmaf(__ldg(s4f + c2 * nx), sbp[c2 * XC], acc0);
                            }
                            reinterpret_cast<float*>(sm.R)[(d * mdk + c3) * XC + xc] = ((acc0 + acc1) + (acc2 + acc3)) * sgn3;
                        } else {
                            const double sgn3 = (double)(k3 + 1) * ((c3 & 1) ? -1.0 : 1.0);
                            const double* sbp = sm.SB + (d * mdk) * XC + xc;
                            double acc0 = 0.0, acc1 = 0.0;
                            if (inbox) {
                                int c2 = 0;
                                for (; c2 + 1 < nk2; c2 += 2) {
                                    acc0 = fma(__ldg(s4p + (int64_t)c2 * sd4.nx), sbp[c2 * XC], acc0);
                                    acc1 = fma(__ldg(s4p + (int64_t)(c2 + 1) * sd4.nx), sbp[(c2 + 1) * XC], acc1);
                                }
                                if (c2 < nk2) acc0 = fma(__ldg(s4p + (int64_t)c2 * sd4.nx), sbp[c2 * XC], acc0);
                            }
                            sm.R[(d * mdk + c3) * XC + xc] = (acc0 + acc1) * sgn3;
                        }
                    }
                    __syncthreads();
                    // C: U[k3u][x][i3] = sum_d R[d][k3][x] B3_d[i3][k3]   (4 consecutive i3 per thread)
                    {
                        const int nb3 = (di3 + 3) / 4;
                        const FDiv f_nb3 = fdiv_make(nb3);
                        for (int q = tid; q < nk3u * nxc * nb3; q += nth) {
                            const int r = fdiv_q(q, f_nb3), b = q - r * nb3, ku = fdiv_q(r, f_nxc), xc = r - ku * nxc;
                            const int i30 = 4 * b;
                            double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
                            if constexpr (MIX) {
                                const float* Rf = reinterpret_cast<const float*>(sm.R);
                                const float* Bf = reinterpret_cast<const float*>(sm.B3s);
                                float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f, f3 = 0.0f;
#pragma unroll 2
                                for (int d = 0; d < D; d++) {
                                    const int2 cn = s_c3n[d];
                                    const int c3 = ku + cn.x;
                                    if ((unsigned)c3 >= (unsigned)cn.y) continue;
                                    const float rr = Rf[(d * mdk + c3) * XC + xc];
                                    const float* bp = Bf + (d * mdk + c3) * di3 + i30;
                                    f0 = fmaf(rr, bp[0], f0);
                                    if (i30 + 1 < di3) f1 = fmaf(rr, bp[1], f1);
                                    if (i30 + 2 < di3) f2 = fmaf(rr, bp[2], f2);
                                    if (i30 + 3 < di3) f3 = fmaf(rr, bp[3], f3);
                                }
                                if constexpr (F32IN) {
                                    float* up = reinterpret_cast<float*>(sm.U) + (ku * nxc + xc) * di3 + i30;
                                    up[0] = f0;
                                    if (i30 + 1 < di3) up[1] = f1;
                                    if (i30 + 2 < di3) up[2] = f2;
                                    if (i30 + 3 < di3) up[3] = f3;
                                    continue;
                                }
                                a0 = f0; a1 = f1; a2 = f2; a3 = f3;
                            } else {
#pragma unroll 2
                                for (int d = 0; d < D; d++) {
                                    const int2 cn = s_c3n[d];
                                    const int c3 = ku + cn.x;
                                    if ((unsigned)c3 >= (unsigned)cn.y) continue;
                                    const double rr = sm.R[(d * mdk + c3) * XC + xc];
                                    const double* bp = sm.B3s + (d * mdk + c3) * di3 + i30;
                                    a0 = fma(rr, bp[0], a0);
                                    if (i30 + 1 < di3) a1 = fma(rr, bp[1], a1);
                                    if (i30 + 2 < di3) a2 = fma(rr, bp[2], a2);
                                    if (i30 + 3 < di3) a3 = fma(rr, bp[3], a3);
                                }
                            }
                            double* up = sm.U + (ku * nxc + xc) * di3 + i30;
                            up[0] = a0;
                            if (i30 + 1 < di3) up[1] = a1;
                            if (i30 + 2 < di3) up[2] = a2;
                            if (i30 + 3 < di3) up[3] = a3;
                        }
                    }
                    __syncthreads();
                    // D: P[k4][x][i3] = sum_k3u S3s[x][k4][k3u] U[k3u][x][i3]        (batch over x)
                    if constexpr (FF)
                        rows_gemm<GEMM_FF_D, 2>(nxc, nk4, di3, nk3u, sm.S3s, nk4 * nk3u, nk3u, sm.U, di3, nxc * di3,
                                                sm.P, di3, nxc * di3, tid, nth);
                    else if constexpr (PX)
                        rows_gemm<GEMM_F32_SETF, 2>(nxc, nk4, di3, nk3u, sm.S3s, nk4 * nk3u, nk3u, sm.U, di3, nxc * di3,
                                                    sm.P, di3, nxc * di3, tid, nth);
                    else if constexpr (TC)
                        rows_gemm<GEMM_F32_SET, 2>(nxc, nk4, di3, nk3u, sm.S3s, nk4 * nk3u, nk3u, sm.U, di3, nxc * di3,
                                                   sm.P, di3, nxc * di3, tid, nth);
                    else
                        flat_gemm<double, false>(nxc, nk4, di3, nk3u, sm.S3s, nk4 * nk3u, nk3u, 1, sm.U, di3, nxc * di3, 1,
                                                 sm.P, di3, nxc * di3, 1, tid, nth);
                    __syncthreads();
                    // F: V[k4][k5][i3] += sum_x Q[k5][k4][x] P[k4][x][i3]             (batch over k4)
                    if constexpr (FF)
                        rows_gemm<GEMM_FF_F, 2>(nk4, nk5, di3, nxc, sm.Q, nxc, nk4 * nxc, sm.P, nxc * di3, di3, sm.V,
                                                nk5 * di3, di3, tid, nth);
                    else if constexpr (PX)
                        rows_gemm<GEMM_FF_DA, 2>(nk4, nk5, di3, nxc, sm.Q, nxc, nk4 * nxc, sm.P, nxc * di3, di3, sm.V,
                                                 nk5 * di3, di3, tid, nth);
                    else
                        flat_gemm<double, true>(nk4, nk5, di3, nxc, sm.Q, nxc, nk4 * nxc, 1, sm.P, nxc * di3, di3, 1,
                                                sm.V, nk5 * di3, di3, 1, tid, nth);
                }
                __syncthreads();
                // G: Y[i4][k5][i3] += sum_k4 B4'[i4][k4] V[k4][k5][i3]             (batch over k5)
                if constexpr (TC) {
                    // on the tensor cores: C[m = (k5, i3)][n = i4] = sum_k4 V[k4][m] B4'[n][k4], V^T split
                    // into BF16 planes over the (now free) chunk buffers, the FP32 result added to Y
                    const int Mv = nk5 * di3, ks = tc_ks(mdk), Mp = (Mv + 15) & ~15, Kp2 = ((nk4 + 15) & ~15) / 2;
                    const int pl = (Mp * ks) / 2;   // one plane, in 32-bit words
                    for (int q = tid; q < Mp * Kp2; q += nth) {
                        const int kk = q / Mp, m = q - kk * Mp, k0 = 2 * kk;
                        const float w0 = (m < Mv && k0 < nk4) ? (float)sm.V[k0 * Mv + m] : 0.0f;
                        const float w1 = (m < Mv && k0 + 1 < nk4) ? (float)sm.V[(k0 + 1) * Mv + m] : 0.0f;
                        unsigned short a0, a1, a2, b0, b1, b2;
                        split3_bf16(w0, a0, a1, a2);
                        split3_bf16(w1, b0, b1, b2);
                        uint32_t* dst = reinterpret_cast<uint32_t*>(sm.Ap + m * ks + k0);
                        dst[0] = (uint32_t)a0 | ((uint32_t)b0 << 16);
                        dst[pl] = (uint32_t)a1 | ((uint32_t)b1 << 16);
                        dst[2 * pl] = (uint32_t)a2 | ((uint32_t)b2 << 16);
                    }
                    __syncthreads();
                    tc_gemm_acc(sm.Ap, sm.Bp, Mv, di4, nk4, ks, sm.Y, tid, nth);
                } else if constexpr (MIX) {
                    for (int q = tid; q < nk4 * nk5 * di3; q += nth) {
                        if constexpr (FF || PX) {
                            const float2 vv = reinterpret_cast<const float2*>(sm.V)[q];
                            sm.Vf[q] = vv.x + vv.y;
                        } else {
                            sm.Vf[q] = (float)sm.V[q];
                        }
                    }
                    if constexpr (!FF && !PX) for (int q = tid; q < di4 * nk4; q += nth) sm.B4f[q] = (float)sm.B4[q];
                    __syncthreads();
                    rows_gemm<FF ? GEMM_F32_FF : GEMM_F32, 2>(nk5, di4, di3, nk4, sm.B4f, 0, nk4, sm.Vf, di3, nk5 * di3,
                                                              sm.Y, di3, nk5 * di3, tid, nth);
                } else {
                    flat_gemm<double, true>(nk5, di4, di3, nk4, sm.B4, 0, nk4, 1, sm.V, di3, nk5 * di3, 1,
                                         sm.Y, di3, nk5 * di3, 1, tid, nth);
                }
            }
            if (!gany) continue;
            __syncthreads();
            if constexpr (FF) {   // the group's pair sums Y to FP64, in place (each thread its own entries)
                for (int q = tid; q < di4 * nk5 * di3; q += nth) {
                    const float2 y = reinterpret_cast<const float2*>(sm.Y)[q];
                    sm.Y[q] = (double)y.x + (double)y.y;
                }
                __syncthreads();
            }
            // H: T[i4][i5][i3] += sum_k5 B5'[i5][k5] Y[i4][k5][i3]   (register-resident output tile)
#pragma unroll
            for (int rr = 0; rr < TRT; rr++) {
                const int b = tid + rr * nth;
                if (b < di4 * tper) {
                    const int i4 = b / tper, r = b - i4 * tper;
                    const int m0 = (r / tb3) * 2, n0 = (r - (r / tb3) * tb3) * 4;
                    for (int c5 = 0; c5 < nk5; c5++) {
                        double a[2], y[4];
#pragma unroll
                        for (int i = 0; i < 2; i++) a[i] = (m0 + i < di5) ? sm.B5[(m0 + i) * nk5 + c5] : 0.0;
#pragma unroll
                        for (int j = 0; j < 4; j++) y[j] = (n0 + j < di3) ? sm.Y[(i4 * nk5 + c5) * di3 + n0 + j] : 0.0;
#pragma unroll
                        for (int i = 0; i < 2; i++)
#pragma unroll
                            for (int j = 0; j < 4; j++) T[rr][i][j] = fma(a[i], y[j], T[rr][i][j]);
                    }
                }
            }
        }
        if (w.single) {
            // one shell's contribution: the squared 2-norm of its output tile, with the factors
            // prod_e sqrt(2 i_e + 1) that the reduction applies (the sign does not matter here)
            const double s12 = (double)(v.ilo[0] + 2 * w.i1 + 1) * (double)(v.ilo[1] + 2 * w.i2 + 1);
            double q2 = 0.0;
#pragma unroll
            for (int rr = 0; rr < TRT; rr++) {
                const int b = tid + rr * nth;
                if (b < di4 * tper) {
                    const int i4 = b / tper, r = b - i4 * tper;
                    const int m0 = (r / tb3) * 2, n0 = (r - (r / tb3) * tb3) * 4;
#pragma unroll
                    for (int i = 0; i < 2; i++)
#pragma unroll
                        for (int j = 0; j < 4; j++)
                            if (m0 + i < di5 && n0 + j < di3) {
                                const double f = (double)(v.ilo[2] + 2 * (i3b + n0 + j) + 1) *
                                                 (double)(v.ilo[3] + 2 * (o4 + i4) + 1) *
                                                 (double)(v.ilo[4] + 2 * (o5 + m0 + i) + 1);
                                q2 = fma(f * T[rr][i][j], T[rr][i][j], q2);
                            }
                }
            }
            for (int off = 16; off > 0; off >>= 1) q2 += __shfl_xor_sync(0xffffffffu, q2, off);
            __syncthreads();   // the chunk buffers are free: reuse the first NT / 32 doubles
            if ((tid & 31) == 0) smem[tid >> 5] = q2;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int q = 0; q < NT / 32; q++) tot += smem[q];
                part[w.part_off] = s12 * tot;
            }
            continue;
        }
        // partial tile in [i3][i4][i5] order
        double* out = part + w.part_off;
#pragma unroll
        for (int rr = 0; rr < TRT; rr++) {
            const int b = tid + rr * nth;
            if (b < di4 * tper) {
                const int i4 = b / tper, r = b - i4 * tper;
                const int m0 = (r / tb3) * 2, n0 = (r - (r / tb3) * tb3) * 4;
#pragma unroll
                for (int i = 0; i < 2; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++)
                        if (m0 + i < di5 && n0 + j < di3) out[((n0 + j) * di4 + i4) * di5 + m0 + i] = T[rr][i][j];
            }
        }
    }
}

template <int MODE, int NT>
static const void* shell_fn() { return (const void*)k_shell<MODE, NT>; }

static const void* shell_kernel(int mode, int nt) {
    if (nt == 1024) return mode == 4 ? shell_fn<4, 1024>() : nullptr;
    if (nt == 256)
        return mode == 4 ? shell_fn<4, 256>() : mode == 3 ? shell_fn<3, 256>() : mode == 2 ? shell_fn<2, 256>() : mode == 1 ? shell_fn<1, 256>() : shell_fn<0, 256>();
    return mode == 4 ? shell_fn<4, 512>() : mode == 3 ? shell_fn<3, 512>() : mode == 2 ? shell_fn<2, 512>() : mode == 1 ? shell_fn<1, 512>() : shell_fn<0, 512>();
}

int sf_shell_prepare(int mode, int nt, int mdi, int mdk, int mk3u, int xc, int Dmax, int mni3, int n_items, int num_sms,
                     int* grid, size_t* smem) {
    if (nt != 256 && nt != 512 && !(nt == 1024 && mode == 4))
        return sf_set_error(SF_ERR_ARG, "shell kernel runs 256 or 512 threads per CTA (1024 in mode 4), not %d", nt);
    if (mode < 0 || mode > 4) return sf_set_error(SF_ERR_ARG, "unknown shell-kernel mode %d", mode);
    const size_t bytes = sf_shell_smem_doubles(mdi, mdk, mk3u, xc, Dmax, mni3, mode) * sizeof(double);
    if (bytes > 200 * 1024) return sf_set_error(SF_ERR_LIMIT, "shell kernel needs %zu bytes of shared memory", bytes);
    const void* fn = shell_kernel(mode, nt);
    SF_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    int per_sm = 0;
    SF_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, bytes));
    if (per_sm < 1) per_sm = 1;
    int g = num_sms * per_sm;
    if (g > n_items) g = n_items;
    *grid = g < 1 ? 1 : g;
    *smem = bytes;
    return SF_OK;
}

int sf_shell_launch_prepared(int mode, int nt, int grid, size_t smem, const VtxDev* d_v, int mdi, int mdk, int mk3u,
                             int xc, int Dmax, int mni3, const WorkItem* d_items, int n_items, int* d_counter,
                             double* d_part, ShellFilter filt, cudaStream_t s) {
    SF_CUDA_TRY(cudaMemsetAsync(d_counter, 0, sizeof(int), s));
#define SF_SHELL_GO(M, N)                                                                                     \
    k_shell<M, N><<<grid, N, smem, s>>>(d_v, mdi, mdk, mk3u, xc, Dmax, mni3, d_items, n_items, d_counter, d_part, filt)
    if (mode < 0 || mode > 4) return sf_set_error(SF_ERR_ARG, "unknown shell-kernel mode %d", mode);
    if (nt == 1024) {
        if (mode != 4) return sf_set_error(SF_ERR_ARG, "1024 threads per CTA run mode 4 only");
        SF_SHELL_GO(4, 1024);
    } else if (nt == 256) {
        if (mode == 4) SF_SHELL_GO(4, 256);
        else if (mode == 3) SF_SHELL_GO(3, 256);
        else if (mode == 2) SF_SHELL_GO(2, 256);
        else if (mode == 1) SF_SHELL_GO(1, 256);
        else SF_SHELL_GO(0, 256);
    } else {
        if (mode == 4) SF_SHELL_GO(4, 512);
        else if (mode == 3) SF_SHELL_GO(3, 512);
        else if (mode == 2) SF_SHELL_GO(2, 512);
        else if (mode == 1) SF_SHELL_GO(1, 512);
        else SF_SHELL_GO(0, 512);
    }
#undef SF_SHELL_GO
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

int sf_shell_fp64_launch(const VtxDev* d_v, int mdi, int mdk, int mk3u, int xc, int Dmax, const WorkItem* d_items,
                         int n_items, int* d_counter, double* d_part, ShellFilter filt, int num_sms, cudaStream_t s) {
    int grid = 0;
    size_t smem = 0;
    SF_TRY(sf_shell_prepare(0, 512, mdi, mdk, mk3u, xc, Dmax, mdi, n_items, num_sms, &grid, &smem));
    return sf_shell_launch_prepared(0, 512, grid, smem, d_v, mdi, mdk, mk3u, xc, Dmax, mdi, d_items, n_items,
                                    d_counter, d_part, filt, s);
}

// A[i1][i2][i3][i4][i5] = (-1)^(n_i1) prod_e sqrt(2 i_e + 1) * sum_{chunks} part[tile, chunk][i3][i4][i5]
// items of one vertex are laid out tile-major with `nchunk` consecutive items per tile
__global__ void k_reduce(const VtxDev* __restrict__ V, int vtx, const WorkItem* __restrict__ items, int item0,
                         int nchunk, const double* __restrict__ part, double* __restrict__ A) {
    const VtxDev& v = V[vtx];
    const int tile = blockIdx.x;
    const int ci1 = v.olo[0] + tile / v.od[1], ci2 = v.olo[1] + tile % v.od[1];
    const int n3 = v.od[2] * v.od[3] * v.od[4];
    const double s12 = sqrt((double)(v.ilo[0] + 2 * ci1 + 1)) * sqrt((double)(v.ilo[1] + 2 * ci2 + 1)) *
                       ((ci1 & 1) ? -1.0 : 1.0);
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < nchunk; c++) acc += part[items[item0 + tile * nchunk + c].part_off + q];
        const int c5 = v.olo[4] + q % v.od[4], c4 = v.olo[3] + (q / v.od[4]) % v.od[3],
                  c3 = v.olo[2] + q / (v.od[4] * v.od[3]);
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

// the same reduction for many vertices in one launch: one CTA per (output tile, i3 range)
__global__ void k_reduce_jobs(const VtxDev* __restrict__ V, const ReduceJob* __restrict__ jobs,
                              const WorkItem* __restrict__ items, const double* __restrict__ part) {
    const ReduceJob jb = jobs[blockIdx.x];
    const VtxDev& v = V[jb.vtx];
    const int ci1 = v.olo[0] + jb.tile / v.od[1], ci2 = v.olo[1] + jb.tile % v.od[1];
    const int n3 = jb.ni3 * v.od[3] * v.od[4];
    const double s12 = sqrt((double)(v.ilo[0] + 2 * ci1 + 1)) * sqrt((double)(v.ilo[1] + 2 * ci2 + 1)) *
                       ((ci1 & 1) ? -1.0 : 1.0);
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < jb.nchunk; c++) acc += part[items[jb.item0 + c * jb.stride].part_off + q];
        const int c5 = v.olo[4] + q % v.od[4], c4 = v.olo[3] + (q / v.od[4]) % v.od[3],
                  c3 = jb.i3b + q / (v.od[4] * v.od[3]);
        const double s = s12 * sqrt((double)(v.ilo[2] + 2 * c3 + 1)) * sqrt((double)(v.ilo[3] + 2 * c4 + 1)) *
                         sqrt((double)(v.ilo[4] + 2 * c5 + 1));
        jb.A[q] = s * acc;
    }
}

int sf_reduce_jobs_launch(const VtxDev* d_v, const ReduceJob* d_jobs, int njobs, const WorkItem* d_items,
                          const double* d_part, cudaStream_t s) {
    if (njobs <= 0) return SF_OK;
    k_reduce_jobs<<<njobs, 256, 0, s>>>(d_v, d_jobs, d_items, d_part);
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
