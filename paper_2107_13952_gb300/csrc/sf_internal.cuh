// Internal declarations shared by the CUDA translation units of the EPRL vertex library.
// Everything here is device/host plumbing for the kernels behind include/sf_eprl.h.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstdarg>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/sf_eprl.h"

// ----------------------------------------------------------------------------------------------
// limits (checked on the host before any launch)
// ----------------------------------------------------------------------------------------------
#define SF_FACT_MAX 170        // factorials up to 170! fit in a double exponent
#define SF_BI_LIMBS 24         // 768-bit magnitudes for the exact Racah sums
#define SF_RACAH_MAX 250       // every integer Racah argument (z+1, beta-z, ...) stays below 256
#define SF_MAX_DL 40           // shells per face (dl+1) handled by one d-table pass set
#define SF_DT_LCHUNK 12        // l values accumulated per d-table pass
#define SF_GL_NMAX 1024        // largest Gauss-Legendre rule of the library (composite rules beyond)
#define SF_MAX_DEVICES 128     // device ordinals with process-wide caches

// ----------------------------------------------------------------------------------------------
// error reporting (thread-local message, set by the host side of every entry point)
// ----------------------------------------------------------------------------------------------
int sf_set_error(int code, const char* fmt, ...);
void sf_note_launch(int n);   // launch counter behind sf_kernel_launches()

#define SF_TRY(x) do { int r_ = (x); if (r_ != SF_OK) return r_; } while (0)

#define SF_CUDA_TRY(call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sf_set_error(e_ == cudaErrorMemoryAllocation ? SF_ERR_OOM : SF_ERR_CUDA,    \
                                "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                                __FILE__, __LINE__);                                           \
    } while (0)

// status word written by kernels (first error wins)
#define SF_DEV_OK 0
#define SF_DEV_BIGINT_OVERFLOW 1
#define SF_DEV_NONREAL_BOOSTER 2
#define SF_DEV_BAD_INDEX 3
#define SF_DEV_TIMEOUT 4

// ----------------------------------------------------------------------------------------------
// small helpers on doubled spins (host + device)
// ----------------------------------------------------------------------------------------------
__host__ __device__ inline int iabs_(int a) { return a < 0 ? -a : a; }
__host__ __device__ inline int imin_(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int imax_(int a, int b) { return a > b ? a : b; }

__host__ __device__ inline bool sf_tri(int a, int b, int c) {
    return iabs_(a - b) <= c && c <= a + b && ((a + b + c) & 1) == 0;
}

// Range of an intertwiner coupling the pair (a,b) to the pair (c,d): doubled lo and count (0 if empty).
__host__ __device__ inline void sf_pair_range(int a, int b, int c, int d, int* lo, int* n) {
    if ((a + b + c + d) & 1) { *lo = 0; *n = 0; return; }
    int l = imax_(iabs_(a - b), iabs_(c - d));
    int h = imin_(a + b, c + d);
    *lo = l;
    *n = (h >= l) ? (h - l) / 2 + 1 : 0;
}

// ----------------------------------------------------------------------------------------------
// double-double arithmetic: error-free transformations of Dekker and Knuth as used by
// Hida, Li and Bailey's double-double library (published algorithms, written out here)
// ----------------------------------------------------------------------------------------------
struct dd { double hi, lo; };

__host__ __device__ inline dd dd_make(double a) { return dd{a, 0.0}; }
__host__ __device__ inline dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return dd{s, e};
}
__host__ __device__ inline dd quick_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return dd{s, e};
}
__host__ __device__ inline dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return dd{p, e};
}
__host__ __device__ inline dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__host__ __device__ inline dd dd_neg(dd a) { return dd{-a.hi, -a.lo}; }
__host__ __device__ inline dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
__host__ __device__ inline dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}
__host__ __device__ inline dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_add(a, dd_neg(dd_mul_d(b, q1)));
    double q2 = r.hi / b.hi;
    r = dd_add(r, dd_neg(dd_mul_d(b, q2)));
    double q3 = r.hi / b.hi;
    dd q = quick_two_sum(q1, q2);
    return dd_add(q, dd_make(q3));
}
__host__ __device__ inline dd dd_sqrt(dd a) {
    if (a.hi <= 0.0) return dd{0.0, 0.0};
    double x = sqrt(a.hi);
    dd x2 = two_prod(x, x);
    dd r = dd_add(a, dd_neg(x2));
    double c = r.hi / (2.0 * x);
    return quick_two_sum(x, c);
}
__host__ __device__ inline double dd_to_d(dd a) { return a.hi + a.lo; }

// ----------------------------------------------------------------------------------------------
// exact unsigned big integers for the Racah sums (limbs of 32 bits, little-endian, fixed
// capacity NL, loops fully unrolled so that the limbs live in registers)
template <int NL> struct BigUT { uint32_t w[NL]; };
using BigU = BigUT<SF_BI_LIMBS>;

template <int NL> __device__ inline void bi_zero(BigUT<NL>& a) {
#pragma unroll
    for (int i = 0; i < NL; i++) a.w[i] = 0u;
}
template <int NL> __device__ inline void bi_set(BigUT<NL>& a, uint32_t v) { bi_zero(a); a.w[0] = v; }
// a *= m; returns the carry out of the top limb (non-zero means overflow)
template <int NL> __device__ inline uint32_t bi_mul(BigUT<NL>& a, uint32_t m) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t t = (uint64_t)a.w[i] * m + c;
        a.w[i] = (uint32_t)t;
        c = t >> 32;
    }
    return (uint32_t)c;
}
// a /= d for a divisor d >= 1 that divides a exactly (quotient by reciprocal multiplication:
// q = mulhi(cur, floor((2^64-1)/d)) is q_true or q_true - 1 because cur < 2^64)
template <int NL> __device__ inline void bi_divexact(BigUT<NL>& a, uint32_t d) {
    const uint64_t M = 0xFFFFFFFFFFFFFFFFull / d;
    uint64_t rem = 0;
#pragma unroll
    for (int i = NL - 1; i >= 0; i--) {
        uint64_t cur = (rem << 32) | a.w[i];
        uint64_t q = __umul64hi(cur, M);
        uint64_t r = cur - q * d;
        if (r >= d) { q++; r -= d; }
        a.w[i] = (uint32_t)q;
        rem = r;
    }
}
template <int NL> __device__ inline uint32_t bi_add(BigUT<NL>& a, const BigUT<NL>& b) {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        uint64_t t = (uint64_t)a.w[i] + b.w[i] + c;
        a.w[i] = (uint32_t)t;
        c = t >> 32;
    }
    return (uint32_t)c;
}
// compare: -1, 0, 1
template <int NL> __device__ inline int bi_cmp(const BigUT<NL>& a, const BigUT<NL>& b) {
    int r = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        if (a.w[i] != b.w[i]) r = (a.w[i] > b.w[i]) ? 1 : -1;   // the highest differing limb wins
    }
    return r;
}
// a -= b, requires a >= b
template <int NL> __device__ inline void bi_sub(BigUT<NL>& a, const BigUT<NL>& b) {
    int64_t br = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
        int64_t t = (int64_t)a.w[i] - (int64_t)b.w[i] - br;
        br = (t < 0) ? 1 : 0;
        a.w[i] = (uint32_t)(t + (br << 32));
    }
}
// value as double-double (top 128 bits, exact up to the dd rounding of the sum)
template <int NL> __device__ inline dd bi_to_dd(const BigUT<NL>& a) {
    int top = -1;
#pragma unroll
    for (int i = 0; i < NL; i++) if (a.w[i]) top = i;
    if (top < 0) return dd{0.0, 0.0};
    dd acc{0.0, 0.0};
    for (int i = top; i >= 0 && i > top - 4; i--) {
        acc = dd_add(acc, dd_make(ldexp((double)a.w[i], 32 * i)));
    }
    return acc;
}

// ----------------------------------------------------------------------------------------------
// device-side descriptors
// ----------------------------------------------------------------------------------------------
// one slot (fixed virtual spins) of a {6j} table: a dense box over (a, b, x), doubled lows
struct SlotDesc {
    int64_t off;
    int32_t alo, blo, xlo, na, nb, nx;
};

// per-vertex parameters visible to kernels
struct VtxDev {
    int32_t tj[10];
    double gamma;
    int32_t dl, D;             // D = dl + 1
    int32_t ilo[5], di[5];     // intertwiner ranges
    int32_t olo[5], od[5];     // output sub-range per edge: first index within the range, count
    int64_t nshell;            // D^6
    const double* S[5];        // {6j} tables S1..S5
    const double* S1x;         // S1 times the x-sum weight (2x+1), rounded once (FP64 paths)
    const float* S4f;          // S4 rounded to FP32 once (mixed paths)
    const float* S5f;          // S5 rounded to FP32 once (SF_MIXED_FF)
    const float2* Sff[3];      // S1, S2, S3 as (hi, lo) float pairs, hi + lo = S to about 2^-48 (SF_MIXED_FF)
    const SlotDesc* slot[5];
    const double* B[4];        // boosters of edges 2..5: [t][i][k - klo(t)], padded to dkmax
    const float* Bf[4];        // the same boosters rounded to FP32 (SF_MIXED_FF)
    const int32_t* klo[4];
    int32_t dkmax[4];
    int64_t ntrip;             // D^3
    const double2* dtab[10];   // d-tables per face [il][im][n]
    int32_t nl[10];            // l values per face (D for free faces, 1 for gauge faces)
};

// face index helpers (order j12 j13 j14 j15 j23 j24 j25 j34 j35 j45)
enum { F12 = 0, F13, F14, F15, F23, F24, F25, F34, F35, F45 };

// ----------------------------------------------------------------------------------------------
// shell-sum scheduling records
// ----------------------------------------------------------------------------------------------
struct WorkItem {              // output tile (i1, i2), i3 in [i3b, i3b + ni3), of one vertex, over groups [g0, g1)
    int32_t vtx, i1, i2, g0, g1;
    int16_t i3b, ni3;
    int64_t part_off;          // its partial tile [i3 - i3b][i4][i5] in the partials buffer
    int32_t single;            // 0: every selected shell of the groups; 1 + 64 p + d23: that one shell only
                               // (p = d24 D + d34 within group g0), whose squared output-tile norm is
                               // written to part[part_off] instead of the tile
};
struct ShellFilter {
    int64_t begin, end;          // linear shell range
    const uint32_t* bitmap;      // optional membership bitmap (single vertex), overrides the range
};
struct ReduceJob {             // one output tile's i3 range: items item0 + c * stride, c = 0..nchunk-1
    int32_t vtx, tile, item0, nchunk, stride, i3b, ni3, pad;
    double* A;                 // the first output entry of the range
};

// ----------------------------------------------------------------------------------------------
// launchers implemented in the kernel translation units (return SF_OK or an error code)
// ----------------------------------------------------------------------------------------------
int sf_fact_table_build(dd* F, cudaStream_t s);
// triangle coefficients of every triad with doubled spins up to m: (m+1)^3 double-doubles
int sf_tri_table_build(int m, const dd* F, dd* d_out, int num_sms, cudaStream_t s);
// d_need (optional): per slot, nonzero if it is built (the others are zero-filled)
int sf_sixj_table_build(int table_id, const VtxDev* d_v, const SlotDesc* d_slots, int nslots, int64_t n,
                        double* d_out, const dd* d_tri, int tri_m, const unsigned char* d_need, int* d_status,
                        int num_sms, cudaStream_t s);
int sf_to_float(const double* d_in, float* d_out, int64_t n, int num_sms, cudaStream_t s);
// (2x+1) S[entry] per slot entry (x = the entry's third argument, doubled)
int sf_scale_x(const double* d_in, const SlotDesc* d_slots, int nslots, double* d_out, cudaStream_t s);
// (hi, lo) float pairs: hi = fl32(d), lo = fl32(d - hi)
int sf_to_ff(const double* d_in, float2* d_out, int64_t n, int num_sms, cudaStream_t s);
// Gauss-Legendre library of the d-table kernel (sizes 64..SF_GL_NMAX in steps of 32), built once
// per device and kept for the life of the process
int sf_gl_library(cudaStream_t s, const double** out);
// stream-ordered scratch (kept by a per-device pool of the library for reuse across calls)
int sf_scratch_alloc(void** p, size_t bytes, cudaStream_t s);
int sf_scratch_free(void* p, cudaStream_t s);
int sf_rule_build(const sf_quad_rule* q, double* d_x, double* d_w, double* d_r, double* d_W, cudaStream_t s);
// d-tables of the ten faces of one vertex (one launch): doubled boundary spins tk, l counts nl
struct DtabFaces {
    int tk[10], nl[10];
    double rho[10];
    double2* out[10];
};
int sf_dtable_build(const int tk[10], double gamma, const int nl[10], int nnodes, const double* d_r, const double* d_gl,
                    double2* const d_out[10], cudaStream_t s);
// node chunk of the booster kernel for the edge's four boundary spins, and its shared memory
int sf_booster_chunk(int tj1, int tj2, int tj3, int tj4);
size_t sf_booster_smem(int tj1, int tj2, int tj3, int tj4, int nk);
// pair tables of a booster edge: per side, the stride of the second strand's offset, the number of
// virtual-spin pairs and of k values of the 3j tables
struct PairDims { int nb[2], npid[2], nkk[2]; };
int sf_pair_dims(const int tj4[4], const int slot4[4], int D, int nnodes, PairDims* pd, size_t pbytes[2], size_t tbytes[2]);
int sf_pair_build(const VtxDev* d_v, int edge, const PairDims& pd, const double* d_W, int nnodes, const dd* F,
                  const int tj4[4], double2* const d_P[2], double* const d_T[2], int* d_status, int num_sms, cudaStream_t s);
// boosters of the triples fill[t] != 0 from their exchanged triples on the pair of free strands at
// coupling positions (pos, pos + 1), whose spins are equal
int sf_booster_mirror(const VtxDev* d_v, int edge, int pos, int ntrip, const unsigned char* d_fill, double* d_B,
                      cudaStream_t s);
// d_need (optional): per virtual-spin triple, nonzero if its booster is computed (the others are zero);
// d_P, d_T: the edge's pair tables (sf_pair_build)
int sf_booster_build(const VtxDev* d_v, int edge, int ntrip, size_t smem, int nc, const double* d_W, int nnodes,
                     const dd* F, double* d_Aj, double* d_Cj, double* d_B, const unsigned char* d_need,
                     const double2* const d_P[2], const double* const d_T[2], const PairDims& pd, int* d_status,
                     cudaStream_t s);
// Shell-kernel modes: the sf_precision values (0 FP64, 1 mixed, 2 mixed with compensated FP32
// pairs for the {6j} contractions).
// shared memory (in doubles) of the shell kernel; mni3 = largest i3 extent of a work item
size_t sf_shell_smem_doubles(int mdi, int mdk, int mk3u, int xc, int D, int mni3, int mode);
// sets the kernel's shared-memory attribute and returns its grid (resident CTAs, at most n_items);
// host-only, so a capturable launch sequence calls it beforehand. nt: 256 or 512 threads per CTA.
int sf_shell_prepare(int mode, int nt, int mdi, int mdk, int mk3u, int xc, int Dmax, int mni3, int n_items, int num_sms,
                     int* grid, size_t* smem);
// zeroes the work counter and launches the persistent shell kernel (stream work only)
int sf_shell_launch_prepared(int mode, int nt, int grid, size_t smem, const VtxDev* d_v, int mdi, int mdk, int mk3u,
                             int xc, int Dmax, int mni3, const WorkItem* d_items, int n_items, int* d_counter,
                             double* d_part, ShellFilter filt, cudaStream_t s);
// FP64 shell kernel with 512 threads over whole-tile items (i3b = 0, ni3 = di3), one call
int sf_shell_fp64_launch(const VtxDev* d_v, int mdi, int mdk, int mk3u, int xc, int Dmax, const WorkItem* d_items,
                         int n_items, int* d_counter, double* d_part, ShellFilter filt, int num_sms, cudaStream_t s);
int sf_reduce_launch(const VtxDev* d_v, int vtx, int ntiles, const WorkItem* d_items, int item0, int nchunk,
                     const double* d_part, double* A, cudaStream_t s);
int sf_reduce_jobs_launch(const VtxDev* d_v, const ReduceJob* d_jobs, int njobs, const WorkItem* d_items,
                          const double* d_part, cudaStream_t s);
int sf_bitmap_launch(const int64_t* d_list, int64_t n, int64_t nshell, uint32_t* d_bm, cudaStream_t s);
int sf_adjoint_launch(const VtxDev* d_v, const VtxDev& h, const double* const psi[5], double* a_out,
                      double* const grad_psi[5], double* const grad_B[4], void* scratch, size_t scratch_bytes,
                      int num_sms, cudaStream_t s);
size_t sf_adjoint_scratch_bytes(const VtxDev& h);
