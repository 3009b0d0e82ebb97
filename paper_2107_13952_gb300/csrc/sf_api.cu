// C ABI of the EPRL vertex library (include/sf_eprl.h): argument checks, table planning,
// device memory ownership and the launch sequence of the kernels.
#include "sf_internal.cuh"
#include <climits>
#include <algorithm>
#include <cmath>
#include <string>

// ----------------------------------------------------------------------------------------------
// errors
// ----------------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";

int sf_set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

extern "C" const char* sf_last_error(void) { return g_err; }
static void sf_clear_error() { g_err[0] = 0; }   // after a probe whose failure is not an error of the call

#include <atomic>
static std::atomic<long long> g_launches{0};
void sf_note_launch(int n) { g_launches += n; }
extern "C" int64_t sf_kernel_launches(void) { return (int64_t)g_launches.load(); }
static thread_local double g_last_kernel_ms = -1.0;
extern "C" double sf_last_kernel_ms(int32_t kind) { return kind == 0 ? g_last_kernel_ms : -1.0; }
extern "C" const char* sf_version(void) { return "sf_eprl 0.1 (sm_103a)"; }

// ----------------------------------------------------------------------------------------------
// host-side tables object
// ----------------------------------------------------------------------------------------------
struct Table6j {
    std::vector<SlotDesc> slots;
    SlotDesc* d_slots = nullptr;
    int64_t n = 0;
    double* d_vals = nullptr;
};

struct VertexHost {
    sf_vertex v;
    int D = 0;
    int32_t ilo[5], di[5];
    int32_t olo[5], od[5];   // output sub-range: first index within each range and count
    int64_t nshell = 0;
    Table6j S[5];
    float* d_S4f = nullptr;
    float* d_S5f = nullptr;
    double* d_S1x = nullptr;
    float2* d_Sff[3] = {nullptr, nullptr, nullptr};
    int64_t ntrip = 0;
    int32_t dkmax[4];
    std::vector<int32_t> klo[4];
    int32_t* d_klo[4] = {nullptr, nullptr, nullptr, nullptr};
    double* d_B[4] = {nullptr, nullptr, nullptr, nullptr};
    float* d_Bf[4] = {nullptr, nullptr, nullptr, nullptr};
    bool boosters_ready = false;
    double2* d_dtab[10] = {nullptr};
    int32_t nl[10];
    int64_t ngroups = 0;
    int mk3u = 1;            // largest union over l23 of the k3 ranges, over (l34, l35)
    int64_t g_lo = 0, g_hi = 0;                 // (l25, l35, l45) groups the tables cover
    bool restricted = false;                    // g_lo > 0 or g_hi < ngroups
    unsigned char* d_need6[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // slots built
    unsigned char* d_needB[4] = {nullptr, nullptr, nullptr, nullptr};            // triples computed
    std::vector<unsigned char> needB_h[4];      // host copies of d_needB (empty: every triple)
};

struct sf_tables {
    int device = 0;
    int num_sms = 0;
    std::vector<VertexHost> vs;
    VtxDev* d_vtx = nullptr;
    dd* d_fact = nullptr;
    int* d_status = nullptr;
    // rule
    bool have_rule = false;
    sf_quad_rule rule{};
    int nnodes = 0;
    const double* d_gl = nullptr;   // process-wide Gauss-Legendre library (not owned)
    double *d_x = nullptr, *d_w = nullptr, *d_r = nullptr, *d_W = nullptr;
    double *d_Aj = nullptr, *d_Cj = nullptr;   // boundary-side 3j scratch (largest edge)
    // amplitude scratch (grown on demand)
    void* d_scratch = nullptr;
    cudaStream_t side = nullptr;   // second stream of the shell sum's launch classes (created on first use)
    size_t scratch_bytes = 0;
    std::vector<void*> owned;
};

static int dev_alloc(sf_tables* t, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return sf_set_error(SF_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    t->owned.push_back(*p);
    return SF_OK;
}

// ----------------------------------------------------------------------------------------------
// argument checks and ranges
// ----------------------------------------------------------------------------------------------
static int check_vertex(const sf_vertex* v) {
    if (!v) return sf_set_error(SF_ERR_ARG, "null vertex");
    for (int f = 0; f < 10; f++)
        if (v->two_j[f] < 0 || v->two_j[f] > 60) return sf_set_error(SF_ERR_ARG, "two_j[%d]=%d out of range [0,60]", f, v->two_j[f]);
    if (!(v->gamma > 0.0) || v->gamma > 1e6) return sf_set_error(SF_ERR_ARG, "gamma must be positive and finite");
    if (v->dl < 0) return sf_set_error(SF_ERR_ARG, "dl must be >= 0");
    if (v->dl > SF_MAX_DL) return sf_set_error(SF_ERR_LIMIT, "dl=%d beyond the compiled limit %d", v->dl, SF_MAX_DL);
    return SF_OK;
}

static void ranges_of(const sf_vertex* v, int32_t lo[5], int32_t n[5]) {
    const int32_t* j = v->two_j;
    sf_pair_range(j[F12], j[F13], j[F14], j[F15], &lo[0], &n[0]);
    sf_pair_range(j[F23], j[F24], j[F25], j[F12], &lo[1], &n[1]);
    sf_pair_range(j[F34], j[F35], j[F13], j[F23], &lo[2], &n[2]);
    sf_pair_range(j[F45], j[F14], j[F24], j[F34], &lo[3], &n[3]);
    sf_pair_range(j[F15], j[F25], j[F35], j[F45], &lo[4], &n[4]);
}

// output sub-range of a vertex (first index, count) within its ranges n[5]
static int sub_range_of(const sf_vertex* v, const int32_t n[5], int32_t first[5], int32_t count[5]) {
    for (int e = 0; e < 5; e++) {
        const int f = v->sub_first[e], c = v->sub_count[e];
        if (f < 0 || c < 0 || f >= n[e] || (c > 0 && f + c > n[e]))
            return sf_set_error(SF_ERR_ARG, "sub-range of edge %d (first %d, count %d) outside its %d intertwiners",
                                e + 1, f, c, n[e]);
        first[e] = f;
        count[e] = c > 0 ? c : n[e] - f;
    }
    return SF_OK;
}

extern "C" int sf_output_ranges(const sf_vertex* v, int32_t two_lo[5], int32_t dim[5]) {
    int32_t lo[5], n[5], f[5], c[5];
    SF_TRY(sf_intertwiner_ranges(v, lo, n));
    if (!two_lo || !dim) return sf_set_error(SF_ERR_ARG, "null output");
    SF_TRY(sub_range_of(v, n, f, c));
    for (int e = 0; e < 5; e++) {
        two_lo[e] = lo[e] + 2 * f[e];
        dim[e] = c[e];
    }
    return SF_OK;
}

extern "C" int sf_intertwiner_ranges(const sf_vertex* v, int32_t two_lo[5], int32_t dim[5]) {
    SF_TRY(check_vertex(v));
    if (!two_lo || !dim) return sf_set_error(SF_ERR_ARG, "null output");
    ranges_of(v, two_lo, dim);
    for (int e = 0; e < 5; e++)
        if (dim[e] == 0) return sf_set_error(SF_ERR_EMPTY, "intertwiner range of edge %d is empty", e + 1);
    return SF_OK;
}

extern "C" int64_t sf_num_shells(const sf_vertex* v) {
    int r = check_vertex(v);
    if (r != SF_OK) return r;
    int64_t D = v->dl + 1;
    return D * D * D * D * D * D;
}

// union over parameter values of pair ranges -> (lo, n)
struct Rng { int lo, n; };
static inline void rng_union(Rng& u, int lo, int n) {
    if (n == 0) return;
    if (u.n == 0) { u.lo = lo; u.n = n; return; }
    int hi = std::max(u.lo + 2 * (u.n - 1), lo + 2 * (n - 1));
    u.lo = std::min(u.lo, lo);
    u.n = (hi - u.lo) / 2 + 1;
}
// x box of tri(a, p) & tri(b, q) for a in A, b in B (union), parity consistent or empty
static Rng x_box(Rng A, int p, Rng B, int q) {
    Rng r{0, 0};
    if (A.n == 0 || B.n == 0) return r;
    if ((A.lo + p + B.lo + q) & 1) return r;
    auto mind = [](Rng R, int c) {
        int hi = R.lo + 2 * (R.n - 1);
        if (c < R.lo) return R.lo - c;
        if (c > hi) return c - hi;
        return (c + R.lo) & 1;
    };
    int lo = std::max(mind(A, p), mind(B, q));
    int hi = std::min(A.lo + 2 * (A.n - 1) + p, B.lo + 2 * (B.n - 1) + q);
    if (lo > hi) return r;
    r.lo = lo;
    r.n = (hi - lo) / 2 + 1;
    return r;
}

static void plan_6j(VertexHost& h) {
    const int32_t* j = h.v.two_j;
    const int D = h.D;
    auto L = [&](int f, int d) { return j[f] + 2 * d; };
    auto pr = [](int a, int b, int c, int d) { Rng r; sf_pair_range(a, b, c, d, &r.lo, &r.n); return r; };
    Rng I1{h.ilo[0], h.di[0]};
    auto add_slot = [](Table6j& T, Rng a, Rng b, Rng x) {
        SlotDesc s{};
        s.off = T.n;
        if (a.n == 0 || b.n == 0 || x.n == 0) { a.n = b.n = x.n = 0; }
        s.alo = a.lo; s.blo = b.lo; s.xlo = x.lo; s.na = a.n; s.nb = b.n; s.nx = x.n;
        T.slots.push_back(s);
        T.n += (int64_t)a.n * b.n * x.n;
    };
    for (int k = 0; k < 5; k++) { h.S[k].slots.clear(); h.S[k].n = 0; }
    // S1[l25][i1, k5, x] = {i1 l25 x; k5 j14 j15}
    for (int d25 = 0; d25 < D; d25++) {
        Rng K5{0, 0};
        for (int d35 = 0; d35 < D; d35++)
            for (int d45 = 0; d45 < D; d45++) { Rng r = pr(j[F15], L(F25, d25), L(F35, d35), L(F45, d45)); rng_union(K5, r.lo, r.n); }
        add_slot(h.S[0], I1, K5, x_box(I1, L(F25, d25), K5, j[F14]));
    }
    // S2[l35, l45][k5, k4, x] = {j14 k5 x; l35 k4 l45}
    for (int d35 = 0; d35 < D; d35++)
        for (int d45 = 0; d45 < D; d45++) {
            Rng K5{0, 0}, K4{0, 0};
            for (int d25 = 0; d25 < D; d25++) { Rng r = pr(j[F15], L(F25, d25), L(F35, d35), L(F45, d45)); rng_union(K5, r.lo, r.n); }
            for (int d24 = 0; d24 < D; d24++)
                for (int d34 = 0; d34 < D; d34++) { Rng r = pr(L(F45, d45), j[F14], L(F24, d24), L(F34, d34)); rng_union(K4, r.lo, r.n); }
            add_slot(h.S[1], K5, K4, x_box(K5, j[F14], K4, L(F35, d35)));
        }
    // S3[l24, l34, l35][k4, k3, x] = {k4 l35 x; k3 l24 l34}
    for (int d24 = 0; d24 < D; d24++)
        for (int d34 = 0; d34 < D; d34++)
            for (int d35 = 0; d35 < D; d35++) {
                Rng K4{0, 0}, K3{0, 0};
                for (int d45 = 0; d45 < D; d45++) { Rng r = pr(L(F45, d45), j[F14], L(F24, d24), L(F34, d34)); rng_union(K4, r.lo, r.n); }
                for (int d23 = 0; d23 < D; d23++) { Rng r = pr(L(F34, d34), L(F35, d35), j[F13], L(F23, d23)); rng_union(K3, r.lo, r.n); }
                add_slot(h.S[2], K4, K3, x_box(K4, L(F35, d35), K3, L(F24, d24)));
            }
    // S4[l23, l24][k3, k2, x] = {l24 k3 x; j13 k2 l23}
    for (int d23 = 0; d23 < D; d23++)
        for (int d24 = 0; d24 < D; d24++) {
            Rng K3{0, 0}, K2{0, 0};
            for (int d34 = 0; d34 < D; d34++)
                for (int d35 = 0; d35 < D; d35++) { Rng r = pr(L(F34, d34), L(F35, d35), j[F13], L(F23, d23)); rng_union(K3, r.lo, r.n); }
            for (int d25 = 0; d25 < D; d25++) { Rng r = pr(L(F23, d23), L(F24, d24), L(F25, d25), j[F12]); rng_union(K2, r.lo, r.n); }
            add_slot(h.S[3], K3, K2, x_box(K3, L(F24, d24), K2, j[F13]));
        }
    // S5[l25][k2, i1, x] = {k2 j13 x; i1 l25 j12}
    for (int d25 = 0; d25 < D; d25++) {
        Rng K2{0, 0};
        for (int d23 = 0; d23 < D; d23++)
            for (int d24 = 0; d24 < D; d24++) { Rng r = pr(L(F23, d23), L(F24, d24), L(F25, d25), j[F12]); rng_union(K2, r.lo, r.n); }
        add_slot(h.S[4], K2, I1, x_box(K2, j[F13], I1, L(F25, d25)));
    }
}

static void plan_boosters(VertexHost& h) {
    const int32_t* j = h.v.two_j;
    const int D = h.D;
    h.ntrip = (int64_t)D * D * D;
    static const int faces[4][4] = {{F23, F24, F25, F12}, {F34, F35, F13, F23}, {F45, F14, F24, F34}, {F15, F25, F35, F45}};
    static const int slotof[4][4] = {{0, 1, 2, -1}, {0, 1, -1, 2}, {0, -1, 1, 2}, {-1, 0, 1, 2}};
    for (int e = 0; e < 4; e++) {
        h.klo[e].assign(h.ntrip, 0);
        int dk = 1;
        for (int t = 0; t < h.ntrip; t++) {
            int off[3] = {t / (D * D), (t / D) % D, t % D};
            int tl[4];
            for (int a = 0; a < 4; a++) tl[a] = j[faces[e][a]] + (slotof[e][a] < 0 ? 0 : 2 * off[slotof[e][a]]);
            int lo, n;
            sf_pair_range(tl[0], tl[1], tl[2], tl[3], &lo, &n);
            h.klo[e][t] = n ? lo : 0;
            dk = std::max(dk, n);
        }
        h.dkmax[e] = dk;
    }
    for (int f = 0; f < 10; f++) h.nl[f] = (f <= F15) ? 1 : D;
    h.mk3u = 1;
    for (int d34 = 0; d34 < D; d34++)
        for (int d35 = 0; d35 < D; d35++) {
            int lo = 1 << 30, hi = -1;
            for (int d23 = 0; d23 < D; d23++) {
                int a, n;
                sf_pair_range(j[F34] + 2 * d34, j[F35] + 2 * d35, j[F13], j[F23] + 2 * d23, &a, &n);
                if (n) { lo = std::min(lo, a); hi = std::max(hi, a + 2 * (n - 1)); }
            }
            if (hi >= lo) h.mk3u = std::max(h.mk3u, (hi - lo) / 2 + 1);
        }
}

static int upload_vtxdev(sf_tables* t) {
    std::vector<VtxDev> hv(t->vs.size());
    for (size_t i = 0; i < t->vs.size(); i++) {
        VertexHost& h = t->vs[i];
        VtxDev& d = hv[i];
        memset(&d, 0, sizeof(d));
        for (int f = 0; f < 10; f++) d.tj[f] = h.v.two_j[f];
        d.gamma = h.v.gamma;
        d.dl = h.v.dl;
        d.D = h.D;
        for (int e = 0; e < 5; e++) { d.ilo[e] = h.ilo[e]; d.di[e] = h.di[e]; d.olo[e] = h.olo[e]; d.od[e] = h.od[e]; }
        d.nshell = h.nshell;
        for (int k = 0; k < 5; k++) { d.S[k] = h.S[k].d_vals; d.slot[k] = h.S[k].d_slots; }
        d.S4f = h.d_S4f;
        d.S1x = h.d_S1x;
        d.S5f = h.d_S5f;
        for (int k = 0; k < 3; k++) d.Sff[k] = h.d_Sff[k];
        for (int e = 0; e < 4; e++) {
            d.B[e] = h.d_B[e];
            d.Bf[e] = h.d_Bf[e];
            d.klo[e] = h.d_klo[e];
            d.dkmax[e] = h.dkmax[e];
        }
        d.ntrip = h.ntrip;
        for (int f = 0; f < 10; f++) { d.dtab[f] = h.d_dtab[f]; d.nl[f] = h.nl[f]; }
    }
    SF_CUDA_TRY(cudaMemcpy(t->d_vtx, hv.data(), hv.size() * sizeof(VtxDev), cudaMemcpyHostToDevice));
    return SF_OK;
}

static int check_status(sf_tables* t, cudaStream_t s, const char* what) {
    int st = 0;
    SF_CUDA_TRY(cudaMemcpyAsync(&st, t->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    SF_CUDA_TRY(cudaStreamSynchronize(s));
    if (st == SF_DEV_OK) return SF_OK;
    if (st == SF_DEV_BIGINT_OVERFLOW) return sf_set_error(SF_ERR_LIMIT, "%s: exact Racah sum overflowed its integer width", what);
    if (st == SF_DEV_NONREAL_BOOSTER) return sf_set_error(SF_ERR_NUMERIC, "%s: a booster has a non-negligible imaginary part", what);
    if (st == SF_DEV_TIMEOUT) return sf_set_error(SF_ERR_TIMEOUT, "%s: a bounded device wait gave up", what);
    return sf_set_error(SF_ERR_NUMERIC, "%s: device status %d", what, st);
}

extern "C" void sf_tables_free(sf_tables* t) {
    if (!t) return;
    for (void* p : t->owned) cudaFree(p);
    if (t->d_scratch) cudaFree(t->d_scratch);
    if (t->side) cudaStreamDestroy(t->side);
    delete t;
}

// The slots and booster triples that the shells of groups [g_lo, g_hi) read: S1, S5 and the edge-2
// boosters by d25, S2 by (d35, d45), S3 and the edge-3 boosters by d35, the edge-4 boosters by
// d45, the edge-5 boosters by the group itself; S4 is read by every group.
static int build_needs(sf_tables* t, VertexHost& h) {
    const int D = h.D;
    std::vector<char> n25(D, 0), n35(D, 0), n45(D, 0), n3545((size_t)D * D, 0);
    for (int64_t g = h.g_lo; g < h.g_hi; g++) {
        const int d25 = (int)(g / ((int64_t)D * D)), d35 = (int)((g / D) % D), d45 = (int)(g % D);
        n25[d25] = n35[d35] = n45[d45] = 1;
        n3545[(size_t)d35 * D + d45] = 1;
    }
    std::vector<unsigned char> m;
    auto put = [&](unsigned char** dst) -> int {
        SF_TRY(dev_alloc(t, (void**)dst, m.size()));
        SF_CUDA_TRY(cudaMemcpy(*dst, m.data(), m.size(), cudaMemcpyHostToDevice));
        return SF_OK;
    };
    m.assign(D, 0);
    for (int d = 0; d < D; d++) m[d] = n25[d];
    SF_TRY(put(&h.d_need6[0]));
    SF_TRY(put(&h.d_need6[4]));
    m.assign((size_t)D * D, 0);
    for (size_t q = 0; q < m.size(); q++) m[q] = n3545[q];
    SF_TRY(put(&h.d_need6[1]));
    m.assign((size_t)D * D * D, 0);
    for (size_t q = 0; q < m.size(); q++) m[q] = n35[q % D];            // slot (d24 D + d34) D + d35
    SF_TRY(put(&h.d_need6[2]));
    // boosters: t = (a D + b) D + c over the edge's three offsets
    for (size_t q = 0; q < m.size(); q++) m[q] = n25[q % D];            // edge 2 (d23, d24, d25)
    SF_TRY(put(&h.d_needB[0]));
    h.needB_h[0] = m;
    for (size_t q = 0; q < m.size(); q++) m[q] = n35[(q / D) % D];      // edge 3 (d34, d35, d23)
    SF_TRY(put(&h.d_needB[1]));
    h.needB_h[1] = m;
    for (size_t q = 0; q < m.size(); q++) m[q] = n45[q / ((size_t)D * D)];   // edge 4 (d45, d24, d34)
    SF_TRY(put(&h.d_needB[2]));
    h.needB_h[2] = m;
    for (size_t q = 0; q < m.size(); q++) m[q] = ((int64_t)q >= h.g_lo && (int64_t)q < h.g_hi) ? 1 : 0;   // edge 5 = g
    SF_TRY(put(&h.d_needB[3]));
    h.needB_h[3] = m;
    return SF_OK;
}

// the shells a call asks for lie in the groups its tables cover
static int check_covered(const sf_tables* t, int64_t shell_begin, int64_t shell_end, const int64_t* shell_list,
                         int64_t n_list) {
    for (size_t i = 0; i < t->vs.size(); i++) {
        const VertexHost& h = t->vs[i];
        if (!h.restricted) continue;
        const int64_t per = (int64_t)h.D * h.D * h.D;
        if (shell_list) {
            std::vector<int64_t> l((size_t)std::max<int64_t>(n_list, 0));
            if (n_list > 0) SF_CUDA_TRY(cudaMemcpy(l.data(), shell_list, (size_t)n_list * sizeof(int64_t), cudaMemcpyDefault));
            for (int64_t s : l)
                if (s >= 0 && s < h.nshell && (s / per < h.g_lo || s / per >= h.g_hi))
                    return sf_set_error(SF_ERR_ARG, "shell %lld lies outside the groups the tables were built for",
                                        (long long)s);
            continue;
        }
        const int64_t b = std::min<int64_t>(std::max<int64_t>(shell_begin, 0), h.nshell);
        const int64_t e = std::min<int64_t>(std::max<int64_t>(shell_end, 0), h.nshell);
        if (e > b && (b < h.g_lo * per || e > h.g_hi * per))
            return sf_set_error(SF_ERR_ARG, "vertex %zu: shells [%lld, %lld) reach beyond the groups [%lld, %lld) its "
                                            "tables were built for", i, (long long)b, (long long)e, (long long)h.g_lo,
                                (long long)h.g_hi);
    }
    return SF_OK;
}

static int build_tables(const sf_vertex* v, int32_t n, int64_t range_begin, int64_t range_end, sf_tables** out,
                        cudaStream_t stream) {
    if (!out) return sf_set_error(SF_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!v || n <= 0) return sf_set_error(SF_ERR_ARG, "need at least one vertex");
    for (int i = 0; i < n; i++) {
        SF_TRY(check_vertex(&v[i]));
        int32_t lo[5], dim[5];
        ranges_of(&v[i], lo, dim);
        for (int e = 0; e < 5; e++)
            if (dim[e] == 0) return sf_set_error(SF_ERR_EMPTY, "vertex %d: intertwiner range of edge %d is empty", i, e + 1);
        {
            int32_t f[5], c[5];
            SF_TRY(sub_range_of(&v[i], dim, f, c));
        }
        // integer Racah arguments and factorials stay within the compiled widths
        int maxl = 0;
        for (int f = 0; f < 10; f++) maxl = std::max(maxl, v[i].two_j[f] + (f > F15 ? 2 * v[i].dl : 0));
        if (2 * maxl + 4 * maxl > 2 * SF_FACT_MAX - 4)
            return sf_set_error(SF_ERR_LIMIT, "vertex %d: spins too large for the exact symbol kernels", i);
    }
    sf_tables* t = new sf_tables();
    int rc = SF_OK;
    do {
        if (cudaGetDevice(&t->device) != cudaSuccess) { rc = sf_set_error(SF_ERR_CUDA, "no CUDA device"); break; }
        cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, t->device);
        t->vs.resize(n);
        for (int i = 0; i < n && rc == SF_OK; i++) {
            VertexHost& h = t->vs[i];
            h.v = v[i];
            h.D = v[i].dl + 1;
            ranges_of(&v[i], h.ilo, h.di);
            sub_range_of(&v[i], h.di, h.olo, h.od);   // validated above
            h.nshell = (int64_t)h.D * h.D * h.D * h.D * h.D * h.D;
            h.ngroups = (int64_t)h.D * h.D * h.D;
            {
                const int64_t per = h.ngroups;   // shells per group
                const int64_t b = std::min<int64_t>(std::max<int64_t>(range_begin, 0), h.nshell);
                const int64_t e = std::min<int64_t>(std::max<int64_t>(range_end, 0), h.nshell);
                h.g_lo = b / per;
                h.g_hi = e > b ? (e + per - 1) / per : h.g_lo;
                h.restricted = h.g_lo > 0 || h.g_hi < h.ngroups;
            }
            plan_6j(h);
            plan_boosters(h);
            for (int k = 0; k < 5 && rc == SF_OK; k++) {
                if (k == 3) rc = dev_alloc(t, (void**)&h.d_S4f, h.S[3].n * sizeof(float));
                if (k == 4) rc = dev_alloc(t, (void**)&h.d_S5f, h.S[4].n * sizeof(float));
                if (k == 0 && rc == SF_OK) rc = dev_alloc(t, (void**)&h.d_S1x, h.S[0].n * sizeof(double));
                if (k < 3) rc = dev_alloc(t, (void**)&h.d_Sff[k], h.S[k].n * sizeof(float2));
                if (rc != SF_OK) break;
                rc = dev_alloc(t, (void**)&h.S[k].d_slots, h.S[k].slots.size() * sizeof(SlotDesc));
                if (rc == SF_OK) rc = dev_alloc(t, (void**)&h.S[k].d_vals, h.S[k].n * sizeof(double));
                if (rc == SF_OK && cudaMemcpy(h.S[k].d_slots, h.S[k].slots.data(), h.S[k].slots.size() * sizeof(SlotDesc),
                                              cudaMemcpyHostToDevice) != cudaSuccess)
                    rc = sf_set_error(SF_ERR_CUDA, "slot upload failed");
            }
            for (int e = 0; e < 4 && rc == SF_OK; e++) {
                rc = dev_alloc(t, (void**)&h.d_klo[e], h.ntrip * sizeof(int32_t));
                if (rc == SF_OK) rc = dev_alloc(t, (void**)&h.d_B[e], (size_t)h.ntrip * h.di[e + 1] * h.dkmax[e] * sizeof(double));
                if (rc == SF_OK) rc = dev_alloc(t, (void**)&h.d_Bf[e], (size_t)h.ntrip * h.di[e + 1] * h.dkmax[e] * sizeof(float));
                if (rc == SF_OK && cudaMemcpy(h.d_klo[e], h.klo[e].data(), h.ntrip * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
                    rc = sf_set_error(SF_ERR_CUDA, "klo upload failed");
                if (rc == SF_OK && (cudaMemsetAsync(h.d_B[e], 0, (size_t)h.ntrip * h.di[e + 1] * h.dkmax[e] * sizeof(double), stream) != cudaSuccess ||
                                    cudaMemsetAsync(h.d_Bf[e], 0, (size_t)h.ntrip * h.di[e + 1] * h.dkmax[e] * sizeof(float), stream) != cudaSuccess))
                    rc = sf_set_error(SF_ERR_CUDA, "booster clear failed");
            }
        }
        if (rc != SF_OK) break;
        if ((rc = dev_alloc(t, (void**)&t->d_vtx, n * sizeof(VtxDev))) != SF_OK) break;
        if ((rc = dev_alloc(t, (void**)&t->d_fact, (SF_FACT_MAX + 1) * sizeof(dd))) != SF_OK) break;
        if ((rc = dev_alloc(t, (void**)&t->d_status, sizeof(int))) != SF_OK) break;
        if (cudaMemsetAsync(t->d_status, 0, sizeof(int), stream) != cudaSuccess) { rc = sf_set_error(SF_ERR_CUDA, "memset"); break; }
        if ((rc = upload_vtxdev(t)) != SF_OK) break;
        for (size_t i = 0; i < t->vs.size() && rc == SF_OK; i++)
            if (t->vs[i].restricted) rc = build_needs(t, t->vs[i]);
        if (rc != SF_OK) break;
        if ((rc = sf_fact_table_build(t->d_fact, stream)) != SF_OK) break;
        // triangle coefficients for every doubled spin that an argument of the tables reaches
        int tri_m = 0;
        for (const VertexHost& h : t->vs) {
            for (int f = 0; f < 10; f++) tri_m = std::max(tri_m, h.v.two_j[f] + (f > F15 ? 2 * h.v.dl : 0));
            for (int k = 0; k < 5; k++)
                for (const SlotDesc& sd : h.S[k].slots)
                    tri_m = std::max(tri_m, std::max(sd.alo + 2 * (sd.na - 1), std::max(sd.blo + 2 * (sd.nb - 1),
                                                                                           sd.xlo + 2 * (sd.nx - 1))));
        }
        dd* d_tri = nullptr;
        if ((rc = dev_alloc(t, (void**)&d_tri, (size_t)(tri_m + 1) * (tri_m + 1) * (tri_m + 1) * sizeof(dd))) != SF_OK) break;
        if ((rc = sf_tri_table_build(tri_m, t->d_fact, d_tri, t->num_sms, stream)) != SF_OK) break;
        for (int i = 0; i < n && rc == SF_OK; i++) {
            VertexHost& h = t->vs[i];
            for (int k = 0; k < 5 && rc == SF_OK; k++)
                rc = sf_sixj_table_build(k + 1, t->d_vtx + i, h.S[k].d_slots, (int)h.S[k].slots.size(), h.S[k].n,
                                         h.S[k].d_vals, d_tri, tri_m, h.d_need6[k], t->d_status, t->num_sms, stream);
            if (rc == SF_OK) rc = sf_to_float(h.S[3].d_vals, h.d_S4f, h.S[3].n, t->num_sms, stream);
            if (rc == SF_OK) rc = sf_scale_x(h.S[0].d_vals, h.S[0].d_slots, (int)h.S[0].slots.size(), h.d_S1x, stream);
            if (rc == SF_OK) rc = sf_to_float(h.S[4].d_vals, h.d_S5f, h.S[4].n, t->num_sms, stream);
            for (int k = 0; k < 3 && rc == SF_OK; k++) rc = sf_to_ff(h.S[k].d_vals, h.d_Sff[k], h.S[k].n, t->num_sms, stream);
        }
        if (rc != SF_OK) break;
        rc = check_status(t, stream, "sf_6j_table");
    } while (0);
    if (rc != SF_OK) { sf_tables_free(t); return rc; }
    *out = t;
    return SF_OK;
}

extern "C" int sf_6j_table(const sf_vertex* v, int32_t n, sf_tables** out, cudaStream_t stream) {
    return build_tables(v, n, 0, INT64_MAX, out, stream);
}

extern "C" int sf_6j_table_range(const sf_vertex* v, int32_t n, int64_t shell_begin, int64_t shell_end, sf_tables** out,
                                 cudaStream_t stream) {
    if (shell_begin < 0 || shell_end < shell_begin) return sf_set_error(SF_ERR_ARG, "bad shell range");
    return build_tables(v, n, shell_begin, shell_end, out, stream);
}

static int boosters_all(sf_tables* t, int nnodes, double2* const d_P[2], double* const d_T[2], cudaStream_t stream);

extern "C" int sf_boosters(sf_tables* t, const sf_quad_rule* q, cudaStream_t stream) {
    if (!t || !q) return sf_set_error(SF_ERR_ARG, "null argument");
    if (q->n_panels < 1 || q->order < 2 || q->order > 1024 || !(q->r_max > 0.0) || q->r_max > 700.0)
        return sf_set_error(SF_ERR_ARG, "bad quadrature rule");
    const int nnodes = q->n_panels * q->order;
    if (!t->have_rule || t->rule.n_panels != q->n_panels || t->rule.order != q->order || t->rule.r_max != q->r_max) {
        if (!t->d_gl) SF_TRY(sf_gl_library(stream, &t->d_gl));
        if (nnodes > t->nnodes) {
            SF_TRY(dev_alloc(t, (void**)&t->d_x, nnodes * sizeof(double)));
            SF_TRY(dev_alloc(t, (void**)&t->d_w, nnodes * sizeof(double)));
            SF_TRY(dev_alloc(t, (void**)&t->d_r, nnodes * sizeof(double)));
            SF_TRY(dev_alloc(t, (void**)&t->d_W, nnodes * sizeof(double)));
        }
        SF_TRY(sf_rule_build(q, t->d_x, t->d_w, t->d_r, t->d_W, stream));
        // d-tables are sized by the node count: reallocate for a different rule
        for (auto& h : t->vs)
            for (int f = 0; f < 10; f++) h.d_dtab[f] = nullptr;
        t->rule = *q;
        t->nnodes = nnodes;
        t->have_rule = true;
    }
    size_t aj = 16;
    for (auto& h : t->vs) {
        for (int f = 0; f < 10; f++) {
            if (!h.d_dtab[f]) SF_TRY(dev_alloc(t, (void**)&h.d_dtab[f], (size_t)h.nl[f] * (h.v.two_j[f] + 1) * nnodes * sizeof(double2)));
        }
        for (int e = 0; e < 4; e++) {
            static const int faces[4][4] = {{F23, F24, F25, F12}, {F34, F35, F13, F23}, {F45, F14, F24, F34}, {F15, F25, F35, F45}};
            size_t a = (size_t)h.di[e + 1] * (h.v.two_j[faces[e][0]] + 1) * (h.v.two_j[faces[e][1]] + 1);
            size_t c = (size_t)h.di[e + 1] * (h.v.two_j[faces[e][2]] + 1) * (h.v.two_j[faces[e][3]] + 1);
            aj = std::max(aj, std::max(a, c));
            for (int a4 = 0; a4 < 4; a4++)
                if (h.v.two_j[faces[e][a4]] > 16)
                    return sf_set_error(SF_ERR_LIMIT, "booster kernel supports boundary spins up to 8");
        }
    }
    static const int bfaces[4][4] = {{F23, F24, F25, F12}, {F34, F35, F13, F23}, {F45, F14, F24, F34}, {F15, F25, F35, F45}};
    static const int bslot[4][4] = {{0, 1, 2, -1}, {0, 1, -1, 2}, {0, -1, 1, 2}, {-1, 0, 1, 2}};
    // per-pair tables of the booster kernel (largest edge), stream-ordered scratch freed on return
    size_t pbytes_max[2] = {16, 16}, tbytes_max[2] = {16, 16};
    for (auto& h : t->vs)
        for (int e = 0; e < 4; e++) {
            int tj4[4];
            for (int a = 0; a < 4; a++) tj4[a] = h.v.two_j[bfaces[e][a]];
            PairDims pd;
            size_t pb[2], tb[2];
            sf_pair_dims(tj4, bslot[e], h.D, nnodes, &pd, pb, tb);
            for (int s = 0; s < 2; s++) {
                pbytes_max[s] = std::max(pbytes_max[s], pb[s]);
                tbytes_max[s] = std::max(tbytes_max[s], tb[s]);
            }
        }
    SF_TRY(dev_alloc(t, (void**)&t->d_Aj, aj * sizeof(double)));
    SF_TRY(dev_alloc(t, (void**)&t->d_Cj, aj * sizeof(double)));
    SF_TRY(upload_vtxdev(t));
    SF_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), stream));
    void* scratch = nullptr;
    const size_t sbytes = pbytes_max[0] + pbytes_max[1] + tbytes_max[0] + tbytes_max[1];
    SF_TRY(sf_scratch_alloc(&scratch, sbytes, stream));
    double2* d_P[2] = {(double2*)scratch, (double2*)((char*)scratch + pbytes_max[0])};
    double* d_T[2] = {(double*)((char*)scratch + pbytes_max[0] + pbytes_max[1]),
                      (double*)((char*)scratch + pbytes_max[0] + pbytes_max[1] + tbytes_max[0])};
    int rc = boosters_all(t, nnodes, d_P, d_T, stream);
    const int fr = sf_scratch_free(scratch, stream);
    if (rc != SF_OK) return rc;
    SF_TRY(fr);
    return check_status(t, stream, "sf_boosters");
}

static int boosters_all(sf_tables* t, int nnodes, double2* const d_P[2], double* const d_T[2], cudaStream_t stream) {
    static const int bslot[4][4] = {{0, 1, 2, -1}, {0, 1, -1, 2}, {0, -1, 1, 2}, {-1, 0, 1, 2}};
    for (size_t i = 0; i < t->vs.size(); i++) {
        VertexHost& h = t->vs[i];
        {
            int nlf[10];
            for (int f = 0; f < 10; f++) nlf[f] = h.nl[f];
            SF_TRY(sf_dtable_build(h.v.two_j, h.v.gamma, nlf, nnodes, t->d_r, t->d_gl, h.d_dtab, stream));
        }
        for (int e = 0; e < 4; e++) {
            static const int faces[4][4] = {{F23, F24, F25, F12}, {F34, F35, F13, F23}, {F45, F14, F24, F34}, {F15, F25, F35, F45}};
            const int32_t* j = h.v.two_j;
            size_t smem = sf_booster_smem(j[faces[e][0]], j[faces[e][1]], j[faces[e][2]], j[faces[e][3]], h.dkmax[e]);
            const int nc = sf_booster_chunk(j[faces[e][0]], j[faces[e][1]], j[faces[e][2]], j[faces[e][3]]);
            int tj4[4];
            for (int a = 0; a < 4; a++) tj4[a] = j[faces[e][a]];
            PairDims pd;
            size_t pb[2], tb[2];
            sf_pair_dims(tj4, bslot[e], h.D, nnodes, &pd, pb, tb);
            SF_TRY(sf_pair_build(t->d_vtx + i, e + 2, pd, t->d_W, nnodes, t->d_fact, tj4, d_P, d_T, t->d_status, t->num_sms,
                                 stream));
            const double2* cP[2] = {d_P[0], d_P[1]};
            const double* cT[2] = {d_T[0], d_T[1]};
            // the edge's pair of free strands (coupling positions pos, pos + 1): with equal spins
            // the triples whose two offsets there decrease are filled from the exchanged triple
            const int pos = e < 2 ? 0 : 2;
            const bool mirror = j[faces[e][pos]] == j[faces[e][pos + 1]];
            const unsigned char* d_need = h.d_needB[e];
            unsigned char* d_masks = nullptr;
            if (mirror) {
                const int D = h.D, sa = bslot[e][pos], sb = bslot[e][pos + 1];
                const std::vector<unsigned char>& need = h.needB_h[e];
                std::vector<unsigned char> masks(2 * (size_t)h.ntrip, 0);   // computed | filled by exchange
                for (int64_t q = 0; q < h.ntrip; q++) {
                    if (!need.empty() && !need[q]) continue;
                    int off[3] = {(int)(q / ((int64_t)D * D)), (int)((q / D) % D), (int)(q % D)};
                    if (off[sa] <= off[sb]) {
                        masks[q] = 1;
                    } else {
                        std::swap(off[sa], off[sb]);
                        masks[((int64_t)off[0] * D + off[1]) * D + off[2]] = 1;
                        masks[h.ntrip + q] = 1;
                    }
                }
                SF_TRY(sf_scratch_alloc((void**)&d_masks, masks.size(), stream));
                const cudaError_t ce = cudaMemcpyAsync(d_masks, masks.data(), masks.size(), cudaMemcpyHostToDevice, stream);
                if (ce != cudaSuccess) {
                    sf_scratch_free(d_masks, stream);
                    return sf_set_error(SF_ERR_CUDA, "booster mask copy: %s", cudaGetErrorString(ce));
                }
                d_need = d_masks;
            }
            int rc = sf_booster_build(t->d_vtx + i, e + 2, (int)h.ntrip, smem, nc, t->d_W, nnodes, t->d_fact, t->d_Aj,
                                      t->d_Cj, h.d_B[e], d_need, cP, cT, pd, t->d_status, stream);
            if (rc == SF_OK && mirror) rc = sf_booster_mirror(t->d_vtx + i, e + 2, pos, (int)h.ntrip, d_masks + h.ntrip,
                                                             h.d_B[e], stream);
            if (d_masks) sf_scratch_free(d_masks, stream);
            SF_TRY(rc);
            SF_TRY(sf_to_float(h.d_B[e], h.d_Bf[e], (int64_t)h.ntrip * h.di[e + 1] * h.dkmax[e], t->num_sms, stream));
        }
        h.boosters_ready = true;
    }
    return SF_OK;
}

static int check_edge(const sf_tables* t, int32_t vertex, int32_t edge) {
    if (!t) return sf_set_error(SF_ERR_ARG, "null tables");
    if (vertex < 0 || vertex >= (int)t->vs.size()) return sf_set_error(SF_ERR_ARG, "vertex index out of range");
    if (edge < 2 || edge > 5) return sf_set_error(SF_ERR_ARG, "edge must be 2..5");
    return SF_OK;
}

extern "C" int sf_booster_shape(const sf_tables* t, int32_t vertex, int32_t edge, int64_t shape[3]) {
    SF_TRY(check_edge(t, vertex, edge));
    const VertexHost& h = t->vs[vertex];
    shape[0] = h.ntrip;
    shape[1] = h.di[edge - 1];
    shape[2] = h.dkmax[edge - 2];
    return SF_OK;
}

extern "C" int sf_boosters_upload(sf_tables* t, int32_t vertex, int32_t edge, const double* B, cudaStream_t stream) {
    SF_TRY(check_edge(t, vertex, edge));
    if (!B) return sf_set_error(SF_ERR_ARG, "null booster pointer");
    VertexHost& h = t->vs[vertex];
    size_t bytes = (size_t)h.ntrip * h.di[edge - 1] * h.dkmax[edge - 2] * sizeof(double);
    SF_CUDA_TRY(cudaMemcpyAsync(h.d_B[edge - 2], B, bytes, cudaMemcpyDefault, stream));
    SF_TRY(sf_to_float(h.d_B[edge - 2], h.d_Bf[edge - 2], (int64_t)h.ntrip * h.di[edge - 1] * h.dkmax[edge - 2], t->num_sms,
                       stream));
    SF_CUDA_TRY(cudaStreamSynchronize(stream));
    h.boosters_ready = true;   // edges never uploaded keep their last (initially zero) contents
    return SF_OK;
}

extern "C" int sf_boosters_download(const sf_tables* t, int32_t vertex, int32_t edge, double* B, cudaStream_t stream) {
    SF_TRY(check_edge(t, vertex, edge));
    if (!B) return sf_set_error(SF_ERR_ARG, "null booster pointer");
    const VertexHost& h = t->vs[vertex];
    size_t bytes = (size_t)h.ntrip * h.di[edge - 1] * h.dkmax[edge - 2] * sizeof(double);
    SF_CUDA_TRY(cudaMemcpyAsync(B, h.d_B[edge - 2], bytes, cudaMemcpyDefault, stream));
    SF_CUDA_TRY(cudaStreamSynchronize(stream));
    return SF_OK;
}

// ----------------------------------------------------------------------------------------------
// vertex amplitude
// ----------------------------------------------------------------------------------------------
static int grow_scratch(sf_tables* t, size_t bytes) {
    if (bytes <= t->scratch_bytes) return SF_OK;
    if (t->d_scratch) { cudaFree(t->d_scratch); t->d_scratch = nullptr; t->scratch_bytes = 0; }
    cudaError_t e = cudaMalloc(&t->d_scratch, bytes);
    if (e != cudaSuccess) { t->d_scratch = nullptr; return sf_set_error(SF_ERR_OOM, "scratch allocation of %zu bytes failed", bytes); }
    t->scratch_bytes = bytes;
    return SF_OK;
}

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Launch configuration of the shell kernel: threads per CTA (512: one CTA per SM; 256: two CTAs
// per SM, so that one CTA's staging and FP32 phases overlap the other's FP64 phases), the number
// of i3 pieces per output tile (2 halves the i3-indexed buffers and the register tile, at the cost
// of staging the i3-independent operands twice), the x chunk and the work granularity.
struct ShellConfig {
    int nt = 512, split = 1, xc = 0, items_per_sm = 8;
};

struct ShellDims {
    int mdi = 1, mdk = 1, mk3u = 1, Dmax = 1, mdi3 = 1;
};

// vertex subsets: mask[i] != 0 selects vertex i; a null mask selects every vertex
typedef std::vector<char> VertexMask;
static bool in_mask(const VertexMask* m, size_t i) { return !m || (*m)[i]; }

static ShellDims shell_dims(const sf_tables* t, const VertexMask* m = nullptr) {
    ShellDims d;
    for (size_t i = 0; i < t->vs.size(); i++) {
        if (!in_mask(m, i)) continue;
        const VertexHost& h = t->vs[i];
        for (int e = 2; e < 5; e++) d.mdi = std::max(d.mdi, (int)h.od[e]);
        for (int e = 0; e < 4; e++) d.mdk = std::max(d.mdk, (int)h.dkmax[e]);
        d.mk3u = std::max(d.mk3u, h.mk3u);
        d.Dmax = std::max(d.Dmax, h.D);
        d.mdi3 = std::max(d.mdi3, (int)h.od[2]);
    }
    return d;
}

static size_t shell_smem_limit(int nt) { return nt == 256 ? 109 * 1024 : 200 * 1024; }   // 256: two CTAs (with static shared memory) per SM
static int shell_tile_blocks(int nt) { return nt >= 1024 ? 1 : 2; }   // register-tile blocks per thread

// the register-resident output tile (blocks of 2 i5 x 4 i3 per i4) fits the blocks per thread
static bool shell_tile_fits(const sf_tables* t, int nt, int split, const VertexMask* m = nullptr) {
    for (size_t i = 0; i < t->vs.size(); i++) {
        if (!in_mask(m, i)) continue;
        const VertexHost& h = t->vs[i];
        const int ni3 = (h.od[2] + split - 1) / split;
        if ((int64_t)h.od[3] * ((h.od[4] + 1) / 2) * ((ni3 + 3) / 4) > shell_tile_blocks(nt) * (int64_t)nt) return false;
    }
    return true;
}

// largest x chunk <= cap whose shared memory fits the CTA size's limit; 0 if none
static int shell_max_xc(const ShellDims& d, int mode, int nt, int split, int cap) {
    const int mni3 = (d.mdi3 + split - 1) / split;
    for (int xc = std::max(1, std::min(cap, 16)); xc >= 1; xc--)
        if (sf_shell_smem_doubles(d.mdi, d.mdk, d.mk3u, xc, d.Dmax, mni3, mode) * sizeof(double) <= shell_smem_limit(nt))
            return xc;
    return 0;
}

// Resolve a requested tiling (0 fields = choose) into a configuration. Default: two CTAs per SM
// on whole tiles when the tile fits with an x chunk of at least 4, else one CTA of 512 threads.
// Half tiles (measured slower at spin 8, where only they give two CTAs per SM: the duplicated
// staging costs more than the overlap gains) are used only when requested.
static int shell_config(const sf_tables* t, int mode, const sf_tiling& req, ShellConfig* out,
                        const VertexMask* m = nullptr) {
    if (req.x_chunk < 0 || req.x_chunk > 16) return sf_set_error(SF_ERR_ARG, "x_chunk must be 0 (default) or 1..16");
    if (req.items_per_sm < 0 || req.items_per_sm > 256) return sf_set_error(SF_ERR_ARG, "items_per_sm must be 0..256");
    if (req.threads != 0 && req.threads != 256 && req.threads != 512 && !(req.threads == 1024 && mode == SF_MIXED_PX))
        return sf_set_error(SF_ERR_ARG, "threads must be 0 (default), 256 or 512 (or 1024 with SF_MIXED_PX)");
    if (req.i3_split < 0 || req.i3_split > 2) return sf_set_error(SF_ERR_ARG, "i3_split must be 0 (default), 1 or 2");
    const ShellDims d = shell_dims(t, m);
    const int cap = req.x_chunk > 0 ? req.x_chunk : 16;
    // SF_MIXED_PX: one CTA of 1024 threads per SM before one of 512 (its staging holds no values
    // in registers, so it fits 64 registers a thread without spilling; 2 % faster at spin 8)
    const int cands[5][2] = {{256, 1}, {1024, 1}, {256, 2}, {512, 1}, {512, 2}};
    const bool explicit_cfg = req.threads != 0 || req.i3_split != 0;
    for (const auto& c : cands) {
        const int nt = c[0], split = c[1];
        if (nt == 1024 && mode != SF_MIXED_PX) continue;
        if (req.threads != 0 && req.threads != nt) continue;
        if (req.i3_split != 0 && req.i3_split != split) continue;
        if (req.i3_split == 0 && split == 2) continue;   // half tiles only on request (duplicated staging)
        if (!shell_tile_fits(t, nt, split, m)) continue;
        const int xc = shell_max_xc(d, mode, nt, split, cap);
        if (xc == 0) continue;
        if (!explicit_cfg && nt == 256 && xc < std::min(4, cap)) continue;
        out->nt = nt;
        out->split = split;
        out->xc = xc;
        // finer items balance the single 512-thread CTA per SM better (measured 3 % at spins 6-8)
        out->items_per_sm = req.items_per_sm > 0 ? req.items_per_sm : (nt >= 512 ? 16 : 8);
        return SF_OK;
    }
    return sf_set_error(SF_ERR_LIMIT, "intertwiner dimensions too large for the shell kernel with this tiling");
}

// Work decomposition of one shell sum: per vertex, output tiles (i1, i2) x i3 pieces x chunks of
// the (l25, l35, l45) groups in the requested range. Chunk counts scale with the estimated cost of
// an item so that items are of similar size (about items_per_sm of them per SM overall), and the
// costliest vertices are queued first (the kernel takes items in order from an atomic counter).
// Within a vertex the items are chunk-major (all tiles of chunk 0, then chunk 1, ...), so the
// CTAs running at one time read the {6j} slots of the same groups and share them in L2. One
// ReduceJob per (tile, i3 piece) names its chunks (items spaced by tiles x pieces).
struct ShellSchedule {
    std::vector<WorkItem> items;
    std::vector<ReduceJob> jobs;
    int64_t part_total = 0;
    ShellDims dims;
    int mni3 = 1;
};

// Appends the items and jobs of the vertices of mask m (every vertex: null) to sc; item indices
// and partial offsets continue those already in sc, and sc->dims, sc->mni3 describe this call's
// vertices.
static int schedule_shells(const sf_tables* t, bool whole_range, int64_t shell_begin, int64_t shell_end,
                           const ShellConfig& cfg, double* const* A_out, ShellSchedule* sc,
                           const VertexMask* m = nullptr) {
    const int nv = (int)t->vs.size();
    std::vector<int64_t> g_lo(nv), g_n(nv);
    std::vector<double> item_cost_v(nv);
    std::vector<int> ns(nv);
    double total_cost = 0.0;
    for (int i = 0; i < nv; i++) {
        const VertexHost& h = t->vs[i];
        const int64_t per_group = (int64_t)h.D * h.D * h.D;   // shells are group-major: D^3 per group
        if (!in_mask(m, i)) {
            g_lo[i] = 0;
            g_n[i] = 0;
            ns[i] = 1;
            item_cost_v[i] = 0.0;
            continue;
        }
        int64_t lo = 0, hi = h.ngroups;
        if (!whole_range) {
            int64_t b = std::min<int64_t>(std::max<int64_t>(shell_begin, 0), h.nshell);
            int64_t e = std::min<int64_t>(std::max<int64_t>(shell_end, 0), h.nshell);
            lo = b / per_group;
            hi = (e > b) ? (e + per_group - 1) / per_group : lo;
        }
        g_lo[i] = lo;
        g_n[i] = std::max<int64_t>(hi - lo, 0);
        ns[i] = std::min(cfg.split, (int)h.od[2]);
        double dmax = std::max(std::max(h.od[2], h.od[3]), h.od[4]);
        item_cost_v[i] = (double)g_n[i] * per_group * dmax * dmax * dmax * dmax / ns[i];
        total_cost += item_cost_v[i] * h.od[0] * h.od[1] * ns[i];
    }
    const double item_cost = std::max(1.0, total_cost / ((double)t->num_sms * std::max(1, cfg.items_per_sm)));
    std::vector<int> order(nv);
    for (int i = 0; i < nv; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return item_cost_v[a] > item_cost_v[b]; });
    std::vector<int> item0(nv), nchunk(nv);
    for (int i : order) {
        if (!in_mask(m, i)) continue;
        const VertexHost& h = t->vs[i];
        const int64_t ntile = (int64_t)h.od[0] * h.od[1];
        const int64_t ng = g_n[i];
        int C = (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(ng, 1),
                                                            (int64_t)std::ceil(item_cost_v[i] / item_cost)));
        item0[i] = (int)sc->items.size();
        nchunk[i] = C;
        for (int c = 0; c < C; c++) {
            for (int64_t tile = 0; tile < ntile; tile++) {
                for (int hp = 0; hp < ns[i]; hp++) {
                    WorkItem w{};
                    w.vtx = i;
                    w.i1 = (int)(h.olo[0] + tile / h.od[1]);
                    w.i2 = (int)(h.olo[1] + tile % h.od[1]);
                    w.g0 = (int)(g_lo[i] + ng * c / C);
                    w.g1 = (int)(g_lo[i] + ng * (c + 1) / C);
                    w.i3b = (int16_t)(h.olo[2] + h.od[2] * hp / ns[i]);
                    w.ni3 = (int16_t)(h.olo[2] + h.od[2] * (hp + 1) / ns[i] - w.i3b);
                    w.part_off = sc->part_total;
                    sc->part_total += (int64_t)w.ni3 * h.od[3] * h.od[4];
                    sc->items.push_back(w);
                }
            }
        }
        if (sc->items.size() > (size_t)0x7FFFFFFF) return sf_set_error(SF_ERR_LIMIT, "too many work items");
    }
    if (!shell_tile_fits(t, cfg.nt, cfg.split, m))
        return sf_set_error(SF_ERR_LIMIT, "intertwiner dimensions too large for the register-resident tile");
    sc->dims = shell_dims(t, m);
    sc->mni3 = (sc->dims.mdi3 + cfg.split - 1) / cfg.split;
    for (int i = 0; i < nv; i++) {
        if (!in_mask(m, i)) continue;
        const VertexHost& h = t->vs[i];
        const int64_t n3 = (int64_t)h.od[2] * h.od[3] * h.od[4];
        for (int tile = 0; tile < h.od[0] * h.od[1]; tile++) {
            for (int hp = 0; hp < ns[i]; hp++) {
                ReduceJob j{};
                j.vtx = i;
                j.tile = tile;
                j.item0 = item0[i] + tile * ns[i] + hp;
                j.nchunk = nchunk[i];
                j.stride = h.od[0] * h.od[1] * ns[i];
                j.i3b = h.olo[2] + h.od[2] * hp / ns[i];
                j.ni3 = h.olo[2] + h.od[2] * (hp + 1) / ns[i] - j.i3b;
                j.A = A_out[i] + tile * n3 + (int64_t)(j.i3b - h.olo[2]) * h.od[3] * h.od[4];
                sc->jobs.push_back(j);
            }
        }
    }
    return SF_OK;
}

// per-shell norms of the kappa pass: for each shell q of a batch, the square root of the sum of its
// items' squared tile norms (nper consecutive items per shell), summed in item order
__global__ void k_kappa_shells(const double* __restrict__ q2, int64_t nshells, int nper, double* __restrict__ out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nshells) return;
    double s = 0.0;
    for (int c = 0; c < nper; c++) s += q2[q * nper + c];
    out[q] = sqrt(s);
}

// kappa_out[v] = sum over the selected non-empty shells s of ||C_s||_2 (FP64): one work item per
// (shell, output tile, i3 piece) restricted to that shell, in batches of at most KAPPA_BATCH items
#define KAPPA_BATCH (1 << 21)
static int kappa_pass(sf_tables* t, const int64_t* shell_list, int64_t n_list, int64_t shell_begin, int64_t shell_end,
                      ShellFilter filt, double* kappa_out, cudaStream_t stream) {
    ShellConfig cfg;
    SF_TRY(shell_config(t, 0, sf_tiling{}, &cfg));
    const ShellDims dm = shell_dims(t);
    const int mni3 = (dm.mdi3 + cfg.split - 1) / cfg.split;
    std::vector<int64_t> list;
    if (shell_list) {
        // the list may be host or device memory (the shell-sum pass copies it the same way)
        list.resize((size_t)n_list);
        if (n_list > 0)
            SF_CUDA_TRY(cudaMemcpy(list.data(), shell_list, (size_t)n_list * sizeof(int64_t), cudaMemcpyDefault));
        std::sort(list.begin(), list.end());
        list.erase(std::unique(list.begin(), list.end()), list.end());
    }
    const size_t o_q2 = align256((size_t)KAPPA_BATCH * sizeof(WorkItem));
    const size_t o_norm = align256(o_q2 + (size_t)KAPPA_BATCH * sizeof(double));
    const size_t o_counter = align256(o_norm + (size_t)KAPPA_BATCH * sizeof(double));
    const size_t need = o_counter + 256;
    void* buf = nullptr;
    {
        cudaError_t e = cudaMalloc(&buf, need);
        if (e != cudaSuccess) return sf_set_error(SF_ERR_OOM, "kappa pass: %zu bytes of scratch: %s", need, cudaGetErrorString(e));
    }
    WorkItem* d_items = (WorkItem*)buf;
    double* d_q2 = (double*)((char*)buf + o_q2);
    double* d_norm = (double*)((char*)buf + o_norm);
    int* d_counter = (int*)((char*)buf + o_counter);
    int grid = 0;
    size_t smem = 0;
    int rc = sf_shell_prepare(0, cfg.nt, dm.mdi, dm.mdk, dm.mk3u, cfg.xc, dm.Dmax, mni3, KAPPA_BATCH, t->num_sms, &grid, &smem);
    std::vector<double> kap(t->vs.size(), 0.0);
    std::vector<WorkItem> items;
    std::vector<double> norms;
    items.reserve(KAPPA_BATCH);
    for (size_t vi = 0; vi < t->vs.size() && rc == SF_OK; vi++) {
        const VertexHost& h = t->vs[vi];
        const int D = h.D;
        const int32_t* j = h.v.two_j;
        const int ns = std::min(cfg.split, (int)h.od[2]);
        const int nper = h.od[0] * h.od[1] * ns;
        int64_t nsel = 0;
        auto flush = [&]() -> int {
            if (items.empty()) return SF_OK;
            const int64_t nsh = (int64_t)items.size() / nper;
            SF_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, stream));
            const int g = std::min<int>(grid, (int)items.size());
            SF_TRY(sf_shell_launch_prepared(0, cfg.nt, g, smem, t->d_vtx, dm.mdi, dm.mdk, dm.mk3u, cfg.xc, dm.Dmax, mni3,
                                            d_items, (int)items.size(), d_counter, d_q2, filt, stream));
            k_kappa_shells<<<(unsigned)((nsh + 127) / 128), 128, 0, stream>>>(d_q2, nsh, nper, d_norm);
            sf_note_launch(1);
            SF_CUDA_TRY(cudaGetLastError());
            norms.resize(nsh);
            SF_CUDA_TRY(cudaMemcpyAsync(norms.data(), d_norm, nsh * sizeof(double), cudaMemcpyDeviceToHost, stream));
            SF_CUDA_TRY(cudaStreamSynchronize(stream));
            for (int64_t q = 0; q < nsh; q++) kap[vi] += norms[q];   // shell order: deterministic
            items.clear();
            return SF_OK;
        };
        auto add_shell = [&](int64_t s) -> int {
            const int d23 = (int)(s % D), d34 = (int)((s / D) % D), d24 = (int)((s / ((int64_t)D * D)) % D);
            const int64_t g = s / ((int64_t)D * D * D);
            const int d45 = (int)(g % D), d35 = (int)((g / D) % D), d25 = (int)(g / ((int64_t)D * D));
            const int l23 = j[F23] + 2 * d23, l24 = j[F24] + 2 * d24, l25 = j[F25] + 2 * d25;
            const int l34 = j[F34] + 2 * d34, l35 = j[F35] + 2 * d35, l45 = j[F45] + 2 * d45;
            int lo, n2, n3, n4, n5;
            sf_pair_range(l23, l24, l25, j[F12], &lo, &n2);
            sf_pair_range(l34, l35, j[F13], l23, &lo, &n3);
            sf_pair_range(l45, j[F14], l24, l34, &lo, &n4);
            sf_pair_range(j[F15], l25, l35, l45, &lo, &n5);
            if (!n2 || !n3 || !n4 || !n5) return SF_OK;   // an empty shell contributes nothing
            nsel++;
            for (int64_t tile = 0; tile < (int64_t)h.od[0] * h.od[1]; tile++)
                for (int hp = 0; hp < ns; hp++) {
                    WorkItem w{};
                    w.vtx = (int)vi;
                    w.i1 = (int)(h.olo[0] + tile / h.od[1]);
                    w.i2 = (int)(h.olo[1] + tile % h.od[1]);
                    w.g0 = (int)g;
                    w.g1 = (int)g + 1;
                    w.i3b = (int16_t)(h.olo[2] + h.od[2] * hp / ns);
                    w.ni3 = (int16_t)(h.olo[2] + h.od[2] * (hp + 1) / ns - w.i3b);
                    w.part_off = (int64_t)items.size();
                    w.single = 1 + 64 * (d24 * D + d34) + d23;
                    items.push_back(w);
                }
            if (items.size() + (size_t)nper > (size_t)KAPPA_BATCH) return flush();
            return SF_OK;
        };
        if (nper > KAPPA_BATCH) { rc = sf_set_error(SF_ERR_LIMIT, "kappa pass: too many tiles per shell"); break; }
        if (shell_list) {
            for (int64_t s : list)
                if (s >= 0 && s < h.nshell && (rc = add_shell(s)) != SF_OK) break;
        } else {
            const int64_t b = std::min<int64_t>(std::max<int64_t>(shell_begin, 0), h.nshell);
            const int64_t e = std::min<int64_t>(std::max<int64_t>(shell_end, 0), h.nshell);
            for (int64_t s = b; s < e && rc == SF_OK; s++) rc = add_shell(s);
        }
        if (rc == SF_OK) rc = flush();
    }
    if (rc == SF_OK) {
        cudaError_t e = cudaMemcpyAsync(kappa_out, kap.data(), kap.size() * sizeof(double), cudaMemcpyDefault, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) rc = sf_set_error(SF_ERR_CUDA, "kappa copy: %s", cudaGetErrorString(e));
    }
    cudaStreamSynchronize(stream);
    cudaFree(buf);
    return rc;
}

// Launch classes of a shell sum with the default tiling. A batch whose largest vertex needs one
// CTA per SM would otherwise run every vertex that way; the vertices whose tiles fit two CTAs of
// 256 threads per SM (with an x chunk of at least 4) then run in a launch of their own on a second
// stream, whose CTAs take the SMs that the first launch's CTAs leave (two CTAs per SM interleave
// their phases: measured 20 % faster at spin 5). One class otherwise.
struct LaunchClass {
    VertexMask mask;
    ShellConfig cfg;
    size_t item0 = 0, nitems = 0;
    ShellDims dims;
    int mni3 = 1;
};

static int launch_classes(const sf_tables* t, int mode, std::vector<LaunchClass>* out) {
    const size_t nv = t->vs.size();
    LaunchClass all;
    all.mask.assign(nv, 1);
    SF_TRY(shell_config(t, mode, sf_tiling{}, &all.cfg));
    if (nv > 1 && all.cfg.nt != 256) {
        LaunchClass large, small;
        large.mask.assign(nv, 0);
        small.mask.assign(nv, 0);
        bool any_small = false, any_large = false;
        for (size_t i = 0; i < nv; i++) {
            VertexMask one(nv, 0);
            one[i] = 1;
            ShellConfig c;
            const bool two = shell_config(t, mode, sf_tiling{}, &c, &one) == SF_OK && c.nt == 256;
            (two ? small.mask : large.mask)[i] = 1;
            any_small = any_small || two;
            any_large = any_large || !two;
        }
        if (any_small && any_large && shell_config(t, mode, sf_tiling{}, &large.cfg, &large.mask) == SF_OK &&
            shell_config(t, mode, sf_tiling{}, &small.cfg, &small.mask) == SF_OK) {
            sf_clear_error();
            out->push_back(std::move(large));
            out->push_back(std::move(small));
            return SF_OK;
        }
        sf_clear_error();
    }
    out->push_back(std::move(all));
    return SF_OK;
}

extern "C" int sf_vertex_amplitude(sf_tables* t, sf_precision precision, int64_t shell_begin, int64_t shell_end,
                                   const int64_t* shell_list, int64_t n_list, double* const* A_out, double* kappa_out,
                                   cudaStream_t stream) {
    if (!t || !A_out) return sf_set_error(SF_ERR_ARG, "null argument");
    if (precision != SF_FP64 && precision != SF_MIXED && precision != SF_MIXED_FF && precision != SF_MIXED_TC &&
        precision != SF_MIXED_PX)
        return sf_set_error(SF_ERR_ARG, "unknown precision");
    if (shell_list && t->vs.size() != 1) return sf_set_error(SF_ERR_ARG, "a shell list needs single-vertex tables");
    if (shell_list && n_list < 0) return sf_set_error(SF_ERR_ARG, "negative list length");
    if (!shell_list && shell_begin < 0) return sf_set_error(SF_ERR_ARG, "negative shell_begin");
    for (size_t i = 0; i < t->vs.size(); i++) {
        if (!t->vs[i].boosters_ready) return sf_set_error(SF_ERR_ARG, "boosters of vertex %zu were never computed or uploaded", i);
        if (!A_out[i]) return sf_set_error(SF_ERR_ARG, "null output for vertex %zu", i);
    }
    SF_TRY(check_covered(t, shell_begin, shell_end, shell_list, n_list));
    const int mix = (int)precision;
    std::vector<LaunchClass> cls;
    SF_TRY(launch_classes(t, mix, &cls));
    ShellSchedule sc;
    for (LaunchClass& c : cls) {
        c.item0 = sc.items.size();
        SF_TRY(schedule_shells(t, shell_list != nullptr, shell_begin, shell_end, c.cfg, A_out, &sc, &c.mask));
        c.nitems = sc.items.size() - c.item0;
        c.dims = sc.dims;
        c.mni3 = sc.mni3;
    }
    // scratch: items | jobs | counters (one per launch) | bitmap | list | partials
    const int64_t nshell0 = t->vs[0].nshell;
    const size_t o_jobs = align256(sc.items.size() * sizeof(WorkItem));
    const size_t o_counter = align256(o_jobs + sc.jobs.size() * sizeof(ReduceJob));
    const size_t o_bitmap = align256(o_counter + cls.size() * sizeof(int));
    const size_t bm_bytes = shell_list ? (size_t)((nshell0 + 31) / 32) * sizeof(uint32_t) : 0;
    const size_t o_list = align256(o_bitmap + bm_bytes);
    const size_t list_bytes = shell_list ? (size_t)std::max<int64_t>(1, n_list) * sizeof(int64_t) : 0;
    const size_t o_part = align256(o_list + list_bytes);
    const size_t total = align256(o_part + (size_t)sc.part_total * sizeof(double));
    SF_TRY(grow_scratch(t, total));
    char* base = (char*)t->d_scratch;
    WorkItem* d_items = (WorkItem*)base;
    ReduceJob* d_jobs = (ReduceJob*)(base + o_jobs);
    int* d_counter = (int*)(base + o_counter);
    double* d_part = (double*)(base + o_part);
    SF_CUDA_TRY(cudaMemcpyAsync(d_items, sc.items.data(), sc.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, stream));
    SF_CUDA_TRY(cudaMemcpyAsync(d_jobs, sc.jobs.data(), sc.jobs.size() * sizeof(ReduceJob), cudaMemcpyHostToDevice, stream));
    ShellFilter filt{};
    filt.begin = shell_begin;
    filt.end = shell_end;
    filt.bitmap = nullptr;
    if (shell_list) {
        uint32_t* d_bm = (uint32_t*)(base + o_bitmap);
        int64_t* d_list = (int64_t*)(base + o_list);
        if (n_list > 0) SF_CUDA_TRY(cudaMemcpyAsync(d_list, shell_list, n_list * sizeof(int64_t), cudaMemcpyDefault, stream));
        SF_TRY(sf_bitmap_launch(d_list, n_list, nshell0, d_bm, stream));
        filt.bitmap = d_bm;
    }
    std::vector<int> grids(cls.size(), 0);
    std::vector<size_t> smems(cls.size(), 0);
    for (size_t c = 0; c < cls.size(); c++) {
        if (cls[c].nitems == 0) continue;
        const ShellDims& dm = cls[c].dims;
        SF_TRY(sf_shell_prepare(mix, cls[c].cfg.nt, dm.mdi, dm.mdk, dm.mk3u, cls[c].cfg.xc, dm.Dmax, cls[c].mni3,
                                (int)cls[c].nitems, t->num_sms, &grids[c], &smems[c]));
    }
    SF_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), stream));
    // events destroyed on every return path (destroying an event with work pending is allowed)
    struct EventPair {
        cudaEvent_t a = nullptr, b = nullptr;
        ~EventPair() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } evs;
    SF_CUDA_TRY(cudaEventCreate(&evs.a));
    SF_CUDA_TRY(cudaEventCreate(&evs.b));
    cudaEvent_t ev0 = evs.a, ev1 = evs.b;
    SF_CUDA_TRY(cudaEventRecord(ev0, stream));
    // the second class runs on a second stream, so that its CTAs take the SMs the first launch's
    // persistent CTAs leave at its tail; the caller's stream waits for both before the reduction
    const bool two = cls.size() > 1 && cls[0].nitems > 0 && cls[1].nitems > 0;
    if (two && !t->side) SF_CUDA_TRY(cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking));
    if (two) SF_CUDA_TRY(cudaStreamWaitEvent(t->side, ev0, 0));
    for (size_t c = 0; c < cls.size(); c++) {
        if (cls[c].nitems == 0) continue;
        const ShellDims& dm = cls[c].dims;
        SF_TRY(sf_shell_launch_prepared(mix, cls[c].cfg.nt, grids[c], smems[c], t->d_vtx, dm.mdi, dm.mdk, dm.mk3u,
                                        cls[c].cfg.xc, dm.Dmax, cls[c].mni3, d_items + cls[c].item0, (int)cls[c].nitems,
                                        d_counter + c, d_part, filt, (two && c > 0) ? t->side : stream));
    }
    if (two) {
        cudaEvent_t join = nullptr;
        SF_CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(join, t->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, join, 0);
        cudaEventDestroy(join);
        SF_CUDA_TRY(e);
    }
    SF_CUDA_TRY(cudaEventRecord(ev1, stream));
    SF_TRY(sf_reduce_jobs_launch(t->d_vtx, d_jobs, (int)sc.jobs.size(), d_items, d_part, stream));
    int rc = check_status(t, stream, "sf_vertex_amplitude");
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess) g_last_kernel_ms = ms;
    if (rc == SF_OK && kappa_out) {
        rc = kappa_pass(t, shell_list, n_list, shell_begin, shell_end, filt, kappa_out, stream);
        if (rc == SF_OK) rc = check_status(t, stream, "sf_vertex_amplitude (kappa)");
    }
    return rc;
}

// ----------------------------------------------------------------------------------------------
// planned shell sums: host decisions once, then stream-only runs (capturable in a CUDA graph)
// ----------------------------------------------------------------------------------------------
struct sf_plan {
    sf_tables* t = nullptr;
    int mix = 0;   // shell-kernel mode (the sf_precision value)
    int64_t begin = 0, end = 0;
    std::vector<double*> A;
    sf_tiling tiling{};
    ShellConfig cfg;
    ShellSchedule sc;
    int grid = 0;
    size_t smem = 0;
    void* d_buf = nullptr;
    size_t buf_bytes = 0;
    WorkItem* d_items = nullptr;
    ReduceJob* d_jobs = nullptr;
    int* d_counter = nullptr;
    double* d_part = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void plan_drop_graph(sf_plan* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

// (re)build the schedule, kernel configuration and device buffer of a plan for a tiling
static int plan_build(sf_plan* p, const sf_tiling& req) {
    plan_drop_graph(p);
    ShellConfig cfg;
    SF_TRY(shell_config(p->t, p->mix, req, &cfg));
    ShellSchedule sc;
    SF_TRY(schedule_shells(p->t, false, p->begin, p->end, cfg, p->A.data(), &sc));
    int grid = 0;
    size_t smem = 0;
    const ShellDims& dm = sc.dims;
    SF_TRY(sf_shell_prepare(p->mix, cfg.nt, dm.mdi, dm.mdk, dm.mk3u, cfg.xc, dm.Dmax, sc.mni3, (int)sc.items.size(),
                            p->t->num_sms, &grid, &smem));
    const size_t o_jobs = align256(sc.items.size() * sizeof(WorkItem));
    const size_t o_counter = align256(o_jobs + sc.jobs.size() * sizeof(ReduceJob));
    const size_t o_part = align256(o_counter + sizeof(int));
    const size_t total = align256(o_part + (size_t)sc.part_total * sizeof(double));
    if (total > p->buf_bytes) {
        if (p->d_buf) cudaFree(p->d_buf);
        p->d_buf = nullptr;
        p->buf_bytes = 0;
        cudaError_t e = cudaMalloc(&p->d_buf, total);
        if (e != cudaSuccess) return sf_set_error(SF_ERR_OOM, "plan buffer of %zu bytes: %s", total, cudaGetErrorString(e));
        p->buf_bytes = total;
    }
    char* base = (char*)p->d_buf;
    p->d_items = (WorkItem*)base;
    p->d_jobs = (ReduceJob*)(base + o_jobs);
    p->d_counter = (int*)(base + o_counter);
    p->d_part = (double*)(base + o_part);
    // synchronous copies: a later run needs nothing from the host
    SF_CUDA_TRY(cudaMemcpy(p->d_items, sc.items.data(), sc.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice));
    SF_CUDA_TRY(cudaMemcpy(p->d_jobs, sc.jobs.data(), sc.jobs.size() * sizeof(ReduceJob), cudaMemcpyHostToDevice));
    p->sc = std::move(sc);
    p->cfg = cfg;
    p->grid = grid;
    p->smem = smem;
    p->tiling.x_chunk = cfg.xc;
    p->tiling.items_per_sm = cfg.items_per_sm;
    p->tiling.threads = cfg.nt;
    p->tiling.i3_split = cfg.split;
    return SF_OK;
}

static int plan_run(sf_plan* p, cudaStream_t s) {
    ShellFilter filt{};
    filt.begin = p->begin;
    filt.end = p->end;
    filt.bitmap = nullptr;
    const ShellDims& dm = p->sc.dims;
    SF_TRY(sf_shell_launch_prepared(p->mix, p->cfg.nt, p->grid, p->smem, p->t->d_vtx, dm.mdi, dm.mdk, dm.mk3u, p->cfg.xc,
                                    dm.Dmax, p->sc.mni3, p->d_items, (int)p->sc.items.size(), p->d_counter, p->d_part,
                                    filt, s));
    return sf_reduce_jobs_launch(p->t->d_vtx, p->d_jobs, (int)p->sc.jobs.size(), p->d_items, p->d_part, s);
}

extern "C" void sf_plan_free(sf_plan* p) {
    if (!p) return;
    plan_drop_graph(p);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->d_buf) cudaFree(p->d_buf);
    delete p;
}

extern "C" int sf_plan_create(sf_tables* t, sf_precision precision, int64_t shell_begin, int64_t shell_end,
                              const sf_tiling* tiling, double* const* A_out, sf_plan** out) {
    if (!out) return sf_set_error(SF_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (!t || !A_out) return sf_set_error(SF_ERR_ARG, "null argument");
    if (precision != SF_FP64 && precision != SF_MIXED && precision != SF_MIXED_FF && precision != SF_MIXED_TC &&
        precision != SF_MIXED_PX)
        return sf_set_error(SF_ERR_ARG, "unknown precision");
    if (shell_begin < 0) return sf_set_error(SF_ERR_ARG, "negative shell_begin");
    for (size_t i = 0; i < t->vs.size(); i++) {
        if (!t->vs[i].boosters_ready) return sf_set_error(SF_ERR_ARG, "boosters of vertex %zu were never computed or uploaded", i);
        if (!A_out[i]) return sf_set_error(SF_ERR_ARG, "null output for vertex %zu", i);
    }
    SF_TRY(check_covered(t, shell_begin, shell_end, nullptr, 0));
    sf_plan* p = new sf_plan();
    p->t = t;
    p->mix = (int)precision;
    p->begin = shell_begin;
    p->end = shell_end;
    p->A.assign(A_out, A_out + t->vs.size());
    sf_tiling req{};
    if (tiling) req = *tiling;
    int rc = plan_build(p, req);
    if (rc != SF_OK) { sf_plan_free(p); return rc; }
    *out = p;
    return SF_OK;
}

extern "C" int sf_plan_run(sf_plan* p, cudaStream_t s) {
    if (!p) return sf_set_error(SF_ERR_ARG, "null plan");
    return plan_run(p, s);
}

extern "C" int sf_plan_graph_launch(sf_plan* p, cudaStream_t s) {
    if (!p) return sf_set_error(SF_ERR_ARG, "null plan");
    if (!p->exec) {
        if (!p->cap) SF_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
        const int64_t before = sf_kernel_launches();
        SF_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        int rc = plan_run(p, p->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        sf_note_launch(-(int)(sf_kernel_launches() - before));   // capture records, it does not launch
        if (rc != SF_OK) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return sf_set_error(SF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        p->graph = g;
        e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) { plan_drop_graph(p); return sf_set_error(SF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
    }
    SF_CUDA_TRY(cudaGraphLaunch(p->exec, s));
    sf_note_launch(p->sc.jobs.empty() ? 1 : 2);
    return SF_OK;
}

extern "C" int sf_plan_sync(sf_plan* p, cudaStream_t s) {
    if (!p) return sf_set_error(SF_ERR_ARG, "null plan");
    SF_CUDA_TRY(cudaStreamSynchronize(s));
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" int sf_plan_info(const sf_plan* p, sf_tiling* tiling, int64_t* n_items, int32_t* grid, int64_t* scratch_bytes) {
    if (!p) return sf_set_error(SF_ERR_ARG, "null plan");
    if (tiling) *tiling = p->tiling;
    if (n_items) *n_items = (int64_t)p->sc.items.size();
    if (grid) *grid = p->grid;
    if (scratch_bytes) *scratch_bytes = (int64_t)p->buf_bytes;
    return SF_OK;
}

extern "C" int sf_plan_autotune(sf_plan* p, int64_t sample_shells, sf_tiling* chosen, cudaStream_t s) {
    if (!p) return sf_set_error(SF_ERR_ARG, "null plan");
    if (sample_shells <= 0) return sf_set_error(SF_ERR_ARG, "sample_shells must be positive");
    // candidates: CTA shapes (threads, i3 pieces) x x chunks x work granularities, each timed on the
    // first sample_shells shells of the plan's range (every vertex), best of two runs after a warm-up
    static const int shapes[5][2] = {{1024, 1}, {512, 1}, {256, 1}, {256, 2}, {512, 2}};   // 1024: SF_MIXED_PX only
    static const int xcs[] = {16, 8, 4};
    static const int ipss[] = {4, 8, 16};
    sf_plan probe;
    probe.t = p->t;
    probe.mix = p->mix;
    probe.begin = p->begin;
    probe.end = std::min<int64_t>(p->end, p->begin + sample_shells);
    probe.A = p->A;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SF_CUDA_TRY(cudaEventCreate(&e0));
    SF_CUDA_TRY(cudaEventCreate(&e1));
    sf_tiling best{};
    float best_ms = 1e30f;
    int rc = SF_OK;
    std::vector<sf_tiling> tried;
    for (const auto& sh : shapes) {
        for (int xc : xcs) {
            for (int ips : ipss) {
                sf_tiling tl{};
                tl.threads = sh[0];
                tl.i3_split = sh[1];
                tl.x_chunk = xc;
                tl.items_per_sm = ips;
                rc = plan_build(&probe, tl);
                if (rc == SF_ERR_LIMIT || rc == SF_ERR_ARG) { rc = SF_OK; continue; }   // shape does not fit
                if (rc != SF_OK) break;
                bool dup = false;                   // x chunk clamped to one already timed
                for (const sf_tiling& q : tried)
                    dup = dup || (q.threads == probe.tiling.threads && q.i3_split == probe.tiling.i3_split &&
                                  q.x_chunk == probe.tiling.x_chunk && q.items_per_sm == probe.tiling.items_per_sm);
                if (dup) continue;
                tried.push_back(probe.tiling);
                float tmin = 1e30f;
                for (int rep = 0; rep < 3 && rc == SF_OK; rep++) {
                    cudaEventRecord(e0, s);
                    rc = plan_run(&probe, s);
                    cudaEventRecord(e1, s);
                    if (cudaEventSynchronize(e1) != cudaSuccess) rc = sf_set_error(SF_ERR_CUDA, "autotune run failed");
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) tmin = std::min(tmin, ms);
                }
                if (rc != SF_OK) break;
                if (tmin < best_ms) { best_ms = tmin; best = probe.tiling; }
            }
            if (rc != SF_OK) break;
        }
        if (rc != SF_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (probe.d_buf) cudaFree(probe.d_buf);
    probe.d_buf = nullptr;
    plan_drop_graph(&probe);
    if (rc != SF_OK) return rc;
    if (best_ms >= 1e30f) return sf_set_error(SF_ERR_LIMIT, "no tiling fits the plan's vertices");
    SF_TRY(plan_build(p, best));
    if (chosen) *chosen = p->tiling;
    return SF_OK;
}

extern "C" int sf_vertex_adjoint(sf_tables* t, sf_precision precision, const double* const psi[5], double* a_out,
                                 double* const grad_psi[5], double* const grad_B[4], cudaStream_t stream) {
    if (!t || !psi || !a_out) return sf_set_error(SF_ERR_ARG, "null argument");
    if (precision != SF_FP64) return sf_set_error(SF_ERR_ARG, "the adjoint runs in FP64 only (precision %d)", (int)precision);
    if (t->vs.size() != 1) return sf_set_error(SF_ERR_ARG, "the adjoint needs single-vertex tables");
    if (!t->vs[0].boosters_ready) return sf_set_error(SF_ERR_ARG, "boosters were never computed or uploaded");
    for (int e = 0; e < 5; e++) if (!psi[e]) return sf_set_error(SF_ERR_ARG, "null boundary vector %d", e + 1);
    if (grad_psi)
        for (int e = 0; e < 5; e++) if (!grad_psi[e]) return sf_set_error(SF_ERR_ARG, "null grad_psi[%d]", e);
    if (grad_B)
        for (int e = 0; e < 4; e++) if (!grad_B[e]) return sf_set_error(SF_ERR_ARG, "null grad_B[%d]", e);
    const VertexHost& hv = t->vs[0];
    if (hv.restricted) return sf_set_error(SF_ERR_ARG, "the adjoint sums every shell: it needs tables of the whole range");
    for (int e = 0; e < 5; e++)
        if (hv.olo[e] != 0 || hv.od[e] != hv.di[e])
            return sf_set_error(SF_ERR_ARG, "the adjoint needs the whole intertwiner range (edge %d has a sub-range)", e + 1);
    VtxDev h;
    memset(&h, 0, sizeof(h));
    for (int e = 0; e < 5; e++) { h.di[e] = hv.di[e]; h.ilo[e] = hv.ilo[e]; }
    for (int e = 0; e < 4; e++) h.dkmax[e] = hv.dkmax[e];
    h.ntrip = hv.ntrip;
    h.nshell = hv.nshell;
    h.D = hv.D;
    SF_TRY(grow_scratch(t, sf_adjoint_scratch_bytes(h)));
    SF_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), stream));
    SF_TRY(sf_adjoint_launch(t->d_vtx, h, psi, a_out, grad_psi, grad_B, t->d_scratch, t->scratch_bytes, t->num_sms, stream));
    return check_status(t, stream, "sf_vertex_adjoint");
}

// ----------------------------------------------------------------------------------------------
// table export
// ----------------------------------------------------------------------------------------------
static int table_ptr(const sf_tables* t, int32_t vertex, int32_t kind, int32_t index, const void** p, int64_t* bytes,
                     std::vector<int64_t>* host_slots) {
    if (!t) return sf_set_error(SF_ERR_ARG, "null tables");
    if (vertex < 0 || vertex >= (int)t->vs.size()) return sf_set_error(SF_ERR_ARG, "vertex index out of range");
    const VertexHost& h = t->vs[vertex];
    switch (kind) {
        case SF_TAB_6J:
            if (index < 1 || index > 5) return sf_set_error(SF_ERR_ARG, "6j table index must be 1..5");
            *p = h.S[index - 1].d_vals;
            *bytes = h.S[index - 1].n * (int64_t)sizeof(double);
            return SF_OK;
        case SF_TAB_6J_SLOTS: {
            if (index < 1 || index > 5) return sf_set_error(SF_ERR_ARG, "6j table index must be 1..5");
            const auto& sl = h.S[index - 1].slots;
            *bytes = (int64_t)sl.size() * 8 * (int64_t)sizeof(int64_t);
            if (host_slots) {
                host_slots->resize(sl.size() * 8);
                for (size_t i = 0; i < sl.size(); i++) {
                    int64_t* o = host_slots->data() + 8 * i;
                    o[0] = sl[i].off; o[1] = sl[i].alo; o[2] = sl[i].blo; o[3] = sl[i].xlo;
                    o[4] = sl[i].na; o[5] = sl[i].nb; o[6] = sl[i].nx; o[7] = 0;
                }
            }
            *p = nullptr;
            return SF_OK;
        }
        case SF_TAB_D:
            if (index < 0 || index > 9) return sf_set_error(SF_ERR_ARG, "face index must be 0..9");
            if (!h.d_dtab[index]) return sf_set_error(SF_ERR_ARG, "d-tables not computed");
            *p = h.d_dtab[index];
            *bytes = (int64_t)h.nl[index] * (h.v.two_j[index] + 1) * t->nnodes * (int64_t)sizeof(double2);
            return SF_OK;
        case SF_TAB_NODES:
            if (!t->have_rule) return sf_set_error(SF_ERR_ARG, "rule not computed");
            if (index < 0 || index > 2) return sf_set_error(SF_ERR_ARG, "node table index must be 0..2");
            *p = index == 0 ? t->d_x : index == 1 ? t->d_w : t->d_r;
            *bytes = t->nnodes * (int64_t)sizeof(double);
            return SF_OK;
        default:
            return sf_set_error(SF_ERR_ARG, "unknown table kind");
    }
}

extern "C" int64_t sf_table_size(const sf_tables* t, int32_t vertex, int32_t kind, int32_t index) {
    const void* p;
    int64_t b = 0;
    int r = table_ptr(t, vertex, kind, index, &p, &b, nullptr);
    return r == SF_OK ? b : r;
}

extern "C" int sf_table_copy(const sf_tables* t, int32_t vertex, int32_t kind, int32_t index, void* dst, int64_t n_bytes,
                             cudaStream_t stream) {
    const void* p;
    int64_t b = 0;
    std::vector<int64_t> hs;
    SF_TRY(table_ptr(t, vertex, kind, index, &p, &b, &hs));
    if (!dst || n_bytes < b) return sf_set_error(SF_ERR_ARG, "destination too small (%lld < %lld bytes)", (long long)n_bytes, (long long)b);
    if (kind == SF_TAB_6J_SLOTS) {
        SF_CUDA_TRY(cudaMemcpyAsync(dst, hs.data(), b, cudaMemcpyDefault, stream));
    } else {
        SF_CUDA_TRY(cudaMemcpyAsync(dst, p, b, cudaMemcpyDefault, stream));
    }
    SF_CUDA_TRY(cudaStreamSynchronize(stream));
    return SF_OK;
}

// ----------------------------------------------------------------------------------------------
// vertex amplitude without any device allocation
//
// For callers that must not allocate device memory once they are running: code that shares the
// GPU with a framework owning a fixed memory pool, hosts that forbid allocation after start-up
// (cudaMalloc/cudaFree can synchronise the device and stall other streams), or callers that keep
// a strict device-memory budget. Such a caller builds its tables during start-up and then calls
// this entry point, which takes every scratch byte from one file-scope device array.
// ----------------------------------------------------------------------------------------------
#include <mutex>

#define SF_NOALLOC_SCRATCH_BYTES (32ull << 20)   // 32 MiB, held on every GPU that loads the library

static __device__ __align__(256) unsigned char g_noalloc_scratch[SF_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_addr[128];   // device address of g_noalloc_scratch, per device ordinal

// once per device, with that device current: the host-side symbol is only a stand-in, the
// kernels need the device address
static int noalloc_scratch(void** out) {
    int dev = 0;
    SF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return sf_set_error(SF_ERR_LIMIT, "device ordinal %d beyond 127", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return sf_set_error(SF_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return SF_OK;
}

extern "C" int sf_vertex_amplitude_noalloc(sf_tables* t, int64_t shell_begin, int64_t shell_end, double* const* A_out,
                                           cudaStream_t stream) {
    if (!t || !A_out) return sf_set_error(SF_ERR_ARG, "null argument");
    if (shell_begin < 0) return sf_set_error(SF_ERR_ARG, "negative shell_begin");
    for (size_t i = 0; i < t->vs.size(); i++) {
        if (!t->vs[i].boosters_ready) return sf_set_error(SF_ERR_ARG, "boosters of vertex %zu were never computed or uploaded", i);
        if (!A_out[i]) return sf_set_error(SF_ERR_ARG, "null output for vertex %zu", i);
    }
    SF_TRY(check_covered(t, shell_begin, shell_end, nullptr, 0));
    const int nv = (int)t->vs.size();
    // one work item per (vertex, i1, i2) tile covering the requested groups: the smallest scratch
    std::vector<WorkItem> items;
    std::vector<int> item0(nv);
    int64_t part_total = 0;
    int mdi = 1, mdk = 1, mk3u = 1, Dmax = 1;
    for (int i = 0; i < nv; i++) {
        VertexHost& h = t->vs[i];
        const int64_t per_group = (int64_t)h.D * h.D * h.D;
        int64_t b = std::min<int64_t>(shell_begin, h.nshell), e = std::min<int64_t>(std::max<int64_t>(shell_end, 0), h.nshell);
        int64_t lo = b / per_group, hi = (e > b) ? (e + per_group - 1) / per_group : lo;
        item0[i] = (int)items.size();
        const int64_t per = (int64_t)h.od[2] * h.od[3] * h.od[4];
        for (int64_t tile = 0; tile < (int64_t)h.od[0] * h.od[1]; tile++) {
            WorkItem w{};
            w.vtx = i;
            w.i1 = (int)(h.olo[0] + tile / h.od[1]);
            w.i2 = (int)(h.olo[1] + tile % h.od[1]);
            w.g0 = (int)lo;
            w.g1 = (int)hi;
            w.i3b = (int16_t)h.olo[2];
            w.ni3 = (int16_t)h.od[2];
            w.part_off = part_total;
            part_total += per;
            items.push_back(w);
        }
        if ((int64_t)h.od[3] * ((h.od[4] + 1) / 2) * ((h.od[2] + 3) / 4) > 4 * 256)
            return sf_set_error(SF_ERR_LIMIT, "vertex %d: intertwiner dimensions too large for the register-resident tile", i);
        for (int k = 2; k < 5; k++) mdi = std::max(mdi, (int)h.od[k]);
        for (int k = 0; k < 4; k++) mdk = std::max(mdk, (int)h.dkmax[k]);
        mk3u = std::max(mk3u, h.mk3u);
        Dmax = std::max(Dmax, h.D);
    }
    int xc = 16;
    while (xc > 1 && sf_shell_smem_doubles(mdi, mdk, mk3u, xc, Dmax, mdi, false) * sizeof(double) > 200 * 1024) xc--;
    if (sf_shell_smem_doubles(mdi, mdk, mk3u, xc, Dmax, mdi, false) * sizeof(double) > 200 * 1024)
        return sf_set_error(SF_ERR_LIMIT, "intertwiner dimensions too large for the shell kernel");
    // scratch layout: items | counter | partial tiles
    const size_t o_counter = align256(items.size() * sizeof(WorkItem));
    const size_t o_part = align256(o_counter + sizeof(int));
    const size_t need = o_part + (size_t)part_total * sizeof(double);
    if (need > SF_NOALLOC_SCRATCH_BYTES)
        return sf_set_error(SF_ERR_LIMIT, "sf_vertex_amplitude_noalloc needs %zu bytes of scratch, above its fixed %llu; "
                                          "split the shell range, the vertex set, or use sf_vertex_amplitude",
                            need, (unsigned long long)SF_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    SF_TRY(noalloc_scratch(&base));
    char* b8 = (char*)base;
    WorkItem* d_items = (WorkItem*)b8;
    int* d_counter = (int*)(b8 + o_counter);   // zeroed by the launcher before the kernel runs
    double* d_part = (double*)(b8 + o_part);   // every partial tile is fully written by its item
    SF_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, stream));
    ShellFilter filt{};
    filt.begin = shell_begin;
    filt.end = shell_end;
    filt.bitmap = nullptr;
    SF_CUDA_TRY(cudaMemsetAsync(t->d_status, 0, sizeof(int), stream));
    SF_TRY(sf_shell_fp64_launch(t->d_vtx, mdi, mdk, mk3u, xc, Dmax, d_items, (int)items.size(), d_counter, d_part, filt,
                                t->num_sms, stream));
    for (int i = 0; i < nv; i++) {
        VertexHost& h = t->vs[i];
        SF_TRY(sf_reduce_launch(t->d_vtx, i, h.od[0] * h.od[1], d_items, item0[i], 1, d_part, A_out[i], stream));
    }
    return check_status(t, stream, "sf_vertex_amplitude_noalloc");
}
