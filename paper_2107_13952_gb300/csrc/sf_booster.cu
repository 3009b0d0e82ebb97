// Boosters B4^gamma (Sec. 2 eq. booster; Sec. 3 "Booster coefficients"):
//   1. Gauss-Legendre nodes (Newton iteration in the angle variable, FP64);
//   2. the rapidity rule: panels in x = e^-r with |I_k| = k |I_1|, `order` nodes per panel;
//   3. d-tables d^{rho,k}_{k l m}(r_n) for every face, l and m, from the compact-picture integral
//        d = i^(k-l) Phi_l sqrt((2k+1)(2l+1)) r/(2 sinh r) int_{-1}^{1} dxi d^k_{mk}(beta) d^l_{mk}(beta_r) e^{i rho v},
//      v = r xi = ln u, t = sin^2(beta/2) = (e^v - e^-r)/(2 sinh r), t_r = sin^2(beta_r/2) = (e^r - e^-v)/(2 sinh r),
//      integrated by Gauss-Legendre in v with an r-dependent node count (no cancellation: the
//      integrand is bounded), d^l for all l by the three-term recurrence in l;
//   4. per (edge, virtual-spin triple): I(m) = sum_n W_n prod_a d_a(m_a, r_n) and
//      B[i][k] = Re sum_m 4jm(j;m)^(i) 4jm(l;m)^(k) I(m).
#include "sf_racah.cuh"
#include <algorithm>
#include <mutex>

#define SF_PI 3.14159265358979323846

// ---------------------------------------------------------------------------------------------
// Gauss-Legendre library: for N = 32q, q = 2..32, arrays (1+xi, 1-xi, w), concatenated.
// ---------------------------------------------------------------------------------------------
__host__ __device__ inline int64_t sf_gl_offset(int N) {   // start of size-N rule
    int q = N / 32;
    return 32ll * ((int64_t)(q - 1) * q / 2 - 1);            // 32 * sum_{q'=2}^{q-1} q'
}
#define SF_GL_TOTAL (32ll * (32ll * 33 / 2 - 1))             // sum_{q=2}^{32} 32 q

__device__ inline void sf_gl_node(int N, int i, double* opx, double* omx, double* w) {
    // i-th root of P_N, theta in (0, pi), descending x
    double th = SF_PI * (i + 0.75) / (N + 0.5);
    double x = cos(th), p0 = 1.0, p1 = x;
    for (int it = 0; it < 12; it++) {
        x = cos(th);
        p0 = 1.0;
        p1 = x;
        for (int k = 2; k <= N; k++) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double s = sin(th);
        double dth = p1 * s / (N * (x * p1 - p0));   // theta-Newton step on P_N(cos theta)
        th -= dth;
        if (fabs(dth) < 1e-17) break;
    }
    x = cos(th);
    p0 = 1.0;
    p1 = x;
    for (int k = 2; k <= N; k++) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    double s = sin(th), sh = sin(0.5 * th), ch = cos(0.5 * th);
    double dp = N * (x * p1 - p0);   // = -(1-x^2) P_N'(x)
    *opx = 2.0 * ch * ch;
    *omx = 2.0 * sh * sh;
    *w = 2.0 * s * s / (dp * dp);
}

__global__ void k_gl_library(double* gl) {
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= SF_GL_TOTAL) return;
    int q = 2;
    while (sf_gl_offset(32 * (q + 1)) <= tid) q++;
    int N = 32 * q;
    int i = (int)(tid - sf_gl_offset(N));
    double a, b, c;
    sf_gl_node(N, i, &a, &b, &c);
    gl[tid] = a;
    gl[SF_GL_TOTAL + tid] = b;
    gl[2 * SF_GL_TOTAL + tid] = c;
}

// rapidity rule nodes: x_n, w_n, r_n = -ln x_n, W_n = w_n (1-x^2)^2 / (16 pi x^3)
__global__ void k_rule_nodes(double r_max, int npan, int order, double* X, double* Wt, double* R, double* Wm) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= npan * order) return;
    int kk = n / order + 1, i = n % order;
    double opx, omx, w;
    sf_gl_node(order, order - 1 - i, &opx, &omx, &w);   // ascending x inside the panel
    double x0 = exp(-r_max);
    double Dx = 2.0 * (1.0 - x0) / ((double)npan * (npan + 1));
    double a = x0 + Dx * 0.5 * kk * (kk - 1);
    double top = (1.0 - x0) - Dx * 0.5 * kk * (kk + 1);   // 1 - b, exactly 0 for the last panel
    double h = 0.5 * Dx * kk;
    double x = a + h * opx;
    double one_minus_x = top + h * omx;
    double r = (x < 0.5) ? -log(x) : -log1p(-one_minus_x);
    double omx2 = one_minus_x * (2.0 - one_minus_x);      // 1 - x^2
    X[n] = x;
    Wt[n] = h * w;
    R[n] = r;
    Wm[n] = h * w * omx2 * omx2 / (16.0 * SF_PI * x * x * x);
}

// The library does not depend on any argument, so it is built once per device, on the first
// call that needs it, and kept until the process exits (0.4 MB per device).
static std::mutex g_gl_mutex;
static double* g_gl_lib[SF_MAX_DEVICES];

int sf_gl_library(cudaStream_t s, const double** out) {
    int dev = 0;
    SF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= SF_MAX_DEVICES) return sf_set_error(SF_ERR_LIMIT, "device ordinal %d beyond %d", dev, SF_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_gl_mutex);
    if (!g_gl_lib[dev]) {
        double* p = nullptr;
        cudaError_t e = cudaMalloc(&p, 3 * SF_GL_TOTAL * sizeof(double));
        if (e != cudaSuccess) return sf_set_error(SF_ERR_OOM, "Gauss-Legendre library allocation failed: %s", cudaGetErrorString(e));
        k_gl_library<<<(unsigned)((SF_GL_TOTAL + 255) / 256), 256, 0, s>>>(p);
        sf_note_launch(1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // complete before any other stream reads it
        if (e != cudaSuccess) {
            cudaFree(p);
            return sf_set_error(SF_ERR_CUDA, "Gauss-Legendre library build failed: %s", cudaGetErrorString(e));
        }
        g_gl_lib[dev] = p;
    }
    *out = g_gl_lib[dev];
    return SF_OK;
}

// Stream-ordered scratch from a memory pool of the library's own on each device. The pool keeps
// the memory that is freed into it (no release threshold), so a scratch buffer of the same size
// on the next call is served without mapping new pages; the runtime's default pool, whose
// threshold is zero, would hand the memory back to the driver at every synchronisation.
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pool[SF_MAX_DEVICES];
static bool g_pool_made[SF_MAX_DEVICES];

int sf_scratch_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int dev = 0;
    SF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= SF_MAX_DEVICES) return sf_set_error(SF_ERR_LIMIT, "device ordinal %d beyond %d", dev, SF_MAX_DEVICES);
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        if (!g_pool_made[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            SF_CUDA_TRY(cudaMemPoolCreate(&g_pool[dev], &props));
            uint64_t keep = UINT64_MAX;
            SF_CUDA_TRY(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
            g_pool_made[dev] = true;
        }
        pool = g_pool[dev];
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return sf_set_error(SF_ERR_OOM, "scratch allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    return SF_OK;
}

int sf_scratch_free(void* p, cudaStream_t s) {
    if (!p) return SF_OK;
    SF_CUDA_TRY(cudaFreeAsync(p, s));
    return SF_OK;
}

int sf_rule_build(const sf_quad_rule* q, double* d_x, double* d_w, double* d_r, double* d_W, cudaStream_t s) {
    int n = q->n_panels * q->order;
    k_rule_nodes<<<(n + 127) / 128, 128, 0, s>>>(q->r_max, q->n_panels, q->order, d_x, d_w, d_r, d_W);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// ---------------------------------------------------------------------------------------------
// d-tables
// ---------------------------------------------------------------------------------------------
// Node count of the v-integral at rapidity r: the integrand oscillates as e^{i rho v} on
// [-r, r] and its d-function factors carry polynomial degrees up to about (l + k)/2 in each of
// t and 1 - t, so the count grows linearly in r with that band; at least 64 nodes.
__device__ inline int sf_gl_count(double r, double rho, int tk, int tlmax) {
    double band = rho + 0.25 * (tlmax + tk) + 1.0;
    int N = (int)ceil((48.0 + r * band) / 32.0) * 32;
    return N < 64 ? 64 : N;
}
// The count is met by a composite rule: P equal panels of [-r, r], each with Np <= SF_GL_NMAX
// library nodes (Np a multiple of 32, P Np >= N). P = 1 is the plain rule.
__device__ inline void sf_gl_split(int N, int* P, int* Np) {
    const int p = (N + SF_GL_NMAX - 1) / SF_GL_NMAX;
    int n = (N + p - 1) / p;
    n = ((n + 31) / 32) * 32;
    *P = p;
    *Np = n < 64 ? 64 : n;
}

__device__ inline double ipow_(double b, int e) {
    double r = 1.0;
    for (int i = 0; i < e; i++) r *= b;
    return r;
}

// grid: x = node blocks, y = m index, z = face; all ten faces of a vertex in one launch
#define SF_DT_NT 64
__global__ void __launch_bounds__(SF_DT_NT) k_dtable(const __grid_constant__ DtabFaces fc, int nnodes,
                                                     const double* __restrict__ R, const double* __restrict__ gl) {
    const int face = blockIdx.z;
    const int tk = fc.tk[face], nl = fc.nl[face];
    const double rho = fc.rho[face];
    double2* __restrict__ out = fc.out[face];
    const int im = blockIdx.y;
    if (im > tk) return;   // this face has fewer m values than the largest one (uniform per CTA)
    const int tm = -tk + 2 * im;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    // recurrence coefficients d^{l+1} = (al cos(b) - gl) d^l - de d^{l-1}, l = k + p
    __shared__ double s_al[SF_MAX_DL + 1], s_ga[SF_MAX_DL + 1], s_de[SF_MAX_DL + 1];
    const double k = 0.5 * tk, m = 0.5 * tm;
    if (threadIdx.x == 0) {
        for (int p = 0; p < nl; p++) {
            double l = k + p;
            if (l == 0.0) {   // k = m = 0: d^1_{00} = cos(beta)
                s_al[p] = 1.0; s_ga[p] = 0.0; s_de[p] = 0.0;
                continue;
            }
            double s2 = sqrt(((l + 1) * (l + 1) - m * m) * ((l + 1) * (l + 1) - k * k));
            double s1 = sqrt(fmax(0.0, (l * l - m * m) * (l * l - k * k)));
            s_al[p] = (2 * l + 1) * (l + 1) / s2;
            s_ga[p] = (2 * l + 1) * m * k / (l * s2);
            s_de[p] = (l + 1) * s1 / (l * s2);
        }
    }
    __syncthreads();
    if (n >= nnodes) return;
    const double r = R[n];
    const double emr = exp(-r);
    const double sh2 = 2.0 * sinh(r);   // 2 sinh r (not e^r - e^-r, which cancels at small r)
    const double ish2 = 1.0 / sh2;      // one division per node; the integrand multiplies by it
    const int kpm = (tk + tm) / 2, kmm = (tk - tm) / 2;
    double sqc = 1.0;              // sqrt(C(2k, k+m))
    {
        double c = 1.0;
        for (int i = 1; i <= kpm; i++) c = c * (kmm + i) / i;
        sqc = sqrt(c);
    }
    const int tlmax = tk + 2 * (nl - 1);
    int P = 1, Np = 64;
    sf_gl_split(sf_gl_count(r, rho, tk, tlmax), &P, &Np);
    const int64_t go = sf_gl_offset(Np);
    const double* gp = gl + go;
    const double* gm = gl + SF_GL_TOTAL + go;
    const double* gw = gl + 2 * SF_GL_TOTAL + go;
    const double rp = r / P, wscale = 1.0 / P;
    for (int c0 = 0; c0 < nl; c0 += SF_DT_LCHUNK) {
        double are[SF_DT_LCHUNK], aim[SF_DT_LCHUNK];
#pragma unroll
        for (int q = 0; q < SF_DT_LCHUNK; q++) { are[q] = 0.0; aim[q] = 0.0; }
        for (int jj = 0; jj < P * Np; jj++) {
            // panel pp covers 1 + xi in [2 pp / P, 2 (pp + 1) / P]; the distances of the node from
            // both ends of [-r, r] are formed directly, so nothing cancels near either end
            const int pp = jj / Np, j = jj - pp * Np;
            const double opx = gp[j], omx = gm[j], w = gw[j] * wscale;
            const double a1 = (P == 1) ? r * opx : rp * (2.0 * pp + opx);              // v + r
            const double a2 = (P == 1) ? r * omx : rp * (2.0 * (P - 1 - pp) + omx);    // r - v
            const double v = (a1 <= a2) ? (a1 - r) : (r - a2);
            const double ev = exp(v), emv = 1.0 / ev;
            const double A = expm1(a1);   // e^{v+r} - 1
            const double Bq = expm1(a2);  // e^{r-v} - 1
            const double t = fmin(1.0, emr * A * ish2), omt = fmin(1.0, ev * Bq * ish2);
            const double tr = fmin(1.0, emv * A * ish2), omtr = fmin(1.0, emr * Bq * ish2);
            const double dk = sqc * ipow_(sqrt(omt), kpm) * ipow_(sqrt(t), kmm);
            double sn, cs;
            sincos(rho * v, &sn, &cs);
            const double wd = w * dk;
            const double pr = wd * cs, pi = wd * sn;
            const double cb = omtr - tr;   // cos(beta_r)
            double dprev = 0.0, dcur = sqc * ipow_(sqrt(omtr), kpm) * ipow_(sqrt(tr), kmm);
            int p = 0;
            for (; p < c0; p++) {
                double dn = (s_al[p] * cb - s_ga[p]) * dcur - s_de[p] * dprev;
                dprev = dcur;
                dcur = dn;
            }
#pragma unroll
            for (int q = 0; q < SF_DT_LCHUNK; q++) {
                if (c0 + q < nl) {
                    are[q] = fma(pr, dcur, are[q]);
                    aim[q] = fma(pi, dcur, aim[q]);
                    if (c0 + q + 1 < nl) {
                        double dn = (s_al[c0 + q] * cb - s_ga[c0 + q]) * dcur - s_de[c0 + q] * dprev;
                        dprev = dcur;
                        dcur = dn;
                    }
                }
            }
        }
        // prefactor i^(k-l) Phi_l sqrt((2k+1)(2l+1)) r / (2 sinh r)
        double phr = 1.0, phi = 0.0;   // Phi_l, built up from l = k
        for (int p = 0; p < c0; p++) {
            double nn = k + p + 1, den = sqrt(nn * nn + rho * rho);
            double ur = nn / den, ui = -rho / den;
            double a = phr * ur - phi * ui, b = phr * ui + phi * ur;
            phr = a; phi = b;
        }
#pragma unroll
        for (int q = 0; q < SF_DT_LCHUNK; q++) {
            int p = c0 + q;
            if (p < nl) {
                double l = k + p;
                double sc = sqrt((2 * k + 1) * (2 * l + 1)) * r / sh2;
                // i^(k-l) = (-i)^p
                double zr = phr, zi = phi;
                switch (p & 3) {
                    case 0: break;
                    case 1: { double a = zi, b = -zr; zr = a; zi = b; } break;   // * (-i)
                    case 2: { zr = -zr; zi = -zi; } break;
                    default: { double a = -zi, b = zr; zr = a; zi = b; } break;  // * i
                }
                double vr = are[q] * zr - aim[q] * zi, vi = are[q] * zi + aim[q] * zr;
                out[((int64_t)p * (tk + 1) + im) * nnodes + n] = make_double2(sc * vr, sc * vi);
                // advance Phi to l+1
                double nn = l + 1, den = sqrt(nn * nn + rho * rho);
                double ur = nn / den, ui = -rho / den;
                double a = phr * ur - phi * ui, b = phr * ui + phi * ur;
                phr = a; phi = b;
            }
        }
    }
}

int sf_dtable_build(const int tk[10], double gamma, const int nl[10], int nnodes, const double* d_r, const double* d_gl,
                    double2* const d_out[10], cudaStream_t s) {
    DtabFaces fc{};
    int mmax = 1;
    for (int f = 0; f < 10; f++) {
        if (nl[f] > SF_MAX_DL + 1) return sf_set_error(SF_ERR_LIMIT, "dl too large for the d-table kernel");
        fc.tk[f] = tk[f];
        fc.nl[f] = nl[f];
        fc.rho[f] = gamma * (0.5 * tk[f] + 1.0);
        fc.out[f] = d_out[f];
        mmax = std::max(mmax, tk[f] + 1);
    }
    dim3 grid((nnodes + SF_DT_NT - 1) / SF_DT_NT, mmax, 10);
    k_dtable<<<grid, SF_DT_NT, 0, s>>>(fc, nnodes, d_r, d_gl);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// ---------------------------------------------------------------------------------------------
// boosters
// ---------------------------------------------------------------------------------------------
// strands of each edge in coupling order: face index and which free-face offset (0..2 of the
// triple, or -1 for the gauge face)
__constant__ int c_edge_face[4][4] = {{F23, F24, F25, F12}, {F34, F35, F13, F23}, {F45, F14, F24, F34}, {F15, F25, F35, F45}};
__constant__ int c_edge_slot[4][4] = {{0, 1, 2, -1}, {0, 1, -1, 2}, {0, -1, 1, 2}, {-1, 0, 1, 2}};

// nodes per staged chunk: as many as keep the staged pair tables within SF_NC_BYTES (so that two
// CTAs fit per SM), a power of two between 16 and 1024; small spins stage many nodes per barrier
#define SF_NC_BYTES (80 * 1024)
int sf_booster_chunk(int tj1, int tj2, int tj3, int tj4) {
    const int n12 = (tj1 + 1) * (tj2 + 1), n34 = (tj3 + 1) * (tj4 + 1);
    const size_t per_node = (size_t)((n12 - n12 / 2) + (n34 - n34 / 2)) * sizeof(double2);
    int nc = 16;
    while (nc < 1024 && per_node * (size_t)(2 * nc) <= SF_NC_BYTES) nc *= 2;
    return nc;
}

// boundary-side 3j tables of one edge (shared by every triple):
//   Aj[i][m1][m2] = (j1 j2 i; m1 m2 mu), Cj[i][m3][m4] = (i j3 j4; -mu m3 m4), mu = -(m1+m2)
__global__ void k_boundary_3j(const VtxDev* __restrict__ vp, int edge, const dd* __restrict__ F, double* Aj, double* Cj,
                              int* status) {
    const VtxDev& v = *vp;
    const int e = edge - 2;
    int tj[4];
    for (int a = 0; a < 4; a++) tj[a] = v.tj[c_edge_face[e][a]];
    const int di = v.di[e + 1], ilo = v.ilo[e + 1];
    const int n1 = tj[0] + 1, n2 = tj[1] + 1, n3 = tj[2] + 1, n4 = tj[3] + 1;
    const int stride = gridDim.x * blockDim.x;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < di * n1 * n2; q += stride) {
        int c = q / (n1 * n2), r = q % (n1 * n2), i1 = r / n2, i2 = r % n2;
        int tm1 = -tj[0] + 2 * i1, tm2 = -tj[1] + 2 * i2;
        Aj[q] = dd_to_d(sf_threej_dd(tj[0], tj[1], ilo + 2 * c, tm1, tm2, -(tm1 + tm2), F, status));
    }
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < di * n3 * n4; q += stride) {
        int c = q / (n3 * n4), r = q % (n3 * n4), i3 = r / n4, i4 = r % n4;
        int tm3 = -tj[2] + 2 * i3, tm4 = -tj[3] + 2 * i4;
        Cj[q] = dd_to_d(sf_threej_dd(ilo + 2 * c, tj[2], tj[3], -(tm3 + tm4), tm3, tm4, F, status));
    }
}

// One CTA per virtual-spin triple t of one edge.
// The m-tuples come in pairs (m, -m) whose terms are complex conjugates: d_{k l -m} =
// (-1)^(k-l) conj(d_{k l m}) and 4jm(-m) = (-1)^(sum j) 4jm(m), and 2 sum_a j_a is even. Hence
//   B[i][k] = sum_m 4jm(j;m)^(i) 4jm(l;m)^(k) Re I(m),
// and with the tuples ordered so that m -> -m reverses the flat index, only the upper half is
// summed (weight 2, the self-conjugate tuple m = 0 weight 1). The node sum is factored through
// pair products P12 = W d1 d2 and P34 = d3 d4 staged per chunk of nodes. The same reflection
// gives P12(-m1, -m2) = s12 conj(P12(m1, m2)) with s12 = (-1)^((k1 - l1) + (k2 - l2)) (likewise
// P34), so only the upper half of each pair table is staged; a tuple whose pair lies in the
// lower half reads its mirror, and Re(conj(a) b) = a.x b.x + a.y b.y flips one sign.
// Pair tables of one side (s = 0: strands 1, 2; s = 1: strands 3, 4) of an edge, for every pair of
// virtual spins (pid = il_a * nb + il_b, il the strands' offsets, 0 on a gauge face): the upper
// halves (flat pair index f >= N/2) of P12 = W d1 d2 and P34 = d3 d4 on every node, the products
// the booster kernel sums; and the virtual-side 3j symbols of that pair of spins for every k from
// |l_a - l_b| to l_a + l_b (zero where the triangle fails). Every triple of virtual spins sharing
// the pair reads them instead of forming them again.
__global__ void k_pair_tables(const VtxDev* __restrict__ vp, int edge, int side, const double* __restrict__ Wm,
                              int nnodes, int64_t total, double2* __restrict__ out) {
    const VtxDev& v = *vp;
    const int e = edge - 2;
    const int fa = c_edge_face[e][2 * side], fb = c_edge_face[e][2 * side + 1];
    const int nb = c_edge_slot[e][2 * side + 1] < 0 ? 1 : v.D;
    const int ta = v.tj[fa], tb = v.tj[fb];
    const int N = (ta + 1) * (tb + 1), h = N / 2, C = N - h;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int n = (int)(q % nnodes);
        const int64_t r = q / nnodes;
        const int f = h + (int)(r % C), pid = (int)(r / C);
        const int ila = pid / nb, ilb = pid % nb;
        const int a1 = f / (tb + 1), a2 = f % (tb + 1);
        const double2 x = v.dtab[fa][((int64_t)ila * (ta + 1) + a1) * nnodes + n];
        const double2 y = v.dtab[fb][((int64_t)ilb * (tb + 1) + a2) * nnodes + n];
        double2 z;
        if (side == 0) {
            const double w = Wm[n];
            z = make_double2(w * (x.x * y.x - x.y * y.y), w * (x.x * y.y + x.y * y.x));
        } else {
            z = make_double2(x.x * y.x - x.y * y.y, x.x * y.y + x.y * y.x);
        }
        out[q] = z;
    }
}

__global__ void k_pair_3j(const VtxDev* __restrict__ vp, int edge, int side, int nkk, int64_t total,
                          const dd* __restrict__ F, double* __restrict__ out, int* status) {
    const VtxDev& v = *vp;
    const int e = edge - 2;
    const int fa = c_edge_face[e][2 * side], fb = c_edge_face[e][2 * side + 1];
    const int nb = c_edge_slot[e][2 * side + 1] < 0 ? 1 : v.D;
    const int ta = v.tj[fa], tb = v.tj[fb];
    const int na1 = ta + 1, nb1 = tb + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int r = (int)(q % (na1 * nb1));
        const int64_t u = q / (na1 * nb1);
        const int kk = (int)(u % nkk), pid = (int)(u / nkk);
        const int tla = ta + 2 * (pid / nb), tlb = tb + 2 * (pid % nb);
        const int k = iabs_(tla - tlb) + 2 * kk;
        const int ia = r / nb1, ib = r % nb1;
        const int tma = -ta + 2 * ia, tmb = -tb + 2 * ib;
        double val = 0.0;
        if (k <= tla + tlb) {
            val = side == 0 ? dd_to_d(sf_threej_dd(tla, tlb, k, tma, tmb, -(tma + tmb), F, status))
                            : dd_to_d(sf_threej_dd(k, tla, tlb, -(tma + tmb), tma, tmb, F, status));
        }
        out[q] = val;
    }
}

int sf_pair_dims(const int tj4[4], const int slot4[4], int D, int nnodes, PairDims* pd, size_t pbytes[2], size_t tbytes[2]) {
    for (int s = 0; s < 2; s++) {
        const int ta = tj4[2 * s], tb = tj4[2 * s + 1];
        const int na = slot4[2 * s] < 0 ? 1 : D, nb = slot4[2 * s + 1] < 0 ? 1 : D;
        const int N = (ta + 1) * (tb + 1), C = N - N / 2;
        pd->nb[s] = nb;
        pd->npid[s] = na * nb;
        pd->nkk[s] = imin_(ta + 2 * (na - 1), tb + 2 * (nb - 1)) + 1;   // k = |la - lb| .. la + lb
        pbytes[s] = (size_t)pd->npid[s] * C * nnodes * sizeof(double2);
        tbytes[s] = (size_t)pd->npid[s] * pd->nkk[s] * (ta + 1) * (tb + 1) * sizeof(double);
    }
    return SF_OK;
}

int sf_pair_build(const VtxDev* d_v, int edge, const PairDims& pd, const double* d_W, int nnodes, const dd* F,
                  const int tj4[4], double2* const d_P[2], double* const d_T[2], int* d_status, int num_sms, cudaStream_t s) {
    for (int side = 0; side < 2; side++) {
        const int ta = tj4[2 * side], tb = tj4[2 * side + 1];
        const int N = (ta + 1) * (tb + 1), C = N - N / 2;
        const int64_t tp = (int64_t)pd.npid[side] * C * nnodes;
        int64_t blocks = std::min<int64_t>((tp + 255) / 256, (int64_t)num_sms * 16);
        k_pair_tables<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(d_v, edge, side, d_W, nnodes, tp, d_P[side]);
        sf_note_launch(1);
        SF_CUDA_TRY(cudaGetLastError());
        const int64_t tt = (int64_t)pd.npid[side] * pd.nkk[side] * (ta + 1) * (tb + 1);
        blocks = std::min<int64_t>((tt + 255) / 256, (int64_t)num_sms * 16);
        k_pair_3j<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(d_v, edge, side, pd.nkk[side], tt, F, d_T[side],
                                                                         d_status);
        sf_note_launch(1);
        SF_CUDA_TRY(cudaGetLastError());
    }
    return SF_OK;
}

#define SF_BT 6         // canonical tuples per thread (upper half of at most 17^3 tuples / 512 threads)
#define SF_BOOST_NT 512
__global__ void __launch_bounds__(SF_BOOST_NT) k_booster(const VtxDev* __restrict__ vp, int edge, const double* __restrict__ Wm,
                                                 int nnodes, int NC, const dd* __restrict__ F, const double* __restrict__ gAj,
                                                 const double* __restrict__ gCj, double* __restrict__ Bout,
                                                 const unsigned char* __restrict__ need, const double2* __restrict__ gP12,
                                                 const double2* __restrict__ gP34, const double* __restrict__ g3A,
                                                 const double* __restrict__ g3C, PairDims pd, int* status) {
    extern __shared__ __align__(16) double sm[];
    const VtxDev& v = *vp;
    const int e = edge - 2;
    const int D = v.D;
    const int t = blockIdx.x;
    const int toff[3] = {t / (D * D), (t / D) % D, t % D};
    int tj[4], tl[4], il[4], fc[4];
    for (int a = 0; a < 4; a++) {
        fc[a] = c_edge_face[e][a];
        tj[a] = v.tj[fc[a]];
        int sl = c_edge_slot[e][a];
        il[a] = sl < 0 ? 0 : toff[sl];
        tl[a] = tj[a] + 2 * il[a];
    }
    const int di = v.di[e + 1], ilo = v.ilo[e + 1];
    const int dkmax = v.dkmax[e];
    double* Bt = Bout + (int64_t)t * di * dkmax;
    int klo, nk;
    sf_pair_range(tl[0], tl[1], tl[2], tl[3], &klo, &nk);
    for (int q = threadIdx.x; q < di * dkmax; q += blockDim.x) Bt[q] = 0.0;
    if (nk == 0 || (need && !need[t])) return;   // an empty range, or a triple no selected shell uses
    const int n1 = tj[0] + 1, n2 = tj[1] + 1, n3 = tj[2] + 1, n4 = tj[3] + 1;
    const int M = n1 * n2 * n3;
    const int Mh = M / 2;   // canonical tuples: [Mh, M); Mh itself is m = 0 when M is odd
    // pair tables: flat pair index f = ia * nb + ib; -m maps f to N - 1 - f; staged f >= N / 2
    const int N12 = n1 * n2, N34 = n3 * n4, h12 = N12 / 2, h34 = N34 / 2;
    const int C12 = N12 - h12, C34 = N34 - h34;
    const double sg12 = ((((tl[0] - tj[0]) + (tl[1] - tj[1])) / 2) & 1) ? -1.0 : 1.0;
    const double sg34 = ((((tl[2] - tj[2]) + (tl[3] - tj[3])) / 2) & 1) ? -1.0 : 1.0;
    // shared: Ir[M] | union { P12[C12][NC], P34[C34][NC] (complex) ; Al[nk][n1 n2], Cl[nk][n3 n4] }
    double* sIr = sm;
    const int Mpad = (M + 1) & ~1;   // keep the complex staging area 16-byte aligned
    double2* P12 = reinterpret_cast<double2*>(sm + Mpad);
    double2* P34 = P12 + C12 * NC;
    double* sAl = sm + Mpad;
    double* sCl = sAl + nk * n1 * n2;
    // this triple's pair tables (upper halves, [pair][node]) and virtual-side 3j tables
    const int pid12 = il[0] * pd.nb[0] + il[1], pid34 = il[2] * pd.nb[1] + il[3];
    const double2* q12 = gP12 + (int64_t)pid12 * C12 * nnodes;
    const double2* q34 = gP34 + (int64_t)pid34 * C34 * nnodes;
    double acc[SF_BT];
#pragma unroll
    for (int q = 0; q < SF_BT; q++) acc[q] = 0.0;
    for (int n0 = 0; n0 < nnodes; n0 += NC) {
        const int nc = imin_(NC, nnodes - n0);
        __syncthreads();
        for (int q = threadIdx.x; q < C12 * NC; q += blockDim.x) {
            const int nn = q % NC, f = q / NC;
            P12[q] = (nn < nc) ? q12[(int64_t)f * nnodes + n0 + nn] : make_double2(0.0, 0.0);
        }
        for (int q = threadIdx.x; q < C34 * NC; q += blockDim.x) {
            const int nn = q % NC, f = q / NC;
            P34[q] = (nn < nc) ? q34[(int64_t)f * nnodes + n0 + nn] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < SF_BT; q++) {
            const int mt = Mh + threadIdx.x + q * blockDim.x;
            if (mt < M) {
                const int i3 = mt % n3, i2 = (mt / n3) % n2, i1 = mt / (n3 * n2);
                const int tm4 = -((-tj[0] + 2 * i1) + (-tj[1] + 2 * i2) + (-tj[2] + 2 * i3));
                if (iabs_(tm4) <= tj[3]) {
                    const int i4 = (tm4 + tj[3]) / 2;
                    const int f12 = i1 * n2 + i2, f34 = i3 * n4 + i4;
                    const bool c12 = f12 < h12, c34 = f34 < h34;   // mirrored (conjugated) pairs
                    const double2* p = P12 + ((c12 ? N12 - 1 - f12 : f12) - h12) * NC;
                    const double2* r = P34 + ((c34 ? N34 - 1 - f34 : f34) - h34) * NC;
                    double s0 = 0.0, s1 = 0.0;
                    for (int nn = 0; nn < nc; nn++) {
                        const double2 a = p[nn], b = r[nn];
                        s0 = fma(a.x, b.x, s0);
                        s1 = fma(a.y, b.y, s1);
                    }
                    // Re of the product: s0 - s1, or s0 + s1 with exactly one factor conjugated
                    const double re = (c12 != c34) ? s0 + s1 : s0 - s1;
                    const double sg = (c12 ? sg12 : 1.0) * (c34 ? sg34 : 1.0);
                    acc[q] = fma(sg, re, acc[q]);
                }
            }
        }
    }
    __syncthreads();   // the staging area is reused for the 3j tables below
    for (int q = threadIdx.x; q < Mh; q += blockDim.x) sIr[q] = 0.0;
#pragma unroll
    for (int q = 0; q < SF_BT; q++) {
        const int mt = Mh + threadIdx.x + q * blockDim.x;
        if (mt < M) sIr[mt] = ((M & 1) && mt == Mh) ? acc[q] : 2.0 * acc[q];
    }
    // ---- virtual-side 3j tables: Al[c][m1][m2] = (l1 l2 k; m1 m2 mu), Cl[c][m3][m4] = (k l3 l4; -mu m3 m4),
    // copied from the per-pair tables (k from |l1 - l2| and from |l3 - l4| in steps of one)
    {
        const int kk12 = (klo - iabs_(tl[0] - tl[1])) / 2, kk34 = (klo - iabs_(tl[2] - tl[3])) / 2;
        const double* a3 = g3A + ((int64_t)pid12 * pd.nkk[0] + kk12) * n1 * n2;
        const double* c3 = g3C + ((int64_t)pid34 * pd.nkk[1] + kk34) * n3 * n4;
        for (int q = threadIdx.x; q < nk * n1 * n2; q += blockDim.x) sAl[q] = a3[q];
        for (int q = threadIdx.x; q < nk * n3 * n4; q += blockDim.x) sCl[q] = c3[q];
    }
    __syncthreads();
    // ---- B[i][k] = sum_m (-1)^((i - mu) + (k - mu)) Aj Cj Al Cl Re I(m)
    for (int q = threadIdx.x; q < di * nk; q += blockDim.x) {
        const int ci = q / nk, ck = q % nk;
        const int ti = ilo + 2 * ci, tk = klo + 2 * ck;
        double br = 0.0;
        for (int i1 = 0; i1 < n1; i1++) {
            const int tm1 = -tj[0] + 2 * i1;
            for (int i2 = 0; i2 < n2; i2++) {
                const int tm2 = -tj[1] + 2 * i2;
                const int tmu = -(tm1 + tm2);
                const double aa = gAj[(ci * n1 + i1) * n2 + i2] * sAl[(ck * n1 + i1) * n2 + i2];
                if (aa == 0.0) continue;
                const int par = ((ti - tmu) / 2 + (tk - tmu) / 2) & 1;
                double sr = 0.0;
                for (int i3 = 0; i3 < n3; i3++) {
                    const int tm3 = -tj[2] + 2 * i3;
                    const int tm4 = tmu - tm3;
                    if (iabs_(tm4) > tj[3]) continue;
                    const int i4 = (tm4 + tj[3]) / 2;
                    const double cc = gCj[(ci * n3 + i3) * n4 + i4] * sCl[(ck * n3 + i3) * n4 + i4];
                    sr = fma(cc, sIr[(i1 * n2 + i2) * n3 + i3], sr);
                }
                br = par ? br - aa * sr : br + aa * sr;
            }
        }
        Bt[ci * dkmax + ck] = br;
    }
}

// Boosters of the triples that sf_boosters fills by exchange. When the two strands of a coupled
// pair carry equal spins, their d-functions coincide, and exchanging the strands multiplies the
// booster by the 3j exchange phase in both 4jm symbols, (-1)^((j_a + j_b + i) + (l_a + l_b + k))
// (eq. booster with the (a1 a2)(a3 a4) coupling): so the booster of a triple whose offsets on the
// pair decrease is the exchanged triple's, times that sign. One CTA per triple; fill[t] != 0
// selects the triples; the exchanged triples were computed by k_booster.
__global__ void k_booster_mirror(const VtxDev* __restrict__ vp, int edge, int pos, const unsigned char* __restrict__ fill,
                                 double* __restrict__ Bout) {
    const VtxDev& v = *vp;
    const int e = edge - 2, D = v.D, t = blockIdx.x;
    if (!fill[t]) return;
    int off[3] = {t / (D * D), (t / D) % D, t % D};
    int tj[4], tl[4];
    for (int a = 0; a < 4; a++) {
        tj[a] = v.tj[c_edge_face[e][a]];
        const int sl = c_edge_slot[e][a];
        tl[a] = tj[a] + 2 * (sl < 0 ? 0 : off[sl]);
    }
    const int sa = c_edge_slot[e][pos], sb = c_edge_slot[e][pos + 1];
    const int tmp = off[sa];
    off[sa] = off[sb];
    off[sb] = tmp;
    const int t2 = (off[0] * D + off[1]) * D + off[2];
    int klo, nk;
    sf_pair_range(tl[0], tl[1], tl[2], tl[3], &klo, &nk);
    const int di = v.di[e + 1], ilo = v.ilo[e + 1], dkmax = v.dkmax[e];
    const double* src = Bout + (int64_t)t2 * di * dkmax;
    double* dst = Bout + (int64_t)t * di * dkmax;
    const int base = tj[pos] + tj[pos + 1] + tl[pos] + tl[pos + 1] + ilo + klo;
    for (int q = threadIdx.x; q < di * nk; q += blockDim.x) {
        const int ci = q / nk, ck = q - ci * nk;
        const int ex = (base + 2 * ci + 2 * ck) / 2;   // (j_a + j_b + i + l_a + l_b + k) in whole units
        const double b = src[ci * dkmax + ck];
        dst[ci * dkmax + ck] = (ex & 1) ? -b : b;
    }
}

int sf_booster_mirror(const VtxDev* d_v, int edge, int pos, int ntrip, const unsigned char* d_fill, double* d_B,
                      cudaStream_t s) {
    if (ntrip <= 0) return SF_OK;
    k_booster_mirror<<<ntrip, 128, 0, s>>>(d_v, edge, pos, d_fill, d_B);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

size_t sf_booster_smem(int tj1, int tj2, int tj3, int tj4, int nk) {
    int n1 = tj1 + 1, n2 = tj2 + 1, n3 = tj3 + 1, n4 = tj4 + 1;
    size_t M = ((size_t)n1 * n2 * n3 + 1) & ~(size_t)1;
    const int c12 = n1 * n2 - (n1 * n2) / 2, c34 = n3 * n4 - (n3 * n4) / 2;
    size_t stage = (size_t)(c12 + c34) * sf_booster_chunk(tj1, tj2, tj3, tj4) * sizeof(double2);
    size_t tabs = sizeof(double) * ((size_t)nk * n1 * n2 + (size_t)nk * n3 * n4);
    return M * sizeof(double) + (stage > tabs ? stage : tabs);
}

int sf_booster_build(const VtxDev* d_v, int edge, int ntrip, size_t smem, int nc, const double* d_W, int nnodes,
                     const dd* F, double* d_Aj, double* d_Cj, double* d_B, const unsigned char* d_need,
                     const double2* const d_P[2], const double* const d_T[2], const PairDims& pd, int* d_status,
                     cudaStream_t s) {
    if (smem > 227 * 1024) return sf_set_error(SF_ERR_LIMIT, "booster kernel needs %zu bytes of shared memory", smem);
    k_boundary_3j<<<64, 256, 0, s>>>(d_v, edge, F, d_Aj, d_Cj, d_status);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    SF_CUDA_TRY(cudaFuncSetAttribute(k_booster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_booster<<<ntrip, SF_BOOST_NT, smem, s>>>(d_v, edge, d_W, nnodes, nc, F, d_Aj, d_Cj, d_B, d_need, d_P[0], d_P[1],
                                               d_T[0], d_T[1], pd, d_status);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}
