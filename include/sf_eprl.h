/*
 * sf_eprl.h -- C ABI of the GB300 library for the Lorentzian EPRL vertex amplitude shell sum
 * (F. Gozzini, "A high-performance code for EPRL spin foam amplitudes", arXiv:2107.13952).
 *
 * The library computes, on one GPU,
 *
 *   A_v(j_f; i_e) = prod_{e=1..5} sqrt(2 i_e + 1)
 *                   * sum_{shells l} sum_{k_2..k_5} prod_{e=2..5} (2k_e+1) B4_e(i_e, k_e) {15j}(j, l; i_1, k_2..k_5)
 *
 * (Sec. 2, eq. vertex-ampl), with the {15j} as the auxiliary-spin sum of five {6j} (Sec. 2, eq. 15j)
 * and the boosters B4 by rapidity quadrature of SL(2,C) boost matrix elements (Sec. 2, eq. booster;
 * Sec. 3 "Booster coefficients"), following the framed vertex algorithm of Sec. 3 "Tensor contractions".
 *
 * Conventions (used by every entry point):
 *   - Spins are DOUBLED integers: two_j = 2*j, so half-integers are exact.
 *   - Boundary order:  two_j[0..9] = (j12, j13, j14, j15, j23, j24, j25, j34, j35, j45)   (Sec. 2).
 *   - Free faces (23, 24, 25, 34, 35, 45) carry l_f = j_f + d_f, d_f = 0..dl; gauge faces l_1b = j_1b.
 *   - Linear shell index  s = ((((d25*D + d35)*D + d45)*D + d24)*D + d34)*D + d23,  D = dl+1,
 *     s in [0, D^6)  (the paper's (Delta s + 1)^6 loops, Sec. 3 "Parallelization"). The order is a
 *     convention of this library: (l25, l35, l45) lead, so a contiguous range is a run of whole
 *     groups that share the edge-5 booster.
 *   - Intertwiner ranges: edge 1 couples (j12 j13 | j14 j15), edge 2 (j23 j24 | j25 j12),
 *     edge 3 (j34 j35 | j13 j23), edge 4 (j45 j14 | j24 j34), edge 5 (j15 j25 | j35 j45)
 *     (the booster index orders of the framed algorithm, step 3).
 *   - Output tensor A[i1][i2][i3][i4][i5], i5 fastest: byte-identical to the paper's column-major
 *     A^{i5 i4 i3 i2 i1} (Sec. 3, footnote on the result layout). Index n_e = (i_e - i_e,lo).
 *   - Booster tensor of edge e: B[t][i - i_lo][k - k_lo(t)], t = (a*D + b)*D + c the mixed-radix
 *     index of the edge's three free-face offsets in argument order: edge 2 (d23, d24, d25),
 *     edge 3 (d34, d35, d23), edge 4 (d45, d24, d34), edge 5 (d25, d35, d45); padded with zeros to
 *     D_kmax columns (the paper's booster tensors B^{l1 l2 l3 l4 i k}, Sec. 3).
 *
 * Memory and streams:
 *   - sf_tables is opaque and owns its device memory (6j tables, d-tables, boosters, scratch); it is
 *     released by sf_tables_free. Every other pointer belongs to the caller; the library never frees it.
 *   - Pointers documented "device" must be device (or managed) memory on the current device.
 *   - Every compute call is enqueued on `stream` and synchronises that stream before returning, so a
 *     returned status covers the device work. Calls on one sf_tables object must not overlap.
 *
 * Errors: every int-returning call returns SF_OK (0) or a negative code; sf_last_error() gives a
 * thread-local message for the last failure on the calling thread.
 */
#ifndef SF_EPRL_H
#define SF_EPRL_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SF_OK           0
#define SF_ERR_ARG     -1   /* bad argument: triangle/parity failure, gamma <= 0, dl < 0, sizes   */
#define SF_ERR_EMPTY   -2   /* an intertwiner range of the boundary is empty                      */
#define SF_ERR_OOM     -3   /* device allocation failed                                           */
#define SF_ERR_CUDA    -4   /* a CUDA runtime call or kernel launch failed                        */
#define SF_ERR_TIMEOUT -5   /* a bounded device wait gave up                                      */
#define SF_ERR_NUMERIC -6   /* a numerical self-check failed (e.g. non-real booster)              */
#define SF_ERR_LIMIT   -7   /* spins or dimensions beyond the compiled limits                     */

/* One vertex boundary (Sec. 3, framed algorithm step 1: ten spins and the number of shells),
 * with an optional reduced set of boundary intertwiners (the paper computes the vertex tensor for a
 * reduced set of intertwiner indices when asked, Sec. 3 after the framed algorithm, and its
 * interface offers a restricted intertwiner range, Sec. 4 "vertex_compute").
 *   sub_first[e], sub_count[e]: the output covers intertwiners i_e = lo_e + 2 (sub_first[e] + n),
 *     n = 0 .. sub_count[e] - 1, of edge e's range (lo_e, dim_e); sub_count[e] = 0 selects
 *     everything from sub_first[e] to the end, so a zero-initialised struct means the whole
 *     tensor. The output tensor of every amplitude call then has shape sub_count[0..4] (same
 *     layout, i5 fastest) and equals the corresponding block of the whole tensor. Boosters keep
 *     the whole intertwiner range. sub_first[e] < 0, beyond the range, or a count running past its
 *     end is SF_ERR_ARG. The adjoint (sf_vertex_adjoint) needs the whole range. */
typedef struct {
    int32_t two_j[10];     /* doubled boundary spins, order above                                */
    double  gamma;         /* Barbero-Immirzi parameter; Y-map (rho, k) = (gamma (j+1), j)         */
    int32_t dl;            /* shell cutoff Delta s: l_f in [j_f, j_f + dl]                        */
    int32_t sub_first[5];  /* first intertwiner index of the output per edge (0 = the range's lo) */
    int32_t sub_count[5];  /* intertwiners per edge in the output (0 = through the range's end)   */
} sf_vertex;

/* Rapidity rule (Sec. 3 "Booster coefficients"): x = e^-r on [e^-r_max, 1] split into n_panels
 * panels with |I_k| = k |I_1| (smallest at x -> 0), `order` Gauss-Legendre nodes per panel. */
typedef struct {
    double  r_max;
    int32_t n_panels;
    int32_t order;
} sf_quad_rule;

typedef enum {
    SF_FP64  = 0,   /* every step in FP64                                                         */
    SF_MIXED = 1,   /* booster contractions over k2, k3, k4 with FP32 inputs and FP32 accumulation
                       within one (l24, l34) set of shells; the {6j} contractions, the k5 contraction
                       and every sum across shells in FP64                                        */
    SF_MIXED_FF = 2, /* booster contractions as SF_MIXED; the {6j} contractions (the S3 contraction
                       over k3 and the x-sum with S1 S2) in compensated FP32 pairs: operands are
                       (hi, lo) float pairs holding about 48 significant bits, products are formed
                       exactly (Dekker) and summed with an error-compensated dot product (Ogita,
                       Rump and Oishi, "Accurate sum and dot product", 2005, Dot2), so these sums
                       keep nearly FP64 accuracy on the FP32 pipe; the sums across the (l24, l34)
                       sets of one (l25, l35, l45) group also in pairs; the k5 contraction and the
                       sums across groups in FP64                                                 */
    SF_MIXED_TC = 3, /* the booster contractions over the virtual intertwiners in FP32-class
                       arithmetic, the {15j} auxiliary-spin sum and the sums across shells in FP64:
                       the k4 contraction with the edge-4 booster on the tensor cores (mma.sync
                       m16n8k16, operands split into three BF16 pieces holding 24 significant
                       bits, the six piece products of order <= 2 accumulated in FP32: split-BF16
                       with FP32 accumulation); the k2 contraction (with S4, S5 and B2), the l23
                       sum with B3 and the k3 contraction with S3 in FP32 on the CUDA cores; the
                       x-sum (2x+1) S1 S2 of eq. 15j, the k5 contraction, and the sums across the
                       (l24, l34) sets and groups in FP64                                         */
    SF_MIXED_PX = 4 /* the booster contractions over k2, k3, k4 (with S4, S5, B2, B3, B4) and the
                       S3 contraction in FP32 on the CUDA cores; the x-sum (2x+1) S1 S2 of eq. 15j
                       in compensated FP32 pairs as in SF_MIXED_FF: the products (2x+1) S1 S2
                       formed as pairs from the (hi, lo) copies of S1 and S2, multiplied by the FP32
                       result of the S3 contraction and summed over x (and across the x chunks of
                       one (l24, l34) set) with Dot2; the k5 contraction and the sums across the
                       (l24, l34) sets and groups in FP64. Faster than SF_MIXED_TC, but beyond the
                       target precision split: the {15j} auxiliary-spin sum is not in FP64       */
} sf_precision;

typedef struct sf_tables sf_tables;

/* Library version string (static). */
const char* sf_version(void);

/* Thread-local message of the last failure on this thread ("" if none). Static storage. */
const char* sf_last_error(void);

/* Host helper (no device work): doubled lower bounds and dimensions of i_1..i_5
 * (framed algorithm step 2), of the whole ranges: the sub-range fields of v are ignored.
 * Returns SF_ERR_EMPTY if a range is empty, SF_ERR_ARG on bad input. */
int sf_intertwiner_ranges(const sf_vertex* v, int32_t two_lo[5], int32_t dim[5]);

/* Host helper: the output ranges of v (its sub-range applied): doubled lower bounds and counts,
 * i.e. the shape of the tensors the amplitude calls write. SF_ERR_ARG for a bad sub-range. */
int sf_output_ranges(const sf_vertex* v, int32_t two_lo[5], int32_t dim[5]);

/* Host helper: number of shells (dl+1)^6 of a vertex, or a negative error code. */
int64_t sf_num_shells(const sf_vertex* v);

/* Build the five {6j} tables S1..S5 of Sec. 3 framed algorithm step 4 for n vertices, exactly
 * (integer Racah sum, rounded once to FP64), and allocate the tables object.
 *   S1[l25][i1, k5, x] = {i1 l25 x; k5 j14 j15}      S2[l35, l45][k5, k4, x] = {j14 k5 x; l35 k4 l45}
 *   S3[l24, l34, l35][k4, k3, x] = {k4 l35 x; k3 l24 l34}
 *   S4[l23, l24][k3, k2, x] = {l24 k3 x; j13 k2 l23}  S5[l25][k2, i1, x] = {k2 j13 x; i1 l25 j12}
 * v: host array of n vertices. *out receives a new object (free with sf_tables_free). */
int sf_6j_table(const sf_vertex* v, int32_t n, sf_tables** out, cudaStream_t stream);

/* The same tables object restricted to what the shells [shell_begin, shell_end) of every vertex
 * read (the range as in sf_vertex_amplitude, widened to whole (l25, l35, l45) groups): the {6j}
 * slots and, in sf_boosters, the booster triples of the other groups are left zero (S1, S5 and the
 * edge-2 boosters are selected by l25, S2 by (l35, l45), S3 and the edge-3 boosters by l35, the
 * edge-4 boosters by l45, the edge-5 boosters by the group; S4 is built whole). For a shell sum over
 * part of the range, as one process of a split sum (Sec. 3 "Parallelization": each node computes
 * its own shells) or one slice of a long sum, building only what it reads. Amplitude calls and
 * plans on these tables must stay inside the groups (else SF_ERR_ARG); sf_vertex_adjoint needs the
 * whole range. Errors: as sf_6j_table, SF_ERR_ARG for a negative or reversed range. */
int sf_6j_table_range(const sf_vertex* v, int32_t n, int64_t shell_begin, int64_t shell_end, sf_tables** out,
                      cudaStream_t stream);

/* Compute the booster tensors of every vertex in t (Sec. 2 eq. booster, Sec. 3): d-tables
 * d^{gamma(j+1), j}_{j l m}(r_n) on the rule's nodes, 4jm symbols, quadrature and m-sum.
 * q: host pointer to the rule. Per edge, the node products of each pair of strands and the
 * virtual-side 3j symbols of each pair of virtual spins are tabulated first, in stream-ordered
 * scratch from a memory pool of the library's own on the current device (kept for reuse by later
 * calls: at dl 10 and spin 8 about 1.2 GB). When the two free strands of an edge's coupled pair
 * carry equal spins, the triples with decreasing offsets on that pair are filled from the
 * exchanged triple times the 3j exchange phase (-1)^(j_a + j_b + i + l_a + l_b + k) instead of
 * being integrated again. Synchronises the stream (status check). */
int sf_boosters(sf_tables* t, const sf_quad_rule* q, cudaStream_t stream);

/* Shape of the booster tensor of (vertex, edge in 2..5): shape = {n_triples, D_i, D_kmax}. */
int sf_booster_shape(const sf_tables* t, int32_t vertex, int32_t edge, int64_t shape[3]);

/* Replace (upload) or read back (download) the booster tensor of (vertex, edge), layout above.
 * B: host or device pointer to shape[0]*shape[1]*shape[2] doubles; padded entries are ignored
 * on upload and written as zero on download. Upload lets a caller inject boosters computed
 * elsewhere (e.g. the SU(2) BF limit (2k+1)B = delta_ik). */
int sf_boosters_upload(sf_tables* t, int32_t vertex, int32_t edge, const double* B, cudaStream_t stream);
int sf_boosters_download(const sf_tables* t, int32_t vertex, int32_t edge, double* B, cudaStream_t stream);

/* Vertex amplitude tensors by the shell sum (framed algorithm steps 5-7).
 *   precision  any sf_precision value (SF_FP64, SF_MIXED, SF_MIXED_FF, SF_MIXED_TC, SF_MIXED_PX).
 *   shell_begin, shell_end: linear shell range [begin, end) of every vertex (clamped to its shell
 *     count; pass 0 and INT64_MAX for all shells). Partial sums over disjoint ranges add up, so a
 *     long sum can be split or resumed.
 *   shell_list, n_list: optional host or device array of linear shell indices (single-vertex tables only);
 *     when non-NULL it replaces the range. Duplicates count once.
 *   A_out: host array of n device pointers, A_out[v] -> prod_e dim_e doubles, overwritten (dim_e
 *     of the vertex's output ranges, sf_output_ranges).
 *   kappa_out: optional (NULL to skip) host or device array of n doubles: kappa_out[v] =
 *     sum over the selected non-empty shells s of ||C_s||_2, C_s the contribution of shell s to the
 *     vertex's output tensor, prod sqrt(2i+1) included, in FP64 whatever the precision. Divided by
 *     ||A_v||_2 it is the cancellation factor kappa of the shell sum, the scale of the mixed paths'
 *     rounding errors (error ~ kappa times the FP32 unit roundoff). It costs one extra pass with
 *     the shell sum unhoisted across shells (about a full framed-algorithm evaluation per shell,
 *     several times the amplitude itself), so ask for it on shell lists or small ranges.
 * Uses library-owned scratch for per-block partial sums, reduced in a fixed order (deterministic).
 * A batch whose vertices need different CTA shapes runs as two launches, the second on a stream
 * the tables own, ordered after the caller's stream's earlier work and joined back into it before
 * the reduction. Synchronises the caller's stream (status check). */
int sf_vertex_amplitude(sf_tables* t, sf_precision precision, int64_t shell_begin, int64_t shell_end,
                        const int64_t* shell_list, int64_t n_list, double* const* A_out, double* kappa_out,
                        cudaStream_t stream);

/* The FP64 shell sum of sf_vertex_amplitude (same tables, same range semantics, same output layout
 * and values) without any device allocation, for callers that must not allocate device memory
 * while they run: programs that share the GPU with a framework owning a fixed memory pool, hosts
 * that forbid allocation after start-up (cudaMalloc/cudaFree may synchronise the whole device),
 * or callers keeping a strict memory budget. The paper has no counterpart; it is a property of
 * this library. Build the tables (sf_6j_table, sf_boosters) during start-up, then call this.
 *   Scratch: one file-scope device array of 32 MiB, present on every GPU that loads the library
 *   until the process exits. The call needs 256-byte-aligned space for one work item and one
 *   partial tile (prod of dim_3..dim_5 doubles) per (vertex, i1, i2) tile; larger requests return
 *   SF_ERR_LIMIT with the size needed (split the shell range or the vertex set).
 *   The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *   that device current and caches it. Every call copies its work list from host memory and
 *   synchronises the stream before returning, so it must not be issued while the stream is being
 *   captured into a CUDA graph; replayable shell sums go through the sf_plan_* calls.
 *   Every call reuses the same array and leaves its contents behind; calls that overlap on the
 *   GPU (other streams, other host threads, same device) race on it and must be serialised by
 *   the caller. A_out: host array of device pointers, as in sf_vertex_amplitude. */
int sf_vertex_amplitude_noalloc(sf_tables* t, int64_t shell_begin, int64_t shell_end, double* const* A_out,
                                cudaStream_t stream);

/* Planned shell sums: many vertex tensors in one persistent launch, replayable as a CUDA graph.
 * The paper distributes the shell loops of one vertex over nodes and cores (Sec. 3,
 * "Parallelization") and names routines for many vertex tensors with few shells each as future
 * work (Sec. 6); a plan serves both. It fixes what the host decides for one sf_vertex_amplitude
 * call over a shell range (the tables, outputs, precision, range, work items and the kernel's
 * tiling) and owns its device scratch, so that running it issues only asynchronous device work:
 * one memset, the persistent shell kernel and one reduction kernel over every vertex's tiles.
 *
 * sf_tiling (0 in a field selects the library's choice):
 *   x_chunk = auxiliary spins x per staged chunk of the {6j} contractions (1..16; the shared-memory
 *     footprint grows with it; default the largest that fits);
 *   items_per_sm = target number of work items per SM (granularity of the cost-balanced split of
 *     tiles x groups; default 16 with 512 or 1024 threads, 8 with 256);
 *   threads = CTA size, 512 (one CTA per SM) or 256 (two CTAs per SM whose phases interleave), and
 *     with SF_MIXED_PX also 1024 (one CTA per SM, twice the warps of 512);
 *   i3_split = 1 or 2 pieces of i3 per output tile (2 halves the per-CTA buffers and register
 *     tile, so that two CTAs of 256 threads fit per SM or one CTA of 512 threads gets larger x
 *     chunks, and stages the i3-independent operands twice). Default: 256 threads on whole tiles
 *     when they fit with an x chunk of at least 4, else 1024 (SF_MIXED_PX) or 512 threads on
 *     whole tiles; half tiles only on request. */
typedef struct sf_tiling {
    int32_t x_chunk;
    int32_t items_per_sm;
    int32_t threads;
    int32_t i3_split;
} sf_tiling;
typedef struct sf_plan sf_plan;

/* Create a plan for the range [shell_begin, shell_end) of every vertex of t (as in
 * sf_vertex_amplitude). tiling: host pointer or NULL (defaults). A_out: host array of device
 * output pointers, fixed for the plan's lifetime. Allocates the plan's scratch and copies its
 * schedule to the device synchronously. t must outlive the plan; tables and boosters are read at
 * run time, so re-uploaded boosters of the same shapes are picked up by later runs.
 * Errors: SF_ERR_ARG (null pointers, boosters missing, bad tiling), SF_ERR_LIMIT (dimensions or
 * x_chunk do not fit the kernel), SF_ERR_OOM. */
int sf_plan_create(sf_tables* t, sf_precision precision, int64_t shell_begin, int64_t shell_end,
                   const sf_tiling* tiling, double* const* A_out, sf_plan** out);

/* Time candidate tilings ((threads, i3_split) in (1024, 1) (SF_MIXED_PX only), (512, 1), (256, 1),
 * (256, 2), (512, 2) x x_chunk 16, 8, 4 (clamped to what fits) x items_per_sm 4, 8, 16) on the
 * first sample_shells shells of the plan's range of every vertex (best of two runs after a
 * warm-up, CUDA events on stream) and rebuild the plan with the fastest; *chosen (optional)
 * receives it. Overwrites the plan's outputs; synchronises the stream; drops a captured graph. */
int sf_plan_autotune(sf_plan* plan, int64_t sample_shells, sf_tiling* chosen, cudaStream_t stream);

/* Run the plan on stream: stream work only (no allocation, no host copy, no synchronisation), so
 * the call itself may be captured into a CUDA graph by the caller. Results: the outputs given at
 * creation, overwritten, equal to sf_vertex_amplitude's over the same range (fixed-order
 * reductions; bitwise reproducible for a fixed tiling). Launch errors are returned; errors
 * during execution surface at the next synchronisation (sf_plan_sync). */
int sf_plan_run(sf_plan* plan, cudaStream_t stream);

/* The same run as one CUDA graph: the first call captures sf_plan_run on a private stream and
 * instantiates it; every call launches the graph on stream. */
int sf_plan_graph_launch(sf_plan* plan, cudaStream_t stream);

/* Wait for stream and report any CUDA error of the plan's runs. */
int sf_plan_sync(sf_plan* plan, cudaStream_t stream);

/* The plan's effective tiling, work-item count, persistent grid size and scratch bytes (each
 * output optional). */
int sf_plan_info(const sf_plan* plan, sf_tiling* tiling, int64_t* n_items, int32_t* grid, int64_t* scratch_bytes);

void sf_plan_free(sf_plan* plan);

/* Boundary-contracted amplitude and its adjoint (single-vertex tables):
 *   a = sum_i A[i1..i5] psi_1[i1] psi_2[i2] psi_3[i3] psi_4[i4] psi_5[i5]
 * (the paper's contraction of a vertex tensor with boundary intertwiner vectors, Sec. 3 usage),
 * recomputing every shell's {15j} ring on the fly (never stored).
 *   psi[e]: device pointer to dim_e complex doubles (interleaved re, im).
 *   a_out: device pointer to one complex double.
 *   grad_psi[e] (optional, NULL to skip): device, dim_e complex doubles: the holomorphic
 *     derivative d a / d psi_e.
 *   grad_B[e-2] (optional): device, shape of the edge-e booster tensor, complex doubles:
 *     d a / d B_e[t][i][k] (zero on padded entries).
 * precision: SF_FP64 (the only value accepted: every step of the contraction and of its adjoint
 *   runs in FP64; other values return SF_ERR_ARG). The tables must cover the whole intertwiner
 *   range (no sub-range). With both grad_psi and grad_B NULL only a is computed. */
int sf_vertex_adjoint(sf_tables* t, sf_precision precision, const double* const psi[5], double* a_out,
                      double* const grad_psi[5], double* const grad_B[4], cudaStream_t stream);

/* ---------------------------------------------------------------------------------------------
 * Vertex-tensor contractions (Sec. 3 "Tensor contractions", eq. vertex-contraction: vertex tensors
 * are contracted with each other and with boundary states over their intertwiner indices; the
 * paper times the complete contraction of two vertices and of one vertex with five boundary
 * states on the GPU, Sec. 4 "Tensor contractions on CPU and GPU", fig. contractions).
 * Tensors use the layout of the amplitude calls: A[i1][i2][i3][i4][i5], i5 fastest, FP64.
 * ------------------------------------------------------------------------------------------- */

/* Partial or complete contraction with boundary vectors over the trailing n_vec indices:
 *   n_vec = 3: out[i1][i2] = sum_{i3 i4 i5} A psi_3[i3] psi_4[i4] psi_5[i5]   (D1 x D2 values)
 *   n_vec = 4: out[i1]     = sum_{i2..i5} A psi_2 ... psi_5                    (D1 values)
 *   n_vec = 5: out[0]      = sum_{i1..i5} A psi_1 ... psi_5                    (1 value)
 * A: device, prod dim doubles. psi[e]: device, dim[e] complex doubles (interleaved re, im), read
 * for e >= 5 - n_vec (others may be NULL). out: device complex doubles. dim: host, each 1..1024.
 * FP64; every sum in a fixed order. Stream-ordered: the call enqueues its kernels (and a small
 * stream-ordered scratch allocation) on `stream` and returns; errors during execution surface at
 * the caller's next synchronisation. Errors: SF_ERR_ARG, SF_ERR_LIMIT (D3 D4 above 12,800),
 * SF_ERR_CUDA, SF_ERR_OOM. */
int sf_contract_vectors(const double* A, const int32_t dim[5], int32_t n_vec, const double* const psi[5],
                        double* out, cudaStream_t stream);

/* Complete contraction of two vertex tensors of n entries: *out = sum_i A[i] B[i] (FP64, fixed
 * order). A, B: device, 16-byte aligned; out: device, one double. Stream-ordered, as
 * sf_contract_vectors. */
int sf_contract_vertices(const double* A, const double* B, int64_t n, double* out, cudaStream_t stream);

/* The Delta_3 spin foam (three vertices joined pairwise by internal edges and sharing one
 * internal face, Sec. 5 "The Delta_3 graph"): for each internal spin x the three vertices have
 * equal tensors A_x (boundary spins (x, J, ..., J), so i1 and i2 run over the same internal range
 * k = k_lo .. ) and each is contracted with three boundary vectors on (i3, i4, i5):
 *   T_v[k][k'] = sum A_x[k][k'][i3][i4][i5] psi[3v][i3] psi[3v+1][i4] psi[3v+2][i5],  v = 0, 1, 2;
 *   amps[x]  = (-1)^x (2x+1) sum_{k1 k2 k3} (-1)^(k1+k2+k3) T_0[k1][k2] T_2[k2][k3] T_1[k3][k1];
 *   total    = sum_x amps[x]  (the amplitude of the graph, summed over the internal face's spin).
 *   n_x: number of internal spins; A: host array of n_x device tensors; dims: host [n_x][5]
 *   (dims[i][0] == dims[i][1]; dims[i][2..4] the same for every x); two_x, two_klo: host [n_x],
 *   doubled x and lowest internal intertwiner (both integer spins); psi: host array of 9 device
 *   vectors (complex doubles, lengths dims[.][2], dims[.][3], dims[.][4] in turn);
 *   amps: device, n_x complex doubles; total: device, one complex double.
 * FP64, fixed-order sums. Synchronises the stream. Errors: SF_ERR_ARG, SF_ERR_LIMIT, SF_ERR_CUDA. */
int sf_delta3_amplitudes(int32_t n_x, const double* const* A, const int32_t* dims, const int32_t* two_x,
                         const int32_t* two_klo, const double* const* psi, double* amps, double* total,
                         cudaStream_t stream);

/* Read-only access to internal tables for verification.
 *   kind SF_TAB_6J:    index 1..5 -> table S_index, all slots concatenated (doubles)
 *   kind SF_TAB_6J_SLOTS: index 1..5 -> slot descriptors, 8 int64 each:
 *                      {offset, a_lo, b_lo, x_lo, n_a, n_b, n_x, 0} (doubled lows, entries
 *                      slot[offset + (ia*n_b + ib)*n_x + ix] for a = a_lo + 2 ia, ...)
 *   kind SF_TAB_D:     index 0..9 -> d-table of that face, complex doubles
 *                      [n_l][2k+1][n_nodes] (l = j + il, m = -k + im)
 *   kind SF_TAB_NODES: index 0 -> rule x_n, 1 -> rule weights w_n, 2 -> r_n = -ln x_n (doubles)
 * sf_table_size returns the byte size; sf_table_copy copies it into dst (host or device). */
#define SF_TAB_6J       1
#define SF_TAB_6J_SLOTS 2
#define SF_TAB_D        3
#define SF_TAB_NODES    4
int64_t sf_table_size(const sf_tables* t, int32_t vertex, int32_t kind, int32_t index);
int sf_table_copy(const sf_tables* t, int32_t vertex, int32_t kind, int32_t index, void* dst,
                  int64_t n_bytes, cudaStream_t stream);

/* Self-check of the compensated-pair dot products of SF_MIXED_FF, on the device, by the very
 * device steps its shell kernel uses (Ogita, Rump and Oishi's Dot2 on (hi, lo) float pairs with
 * Dekker's FMA TwoProduct): n_dots dot products of length len, terms taken in increasing index.
 *   kind 0: pair x float  (a: [n_dots][len][2] floats (hi, lo); b: [n_dots][len] floats)
 *   kind 1: pair x pair   (a and b: [n_dots][len][2] floats)
 *   out: [n_dots][2] floats, the normalised (hi, lo) result. All three are device pointers.
 * Synchronises the stream. Errors: SF_ERR_ARG (kind, sizes or null pointers), SF_ERR_CUDA. */
int sf_check_dot2(int32_t kind, int32_t n_dots, int32_t len, const float* a, const float* b, float* out,
                  cudaStream_t stream);

/* Number of kernels this library has launched in the process (all entry points). */
int64_t sf_kernel_launches(void);

/* Device time in milliseconds of the last shell-sum kernel launched by sf_vertex_amplitude on
 * the calling thread (kind 0), measured with CUDA events recorded on the call's stream around
 * that launch; -1 if none. */
double sf_last_kernel_ms(int32_t kind);

/* Release the tables object and all its device memory (NULL is a no-op). */
void sf_tables_free(sf_tables* t);

#ifdef __cplusplus
}
#endif
#endif /* SF_EPRL_H */
