// Contractions of vertex tensors (Sec. 3 "Tensor contractions"; eq. vertex-contraction; the GPU
// workload of Sec. 4 "Tensor contractions on CPU and GPU", fig. contractions) and the three-vertex
// Delta_3 network with one internal face (Sec. 5 "The Delta_3 graph").
//
//   sf_contract_vectors   T[lead] = sum over the trailing 3, 4 or 5 intertwiner indices of
//                         A[i1][i2][i3][i4][i5] prod_e psi_e[i_e]          (psi complex, A real)
//   sf_contract_vertices  sum_i A[i] B[i]                                   (complete contraction)
//   sf_delta3_amplitudes  per internal spin x: (-1)^x (2x+1) sum_{k1 k2 k3} (-1)^(k1+k2+k3)
//                         T_A[k1][k2] T_C[k2][k3] T_B[k3][k1], and the sum over x
//
// A vertex tensor is read from HBM exactly once. The vector contraction costs two FP64 FMAs per
// entry (a real entry times a complex weight), which on this GPU (2 FP64 FMAs per clock per SM)
// is below the HBM rate, so it is bound by the FP64 pipe; the two-vertex contraction (one FMA per
// 16 bytes) is bound by HBM. Every reduction runs in a fixed order (bitwise reproducible).
#include "sf_internal.cuh"

struct c2 { double x, y; };
__device__ __forceinline__ c2 c2mul(c2 a, c2 b) { return c2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

// block-wide sum of a complex value (blockDim.x a multiple of 32, at most 1024); result in lane 0
// of warp 0
__device__ __forceinline__ c2 block_sum_c2(c2 v, c2* red) {
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    c2 s{0.0, 0.0};
    if (warp == 0) {
        for (int w = lane; w < nw; w += 32) { s.x += red[w].x; s.y += red[w].y; }
        for (int off = 16; off > 0; off >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
        }
    }
    return s;
}

// One CTA per slab (i1, i2): P[i1][i2] = sum_{i3 i4 i5} A[i1][i2][i3][i4][i5] psi3[i3] psi4[i4] psi5[i5].
// Thread (c5, g) with c5 = tid % D5 handles the rows r = g, g + R, ... of the slab's D3 D4 rows
// (R = blockDim / D5 row groups), so a warp reads consecutive addresses of consecutive rows; it
// accumulates w[r] A[r][c5] with the row weight w = psi3 psi4 from shared memory (two FMAs per
// entry) and multiplies by psi5[c5] once at the end.
__global__ void __launch_bounds__(1024) k_contract_slab(const double* __restrict__ A, int D3, int D4, int D5,
                                                        const c2* __restrict__ p3, const c2* __restrict__ p4,
                                                        const c2* __restrict__ p5, c2* __restrict__ P) {
    extern __shared__ __align__(16) unsigned char cs_smem[];
    c2* w34 = reinterpret_cast<c2*>(cs_smem);          // [D3 D4]
    c2* red = w34 + D3 * D4;                            // [32]
    const int nrow = D3 * D4;
    for (int q = threadIdx.x; q < nrow; q += blockDim.x) w34[q] = c2mul(p3[q / D4], p4[q % D4]);
    __syncthreads();
    const int R = blockDim.x / D5;
    const int c5 = threadIdx.x % D5, g = threadIdx.x / D5;
    c2 acc{0.0, 0.0};
    if (g < R) {
        const double* slab = A + (int64_t)blockIdx.x * nrow * D5 + c5;
        int r = g;
        for (; r + 3 * R < nrow; r += 4 * R) {   // four loads in flight
            const double a0 = __ldg(slab + (int64_t)r * D5), a1 = __ldg(slab + (int64_t)(r + R) * D5);
            const double a2 = __ldg(slab + (int64_t)(r + 2 * R) * D5), a3 = __ldg(slab + (int64_t)(r + 3 * R) * D5);
            const c2 w0 = w34[r], w1 = w34[r + R], w2 = w34[r + 2 * R], w3 = w34[r + 3 * R];
            acc.x = fma(w0.x, a0, acc.x); acc.y = fma(w0.y, a0, acc.y);
            acc.x = fma(w1.x, a1, acc.x); acc.y = fma(w1.y, a1, acc.y);
            acc.x = fma(w2.x, a2, acc.x); acc.y = fma(w2.y, a2, acc.y);
            acc.x = fma(w3.x, a3, acc.x); acc.y = fma(w3.y, a3, acc.y);
        }
        for (; r < nrow; r += R) {
            const double a = __ldg(slab + (int64_t)r * D5);
            const c2 w = w34[r];
            acc.x = fma(w.x, a, acc.x);
            acc.y = fma(w.y, a, acc.y);
        }
        acc = c2mul(acc, p5[c5]);
    }
    const c2 s = block_sum_c2(acc, red);
    if (threadIdx.x == 0) P[blockIdx.x] = s;
}

// out[i1] = sum_{i2} psi2[i2] P[i1][i2] (n_vec = 4), or out[0] = sum_{i1 i2} psi1[i1] psi2[i2] P[i1][i2]
// (n_vec = 5); one CTA per output, terms in index order
__global__ void k_contract_lead(const c2* __restrict__ P, int D1, int D2, int n_vec, const c2* __restrict__ p1,
                                const c2* __restrict__ p2, c2* __restrict__ out) {
    __shared__ c2 red[32];
    const int n = n_vec == 5 ? D1 * D2 : D2;
    const int base = n_vec == 5 ? 0 : blockIdx.x * D2;
    c2 acc{0.0, 0.0};
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const int i1 = n_vec == 5 ? q / D2 : blockIdx.x, i2 = n_vec == 5 ? q % D2 : q;
        c2 w = p2[i2];
        if (n_vec == 5) w = c2mul(w, p1[i1]);
        const c2 z = c2mul(w, P[base + q]);
        acc.x += z.x;
        acc.y += z.y;
    }
    const c2 s = block_sum_c2(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

static int slab_threads(int D5) {
    const int R = imax_(1, 1024 / D5);
    int nt = R * D5;
    nt = ((nt + 31) / 32) * 32;
    return nt > 1024 ? 1024 : nt;
}

static int launch_slabs(const double* A, const int32_t dim[5], const c2* p3, const c2* p4, const c2* p5, c2* P,
                        cudaStream_t s) {
    const int nt = slab_threads(dim[4]);
    const size_t smem = ((size_t)dim[2] * dim[3] + 32) * sizeof(c2);
    if (smem > 200 * 1024) return sf_set_error(SF_ERR_LIMIT, "slab of %d x %d rows too large", dim[2], dim[3]);
    SF_CUDA_TRY(cudaFuncSetAttribute(k_contract_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_contract_slab<<<dim[0] * dim[1], nt, smem, s>>>(A, dim[2], dim[3], dim[4], p3, p4, p5, P);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

static int check_dims(const int32_t dim[5]) {
    if (!dim) return sf_set_error(SF_ERR_ARG, "null dimensions");
    int64_t n = 1;
    for (int e = 0; e < 5; e++) {
        if (dim[e] < 1 || dim[e] > 1024) return sf_set_error(SF_ERR_ARG, "dimension %d = %d out of range", e + 1, dim[e]);
        n *= dim[e];
    }
    if ((int64_t)dim[0] * dim[1] > 0x7FFFFFFF) return sf_set_error(SF_ERR_LIMIT, "too many slabs");
    return SF_OK;
}

extern "C" int sf_contract_vectors(const double* A, const int32_t dim[5], int32_t n_vec, const double* const psi[5],
                                   double* out, cudaStream_t stream) {
    SF_TRY(check_dims(dim));
    if (!A || !psi || !out) return sf_set_error(SF_ERR_ARG, "null argument");
    if (n_vec < 3 || n_vec > 5) return sf_set_error(SF_ERR_ARG, "n_vec must be 3, 4 or 5");
    for (int e = 5 - n_vec; e < 5; e++)
        if (!psi[e]) return sf_set_error(SF_ERR_ARG, "null vector for index %d", e + 1);
    const c2* p[5];
    for (int e = 0; e < 5; e++) p[e] = reinterpret_cast<const c2*>(psi[e]);
    c2* P = reinterpret_cast<c2*>(out);
    void* tmp = nullptr;
    if (n_vec > 3) {
        SF_TRY(sf_scratch_alloc(&tmp, (size_t)dim[0] * dim[1] * sizeof(c2), stream));
        P = reinterpret_cast<c2*>(tmp);
    }
    int rc = launch_slabs(A, dim, p[2], p[3], p[4], P, stream);
    if (rc == SF_OK && n_vec > 3) {
        k_contract_lead<<<n_vec == 5 ? 1 : dim[0], 256, 0, stream>>>(P, dim[0], dim[1], n_vec, p[0], p[1],
                                                                     reinterpret_cast<c2*>(out));
        sf_note_launch(1);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = sf_set_error(SF_ERR_CUDA, "contraction launch: %s", cudaGetErrorString(e));
    }
    if (tmp) sf_scratch_free(tmp, stream);
    return rc;
}

// sum_i A[i] B[i]: CTA b takes the contiguous chunk [b n / G, (b+1) n / G) with 16-byte loads
// where both operands are 16-byte aligned; partial sums reduced in block order
__global__ void __launch_bounds__(256) k_dot_chunks(const double* __restrict__ A, const double* __restrict__ B, int64_t n,
                                                    double* __restrict__ part) {
    __shared__ c2 red[32];
    const int64_t lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
    double s0 = 0.0, s1 = 0.0;
    int64_t q = lo;
    // align the start of the vector loop to an even index (16 bytes, given 16-byte-aligned bases)
    if ((q & 1) && q < hi) {
        if (threadIdx.x == 0) s0 = fma(__ldg(A + q), __ldg(B + q), s0);
        q++;
    }
    const int64_t nv = (hi - q) / 2;
    const double2* A2 = reinterpret_cast<const double2*>(A + q);
    const double2* B2 = reinterpret_cast<const double2*>(B + q);
    int64_t v = threadIdx.x;
    for (; v + 3 * (int64_t)blockDim.x < nv; v += 4 * (int64_t)blockDim.x) {
        const double2 a0 = __ldg(A2 + v), b0 = __ldg(B2 + v);
        const double2 a1 = __ldg(A2 + v + blockDim.x), b1 = __ldg(B2 + v + blockDim.x);
        const double2 a2 = __ldg(A2 + v + 2 * blockDim.x), b2 = __ldg(B2 + v + 2 * blockDim.x);
        const double2 a3 = __ldg(A2 + v + 3 * blockDim.x), b3 = __ldg(B2 + v + 3 * blockDim.x);
        s0 = fma(a0.x, b0.x, s0); s1 = fma(a0.y, b0.y, s1);
        s0 = fma(a1.x, b1.x, s0); s1 = fma(a1.y, b1.y, s1);
        s0 = fma(a2.x, b2.x, s0); s1 = fma(a2.y, b2.y, s1);
        s0 = fma(a3.x, b3.x, s0); s1 = fma(a3.y, b3.y, s1);
    }
    for (; v < nv; v += blockDim.x) {
        const double2 a = __ldg(A2 + v), b = __ldg(B2 + v);
        s0 = fma(a.x, b.x, s0);
        s1 = fma(a.y, b.y, s1);
    }
    const int64_t tail = q + 2 * nv;
    if (threadIdx.x == 0 && tail < hi) s0 = fma(__ldg(A + tail), __ldg(B + tail), s0);
    const c2 s = block_sum_c2(c2{s0 + s1, 0.0}, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s.x;
}

__global__ void k_sum_parts(const double* __restrict__ part, int n, double* out) {
    __shared__ c2 red[32];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
    const c2 t = block_sum_c2(c2{s, 0.0}, red);
    if (threadIdx.x == 0) *out = t.x;
}

extern "C" int sf_contract_vertices(const double* A, const double* B, int64_t n, double* out, cudaStream_t stream) {
    if (!A || !B || !out || n < 0) return sf_set_error(SF_ERR_ARG, "bad arguments");
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return sf_set_error(SF_ERR_ARG, "tensors must be 16-byte aligned");
    int dev = 0, sms = 0;
    SF_CUDA_TRY(cudaGetDevice(&dev));
    SF_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t G = (int64_t)sms * 8;   // resident CTAs: 8 x 256 threads per SM
    if (G > (n + 511) / 512) G = (n + 511) / 512;
    if (G < 1) G = 1;
    double* part = nullptr;
    SF_TRY(sf_scratch_alloc((void**)&part, (size_t)G * sizeof(double), stream));
    k_dot_chunks<<<(unsigned)G, 256, 0, stream>>>(A, B, n, part);
    sf_note_launch(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_sum_parts<<<1, 256, 0, stream>>>(part, (int)G, out);
        sf_note_launch(1);
        e = cudaGetLastError();
    }
    sf_scratch_free(part, stream);
    if (e != cudaSuccess) return sf_set_error(SF_ERR_CUDA, "contraction launch: %s", cudaGetErrorString(e));
    return SF_OK;
}

// Delta_3: for each internal spin x (one CTA each), the three partial contractions T_A, T_B, T_C
// (each [k1][k2] = P of k_contract_slab with the vertex's three boundary vectors) are combined as
//   amp(x) = (-1)^x (2x+1) sum_{k1 k2 k3} (-1)^(k1+k2+k3) T_A[k1][k2] T_C[k2][k3] T_B[k3][k1]
// (the internal edges: the first vertex's (k1, k2), the second's (k1, k3) read in that order as
// T_B[k3][k1]'s transpose, the third's (k3, k2)); k = k_lo + 2 n in doubled units.
__global__ void k_delta3(const c2* __restrict__ T, const int* __restrict__ meta, int n_x, c2* __restrict__ amps) {
    __shared__ c2 red[32];
    const int xi = blockIdx.x;
    const int two_x = meta[3 * xi], two_klo = meta[3 * xi + 1], nk = meta[3 * xi + 2];
    int64_t off = 0;
    for (int q = 0; q < xi; q++) off += 3 * (int64_t)meta[3 * q + 2] * meta[3 * q + 2];
    const c2* TA = T + off;
    const c2* TB = TA + nk * nk;
    const c2* TC = TB + nk * nk;
    c2 acc{0.0, 0.0};
    for (int q = threadIdx.x; q < nk * nk * nk; q += blockDim.x) {
        const int n1 = q / (nk * nk), n2 = (q / nk) % nk, n3 = q % nk;
        const int ksum = (3 * two_klo + 2 * (n1 + n2 + n3)) / 2;
        c2 z = c2mul(c2mul(TA[n1 * nk + n2], TC[n2 * nk + n3]), TB[n3 * nk + n1]);
        if (ksum & 1) { z.x = -z.x; z.y = -z.y; }
        acc.x += z.x;
        acc.y += z.y;
    }
    c2 s = block_sum_c2(acc, red);
    if (threadIdx.x == 0) {
        const double f = (double)(two_x + 1) * (((two_x / 2) & 1) ? -1.0 : 1.0);
        amps[xi] = c2{f * s.x, f * s.y};
    }
}

__global__ void k_sum_c2(const c2* __restrict__ v, int n, c2* out) {
    __shared__ c2 red[32];
    c2 acc{0.0, 0.0};
    for (int q = threadIdx.x; q < n; q += blockDim.x) { acc.x += v[q].x; acc.y += v[q].y; }
    const c2 s = block_sum_c2(acc, red);
    if (threadIdx.x == 0) *out = s;
}

extern "C" int sf_delta3_amplitudes(int32_t n_x, const double* const* A, const int32_t* dims, const int32_t* two_x,
                                    const int32_t* two_klo, const double* const* psi, double* amps, double* total,
                                    cudaStream_t stream) {
    if (n_x < 1 || !A || !dims || !two_x || !two_klo || !psi || !amps || !total)
        return sf_set_error(SF_ERR_ARG, "null argument");
    for (int b = 0; b < 9; b++)
        if (!psi[b]) return sf_set_error(SF_ERR_ARG, "null boundary vector %d", b + 1);
    int64_t tot = 0;
    std::vector<int> meta(3 * n_x);
    for (int i = 0; i < n_x; i++) {
        const int32_t* d = dims + 5 * i;
        SF_TRY(check_dims(d));
        if (!A[i]) return sf_set_error(SF_ERR_ARG, "null vertex tensor %d", i);
        if (d[0] != d[1]) return sf_set_error(SF_ERR_ARG, "x %d: the two internal intertwiner ranges differ", i);
        if (two_x[i] < 0 || (two_x[i] & 1) || (two_klo[i] & 1))
            return sf_set_error(SF_ERR_ARG, "x %d: the internal spin and intertwiners must be integers", i);
        if (i > 0)
            for (int e = 2; e < 5; e++)
                if (d[e] != dims[e]) return sf_set_error(SF_ERR_ARG, "boundary dimensions must agree across x");
        meta[3 * i] = two_x[i];
        meta[3 * i + 1] = two_klo[i];
        meta[3 * i + 2] = d[0];
        tot += 3 * (int64_t)d[0] * d[0];
    }
    c2* T = nullptr;
    int* d_meta = nullptr;
    SF_TRY(sf_scratch_alloc((void**)&T, (size_t)tot * sizeof(c2), stream));
    int rc = sf_scratch_alloc((void**)&d_meta, meta.size() * sizeof(int), stream);
    cudaError_t e = cudaSuccess;
    if (rc == SF_OK) {
        e = cudaMemcpyAsync(d_meta, meta.data(), meta.size() * sizeof(int), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) rc = sf_set_error(SF_ERR_CUDA, "delta3 copy: %s", cudaGetErrorString(e));
    }
    int64_t off = 0;
    for (int i = 0; i < n_x && rc == SF_OK; i++) {
        const int32_t* d = dims + 5 * i;
        for (int v = 0; v < 3 && rc == SF_OK; v++) {
            // vertex v contracts its (i3, i4, i5) with psi[3v], psi[3v+1], psi[3v+2]
            rc = launch_slabs(A[i], d, reinterpret_cast<const c2*>(psi[3 * v]), reinterpret_cast<const c2*>(psi[3 * v + 1]),
                              reinterpret_cast<const c2*>(psi[3 * v + 2]), T + off, stream);
            off += (int64_t)d[0] * d[1];
        }
    }
    if (rc == SF_OK) {
        k_delta3<<<n_x, 256, 0, stream>>>(T, d_meta, n_x, reinterpret_cast<c2*>(amps));
        sf_note_launch(1);
        k_sum_c2<<<1, 256, 0, stream>>>(reinterpret_cast<const c2*>(amps), n_x, reinterpret_cast<c2*>(total));
        sf_note_launch(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = sf_set_error(SF_ERR_CUDA, "delta3 launch: %s", cudaGetErrorString(e));
    }
    sf_scratch_free(T, stream);
    if (d_meta) sf_scratch_free(d_meta, stream);
    if (rc != SF_OK) return rc;
    // the metadata was copied from this call's host vector: wait for the copy before it goes away
    SF_CUDA_TRY(cudaStreamSynchronize(stream));
    return SF_OK;
}
