// {6j} tables S1..S5 of the vertex algorithm (Sec. 3, framed algorithm step 4), exact.
#include "sf_racah.cuh"

// n! for n = 0..SF_FACT_MAX as double-double (sequential products, relative error ~n 2^-106)
__global__ void k_fact_table(dd* F) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    dd f = dd_make(1.0);
    F[0] = f;
    for (int n = 1; n <= SF_FACT_MAX; n++) {
        f = dd_mul_d(f, (double)n);
        F[n] = f;
    }
}

// triangle coefficients of all triads with doubled spins up to m (one thread per entry)
__global__ void k_tri_table(int m, const dd* __restrict__ F, dd* __restrict__ out) {
    const int m1 = m + 1;
    const int64_t n = (int64_t)m1 * m1 * m1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const int z = (int)(e % m1), y = (int)((e / m1) % m1), x = (int)(e / ((int64_t)m1 * m1));
        // triads beyond the factorial table never occur in a table the host admits
        const bool ok = sf_tri(x, y, z) && (x + y + z) / 2 + 1 <= SF_FACT_MAX;
        out[e] = ok ? sf_delta(F, x, y, z) : dd{0.0, 0.0};
    }
}

int sf_tri_table_build(int m, const dd* F, dd* d_out, int num_sms, cudaStream_t s) {
    const int64_t n = (int64_t)(m + 1) * (m + 1) * (m + 1);
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_tri_table<<<(unsigned)blocks, 256, 0, s>>>(m, F, d_out);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// one thread per table entry (grid-stride); the slot of an entry is found by binary search. The
// six arguments are selected per table and the symbol is evaluated at one call site (one copy of
// the exact-arithmetic code in the instruction cache). need (optional): per slot, nonzero if the
// slot is built; entries of the other slots are set to zero.
__global__ void __launch_bounds__(256) k_sixj_table(int table_id, const VtxDev* __restrict__ vp,
                                                    const SlotDesc* __restrict__ slots, int nslots,
                                                    int64_t n, double* __restrict__ out,
                                                    const TriTable tt, const unsigned char* __restrict__ need,
                                                    int* status) {
    const VtxDev& v = *vp;
    const int D = v.D;
    const int j12 = v.tj[F12], j13 = v.tj[F13], j14 = v.tj[F14], j15 = v.tj[F15];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        int lo = 0, hi = nslots - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (slots[mid].off <= e) lo = mid; else hi = mid - 1;
        }
        if (need && !need[lo]) {
            out[e] = 0.0;
            continue;
        }
        const SlotDesc s = slots[lo];
        int64_t r = e - s.off;
        const int ix = (int)(r % s.nx);
        r /= s.nx;
        const int ib = (int)(r % s.nb);
        const int ia = (int)(r / s.nb);
        const int a = s.alo + 2 * ia, b = s.blo + 2 * ib, x = s.xlo + 2 * ix;
        int g[6];
        switch (table_id) {
            case 1: {   // slot d25: {i1 l25 x; k5 j14 j15}, a = i1, b = k5
                const int l25 = v.tj[F25] + 2 * lo;
                g[0] = a; g[1] = l25; g[2] = x; g[3] = b; g[4] = j14; g[5] = j15;
            } break;
            case 2: {   // slot (d35, d45): {j14 k5 x; l35 k4 l45}, a = k5, b = k4
                const int l35 = v.tj[F35] + 2 * (lo / D), l45 = v.tj[F45] + 2 * (lo % D);
                g[0] = j14; g[1] = a; g[2] = x; g[3] = l35; g[4] = b; g[5] = l45;
            } break;
            case 3: {   // slot (d24, d34, d35): {k4 l35 x; k3 l24 l34}, a = k4, b = k3
                const int l24 = v.tj[F24] + 2 * (lo / (D * D));
                const int l34 = v.tj[F34] + 2 * ((lo / D) % D);
                const int l35 = v.tj[F35] + 2 * (lo % D);
                g[0] = a; g[1] = l35; g[2] = x; g[3] = b; g[4] = l24; g[5] = l34;
            } break;
            case 4: {   // slot (d23, d24): {l24 k3 x; j13 k2 l23}, a = k3, b = k2
                const int l23 = v.tj[F23] + 2 * (lo / D), l24 = v.tj[F24] + 2 * (lo % D);
                g[0] = l24; g[1] = a; g[2] = x; g[3] = j13; g[4] = b; g[5] = l23;
            } break;
            default: {  // 5, slot d25: {k2 j13 x; i1 l25 j12}, a = k2, b = i1
                const int l25 = v.tj[F25] + 2 * lo;
                g[0] = a; g[1] = j13; g[2] = x; g[3] = b; g[4] = l25; g[5] = j12;
            } break;
        }
        out[e] = sf_sixj(g[0], g[1], g[2], g[3], g[4], g[5], tt, status);
    }
}

int sf_fact_table_build(dd* F, cudaStream_t s) {
    k_fact_table<<<1, 1, 0, s>>>(F);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

int sf_sixj_table_build(int table_id, const VtxDev* d_v, const SlotDesc* d_slots, int nslots, int64_t n,
                        double* d_out, const dd* d_tri, int tri_m, const unsigned char* d_need, int* d_status,
                        int num_sms, cudaStream_t s) {
    if (n <= 0) return SF_OK;
    int64_t blocks = (n + 255) / 256;
    int64_t cap = (int64_t)num_sms * 16;
    if (blocks > cap) blocks = cap;
    TriTable tt;
    tt.d = d_tri;
    tt.m1 = tri_m + 1;
    k_sixj_table<<<(unsigned)blocks, 256, 0, s>>>(table_id, d_v, d_slots, nslots, n, d_out, tt, d_need, d_status);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)in[i];
}

// S1 with the weight (x+1) = 2x+1 (doubled x) of the x-sum folded in: one CTA per slot
__global__ void k_scale_x(const double* __restrict__ in, const SlotDesc* __restrict__ slots, double* __restrict__ out) {
    const SlotDesc sd = slots[blockIdx.x];
    const int64_t n = (int64_t)sd.na * sd.nb * sd.nx;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int ix = (int)(i % sd.nx);
        out[sd.off + i] = (double)(sd.xlo + 2 * ix + 1) * in[sd.off + i];
    }
}

int sf_scale_x(const double* d_in, const SlotDesc* d_slots, int nslots, double* d_out, cudaStream_t s) {
    if (nslots <= 0) return SF_OK;
    k_scale_x<<<nslots, 256, 0, s>>>(d_in, d_slots, d_out);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

__global__ void k_to_ff(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double d = in[i];
        const float hi = (float)d;
        out[i] = make_float2(hi, (float)(d - (double)hi));
    }
}

int sf_to_ff(const double* d_in, float2* d_out, int64_t n, int num_sms, cudaStream_t s) {
    if (n <= 0) return SF_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_to_ff<<<(unsigned)blocks, 256, 0, s>>>(d_in, d_out, n);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

int sf_to_float(const double* d_in, float* d_out, int64_t n, int num_sms, cudaStream_t s) {
    if (n <= 0) return SF_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > (int64_t)num_sms * 16) blocks = (int64_t)num_sms * 16;
    k_to_float<<<(unsigned)blocks, 256, 0, s>>>(d_in, d_out, n);
    sf_note_launch(1);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}
