// pdf.cu -- inverse transform sampling from piecewise-constant PDFs
// (nacc_sample_pdf): Eq. 1 t = F^-1(u), with the CDF read as 1 - T (Eq. 3,
// Table 1 "PDF Approaches").
//
// One thread per ray walks bins and outputs together (both are monotone), so
// no per-ray CDF array is stored: F_j is formed on the fly with exactly the
// sequential FP32 prefix sums of the definition, and the bin of u_k is the
// largest j with F_j <= u_k and F_j < 1.  The weight rows of a CTA's rays
// are staged through shared memory with coalesced loads when they fit.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kPdfThreads = 64;

struct PdfArgs {
    int64_t n_rays;
    int n_bins, n_out;
    const float* edges;
    const float* weights;
    float* out;
    int stratified;
    uint64_t seed;
    int staged;  // rows staged in shared memory
};

// Copies nr contiguous rows of length w between global memory (row stride
// w) and shared memory (row stride ws), in either direction, with eight
// accesses in flight per thread.  Equal strides: one flat copy.  Otherwise
// each warp copies 32-column pieces of whole rows (one division per piece).
template <bool kToShared>
__device__ __forceinline__ void copy_rows(float* g, int nr, int w, float* s, int ws) {
    constexpr int kU = 8;
    if (ws == w) {
        const int n = nr * w;
        for (int q0 = threadIdx.x; q0 < n; q0 += kU * kPdfThreads) {
            float v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * kPdfThreads;
                if (q < n) v[u] = kToShared ? __ldcs(g + q) : s[q];
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int q = q0 + u * kPdfThreads;
                if (q < n) {
                    if (kToShared)
                        s[q] = v[u];
                    else
                        g[q] = v[u];
                }
            }
        }
        return;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = kPdfThreads / 32;
    const int nch = (w + 31) / 32, items = nr * nch;
    for (int i0 = wid; i0 < items; i0 += kU * nw) {
        float v[kU];
        int gi[kU], si[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * nw;
            gi[u] = -1;
            if (i < items) {
                const int rr = i / nch;
                const int col = (i - rr * nch) * 32 + lane;
                if (col < w) {
                    gi[u] = rr * w + col;
                    si[u] = rr * ws + col;
                    v[u] = kToShared ? __ldcs(g + gi[u]) : s[si[u]];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (gi[u] >= 0) {
                if (kToShared)
                    s[si[u]] = v[u];
                else
                    g[gi[u]] = v[u];
            }
        }
    }
}

// The walk of one ray; outputs to `o` (shared memory) or, if NULL, to the
// ray's global output row.
__device__ __forceinline__ void sample_one(const PdfArgs& A, int64_t r, const float* E, const float* W, float* o) {
    const int nb = A.n_bins, no = A.n_out;
    float tot = 0.0f;
    for (int j = 0; j < nb; ++j) tot = __fadd_rn(tot, W[j]);
    const bool uni = !(tot > 0.0f);
    const float fnb = (float)nb, fno = (float)no;
    const float U = A.stratified ? u01_from_bits(splitmix64(A.seed, (uint64_t)r)) : 0.0f;
    // F_j for the current bin j and the next, formed incrementally
    int j = 0;
    float cj = 0.0f;  // w_0 + ... + w_{j-1}
    float Fj = 0.0f;
    float cn = uni ? 0.0f : __fadd_rn(cj, W[0]);
    auto F_of = [&](int jj, float c) -> float {
        if (jj >= nb) return 1.0f;
        if (uni) return __fdiv_rn((float)jj, fnb);
        return __fdiv_rn(c, tot);
    };
    float Fn = F_of(1, cn);
    float* out = o ? o : A.out + r * (no + 1);
    for (int k = 0; k <= no; ++k) {
        float u = __fdiv_rn((float)k, fno);
        if (A.stratified && k > 0 && k < no) {
            u = __fdiv_rn(__fadd_rn((float)k, U), fno);
            if (u > 1.0f) u = 1.0f;
        }
        // advance while the next bin start qualifies: F_{j+1} <= u, F_{j+1} < 1, j+1 <= n-1
        while (j + 1 <= nb - 1 && Fn <= u && Fn < 1.0f) {
            ++j;
            cj = cn;
            Fj = Fn;
            if (!uni) cn = __fadd_rn(cj, W[j]);
            Fn = F_of(j + 1, cn);
        }
        float den = __fsub_rn(Fn, Fj);
        float e0 = E[j];
        float t = e0;
        if (den > 0.0f) {
            float fr = __fdiv_rn(__fsub_rn(u, Fj), den);
            t = __fadd_rn(e0, __fmul_rn(fr, __fsub_rn(E[j + 1], e0)));
        }
        out[k] = t;
    }
}

__global__ void __launch_bounds__(kPdfThreads) k_sample_pdf(PdfArgs A) {
    extern __shared__ float s_rows[];
    const int nb = A.n_bins;
    const int ew = nb + 1, ww = nb;
    const int64_t r0 = (int64_t)blockIdx.x * kPdfThreads;
    const int64_t left = A.n_rays - r0;
    const int nr = left < kPdfThreads ? (int)left : kPdfThreads;
    const float* E;
    const float* W;
    // the weights, read in sequence by the walk, are staged (row stride
    // ww|1, odd: no bank conflicts); the edges are read twice per output
    // straight from global memory (each row stays in L1), the outputs are
    // stored directly: small shared memory keeps many warps resident
    E = A.edges + (r0 + threadIdx.x) * ew;
    if (A.staged) {
        const int sw = ww | 1;
        copy_rows<true>(const_cast<float*>(A.weights + r0 * ww), nr, ww, s_rows, sw);
        __syncthreads();
        W = s_rows + threadIdx.x * sw;
    } else {
        W = A.weights + (r0 + threadIdx.x) * ww;
    }
    if (threadIdx.x < nr) sample_one(A, r0 + threadIdx.x, E, W, nullptr);
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_sample_pdf(int64_t n_rays, int32_t n_bins, const float* edges,
                               const float* weights, int32_t n_out, int32_t stratified,
                               uint64_t seed, float* edges_out, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    NACC_CHECK_ARG(n_out >= 1 && n_out <= 4096, "n_out=%d outside [1, 4096]", n_out);
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(edges && weights && edges_out, "edges / weights / edges_out is NULL");
    PdfArgs A{n_rays, n_bins, n_out, edges, weights, edges_out, stratified ? 1 : 0, seed, 0};
    size_t shm = (size_t)kPdfThreads * (size_t)(n_bins | 1) * sizeof(float);
    if (shm <= 96 * 1024) {
        A.staged = 1;
        if (shm > 48 * 1024)
            NACC_CUDA_TRY(cudaFuncSetAttribute(k_sample_pdf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    } else {
        shm = 0;
    }
    int64_t blocks = (n_rays + kPdfThreads - 1) / kPdfThreads;
    NACC_CHECK_ARG(blocks < (int64_t(1) << 31), "too many rays");
    k_sample_pdf<<<(unsigned)blocks, kPdfThreads, shm, as_stream(stream)>>>(A);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
