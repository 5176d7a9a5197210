// pdf.cu -- inverse transform sampling from piecewise-constant PDFs
// (nacc_sample_pdf): Eq. 1 t = F^-1(u), with the CDF read as 1 - T (Eq. 3,
// Table 1 "PDF Approaches").
//
// One thread per ray walks bins and outputs together (both are monotone), so
// no per-ray CDF array is stored: F_j is formed on the fly with exactly the
// sequential FP32 prefix sums of the definition, and the bin of u_k is the
// largest j with F_j <= u_k and F_j < 1.  The rows of a CTA's rays are
// staged through shared memory with coalesced loads when they fit.
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

__global__ void __launch_bounds__(kPdfThreads) k_sample_pdf(PdfArgs A) {
    extern __shared__ float s_rows[];
    const int nb = A.n_bins, no = A.n_out;
    const int ew = nb + 1, ww = nb;
    const int64_t r0 = (int64_t)blockIdx.x * kPdfThreads;
    const int64_t left = A.n_rays - r0;
    const int nr = left < kPdfThreads ? (int)left : kPdfThreads;
    const float* E;
    const float* W;
    int es, ws;  // row strides
    if (A.staged) {
        // stage rows [r0, r0+nr): edges then weights, row strides ew|1, ww|1 (odd: no conflicts)
        const int se = ew | 1, sw = ww | 1;
        float* sE = s_rows;
        float* sW = s_rows + kPdfThreads * se;
        const float* gE = A.edges + r0 * ew;
        const float* gW = A.weights + r0 * ww;
        for (int q = threadIdx.x; q < nr * ew; q += kPdfThreads) {
            int rr = q / ew;
            sE[rr * se + (q - rr * ew)] = __ldcs(gE + q);
        }
        for (int q = threadIdx.x; q < nr * ww; q += kPdfThreads) {
            int rr = q / ww;
            sW[rr * sw + (q - rr * ww)] = __ldcs(gW + q);
        }
        __syncthreads();
        E = sE + threadIdx.x * se;
        W = sW + threadIdx.x * sw;
        es = se;
        ws = sw;
    } else {
        E = A.edges + (r0 + threadIdx.x) * ew;
        W = A.weights + (r0 + threadIdx.x) * ww;
        es = ew;
        ws = ww;
    }
    (void)es;
    (void)ws;
    if (threadIdx.x >= nr) return;
    const int64_t r = r0 + threadIdx.x;
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
    float* out = A.out + r * (no + 1);
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
    size_t shm = (size_t)kPdfThreads * (size_t)(((n_bins + 1) | 1) + (n_bins | 1)) * sizeof(float);
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
