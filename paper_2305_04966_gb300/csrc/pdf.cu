// pdf.cu -- inverse transform sampling from piecewise-constant PDFs
// (nacc_sample_pdf): Eq. 1 t = F^-1(u), with the CDF read as 1 - T (Eq. 3,
// Table 1 "PDF Approaches").
//
// One thread per ray; each warp owns 32 consecutive rays.  Their weight and
// edge rows come into the warp's shared memory by asynchronous 4-byte copies,
// issued all at once (one coalesced 128-byte segment per row piece and
// instruction), into rows of odd stride, so that each lane then reads its
// own ray's row without bank conflicts.  The total W and the prefix sums
// c_j are the definition's sequential FP32 sums.
//  - Rows of at most 64 bins (k_sample_pdf_rows): the whole rows are staged;
//    the lane turns its weight row into F_0..F_n in place (F_j = c_j / W),
//    then takes the outputs in a loop that is the same for every lane: u_k,
//    the bin by binary search over the non-decreasing F (the largest j with
//    F_j <= u_k and F_j < 1, a prefix predicate), t_k.  The outputs go out
//    through a small shared-memory buffer, eight columns of the 32 rows at a
//    time, as 32-byte row segments.
//  - Longer rows (k_sample_pdf_stream): chunks of 64 bins, two passes (the
//    total, then the walk over bins and outputs together, both monotone,
//    emitting every output whose bin is j).
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kPdfWarps = 2;
constexpr int kChunk = 64;               // bins per chunk
constexpr int kRowStride = kChunk + 1;   // odd: lane-per-row reads are conflict-free; holds kChunk + 1 edges
constexpr int kMaxStagedOut = 33;        // n_out + 1 <= this: outputs staged in shared memory

struct PdfArgs {
    int64_t n_rays;
    int n_bins, n_out;
    const float* edges;
    const float* weights;
    float* out;
    int stratified;
    uint64_t seed;
    int out_stride;  // > 0: outputs staged with this (odd) row stride; 0: stored directly
};

// floats of shared memory per warp: weight chunk, edge chunk, staged outputs
__host__ __device__ inline int pdf_warp_floats(int out_stride) { return 2 * 32 * kRowStride + 32 * out_stride; }

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src)
                 : "memory");
}

// dst[i][q] = src[(r0 + i) * stride + col0 + q] for rows i < nr, q < len: the
// lanes take consecutive q (one coalesced segment per row and instruction).
__device__ __forceinline__ void copy_chunk(float* dst, const float* src, int64_t r0, int nr, int64_t stride,
                                           int64_t col0, int len, int lane) {
    const float* p = src + r0 * stride + col0;
    for (int i = 0; i < nr; ++i)
        for (int q = lane; q < len; q += 32) cp_async4(dst + i * kRowStride + q, p + (int64_t)i * stride + q);
}

__device__ __forceinline__ void copies_done() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

__device__ __forceinline__ float u_of(int k, int no, float fno, bool strat, float U) {
    float u = __fdiv_rn((float)k, fno);
    if (strat && k > 0 && k < no) {
        u = __fdiv_rn(__fadd_rn((float)k, U), fno);
        if (u > 1.0f) u = 1.0f;
    }
    return u;
}

constexpr int kOutCols = 8;               // output columns per flush of the row kernel
constexpr int kOutStride = kOutCols + 1;
constexpr int kIlp = 4;                  // outputs searched together (kOutCols is a multiple)

// floats of shared memory per warp of the row kernel: F rows, edge rows, output buffer
__host__ __device__ inline int pdf_rows_warp_floats() { return 2 * 32 * kRowStride + 32 * kOutStride; }

__global__ void __launch_bounds__(kPdfWarps * 32) k_sample_pdf_rows(PdfArgs A) {
    extern __shared__ float s_pdf[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * kPdfWarps + wid) * 32;
    if (r0 >= A.n_rays) return;  // whole warps only: no block-wide barrier below
    const int nb = A.n_bins, no = A.n_out;
    float* Fs = s_pdf + (size_t)wid * pdf_rows_warp_floats();
    float* Es = Fs + 32 * kRowStride;
    float* Os = Es + 32 * kRowStride;
    const int nr = A.n_rays - r0 < 32 ? (int)(A.n_rays - r0) : 32;
    const int64_t r = r0 + lane;
    float* F = Fs + lane * kRowStride;
    const float* E = Es + lane * kRowStride;
    copy_chunk(Fs, A.weights, r0, nr, nb, 0, nb, lane);
    copy_chunk(Es, A.edges, r0, nr, nb + 1, 0, nb + 1, lane);
    copies_done();
    // c_j in place of w_j (lanes past the last ray work on rows never stored)
    float tot = 0.0f;
#pragma unroll 8
    for (int j = 0; j < nb; ++j) {
        const float w = F[j];
        F[j] = tot;
        tot = __fadd_rn(tot, w);
    }
    const bool uni = !(tot > 0.0f);
    const float fnb = (float)nb, fno = (float)no;
#pragma unroll 4
    for (int j = 0; j < nb; ++j) F[j] = uni ? __fdiv_rn((float)j, fnb) : __fdiv_rn(F[j], tot);
    F[nb] = 1.0f;
    const bool strat = A.stratified != 0;
    const float U = strat ? u01_from_bits(splitmix64(A.seed, (uint64_t)r)) : 0.0f;
    const int top = nb > 1 ? 1 << (31 - __clz(nb - 1)) : 0;  // largest power of two <= nb - 1
    for (int k0 = 0; k0 <= no; k0 += kOutCols) {
        const int ncol = no + 1 - k0 < kOutCols ? no + 1 - k0 : kOutCols;
        // kIlp outputs at a time, their searches interleaved (independent chains of shared-memory loads)
        for (int c0 = 0; c0 < ncol; c0 += kIlp) {
            float u[kIlp];
            int j[kIlp];
#pragma unroll
            for (int g = 0; g < kIlp; ++g) {
                u[g] = u_of(min(k0 + c0 + g, no), no, fno, strat, U);
                j[g] = 0;  // largest j in [0, nb-1] with F_j <= u and F_j < 1 (true at j = 0)
            }
            for (int st = top; st > 0; st >>= 1) {
#pragma unroll
                for (int g = 0; g < kIlp; ++g) {
                    const int q = j[g] + st;
                    if (q <= nb - 1) {
                        const float f = F[q];
                        if (f <= u[g] && f < 1.0f) j[g] = q;
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < kIlp; ++g) {
                const float Fj = F[j[g]], den = __fsub_rn(F[j[g] + 1], Fj);
                const float e0 = E[j[g]];
                float t = e0;
                if (den > 0.0f) {
                    const float fr = __fdiv_rn(__fsub_rn(u[g], Fj), den);
                    t = __fadd_rn(e0, __fmul_rn(fr, __fsub_rn(E[j[g] + 1], e0)));
                }
                if (c0 + g < ncol) Os[lane * kOutStride + c0 + g] = t;
            }
        }
        __syncwarp();
        // columns k0 .. k0+ncol-1 of the 32 rows: lane = (row group, column)
        for (int i = lane / kOutCols; i < nr; i += 32 / kOutCols) {
            const int c = lane % kOutCols;
            if (c < ncol) A.out[(r0 + i) * (no + 1) + k0 + c] = Os[i * kOutStride + c];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kPdfWarps * 32) k_sample_pdf_stream(PdfArgs A) {
    extern __shared__ float s_pdf[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * kPdfWarps + wid) * 32;
    if (r0 >= A.n_rays) return;  // whole warps only: no block-wide barrier below
    const int nb = A.n_bins, no = A.n_out, os = A.out_stride;
    float* Ws = s_pdf + (size_t)wid * pdf_warp_floats(os);
    float* Es = Ws + 32 * kRowStride;
    float* Os = Es + 32 * kRowStride;
    const int nr = A.n_rays - r0 < 32 ? (int)(A.n_rays - r0) : 32;
    const bool act = lane < nr;
    const int64_t r = r0 + lane;
    const float* wrow = Ws + lane * kRowStride;
    const float* erow = Es + lane * kRowStride;
    const bool one_chunk = nb <= kChunk;

    // W = w_0 + ... + w_{n-1}, in sequence
    float tot = 0.0f;
    for (int c0 = 0; c0 < nb; c0 += kChunk) {
        const int len = nb - c0 < kChunk ? nb - c0 : kChunk;
        copy_chunk(Ws, A.weights, r0, nr, nb, c0, len, lane);
        if (one_chunk) copy_chunk(Es, A.edges, r0, nr, nb + 1, 0, nb + 1, lane);
        copies_done();
        if (act) {
#pragma unroll 8
            for (int q = 0; q < len; ++q) tot = __fadd_rn(tot, wrow[q]);
        }
        __syncwarp();
    }
    const bool uni = !(tot > 0.0f);
    const float fnb = (float)nb, fno = (float)no;
    const bool strat = A.stratified != 0;
    const float U = strat ? u01_from_bits(splitmix64(A.seed, (uint64_t)r)) : 0.0f;

    // the walk: bin j (F_j, prefix c_j) against output k (u_k)
    int k = act ? 0 : no + 1;
    float u = u_of(0, no, fno, strat, U);
    float cj = 0.0f, Fj = 0.0f;
    float* orow = os ? Os + lane * os : A.out + r * (no + 1);
    for (int c0 = 0; c0 < nb; c0 += kChunk) {
        const int len = nb - c0 < kChunk ? nb - c0 : kChunk;
        if (!one_chunk) {  // e_{c0} .. e_{c0+len}
            copy_chunk(Ws, A.weights, r0, nr, nb, c0, len, lane);
            copy_chunk(Es, A.edges, r0, nr, nb + 1, c0, len + 1, lane);
            copies_done();
        }
        if (k <= no) {
            for (int q = 0; q < len; ++q) {
                const int j = c0 + q;
                const float cn = uni ? 0.0f : __fadd_rn(cj, wrow[q]);
                const float Fn = j + 1 >= nb ? 1.0f : (uni ? __fdiv_rn((float)(j + 1), fnb) : __fdiv_rn(cn, tot));
                const bool last = j == nb - 1;
                // every remaining output whose bin is j: bin j+1 does not qualify for it
                while (k <= no && (last || !(Fn <= u && Fn < 1.0f))) {
                    const float den = __fsub_rn(Fn, Fj);
                    const float e0 = erow[q];
                    float t = e0;
                    if (den > 0.0f) {
                        const float fr = __fdiv_rn(__fsub_rn(u, Fj), den);
                        t = __fadd_rn(e0, __fmul_rn(fr, __fsub_rn(erow[q + 1], e0)));
                    }
                    orow[k] = t;
                    ++k;
                    u = u_of(k, no, fno, strat, U);
                }
                if (k > no) break;
                cj = cn;
                Fj = Fn;
            }
        }
        __syncwarp();
    }
    if (os) {  // staged rows out, coalesced
        for (int i = 0; i < nr; ++i)
            for (int q = lane; q <= no; q += 32) A.out[(r0 + i) * (no + 1) + q] = Os[i * os + q];
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
    const int64_t blocks = (n_rays + 32 * kPdfWarps - 1) / (32 * kPdfWarps);
    NACC_CHECK_ARG(blocks < (int64_t(1) << 31), "too many rays");
    if (n_bins <= kChunk) {
        PdfArgs A{n_rays, n_bins, n_out, edges, weights, edges_out, stratified ? 1 : 0, seed, 0};
        const size_t shm = (size_t)kPdfWarps * pdf_rows_warp_floats() * sizeof(float);
        k_sample_pdf_rows<<<(unsigned)blocks, kPdfWarps * 32, shm, as_stream(stream)>>>(A);
    } else {
        const int os = n_out + 1 <= kMaxStagedOut ? ((n_out + 1) | 1) : 0;
        PdfArgs A{n_rays, n_bins, n_out, edges, weights, edges_out, stratified ? 1 : 0, seed, os};
        const size_t shm = (size_t)kPdfWarps * pdf_warp_floats(os) * sizeof(float);
        k_sample_pdf_stream<<<(unsigned)blocks, kPdfWarps * 32, shm, as_stream(stream)>>>(A);
    }
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
