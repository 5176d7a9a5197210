// proposal.cu -- the glue kernels of the learned-proposal estimator
// (nacc_proposal.h): uniform initial bins per ray, transmittance weights of
// a dense [ray][bin] layout (the PDF of Table 1 "PDF Approaches": w_j =
// T_j (1 - exp(-sigma_j dt_j)), Eq. 2), and the final bins as packed samples
// (Sec. 4.2 "Packed Tensor") for the radiance field and the renderer.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

// Ray clip against the box of level 0, the same individually rounded
// operations as the lattice march's clip.
__device__ __forceinline__ bool clip_box(const Level& lv, const float o[3], const float d[3], float t_min,
                                         float t_max, float& tn, float& tf) {
    float near = t_min, far = t_max;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < lv.lmin[a] || o[a] > lv.lmax[a]) return false;
            continue;
        }
        const float inv = __fdiv_rn(1.0f, d[a]);
        const float ta = __fmul_rn(__fsub_rn(lv.lmin[a], o[a]), inv);
        const float tb = __fmul_rn(__fsub_rn(lv.lmax[a], o[a]), inv);
        const float lo = (ta < tb) ? ta : tb;
        const float hi = (ta < tb) ? tb : ta;
        if (lo > near) near = lo;
        if (hi < far) far = hi;
    }
    tn = near;
    tf = far;
    return near < far;
}

__global__ void k_uniform_edges(GridGeom g, const float* __restrict__ o, const float* __restrict__ d, int64_t n,
                                float t_min, float t_max, int nb, float* __restrict__ edges) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const float oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
        const float dd[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
        float tn, tf;
        if (!clip_box(g.lv[0], oo, dd, t_min, t_max, tn, tf)) {
            tn = fmaxf(t_min, 0.0f);
            tf = tn;  // a miss: empty bins
        }
        const float span = __fsub_rn(tf, tn);
        float* e = edges + r * (nb + 1);
        for (int j = 0; j < nb; ++j) e[j] = __fadd_rn(tn, __fmul_rn(span, __fdiv_rn((float)j, (float)nb)));
        e[nb] = tf;
    }
}

__global__ void k_range_edges(const float* __restrict__ lo, const float* __restrict__ hi, int64_t n, int nb,
                              float* __restrict__ edges) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const float tn = lo[r], tf = hi[r];
        const float span = __fsub_rn(tf, tn);
        float* e = edges + r * (nb + 1);
        for (int j = 0; j < nb; ++j) e[j] = __fadd_rn(tn, __fmul_rn(span, __fdiv_rn((float)j, (float)nb)));
        e[nb] = tf;
    }
}

// One warp per ray: tau_j = sigma_j (e_{j+1} - e_j), exclusive prefix P_j by
// warp scans (carry across 32-bin chunks), w_j = exp(-P_j) (1 - exp(-tau_j)).
__global__ void __launch_bounds__(256) k_dense_weights(int64_t n, int nb, const float* __restrict__ edges,
                                                       const float* __restrict__ sigma, float* __restrict__ w,
                                                       float* __restrict__ trans) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        const float* e = edges + r * (nb + 1);
        const float* s = sigma + r * nb;
        float* wr = w + r * nb;
        float carry = 0.0f;
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int j = j0 + lane;
            const float tau = j < nb ? s[j] * (e[j + 1] - e[j]) : 0.0f;
            float incl = tau;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            const float P = carry + (incl - tau);
            if (j < nb) {
                const float a = tau < 0.0625f ? tau * (1.0f - 0.5f * tau * (1.0f - tau * (1.0f / 3.0f) * (1.0f - 0.25f * tau)))
                                              : 1.0f - __expf(-tau);
                wr[j] = __expf(-P) * a;
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (trans && lane == 0) trans[r] = __expf(-carry);
    }
}

__global__ void k_edges_to_packed(int64_t n, int nb, const float* __restrict__ edges, int64_t* __restrict__ offsets,
                                  float* __restrict__ t0, float* __restrict__ t1, int64_t* __restrict__ n_samples) {
    const int64_t total = n * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / nb, j = i - r * nb;
        const float* e = edges + r * (nb + 1) + j;
        t0[i] = e[0];
        t1[i] = e[1];
        if (j == 0) offsets[r] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        offsets[n] = total;
        *n_samples = total;
    }
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_uniform_edges(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                                  float t_min, float t_max, int32_t n_bins, float* edges, void* stream) {
    clear_error();
    GridGeom g;
    if (!make_geom(grid, &g, false)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    NACC_CHECK_ARG(!std::isnan(t_min) && !std::isnan(t_max), "t_min/t_max is NaN");
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(rays_o && rays_d && edges, "a pointer argument is NULL");
    const int blocks = (int)min64((n_rays + 255) / 256, (int64_t)sm_count() * 8);
    k_uniform_edges<<<blocks, 256, 0, as_stream(stream)>>>(g, rays_o, rays_d, n_rays, t_min, t_max, n_bins, edges);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_range_edges(int64_t n_rays, const float* t_lo, const float* t_hi, int32_t n_bins, float* edges,
                                void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(t_lo && t_hi && edges, "a pointer argument is NULL");
    const int blocks = (int)min64((n_rays + 255) / 256, (int64_t)sm_count() * 8);
    k_range_edges<<<blocks, 256, 0, as_stream(stream)>>>(t_lo, t_hi, n_rays, n_bins, edges);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_dense_weights(int64_t n_rays, int32_t n_bins, const float* edges, const float* sigmas,
                                  float* weights, float* trans_out, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(edges && sigmas && weights, "a pointer argument is NULL");
    const int blocks = (int)min64((n_rays + 7) / 8, (int64_t)sm_count() * 8);
    k_dense_weights<<<blocks, 256, 0, as_stream(stream)>>>(n_rays, n_bins, edges, sigmas, weights, trans_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_edges_to_packed(int64_t n_rays, int32_t n_bins, const float* edges, int64_t* offsets,
                                    float* t_starts, float* t_ends, int64_t* n_samples, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 34), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    NACC_CHECK_ARG(offsets && n_samples, "offsets / n_samples is NULL");
    if (n_rays == 0) {
        NACC_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), as_stream(stream)));
        NACC_CUDA_TRY(cudaMemsetAsync(n_samples, 0, sizeof(int64_t), as_stream(stream)));
        return NACC_OK;
    }
    NACC_CHECK_ARG(edges && t_starts && t_ends, "a pointer argument is NULL");
    const int blocks = (int)min64((n_rays * n_bins + 255) / 256, (int64_t)sm_count() * 8);
    k_edges_to_packed<<<blocks, 256, 0, as_stream(stream)>>>(n_rays, n_bins, edges, offsets, t_starts, t_ends,
                                                             n_samples);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
