// harness.cu -- stand-ins for the user's radiance field and loss
// (nacc_harness.h).  Not the method: they let a full sampling -> rendering
// -> gradient step run on synthetic Gaussian-blob scenes.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

__global__ void __launch_bounds__(256)
    k_field(const float* __restrict__ o, const float* __restrict__ d, const int32_t* __restrict__ ri,
            const float* __restrict__ t0, const float* __restrict__ t1,
            const int64_t* __restrict__ n_samples, nacc_blob_field f, float* __restrict__ sig,
            float* __restrict__ rgb) {
    extern __shared__ BlobS s_blobs[];
    stage_blobs(s_blobs, f, true);
    __syncthreads();
    const int64_t S = *n_samples;
    const int nb = f.n_blobs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = __ldcs(ri + i);
        const float m = 0.5f * (__ldcs(t0 + i) + __ldcs(t1 + i));
        const float x = __ldg(o + 3 * r) + __ldg(d + 3 * r) * m;
        const float y = __ldg(o + 3 * r + 1) + __ldg(d + 3 * r + 1) * m;
        const float z = __ldg(o + 3 * r + 2) + __ldg(d + 3 * r + 2) * m;
        float s = 0.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        for (int b = 0; b < nb; ++b) {
            const BlobS& v = s_blobs[b];
            float dx = x - v.mx, dy = y - v.my, dz = z - v.mz;
            float sb = v.peak * __expf((dx * dx + dy * dy + dz * dz) * v.coef);
            s += sb;
            cr += sb * v.r;
            cg += sb * v.g;
            cb += sb * v.b;
        }
        float inv = s > 0.0f ? 1.0f / s : 0.0f;
        __stcs(sig + i, s);
        __stcs(rgb + 3 * i, cr * inv);
        __stcs(rgb + 3 * i + 1, cg * inv);
        __stcs(rgb + 3 * i + 2, cb * inv);
    }
}

__global__ void __launch_bounds__(256)
    k_field_points(const float* __restrict__ xyz, int64_t n, nacc_blob_field f, float* __restrict__ sig) {
    extern __shared__ BlobS s_blobs[];
    stage_blobs(s_blobs, f, false);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        sig[i] = blob_sigma(s_blobs, f.n_blobs, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
    }
}

__global__ void __launch_bounds__(256)
    k_l2(const float* __restrict__ rgb, const float* __restrict__ tgt, int64_t m, float scale,
         float* __restrict__ g, float* __restrict__ loss) {
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        float e = rgb[i] - tgt[i];
        g[i] = 2.0f * scale * e;
        acc += e * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ float s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        atomicAdd(loss, t * scale);
    }
}

int check_field(const nacc_blob_field* f, bool rgb) {
    NACC_CHECK_ARG(f != nullptr, "field is NULL");
    NACC_CHECK_ARG(f->n_blobs >= 0 && f->n_blobs <= kMaxBlobs, "n_blobs=%d outside [0, %d]", f->n_blobs, kMaxBlobs);
    NACC_CHECK_ARG(f->n_blobs == 0 || (f->mu && f->std && f->peak && (!rgb || f->rgb)),
                   "field arrays are NULL");
    return NACC_OK;
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" int nacc_harness_field(const float* rays_o, const float* rays_d, const int32_t* ray_indices,
                                  const float* t_starts, const float* t_ends,
                                  const int64_t* n_samples, const nacc_blob_field* field,
                                  float* sigmas, float* rgbs, void* stream) {
    clear_error();
    int rc = check_field(field, true);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(rays_o && rays_d && ray_indices && t_starts && t_ends && n_samples && sigmas && rgbs,
                   "a pointer argument is NULL");
    size_t shm = sizeof(BlobS) * (size_t)field->n_blobs;
    if (shm > 48 * 1024)
        NACC_CUDA_TRY(cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_field<<<sm_count() * 8, 256, shm, as_stream(stream)>>>(rays_o, rays_d, ray_indices, t_starts,
                                                             t_ends, n_samples, *field, sigmas, rgbs);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_harness_field_points(int64_t n, const float* xyz, const nacc_blob_field* field,
                                         float* sigma, void* stream) {
    clear_error();
    int rc = check_field(field, false);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(n >= 0, "n < 0");
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(xyz && sigma, "xyz / sigma is NULL");
    size_t shm = sizeof(BlobS) * (size_t)field->n_blobs;
    if (shm > 48 * 1024)
        NACC_CUDA_TRY(cudaFuncSetAttribute(k_field_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_field_points<<<blocks, 256, shm, as_stream(stream)>>>(xyz, n, *field, sigma);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_harness_l2_loss(int64_t n, const float* rgb, const float* target, float* g_rgb,
                                    float* loss, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0, "n < 0");
    NACC_CHECK_ARG(loss != nullptr, "loss is NULL");
    cudaStream_t st = as_stream(stream);
    NACC_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(rgb && target && g_rgb, "rgb / target / g_rgb is NULL");
    const int64_t m = 3 * n;
    int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)sm_count() * 8);
    k_l2<<<blocks, 256, 0, st>>>(rgb, target, m, 1.0f / (float)m, g_rgb, loss);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
