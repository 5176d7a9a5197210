// march.cu -- occupancy-grid lattice marching into packed samples
// (nacc_march_grid): count pass, block-offset scan, fill pass.
//
// Table 1 "Spatial Skipping" (occupied <=> bit set), Sec. 3.1 (skip empty
// space), Sec. 4.2 "Sample as Interval" / "Packed Tensor" / "No Gradient
// Filtering", Appendix B (step, resolution, threshold).
//
// One thread marches one ray.  The lattice arithmetic (t0, t1, midpoint,
// position, level, cell) uses explicitly rounded FP32 intrinsics so that the
// occupancy test of every lattice point is bit-identical to the dense-march
// definition.  Empty cells are skipped with a DDA step that is conservative
// by construction:
//   * along each axis the computed cell index is monotone in k (every
//     rounding step is monotone), so inside a cell it can only change when
//     the exact position crosses a face;
//   * the skip target is the exit of the cell shrunk by 1/256 cell per face
//     (and the entry of the next finer level's box grown by the same
//     margin), far larger than the ~1e-5-cell error of the rounded position;
//   * the resume index floor((t_exit - t_near)/dt) - 1 keeps 1.5 steps of
//     slack on top.
// So every skipped lattice point provably lies in the same empty cell and
// the emitted set equals the dense march's.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kMarchThreads = 128;
constexpr float kSkipMargin = 1.0f / 256.0f;  // cells

struct MarchArgs {
    GridGeom g;
    const float* o;
    const float* d;
    int64_t n;
    float step;
    int max_steps;
    float t_min, t_max;
    float thr;  // optical-depth threshold (+inf: no early stop)
    nacc_blob_field field;
};

// Slab clip against the outermost level's box (same comparisons as the
// definition: ternary min/max, NaN never tightens the interval).
__device__ __forceinline__ bool clip_ray(const Level& outer, const float o[3], const float d[3],
                                         float t_min, float t_max, float& tn, float& tf) {
    float near = t_min, far = t_max;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < outer.lmin[a] || o[a] > outer.lmax[a]) return false;
            continue;
        }
        float inv = __fdiv_rn(1.0f, d[a]);
        float ta = __fmul_rn(__fsub_rn(outer.lmin[a], o[a]), inv);
        float tb = __fmul_rn(__fsub_rn(outer.lmax[a], o[a]), inv);
        float lo = (ta < tb) ? ta : tb;
        float hi = (ta < tb) ? tb : ta;
        if (lo > near) near = lo;
        if (hi < far) far = hi;
    }
    tn = near;
    tf = far;
    return near < far;
}

// March one ray.  kCount: only count (and report the stop index); otherwise
// write at out[base .. base+limit).  kField: early termination with the
// staged blob field.  Returns the number of samples.
template <bool kCount, bool kField>
__device__ int march_ray(const MarchArgs& A, const BlobS* blobs, int64_t r, int kend, int limit,
                         int64_t base, int32_t* ray_idx, float* t0s, float* t1s, int& kstop) {
    float o[3], d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o[a] = __ldg(&A.o[3 * r + a]);
        d[a] = __ldg(&A.d[3 * r + a]);
    }
    kstop = kend;
    const int L = A.g.n_levels;
    const int res = A.g.res;
    float tn, tf;
    if (!clip_ray(A.g.lv[L - 1], o, d, A.t_min, A.t_max, tn, tf)) return 0;
    float invd[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) invd[a] = 1.0f / d[a];
    const uint64_t r3 = (uint64_t)res * res * res;
    float tau = 0.0f;
    int n = 0;
    int k = 0;
    while (k < kend) {
        float t0 = __fadd_rn(tn, __fmul_rn((float)k, A.step));
        if (!(t0 < tf)) break;
        float t1 = __fadd_rn(t0, A.step);
        float tm = __fmul_rn(__fadd_rn(t0, t1), 0.5f);
        float x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(d[a], tm));
        int l = 0;
        for (; l < L; ++l) {
            const Level& lv = A.g.lv[l];
            if (x[0] >= lv.lmin[0] && x[0] <= lv.lmax[0] && x[1] >= lv.lmin[1] &&
                x[1] <= lv.lmax[1] && x[2] >= lv.lmin[2] && x[2] <= lv.lmax[2])
                break;
        }
        if (l == L) {  // outside every level (only possible at the ray's ends)
            ++k;
            continue;
        }
        const Level& lv = A.g.lv[l];
        int ic[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float u = __fmul_rn(__fsub_rn(x[a], lv.lmin[a]), lv.scale[a]);
            int c = (int)floorf(u);
            ic[a] = c < 0 ? 0 : (c > res - 1 ? res - 1 : c);
        }
        uint64_t idx = (uint64_t)l * r3 + ((uint64_t)ic[0] * res + ic[1]) * res + ic[2];
        bool occ = (__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u;
        if (occ) {
            if (kField) {
                if (tau > A.thr) {
                    kstop = k;
                    return n;
                }
            }
            if (!kCount) {
                if (n >= limit) return n;
                if (ray_idx) ray_idx[base + n] = (int32_t)r;
                t0s[base + n] = t0;
                t1s[base + n] = t1;
            }
            ++n;
            if (kField) {
                float s = blob_sigma(blobs, A.field.n_blobs, x[0], x[1], x[2]);
                tau = __fadd_rn(tau, __fmul_rn(s, __fsub_rn(t1, t0)));
            }
            ++k;
        } else {
            // Conservative exit of the empty cell (shrunk by kSkipMargin).
            float ts = INFINITY;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (d[a] > 0.0f) {
                    float face = lv.lmin[a] + ((float)ic[a] + (1.0f - kSkipMargin)) * lv.width[a];
                    ts = fminf(ts, (face - o[a]) * invd[a]);
                } else if (d[a] < 0.0f) {
                    float face = lv.lmin[a] + ((float)ic[a] + kSkipMargin) * lv.width[a];
                    ts = fminf(ts, (face - o[a]) * invd[a]);
                }
            }
            if (l > 0) {  // do not skip into the next finer level's (grown) box
                const Level& fl = A.g.lv[l - 1];
                float tin = -INFINITY, tout = INFINITY;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float m = kSkipMargin * lv.width[a];
                    float lo = fl.lmin[a] - m, hi = fl.lmax[a] + m;
                    if (d[a] == 0.0f) {
                        if (o[a] < lo || o[a] > hi) {
                            tin = INFINITY;
                            tout = -INFINITY;
                        }
                    } else {
                        float ta = (lo - o[a]) * invd[a], tb = (hi - o[a]) * invd[a];
                        tin = fmaxf(tin, fminf(ta, tb));
                        tout = fminf(tout, fmaxf(ta, tb));
                    }
                }
                if (tin <= tout && tout > tm) ts = fminf(ts, tin);
            }
            int kn = k + 1;
            float q = (ts - tn) / A.step;
            if (q > (float)(k + 2)) kn = (q < (float)kend) ? (int)floorf(q) - 1 : kend;
            k = kn > k + 1 ? kn : k + 1;
        }
    }
    return n;
}

template <bool kField>
__global__ void __launch_bounds__(kMarchThreads)
    k_march_count(MarchArgs A, int32_t* __restrict__ counts, int32_t* __restrict__ kstops,
                  long long* __restrict__ block_sums) {
    extern __shared__ BlobS s_blobs[];
    if (kField) {
        stage_blobs(s_blobs, A.field, false);
        __syncthreads();
    }
    int64_t r = (int64_t)blockIdx.x * kMarchThreads + threadIdx.x;
    int cnt = 0;
    if (r < A.n) {
        int ks = 0;
        cnt = march_ray<true, kField>(A, s_blobs, r, A.max_steps, 0, 0, nullptr, nullptr, nullptr, ks);
        counts[r] = cnt;
        kstops[r] = ks;
    }
    // block total
    __shared__ int s_w[kMarchThreads / 32];
    int v = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < kMarchThreads / 32; ++w) t += s_w[w];
        block_sums[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of the per-block totals in place; writes the
// grand total to *n_samples and offsets[n_rays].
__global__ void __launch_bounds__(1024)
    k_scan_block_sums(long long* __restrict__ sums, int64_t nb, int64_t* __restrict__ off_last,
                      int64_t* __restrict__ n_samples) {
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        int64_t i = base + threadIdx.x;
        long long v = i < nb ? sums[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        long long carry = s_carry;
        long long incl = x + (wid > 0 ? s_w[wid - 1] : 0);
        if (i < nb) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) s_carry = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *off_last = s_carry;
        *n_samples = s_carry;
    }
}

__global__ void __launch_bounds__(kMarchThreads)
    k_march_fill(MarchArgs A, const int32_t* __restrict__ counts, const int32_t* __restrict__ kstops,
                 const long long* __restrict__ block_off, const int64_t* __restrict__ n_samples,
                 int64_t capacity, int64_t* __restrict__ offsets, int32_t* __restrict__ ray_idx,
                 float* __restrict__ t0s, float* __restrict__ t1s) {
    int64_t r = (int64_t)blockIdx.x * kMarchThreads + threadIdx.x;
    int cnt = r < A.n ? counts[r] : 0;
    // block exclusive scan of counts
    __shared__ int s_w[kMarchThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < wid; ++w) wbase += s_w[w];
    long long off = block_off[blockIdx.x] + wbase + x - cnt;
    if (r < A.n) {
        offsets[r] = off;
        bool fits = *n_samples <= capacity;
        if (cnt > 0 && fits) {
            int ks;
            march_ray<false, false>(A, nullptr, r, kstops[r], cnt, off, ray_idx, t0s, t1s, ks);
        }
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_march_scratch_bytes(int64_t n_rays) {
    if (n_rays < 0) return 0;
    int64_t nb = (n_rays + kMarchThreads - 1) / kMarchThreads;
    return align256(4 * (size_t)n_rays) * 2 + align256(8 * (size_t)(nb > 0 ? nb : 1));
}

extern "C" int nacc_march_grid(const nacc_grid* grid, const float* rays_o, const float* rays_d,
                               int64_t n_rays, const nacc_march_params* params,
                               const nacc_blob_field* field, nacc_packed* out, void* scratch,
                               size_t scratch_bytes, void* stream) {
    clear_error();
    MarchArgs A;
    if (!make_geom(grid, &A.g, true)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(params != nullptr, "params is NULL");
    NACC_CHECK_ARG(out != nullptr, "out is NULL");
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range",
                   (long long)n_rays);
    NACC_CHECK_ARG(params->step > 0.0f && std::isfinite(params->step), "step must be finite and > 0");
    NACC_CHECK_ARG(params->max_steps >= 1 && params->max_steps <= (1 << 24),
                   "max_steps=%d outside [1, 2^24]", params->max_steps);
    NACC_CHECK_ARG(!std::isnan(params->t_min) && !std::isnan(params->t_max), "t_min/t_max is NaN");
    NACC_CHECK_ARG(out->offsets && out->n_samples, "out->offsets / out->n_samples is NULL");
    NACC_CHECK_ARG(out->capacity >= 0, "capacity < 0");
    NACC_CHECK_ARG(out->capacity == 0 || (out->t_starts && out->t_ends),
                   "out->t_starts / out->t_ends is NULL");
    NACC_CHECK_ARG(out->capacity < (int64_t(1) << 40), "capacity too large");
    bool with_field = field != nullptr && field->n_blobs > 0 && params->early_stop_eps > 0.0f;
    if (with_field) {
        NACC_CHECK_ARG(field->n_blobs <= kMaxBlobs, "n_blobs=%d > %d", field->n_blobs, kMaxBlobs);
        NACC_CHECK_ARG(field->mu && field->std && field->peak, "field mu/std/peak is NULL");
    }
    cudaStream_t st = as_stream(stream);
    if (n_rays == 0) {
        NACC_CUDA_TRY(cudaMemsetAsync(out->offsets, 0, sizeof(int64_t), st));
        NACC_CUDA_TRY(cudaMemsetAsync(out->n_samples, 0, sizeof(int64_t), st));
        return NACC_OK;
    }
    NACC_CHECK_ARG(rays_o && rays_d, "rays_o / rays_d is NULL");
    size_t need = nacc_march_scratch_bytes(n_rays);
    NACC_CHECK_ARG(scratch != nullptr && scratch_bytes >= need,
                   "scratch too small: %zu < %zu bytes", scratch_bytes, need);
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch not 256-byte aligned");

    A.o = rays_o;
    A.d = rays_d;
    A.n = n_rays;
    A.step = params->step;
    A.max_steps = params->max_steps;
    A.t_min = params->t_min;
    A.t_max = params->t_max;
    A.thr = with_field ? tau_threshold(params->early_stop_eps) : INFINITY;
    A.field = with_field ? *field : nacc_blob_field{0, nullptr, nullptr, nullptr, nullptr};

    char* sp = static_cast<char*>(scratch);
    int32_t* counts = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int32_t* kstops = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    long long* bsums = reinterpret_cast<long long*>(sp);

    int64_t nb = (n_rays + kMarchThreads - 1) / kMarchThreads;
    NACC_CHECK_ARG(nb < (int64_t(1) << 31), "too many rays for one launch");
    if (with_field) {
        size_t shm = sizeof(BlobS) * (size_t)A.field.n_blobs;
        if (shm > 48 * 1024)
            NACC_CUDA_TRY(cudaFuncSetAttribute(k_march_count<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        k_march_count<true><<<(unsigned)nb, kMarchThreads, shm, st>>>(A, counts, kstops, bsums);
    } else {
        k_march_count<false><<<(unsigned)nb, kMarchThreads, 0, st>>>(A, counts, kstops, bsums);
    }
    NACC_LAUNCH_CHECK();
    k_scan_block_sums<<<1, 1024, 0, st>>>(bsums, nb, out->offsets + n_rays, out->n_samples);
    NACC_LAUNCH_CHECK();
    k_march_fill<<<(unsigned)nb, kMarchThreads, 0, st>>>(A, counts, kstops, bsums, out->n_samples,
                                                          out->capacity, out->offsets,
                                                          out->ray_indices, out->t_starts,
                                                          out->t_ends);
    NACC_LAUNCH_CHECK();
    // Overflow is impossible when the capacity covers every lattice point.
    bool may_overflow = (double)out->capacity < (double)n_rays * (double)params->max_steps;
    if (may_overflow) {
        int64_t total = 0;
        NACC_CUDA_TRY(cudaMemcpyAsync(&total, out->n_samples, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, st));
        NACC_CUDA_TRY(cudaStreamSynchronize(st));
        if (total > out->capacity) {
            set_error("packed capacity %lld < %lld samples", (long long)out->capacity,
                      (long long)total);
            return NACC_ERR_CAPACITY;
        }
    }
    return NACC_OK;
}
