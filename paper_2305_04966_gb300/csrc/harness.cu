// harness.cu -- stand-ins for the user's radiance field and loss
// (nacc_harness.h).  Not the method: they let a full sampling -> rendering
// -> gradient step run on synthetic Gaussian-blob scenes.
#include "nacc_internal.cuh"

namespace nacc {
namespace {

__device__ __forceinline__ float ex2_approx(float a) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

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

// The blob field at the sample midpoints of a packed set, one warp per ray
// (persistent grid).  On the ray x(t) = o + t d blob b contributes peak_b
// 2^(A_b (t - t*_b)^2 + C_b) with A_b = c_b |d|^2, C_b = c_b p_b^2, c_b the
// log2-scaled coefficient, t*_b the closest approach and p_b the distance
// there (cross product, no cancellation): set up once per ray by the lanes,
// then each lane evaluates four consecutive samples per chunk (128-bit
// loads of t0, t1; 128-bit stores of sigma and rgb for groups inside the
// ray, scalar accesses at its ends).
//
// Fields of more than kCullAbove blobs keep, per ray, only the blobs whose
// integral along the whole ray line is above kCullEps (bound: peak 2^C_b
// sqrt(2 pi) sd / |d|); each dropped blob changes sigma by at most
// peak 2^C_b <= kCullEps |d| / (sqrt(2 pi) sd) at any point of the ray.
// Fields of at least kGroupAbove blobs first list, per group of kFieldGroup
// consecutive rays, the blobs any of them may keep (field_group_candidates),
// so each ray's table is built from that list: the same tables, in the same
// order, for less work.
constexpr int kFieldWarps = 8;
constexpr int kFieldRayBlobs = 256;  // per-warp shared table limit
constexpr int kCullAbove = 16;
constexpr float kCullEps = 1e-7f;

// t0, t1 of positions p..p+3 of the ray's range [s, e) (zero outside it);
// true if all four lie inside (one 128-bit load per plane).
__device__ __forceinline__ bool load_t4(const float* __restrict__ t0, const float* __restrict__ t1, long long p,
                                        long long s, long long e, float ta[4], float tb[4]) {
    const bool whole = p >= s && p + 4 <= e;
    if (whole) {
        const float4 u = __ldcs(reinterpret_cast<const float4*>(t0 + p));
        const float4 w = __ldcs(reinterpret_cast<const float4*>(t1 + p));
        ta[0] = u.x, ta[1] = u.y, ta[2] = u.z, ta[3] = u.w;
        tb[0] = w.x, tb[1] = w.y, tb[2] = w.z, tb[3] = w.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = p + j >= s && p + j < e;
            ta[j] = in ? t0[p + j] : 0.0f;
            tb[j] = in ? t1[p + j] : 0.0f;
        }
    }
    return whole;
}

constexpr int kFieldGroup = 8;    // consecutive rays sharing one candidate list
constexpr int kGroupAbove = 128;  // fields of at least this many blobs use the lists

// The blobs some ray of the group rbase .. rbase+kFieldGroup-1 may keep in its table
// (integral bound along the line above kCullEps), as an ascending list in
// cand; returns its length, or -1 (every blob) when a ray of the group has a
// zero direction.  With c = the first ray's line (origin o_c, unit direction
// u_c), delta the largest distance of a group ray's origin from o_c and s the
// largest sine of a group direction's angle to u_c, blob b lies at least
// p_lo = p_c - delta - (|mu - o_c| + delta) s from every group ray's line
// (the closest point of line i lies within |mu - o_i| of o_i), so each ray's
// bound is at most peak 2^(coef p_lo^2) sqrt(2 pi) sd / min |d|; a blob whose
// bound is below kCullEps / 4 (slack for the FP32 distances and exponential)
// is kept by none of them.
__device__ int field_group_candidates(const BlobS* sb, int nb, const float* __restrict__ ro,
                                      const float* __restrict__ rd, int64_t rbase, int64_t n, uint16_t* cand,
                                      int lane) {
    const int64_t r = rbase + lane;
    const bool lv = lane < kFieldGroup && r < n;
    float oi[3] = {0.0f, 0.0f, 0.0f}, di[3] = {0.0f, 0.0f, 0.0f};
    if (lv) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            oi[a] = __ldg(ro + 3 * r + a);
            di[a] = __ldg(rd + 3 * r + a);
        }
    }
    float oc[3], dc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        oc[a] = __shfl_sync(0xffffffffu, oi[a], 0);
        dc[a] = __shfl_sync(0xffffffffu, di[a], 0);
    }
    const float lc = sqrtf(fmaf(dc[2], dc[2], fmaf(dc[1], dc[1], dc[0] * dc[0])));
    const float li = sqrtf(fmaf(di[2], di[2], fmaf(di[1], di[1], di[0] * di[0])));
    const bool bad = lv && !(li > 0.0f && li < 1e30f);
    if (__any_sync(0xffffffffu, bad) || !(lc > 0.0f && lc < 1e30f)) return -1;
    float sn = 0.0f, dl = 0.0f, il = 0.0f;
    if (lv) {
        const float cx = fmaf(di[1], dc[2], -di[2] * dc[1]), cy = fmaf(di[2], dc[0], -di[0] * dc[2]),
                    cz = fmaf(di[0], dc[1], -di[1] * dc[0]);
        sn = sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx))) / (li * lc) * 1.0001f + 1e-6f;
        const float e0 = oi[0] - oc[0], e1 = oi[1] - oc[1], e2 = oi[2] - oc[2];
        dl = sqrtf(fmaf(e2, e2, fmaf(e1, e1, e0 * e0))) * 1.0001f;
        il = 1.0001f / li;
    }
    float s_max = sn, delta = dl, ilen = il;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        s_max = fmaxf(s_max, __shfl_xor_sync(0xffffffffu, s_max, o2));
        delta = fmaxf(delta, __shfl_xor_sync(0xffffffffu, delta, o2));
        ilen = fmaxf(ilen, __shfl_xor_sync(0xffffffffu, ilen, o2));
    }
    if (!(s_max < 1e30f && delta < 1e30f && ilen < 1e30f)) return -1;
    const float u0 = dc[0] / lc, u1 = dc[1] / lc, u2 = dc[2] / lc;
    const float lim = __log2f(kCullEps) - 2.0f;
    int nc = 0;
    for (int b0 = 0; b0 < nb; b0 += 32) {
        const int b = b0 + lane;
        bool keep = false;
        if (b < nb) {
            const BlobS v = sb[b];
            keep = v.peak > 0.0f;
            if (keep) {
                const float m0 = v.mx - oc[0], m1 = v.my - oc[1], m2 = v.mz - oc[2];
                const float cx = fmaf(m1, u2, -m2 * u1), cy = fmaf(m2, u0, -m0 * u2), cz = fmaf(m0, u1, -m1 * u0);
                const float pc = sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)));
                const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
                const float plo = fmaxf(0.0f, pc - delta - (mn + delta) * s_max - 1e-4f * (mn + delta + 1.0f));
                const float sd = sqrtf(-0.72134752f / v.coef);  // coef = -log2(e) / (2 sd^2)
                const float lb = __log2f(v.peak * 2.5066283f * sd * ilen) + v.coef * (plo * plo) * 0.9998f;
                keep = !(lb < lim);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) cand[nc + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)b;
        nc += __popc(bal);
    }
    return nc;
}

// One ray of k_field_rays: its table {A_b, t*_b, C_b + log2 peak_b, b} from the blobs
// cand[0 .. nc) (ascending; NULL or !kGroups: blobs 0 .. nc-1), culled per
// ray when kCull, then its samples, four consecutive ones per lane per chunk
// of 128.
template <bool kCull, bool kGroups>
__device__ __forceinline__ void field_ray(int64_t r, const uint16_t* cand, int nc, const float* __restrict__ o,
                                          const float* __restrict__ d, const int64_t* __restrict__ off,
                                          const float* __restrict__ t0, const float* __restrict__ t1,
                                          const BlobS* sb, int nb, float4* q, float* __restrict__ sig,
                                          float* __restrict__ rgb, int lane) {
        const long long s = off[r], e = off[r + 1];
        if (e <= s) return;
        // the first chunk's loads are in flight during the table set-up; each
        // chunk's compute overlaps the next chunk's loads
        long long p = (s & ~3ll) + 4 * lane;
        float ta[4], tb[4];
        bool whole = p < e ? load_t4(t0, t1, p, s, e, ta, tb) : false;
        const float ox = __ldg(o + 3 * r), oy = __ldg(o + 3 * r + 1), oz = __ldg(o + 3 * r + 2);
        const float dx = __ldg(d + 3 * r), dy = __ldg(d + 3 * r + 1), dz = __ldg(d + 3 * r + 2);
        const float dd = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
        const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
        // table entries {A_b, t*_b, C_b, b}, compacted in blob order
        int nt = 0;
        for (int i0 = 0; i0 < nc; i0 += 32) {
            const int b = kGroups ? (i0 + lane < nc ? (cand ? (int)cand[i0 + lane] : i0 + lane) : nb) : i0 + lane;
            bool keep = false;
            float4 ent;
            if (b < nb) {
                const BlobS v = sb[b];
                const float m0 = v.mx - ox, m1 = v.my - oy, m2 = v.mz - oz;
                float ts, pp;
                if (dd > 0.0f) {
                    const float cx = fmaf(m1, dz, -m2 * dy), cy = fmaf(m2, dx, -m0 * dz),
                                cz = fmaf(m0, dy, -m1 * dx);
                    ts = fmaf(m2, dz, fmaf(m1, dy, m0 * dx)) * idd;
                    pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
                } else {
                    ts = 0.0f;
                    pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
                }
                // the peak rides in the exponent: density 2^(A (t - t*)^2 + C + log2 peak)
                ent = make_float4(v.coef * dd, ts, fmaf(v.coef, pp, __log2f(v.peak)), __int_as_float(b));
                keep = true;
                if (nb > kCullAbove) {
                    const float sd = sqrtf(-0.72134752f / v.coef);  // coef = -log2(e) / (2 sd^2)
                    const float peak_line = ex2_approx(ent.z);
                    const float bound = dd > 0.0f ? peak_line * 2.5066283f * sd * ilen : peak_line * 1e30f;
                    keep = bound > kCullEps;
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) q[nt + __popc(bal & ((1u << lane) - 1u))] = ent;
            nt += __popc(bal);
        }
        __syncwarp();
        for (; p < e; p += 128) {
            float tm[4], sg[4] = {0.0f, 0.0f, 0.0f, 0.0f}, c[12] = {};
#pragma unroll
            for (int j = 0; j < 4; ++j) tm[j] = 0.5f * (ta[j] + tb[j]);
            const bool cur_whole = whole;
            if (p + 128 < e) whole = load_t4(t0, t1, p + 128, s, e, ta, tb);
            for (int i = 0; i < nt; ++i) {
                const float4 v = q[i];
                const BlobS& w = sb[__float_as_int(v.w)];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float u = tm[j] - v.y;
                    const float sj = ex2_approx(fmaf(v.x * u, u, v.z));
                    sg[j] += sj;
                    c[3 * j] = fmaf(sj, w.r, c[3 * j]);
                    c[3 * j + 1] = fmaf(sj, w.g, c[3 * j + 1]);
                    c[3 * j + 2] = fmaf(sj, w.b, c[3 * j + 2]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float inv = sg[j] > 0.0f ? __frcp_rn(sg[j]) : 0.0f;
                c[3 * j] *= inv;
                c[3 * j + 1] *= inv;
                c[3 * j + 2] *= inv;
            }
            if (cur_whole) {
                __stcs(reinterpret_cast<float4*>(sig + p), make_float4(sg[0], sg[1], sg[2], sg[3]));
                float4* q4 = reinterpret_cast<float4*>(rgb + 3 * p);
                __stcs(q4, make_float4(c[0], c[1], c[2], c[3]));
                __stcs(q4 + 1, make_float4(c[4], c[5], c[6], c[7]));
                __stcs(q4 + 2, make_float4(c[8], c[9], c[10], c[11]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (p + j >= s && p + j < e) {
                        sig[p + j] = sg[j];
                        rgb[3 * (p + j)] = c[3 * j];
                        rgb[3 * (p + j) + 1] = c[3 * j + 1];
                        rgb[3 * (p + j) + 2] = c[3 * j + 2];
                    }
                }
            }
        }
        __syncwarp();  // the next ray's set-up rewrites q
}

// kCull: fields of more than kCullAbove blobs (tables culled per ray); kGroups:
// of at least kGroupAbove blobs (candidate lists per group of rays first)
template <bool kCull, bool kGroups>
__global__ void __launch_bounds__(kFieldWarps * 32, 4)
    k_field_rays(const float* __restrict__ o, const float* __restrict__ d, int64_t n_rays,
                 const int64_t* __restrict__ off, const float* __restrict__ t0, const float* __restrict__ t1,
                 nacc_blob_field f, float* __restrict__ sig, float* __restrict__ rgb) {
    extern __shared__ float4 s_dyn[];
    const int nb = f.n_blobs;
    BlobS* sb = reinterpret_cast<BlobS*>(s_dyn + kFieldWarps * nb);
    stage_blobs(sb, f, true);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sb[b].coef *= 1.4426950408889634f;  // log2 e
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* q = s_dyn + wid * nb;
    const int64_t warps = (int64_t)gridDim.x * kFieldWarps;

    if (kGroups) {
        // groups of kFieldGroup consecutive rays: the blobs none of the group's
        // rays can keep are left out of every table before the rays are set up
        uint16_t* cand = reinterpret_cast<uint16_t*>(sb + nb) + (size_t)wid * nb;
        const int64_t n_groups = (n_rays + kFieldGroup - 1) / kFieldGroup;
        for (int64_t grp = (int64_t)blockIdx.x * kFieldWarps + wid; grp < n_groups; grp += warps) {
            const int64_t rbase = grp * kFieldGroup;
            const int nc = field_group_candidates(sb, nb, o, d, rbase, n_rays, cand, lane);
            __syncwarp();
            for (int i = 0; i < kFieldGroup && rbase + i < n_rays; ++i)
                field_ray<kCull, true>(rbase + i, nc >= 0 ? cand : nullptr, nc >= 0 ? nc : nb, o, d, off, t0, t1, sb,
                                       nb, q, sig, rgb, lane);
            __syncwarp();  // the next group rewrites the candidate list
        }
    } else {
        for (int64_t r = (int64_t)blockIdx.x * kFieldWarps + wid; r < n_rays; r += warps)
            field_ray<kCull, false>(r, nullptr, nb, o, d, off, t0, t1, sb, nb, q, sig, rgb, lane);
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

extern "C" int nacc_harness_field_rays(const float* rays_o, const float* rays_d, int64_t n_rays,
                                       const int64_t* offsets, const float* t_starts, const float* t_ends,
                                       const nacc_blob_field* field, float* sigmas, float* rgbs, void* stream) {
    clear_error();
    int rc = check_field(field, true);
    if (rc != NACC_OK) return rc;
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(rays_o && rays_d && offsets && t_starts && t_ends && sigmas && rgbs, "a pointer argument is NULL");
    NACC_CHECK_ARG(field->n_blobs <= kFieldRayBlobs, "n_blobs=%d > %d (use nacc_harness_field)", field->n_blobs,
                   kFieldRayBlobs);
    auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    NACC_CHECK_ARG(a16(t_starts) && a16(t_ends) && a16(sigmas) && a16(rgbs),
                   "t_starts, t_ends, sigmas and rgbs must be 16-byte aligned");
    // per-warp tables, the staged blobs, per-warp candidate lists (culled fields)
    const size_t shm = (sizeof(float4) * kFieldWarps + sizeof(BlobS) + sizeof(uint16_t) * kFieldWarps) *
                       (size_t)field->n_blobs;
    const int nbl = field->n_blobs;
    const auto kern = nbl >= kGroupAbove ? k_field_rays<true, true>
                                         : (nbl > kCullAbove ? k_field_rays<true, false> : k_field_rays<false, false>);
    if (shm > 48 * 1024)
        NACC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    int per_sm = 1;
    NACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFieldWarps * 32, shm));
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = min64((int64_t)per_sm * sm_count(), (n_rays + kFieldWarps - 1) / kFieldWarps);
    kern<<<(unsigned)grid, kFieldWarps * 32, shm, as_stream(stream)>>>(rays_o, rays_d, n_rays, offsets, t_starts,
                                                                      t_ends, *field, sigmas, rgbs);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

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
