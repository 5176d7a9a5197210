// march_unbounded.cu -- lattice marching for unbounded scenes
// (nacc_march_unbounded): sampling in s-space and an occupancy grid over the
// contracted space.
//
// Sec. 3.2 "Handling Unbounded Scenes": a bijection Phi: s in [0, 1] ->
// t in [t_near, t_far] makes the samples coarser with distance; the lattice
// is uniform in s.  Phi is disparity-linear: 1/t = (1 - s)/t_near + s/t_far.
// The grid is looked up at c(x), the L-infinity contraction of the sample's
// midpoint into [-2, 2]^3.  Every lattice point is tested (the contraction
// mixes the axes, so the per-axis monotonicity behind the bounded march's
// cell runs does not hold); the early stop is the bounded march's rule with
// the field at the uncontracted point.
//
// Passes: a table of t_k and of the midpoints; the count (one thread per
// ray, every lattice point, 4 grid words in flight, runs of consecutive
// points recorded); with a field, the early stop (one warp per ray over its
// occupied points, 32 at a time); the scan of the block totals; the fill
// (recorded runs expanded by the warp, coalesced stores).  The early-stop
// density of a ray keeps only the blobs whose integral along the whole ray
// line is above 1e-7 (a bound on everything dropped: at most 1e-7 per blob
// of optical depth), in the warp's shared table of the closed form
// peak_b 2^(A_b (t - t*_b)^2 + C_b); a ray with more than kStopTable such
// blobs sums every blob directly.
#include <algorithm>

#include "early_stop.cuh"
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kThreads = 128;  // rays per block (4 warps)
constexpr int kWarps = kThreads / 32;
constexpr int kStopTable = 256;  // early-stop table entries per ray (one warp's shared table)
constexpr int kRunSlots = 16;  // recorded runs of consecutive lattice points per ray
constexpr int kBatch = 4;      // lattice points whose grid words are loaded together
constexpr float kCullEps = 1e-7f;
constexpr float kMaxContracted = 1.99999988f;  // largest float below 2
constexpr int kChunk = 32;      // lattice points whose contracted box is tested for emptiness together
constexpr int kLogF = 2, kLogC = 4;  // "any cell occupied" summaries over 4^3 and 16^3 cells
constexpr size_t any_bytes(int log) {  // one summary bitfield, sized for 8 levels of 1024^3 cells
    return size_t(NACC_MAX_LEVELS) * (size_t(1024) >> log) * (size_t(1024) >> log) * (size_t(1024) >> log) / 8;
}

struct UArgs {
    GridGeom g;
    const float* o;
    const float* d;
    const float* tt;  // t_k = Phi(k / K), k = 0..K
    const float* tm;  // (t_k + t_k+1) * 0.5, k = 0..K-1
    const uint32_t* f_any;  // bit set iff any cell of the 4^3 block is occupied (NULL: no culling)
    const uint32_t* c_any;  // the same over 16^3 blocks
    int nbf, nbc;           // blocks per axis
    int64_t n;
    int K;
    float thr;
    int exact_all;  // every early-stop decision on the exact path (validation)
    nacc_blob_field field;
};

__device__ __forceinline__ float ex2_approx(float a) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

__device__ __forceinline__ float phi(int k, int K, float inv_tn, float inv_tf) {
    const float s = __fdiv_rn((float)k, (float)K);
    return __fdiv_rn(1.0f, __fadd_rn(__fmul_rn(inv_tn, __fsub_rn(1.0f, s)), __fmul_rn(inv_tf, s)));
}

// t_k = 1 / (a (1 - s) + b s) with a = 1/t_near, b = 1/t_far, s = k / K, each
// operation rounded, and the midpoints (t_k + t_k+1) * 0.5.
__global__ void __launch_bounds__(256) k_unb_table(int K, float inv_tn, float inv_tf, float* __restrict__ tt,
                                                   float* __restrict__ tm) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
        const float t0 = phi(k, K, inv_tn, inv_tf);
        tt[k] = t0;
        if (k < K) tm[k] = __fmul_rn(__fadd_rn(t0, phi(k + 1, K, inv_tn, inv_tf)), 0.5f);
    }
}

// Flat cell index of c(x), x = o + d tm on the ray, in the finest level whose
// box holds it; -1 (all ones for unsigned I) outside every level.  I is
// uint32_t when every cell index fits.
__device__ __forceinline__ bool in_level(const Level& lv, const float c[3]) {
    return c[0] >= lv.lmin[0] && c[0] <= lv.lmax[0] && c[1] >= lv.lmin[1] && c[1] <= lv.lmax[1] &&
           c[2] >= lv.lmin[2] && c[2] <= lv.lmax[2];
}

// `hint`: a level to try first (the level of a nearby point); taken only
// if the point lies in it and not in the next finer one -- the levels'
// boxes are nested, so that is the finest level holding it.  The level
// found (or L) goes to `lvl`.
template <typename I>
__device__ __forceinline__ I cell_index(const UArgs& A, const float o[3], const float d[3], float tm, int hint,
                                        int& lvl) {
    float c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = __fadd_rn(o[a], __fmul_rn(d[a], tm));
    const float m = fmaxf(fmaxf(fabsf(c[0]), fabsf(c[1])), fabsf(c[2]));
    if (m > 1.0f) {  // c = x (2 - 1/m) / m; the reciprocal correctly rounded, as 1.0f / m
        const float inv = __frcp_rn(m);
        const float g = __fmul_rn(__fsub_rn(2.0f, inv), inv);
#pragma unroll
        for (int a = 0; a < 3; ++a) c[a] = __fmul_rn(c[a], g);
    }
    const int L = A.g.n_levels;
    int l;
    if (in_level(A.g.lv[hint], c) && (hint == 0 || !in_level(A.g.lv[hint - 1], c))) {
        l = hint;
    } else {
        for (l = 0; l < L; ++l)
            if (in_level(A.g.lv[l], c)) break;
    }
    lvl = l;
    if (l == L) return (I)-1;
    const Level& lv = A.g.lv[l];
    const I res = (I)A.g.res;
    I ic[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int q = (int)floorf(__fmul_rn(__fsub_rn(c[a], lv.lmin[a]), lv.scale[a]));
        ic[a] = (I)(q < 0 ? 0 : (q > A.g.res - 1 ? A.g.res - 1 : q));
    }
    return (I)l * res * res * res + (ic[0] * res + ic[1]) * res + ic[2];
}

// Occupancy of lattice points kb..kb+kBatch-1 (bit j set = point kb+j
// occupied; points >= K are not); t[0..kBatch] receives t_kb..t_(kb+kBatch).
template <typename I>
__device__ __forceinline__ unsigned batch_mask(const UArgs& A, const float o[3], const float d[3], int kb,
                                               float t[kBatch + 1], int& hint) {
#pragma unroll
    for (int j = 0; j <= kBatch; ++j) t[j] = __ldg(A.tt + min(kb + j, A.K));
    I idx[kBatch];
    int lv[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        lv[j] = hint;
        idx[j] = kb + j < A.K ? cell_index<I>(A, o, d, __ldg(A.tm + kb + j), hint, lv[j]) : (I)-1;
    }
    // the next batch starts from the level of this batch's last point inside the grid
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
        if (lv[j] < A.g.n_levels) hint = lv[j];
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
        const uint32_t w = idx[j] != (I)-1 ? __ldg(&A.g.bits[idx[j] >> 5]) : 0u;
        m |= ((w >> (idx[j] & 31)) & 1u) << j;
    }
    return m;
}

// Runs of consecutive emitted points: merged while they continue one
// another; up to kRunSlots stored as {first k, count}; n = -1 on overflow.
struct RunRec {
    int2* slots;
    int n;
    int k0, k1;
};

__device__ __forceinline__ void rec_point(RunRec& q, int k) {
    if (q.k1 == k) {
        q.k1 = k + 1;
        return;
    }
    if (q.k1 > q.k0 && q.n >= 0) {
        if (q.n < kRunSlots)
            q.slots[q.n++] = make_int2(q.k0, q.k1 - q.k0);
        else
            q.n = -1;
    }
    q.k0 = k;
    q.k1 = k + 1;
}

__device__ __forceinline__ void rec_flush(RunRec& q) {
    if (q.k1 > q.k0 && q.n >= 0) {
        if (q.n < kRunSlots)
            q.slots[q.n++] = make_int2(q.k0, q.k1 - q.k0);
        else
            q.n = -1;
    }
}

// Per-blob constants of the early-stop table, staged once per block:
// {mu_x, mu_y, mu_z, c} with c = -log2(e) / (2 std^2), and {log2 peak,
// sqrt(2 pi) std} (peak <= 0: log2 peak = -inf, never kept).
constexpr int kStageBlobs = 256;  // blobs staged in shared memory; more are read from global memory

__device__ __forceinline__ void blob_consts(const nacc_blob_field& f, int b, float4& m, float4& k) {
    const float sd = __ldg(f.std + b), pk = __ldg(f.peak + b);
    m = make_float4(__ldg(f.mu + 3 * b), __ldg(f.mu + 3 * b + 1), __ldg(f.mu + 3 * b + 2), -0.72134752f / (sd * sd));
    k = make_float4(pk > 0.0f ? __log2f(pk) : -INFINITY, 2.5066283f * sd, 1.0f / sd, sd);
}

// The longest lattice interval within 4 std of a blob's closest approach
// t*: the lattice's intervals grow with t (1/t falls by the same `dinv` =
// (1/t_near - 1/t_far) / K per step), so the interval holding t ends before
// 1 / (1/t - dinv) and is at most that squared times dinv; dt_max = t_far -
// t_near bounds every interval.  The intervals [t_k, t_k+1] of the table are
// contiguous (no overlap).
__device__ __forceinline__ float blob_interval(float ts, float sd, float ilen, float dinv, float dt_max) {
    const float t_hi = (fabsf(ts) + 4.0f * sd * ilen) * 1.0001f;
    // fast reciprocals (within 2 ulp) with margins that keep the result an upper bound
    const float den = __fdividef(1.0f, t_hi) * (1.0f - 1e-5f) - 2.0f * dinv;
    return den > 0.0f ? fminf(dt_max, dinv * __fdividef(1.0f, den * den) * 1.01f) : dt_max;
}

// The ray's early-stop table and depth bound (early_stop.cuh), built by the
// warp, lane b0 + lane handling blob b0 + lane: the per-ray closed form in
// FP32; the blobs whose integral along the whole ray line exceeds kCullEps
// (bound peak 2^C sqrt(2 pi) sd / |d|) are compacted in blob order into the
// table as {A_b, t*_b, C_b + log2 peak_b} (log2-scaled: density peak_b
// 2^(A_b (t - t*_b)^2 + C_b); blob index in tidx).  U bounds the
// definition's depth at every sample (every blob's weight, the closed
// form's own FP32 rounding included); e_out is the error bound's share of
// the blobs left out (their whole weight).  Returns the number of kept blobs
// (the table holds the first kStopTable).  onorm =
// |o|, dnorm = |d|, cnt = the ray's samples, dinv and dt_max as in
// blob_interval.  The blobs visited are cand[0 .. n_cand) (ascending; NULL:
// all blobs): any other blob must give S = 0 on this ray (group_candidates).
__device__ int build_warp_table(const nacc_blob_field& f, const float4* sm, const float4* sk, const uint16_t* cand,
                                int n_cand, const float o[3], const float d[3], float onorm, float dnorm, float dinv,
                                float dt_max, int cnt, float4* tab, uint16_t* tidx, float& U, float& e_out,
                                int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
    int n = 0;
    float u = 0.0f, e = 0.0f;
    for (int i0 = 0; i0 < n_cand; i0 += 32) {
        const int b = i0 + lane < n_cand ? (cand ? (int)cand[i0 + lane] : i0 + lane) : f.n_blobs;
        bool keep = false;
        float4 ent = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (b < f.n_blobs) {
            float4 mc, kc;
            if (b < kStageBlobs) {
                mc = sm[b];
                kc = sk[b];
            } else {
                blob_consts(f, b, mc, kc);
            }
            const float m0 = mc.x - o[0], m1 = mc.y - o[1], m2 = mc.z - o[2];
            float ts, pp;
            if (dd > 0.0f) {
                const float cx = fmaf(m1, d[2], -m2 * d[1]), cy = fmaf(m2, d[0], -m0 * d[2]),
                            cz = fmaf(m0, d[1], -m1 * d[0]);
                ts = fmaf(m2, d[2], fmaf(m1, d[1], m0 * d[0])) * idd;
                pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
            } else {
                ts = 0.0f;
                pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
            }
            const float C = fmaf(mc.w, pp, kc.x);
            const float S = ex2_approx(C);  // largest density on the line
            float I;                         // integral along the line
            if (dd > 0.0f) {
                I = S * kc.y * ilen;
                keep = I > kCullEps;
            } else {
                I = S * dt_max * (float)cnt;
                keep = true;
            }
            if (S > 0.0f) {
                // growth with the FP32 closed form's own error (within 11u |mu - o|) included
                const float sd = kc.w * 1.0001f;
                const float p = sqrtf(pp);
                const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
                const float dt_b = dd > 0.0f ? blob_interval(ts, sd, ilen, dinv, dt_max) : dt_max;
                const float W = blob_weight(
                    S, I, dt_b, dt_max, 0.0f,
                    blob_growth(p, kc.z, onorm + 2.5f * fabsf(ts) * dnorm + 16.0f * p + 12.0f * mn));
                u += W;
                if (!keep) e += W;
            }
            ent = make_float4(mc.w * dd, ts, C, 0.0f);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = n + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < kStopTable) {
            tab[pos] = ent;
            tidx[pos] = (uint16_t)b;
        }
        n += __popc(bal);
    }
    U = warp_sum(u);
    e_out = warp_sum(e);
    return n;
}

// Error bound of the kept blobs (early_stop.cuh), one lane per kept blob:
// t* and p^2 again by closest_approach, the table entry rewritten (when the
// table holds the nt kept blobs; otherwise every kept blob is bounded from
// its FP32 values, for the direct form).  Returns the whole-ray bound, and
// the relative one in eps.  Arguments as build_warp_table.
__device__ float refine_warp_table(const nacc_blob_field& f, const float4* sm, const float4* sk, int nt,
                                   const float o[3], const float d[3], float onorm, float dnorm, float dinv,
                                   float dt_max, int cnt, float4* tab, const uint16_t* tidx, float& eps, int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
    const bool have_tab = nt <= kStopTable;
    float e = 0.0f, em = 0.0f;
    for (int i = lane; i < (have_tab ? nt : f.n_blobs); i += 32) {
        const int b = have_tab ? tidx[i] : i;
        float4 mc, kc;
        if (b < kStageBlobs) {
            mc = sm[b];
            kc = sk[b];
        } else {
            blob_consts(f, b, mc, kc);
        }
        float ts, pp;
        if (dd > 0.0f) {
            const float mu[3] = {mc.x, mc.y, mc.z};
            closest_approach(mu, o, d, idd, ts, pp);
        } else {
            const float m0 = mc.x - o[0], m1 = mc.y - o[1], m2 = mc.z - o[2];
            ts = 0.0f;
            pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
        }
        const float C = fmaf(mc.w, pp, kc.x);
        const float S = ex2_approx(C);
        const float I = dd > 0.0f ? S * kc.y * ilen : S * dt_max * (float)cnt;
        if (!have_tab && !(I > kCullEps) && dd > 0.0f) continue;  // left out: counted whole in build_warp_table
        const float sd = kc.w * 1.0001f;
        const float dt_b = dd > 0.0f ? blob_interval(ts, sd, ilen, dinv, dt_max) : dt_max;
        const float p = sqrtf(pp);
        const float pos0 = onorm + 2.5f * fabsf(ts) * dnorm + 16.0f * p;
        const float gm1 = blob_growth(p, kc.z, pos0);
        e += blob_error(blob_weight(S, I, dt_b, dt_max, 0.0f, gm1), gm1, p * kc.z, f.n_blobs, true);
        em = fmaxf(em, blob_rel_error(kc.z, pos0, f.n_blobs));
        if (have_tab) tab[i] = make_float4(mc.w * dd, ts, C, 0.0f);
    }
    eps = warp_max(em);
    return warp_sum(e);
}

// The ascending list of the blobs that may be non-zero somewhere on the ray
// in the definition's arithmetic (early_stop.cuh, blob_may_count), built by
// the warp; returns its length.  pos_far = |o| + t_far |d|.
__device__ int build_exact_list(const nacc_blob_field& f, const float4* sm, const float4* sk, const float o[3],
                                const float d[3], float pos_far, uint16_t* ex_list, int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    int ne = 0;
    for (int b0 = 0; b0 < f.n_blobs; b0 += 32) {
        const int b = b0 + lane;
        bool in_ex = false;
        if (b < f.n_blobs) {
            float4 mc;
            float4 kc;
            if (b < kStageBlobs) {
                mc = sm[b];
                kc = sk[b];
            } else {
                blob_consts(f, b, mc, kc);
            }
            const float m0 = mc.x - o[0], m1 = mc.y - o[1], m2 = mc.z - o[2];
            float pp;
            if (dd > 0.0f) {
                const float cx = fmaf(m1, d[2], -m2 * d[1]), cy = fmaf(m2, d[0], -m0 * d[2]),
                            cz = fmaf(m0, d[1], -m1 * d[0]);
                pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
            } else {
                pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
            }
            // the FP32 distance is within 8u |mu - o| of exact: widen the margin by |mu - o|
            const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
            in_ex = blob_may_count(sqrtf(pp), kc.w * 1.0001f, pos_far + mn);
        }
        const unsigned bex = __ballot_sync(0xffffffffu, in_ex);
        if (in_ex) ex_list[ne + __popc(bex & ((1u << lane) - 1u))] = (uint16_t)b;
        ne += __popc(bex);
    }
    return ne;
}

__device__ __forceinline__ float sigma_table(const float4* tab, int nt, float tm) {
    float s = 0.0f;
    for (int b = 0; b < nt; ++b) {
        const float4 v = tab[b];
        const float u = tm - v.y;
        s += ex2_approx(fmaf(v.x * u, u, v.z));
    }
    return s;
}

// A table entry contributes to the optical depth of a group of points whose
// midpoints lie in [t_lo, t_hi] and whose intervals sum to at most span at
// most (its density at the point of [t_lo, t_hi] nearest its closest
// approach, the largest there) x span; entries below kGroupEps are left out
// for that group.  Over a ray of at most 2^24 points in groups of 64, with
// at most kStopTable entries, that moves the optical depth by at most
// 6.7e-3 (and by 4.1e-7 at 1,024 points): only decisions within that of
// the threshold.
constexpr float kGroupEps = 1e-10f;

// The table's density at two points, summing only the entries that the
// bound above keeps for the warp's group (each lane tests one entry, the
// warp takes the kept ones in table order); every lane of the warp calls
// it, `active` lanes get sums.
__device__ __forceinline__ void sigma_table2_group(const float4* tab, int nt, float t_lo, float t_hi, float span,
                                                   float tma, float tmb, float& sa, float& sb, bool active,
                                                   int lane) {
    float a = 0.0f, b = 0.0f;
    for (int e0 = 0; e0 < nt; e0 += 32) {
        bool on = false;
        if (e0 + lane < nt) {
            const float4 v = tab[e0 + lane];
            const float u = fminf(fmaxf(v.y, t_lo), t_hi) - v.y;
            on = ex2_approx(fmaf(v.x * u, u, v.z)) * span > kGroupEps;
        }
        unsigned m = __ballot_sync(0xffffffffu, on);
        if (!active) continue;
        while (m) {
            const float4 v = tab[e0 + __ffs(m) - 1];
            m &= m - 1;
            const float ua = tma - v.y, ub = tmb - v.y;
            a += ex2_approx(fmaf(v.x * ua, ua, v.z));
            b += ex2_approx(fmaf(v.x * ub, ub, v.z));
        }
    }
    sa = a;
    sb = b;
}

__device__ __forceinline__ float sigma_all(const nacc_blob_field& f, const float x[3]) {
    float s = 0.0f;
    for (int b = 0; b < f.n_blobs; ++b) {
        const float sd = __ldg(f.std + b);
        const float dx = x[0] - __ldg(f.mu + 3 * b), dy = x[1] - __ldg(f.mu + 3 * b + 1),
                    dz = x[2] - __ldg(f.mu + 3 * b + 2);
        s = fmaf(__ldg(f.peak + b), __expf(-fmaf(dz, dz, fmaf(dy, dy, dx * dx)) / (2.0f * sd * sd)), s);
    }
    return s;
}

// Any-occupied summaries: one bit per (1 << kLog)^3 block of cells of each
// level (partial blocks at the high edge), from the bits, and the coarse one
// from the fine one.
__global__ void __launch_bounds__(256) k_unb_fine_summary(GridGeom g, int nb, uint32_t* __restrict__ any) {
    constexpr int kB = 1 << kLogF;
    const uint64_t nblocks = (uint64_t)g.n_levels * nb * nb * nb;
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool occ = false;
    if (b < nblocks) {
        const int res = g.res;
        const uint64_t per_level = (uint64_t)nb * nb * nb;
        const int l = (int)(b / per_level);
        const uint32_t rem = (uint32_t)(b % per_level);
        const int bx = rem / (nb * nb), by = (rem / nb) % nb, bz = rem % nb;
        const uint64_t r3 = (uint64_t)res * res * res;
        for (int x = bx * kB; x < min(bx * kB + kB, res); ++x)
            for (int y = by * kB; y < min(by * kB + kB, res); ++y)
                for (int z = bz * kB; z < min(bz * kB + kB, res); ++z) {
                    const uint64_t i = (uint64_t)l * r3 + ((uint64_t)x * res + y) * res + z;
                    occ = occ || ((g.bits[i >> 5] >> (i & 31)) & 1u);
                }
    }
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && b < nblocks) any[b >> 5] = m;
}

__global__ void __launch_bounds__(256) k_unb_coarse_summary(int n_levels, int nbc, int nbf,
                                                            const uint32_t* __restrict__ f_any,
                                                            uint32_t* __restrict__ c_any) {
    constexpr int kR = 1 << (kLogC - kLogF);
    const uint64_t ncb = (uint64_t)n_levels * nbc * nbc * nbc;
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool occ = false;
    if (b < ncb) {
        const uint64_t per_level = (uint64_t)nbc * nbc * nbc;
        const int l = (int)(b / per_level);
        const uint32_t rem = (uint32_t)(b % per_level);
        const int bx = rem / (nbc * nbc), by = (rem / nbc) % nbc, bz = rem % nbc;
        for (int x = bx * kR; x < min(bx * kR + kR, nbf); ++x)
            for (int y = by * kR; y < min(by * kR + kR, nbf); ++y)
                for (int z = bz * kR; z < min(bz * kR + kR, nbf); ++z) {
                    const uint32_t f = (((uint32_t)l * nbf + x) * nbf + y) * nbf + z;
                    occ = occ || ((__ldg(&f_any[f >> 5]) >> (f & 31)) & 1u);
                }
    }
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if ((threadIdx.x & 31) == 0 && b < ncb) c_any[b >> 5] = m;
}

// True if every block of the summary (nb blocks per axis, 1 << log cells)
// covering cells [ilo, ihi] of level l is empty; false also when more than
// `cap` blocks would have to be read.
__device__ __forceinline__ bool blocks_empty(const uint32_t* any, int nb, int log, int l, const int ilo[3],
                                             const int ihi[3], int cap) {
    const int b0x = ilo[0] >> log, b1x = ihi[0] >> log, b0y = ilo[1] >> log, b1y = ihi[1] >> log,
              b0z = ilo[2] >> log, b1z = ihi[2] >> log;
    if ((b1x - b0x + 1) * (b1y - b0y + 1) * (b1z - b0z + 1) > cap) return false;
    for (int x = b0x; x <= b1x; ++x)
        for (int y = b0y; y <= b1y; ++y)
            for (int z = b0z; z <= b1z; ++z) {
                const uint32_t b = (((uint32_t)l * nb + x) * nb + y) * nb + z;
                if ((__ldg(&any[b >> 5]) >> (b & 31)) & 1u) return false;
            }
    return true;
}

// The contraction's scale factor as a function of the max-norm: 1 inside the
// unit cube, (2 - 1/m)/m beyond (continuous, non-increasing).
__device__ __forceinline__ float contract_scale(float m) { return m <= 1.0f ? 1.0f : (2.0f - 1.0f / m) / m; }

// True if no lattice point k0..k1 (midpoints tm_k0 <= tm_k <= tm_k1 on the
// ray) can lie in an occupied cell: the exact contracted segment is bounded
// per axis by interval products (x_a(t) is linear in t, the max-norm m(t) is
// bounded by its endpoint values above and by max_a min_t |x_a(t)| below,
// the scale factor is non-increasing in m), the box is grown by far more
// than the FP32 rounding of the computed points (1e-5 absolute + 1e-5
// relative), it must lie inside one level and clear of the next finer
// level's box, and every cell of that level within one cell of it must be
// empty.
__device__ bool chunk_empty(const UArgs& A, const float o[3], const float d[3], float ta, float tb) {
    float xlo[3], xhi[3], mlo = 0.0f, mhi = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xa = fmaf(d[a], ta, o[a]), xb = fmaf(d[a], tb, o[a]);
        const float e = 1e-5f * (fabsf(o[a]) + fabsf(d[a]) * fmaxf(fabsf(ta), fabsf(tb))) + 1e-5f;
        xlo[a] = fminf(xa, xb) - e;
        xhi[a] = fmaxf(xa, xb) + e;
        mhi = fmaxf(mhi, fmaxf(fabsf(xlo[a]), fabsf(xhi[a])));
        const float amin = (xlo[a] <= 0.0f && xhi[a] >= 0.0f) ? 0.0f : fminf(fabsf(xlo[a]), fabsf(xhi[a]));
        mlo = fmaxf(mlo, amin);
    }
    const float glo = contract_scale(mhi) * (1.0f - 1e-5f), ghi = contract_scale(mlo) * (1.0f + 1e-5f);
    float clo[3], chi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float p0 = xlo[a] * glo, p1 = xlo[a] * ghi, p2 = xhi[a] * glo, p3 = xhi[a] * ghi;
        clo[a] = fminf(fminf(p0, p1), fminf(p2, p3)) - 1e-5f;
        chi[a] = fmaxf(fmaxf(p0, p1), fmaxf(p2, p3)) + 1e-5f;
    }
    const int L = A.g.n_levels;
    int l = 0;
    for (; l < L; ++l) {
        const Level& lv = A.g.lv[l];
        if (clo[0] >= lv.lmin[0] && chi[0] <= lv.lmax[0] && clo[1] >= lv.lmin[1] && chi[1] <= lv.lmax[1] &&
            clo[2] >= lv.lmin[2] && chi[2] <= lv.lmax[2])
            break;
    }
    if (l == L) return false;
    if (l > 0) {  // the box must not reach the next finer level's box
        const Level& fl = A.g.lv[l - 1];
        if (chi[0] >= fl.lmin[0] && clo[0] <= fl.lmax[0] && chi[1] >= fl.lmin[1] && clo[1] <= fl.lmax[1] &&
            chi[2] >= fl.lmin[2] && clo[2] <= fl.lmax[2])
            return false;
    }
    const Level& lv = A.g.lv[l];
    const int res = A.g.res;
    int ilo[3], ihi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ilo[a] = max((int)floorf((clo[a] - lv.lmin[a]) * lv.scale[a]) - 1, 0);
        ihi[a] = min((int)floorf((chi[a] - lv.lmin[a]) * lv.scale[a]) + 1, res - 1);
    }
    return blocks_empty(A.c_any, A.nbc, kLogC, l, ilo, ihi, 8) ||
           blocks_empty(A.f_any, A.nbf, kLogF, l, ilo, ihi, 27);
}

// Count pass: per ray (one thread), the number of occupied lattice points
// and their runs; chunks of kChunk points whose contracted box is empty are
// skipped whole.
template <typename I>
__global__ void __launch_bounds__(kThreads) k_unb_count(UArgs A, int32_t* __restrict__ counts,
                                                        int32_t* __restrict__ kstops, int32_t* __restrict__ nruns,
                                                        int2* __restrict__ runs, long long* __restrict__ block_sums) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t r = (int64_t)blockIdx.x * kThreads + tid;
    int cnt = 0;
    if (r < A.n) {
        const float o[3] = {A.o[3 * r], A.o[3 * r + 1], A.o[3 * r + 2]};
        const float d[3] = {A.d[3 * r], A.d[3 * r + 1], A.d[3 * r + 2]};
        RunRec q{runs + r * kRunSlots, 0, -1, -1};
        int hint = 0;  // level of the previous batch's last point in the grid
        for (int kc = 0; kc < A.K; kc += kChunk) {
            const int ke = min(kc + kChunk, A.K);
            if (A.f_any && chunk_empty(A, o, d, __ldg(A.tm + kc), __ldg(A.tm + ke - 1))) continue;
            for (int kb = kc; kb < ke; kb += kBatch) {
                float t[kBatch + 1];
                const unsigned m = batch_mask<I>(A, o, d, kb, t, hint);
#pragma unroll
                for (int j = 0; j < kBatch; ++j) {
                    if (!((m >> j) & 1u)) continue;
                    rec_point(q, kb + j);
                    ++cnt;
                }
            }
        }
        rec_flush(q);
        counts[r] = cnt;
        kstops[r] = A.K;
        nruns[r] = q.n;
    }
    __shared__ int s_w[kWarps];
    int v = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[wid] = v;
    __syncthreads();
    if (tid == 0) {
        long long t = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) t += s_w[w];
        block_sums[blockIdx.x] = t;
    }
}

// sigma*dt at lattice point k of the ray in the definition's arithmetic
// (early_stop.cuh): t from the lattice table, the blob parameters from
// global memory, entries that are 0 over the whole chunk left out; 0 for
// lanes without a point (`valid` false).  Every lane of the warp calls it.
// The definition's per-blob constants (centre, coefficient -1/2 / std^2 as
// the definition rounds it, peak), staged once per CTA of the exact kernel.
struct UExact {
    float mx, my, mz, coef, peak;
};

__device__ __forceinline__ void stage_exact_blobs(UExact* eb, const nacc_blob_field& f) {
    for (int b = threadIdx.x; b < f.n_blobs; b += blockDim.x) {
        const float sd = __ldg(f.std + b);
        eb[b] = UExact{__ldg(f.mu + 3 * b), __ldg(f.mu + 3 * b + 1), __ldg(f.mu + 3 * b + 2),
                       __fdiv_rn(-0.5f, __fmul_rn(sd, sd)), __ldg(f.peak + b)};
    }
}

__device__ __forceinline__ float unb_exact_tau(const UArgs& A, const UExact* eb, const uint16_t* ex_list, int n_ex,
                                               const float o[3], const float d[3], int k, bool valid, float pos_far,
                                               int lane) {
    const int kk = valid ? k : 0;
    const float t0 = __ldg(A.tt + kk), t1 = __ldg(A.tt + kk + 1), tm = __ldg(A.tm + kk);
    float x[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(o[a], __fmul_rn(d[a], tm));
    const unsigned vm = __ballot_sync(0xffffffffu, valid);
    if (!vm) return 0.0f;
    const float t_lo = __shfl_sync(0xffffffffu, tm, __ffs(vm) - 1);
    const float t_hi = __shfl_sync(0xffffffffu, tm, 31 - __clz(vm));
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float s = exact_sigma_chunk(
        x, ex_list, n_ex,
        [eb](int b) {
            const UExact& v = eb[b];
            return ExactBlob{v.mx, v.my, v.mz, v.coef, v.peak};
        },
        o, d, dd, dd > 0.0f ? 1.0f / dd : 0.0f, t_lo, t_hi, pos_far, lane);
    return valid ? __fmul_rn(s, __fsub_rn(t1, t0)) : 0.0f;
}

// Occupancy of lattice point k (the lattice walk of rays whose runs overflowed).
template <typename I>
__device__ __forceinline__ bool unb_occupied(const UArgs& A, const float o[3], const float d[3], int k) {
    int lvl;
    const I idx = cell_index<I>(A, o, d, __ldg(A.tm + k), 0, lvl);
    return idx != (I)-1 && ((__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u);
}

// The exact path of the early stop (early_stop.cuh): the ray's occupied
// points in lattice order, 32 at a time (from the recorded runs, or by
// walking the lattice when the runs overflowed); each lane evaluates one
// point's sigma*dt in the definition's arithmetic into the warp's buffer
// `buf` (32 floats of shared memory), then lane 0 adds the terms in order
// one at a time -- the definition's own sum -- and finds the first point
// whose depth before it exceeds the threshold, which cuts the ray.  cut /
// kstop are left as given if the ray never stops.
template <typename I>
__device__ __forceinline__ void unb_stop_exact(const UArgs& A, const UExact* eb, const uint16_t* ex_list, int n_ex,
                                              const float o[3],
                                              const float d[3], int cnt, int nr, int2 run, float pos_far, int lane,
                                              float* buf, int& cut, int& kstop) {
    int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ex, o2);
        if (lane >= o2) ex += y;
    }
    ex -= run.y;
    const int kend = nr >= 0 ? cnt : A.K;  // positions (runs) or lattice indices (walk)
    float P = 0.0f;                       // the sequential sum (lane 0's)
    int seen = 0;
    for (int q0 = 0; q0 < kend && seen < cnt; q0 += 32) {
        const int q = q0 + lane;
        int k = 0;
        bool on;
        if (nr >= 0) {
            for (int j = 0; j < nr; ++j) {
                const int ej = __shfl_sync(0xffffffffu, ex, j);
                const int kj = __shfl_sync(0xffffffffu, run.x, j);
                if (q >= ej) k = kj + (q - ej);
            }
            on = q < cnt;
        } else {
            k = q;
            on = q < A.K && unb_occupied<I>(A, o, d, q);
        }
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (!m) continue;
        buf[lane] = unb_exact_tau(A, eb, ex_list, n_ex, o, d, k, on, pos_far, lane);
        __syncwarp();
        int jc = -1, sc = seen;
        if (lane == 0) {
            unsigned mm = m;
            while (mm && sc < cnt) {
                const int j = __ffs(mm) - 1;
                mm &= mm - 1;
                if (P > A.thr) {
                    jc = j;
                    break;
                }
                P = __fadd_rn(P, buf[j]);
                ++sc;
            }
        }
        jc = __shfl_sync(0xffffffffu, jc, 0);
        const int sc0 = __shfl_sync(0xffffffffu, sc, 0);
        const int kc = __shfl_sync(0xffffffffu, k, jc < 0 ? 0 : jc);
        __syncwarp();
        if (jc >= 0) {
            cut = sc0;
            kstop = kc;
            return;
        }
        seen = sc0;
    }
}

// The fast depth of one ray (early_stop.cuh): its occupied points in lattice
// order, 64 (runs) or 32 (lattice walk when the runs overflowed) at a time,
// each lane adding its points' sigma dt from the ray's table (nt entries; -1:
// none, every blob directly), a warp scan giving the optical depth before
// each point.  Returns 0 if no point's fast depth comes within the error
// bound rb of the threshold (no cut), 1 if the first one that does passes it
// by more than the bound (cut / kstop set there), 2 otherwise (undecided).
template <typename I>
__device__ __forceinline__ int unb_fast_cut(const UArgs& A, const float4* tab, int nt, const RayBound& rb,
                                            const float o[3], const float d[3], int cnt, int nr, int2 run, int lane,
                                            int& cut, int& kstop) {
    float Q = 0.0f;  // sum of the depths before the points visited
    float carry = 0.0f;
    if (nr >= 0) {
        int ex = run.y;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ex, o2);
            if (lane >= o2) ex += y;
        }
        ex -= run.y;
        // two consecutive points per lane (64 per pass): each table
        // entry is read once for both
        for (int p0 = 0; p0 < cnt; p0 += 64) {
            const int pa = p0 + 2 * lane, pb = pa + 1;
            int ka = 0, kb = 0;
            for (int j = 0; j < nr; ++j) {
                const int ej = __shfl_sync(0xffffffffu, ex, j);
                const int kj = __shfl_sync(0xffffffffu, run.x, j);
                if (pa >= ej) ka = kj + (pa - ej);
                if (pb >= ej) kb = kj + (pb - ej);
            }
            float taua = 0.0f, taub = 0.0f;
            const bool two = pb < cnt;
            const float a0 = __ldg(A.tt + ka), a1 = __ldg(A.tt + ka + 1);
            const float b0 = two ? __ldg(A.tt + kb) : a0, b1 = two ? __ldg(A.tt + kb + 1) : a1;
            const float tca = 0.5f * (a0 + a1), tcb = 0.5f * (b0 + b1);
            float sa = 0.0f, sb = 0.0f;
            if (nt > 0) {  // the group's midpoints span [first, last] (lattice order)
                const int last = min(cnt - p0, 64) - 1;
                const float t_lo = __shfl_sync(0xffffffffu, tca, 0);
                const float t_hi = __shfl_sync(0xffffffffu, (last & 1) ? tcb : tca, last >> 1);
                const float t_end = __shfl_sync(0xffffffffu, (last & 1) ? b1 : a1, last >> 1);
                const float span = t_end - __shfl_sync(0xffffffffu, a0, 0);
                sigma_table2_group(tab, nt, t_lo, t_hi, span, tca, tcb, sa, sb, pa < cnt, lane);
            }
            if (pa < cnt) {
                if (nt < 0) {
                    const float tma = __ldg(A.tm + ka), tmb = __ldg(A.tm + (two ? kb : ka));
                    const float xa[3] = {__fadd_rn(o[0], __fmul_rn(d[0], tma)), __fadd_rn(o[1], __fmul_rn(d[1], tma)),
                                         __fadd_rn(o[2], __fmul_rn(d[2], tma))};
                    const float xb[3] = {__fadd_rn(o[0], __fmul_rn(d[0], tmb)), __fadd_rn(o[1], __fmul_rn(d[1], tmb)),
                                         __fadd_rn(o[2], __fmul_rn(d[2], tmb))};
                    sa = sigma_all(A.field, xa);
                    sb = sigma_all(A.field, xb);
                }
                taua = __fmul_rn(sa, __fsub_rn(a1, a0));
                if (two) taub = __fmul_rn(sb, __fsub_rn(b1, b0));
            }
            const float pair = taua + taub;
            float x = pair;  // -> inclusive prefix over the lanes' pairs
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, x, o2);
                if (lane >= o2) x += y;
            }
            const float before_a = carry + (x - pair), before_b = before_a + taua;
            const float Qc = Q + warp_sum((pa < cnt ? before_a : 0.0f) + (pb < cnt ? before_b : 0.0f));
            const float lo_thr = A.thr - depth_error(rb, cnt, Qc, A.thr);
            const unsigned over_a = __ballot_sync(0xffffffffu, pa < cnt && before_a > lo_thr);
            const unsigned over_b = __ballot_sync(0xffffffffu, pb < cnt && before_b > lo_thr);
            if (over_a | over_b) {  // the first point near or past the threshold, in lattice order
                const int ja = over_a ? __ffs(over_a) - 1 : 32, jb = over_b ? __ffs(over_b) - 1 : 32;
                const bool at_a = ja <= jb;
                const int j = at_a ? ja : jb;
                const float bc = __shfl_sync(0xffffffffu, at_a ? before_a : before_b, j);
                const int kc = __shfl_sync(0xffffffffu, at_a ? ka : kb, j);
                if (bc - depth_error(rb, cnt, Qc, bc) > A.thr) {
                    cut = p0 + 2 * j + (at_a ? 0 : 1);
                    kstop = kc;
                    return 1;
                }
                return 2;
            }
            Q = Qc;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    } else {
        int seen = 0;
        for (int kb = 0; kb < A.K && seen < cnt; kb += 32) {
            const int k = kb + lane;
            bool occ = false;
            if (k < A.K) {
                int lvl;
                const I idx = cell_index<I>(A, o, d, __ldg(A.tm + k), 0, lvl);
                occ = idx != (I)-1 && ((__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u);
            }
            const unsigned m = __ballot_sync(0xffffffffu, occ);
            if (!m) continue;
            float tau = 0.0f;
            if (occ) {
                const float t0 = __ldg(A.tt + k), t1 = __ldg(A.tt + k + 1);
                float sg;
                if (nt >= 0) {
                    sg = sigma_table(tab, nt, 0.5f * (t0 + t1));
                } else {
                    const float tm = __ldg(A.tm + k);
                    const float x[3] = {__fadd_rn(o[0], __fmul_rn(d[0], tm)), __fadd_rn(o[1], __fmul_rn(d[1], tm)),
                                        __fadd_rn(o[2], __fmul_rn(d[2], tm))};
                    sg = sigma_all(A.field, x);
                }
                tau = __fmul_rn(sg, __fsub_rn(t1, t0));
            }
            float x = tau;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, x, o2);
                if (lane >= o2) x += y;
            }
            const float before = carry + (x - tau);
            const float Qc = Q + warp_sum(occ ? before : 0.0f);
            const float lo_thr = A.thr - depth_error(rb, cnt, Qc, A.thr);
            const unsigned over = __ballot_sync(0xffffffffu, occ && before > lo_thr);
            if (over) {
                const int j = __ffs(over) - 1;
                const float bc = __shfl_sync(0xffffffffu, before, j);
                if (bc - depth_error(rb, cnt, Qc, bc) > A.thr) {
                    cut = seen + __popc(m & ((1u << j) - 1u));
                    kstop = kb + j;
                    return 1;
                }
                return 2;
            }
            seen += __popc(m);
            Q = Qc;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    return 0;
}

// The blobs that can have S > 0 (a density above 2^-126 somewhere on the
// line) on some ray of a group of rays, as an ascending list; every other
// blob gives S = 0 exactly in build_warp_table on each of the group's rays,
// so leaving it out changes no result.  With c = the line of the group's
// first ray (origin o_c, unit direction d_c), delta = the largest distance of
// a group ray's origin from o_c and s_max = the largest sine of the angle of
// a group ray's direction to d_c, the distance of blob centre mu from ray i's
// line is at least p_c - delta - (|mu - o_c| + delta) s_max (p_c its distance
// from line c; the closest point of line i lies within |mu - o_i| of o_i).
// S = 0 once C = log2 peak - log2(e) p^2 / (2 std^2) < -140, i.e. p above
// R_b = std sqrt((141 + log2 peak) / 0.7213) (one unit of slack in the
// exponent for the FP32 rounding of C), with relative slack 1e-4 for the
// FP32 distances.  Returns the list length; -1 (use every blob) when a ray
// of the group has a zero or non-finite direction.
// oi, di: this lane's ray (lv: the lane has one; lane 0 always has).
__device__ int group_candidates(const nacc_blob_field& f, const float4* sm, const float4* sk, const float oi[3],
                                const float di[3], bool lv, uint16_t* cand, int lane) {
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
    float sn = 0.0f, dl = 0.0f;
    if (lv) {
        const float cx = fmaf(di[1], dc[2], -di[2] * dc[1]), cy = fmaf(di[2], dc[0], -di[0] * dc[2]),
                    cz = fmaf(di[0], dc[1], -di[1] * dc[0]);
        sn = sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx))) / (li * lc) * 1.0001f + 1e-6f;
        const float e0 = oi[0] - oc[0], e1 = oi[1] - oc[1], e2 = oi[2] - oc[2];
        dl = sqrtf(fmaf(e2, e2, fmaf(e1, e1, e0 * e0))) * 1.0001f;
    }
    const float s_max = warp_max(sn), delta = warp_max(dl);
    if (!(s_max < 1e30f && delta < 1e30f)) return -1;
    const float u0 = dc[0] / lc, u1 = dc[1] / lc, u2 = dc[2] / lc;
    int nc = 0;
    for (int b0 = 0; b0 < f.n_blobs; b0 += 32) {
        const int b = b0 + lane;
        bool keep = false;
        if (b < f.n_blobs) {
            float4 mc, kc;
            if (b < kStageBlobs) {
                mc = sm[b];
                kc = sk[b];
            } else {
                blob_consts(f, b, mc, kc);
            }
            keep = true;
            if (!(kc.x > -141.0f)) {
                keep = false;  // peak below 2^-141 (or none): C < -140 everywhere
            } else {
                const float m0 = mc.x - oc[0], m1 = mc.y - oc[1], m2 = mc.z - oc[2];
                const float cx = fmaf(m1, u2, -m2 * u1), cy = fmaf(m2, u0, -m0 * u2), cz = fmaf(m0, u1, -m1 * u0);
                const float pc = sqrtf(fmaf(cz, cz, fmaf(cy, cy, cx * cx)));
                const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
                const float rb = kc.w * sqrtf((141.0f + kc.x) * 1.38629436f);  // std sqrt((141 + log2 peak) / 0.7213)
                const float lower = pc - delta - (mn + delta) * s_max - 1e-4f * (mn + delta + 1.0f);
                keep = !(lower > rb * 1.0001f + 1e-5f * (mn + delta));
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (keep) cand[nc + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)b;
        nc += __popc(bal);
    }
    return nc;
}

// Early stop (after the count pass): one warp per ray, the block's rays in
// turn, each decided as early_stop.cuh describes: no density at all when the
// ray's depth bound stays below the threshold; else the fast depth -- the
// ray's occupied points visited 64 (runs) or 32 (lattice walk when the runs
// overflowed) at a time in lattice order, each lane adding its points'
// sigma dt from the ray's table, a warp scan giving the optical depth
// before each point -- cut at the first point whose fast depth passes the
// threshold by more than the bound; else (a fast depth within the bound of
// the threshold, or A.exact_all) the exact path.  The count and stop index
// are cut there and the block's total is rewritten.
template <typename I>
__global__ void __launch_bounds__(kThreads, 5) k_unb_stop(UArgs A, int32_t* __restrict__ counts,
                                                       int32_t* __restrict__ kstops,
                                                       const int32_t* __restrict__ nruns,
                                                       const int2* __restrict__ runs,
                                                       long long* __restrict__ block_sums,
                                                       unsigned long long* __restrict__ ticket,
                                                       long long* __restrict__ queue,
                                                       unsigned long long* __restrict__ qlen) {
    __shared__ float4 s_tab[kWarps][kStopTable];
    __shared__ uint16_t s_tidx[kWarps][kStopTable];
    __shared__ float4 s_bm[kStageBlobs];
    __shared__ float4 s_bk[kStageBlobs];
    __shared__ uint16_t s_cand[kWarps][kMaxBlobs];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float4* tab = s_tab[wid];
    uint16_t* tidx = s_tidx[wid];
    for (int b = tid; b < min(A.field.n_blobs, kStageBlobs); b += kThreads) blob_consts(A.field, b, s_bm[b], s_bk[b]);
    __syncthreads();
    const float t_near = __ldg(A.tt), t_far = __ldg(A.tt + A.K);
    const float dinv = (1.0f / t_near - 1.0f / t_far) / (float)A.K * 1.01f;
    const float dt_max = (t_far - t_near) * 1.0001f;
    const int nblobs = A.field.n_blobs;
    const int64_t n_groups = (A.n + 31) / 32;
    for (;;) {  // groups of 32 rays by ticket: rays that stop cost far more than rays that cannot
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const int64_t grp = (int64_t)__shfl_sync(0xffffffffu, tk, 0);
        if (grp >= n_groups) break;
        const int64_t rbase = grp * 32;
        long long delta = 0;  // change of the block's total
        // lane i loads the header of ray rbase + i (coalesced); the rays are then
        // taken in turn, their values broadcast by shuffles, and lane i keeps the
        // results of ray i
        const int64_t rl = rbase + lane;
        const bool lv = rl < A.n;
        const int l_cnt = lv ? counts[rl] : 0;
        const int l_nr = lv ? nruns[rl] : 0;
        float l_o[3] = {0.0f, 0.0f, 0.0f}, l_d[3] = {0.0f, 0.0f, 0.0f};
        if (lv) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                l_o[a] = A.o[3 * rl + a];
                l_d[a] = A.d[3 * rl + a];
            }
        }
        const int n_cand = group_candidates(A.field, s_bm, s_bk, l_o, l_d, lv, s_cand[wid], lane);
        __syncwarp();
        const uint16_t* cand = n_cand >= 0 ? s_cand[wid] : nullptr;
        const int nc = n_cand >= 0 ? n_cand : nblobs;
        int l_cut = l_cnt, l_kstop = A.K;
        unsigned todo = __ballot_sync(0xffffffffu, l_cnt > 0);
        // the next ray's runs are loaded while the current one is evaluated
        int2 run_next = make_int2(0, 0);
        if (todo) {
            const int i0 = __ffs(todo) - 1;
            const int nr0 = __shfl_sync(0xffffffffu, l_nr, i0);
            if (nr0 >= 0 && lane < nr0) run_next = runs[(rbase + i0) * kRunSlots + lane];
        }
        while (todo) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t r = rbase + i;
            const int cnt = __shfl_sync(0xffffffffu, l_cnt, i);
            const int nr = __shfl_sync(0xffffffffu, l_nr, i);
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __shfl_sync(0xffffffffu, l_o[a], i);
                d[a] = __shfl_sync(0xffffffffu, l_d[a], i);
            }
            const int2 run = run_next;
            if (todo) {
                const int in = __ffs(todo) - 1;
                const int nrn = __shfl_sync(0xffffffffu, l_nr, in);
                run_next = nrn >= 0 && lane < nrn ? runs[(rbase + in) * kRunSlots + lane] : make_int2(0, 0);
            }
            const float onorm = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) * 1.0001f;
            const float dnorm = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * 1.0001f;
            int cut = cnt, kstop = A.K;
            float U, e_out;
            const int nk = build_warp_table(A.field, s_bm, s_bk, cand, nc, o, d, onorm, dnorm, dinv, dt_max, cnt, tab,
                                            tidx, U, e_out, lane);
            __syncwarp();
            if (A.exact_all != 0 || !(depth_upper(U, cnt, nblobs) <= A.thr)) {  // the ray may stop
                const int nt = nk <= kStopTable ? nk : -1;
                const float e_grp = nt > 0 ? 2.0f * kGroupEps * (float)nt * (float)((cnt + 63) / 64) : 0.0f;
                // the refined table and its error bound
                float eps;
                const float ek = refine_warp_table(A.field, s_bm, s_bk, nk, o, d, onorm, dnorm, dinv, dt_max, cnt, tab,
                                                   tidx, eps, lane);
                __syncwarp();
                const RayBound rb{U, ek, eps, e_out + e_grp};
                const int st = A.exact_all != 0 || !bounds_usable(rb, cnt, A.thr)
                                   ? 2
                                   : unb_fast_cut<I>(A, tab, nt, rb, o, d, cnt, nr, run, lane, cut, kstop);
                const bool exact = st == 2;
                if (exact && lane == 0) queue[atomicAdd(qlen, 1ull)] = r;  // decided exactly by k_unb_stop_exact
            }
            if (lane == i) {
                l_cut = cut;
                l_kstop = kstop;
            }
            delta += cut - cnt;
            __syncwarp();  // the next ray rewrites the table
        }
        if (lv && l_cnt > 0) {
            counts[rl] = l_cut;
            kstops[rl] = l_kstop;
        }
        if (lane == 0 && delta != 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(block_sums + rbase / kThreads), (unsigned long long)delta);
        __syncwarp();  // the next group rewrites the candidate list
    }
}

// Exact decisions of the rays the early-stop pass queued (early_stop.cuh):
// persistent CTAs take queued rays one at a time (ticket `qhead` over the
// `*qlen` entries); warp 0 builds the ray's exact blob list, then the four
// warps evaluate the definition's sigma*dt at 128 consecutive points at a
// time (32 each) into shared memory and thread 0 adds them in order one at a
// time -- the definition's own sum -- stopping at the first point whose depth
// before it exceeds the threshold.  Rays whose runs overflowed walk the
// lattice on warp 0 alone (unb_stop_exact).  The cut and its lattice index
// replace the ray's count and stop, and the change of the count is added to
// its block's total.  Dynamic shared memory: the blobs' exact constants
// (UExact, n_blobs of them).
template <typename I>
__global__ void __launch_bounds__(kThreads) k_unb_stop_exact(UArgs A, int32_t* __restrict__ counts,
                                                             int32_t* __restrict__ kstops,
                                                             const int32_t* __restrict__ nruns,
                                                             const int2* __restrict__ runs,
                                                             long long* __restrict__ block_sums,
                                                             const long long* __restrict__ queue,
                                                             const unsigned long long* __restrict__ qlen,
                                                             unsigned long long* __restrict__ qhead) {
    extern __shared__ UExact s_eb[];
    __shared__ float4 s_bm[kStageBlobs];
    __shared__ float4 s_bk[kStageBlobs];
    __shared__ uint16_t s_ex[kMaxBlobs];
    __shared__ __align__(16) float s_tau[kThreads];
    __shared__ int s_k[kThreads];
    __shared__ float s_seq[32];
    __shared__ unsigned long long s_tk;
    __shared__ int s_nex, s_jc;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int b = tid; b < min(A.field.n_blobs, kStageBlobs); b += kThreads) blob_consts(A.field, b, s_bm[b], s_bk[b]);
    stage_exact_blobs(s_eb, A.field);
    __syncthreads();
    const float t_far = __ldg(A.tt + A.K);
    const unsigned long long nq = *qlen;
    for (;;) {
        if (tid == 0) s_tk = atomicAdd(qhead, 1ull);
        __syncthreads();
        const unsigned long long tk = s_tk;
        if (tk >= nq) break;  // the same for the whole CTA
        const int64_t r = queue[tk];
        const int cnt = counts[r], nr = nruns[r];
        const float o[3] = {A.o[3 * r], A.o[3 * r + 1], A.o[3 * r + 2]};
        const float d[3] = {A.d[3 * r], A.d[3 * r + 1], A.d[3 * r + 2]};
        const int2 run = (nr >= 0 && lane < nr) ? runs[r * kRunSlots + lane] : make_int2(0, 0);
        const float pos_far = (sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) +
                               t_far * sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])) * 1.0002f;
        if (wid == 0) {
            const int n = build_exact_list(A.field, s_bm, s_bk, o, d, pos_far, s_ex, lane);
            if (lane == 0) s_nex = n;
        }
        __syncthreads();
        const int n_ex = s_nex;
        int cut = cnt, kstop = A.K;
        if (nr >= 0) {
            int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ex, o2);
                if (lane >= o2) ex += y;
            }
            ex -= run.y;
            float P = 0.0f;  // the sequential sum (thread 0's)
            for (int pr = 0; pr < cnt; pr += kThreads) {
                const int p = pr + tid;
                int k = 0;
                for (int j = 0; j < nr; ++j) {
                    const int ej = __shfl_sync(0xffffffffu, ex, j);
                    const int kj = __shfl_sync(0xffffffffu, run.x, j);
                    if (p >= ej) k = kj + (p - ej);
                }
                s_tau[tid] = unb_exact_tau(A, s_eb, s_ex, n_ex, o, d, k, p < cnt, pos_far, lane);
                s_k[tid] = k;
                __syncthreads();
                if (tid == 0) s_jc = seq_depth_cut<kThreads>(s_tau, min(kThreads, cnt - pr), A.thr, P);
                __syncthreads();
                const int jc = s_jc;
                if (jc >= 0) {
                    cut = pr + jc;
                    kstop = s_k[jc];
                    break;
                }
            }
        } else if (wid == 0) {  // runs overflowed: the lattice walk, on one warp
            unb_stop_exact<I>(A, s_eb, s_ex, n_ex, o, d, cnt, nr, run, pos_far, lane, s_seq, cut, kstop);
        }
        if (tid == 0) {
            counts[r] = cut;
            kstops[r] = kstop;
            if (cut != cnt)
                atomicAdd(reinterpret_cast<unsigned long long*>(block_sums + r / kThreads),
                          (unsigned long long)(long long)(cut - cnt));
        }
        __syncthreads();  // the next ray rewrites the list, the buffers and the ticket
    }
}

// One block: exclusive scan of the block totals in place; total -> *n_samples, offsets[n].
__global__ void __launch_bounds__(1024) k_unb_scan(long long* __restrict__ sums, int64_t nb,
                                                   int64_t* __restrict__ off_last, int64_t* __restrict__ n_samples) {
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const long long v = i < nb ? sums[i] : 0;
        long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const long long carry = s_carry;
        const long long incl = x + (wid > 0 ? s_w[wid - 1] : 0);
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

// Fill pass.  Recorded rays are expanded one at a time by their warp (sample
// p of a ray is point p of its concatenated runs; coalesced stores); rays
// whose runs overflowed the slots re-walk the lattice per lane up to their
// recorded stop.
__global__ void __launch_bounds__(kThreads) k_unb_fill(UArgs A, const int32_t* __restrict__ counts,
                                                       const int32_t* __restrict__ kstops,
                                                       const int32_t* __restrict__ nruns,
                                                       const int2* __restrict__ runs,
                                                       const long long* __restrict__ block_off,
                                                       const int64_t* __restrict__ n_samples, int64_t capacity,
                                                       int64_t* __restrict__ offsets, int32_t* __restrict__ ray_idx,
                                                       float* __restrict__ t0s, float* __restrict__ t1s) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t r = (int64_t)blockIdx.x * kThreads + tid;
    const int cnt = r < A.n ? counts[r] : 0;
    __shared__ int s_w[kWarps];
    int x = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    int wbase = 0;
    for (int w = 0; w < wid; ++w) wbase += s_w[w];
    long long pos = block_off[blockIdx.x] + wbase + x - cnt;
    if (r < A.n) offsets[r] = pos;
    if (*n_samples > capacity) return;  // overflow: offsets only (the whole grid agrees)
    const int nr = cnt > 0 ? nruns[r] : 0;
    const int64_t r_lane0 = r - lane;

    unsigned todo = __ballot_sync(0xffffffffu, nr > 0);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        const int cj = __shfl_sync(0xffffffffu, cnt, j);
        const int nj = __shfl_sync(0xffffffffu, nr, j);
        const long long pj = __shfl_sync(0xffffffffu, pos, j);
        const int64_t rj = r_lane0 + j;
        const int2 run = lane < nj ? runs[rj * kRunSlots + lane] : make_int2(0, 0);
        int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ex, o);
            if (lane >= o) ex += y;
        }
        ex -= run.y;
        // lane l writes positions q..q+3, q = 4l + a multiple of 128 from pj
        // rounded down to a multiple of 4: groups of four inside the ray as
        // one 128-bit store per array, the ragged head and tail position by
        // position (nothing outside the ray is read from the table or written)
        const long long a4 = pj & ~3ll, pend = pj + cj;
        for (long long q0 = a4; q0 < pend; q0 += 128) {
            const long long q = q0 + 4 * lane;
            const int p0 = (int)(q - pj);  // sample index of position q within the ray (may be < 0)
            int k[4] = {p0, p0 + 1, p0 + 2, p0 + 3};
            for (int i = 0; i < nj; ++i) {
                const int ei = __shfl_sync(0xffffffffu, ex, i);
                const int ki = __shfl_sync(0xffffffffu, run.x, i);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (p0 + u >= ei) k[u] = ki + (p0 + u - ei);
            }
            float t0[4], t1[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool in = p0 + u >= 0 && p0 + u < cj;
                t0[u] = in ? __ldg(A.tt + k[u]) : 0.0f;
                t1[u] = in ? __ldg(A.tt + k[u] + 1) : 0.0f;
            }
            if (q >= pj && q + 4 <= pend) {
                *reinterpret_cast<float4*>(t0s + q) = make_float4(t0[0], t0[1], t0[2], t0[3]);
                *reinterpret_cast<float4*>(t1s + q) = make_float4(t1[0], t1[1], t1[2], t1[3]);
                if (ray_idx) *reinterpret_cast<int4*>(ray_idx + q) = make_int4((int)rj, (int)rj, (int)rj, (int)rj);
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (q + u < pj || q + u >= pend) continue;
                    t0s[q + u] = t0[u];
                    t1s[q + u] = t1[u];
                    if (ray_idx) ray_idx[q + u] = (int32_t)rj;
                }
            }
        }
    }

    if (nr >= 0) return;
    const float o[3] = {A.o[3 * r], A.o[3 * r + 1], A.o[3 * r + 2]};
    const float d[3] = {A.d[3 * r], A.d[3 * r + 1], A.d[3 * r + 2]};
    const int kend = kstops[r];
    int written = 0, hint = 0;
    for (int kb = 0; kb < kend && written < cnt; kb += kBatch) {
        float t[kBatch + 1];
        unsigned m = batch_mask<int64_t>(A, o, d, kb, t, hint);
        while (m && written < cnt) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            if (kb + j >= kend) break;
            t0s[pos] = __ldg(A.tt + kb + j);
            t1s[pos] = __ldg(A.tt + kb + j + 1);
            if (ray_idx) ray_idx[pos] = (int32_t)r;
            ++pos;
            ++written;
        }
    }
}

// x = c if m' = max|c_a| <= 1, else c * (inv / m'), inv = 1 / (2 - min(m', 2 - 2^-23)).
__global__ void __launch_bounds__(256) k_uncontract(int64_t n, const float* __restrict__ c, float* __restrict__ x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float c0 = c[3 * i], c1 = c[3 * i + 1], c2 = c[3 * i + 2];
        const float mp = fmaxf(fmaxf(fabsf(c0), fabsf(c1)), fabsf(c2));
        float g = 1.0f;
        if (mp > 1.0f) {
            const float inv = __fdiv_rn(1.0f, __fsub_rn(2.0f, fminf(mp, kMaxContracted)));
            g = __fdiv_rn(inv, mp);
        }
        x[3 * i] = __fmul_rn(c0, g);
        x[3 * i + 1] = __fmul_rn(c1, g);
        x[3 * i + 2] = __fmul_rn(c2, g);
    }
}

// c = x if m = max|x_a| <= 1, else x * ((2 - 1/m) * (1/m)).
__global__ void __launch_bounds__(256) k_contract(int64_t n, const float* __restrict__ x, float* __restrict__ c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
        const float m = fmaxf(fmaxf(fabsf(x0), fabsf(x1)), fabsf(x2));
        float g = 1.0f;
        if (m > 1.0f) {
            const float inv = __fdiv_rn(1.0f, m);
            g = __fmul_rn(__fsub_rn(2.0f, inv), inv);
        }
        c[3 * i] = m > 1.0f ? __fmul_rn(x0, g) : x0;
        c[3 * i + 1] = m > 1.0f ? __fmul_rn(x1, g) : x1;
        c[3 * i + 2] = m > 1.0f ? __fmul_rn(x2, g) : x2;
    }
}

// edges[r][j] = Phi(j / n_bins), the s-lattice of n_bins bins, for every ray.
__global__ void __launch_bounds__(256) k_phi_edges(int64_t n_rays, int nb, float inv_tn, float inv_tf,
                                                   float* __restrict__ edges) {
    const int64_t total = n_rays * (nb + 1);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % (nb + 1));
        const float s = __fdiv_rn((float)j, (float)nb);
        edges[i] = __fdiv_rn(1.0f, __fadd_rn(__fmul_rn(inv_tn, __fsub_rn(1.0f, s)), __fmul_rn(inv_tf, s)));
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_march_unbounded_scratch_bytes(int64_t n_rays, int32_t max_steps) {
    if (n_rays < 0 || max_steps < 1) return 0;
    const int64_t nb = (n_rays + kThreads - 1) / kThreads;
    return align256(4 * (size_t)n_rays) * 3 + align256(sizeof(int2) * kRunSlots * (size_t)n_rays) +
           align256(8 * (size_t)(nb > 0 ? nb : 1)) + align256(4 * ((size_t)max_steps + 1)) +
           align256(4 * (size_t)max_steps) + align256(any_bytes(kLogF)) + align256(any_bytes(kLogC)) +
           256 + align256(8 * (size_t)n_rays);  // work tickets and exact queue of the early-stop pass
}

extern "C" int nacc_march_unbounded(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                                    const nacc_march_params* params, const nacc_blob_field* field, nacc_packed* out,
                                    void* scratch, size_t scratch_bytes, void* stream) {
    clear_error();
    UArgs A;
    if (!make_geom(grid, &A.g, true)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(params != nullptr && out != nullptr, "params / out is NULL");
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(params->max_steps >= 1 && params->max_steps <= (1 << 24), "max_steps=%d outside [1, 2^24]",
                   params->max_steps);
    NACC_CHECK_ARG(params->t_min > 0.0f && std::isfinite(params->t_max) && params->t_max > params->t_min,
                   "need 0 < t_min < t_max < inf (t_near, t_far of the s-lattice)");
    NACC_CHECK_ARG(out->offsets && out->n_samples, "out->offsets / out->n_samples is NULL");
    NACC_CHECK_ARG(out->capacity >= 0 && (out->capacity == 0 || (out->t_starts && out->t_ends)),
                   "out->t_starts / out->t_ends is NULL");
    NACC_CHECK_ARG(((reinterpret_cast<uintptr_t>(out->t_starts) | reinterpret_cast<uintptr_t>(out->t_ends) |
                     reinterpret_cast<uintptr_t>(out->ray_indices)) & 15) == 0,
                   "out->t_starts, t_ends and ray_indices must be 16-byte aligned");
    const bool with_field = field != nullptr && field->n_blobs > 0 && params->early_stop_eps > 0.0f;
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
    const size_t need = nacc_march_unbounded_scratch_bytes(n_rays, params->max_steps);
    NACC_CHECK_ARG(scratch && scratch_bytes >= need, "scratch too small: %zu < %zu bytes", scratch_bytes, need);
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch not 256-byte aligned");
    const int64_t nb = (n_rays + kThreads - 1) / kThreads;
    NACC_CHECK_ARG(nb < (int64_t(1) << 31), "too many rays for one launch");
    A.o = rays_o;
    A.d = rays_d;
    A.n = n_rays;
    A.K = params->max_steps;
    A.thr = with_field ? tau_threshold(params->early_stop_eps) : INFINITY;
    A.exact_all = params->exact_stops != 0 ? 1 : 0;
    A.field = with_field ? *field : nacc_blob_field{0, nullptr, nullptr, nullptr, nullptr};
    char* sp = static_cast<char*>(scratch);
    int32_t* counts = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int32_t* kstops = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int32_t* nruns = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int2* runs = reinterpret_cast<int2*>(sp);
    sp += align256(sizeof(int2) * kRunSlots * (size_t)n_rays);
    long long* bsums = reinterpret_cast<long long*>(sp);
    sp += align256(8 * (size_t)nb);
    float* tt = reinterpret_cast<float*>(sp);
    sp += align256(4 * ((size_t)A.K + 1));
    float* tm = reinterpret_cast<float*>(sp);
    sp += align256(4 * (size_t)A.K);
    uint32_t* f_any = reinterpret_cast<uint32_t*>(sp);
    sp += align256(any_bytes(kLogF));
    uint32_t* c_any = reinterpret_cast<uint32_t*>(sp);
    sp += align256(any_bytes(kLogC));
    unsigned long long* tickets = reinterpret_cast<unsigned long long*>(sp);  // ticket, qlen, qhead
    sp += 256;
    long long* queue = reinterpret_cast<long long*>(sp);
    A.tt = tt;
    A.tm = tm;
    A.nbf = (A.g.res + (1 << kLogF) - 1) >> kLogF;
    A.nbc = (A.g.res + (1 << kLogC) - 1) >> kLogC;
    A.f_any = f_any;
    A.c_any = c_any;
    {
        const int64_t nfb = (int64_t)A.g.n_levels * A.nbf * A.nbf * A.nbf;
        k_unb_fine_summary<<<(unsigned)((nfb + 255) / 256), 256, 0, st>>>(A.g, A.nbf, f_any);
        NACC_LAUNCH_CHECK();
        const int64_t ncb = (int64_t)A.g.n_levels * A.nbc * A.nbc * A.nbc;
        k_unb_coarse_summary<<<(unsigned)((ncb + 255) / 256), 256, 0, st>>>(A.g.n_levels, A.nbc, A.nbf, f_any,
                                                                           c_any);
        NACC_LAUNCH_CHECK();
    }
    {
        const int K = A.K;
        const int blocks = (int)std::min<int64_t>(((int64_t)K + 1 + 255) / 256, (int64_t)sm_count() * 4);
        k_unb_table<<<blocks, 256, 0, st>>>(K, 1.0f / params->t_min, 1.0f / params->t_max, tt, tm);
        NACC_LAUNCH_CHECK();
    }
    // 32-bit cell indices when every index (and the all-ones "outside") fits
    const bool idx32 = (int64_t)A.g.n_levels * A.g.res * A.g.res * A.g.res < (int64_t(1) << 32) - 1;
    if (cudaEvent_t e = march_count_events()[0]) NACC_CUDA_TRY(cudaEventRecord(e, st));
    if (idx32)
        k_unb_count<uint32_t><<<(unsigned)nb, kThreads, 0, st>>>(A, counts, kstops, nruns, runs, bsums);
    else
        k_unb_count<int64_t><<<(unsigned)nb, kThreads, 0, st>>>(A, counts, kstops, nruns, runs, bsums);
    NACC_LAUNCH_CHECK();
    if (with_field) {
        // persistent warps taking 32-ray groups by ticket; rays they cannot
        // decide from bounds go to a queue decided exactly by a second kernel
        NACC_CUDA_TRY(cudaMemsetAsync(tickets, 0, 3 * sizeof(unsigned long long), st));
        int per_sm = 0, per_sm_x = 0;
        const size_t shm_x = sizeof(UExact) * (size_t)A.field.n_blobs;  // <= 20 KiB (kMaxBlobs blobs)
        if (idx32) {
            NACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unb_stop<uint32_t>, kThreads, 0));
            NACC_CUDA_TRY(
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, k_unb_stop_exact<uint32_t>, kThreads, shm_x));
        } else {
            NACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_unb_stop<int64_t>, kThreads, 0));
            NACC_CUDA_TRY(
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, k_unb_stop_exact<int64_t>, kThreads, shm_x));
        }
        const unsigned blocks =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sm_count() * std::max(per_sm, 1)));
        const unsigned blocks_x =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(nb, (int64_t)sm_count() * std::max(per_sm_x, 1)));
        if (idx32) {
            k_unb_stop<uint32_t><<<blocks, kThreads, 0, st>>>(A, counts, kstops, nruns, runs, bsums, tickets, queue,
                                                             tickets + 1);
            NACC_LAUNCH_CHECK();
            k_unb_stop_exact<uint32_t><<<blocks_x, kThreads, shm_x, st>>>(A, counts, kstops, nruns, runs, bsums, queue,
                                                                     tickets + 1, tickets + 2);
        } else {
            k_unb_stop<int64_t><<<blocks, kThreads, 0, st>>>(A, counts, kstops, nruns, runs, bsums, tickets, queue,
                                                            tickets + 1);
            NACC_LAUNCH_CHECK();
            k_unb_stop_exact<int64_t><<<blocks_x, kThreads, shm_x, st>>>(A, counts, kstops, nruns, runs, bsums, queue,
                                                                    tickets + 1, tickets + 2);
        }
        NACC_LAUNCH_CHECK();
    }
    if (cudaEvent_t e = march_count_events()[1]) NACC_CUDA_TRY(cudaEventRecord(e, st));
    k_unb_scan<<<1, 1024, 0, st>>>(bsums, nb, out->offsets + n_rays, out->n_samples);
    NACC_LAUNCH_CHECK();
    k_unb_fill<<<(unsigned)nb, kThreads, 0, st>>>(A, counts, kstops, nruns, runs, bsums, out->n_samples,
                                                  out->capacity, out->offsets, out->ray_indices, out->t_starts,
                                                  out->t_ends);
    NACC_LAUNCH_CHECK();
    const bool may_overflow = (double)out->capacity < (double)n_rays * (double)params->max_steps;
    if (may_overflow) {
        int64_t total = 0;
        NACC_CUDA_TRY(cudaMemcpyAsync(&total, out->n_samples, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        NACC_CUDA_TRY(cudaStreamSynchronize(st));
        if (total > out->capacity) {
            set_error("packed capacity %lld < %lld samples", (long long)out->capacity, (long long)total);
            return NACC_ERR_CAPACITY;
        }
    }
    return NACC_OK;
}

extern "C" int nacc_uncontract_points(int64_t n, const float* c_in, float* x_out, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0, "n=%lld < 0", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(c_in && x_out, "c_in / x_out is NULL");
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_uncontract<<<blocks, 256, 0, as_stream(stream)>>>(n, c_in, x_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_contract_points(int64_t n, const float* x_in, float* c_out, void* stream) {
    clear_error();
    NACC_CHECK_ARG(n >= 0, "n=%lld < 0", (long long)n);
    if (n == 0) return NACC_OK;
    NACC_CHECK_ARG(x_in && c_out, "x_in / c_out is NULL");
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    k_contract<<<blocks, 256, 0, as_stream(stream)>>>(n, x_in, c_out);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_phi_edges(int64_t n_rays, int32_t n_bins, float t_near, float t_far, float* edges,
                              void* stream) {
    clear_error();
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 34), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(n_bins >= 1 && n_bins <= 4096, "n_bins=%d outside [1, 4096]", n_bins);
    NACC_CHECK_ARG(t_near > 0.0f && std::isfinite(t_far) && t_far > t_near, "need 0 < t_near < t_far < inf");
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(edges, "edges is NULL");
    const int64_t total = n_rays * (n_bins + 1);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)sm_count() * 16);
    k_phi_edges<<<blocks, 256, 0, as_stream(stream)>>>(n_rays, n_bins, 1.0f / t_near, 1.0f / t_far, edges);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}
