// march.cu -- occupancy-grid lattice marching into packed samples
// (nacc_march_grid): count pass (run walk), early-stop pass, block-offset
// scan, fill pass.
//
// Table 1 "Spatial Skipping" (occupied <=> bit set), Sec. 3.1 (skip empty
// space), Sec. 4.2 "Sample as Interval" / "Packed Tensor" / "No Gradient
// Filtering", Appendix B (step, resolution, threshold).
//
// One thread marches one ray cell by cell.  At a lattice point the full
// test runs (t0, t1, midpoint, position, level, cell, bit) in explicitly
// rounded FP32 intrinsics, bit-identical to the dense-march definition; then
// the exit of the cell is computed conservatively and every lattice point up
// to it shares the cell, hence the occupancy:
//   * along each axis the computed cell index is monotone in k (every
//     rounding step is monotone), so inside a cell it can only change when
//     the exact position crosses a face;
//   * the run ends at the exit of the cell shrunk by 1/256 cell per face (and
//     at the entry of the next finer level's box grown by the same margin);
//     a forward error analysis of the rounded position, face and exit time
//     bounds their error by about 11u|o| + 15u|x|max (u = 2^-24), and the
//     skip is taken only at levels where 16x that bound is below the margin
//     (else the run is one point);
//   * the run holds the lattice points whose rounded midpoint lies before the
//     exit: k < floor(q + 1/2 - slack) with q = (t_exit - t_near)/dt and a
//     slack of 1/64 step plus 2^-16 (|q| + |t_near|/dt) for the rounding of
//     t0, t1, the midpoint and q (at least 16x their bound).
// A cell inside an empty (or a fully occupied) block of cells runs to the
// block's exit -- its 16^3 block if that is uniform, else its 4^3 block if
// that is (per-call summaries of the bits): the same argument holds for any
// box of cells whose bits all agree.
// The count pass visits only run starts: it records each ray's occupied runs
// and their total, so the emitted set equals the dense march's at a fraction
// of its cost.  With a field, an early-stop pass gives each ray to a warp,
// which evaluates the density at the emitted points in lattice order, 64 at
// a time, and cuts the ray at the first point whose optical depth before it
// exceeds the threshold (the depth is a warp scan of FP32 sigma dt: the
// rounding order of the sum differs from a sequential one by a few ulps,
// which moves only decisions within that of the threshold); the fill pass
// never evaluates the field.  The fill pass expands the recorded runs
// warp-cooperatively as coalesced stores (rays whose runs overflowed the
// slots are re-marched per lane and flushed by the warp).
#include <algorithm>

#include "early_stop.cuh"
#include "nacc_internal.cuh"

namespace nacc {
namespace {

constexpr int kBlockThreads = 32;               // one ray per thread; one warp per block
constexpr int kRaysPerBlock = kBlockThreads;    // rays per block-sum entry
constexpr int kBuf = 32;                        // lattice indices buffered per lane
constexpr int kRunSlots = 16;                   // recorded lattice runs per ray
constexpr int kLogC = 4, kLogF = 2;             // block summaries: coarse 16^3 and fine 4^3 cells
constexpr size_t summary_bytes(int log) {       // one any- or all-bitfield, 8 levels of 1024^3 cells
    return size_t(NACC_MAX_LEVELS) * (size_t(1024) >> log) * (size_t(1024) >> log) * (size_t(1024) >> log) / 8;
}
constexpr size_t kBlockBitsBytes = 2 * summary_bytes(kLogC) + 2 * summary_bytes(kLogF);
constexpr float kSkipMargin = 1.0f / 256.0f;    // cells

struct MarchArgs {
    GridGeom g;
    const float* o;
    const float* d;
    int64_t n;
    float step;
    int max_steps;
    float t_min, t_max;
    float thr;  // optical-depth threshold (+inf: no early stop)
    int exact_all;  // every early-stop decision on the exact path (validation)
    float inv_step;  // 1/step, only for the conservative skip (never for lattice values)
    int idx32;       // every flat cell index fits 32 bits
    float skip_lim[NACC_MAX_LEVELS];  // skip allowed at level l iff max|o| <= skip_lim[l]
    // block summaries (NULL: none): bit set iff any (all) cells of the block are occupied
    const uint32_t* c_any;  // coarse blocks of (1 << kLogC)^3 cells
    const uint32_t* c_all;
    const uint32_t* f_any;  // fine blocks of (1 << kLogF)^3 cells
    const uint32_t* f_all;
    int nbc, nbf;           // blocks per axis
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
        const float inv = __fdiv_rn(1.0f, d[a]);
        const float ta = __fmul_rn(__fsub_rn(outer.lmin[a], o[a]), inv);
        const float tb = __fmul_rn(__fsub_rn(outer.lmax[a], o[a]), inv);
        const float lo = (ta < tb) ? ta : tb;
        const float hi = (ta < tb) ? tb : ta;
        if (lo > near) near = lo;
        if (hi < far) far = hi;
    }
    tn = near;
    tf = far;
    return near < far;
}

struct Ray {
    float o[3], d[3], invd[3];
    float tn, tf;
    float omax;  // max |o|
};

// One lattice point: interval [t0, t1], midpoint position x, level l (L if
// outside every level) and cell ic; returns the occupancy bit.
__device__ __forceinline__ bool lattice_point(const MarchArgs& A, const Ray& R, int k, float& t0, float& t1,
                                              float x[3], int& l, int ic[3]) {
    t0 = __fadd_rn(R.tn, __fmul_rn((float)k, A.step));
    t1 = __fadd_rn(t0, A.step);
    const float tm = __fmul_rn(__fadd_rn(t0, t1), 0.5f);
#pragma unroll
    for (int a = 0; a < 3; ++a) x[a] = __fadd_rn(R.o[a], __fmul_rn(R.d[a], tm));
    const int L = A.g.n_levels;
    for (l = 0; l < L; ++l) {
        const Level& lv = A.g.lv[l];
        if (x[0] >= lv.lmin[0] && x[0] <= lv.lmax[0] && x[1] >= lv.lmin[1] && x[1] <= lv.lmax[1] &&
            x[2] >= lv.lmin[2] && x[2] <= lv.lmax[2])
            break;
    }
    if (l == L) return false;
    const Level& lv = A.g.lv[l];
    const int res = A.g.res;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = __fmul_rn(__fsub_rn(x[a], lv.lmin[a]), lv.scale[a]);
        const int c = (int)floorf(u);
        ic[a] = c < 0 ? 0 : (c > res - 1 ? res - 1 : c);
    }
    if (A.idx32) {
        const uint32_t r3 = (uint32_t)res * res * res;
        const uint32_t idx = (uint32_t)l * r3 + ((uint32_t)ic[0] * res + ic[1]) * res + ic[2];
        return (__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u;
    }
    const uint64_t r3 = (uint64_t)res * res * res;
    const uint64_t idx = (uint64_t)l * r3 + ((uint64_t)ic[0] * res + ic[1]) * res + ic[2];
    return (__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u;
}

// First lattice index that may leave the box of cells lo[a] <= c_a <= hi[a]
// of level l, holding the point of lattice index k at midpoint tm
// (conservative, see the header).
__device__ __forceinline__ int skip_target(const MarchArgs& A, const Ray& R, int k, float tm, int l,
                                           const int lo[3], const int hi[3], int kend) {
    if (R.omax > A.skip_lim[l]) return k + 1;
    const Level& lv = A.g.lv[l];
    float ts = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] > 0.0f) {
            const float face = lv.lmin[a] + ((float)hi[a] + (1.0f - kSkipMargin)) * lv.width[a];
            ts = fminf(ts, (face - R.o[a]) * R.invd[a]);
        } else if (R.d[a] < 0.0f) {
            const float face = lv.lmin[a] + ((float)lo[a] + kSkipMargin) * lv.width[a];
            ts = fminf(ts, (face - R.o[a]) * R.invd[a]);
        }
    }
    if (l > 0) {  // do not skip into the next finer level's (grown) box
        const Level& fl = A.g.lv[l - 1];
        float tin = -INFINITY, tout = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float m = kSkipMargin * lv.width[a];
            const float lo = fl.lmin[a] - m, hi = fl.lmax[a] + m;
            if (R.d[a] == 0.0f) {
                if (R.o[a] < lo || R.o[a] > hi) {
                    tin = INFINITY;
                    tout = -INFINITY;
                }
            } else {
                const float ta = (lo - R.o[a]) * R.invd[a], tb = (hi - R.o[a]) * R.invd[a];
                tin = fmaxf(tin, fminf(ta, tb));
                tout = fminf(tout, fmaxf(ta, tb));
            }
        }
        if (tin <= tout && tout > tm) ts = fminf(ts, tin);
    }
    const float q = (ts - R.tn) * A.inv_step;
    const float slack = 0.015625f + 1.52587890625e-5f * (fabsf(R.tn) * A.inv_step + fminf(fabsf(q), 16777216.0f));
    const float e = q + 0.5f - slack;  // exclusive run end (before flooring); NaN -> no skip
    if (!(e >= (float)(k + 2))) return k + 1;
    return e < (float)kend ? (int)floorf(e) : kend;
}

__device__ __forceinline__ float ex2_approx(float a) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a));
    return y;
}

// Blob parameters of the early-stop pass, staged in shared memory: centre,
// c2 = coef * log2 e (the base-2 exponent's coefficient), peak, the
// definition's coef = fl(-0.5 / fl(std * std)), std, 1/std.
struct StopBlob {
    float mx, my, mz, c2;
    float peak, coef, sd, isd;
};

__device__ inline void stage_stop_blobs(StopBlob* s, const nacc_blob_field& f) {
    for (int b = threadIdx.x; b < f.n_blobs; b += blockDim.x) {
        StopBlob v;
        v.mx = f.mu[3 * b + 0];
        v.my = f.mu[3 * b + 1];
        v.mz = f.mu[3 * b + 2];
        v.sd = f.std[b];
        v.coef = __fdiv_rn(-0.5f, __fmul_rn(v.sd, v.sd));
        v.c2 = v.coef * 1.4426950408889634f;  // log2 e
        v.peak = f.peak[b];
        v.isd = 1.0f / v.sd;
        s[b] = v;
    }
}

// Early-stop density: the blob field of the harness evaluated with fused
// multiply-adds and the hardware base-2 exponent (exp(a) = 2^(a log2 e)),
// at two points per blob load (two buffered samples of a lane share every
// shared-memory read of the blob parameters).  Used for rays whose table
// would exceed kTab entries; its error is inside the per-ray bound of
// early_stop.cuh.
__device__ __forceinline__ void sigma_early_stop2(const StopBlob* s, int n, const float xa[3], const float xb[3],
                                                  float& sa, float& sb) {
    float acc_a = 0.0f, acc_b = 0.0f;
#pragma unroll 2
    for (int b = 0; b < n; ++b) {
        const float4 v = *reinterpret_cast<const float4*>(&s[b].mx);  // centre, coefficient
        const float pk = s[b].peak;
        const float ax = xa[0] - v.x, ay = xa[1] - v.y, az = xa[2] - v.z;
        const float bx = xb[0] - v.x, by = xb[1] - v.y, bz = xb[2] - v.z;
        const float ra = fmaf(az, az, fmaf(ay, ay, ax * ax));
        const float rb = fmaf(bz, bz, fmaf(by, by, bx * bx));
        acc_a = fmaf(pk, ex2_approx(ra * v.w), acc_a);
        acc_b = fmaf(pk, ex2_approx(rb * v.w), acc_b);
    }
    sa = acc_a;
    sb = acc_b;
}

// Early-stop density along one ray, set up per ray by its warp: along the
// ray x(t) = o + t d, |x(t) - mu_b|^2 = |d|^2 (t - t*_b)^2 + p_b^2 with the
// closest approach t*_b = (mu_b - o).d / |d|^2 and p_b^2 = |(mu_b - o) x d|^2
// / |d|^2 (cross product: no cancellation near the centre).  The table keeps
// {A_b = c_b |d|^2, t*_b, C_b = c_b p_b^2, peak_b} (c_b the log2-scaled
// coefficient) in shared memory, and a sample costs one broadcast 128-bit
// load, three FP32 operations, one exp2 and one FMA per kept blob.  Rounding
// of t - t*_b is of the order of that of the position in the direct form.
constexpr int kTab = 64;  // table entries per ray; a ray with more kept blobs uses the direct form

// Blobs whose integral along the whole ray line is at most kCullEps
// (bound peak 2^C sqrt(2 pi) std / |d|, C = c_b p_b^2) are left out of the
// ray's table: each changes the optical depth by at most kCullEps.
constexpr float kCullEps = 1e-7f;

// The ray's early-stop table and depth bound (early_stop.cuh), built by the
// warp, lane b0 + lane handling blob b0 + lane: the per-ray closed form in
// FP32; blobs whose line integral exceeds kCullEps are compacted in blob
// order into the table (entry {c2 |d|^2, t*, C, peak}, blob index in tidx).
// U bounds the definition's depth at every sample (every blob's weight, the
// closed form's own FP32 rounding included); e_out is the error bound's
// share of the blobs left out (their whole weight).  Returns the number of
// kept blobs (the table holds the first kTab).  onorm = |o|, dnorm = |d|, tmax bounds |t| of every midpoint, cnt =
// the ray's samples.  Every lattice interval is within 8u tmax of dt long,
// and consecutive intervals, rounded apart, overlap by at most that much.
// One blob's part of the table and bound of a ray (below): its entry, whether
// it is kept, and its weight in U and in e_out.  dd = |d|^2, idd = 1/dd,
// ilen = 1/|d| (0 for a ray that does not move), dt_b and ov as below.
__device__ __forceinline__ void ray_blob_entry(const StopBlob& v, const float o[3], const float d[3], float dd,
                                               float idd, float ilen, float onorm, float dnorm, float dt_b, float ov,
                                               int cnt, float4& ent, bool& keep, float& u, float& e) {
    const float m0 = v.mx - o[0], m1 = v.my - o[1], m2 = v.mz - o[2];
    float ts, pp, I;
    if (dd > 0.0f) {
        const float md = fmaf(m2, d[2], fmaf(m1, d[1], m0 * d[0]));
        const float cx = fmaf(m1, d[2], -m2 * d[1]);
        const float cy = fmaf(m2, d[0], -m0 * d[2]);
        const float cz = fmaf(m0, d[1], -m1 * d[0]);
        ts = md * idd;
        pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
    } else {  // a ray that does not move: the distance is |mu - o|
        ts = 0.0f;
        pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
    }
    const float C = v.c2 * pp;
    const float S = v.peak * ex2_approx(C);  // largest density on the line
    if (dd > 0.0f) {
        I = S * 2.5066283f * v.sd * ilen;  // integral along the line
        keep = I > kCullEps;
    } else {
        I = S * dt_b * (float)cnt;  // every sample at the same point
        keep = true;
    }
    u = 0.0f;
    e = 0.0f;
    if (S > 0.0f) {
        // growth with the FP32 closed form's own error (within 11u |mu - o|) included
        const float p = sqrtf(pp);
        const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
        const float W = blob_weight(
            S, I, dt_b, dt_b, ov, blob_growth(p, v.isd, onorm + 2.5f * fabsf(ts) * dnorm + 16.0f * p + 12.0f * mn));
        u = W;
        if (!keep) e = W;
    }
    ent = make_float4(v.c2 * dd, ts, C, v.peak);
}

__device__ int build_ray_table(const StopBlob* sb, int n, const float o[3], const float d[3], float onorm,
                               float dnorm, float tmax, float dt, int cnt, float4* tab, uint16_t* tidx, float& U,
                               float& e_out, int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
    const float dt_b = dt + 8.0f * kU * tmax, ov = (float)cnt * 8.0f * kU * tmax;
    int nt = 0;
    float u = 0.0f, e = 0.0f;
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int b = b0 + lane;
        bool keep = false;
        float4 ent = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (b < n) {
            float ub, eb;
            ray_blob_entry(sb[b], o, d, dd, idd, ilen, onorm, dnorm, dt_b, ov, cnt, ent, keep, ub, eb);
            u += ub;
            e += eb;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        const int pos = nt + __popc(bal & ((1u << lane) - 1u));
        if (keep && pos < kTab) {
            tab[pos] = ent;
            tidx[pos] = (uint16_t)b;
        }
        nt += __popc(bal);
    }
    U = warp_sum(u);
    e_out = warp_sum(e);
    return nt;
}

// Error bound of the kept blobs (early_stop.cuh), one lane per kept blob:
// t* and p^2 again by closest_approach, the table entry rewritten (when the
// table holds the nt kept blobs; otherwise every kept blob is bounded from its
// FP32 values, for the direct form).  Returns the whole-ray bound, and the
// relative one in eps.  Arguments as build_ray_table.
// One kept blob's refined table entry and its terms of the ray's error
// bounds (absolute eb, relative er); false for a blob the direct form leaves
// out (only without a table: it is counted whole in the table build).
__device__ __forceinline__ bool refine_blob(const StopBlob& v, const float o[3], const float d[3], float dd, float idd,
                                            float ilen, float onorm, float dnorm, float dt_b, float ov, int cnt, int n,
                                            bool have_tab, float4& ent, float& eb, float& er) {
    float ts, pp;
    if (dd > 0.0f) {
        const float mu[3] = {v.mx, v.my, v.mz};
        closest_approach(mu, o, d, idd, ts, pp);
    } else {
        const float m0 = v.mx - o[0], m1 = v.my - o[1], m2 = v.mz - o[2];
        ts = 0.0f;
        pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
    }
    const float C = v.c2 * pp;
    const float S = v.peak * ex2_approx(C);
    const float I = dd > 0.0f ? S * 2.5066283f * v.sd * ilen : S * dt_b * (float)cnt;
    if (!have_tab && !(I > kCullEps) && dd > 0.0f) return false;
    const float p = sqrtf(pp);
    const float pos0 = onorm + 2.5f * fabsf(ts) * dnorm + 16.0f * p;
    const float gm1 = blob_growth(p, v.isd, pos0);
    eb = blob_error(blob_weight(S, I, dt_b, dt_b, ov, gm1), gm1, p * v.isd, n, true);
    er = blob_rel_error(v.isd, pos0, n);
    ent = make_float4(v.c2 * dd, ts, C, v.peak);
    return true;
}

__device__ float refine_ray_table(const StopBlob* sb, int n, int nt, const float o[3], const float d[3], float onorm,
                                  float dnorm, float tmax, float dt, int cnt, float4* tab, const uint16_t* tidx,
                                  float& eps, int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
    const float dt_b = dt + 8.0f * kU * tmax, ov = (float)cnt * 8.0f * kU * tmax;
    const bool have_tab = nt <= kTab;
    float e = 0.0f, em = 0.0f;
    for (int i = lane; i < (have_tab ? nt : n); i += 32) {
        float4 ent;
        float eb, er;
        if (!refine_blob(sb[have_tab ? tidx[i] : i], o, d, dd, idd, ilen, onorm, dnorm, dt_b, ov, cnt, n, have_tab, ent,
                         eb, er))
            continue;  // left out: counted whole in build_ray_table
        e += eb;
        em = fmaxf(em, er);
        if (have_tab) tab[i] = ent;
    }
    eps = warp_max(em);
    return warp_sum(e);
}

// The tables of a whole 32-ray entry when the field has at most kSmallBlobs
// blobs: eight lanes per ray, four rays per pass (lane 8s + b takes blob b of
// ray 4 pass + s), each ray's kept blobs compacted in blob order into its
// own kSmallBlobs entries of tab8, and U / e_out summed over the eight lanes
// in the order warp_sum takes for blobs 0..7 (the other lanes hold zeros
// there), so that every ray's table, nt, U and e_out are those
// build_ray_table gives; for a ray that may stop, the refined entries and
// bounds as refine_ray_table gives them, the same way.  Ray i's values come
// from lane i (l_*).
constexpr int kSmallBlobs = 8;
__device__ __forceinline__ void build_entry_tables(const StopBlob* sb, int n, const float l_o[3],
                                                   const float l_d[3], int l_cnt, float l_tn, int l_ke, float dt,
                                                   bool exact_all, float thr, float4* tab8, uint16_t* tidx8,
                                                   float* s_U, float* s_e, int* s_nt, float* s_ek, float* s_eps,
                                                   int lane) {
    const int slot = lane >> 3, b = lane & 7;
#pragma unroll 1
    for (int pass = 0; pass < 32 / 4; ++pass) {
        const int i = 4 * pass + slot;
        const int cnt = __shfl_sync(0xffffffffu, l_cnt, i);
        if (!__any_sync(0xffffffffu, cnt > 0)) continue;
        const float tn = __shfl_sync(0xffffffffu, l_tn, i);
        const int ke = __shfl_sync(0xffffffffu, l_ke, i);
        float o[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __shfl_sync(0xffffffffu, l_o[a], i);
            d[a] = __shfl_sync(0xffffffffu, l_d[a], i);
        }
        // the per-ray values as the ray loop forms them
        const float tmax = fabsf(tn) + (float)(ke + 1) * dt * 1.0001f;
        const float onorm = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) * 1.0001f;
        const float dnorm = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * 1.0001f;
        const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
        const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
        const float ilen = dd > 0.0f ? rsqrtf(dd) : 0.0f;
        const float dt_b = dt + 8.0f * kU * tmax, ov = (float)cnt * 8.0f * kU * tmax;
        bool keep = false;
        float4 ent = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float u = 0.0f, e = 0.0f;
        if (b < n && cnt > 0) ray_blob_entry(sb[b], o, d, dd, idd, ilen, onorm, dnorm, dt_b, ov, cnt, ent, keep, u, e);
        const unsigned grp = (__ballot_sync(0xffffffffu, keep) >> (8 * slot)) & 0xffu;
        if (keep) {
            const int pos = __popc(grp & ((1u << b) - 1u));
            tab8[i * kSmallBlobs + pos] = ent;
            tidx8[i * kSmallBlobs + pos] = (uint16_t)b;
        }
#pragma unroll
        for (int o2 = 4; o2 > 0; o2 >>= 1) {
            u += __shfl_xor_sync(0xffffffffu, u, o2);
            e += __shfl_xor_sync(0xffffffffu, e, o2);
        }
        // the refined table and bounds of a ray that may stop (the ray loop's
        // condition), lane 8s + j taking the ray's j-th kept blob as
        // refine_ray_table's lane j does
        const int nt = __popc(grp);
        const bool may = cnt > 0 && (exact_all || !(depth_upper(u, cnt, n) <= thr));
        __syncwarp();  // this pass's blob indices are in place
        float eb = 0.0f, er = 0.0f;
        if (may && b < nt) {
            float4 ent2;
            refine_blob(sb[tidx8[i * kSmallBlobs + b]], o, d, dd, idd, ilen, onorm, dnorm, dt_b, ov, cnt, n, true, ent2,
                        eb, er);
            tab8[i * kSmallBlobs + b] = ent2;
        }
#pragma unroll
        for (int o2 = 4; o2 > 0; o2 >>= 1) {
            eb += __shfl_xor_sync(0xffffffffu, eb, o2);
            er = fmaxf(er, __shfl_xor_sync(0xffffffffu, er, o2));
        }
        if (b == 0) {
            s_U[i] = u;
            s_e[i] = e;
            s_nt[i] = nt;
            s_ek[i] = eb;
            s_eps[i] = er;
        }
    }
    __syncwarp();
}

// The ascending list of the blobs that may be non-zero somewhere on the ray
// in the definition's arithmetic (early_stop.cuh, blob_may_count), built by
// the warp; returns its length.  pos_far = |o| + t_max |d|.
__device__ int build_exact_list(const StopBlob* sb, int n, const float o[3], const float d[3], float pos_far,
                                uint16_t* ex_list, int lane) {
    const float dd = fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
    const float idd = dd > 0.0f ? 1.0f / dd : 0.0f;
    int ne = 0;
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int b = b0 + lane;
        bool in_ex = false;
        if (b < n) {
            const StopBlob v = sb[b];
            const float m0 = v.mx - o[0], m1 = v.my - o[1], m2 = v.mz - o[2];
            float pp;
            if (dd > 0.0f) {
                const float cx = fmaf(m1, d[2], -m2 * d[1]), cy = fmaf(m2, d[0], -m0 * d[2]),
                            cz = fmaf(m0, d[1], -m1 * d[0]);
                pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
            } else {
                pp = fmaf(m2, m2, fmaf(m1, m1, m0 * m0));
            }
            // the FP32 distance is within 8u |mu - o| of exact; blob_may_count's
            // margin is 8u pos_far, so widen it by |mu - o|
            const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
            in_ex = blob_may_count(sqrtf(pp), v.sd, pos_far + mn);
        }
        const unsigned bex = __ballot_sync(0xffffffffu, in_ex);
        if (in_ex) ex_list[ne + __popc(bex & ((1u << lane) - 1u))] = (uint16_t)b;
        ne += __popc(bex);
    }
    return ne;
}

// Density at ray parameters ta, tb from the ray's table (every lane reads
// the same entry: a shared-memory broadcast).
__device__ __forceinline__ void sigma_tab2(const float4* tab, int nt, float ta, float tb, float& sa, float& sb) {
    float acc_a = 0.0f, acc_b = 0.0f;
#pragma unroll 4
    for (int b = 0; b < nt; ++b) {
        const float4 v = tab[b];
        const float ua = ta - v.y, ub = tb - v.y;
        acc_a = fmaf(v.w, ex2_approx(fmaf(v.x * ua, ua, v.z)), acc_a);
        acc_b = fmaf(v.w, ex2_approx(fmaf(v.x * ub, ub, v.z)), acc_b);
    }
    sa = acc_a;
    sb = acc_b;
}

// A table entry contributes to the optical depth of a group of points whose
// midpoints lie in [t_lo, t_hi] and whose intervals sum to at most span at
// most (its density at the point of [t_lo, t_hi] nearest its closest
// approach, the largest there) x span; entries below kGroupEps are left out
// for that group.  Over a ray of at most 2^24 points in groups of 64, with
// at most kTab entries, that moves the optical depth by at most 1.7e-3 (and
// by 1.0e-7 at 1,024 points): only decisions within that of the threshold.
// (The fast depth takes groups of 128 points: half as many groups, so the
// error bound's count of groups of 64 over-estimates.)
constexpr float kGroupEps = 1e-10f;
constexpr int kGroupMin = 16;  // tables of at most this many entries are summed whole (cheaper)

// The same densities at four points of a lane (each table entry read once).
__device__ __forceinline__ void sigma_tab4(const float4* tab, int nt, const float t[4], float sg[4]) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 2
    for (int b = 0; b < nt; ++b) {
        const float4 v = tab[b];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float d = t[u] - v.y;
            acc[u] = fmaf(v.w, ex2_approx(fmaf(v.x * d, d, v.z)), acc[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sg[u] = acc[u];
}

__device__ __forceinline__ void sigma_tab4_group(const float4* tab, int nt, float t_lo, float t_hi, float span,
                                                 const float t[4], float sg[4], bool active) {
    const int lane = threadIdx.x & 31;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int e0 = 0; e0 < nt; e0 += 32) {
        bool on = false;
        if (e0 + lane < nt) {
            const float4 v = tab[e0 + lane];
            const float u = fminf(fmaxf(v.y, t_lo), t_hi) - v.y;
            on = v.w * ex2_approx(fmaf(v.x * u, u, v.z)) * span > kGroupEps;
        }
        unsigned m = __ballot_sync(0xffffffffu, on);
        if (!active) continue;
        while (m) {
            const float4 v = tab[e0 + __ffs(m) - 1];
            m &= m - 1;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float d = t[u] - v.y;
                acc[u] = fmaf(v.w, ex2_approx(fmaf(v.x * d, d, v.z)), acc[u]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sg[u] = acc[u];
}

// Per-thread march state of one ray.
struct Lane {
    Ray R;
    int k;        // next lattice index
    int run_end;  // end (exclusive) of the current cell run
    bool occ;     // the current run is occupied
    bool done;
    float tau;    // optical depth of the emitted samples (early stop)
    int n;        // samples emitted
};

__device__ __forceinline__ bool lane_init(const MarchArgs& A, int64_t r, Lane& s) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        s.R.o[a] = __ldg(&A.o[3 * r + a]);
        s.R.d[a] = __ldg(&A.d[3 * r + a]);
        s.R.invd[a] = 1.0f / s.R.d[a];
    }
    s.R.omax = fmaxf(fabsf(s.R.o[0]), fmaxf(fabsf(s.R.o[1]), fabsf(s.R.o[2])));
    s.k = 0;
    s.run_end = 0;
    s.occ = false;
    s.tau = 0.0f;
    s.n = 0;
    s.done = !clip_ray(A.g.lv[A.g.n_levels - 1], s.R.o, s.R.d, A.t_min, A.t_max, s.R.tn, s.R.tf);
    return !s.done;
}

// Record of a ray's occupied lattice ranges for the fill pass: runs that
// continue one another are merged, up to kRunSlots ranges are stored as
// {first k, count} in this ray's slots; n = -1 marks an overflow.
struct RunRec {
    int2* slots;
    int n;
    int k0, k1;  // pending range [k0, k1)
};

__device__ __forceinline__ void rec_flush(RunRec& q) {
    if (q.k1 > q.k0 && q.n >= 0) {
        if (q.n < kRunSlots)
            q.slots[q.n++] = make_int2(q.k0, q.k1 - q.k0);
        else
            q.n = -1;
    }
}

__device__ __forceinline__ void rec_run(RunRec& q, int k0, int k1) {
    if (q.k1 == k0) {
        q.k1 = k1;
        return;
    }
    rec_flush(q);
    q.k0 = k0;
    q.k1 = k1;
}

__device__ __forceinline__ bool cell_bit(const MarchArgs& A, int l, int x, int y, int z) {
    const uint32_t res = (uint32_t)A.g.res;
    const uint32_t idx = ((uint32_t)l * res + (uint32_t)x) * res * res + (uint32_t)y * res + (uint32_t)z;
    return (__ldg(&A.g.bits[idx >> 5]) >> (idx & 31)) & 1u;
}

// Exit axis of the box [lo, hi] of level l along the ray (-1 if none): the
// face reached first.  Any answer keeps a box extended across it uniform.
__device__ __forceinline__ int exit_axis(const MarchArgs& A, const Ray& R, int l, const int lo[3], const int hi[3]) {
    const Level& lv = A.g.lv[l];
    int ax = -1;
    float tx = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (R.d[a] == 0.0f) continue;
        const float face = lv.lmin[a] + (float)(R.d[a] > 0.0f ? hi[a] + 1 : lo[a]) * lv.width[a];
        const float t = (face - R.o[a]) * R.invd[a];
        if (t < tx) {
            tx = t;
            ax = a;
        }
    }
    return ax;
}

// Occupancy summary bit of block (bx, by, bz) of level l in a summary with nb blocks per axis.
__device__ __forceinline__ bool summary_bit(const uint32_t* sum, int nb, int l, int bx, int by, int bz) {
    const uint32_t n = (uint32_t)nb;
    const uint32_t b = (((uint32_t)l * n + (uint32_t)bx) * n + (uint32_t)by) * n + (uint32_t)bz;
    return (__ldg(&sum[b >> 5]) >> (b & 31)) & 1u;
}

// The box of cells a run starting in cell ic of level l (occupancy occ)
// may span: the cell's coarse block if all its cells share occ, else its
// fine block if they do, else the cell; then, if the unit across the face
// the ray leaves through (the next block of the same size, or the next
// cell) shares occ too, the box spans it as well (32-bit cell indices only
// for the cell case).
__device__ __forceinline__ void run_box(const MarchArgs& A, const Ray& R, int l, const int ic[3], bool occ,
                                        int lo[3], int hi[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) lo[a] = hi[a] = ic[a];
    if (!A.c_any) return;
    int log = -1;  // unit of the box: 1 << log cells per edge; -1 a single cell
    if (summary_bit(occ ? A.c_all : A.c_any, A.nbc, l, ic[0] >> kLogC, ic[1] >> kLogC, ic[2] >> kLogC) == occ)
        log = kLogC;
    else if (summary_bit(occ ? A.f_all : A.f_any, A.nbf, l, ic[0] >> kLogF, ic[1] >> kLogF, ic[2] >> kLogF) == occ)
        log = kLogF;
    if (log >= 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = (ic[a] >> log) << log;
            hi[a] = min(lo[a] + (1 << log), A.g.res) - 1;
        }
    } else if (!A.idx32) {
        return;
    }
    const int ax = exit_axis(A, R, l, lo, hi);
    if (ax < 0) return;
    const int unit = log >= 0 ? 1 << log : 1;
    // the unit across that face (selects, not a run-time array index)
    int nlo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) nlo[a] = lo[a] + (a == ax ? (R.d[a] > 0.0f ? unit : -unit) : 0);
    if (nlo[0] < 0 || nlo[0] >= A.g.res || nlo[1] < 0 || nlo[1] >= A.g.res || nlo[2] < 0 || nlo[2] >= A.g.res)
        return;
    bool same;
    if (log == kLogC)
        same = summary_bit(occ ? A.c_all : A.c_any, A.nbc, l, nlo[0] >> kLogC, nlo[1] >> kLogC, nlo[2] >> kLogC) == occ;
    else if (log == kLogF)
        same = summary_bit(occ ? A.f_all : A.f_any, A.nbf, l, nlo[0] >> kLogF, nlo[1] >> kLogF, nlo[2] >> kLogF) == occ;
    else
        same = cell_bit(A, l, nlo[0], nlo[1], nlo[2]) == occ;
    if (!same) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int nhi = min(nlo[a] + unit, A.g.res) - 1;
        lo[a] = min(lo[a], nlo[a]);
        hi[a] = max(hi[a], nhi);
    }
}

// Advance the march of one ray: append the lattice indices of its occupied
// points k < kend, in order, to buf[0..kBuf) (at most `limit` in total) and
// return when the buffer is full or the ray is finished.
__device__ void advance(const MarchArgs& A, Lane& s, int kend, int limit, int* buf, int& bn) {
    const int L = A.g.n_levels;
    while (!s.done && bn < kBuf) {
        if (s.k >= s.run_end) {  // start a new cell run at s.k
            if (s.k >= kend) {
                s.done = true;
                break;
            }
            float t0, t1, x[3];
            int l, ic[3];
            const bool occ = lattice_point(A, s.R, s.k, t0, t1, x, l, ic);
            if (!(t0 < s.R.tf)) {
                s.done = true;
                break;
            }
            if (l < L) {
                int lo[3], hi[3];
                run_box(A, s.R, l, ic, occ, lo, hi);  // a cell in a uniform block: the run spans the block
                s.run_end = skip_target(A, s.R, s.k, __fmul_rn(__fadd_rn(t0, t1), 0.5f), l, lo, hi, kend);
            } else {
                s.run_end = s.k + 1;
            }
            s.occ = occ;
            if (!occ) {
                s.k = s.run_end;
                continue;
            }
        }
        // the points of the occupied run, as many as the buffer takes (one run
        // per outer iteration keeps the run starts of the warp's lanes aligned)
        const int n_emit = min(s.run_end - s.k, kBuf - bn);
        for (int i = 0; i < n_emit; ++i) {
            const float t0 = __fadd_rn(s.R.tn, __fmul_rn((float)s.k, A.step));
            if (!(t0 < s.R.tf)) {
                s.done = true;
                break;
            }
            buf[bn++] = s.k;
            ++s.n;
            ++s.k;
            if (s.n >= limit) {
                s.done = true;
                break;
            }
        }
    }
}

// Empty-block summary of the occupancy bits: one bit per kBlk^3 block of
// cells of each level (partial blocks at the high edge when kBlk does not
// divide res), set iff any cell of the block is occupied.  Block b =
// (l*nb + bx)*nb*nb + by*nb + bz.  An acceleration structure only: a run
// that stays inside an empty block skips every cell of it.
template <int kLog>
__global__ void __launch_bounds__(256)
    k_block_summary(GridGeom g, int nb, uint32_t* __restrict__ blk, uint32_t* __restrict__ blkf) {
    constexpr int kBlk = 1 << kLog;
    const uint64_t nblocks = (uint64_t)g.n_levels * nb * nb * nb;
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false, all = b < nblocks;
    if (b < nblocks) {
        const int res = g.res;
        const uint64_t per_level = (uint64_t)nb * nb * nb;
        const int l = (int)(b / per_level);
        const uint32_t rem = (uint32_t)(b % per_level);
        const int bx = rem / (nb * nb), by = (rem / nb) % nb, bz = rem % nb;
        const int x1 = min(bx * kBlk + kBlk, res), y1 = min(by * kBlk + kBlk, res);
        const int z0 = bz * kBlk, nz = min(z0 + kBlk, res) - z0;
        const uint64_t r3 = (uint64_t)res * res * res;
        const uint64_t mask = (1ull << nz) - 1;
        for (int x = bx * kBlk; x < x1; ++x) {
            for (int y = by * kBlk; y < y1; ++y) {
                const uint64_t i0 = (uint64_t)l * r3 + ((uint64_t)x * res + y) * res + z0;
                const uint64_t w = i0 >> 5;
                const int off = (int)(i0 & 31);
                uint64_t bits = g.bits[w];
                if (off + nz > 32) bits |= (uint64_t)g.bits[w + 1] << 32;
                const uint64_t row = (bits >> off) & mask;
                any = any || row != 0;
                all = all && row == mask;
            }
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, any);
    const unsigned mf = __ballot_sync(0xffffffffu, all);
    if ((threadIdx.x & 31) == 0 && b < nblocks) {
        blk[b >> 5] = m;
        blkf[b >> 5] = mf;
    }
}

// K_end of a ray: the first lattice index k whose t0 = t_near + k dt is not
// below t_far, or max_steps (t0 is monotone in k: binary search).
__device__ __forceinline__ int lattice_end(const MarchArgs& A, const Ray& R) {
    int lo = 0, hi = A.max_steps;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__fadd_rn(R.tn, __fmul_rn((float)mid, A.step)) < R.tf)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Count pass: one thread per ray walks its cell runs up to K_end without
// visiting the points inside a run, and records the occupied runs ({first
// k, count}, merged when they continue one another) and their total.
// kstops[r] = K_end; the per-32-ray totals go to block_sums.
constexpr int kRunsThreads = 128;
__global__ void __launch_bounds__(kRunsThreads)
    k_march_runs(MarchArgs A, int32_t* __restrict__ counts, int32_t* __restrict__ kstops,
                 int32_t* __restrict__ nruns, float* __restrict__ tnear, int2* __restrict__ runs,
                 long long* __restrict__ block_sums) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * kRunsThreads + threadIdx.x;
    int cnt = 0;
    if (r < A.n) {
        Lane s;
        s.R.tn = 0.0f;
        const bool hit = lane_init(A, r, s);
        RunRec q{runs + r * kRunSlots, 0, -1, -1};
        int ke = 0;
        if (hit) {
            ke = lattice_end(A, s.R);
            const int L = A.g.n_levels;
            int k = 0;
            while (k < ke) {
                float t0, t1, x[3];
                int l, ic[3];
                const bool occ = lattice_point(A, s.R, k, t0, t1, x, l, ic);
                int run_end = k + 1;
                if (l < L) {
                    int lo[3], hi[3];
                    run_box(A, s.R, l, ic, occ, lo, hi);  // a cell in a uniform block: the run spans the block
                    run_end = skip_target(A, s.R, k, __fmul_rn(__fadd_rn(t0, t1), 0.5f), l, lo, hi, ke);
                }
                if (occ) {
                    rec_run(q, k, run_end);
                    cnt += run_end - k;
                }
                k = run_end;
            }
        }
        rec_flush(q);
        counts[r] = cnt;
        kstops[r] = ke;
        nruns[r] = q.n;
        tnear[r] = s.R.tn;
    }
    int v = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int64_t r0 = r - lane;
    if (lane == 0 && r0 < A.n) block_sums[r0 / kRaysPerBlock] = v;
}

// sigma*dt at lattice point k of the ray in the definition's arithmetic
// (early_stop.cuh): the lattice interval, its rounded midpoint and point, the
// density over the ray's exact blob list (entries that are 0 over the whole
// chunk left out), the rounded interval length; 0 for lanes without a point
// (`valid` false).  Every lane of the warp calls it.
__device__ __forceinline__ float exact_tau(const MarchArgs& A, const StopBlob* sb, const uint16_t* ex_list,
                                           int n_ex, const float o[3], const float d[3], float tn, int k, bool valid,
                                           float pos_far, int lane) {
    const float t0 = __fadd_rn(tn, __fmul_rn((float)k, A.step));
    const float t1 = __fadd_rn(t0, A.step);
    const float tm = __fmul_rn(__fadd_rn(t0, t1), 0.5f);
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
        [sb](int b) {
            const StopBlob& v = sb[b];
            return ExactBlob{v.mx, v.my, v.mz, v.coef, v.peak};
        },
        o, d, dd, dd > 0.0f ? 1.0f / dd : 0.0f, t_lo, t_hi, pos_far, lane);
    return valid ? __fmul_rn(s, __fsub_rn(t1, t0)) : 0.0f;
}

// The exact path of the early stop (early_stop.cuh): the ray's emitted
// points in lattice order, 32 at a time (from its recorded runs, or by
// walking the lattice up to K_end when the runs overflowed); each lane
// evaluates one point's sigma*dt in the definition's arithmetic into the
// warp's buffer `buf` (32 floats of shared memory), then lane 0 adds the
// terms in order one at a time -- the definition's own sum -- and finds the
// first point whose depth before it exceeds the threshold, which cuts the
// ray.  cut / kstop are left as given if the ray never stops.
__device__ __noinline__ void stop_exact(const MarchArgs& A, const StopBlob* sb, const uint16_t* ex_list, int n_ex,
                                        int64_t r, const float o[3], const float d[3], float tn, int cnt, int nr,
                                        int2 run, int ke, float pos_far, int lane, float* buf, int& cut, int& kstop) {
    int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
    for (int o2 = 1; o2 < 32; o2 <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ex, o2);
        if (lane >= o2) ex += y;
    }
    ex -= run.y;
    float P = 0.0f;  // the sequential sum (lane 0's)
    if (nr >= 0) {
        for (int p0 = 0; p0 < cnt; p0 += 32) {
            const int p = p0 + lane;
            int k = 0;
            for (int j = 0; j < nr; ++j) {
                const int ej = __shfl_sync(0xffffffffu, ex, j);
                const int kj = __shfl_sync(0xffffffffu, run.x, j);
                if (p >= ej) k = kj + (p - ej);
            }
            buf[lane] = exact_tau(A, sb, ex_list, n_ex, o, d, tn, k, p < cnt, pos_far, lane);
            __syncwarp();
            int jc = -1;
            if (lane == 0) {
                const int nv = min(32, cnt - p0);
                for (int j = 0; j < nv; ++j) {
                    if (P > A.thr) {
                        jc = j;
                        break;
                    }
                    P = __fadd_rn(P, buf[j]);
                }
            }
            jc = __shfl_sync(0xffffffffu, jc, 0);
            const int kc = __shfl_sync(0xffffffffu, k, jc < 0 ? 0 : jc);
            __syncwarp();
            if (jc >= 0) {
                cut = p0 + jc;
                kstop = kc;
                return;
            }
        }
        return;
    }
    Lane s;
    s.R.tn = 0.0f;
    lane_init(A, r, s);  // the count pass found this ray inside the grid
    int seen = 0;
    for (int kb = 0; kb < ke && seen < cnt; kb += 32) {
        const int k = kb + lane;
        bool occ = false;
        float t0 = 0.0f, t1 = 0.0f, xp[3];
        if (k < ke) {
            int l, ic[3];
            occ = lattice_point(A, s.R, k, t0, t1, xp, l, ic);
        }
        const unsigned m = __ballot_sync(0xffffffffu, occ);
        buf[lane] = exact_tau(A, sb, ex_list, n_ex, o, d, tn, k, occ, pos_far, lane);
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
        __syncwarp();
        if (jc >= 0) {
            cut = sc0;
            kstop = kb + jc;
            return;
        }
        seen = sc0;
    }
}

// The fast depth of one ray (early_stop.cuh): the ray's table (nt entries; -1:
// none, the direct form over every blob), its points in lattice order 64 at a
// time (two consecutive points per lane, from the recorded runs; a ray whose
// runs overflowed the slots walks the lattice 32 points at a time up to
// K_end), each lane adding its points' sigma dt, a warp scan giving the
// optical depth before each point.  Returns 0 if no point's fast depth comes
// within the error bound rb of the threshold (no cut), 1 if the first one
// that does passes it by more than the bound (cut / kstop set there), 2
// otherwise (undecided).
__device__ __forceinline__ int fast_cut(const MarchArgs& A, const StopBlob* s_blobs, int nblobs, const float4* tab,
                                        int nt, const RayBound& rb, int64_t r, const float o[3], const float d[3],
                                        float tn, int cnt, int nr, int2 run, int ke, int lane, int& cut, int& kstop) {
    float Q = 0.0f;  // sum of the depths before the points visited
    float carry = 0.0f;
    if (nr >= 0) {
        int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, ex, o2);
            if (lane >= o2) ex += y;
        }
        ex -= run.y;
        // four consecutive points per lane (128 per pass): each table entry
        // is read once for all four
        for (int p0 = 0; p0 < cnt; p0 += 128) {
            const int pq = p0 + 4 * lane;
            int kq[4] = {0, 0, 0, 0};
            for (int j = 0; j < nr; ++j) {
                const int ej = __shfl_sync(0xffffffffu, ex, j);
                const int kj = __shfl_sync(0xffffffffu, run.x, j);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (pq + u >= ej) kq[u] = kj + (pq + u - ej);
            }
            float t0[4], t1[4], tm[4], sg[4] = {0.0f, 0.0f, 0.0f, 0.0f}, tau[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = pq + u < cnt ? kq[u] : kq[0];
                t0[u] = __fadd_rn(tn, __fmul_rn((float)k, A.step));
                t1[u] = __fadd_rn(t0[u], A.step);
                tm[u] = __fmul_rn(__fadd_rn(t0[u], t1[u]), 0.5f);
            }
            if (nt > 0 && nt <= kGroupMin) {
                if (pq < cnt) sigma_tab4(tab, nt, tm, sg);
            } else if (nt > 0) {  // the pass's midpoints span [first, last] (lattice order)
                const int last = min(cnt - p0, 128) - 1, ll = last >> 2, lu = last & 3;
                const float t_lo = __shfl_sync(0xffffffffu, tm[0], 0);
                const float tm_l = lu == 0 ? tm[0] : lu == 1 ? tm[1] : lu == 2 ? tm[2] : tm[3];
                const float t1_l = lu == 0 ? t1[0] : lu == 1 ? t1[1] : lu == 2 ? t1[2] : t1[3];
                const float t_hi = __shfl_sync(0xffffffffu, tm_l, ll);
                const float t_end = __shfl_sync(0xffffffffu, t1_l, ll);
                const float span = t_end - __shfl_sync(0xffffffffu, t0[0], 0);
                sigma_tab4_group(tab, nt, t_lo, t_hi, span, tm, sg, pq < cnt);
            }
            if (pq < cnt && nt < 0) {
#pragma unroll
                for (int u = 0; u < 4; u += 2) {
                    float xa[3], xb[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        xa[a] = fmaf(d[a], tm[u], o[a]);
                        xb[a] = fmaf(d[a], tm[u + 1], o[a]);
                    }
                    sigma_early_stop2(s_blobs, nblobs, xa, xb, sg[u], sg[u + 1]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) tau[u] = pq + u < cnt ? __fmul_rn(sg[u], __fsub_rn(t1[u], t0[u])) : 0.0f;
            const float l1 = tau[0], l2 = l1 + tau[1], l3 = l2 + tau[2], quad = l3 + tau[3];
            float x = quad;  // -> inclusive prefix over the lanes' quads
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, x, o2);
                if (lane >= o2) x += y;
            }
            float before[4];
            before[0] = carry + (x - quad);
            before[1] = before[0] + tau[0];
            before[2] = before[1] + tau[1];
            before[3] = before[2] + tau[2];
            float qs = 0.0f;
#pragma unroll
            for (int u = 0; u < 4; ++u) qs += pq + u < cnt ? before[u] : 0.0f;
            const float Qc = Q + warp_sum(qs);
            const float lo_thr = A.thr - depth_error(rb, cnt, Qc, A.thr);
            int first = 128;  // the first point near or past the threshold, in lattice order
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const unsigned ov = __ballot_sync(0xffffffffu, pq + u < cnt && before[u] > lo_thr);
                if (ov) first = min(first, 4 * (__ffs(ov) - 1) + u);
            }
            if (first < 128) {
                const int jl = first >> 2, ju = first & 3;
                const float bsel = ju == 0 ? before[0] : ju == 1 ? before[1] : ju == 2 ? before[2] : before[3];
                const int ksel = ju == 0 ? kq[0] : ju == 1 ? kq[1] : ju == 2 ? kq[2] : kq[3];
                const float bc = __shfl_sync(0xffffffffu, bsel, jl);
                const int kc = __shfl_sync(0xffffffffu, ksel, jl);
                if (bc - depth_error(rb, cnt, Qc, bc) > A.thr) {
                    cut = p0 + first;
                    kstop = kc;
                    return 1;
                }
                return 2;
            }
            Q = Qc;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    } else {
        Lane s;
        s.R.tn = 0.0f;
        lane_init(A, r, s);  // the count pass found this ray inside the grid
        int seen = 0;
        for (int kb = 0; kb < ke && seen < cnt; kb += 32) {
            const int k = kb + lane;
            bool occ = false;
            float t0 = 0.0f, t1 = 0.0f, xp[3];
            if (k < ke) {
                int l, ic[3];
                occ = lattice_point(A, s.R, k, t0, t1, xp, l, ic);
            }
            const unsigned m = __ballot_sync(0xffffffffu, occ);
            if (!m) continue;
            float tau = 0.0f;
            if (occ) {
                const float tm = __fmul_rn(__fadd_rn(t0, t1), 0.5f);
                float sg, unused;
                if (nt >= 0) {
                    sigma_tab2(tab, nt, tm, tm, sg, unused);
                } else {
                    float xa[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) xa[a] = fmaf(d[a], tm, o[a]);
                    sigma_early_stop2(s_blobs, nblobs, xa, xa, sg, unused);
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

// Early termination (with a field, after the count pass): each warp takes
// the 32 rays of one block-sum entry in turn and decides each ray's cut as
// early_stop.cuh describes: no density at all when the ray's depth bound
// stays below the threshold; else the fast depth -- the ray's table, its
// points in lattice order 64 at a time (two consecutive points per lane, from
// the recorded runs; a ray whose runs overflowed the slots walks the lattice
// 32 points at a time up to K_end), each lane adding its points' sigma dt, a
// warp scan giving the optical depth before each point -- and the cut at the
// first point whose fast depth passes the threshold by more than the bound;
// else (a fast depth within the bound of the threshold, or A.exact_all) the
// exact path.  counts[r] and kstops[r] (the cut's lattice index) are
// rewritten, and so is the entry's total.
constexpr int kStopThreads = 128;
constexpr int kStopWarps = kStopThreads / 32;
__global__ void __launch_bounds__(kStopThreads, 7)
    k_march_stop(MarchArgs A, int32_t* __restrict__ counts, int32_t* __restrict__ kstops,
                 const int32_t* __restrict__ nruns, const float* __restrict__ tnear,
                 const int2* __restrict__ runs, long long* __restrict__ block_sums,
                 unsigned long long* __restrict__ ticket, long long* __restrict__ queue,
                 unsigned long long* __restrict__ qlen) {
    extern __shared__ StopBlob s_blobs[];
    constexpr int kTabWarp = kTab > 32 * kSmallBlobs ? kTab : 32 * kSmallBlobs;
    __shared__ float4 s_tab[kStopWarps][kTabWarp];  // one ray's table, or a small field's 32
    __shared__ uint16_t s_tidx[kStopWarps][kTabWarp];
    __shared__ float s_U[kStopWarps][32], s_eo[kStopWarps][32], s_ek[kStopWarps][32], s_eps[kStopWarps][32];
    __shared__ int s_nt[kStopWarps][32];
    stage_stop_blobs(s_blobs, A.field);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* tab = s_tab[wid];
    uint16_t* tidx = s_tidx[wid];
    const int nblobs = A.field.n_blobs;
    const int64_t n_entries = (A.n + kRaysPerBlock - 1) / kRaysPerBlock;
    for (;;) {  // entries of 32 rays by ticket: rays that stop cost far more than rays that cannot
        unsigned long long tk = 0;
        if (lane == 0) tk = atomicAdd(ticket, 1ull);
        const int64_t cb = (int64_t)__shfl_sync(0xffffffffu, tk, 0);  // this warp's block-sum entry
        if (cb >= n_entries) break;
        const int64_t rbase = cb * kRaysPerBlock;
        // lane i loads the header of ray rbase + i (coalesced); the rays are then
        // taken in turn, their values broadcast by shuffles, and lane i keeps the
        // results of ray i
        const int64_t rl = rbase + lane;
        const bool lv = rl < A.n;
        const int l_cnt = lv ? counts[rl] : 0;
        const int l_nr = lv ? nruns[rl] : 0;
        const float l_tn = lv ? tnear[rl] : 0.0f;
        const int l_ke = lv ? kstops[rl] : 0;
        float l_o[3], l_d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            l_o[a] = lv ? __ldg(A.o + 3 * rl + a) : 0.0f;
            l_d[a] = lv ? __ldg(A.d + 3 * rl + a) : 0.0f;
        }
        int l_cut = l_cnt, l_kstop = l_ke;
        unsigned todo = __ballot_sync(0xffffffffu, l_cnt > 0);
        const bool small = nblobs <= kSmallBlobs;  // every ray's table built up front, 8 lanes per ray
        if (small && todo)
            build_entry_tables(s_blobs, nblobs, l_o, l_d, l_cnt, l_tn, l_ke, A.step, A.exact_all != 0, A.thr, tab, tidx,
                               s_U[wid], s_eo[wid], s_nt[wid], s_ek[wid], s_eps[wid], lane);
        // the next ray's runs are loaded while the current one is evaluated
        int2 run_next = make_int2(0, 0);
        if (todo) {
            const int i0 = __ffs(todo) - 1;
            if (lane < __shfl_sync(0xffffffffu, l_nr, i0)) run_next = runs[(rbase + i0) * kRunSlots + lane];
        }
        while (todo) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t r = rbase + i;
            const int cnt = __shfl_sync(0xffffffffu, l_cnt, i);
            const int nr = __shfl_sync(0xffffffffu, l_nr, i);
            const float tn = __shfl_sync(0xffffffffu, l_tn, i);
            const int ke = __shfl_sync(0xffffffffu, l_ke, i);
            float o[3], d[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o[a] = __shfl_sync(0xffffffffu, l_o[a], i);
                d[a] = __shfl_sync(0xffffffffu, l_d[a], i);
            }
            const int2 run = run_next;
            if (todo) {
                const int in = __ffs(todo) - 1;
                run_next = lane < __shfl_sync(0xffffffffu, l_nr, in) ? runs[(rbase + in) * kRunSlots + lane]
                                                                    : make_int2(0, 0);
            }
            // bounds of the ray (every sample's midpoint lies before t_near + (K_end + 1) dt)
            const float tmax = fabsf(tn) + (float)(ke + 1) * A.step * 1.0001f;
            const float onorm = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) * 1.0001f;
            const float dnorm = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) * 1.0001f;
            int cut = cnt, kstop = ke;
            float U, e_out;
            int nk;
            float4* tab_r = tab;
            uint16_t* tidx_r = tidx;
            if (small) {
                tab_r = tab + i * kSmallBlobs;
                tidx_r = tidx + i * kSmallBlobs;
                nk = s_nt[wid][i];
                U = s_U[wid][i];
                e_out = s_eo[wid][i];
            } else {
                nk = build_ray_table(s_blobs, nblobs, o, d, onorm, dnorm, tmax, A.step, cnt, tab, tidx, U, e_out, lane);
            }
            if (A.exact_all != 0 || !(depth_upper(U, cnt, nblobs) <= A.thr)) {  // the ray may stop
                __syncwarp();
                const int nt = nk <= kTab ? nk : -1;
                const float e_grp = nt > kGroupMin ? 2.0f * kGroupEps * (float)nt * (float)((cnt + 63) / 64) : 0.0f;
                // the refined table and its (tight) error bound
                float eps;
                const float ek = small ? s_ek[wid][i]
                                       : refine_ray_table(s_blobs, nblobs, nk, o, d, onorm, dnorm, tmax, A.step, cnt,
                                                          tab_r, tidx_r, eps, lane);
                if (small) eps = s_eps[wid][i];
                const RayBound rb{U, ek, eps, e_out + e_grp};
                __syncwarp();
                const int st = A.exact_all != 0 || !bounds_usable(rb, cnt, A.thr)
                                   ? 2
                                   : fast_cut(A, s_blobs, nblobs, tab_r, nt, rb, r, o, d, tn, cnt, nr, run, ke, lane,
                                              cut, kstop);
                const bool exact = st == 2;
                if (exact && lane == 0) queue[atomicAdd(qlen, 1ull)] = r;  // decided exactly by k_march_stop_exact
            }
            if (lane == i) {
                l_cut = cut;
                l_kstop = kstop;
            }
            __syncwarp();  // the next ray rewrites the table
        }
        if (lv) {
            counts[rl] = l_cut;
            kstops[rl] = l_kstop;
        }
        int wsum = l_cut;
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, o2);
        if (lane == 0) block_sums[cb] = wsum;
    }
}

// Exact decisions of the rays the early-stop pass queued (early_stop.cuh):
// persistent CTAs take queued rays one at a time (ticket `qhead` over the
// `*qlen` entries); warp 0 builds the ray's exact blob list, then the four
// warps evaluate the definition's sigma*dt at 128 consecutive points at a
// time (32 each, exact_tau) into shared memory and thread 0 adds them in
// order one at a time -- the definition's own sum -- stopping at the first
// point whose depth before it exceeds the threshold.  Rays whose runs
// overflowed walk the lattice on warp 0 alone (stop_exact).  The cut and its
// lattice index replace the ray's count and K_end, and the change of the
// count is added to its 32-ray entry's total.
__global__ void __launch_bounds__(kStopThreads)
    k_march_stop_exact(MarchArgs A, int32_t* __restrict__ counts, int32_t* __restrict__ kstops,
                       const int32_t* __restrict__ nruns, const float* __restrict__ tnear,
                       const int2* __restrict__ runs, long long* __restrict__ block_sums,
                       const long long* __restrict__ queue, const unsigned long long* __restrict__ qlen,
                       unsigned long long* __restrict__ qhead) {
    extern __shared__ StopBlob s_blobs[];
    __shared__ uint16_t s_ex[kMaxBlobs];
    __shared__ __align__(16) float s_tau[kStopThreads];
    __shared__ int s_k[kStopThreads];
    __shared__ float s_seq[32];
    __shared__ unsigned long long s_tk;
    __shared__ int s_nex, s_jc;
    stage_stop_blobs(s_blobs, A.field);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long nq = *qlen;
    for (;;) {
        if (threadIdx.x == 0) s_tk = atomicAdd(qhead, 1ull);
        __syncthreads();
        const unsigned long long tk = s_tk;
        if (tk >= nq) break;  // the same for the whole CTA
        const int64_t r = queue[tk];
        const int cnt = counts[r], nr = nruns[r], ke = kstops[r];
        const float tn = tnear[r];
        float o[3], d[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = __ldg(A.o + 3 * r + a);
            d[a] = __ldg(A.d + 3 * r + a);
        }
        const int2 run = (nr >= 0 && lane < nr) ? runs[r * kRunSlots + lane] : make_int2(0, 0);
        const float tmax = fabsf(tn) + (float)(ke + 1) * A.step * 1.0001f;
        const float pos_far = (sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]) +
                               tmax * sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])) * 1.0002f;
        if (wid == 0) {
            const int n = build_exact_list(s_blobs, A.field.n_blobs, o, d, pos_far, s_ex, lane);
            if (lane == 0) s_nex = n;
        }
        __syncthreads();
        const int n_ex = s_nex;
        int cut = cnt, kstop = ke;
        if (nr >= 0) {
            int ex = run.y;  // -> exclusive prefix of the run lengths
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, ex, o2);
                if (lane >= o2) ex += y;
            }
            ex -= run.y;
            float P = 0.0f;  // the sequential sum (thread 0's)
            for (int pr = 0; pr < cnt; pr += kStopThreads) {
                const int p = pr + (int)threadIdx.x;
                int k = 0;
                for (int j = 0; j < nr; ++j) {
                    const int ej = __shfl_sync(0xffffffffu, ex, j);
                    const int kj = __shfl_sync(0xffffffffu, run.x, j);
                    if (p >= ej) k = kj + (p - ej);
                }
                s_tau[threadIdx.x] = exact_tau(A, s_blobs, s_ex, n_ex, o, d, tn, k, p < cnt, pos_far, lane);
                s_k[threadIdx.x] = k;
                __syncthreads();
                if (threadIdx.x == 0) s_jc = seq_depth_cut<kStopThreads>(s_tau, min(kStopThreads, cnt - pr), A.thr, P);
                __syncthreads();
                const int jc = s_jc;
                if (jc >= 0) {
                    cut = pr + jc;
                    kstop = s_k[jc];
                    break;
                }
            }
        } else if (wid == 0) {  // runs overflowed: the lattice walk, on one warp
            stop_exact(A, s_blobs, s_ex, n_ex, r, o, d, tn, cnt, nr, run, ke, pos_far, lane, s_seq, cut, kstop);
        }
        if (threadIdx.x == 0) {
            counts[r] = cut;
            kstops[r] = kstop;
            if (cut != cnt)
                atomicAdd(reinterpret_cast<unsigned long long*>(block_sums + r / kRaysPerBlock),
                          (unsigned long long)(long long)(cut - cnt));
        }
        __syncthreads();  // the next ray rewrites the list, the buffers and the ticket
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
            s_w[lane] = w;  // inclusive over warps
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

// A warp's re-marched rays (lane flag `mine`): each such lane walks its ray
// up to the recorded stop kend, emitting cnt points from offset pos into its
// buffer `buf` (row of wbuf), which the whole warp flushes, lane by lane.
__device__ __forceinline__ void fill_long_group(const MarchArgs& A, int64_t r, bool mine, int cnt, int kend,
                                                long long pos, int* buf, const int (*wbuf)[kBuf + 1],
                                                int32_t* __restrict__ ray_idx, float* __restrict__ t0s,
                                                float* __restrict__ t1s) {
    const int lane = threadIdx.x & 31;
    Lane s;
    s.done = true;
    s.R.tn = 0.0f;
    if (mine) lane_init(A, r, s);
    while (true) {
        int bn = 0;
        if (!s.done) advance(A, s, kend, cnt, buf, bn);
        __syncwarp();
        unsigned m = __ballot_sync(0xffffffffu, bn > 0);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const int nj = __shfl_sync(0xffffffffu, bn, j);
            const long long pj = __shfl_sync(0xffffffffu, pos, j);
            const int rj = __shfl_sync(0xffffffffu, (int)r, j);
            const float tnj = __shfl_sync(0xffffffffu, s.R.tn, j);
            if (lane < nj) {
                const int k = wbuf[j][lane];
                const float t0 = __fadd_rn(tnj, __fmul_rn((float)k, A.step));
                t0s[pj + lane] = t0;
                t1s[pj + lane] = __fadd_rn(t0, A.step);
                if (ray_idx) ray_idx[pj + lane] = rj;
            }
        }
        __syncwarp();
        pos += bn;
        if (__all_sync(0xffffffffu, s.done)) break;
    }
}

// Expansion of a ray whose runs were recorded (whole warp; run = slot `lane`
// of its record, or zero): sample p of the ray is point p of its
// concatenated ranges.  Lane l writes positions q..q+3 of the sample arrays,
// q = 4l + a multiple of 128 from pj rounded down to a multiple of 4: groups
// of four inside the ray as one 128-bit store per array, the ray's ragged
// head and tail position by position (nothing outside the ray is written).
__device__ __forceinline__ void fill_runs(const MarchArgs& A, int64_t r, int cj, long long pj, int nr, float tn,
                                          int2 run, int32_t* __restrict__ ray_idx, float* __restrict__ t0s,
                                          float* __restrict__ t1s) {
    const int lane = threadIdx.x & 31;
    if (lane >= nr) run = make_int2(0, 0);
    int ex = run.y;  // -> exclusive prefix of the range lengths
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, ex, o);
        if (lane >= o) ex += y;
    }
    ex -= run.y;
    const long long a4 = pj & ~3ll, pend = pj + cj;
    for (long long q0 = a4; q0 < pend; q0 += 128) {
        const long long q = q0 + 4 * lane;
        const int p0 = (int)(q - pj);  // sample index of position q within the ray (may be < 0)
        int k[4] = {p0, p0 + 1, p0 + 2, p0 + 3};
        for (int i = 0; i < nr; ++i) {
            const int ei = __shfl_sync(0xffffffffu, ex, i);
            const int ki = __shfl_sync(0xffffffffu, run.x, i);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (p0 + u >= ei) k[u] = ki + (p0 + u - ei);
        }
        float t0[4], t1[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            t0[u] = __fadd_rn(tn, __fmul_rn((float)k[u], A.step));
            t1[u] = __fadd_rn(t0[u], A.step);
        }
        if (q >= pj && q + 4 <= pend) {
            __stcs(reinterpret_cast<float4*>(t0s + q), make_float4(t0[0], t0[1], t0[2], t0[3]));
            __stcs(reinterpret_cast<float4*>(t1s + q), make_float4(t1[0], t1[1], t1[2], t1[3]));
            if (ray_idx) __stcs(reinterpret_cast<int4*>(ray_idx + q), make_int4((int)r, (int)r, (int)r, (int)r));
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (q + u < pj || q + u >= pend) continue;
                t0s[q + u] = t0[u];
                t1s[q + u] = t1[u];
                if (ray_idx) ray_idx[q + u] = (int)r;
            }
        }
    }
}

// Fill pass: each warp takes kFillRays consecutive rays, the blocks in ray
// order, so that the warps in flight write neighbouring stretches of the
// packed arrays (scattered concurrent write streams cost DRAM efficiency).
// All loads of the warp's rays are issued before the first is used; the
// rays' CSR offsets come from their 32-ray entry's start and the counts
// before them.  A ray whose runs were recorded is expanded from them
// (fill_runs); a ray whose runs overflowed the slots is re-marched by lane 0
// up to its recorded stop, without the field, and flushed by the whole warp.
// Four-warp blocks at 40 registers keep 48 warps per SM (32 or 64 per SM
// measured slower: too few rays in flight, or spills in the expansion).
constexpr int kFillWarps = 4;
constexpr int kFillRays = 1;  // 2 and 4 measured slower (registers spill around the re-march)
static_assert(32 % kFillRays == 0, "a warp's rays share one 32-ray entry");
__global__ void __launch_bounds__(kFillWarps * 32, 12)
    k_march_fill(MarchArgs A, const int32_t* __restrict__ counts, const int32_t* __restrict__ kstops,
                 const int32_t* __restrict__ nruns, const float* __restrict__ tnear,
                 const int2* __restrict__ runs, const long long* __restrict__ block_off,
                 const int64_t* __restrict__ n_samples, int64_t capacity, int64_t* __restrict__ offsets,
                 int32_t* __restrict__ ray_idx, float* __restrict__ t0s, float* __restrict__ t1s) {
    __shared__ int s_lb[kFillWarps][kBuf + 1];  // lattice indices of a re-marched ray
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t r0 = ((int64_t)blockIdx.x * kFillWarps + wid) * kFillRays;
    if (r0 >= A.n) return;  // whole warp
    const int64_t g0 = r0 & ~31ll;
    const int j0 = (int)(r0 - g0);
    const int c = g0 + lane < A.n ? counts[g0 + lane] : 0;
    const long long base = block_off[g0 / kRaysPerBlock];
    const bool hl = lane < kFillRays && r0 + lane < A.n;  // lane i holds ray r0 + i's header
    const int nr_l = hl ? nruns[r0 + lane] : 0;
    const float tn_l = hl ? tnear[r0 + lane] : 0.0f;
    int2 run0[kFillRays];
#pragma unroll
    for (int i = 0; i < kFillRays; ++i)
        run0[i] = lane < kRunSlots && r0 + i < A.n ? runs[(r0 + i) * kRunSlots + lane] : make_int2(0, 0);
    const bool over = *n_samples > capacity;
    int x = c;  // -> inclusive prefix of the entry's counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
#pragma unroll
    for (int i = 0; i < kFillRays; ++i) {
        const int64_t r = r0 + i;
        if (r >= A.n) break;  // whole warp
        const int cj = __shfl_sync(0xffffffffu, c, j0 + i);
        const long long pj = base + (__shfl_sync(0xffffffffu, x, j0 + i) - cj);
        const int nr = __shfl_sync(0xffffffffu, nr_l, i);
        const float tn = __shfl_sync(0xffffffffu, tn_l, i);
        if (lane == 0) offsets[r] = pj;
        if (over || cj == 0) continue;  // overflow: offsets only (the whole grid agrees)
        if (nr < 0)
            fill_long_group(A, r, lane == 0, cj, kstops[r], pj, s_lb[wid], &s_lb[wid], ray_idx, t0s, t1s);
        else
            fill_runs(A, r, cj, pj, nr, tn, run0[i], ray_idx, t0s, t1s);
    }
}

// The occupied range of each ray for the combined estimator: t0 of its first
// and t1 of its last occupied lattice point (the march's emitted set
// without a field: the same lattice definition).  Walks cell runs only (the
// block summaries skip empty and fully occupied blocks) and never emits a
// point: the last occupied point of a run is min(run end, K_end) - 1 with
// K_end the first lattice index that is not visited (t0 >= t_far or
// max_steps).  A ray with no occupied point gets t_lo = t_hi = t_near
// (max(t_min, 0) if it misses).
__global__ void __launch_bounds__(kBlockThreads) k_occupied_range(MarchArgs A, float* __restrict__ t_lo,
                                                                  float* __restrict__ t_hi) {
    const int64_t r = (int64_t)blockIdx.x * kBlockThreads + threadIdx.x;
    if (r >= A.n) return;
    Lane s;
    const bool hit = lane_init(A, r, s);
    int first = -1, last = -1;
    if (hit) {
        const int ke = lattice_end(A, s.R);
        const int L = A.g.n_levels;
        int k = 0;
        while (k < ke) {
            float t0, t1, x[3];
            int l, ic[3];
            const bool occ = lattice_point(A, s.R, k, t0, t1, x, l, ic);
            int run_end = k + 1;
            if (l < L) {
                int lo[3], hi[3];
                run_box(A, s.R, l, ic, occ, lo, hi);
                run_end = skip_target(A, s.R, k, __fmul_rn(__fadd_rn(t0, t1), 0.5f), l, lo, hi, ke);
            }
            if (occ) {
                if (first < 0) first = k;
                last = min(run_end, ke) - 1;
            }
            k = run_end;
        }
    }
    if (first < 0) {
        const float t = hit ? s.R.tn : fmaxf(A.t_min, 0.0f);
        t_lo[r] = t;
        t_hi[r] = t;
    } else {
        t_lo[r] = __fadd_rn(s.R.tn, __fmul_rn((float)first, A.step));
        t_hi[r] = __fadd_rn(__fadd_rn(s.R.tn, __fmul_rn((float)last, A.step)), A.step);
    }
}

// The coarse summary from the fine one: a coarse block is any- (all-)
// occupied iff any (every) fine block inside it is; fine blocks past the
// grid's edge do not exist.
__global__ void __launch_bounds__(256)
    k_coarse_summary(int n_levels, int nbc, int nbf, const uint32_t* __restrict__ f_any,
                     const uint32_t* __restrict__ f_all, uint32_t* __restrict__ c_any, uint32_t* __restrict__ c_all) {
    constexpr int kR = 1 << (kLogC - kLogF);  // fine blocks per coarse block edge
    const uint64_t ncb = (uint64_t)n_levels * nbc * nbc * nbc;
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false, all = b < ncb;
    if (b < ncb) {
        const uint64_t per_level = (uint64_t)nbc * nbc * nbc;
        const int l = (int)(b / per_level);
        const uint32_t rem = (uint32_t)(b % per_level);
        const int bx = rem / (nbc * nbc), by = (rem / nbc) % nbc, bz = rem % nbc;
        for (int x = bx * kR; x < min(bx * kR + kR, nbf); ++x)
            for (int y = by * kR; y < min(by * kR + kR, nbf); ++y)
                for (int z = bz * kR; z < min(bz * kR + kR, nbf); ++z) {
                    const uint32_t f = (((uint32_t)l * nbf + x) * nbf + y) * nbf + z;
                    any = any || ((__ldg(&f_any[f >> 5]) >> (f & 31)) & 1u);
                    all = all && ((__ldg(&f_all[f >> 5]) >> (f & 31)) & 1u);
                }
    }
    const unsigned m = __ballot_sync(0xffffffffu, any);
    const unsigned mf = __ballot_sync(0xffffffffu, all);
    if ((threadIdx.x & 31) == 0 && b < ncb) {
        c_any[b >> 5] = m;
        c_all[b >> 5] = mf;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Points A's block summaries into `mem` (kBlockBitsBytes) and rebuilds them from the bits.
int build_summaries(MarchArgs& A, void* mem, cudaStream_t st) {
    char* p = static_cast<char*>(mem);
    uint32_t* c_any = reinterpret_cast<uint32_t*>(p);
    uint32_t* c_all = reinterpret_cast<uint32_t*>(p + summary_bytes(kLogC));
    uint32_t* f_any = reinterpret_cast<uint32_t*>(p + 2 * summary_bytes(kLogC));
    uint32_t* f_all = reinterpret_cast<uint32_t*>(p + 2 * summary_bytes(kLogC) + summary_bytes(kLogF));
    A.nbc = (A.g.res + (1 << kLogC) - 1) >> kLogC;
    A.nbf = (A.g.res + (1 << kLogF) - 1) >> kLogF;
    A.c_any = c_any;
    A.c_all = c_all;
    A.f_any = f_any;
    A.f_all = f_all;
    const uint64_t nfb = (uint64_t)A.g.n_levels * A.nbf * A.nbf * A.nbf;
    k_block_summary<kLogF><<<(unsigned)((nfb + 255) / 256), 256, 0, st>>>(A.g, A.nbf, f_any, f_all);
    NACC_LAUNCH_CHECK();
    const uint64_t ncb = (uint64_t)A.g.n_levels * A.nbc * A.nbc * A.nbc;
    k_coarse_summary<<<(unsigned)((ncb + 255) / 256), 256, 0, st>>>(A.g.n_levels, A.nbc, A.nbf, f_any, f_all, c_any,
                                                                     c_all);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

}  // namespace
}  // namespace nacc

using namespace nacc;

extern "C" size_t nacc_march_scratch_bytes(int64_t n_rays) {
    if (n_rays < 0) return 0;
    const int64_t nb = (n_rays + kRaysPerBlock - 1) / kRaysPerBlock;
    // counts, kstops, nruns, tnear, block sums, run slots
    return align256(4 * (size_t)n_rays) * 4 + align256(8 * (size_t)(nb > 0 ? nb : 1)) +
           align256(sizeof(int2) * kRunSlots * (size_t)n_rays) + kBlockBitsBytes + 256 +  // + work tickets
           align256(8 * (size_t)n_rays);                                                       // + exact queue
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
    const size_t need = nacc_march_scratch_bytes(n_rays);
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
    A.exact_all = params->exact_stops != 0 ? 1 : 0;
    A.inv_step = 1.0f / params->step;
    A.idx32 = ((uint64_t)A.g.n_levels * A.g.res * A.g.res * A.g.res) <= 0xffffffffull ? 1 : 0;
    A.field = with_field ? *field : nacc_blob_field{0, nullptr, nullptr, nullptr, nullptr};
    for (int l = 0; l < NACC_MAX_LEVELS; ++l) {
        A.skip_lim[l] = -1.0f;  // never skip
        if (l >= A.g.n_levels) continue;
        const Level& lv = A.g.lv[l];
        double wmin = INFINITY, xmax = 0.0;
        for (int a = 0; a < 3; ++a) {
            wmin = std::fmin(wmin, (double)lv.width[a]);
            xmax = std::fmax(xmax, std::fmax(std::fabs((double)lv.lmin[a]), std::fabs((double)lv.lmax[a])));
        }
        const double lim = (wmin * kSkipMargin / (16.0 * 0x1p-24) - 15.0 * xmax) / 11.0;
        if (lim > 0.0) A.skip_lim[l] = (float)lim;
    }

    char* sp = static_cast<char*>(scratch);
    int32_t* counts = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int32_t* kstops = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    int32_t* nruns = reinterpret_cast<int32_t*>(sp);
    sp += align256(4 * (size_t)n_rays);
    float* tnear = reinterpret_cast<float*>(sp);
    sp += align256(4 * (size_t)n_rays);
    long long* bsums = reinterpret_cast<long long*>(sp);
    sp += align256(8 * (size_t)((n_rays + kRaysPerBlock - 1) / kRaysPerBlock));
    int2* runs = reinterpret_cast<int2*>(sp);
    sp += align256(sizeof(int2) * kRunSlots * (size_t)n_rays);
    const int64_t nb = (n_rays + kRaysPerBlock - 1) / kRaysPerBlock;
    NACC_CHECK_ARG(nb < (int64_t(1) << 31), "too many rays for one launch");
    {
        const int rc = build_summaries(A, sp, st);
        if (rc != NACC_OK) return rc;
    }
    if (cudaEvent_t e = march_count_events()[0]) NACC_CUDA_TRY(cudaEventRecord(e, st));
    k_march_runs<<<(unsigned)((n_rays + kRunsThreads - 1) / kRunsThreads), kRunsThreads, 0, st>>>(
        A, counts, kstops, nruns, tnear, runs, bsums);
    NACC_LAUNCH_CHECK();
    if (with_field) {
        const size_t shm = sizeof(StopBlob) * (size_t)A.field.n_blobs;
        if (shm > 32 * 1024)
            NACC_CUDA_TRY(cudaFuncSetAttribute(k_march_stop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        // persistent warps taking 32-ray entries by ticket; rays they cannot
        // decide from bounds go to a queue decided exactly by a second kernel
        unsigned long long* tickets = reinterpret_cast<unsigned long long*>(sp + kBlockBitsBytes);  // ticket, qlen, qhead
        long long* queue = reinterpret_cast<long long*>(sp + kBlockBitsBytes + 256);
        NACC_CUDA_TRY(cudaMemsetAsync(tickets, 0, 3 * sizeof(unsigned long long), st));
        int per_sm = 0;
        NACC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march_stop, kStopThreads, shm));
        const int64_t want = (nb + kStopWarps - 1) / kStopWarps;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * std::max(per_sm, 1)));
        k_march_stop<<<(unsigned)blocks, kStopThreads, shm, st>>>(A, counts, kstops, nruns, tnear, runs, bsums,
                                                                   tickets, queue, tickets + 1);
        NACC_LAUNCH_CHECK();
        if (shm > 32 * 1024 - 8192)
            NACC_CUDA_TRY(cudaFuncSetAttribute(k_march_stop_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)shm));
        int per_sm_x = 0;
        NACC_CUDA_TRY(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, k_march_stop_exact, kStopThreads, shm));
        const int64_t blocks_x = std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * std::max(per_sm_x, 1)));
        k_march_stop_exact<<<(unsigned)blocks_x, kStopThreads, shm, st>>>(A, counts, kstops, nruns, tnear, runs, bsums,
                                                                           queue, tickets + 1, tickets + 2);
        NACC_LAUNCH_CHECK();
    }
    if (cudaEvent_t e = march_count_events()[1]) NACC_CUDA_TRY(cudaEventRecord(e, st));
    k_scan_block_sums<<<1, 1024, 0, st>>>(bsums, nb, out->offsets + n_rays, out->n_samples);
    NACC_LAUNCH_CHECK();
    k_march_fill<<<(unsigned)((n_rays + kFillWarps * kFillRays - 1) / (kFillWarps * kFillRays)), kFillWarps * 32, 0,
                   st>>>(
        A, counts, kstops, nruns, tnear, runs, bsums, out->n_samples, out->capacity, out->offsets, out->ray_indices,
        out->t_starts, out->t_ends);
    NACC_LAUNCH_CHECK();
    // Overflow is impossible when the capacity covers every lattice point.
    const bool may_overflow = (double)out->capacity < (double)n_rays * (double)params->max_steps;
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

extern "C" size_t nacc_occupied_range_scratch_bytes(void) { return kBlockBitsBytes; }

extern "C" int nacc_occupied_range(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                                   const nacc_march_params* params, float* t_lo, float* t_hi, void* scratch,
                                   size_t scratch_bytes, void* stream) {
    clear_error();
    MarchArgs A;
    if (!make_geom(grid, &A.g, true)) return NACC_ERR_INVALID_ARG;
    NACC_CHECK_ARG(params != nullptr, "params is NULL");
    NACC_CHECK_ARG(n_rays >= 0 && n_rays < (int64_t(1) << 40), "n_rays=%lld out of range", (long long)n_rays);
    NACC_CHECK_ARG(params->step > 0.0f && std::isfinite(params->step), "step must be finite and > 0");
    NACC_CHECK_ARG(params->max_steps >= 1 && params->max_steps <= (1 << 24), "max_steps=%d outside [1, 2^24]",
                   params->max_steps);
    NACC_CHECK_ARG(!std::isnan(params->t_min) && !std::isnan(params->t_max), "t_min/t_max is NaN");
    if (n_rays == 0) return NACC_OK;
    NACC_CHECK_ARG(rays_o && rays_d && t_lo && t_hi, "a pointer argument is NULL");
    NACC_CHECK_ARG(scratch != nullptr && scratch_bytes >= kBlockBitsBytes, "scratch too small: %zu < %zu bytes",
                   scratch_bytes, kBlockBitsBytes);
    NACC_CHECK_ARG((reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "scratch not 256-byte aligned");
    A.o = rays_o;
    A.d = rays_d;
    A.n = n_rays;
    A.step = params->step;
    A.max_steps = params->max_steps;
    A.t_min = params->t_min;
    A.t_max = params->t_max;
    A.thr = INFINITY;
    A.exact_all = 0;
    A.inv_step = 1.0f / params->step;
    A.idx32 = ((uint64_t)A.g.n_levels * A.g.res * A.g.res * A.g.res) <= 0xffffffffull ? 1 : 0;
    A.field = nacc_blob_field{0, nullptr, nullptr, nullptr, nullptr};
    for (int l = 0; l < NACC_MAX_LEVELS; ++l) {
        A.skip_lim[l] = -1.0f;
        if (l >= A.g.n_levels) continue;
        const Level& lv = A.g.lv[l];
        double wmin = INFINITY, xmax = 0.0;
        for (int a = 0; a < 3; ++a) {
            wmin = std::fmin(wmin, (double)lv.width[a]);
            xmax = std::fmax(xmax, std::fmax(std::fabs((double)lv.lmin[a]), std::fabs((double)lv.lmax[a])));
        }
        const double lim = (wmin * kSkipMargin / (16.0 * 0x1p-24) - 15.0 * xmax) / 11.0;
        if (lim > 0.0) A.skip_lim[l] = (float)lim;
    }
    const int64_t nb = (n_rays + kBlockThreads - 1) / kBlockThreads;
    NACC_CHECK_ARG(nb < (int64_t(1) << 31), "too many rays for one launch");
    {
        const int rc = build_summaries(A, scratch, as_stream(stream));
        if (rc != NACC_OK) return rc;
    }
    k_occupied_range<<<(unsigned)nb, kBlockThreads, 0, as_stream(stream)>>>(A, t_lo, t_hi);
    NACC_LAUNCH_CHECK();
    return NACC_OK;
}

extern "C" int nacc_set_march_count_events(void* before, void* after) {
    clear_error();
    NACC_CHECK_ARG((before == nullptr) == (after == nullptr), "give both events or neither");
    march_count_events()[0] = static_cast<cudaEvent_t>(before);
    march_count_events()[1] = static_cast<cudaEvent_t>(after);
    return NACC_OK;
}
