// early_stop.cuh -- exact early-termination decisions for the march kernels
// (Sec. 4.2 "No Gradient Filtering": samples whose transmittance has fallen
// below eps are dropped).
//
// The decision is defined on an FP32 optical depth: sample k is emitted iff
// the lattice-order FP32 sum of sigma*(t1 - t0) over the emitted samples
// before it is <= fl(-ln eps), where sigma is the blob density with a fixed
// operation order (x = o + d*tm; per blob, in blob order, r2 = (dx*dx +
// dy*dy) + dz*dz, e = exp_steps(r2 * coef), s = s + peak*e; coef =
// -0.5/(std*std)) and exp_steps is the exponential defined by its steps
// below.  Evaluating that per sample costs a division-free but long chain
// per blob and a sequential sum per ray, so the kernels decide most rays
// another way, each choice provably giving the definition's answer:
//
//   * an upper bound U on the depth at every sample (per blob: its integral
//     along the whole ray line plus three times its largest value on the
//     line times the longest lattice interval where it is not negligible,
//     grown for rounding): U <= threshold means the ray never stops, and no
//     density is evaluated.  Over contiguous intervals, a unimodal function's
//     midpoint sum is at most its right-endpoint sum on the rising side, its
//     left-endpoint sum on the falling side and one term at the mode; each
//     endpoint sum exceeds the integral by at most dt_max times the
//     function's total rise (or fall), itself at most its maximum;
//   * otherwise the fast depth (the per-ray closed form of each blob with
//     the hardware exp2, a warp scan) together with a bound E on its
//     difference from the definition's depth at any sample: when the first
//     sample whose fast depth exceeds threshold - E also exceeds threshold
//     + E, the definition cuts the ray there;
//   * otherwise (the fast depth comes within E of the threshold) the ray is
//     queued and decided in the definition's own arithmetic by a second
//     kernel: the warp evaluates the exact density at 32 samples at a time,
//     and one lane adds their sigma*dt in lattice order one by one.
//
// E bounds, per blob b with line maximum S_b (= peak 2^C_b), line integral
// I_b, perpendicular distance p_b, std s_b and dt_b the longest lattice
// interval within 4 std of its closest approach, weight W_b = (I_b + 3 S_b
// dt_b + tail) g_b (1 + 2^-7) (blob_weight): the position-type errors (the definition's rounded point,
// the closed form's rounded closest approach and perpendicular distance)
// are all within delta_b = 16u (|o| + |mu_b| + t |d|) of the exact point on
// the line at t (u = 2^-24; t within 16 std of the blob's closest approach,
// where alone its density is not negligible), which multiplies it by at most
// exp(z delta_b / s_b + (delta_b/s_b)^2) at distance z std; integrated along
// the line this gives g_b = exp((p_b/s_b + 2) delta_b / s_b + (delta_b /
// s_b)^2).  Relative errors (the exponentials, at most 2 ulp for exp_steps
// and 2^-22 for ex2.approx; coefficient, exponent and product roundings,
// proportional to the exponent's size; the sums over blobs) are covered by
// u (2 n_blobs + 32 + 8 (z_p^2 + 2)) W_b.  Blobs the fast table leaves out
// contribute their whole W_b, groups culled per 64 samples their bound.
// The sums over samples: the definition's sequential sum is within u times
// the sum of its partial sums of the exact sum of its terms (tracked from the
// scanned depths), the warp scan within u (8 + chunks) P.
#pragma once

#include "nacc_internal.cuh"

namespace nacc {

// ---------------------------------------------------------------------------
// The exponential of the definition: Cody and Waite's reduction and the
// degree-7 Taylor polynomial of e^r, each step one rounded FP32 operation.
//   a < -86 or NaN: 0;  a > 88: +inf
//   n = rint(a * fl(log2 e)),  r = (a - n * LN2_HI) - n * LN2_LO,
//   LN2_HI = fl(ln 2) with its 12 low significand bits cleared,
//   LN2_LO = fl(ln 2 - LN2_HI),
//   p = (((((((c7 r + c6) r + c5) r + c4) r + c3) r + c2) r + c1) r + c0,
//   c_k = fl(1/k!),  result = p * 2^n.
// ---------------------------------------------------------------------------
constexpr float kU = 5.9604644775390625e-8f;  // 2^-24, the unit roundoff of FP32

constexpr float kExpL2E = 0x1.715476p+0f;     // fl(log2 e)
constexpr float kExpLn2Hi = 0x1.62ep-1f;      // 0.693115234375
constexpr float kExpLn2Lo = 0x1.0bfbe8p-15f;  // fl(ln 2 - LN2_HI)
constexpr float kExpC2 = 0x1p-1f;             // 1/2!
constexpr float kExpC3 = 0x1.555556p-3f;      // fl(1/3!)
constexpr float kExpC4 = 0x1.555556p-5f;      // fl(1/4!)
constexpr float kExpC5 = 0x1.111112p-7f;      // fl(1/5!)
constexpr float kExpC6 = 0x1.6c16c2p-10f;     // fl(1/6!)
constexpr float kExpC7 = 0x1.a01a02p-13f;     // fl(1/7!)

__device__ __forceinline__ float exp_steps(float a) {
    if (!(a >= -86.0f)) return 0.0f;
    if (a > 88.0f) return INFINITY;
    const float n = rintf(__fmul_rn(a, kExpL2E));
    float r = __fsub_rn(a, __fmul_rn(n, kExpLn2Hi));
    r = __fsub_rn(r, __fmul_rn(n, kExpLn2Lo));
    float p = kExpC7;
    p = __fadd_rn(__fmul_rn(p, r), kExpC6);
    p = __fadd_rn(__fmul_rn(p, r), kExpC5);
    p = __fadd_rn(__fmul_rn(p, r), kExpC4);
    p = __fadd_rn(__fmul_rn(p, r), kExpC3);
    p = __fadd_rn(__fmul_rn(p, r), kExpC2);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    return __fmul_rn(p, __int_as_float(((int)n + 127) << 23));
}

// Exact-path blob parameters: centre, -0.5/(std*std) computed as
// fl(-0.5 / fl(std*std)), peak.
struct ExactBlob {
    float mx, my, mz, coef, peak;
};

// The definition's density at x over the blobs of `list` (ascending blob
// indices; every blob left out has exp_steps(...) == 0 at every point of the
// ray, adding exactly nothing), each operation rounded as in the definition.
template <class Get>
__device__ __forceinline__ float exact_sigma(const float x[3], const uint16_t* list, int n, Get get) {
    float s = 0.0f;
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
        const ExactBlob v = get(list[i]);
        const float dx = __fsub_rn(x[0], v.mx);
        const float dy = __fsub_rn(x[1], v.my);
        const float dz = __fsub_rn(x[2], v.mz);
        float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
        const float e = exp_steps(__fmul_rn(r2, v.coef));
        s = __fadd_rn(s, __fmul_rn(v.peak, e));
    }
    return s;
}

// The same density at each lane's point x_lane of a chunk of points on the
// ray o + t d whose midpoints lie in [t_lo, t_hi] (every lane of the warp
// calls it; lanes without a point pass any x and ignore the result).  An
// entry of `list` is left out for the chunk when its exponent is below -86 at
// every point of the chunk in the definition's arithmetic -- it then adds
// exactly 0 there: the exact distance from its centre to the segment is
// r_min (closest approach clamped to [t_lo, t_hi]), the definition's rounded
// point lies within u (|o| + t |d| + |x|) of the exact one, the FP32 test here
// within 8u |mu - o| of exact; below r_min - 16u (pos_far + |mu - o|) > 13.19
// std, the exponent (-r^2 / (2 std^2), relative rounding a few u) is below
// -87.  Each lane tests one entry, the warp takes the kept ones in order.
template <class Get>
__device__ __forceinline__ float exact_sigma_chunk(const float x[3], const uint16_t* list, int n, Get get,
                                                   const float o[3], const float d[3], float dd, float idd,
                                                   float t_lo, float t_hi, float pos_far, int lane) {
    float s = 0.0f;
    for (int g = 0; g < n; g += 32) {
        bool on = false;
        if (g + lane < n) {
            const ExactBlob v = get(list[g + lane]);
            const float m0 = v.mx - o[0], m1 = v.my - o[1], m2 = v.mz - o[2];
            const float mn = sqrtf(fmaf(m2, m2, fmaf(m1, m1, m0 * m0)));
            float r2;
            if (dd > 0.0f) {
                const float ts = fmaf(m2, d[2], fmaf(m1, d[1], m0 * d[0])) * idd;
                const float cx = fmaf(m1, d[2], -m2 * d[1]), cy = fmaf(m2, d[0], -m0 * d[2]),
                            cz = fmaf(m0, d[1], -m1 * d[0]);
                const float uc = fminf(fmaxf(ts, t_lo), t_hi) - ts;
                r2 = fmaf(dd * uc, uc, fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd);
            } else {
                r2 = mn * mn;
            }
            const float rmin = sqrtf(r2) * (1.0f - 1e-5f) - 16.0f * kU * (pos_far + mn) * 1.01f;
            const float sd2 = -0.5f / v.coef;  // std^2
            on = !(rmin > 0.0f && rmin * rmin > 174.0f * sd2);
        }
        unsigned m = __ballot_sync(0xffffffffu, on);
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const ExactBlob v = get(list[g + j]);
            const float dx = __fsub_rn(x[0], v.mx);
            const float dy = __fsub_rn(x[1], v.my);
            const float dz = __fsub_rn(x[2], v.mz);
            float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
            const float e = exp_steps(__fmul_rn(r2, v.coef));
            s = __fadd_rn(s, __fmul_rn(v.peak, e));
        }
    }
    return s;
}

// ---------------------------------------------------------------------------
// Double-float helpers (value = hi + lo), every operation explicitly rounded
// so that nothing is contracted: the closest approach t*_b and the squared
// distance p_b^2 of the fast table are formed to about u^2 and rounded once.
// ---------------------------------------------------------------------------
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ F2 f2_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return F2{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const F2 s = f2_two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s.hi, lo);
    return F2{h, __fsub_rn(lo, __fsub_rn(h, s.hi))};
}

__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const F2 p = f2_two_prod(a.hi, b.hi);
    const float lo = __fadd_rn(p.lo, __fadd_rn(__fmul_rn(a.hi, b.lo), __fmul_rn(a.lo, b.hi)));
    const float h = __fadd_rn(p.hi, lo);
    return F2{h, __fsub_rn(lo, __fsub_rn(h, p.hi))};
}

__device__ __forceinline__ F2 f2_div(F2 a, F2 b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const F2 r = f2_add(a, f2_mul(F2{-q1, 0.0f}, b));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    const float h = __fadd_rn(q1, q2);
    return F2{h, __fsub_rn(q2, __fsub_rn(h, q1))};
}

// Closest approach t* = (mu - o).d / |d|^2 and squared distance p^2 =
// |(mu - o) x d|^2 / |d|^2 of a centre from the line o + t d (|d| > 0,
// idd = fl(1/|d|^2)).  A first FP32 estimate t_ref of t* moves the origin to
// o' = o + t_ref d, formed in double-float (exact up to u^2), so the rest
// works on m' = mu - o', whose size is about p instead of |mu - o|: t* =
// t_ref + m'.d / |d|^2 within 0.5u |t*| (the final rounding) + 8u |m'| / |d|,
// p within 8u |m'|.
__device__ __forceinline__ void closest_approach(const float mu[3], const float o[3], const float d[3], float idd,
                                                 float& ts, float& pp) {
    const float m0 = mu[0] - o[0], m1 = mu[1] - o[1], m2 = mu[2] - o[2];
    const float t_ref = fmaf(m2, d[2], fmaf(m1, d[1], m0 * d[0])) * idd;
    float mp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const F2 q = f2_two_prod(d[a], t_ref);
        const F2 s = f2_two_sum(o[a], q.hi);
        // mu - (s.hi + s.lo + q.lo), the small parts last
        mp[a] = __fsub_rn(__fsub_rn(mu[a], s.hi), __fadd_rn(s.lo, q.lo));
    }
    const float cx = fmaf(mp[1], d[2], -mp[2] * d[1]);
    const float cy = fmaf(mp[2], d[0], -mp[0] * d[2]);
    const float cz = fmaf(mp[0], d[1], -mp[1] * d[0]);
    ts = t_ref + fmaf(mp[2], d[2], fmaf(mp[1], d[1], mp[0] * d[0])) * idd;
    pp = fmaf(cz, cz, fmaf(cy, cy, cx * cx)) * idd;
}

// ---------------------------------------------------------------------------
// Per-ray bounds, accumulated blob by blob (each lane one blob), then summed
// over the warp.
// ---------------------------------------------------------------------------
constexpr float kExactZ = 13.5f;  // a blob farther than this many std from the line is 0 on it

struct RayBound {
    float U;    // upper bound on the definition's optical depth at any sample
    float Ek;   // bound on |fast - definition| of the kept blobs' terms, whole ray
    float eps;  // the same relative to the depth: at most eps times the terms summed
    float Ea;   // absolute part: blobs left out (whole weights), per-group culling
};

// A blob's weight: an upper bound on the sum of its share of sigma*dt over
// the ray's samples in the definition's arithmetic (S = its largest density
// on the line, I = its integral along the line, dt = the longest lattice
// interval within 4 std of its closest approach, dt_max = the longest
// anywhere -- beyond 4 std the density is below e^-8 S, so those intervals
// add at most 3 e^-8 S dt_max to the endpoint sums --, ov = the total
// length by which the ray's rounded intervals may overlap one another; the
// margin 2^-7 covers its FP32 evaluation here -- the line values from a
// closed form rounded in FP32 -- and the rounding of the definition's terms).
__device__ __forceinline__ float blob_weight(float S, float I, float dt, float dt_max, float ov, float gm1) {
    return (I + S * (3.0f * dt + 1.01e-3f * dt_max + ov)) * (1.0f + gm1) * (1.0f + 0x1p-7f);
}

// Growth g - 1 of a blob's density under the position-type errors (above).
// The errors at a point w std along the line from the closest approach are
// within 1.5u (pos0 + 3 |w| sd): pos0 = |o| + 2.5 |t*| |d| + 16 p (the
// definition's rounded point u (|d| |tm| + |x|), the fast form's rounded
// closest approach and distance, closest_approach, its rounded t - t*),
// which moves the exponent by at most z delta / sd at distance z <= p/sd +
// |w| std; weighted by the density along the line this stays below the
// returned factor (isd = 1/sd).
__device__ __forceinline__ float blob_growth(float p, float isd, float pos0) {
    const float zp = p * isd * 1.0001f;  // isd = 1/sd (rounded: the margin covers it)
    const float dl = 1.5f * kU * pos0 * isd * 1.0001f;
    const float x = fminf(1.02f * ((zp + 2.0f) * dl + 4.5f * kU * (zp + 2.0f)) + dl * dl, 60.0f);
    return x < 1e-3f ? x * 1.001f : __expf(x) * 1.0001f - 1.0f;
}

// A blob's share of the error bound: its whole weight if the fast table
// leaves it out, else the growth (the two evaluations' points lie within the
// combined position error of each other) and the relative errors (the
// exponentials: at most 2 ulp for exp_steps and 2^-22 for ex2.approx; the
// peak, interval and sum roundings; the exponent's roundings, proportional
// to its size, about (z_p^2 + w^2)/2; the sums over n_blobs blobs).
__device__ __forceinline__ float blob_error(float W, float gm1, float zp, int n_blobs, bool kept) {
    const float rel = kU * (2.0f * (float)n_blobs + 32.0f + 8.0f * (zp * zp + 2.0f));
    return kept ? W * (gm1 + rel) : W;
}

// A kept blob's relative error bound at any point where either evaluation is
// not negligible: there the definition's exponent is at least -86, so the
// point lies within 13.2 std of the centre (z <= 13.2, |w| <= 13.2), where
// the position-type errors move the density by at most exp(13.2 * 1.5u
// (pos0 / sd + 40)) and the relative-type ones by u (2 n_blobs + 32 + 16 *
// 87) (exponent roundings proportional to |a| <= 87).
__device__ __forceinline__ float blob_rel_error(float isd, float pos0, int n_blobs) {
    const float x = 1.02f * 13.2f * 1.5f * kU * (pos0 * isd * 1.0001f + 40.0f);
    return (x < 1e-3f ? x * 1.001f : __expf(fminf(x, 60.0f)) * 1.0001f - 1.0f) +
           kU * (2.0f * (float)n_blobs + 32.0f + 16.0f * 87.0f);
}

// True if the blob may be non-zero somewhere on the ray in the definition's
// arithmetic: its exponent is below -(p - pos_err)^2 / (2 sd^2) everywhere,
// pos_err = 8u pos_far covering the rounded point (pos_far = |o| + t_max |d|).
__device__ __forceinline__ bool blob_may_count(float p, float sd, float pos_far) {
    return fmaxf(p - 8.0f * kU * pos_far, 0.0f) / sd < kExactZ;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Rounding of the sums over samples.  The definition's sequential sum of n
// terms is within u times the sum of its partial sums of the exact sum of
// its terms; Q (the sum of the depths before every sample up to the one
// tested, from the warp scan, which is within E of the definition's) bounds
// that sum with cnt * E for the difference.  The warp scan itself is
// within u (16 + chunks) P of its terms' exact sum: a lane's up to three
// sequential additions of its own points, the five levels of the scan, the
// subtraction of the lane's total, the carry, and one addition per earlier
// chunk of at least 32 points.
__device__ __forceinline__ float sum_bound(int cnt, float Q, float E, float P) {
    const float n = (float)cnt;
    return kU * ((Q + n * E) * 1.01f + (n * (1.0f / 32.0f) + 16.0f) * P * 1.01f);
}

// Bound on |fast - definition| of the density terms before a sample whose
// fast depth is P: the absolute part plus the smaller of the whole-ray bound
// and the relative one (the terms before the sample sum to at most P plus
// the error, so their errors sum to at most eps times that; eps < 1e-2).
__device__ __forceinline__ float density_error(const RayBound& rb, float P) {
    return rb.Ea + fminf(rb.Ek, rb.eps * (P + rb.Ea) * 1.02f);
}

// Bound on |fast - definition| of the depth before any sample whose fast
// depth is at most P (cnt: the ray's emitted samples; Q as in sum_bound),
// including the far tails (below 1e-30 per sample: peak 2^-124 or less on
// either side).
__device__ __forceinline__ float depth_error(const RayBound& rb, int cnt, float Q, float P) {
    const float Es = density_error(rb, P);
    return Es + 1e-30f * (float)cnt + sum_bound(cnt, Q, Es, P + Es);
}

// Upper bound on the definition's depth at any sample of the ray, from the
// sum U of the blobs' weights (the sums over blobs and samples round up by
// at most that much).
__device__ __forceinline__ float depth_upper(float U, int cnt, int n_blobs) {
    return U * (1.0f + kU * ((float)cnt + (float)n_blobs + 24.0f) * 1.01f);
}

// A ray whose counts make the sequential-sum bound meaningless (or whose
// bounds are not finite / not small) is decided exactly.
__device__ __forceinline__ bool bounds_usable(const RayBound& rb, int cnt, float thr) {
    return cnt < 16384 && density_error(rb, thr) < 0.25f * thr && rb.eps < 1e-2f && rb.U < 3.0e38f;
}

// The definition's sequential depth over one round of n <= N terms (tau in
// shared memory, 16-byte aligned), added one at a time onto P in order:
// returns the first j whose depth before it (P plus tau[0..j)) exceeds thr,
// or -1.  The adds run to the end of the round without a branch (P's later
// value is unused once a cut is found), so only their own latency chains.
template <int N>
__device__ __forceinline__ int seq_depth_cut(const float* tau, int n, float thr, float& P) {
    int jc = -1;
    if (n == N) {
#pragma unroll
        for (int j = 0; j < N; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(tau + j);
            jc = (jc < 0 && P > thr) ? j : jc;
            P = __fadd_rn(P, v.x);
            jc = (jc < 0 && P > thr) ? j + 1 : jc;
            P = __fadd_rn(P, v.y);
            jc = (jc < 0 && P > thr) ? j + 2 : jc;
            P = __fadd_rn(P, v.z);
            jc = (jc < 0 && P > thr) ? j + 3 : jc;
            P = __fadd_rn(P, v.w);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < n; ++j) {
            jc = (jc < 0 && P > thr) ? j : jc;
            P = __fadd_rn(P, tau[j]);
        }
    }
    return jc;
}

}  // namespace nacc
