/*
 * oracle.c -- plain, slow, CPU reference for occupancy-grid sampling and
 * differentiable volume rendering as described in NerfAcc (arXiv 2305.04966).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference legs call this file.  It shares no
 * code, header, table or constant generator with the CUDA library.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off [-fopenmp] oracle.c -lm
 * (-ffp-contract=off is REQUIRED: the lattice march is defined with every FP32
 * operation individually rounded; a fused multiply-add would change it.)
 *
 * Functions and the passage each follows:
 *   orc_march          Table 1 "Spatial Skipping" row (occupied <=> bit set),
 *                      Sec. 4.2 "Sample as Interval" and "Packed Tensor",
 *                      Sec. 4.2 "No Gradient Filtering" (drop T < 1e-4),
 *                      Appendix B (step size, resolution L^3, threshold).
 *                      FP32 lattice arithmetic; this dense march IS the
 *                      definition of the emitted sample set.
 *   orc_field_*        analytic Gaussian-blob density / colour (stands in for
 *                      the radiance field of Algorithm 1; not the method).
 *   orc_render_fwd     Eq. 2 discretised: T_i = exp(-sum_{j<i} sigma_j dt_j),
 *                      w_i = T_i (1 - exp(-sigma_i dt_i)); Table 1 PDF row;
 *                      Algorithm 1 "rendering".  FP64.
 *   orc_render_bwd     gradient of orc_render_fwd w.r.t. sigma_i and c_i
 *                      (Algorithm 1: the field receives gradients).  FP64.
 *   orc_grid_points    jittered cell centres for the estimator update (Eq. 4,
 *                      Sec. 3.1 "Spatial Skipping" EMA paragraph).
 *   orc_update_grid    EMA update F: T^{k-1} -> T^k (Eq. 4) and binarisation
 *                      1[sigma > tau] (Table 1).  FP32 EMA, FP64 mean.
 *   orc_sample_pdf     inverse transform sampling t = F^-1(u) (Eq. 1) with the
 *                      CDF built from 1 - T (Eq. 3).  FP32 (the bin choice is
 *                      a float decision taken in the kernel's precision).
 *   orc_splitmix64_at  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) stream
 *                      element, used as a counter-based generator.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LEVELS 16

typedef struct {
    float lmin[3], lmax[3], scale[3], width[3];
} orc_level;

/* Level l's box is the level-0 box scaled by 2^l about its centre.  All in
 * FP32: cen = (min+max)*0.5, half = (max-min)*0.5, lmin = cen - half*2^l,
 * lmax = cen + half*2^l, scale = res / (lmax-lmin), width = (lmax-lmin)/res. */
static void orc_levels(const float amin[3], const float amax[3], int res, int L, orc_level* lv)
{
    for (int l = 0; l < L; ++l) {
        float f = (float)(1 << l);
        for (int a = 0; a < 3; ++a) {
            float cen = (amin[a] + amax[a]) * 0.5f;
            float half = (amax[a] - amin[a]) * 0.5f;
            float hs = half * f;
            lv[l].lmin[a] = cen - hs;
            lv[l].lmax[a] = cen + hs;
            float ext = lv[l].lmax[a] - lv[l].lmin[a];
            lv[l].scale[a] = (float)res / ext;
            lv[l].width[a] = ext / (float)res;
        }
    }
}

/* Early-stop threshold on optical depth: T < eps  <=>  sum(sigma dt) > -ln(eps). */
static float orc_tau_threshold(float eps)
{
    if (!(eps > 0.0f)) return INFINITY;
    return (float)(-log((double)eps));
}

/* SplitMix64 output number (counter+1) of the stream seeded with `seed`. */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t counter)
{
    uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Top 24 bits as a float in [0, 1). */
static float orc_u01(uint64_t h) { return (float)(h >> 40) * 0x1p-24f; }

/* ------------------------------------------------------------------------ */
/* Analytic field (harness, not the method)                                  */
/* ------------------------------------------------------------------------ */

/* Natural exponential of an FP32 argument, defined by its steps so that the
 * early-stop decision it feeds is one function of the inputs on every
 * platform (a host libm's expf and a GPU's differ in the last bits).  The
 * method is Cody and Waite's argument reduction followed by the degree-7
 * Taylor polynomial of e^r, every operation one rounded FP32 operation:
 *   a < -86 or NaN:  0        (e^-86 < 2^-124: below the significance of any
 *                              density sum it is added to)
 *   n = rint(a * L2E)         L2E = fl(log2 e), rint rounds half to even
 *   r = (a - n * LN2_HI) - n * LN2_LO
 *                             LN2_HI = fl(ln 2) with its 12 low significand
 *                             bits cleared (n * LN2_HI is exact),
 *                             LN2_LO = fl(ln 2 - LN2_HI)
 *   p = (((((((c7 r + c6) r + c5) r + c4) r + c3) r + c2) r + c1) r + c0,
 *                             c_k = fl(1 / k!)
 *   e^a = p * 2^n             (2^n exact and normal: n >= -124 here)
 * Measured against the FP64 exponential: at most 1.19 units in the last
 * place on [-86, 0]; pinned at 2. */
float orc_exp_steps(float a)
{
    if (!(a >= -86.0f)) return 0.0f;
    if (a > 88.0f) return INFINITY;
    const double ln2 = 0.69314718055994530942;
    float hi = (float)ln2;
    uint32_t hb;
    memcpy(&hb, &hi, sizeof hb);
    hb &= ~0xFFFu;
    memcpy(&hi, &hb, sizeof hi);
    const float lo = (float)(ln2 - (double)hi);
    const float l2e = (float)1.44269504088896340736;
    float c[8];
    double fact = 1.0;
    for (int k = 0; k < 8; ++k) {
        if (k > 0) fact *= (double)k;
        c[k] = (float)(1.0 / fact);
    }
    float n = rintf(a * l2e);
    float r = a - n * hi;
    r = r - n * lo;
    float p = c[7];
    for (int k = 6; k >= 0; --k) {
        p = p * r;
        p = p + c[k];
    }
    uint32_t sb = (uint32_t)((int)n + 127) << 23;
    float scale;
    memcpy(&scale, &sb, sizeof scale);
    return p * scale;
}

void orc_exp_steps_array(int64_t n, const float* a, float* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_exp_steps(a[i]);
}

/* FP32 density with a fixed operation order; used only for the early-stop
 * decision inside the march, which is taken in FP32 like the kernel's.  The
 * exponential is orc_exp_steps (defined above by its steps). */
static float orc_sigma_f32(const float x[3], int nb, const float* mu, const float* stdv,
                           const float* peak)
{
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) {
        float sd2 = stdv[b] * stdv[b];
        float coef = -0.5f / sd2;
        float dx = x[0] - mu[3 * b + 0];
        float dy = x[1] - mu[3 * b + 1];
        float dz = x[2] - mu[3 * b + 2];
        float r2 = dx * dx + dy * dy;
        r2 = r2 + dz * dz;
        float e = orc_exp_steps(r2 * coef);
        s = s + peak[b] * e;
    }
    return s;
}

/* FP64 density and density-weighted colour at a point. */
static void orc_field_f64(const double x[3], int nb, const float* mu, const float* stdv,
                          const float* peak, const float* rgb, double* sigma, double c[3])
{
    double s = 0.0, acc[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b) {
        double dx = x[0] - mu[3 * b], dy = x[1] - mu[3 * b + 1], dz = x[2] - mu[3 * b + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        double sd = stdv[b];
        double sb = (double)peak[b] * exp(-r2 / (2.0 * sd * sd));
        s += sb;
        for (int a = 0; a < 3; ++a) acc[a] += sb * (double)rgb[3 * b + a];
    }
    *sigma = s;
    for (int a = 0; a < 3; ++a) c[a] = s > 0.0 ? acc[a] / s : 0.0;
}

/* Field at interval midpoints of packed samples: x = o[r] + d[r] * (t0+t1)/2. */
void orc_field_samples(int64_t n_samples, const float* rays_o, const float* rays_d,
                       const int32_t* ray_idx, const float* t0, const float* t1, int nb,
                       const float* mu, const float* stdv, const float* peak, const float* rgb,
                       double* sigma_out, double* rgb_out, int n_threads)
{
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int64_t i = 0; i < n_samples; ++i) {
        int64_t r = ray_idx[i];
        double m = 0.5 * ((double)t0[i] + (double)t1[i]);
        double x[3];
        for (int a = 0; a < 3; ++a) x[a] = (double)rays_o[3 * r + a] + (double)rays_d[3 * r + a] * m;
        orc_field_f64(x, nb, mu, stdv, peak, rgb, &sigma_out[i], &rgb_out[3 * i]);
    }
}

/* Field at arbitrary points (FP64 density only). */
void orc_field_points(int64_t n, const float* xyz, int nb, const float* mu, const float* stdv,
                      const float* peak, const float* rgb, double* sigma_out, int n_threads)
{
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int64_t i = 0; i < n; ++i) {
        double x[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        double c[3];
        orc_field_f64(x, nb, mu, stdv, peak, rgb, &sigma_out[i], c);
    }
}

/* ------------------------------------------------------------------------ */
/* Occupancy-grid lattice march (the definition of the packed sample set)    */
/* ------------------------------------------------------------------------ */

/* Slab clip of the ray against the outermost level's box; returns 0 on miss. */
static int orc_clip(const float o[3], const float d[3], const orc_level* outer, float t_min,
                    float t_max, float* tn, float* tf)
{
    float near = t_min, far = t_max;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0f) {
            if (o[a] < outer->lmin[a] || o[a] > outer->lmax[a]) return 0;
            continue;
        }
        float inv = 1.0f / d[a];
        float ta = (outer->lmin[a] - o[a]) * inv;
        float tb = (outer->lmax[a] - o[a]) * inv;
        float lo = (ta < tb) ? ta : tb;
        float hi = (ta < tb) ? tb : ta;
        if (lo > near) near = lo;
        if (hi < far) far = hi;
    }
    *tn = near;
    *tf = far;
    return near < far;
}

/* Occupancy of the point x: the finest level whose (closed) box holds x,
 * then the clamped cell of that level.  Returns 1 if the bit is set. */
static int orc_occupied(const float x[3], const orc_level* lv, int L, int res, const uint32_t* bits)
{
    for (int l = 0; l < L; ++l) {
        int inside = 1;
        for (int a = 0; a < 3; ++a)
            if (!(x[a] >= lv[l].lmin[a] && x[a] <= lv[l].lmax[a])) inside = 0;
        if (!inside) continue;
        int64_t i[3];
        for (int a = 0; a < 3; ++a) {
            float u = (x[a] - lv[l].lmin[a]) * lv[l].scale[a];
            int64_t c = (int64_t)floorf(u);
            if (c < 0) c = 0;
            if (c > res - 1) c = res - 1;
            i[a] = c;
        }
        int64_t r3 = (int64_t)res * res * res;
        int64_t idx = (int64_t)l * r3 + (i[0] * res + i[1]) * res + i[2];
        return (int)((bits[idx >> 5] >> (idx & 31)) & 1u);
    }
    return 0; /* outside every level */
}

typedef struct {
    int n_blobs;
    const float *mu, *stdv, *peak;
    float thr;
} orc_march_field;

/* March one ray over the lattice t0_k = t_near + k*step (k < max_steps,
 * t0_k < t_far), emitting [t0_k, t0_k + step] whenever the interval midpoint
 * is in an occupied cell.  With a field, sample k is emitted only while the
 * optical depth accumulated over the emitted samples before it is <= thr
 * (T >= eps); the ray stops at the first occupied k that fails this. */
static int64_t orc_march_ray(const float o[3], const float d[3], const orc_level* lv, int L,
                             int res, const uint32_t* bits, float step, int max_steps,
                             float t_min, float t_max, const orc_march_field* fld,
                             int64_t base, int32_t ray, int32_t* ray_idx, float* t0s, float* t1s)
{
    float tn, tf;
    if (!orc_clip(o, d, &lv[L - 1], t_min, t_max, &tn, &tf)) return 0;
    float tau = 0.0f;
    int64_t n = 0;
    for (int k = 0; k < max_steps; ++k) {
        float t0 = tn + (float)k * step;
        if (!(t0 < tf)) break;
        float t1 = t0 + step;
        float tm = (t0 + t1) * 0.5f;
        float x[3];
        for (int a = 0; a < 3; ++a) x[a] = o[a] + d[a] * tm;
        if (!orc_occupied(x, lv, L, res, bits)) continue;
        if (fld && tau > fld->thr) break;
        if (t0s) {
            ray_idx[base + n] = ray;
            t0s[base + n] = t0;
            t1s[base + n] = t1;
        }
        ++n;
        if (fld) {
            float s = orc_sigma_f32(x, fld->n_blobs, fld->mu, fld->stdv, fld->peak);
            float dt = t1 - t0;
            tau = tau + s * dt;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Unbounded scenes: sampling in s-space and a contracted grid               */
/* ------------------------------------------------------------------------ */

/* Disparity-linear bijection s in [0, 1] -> t in [t_near, t_far]:
 * 1/t = (1 - s)/t_near + s/t_far, as FP32 operations in this order:
 * a = 1/t_near, b = 1/t_far, t = 1 / (a * (1 - s) + b * s)
 * (both ends exact up to the reciprocal's rounding, no cancellation). */
float orc_s_to_t(float s, float t_near, float t_far)
{
    float a = 1.0f / t_near;
    float b = 1.0f / t_far;
    float den = a * (1.0f - s) + b * s;
    return 1.0f / den;
}

/* L-infinity contraction: c(x) = x if max|x_a| <= 1, else
 * (2 - 1/m) x / m with m = max|x_a|, as inv = 1/m, f = 2 - inv, g = f * inv,
 * c_a = x_a * g (FP32, each rounded). */
void orc_contract(const float x[3], float c[3])
{
    float ax = fabsf(x[0]), ay = fabsf(x[1]), az = fabsf(x[2]);
    float m = ax > ay ? ax : ay;
    m = m > az ? m : az;
    if (m <= 1.0f) {
        c[0] = x[0];
        c[1] = x[1];
        c[2] = x[2];
        return;
    }
    float inv = 1.0f / m;
    float f = 2.0f - inv;
    float g = f * inv;
    for (int a = 0; a < 3; ++a) c[a] = x[a] * g;
}

void orc_contract_points(int64_t n, const float* xyz, float* out)
{
    for (int64_t i = 0; i < n; ++i) orc_contract(&xyz[3 * i], &out[3 * i]);
}

/* Inverse contraction in FP32 (the scene point of a grid point): m' = max|c_a|;
 * x = c if m' <= 1, else x_a = c_a * (inv / m') with
 * inv = 1 / (2 - min(m', largest float below 2)). */
void orc_uncontract_points(int64_t n, const float* c, float* x)
{
    const float mmax = 1.99999988f;
    for (int64_t i = 0; i < n; ++i) {
        const float* ci = &c[3 * i];
        float ax = fabsf(ci[0]), ay = fabsf(ci[1]), az = fabsf(ci[2]);
        float mp = ax > ay ? ax : ay;
        mp = mp > az ? mp : az;
        float g = 1.0f;
        if (mp > 1.0f) {
            float mc = mp < mmax ? mp : mmax;
            float den = 2.0f - mc;
            float inv = 1.0f / den;
            g = inv / mp;
        }
        for (int a = 0; a < 3; ++a) x[3 * i + a] = ci[a] * g;
    }
}

/* One ray of the unbounded march: for k = 0..K-1, s0 = k / K, s1 = (k+1) / K
 * (FP32 divisions), t0 = Phi(s0), t1 = Phi(s1), tm = (t0 + t1) * 0.5,
 * x = o + d * tm; the sample is emitted iff the cell of c(x) is occupied,
 * with the same early-stop rule as the bounded march (sigma at x). */
static int64_t orc_march_unb_ray(const float o[3], const float d[3], const orc_level* lv, int L, int res,
                                 const uint32_t* bits, int K, float t_near, float t_far,
                                 const orc_march_field* fld, int64_t base, int32_t ray, int32_t* ray_idx,
                                 float* t0s, float* t1s)
{
    float tau = 0.0f;
    int64_t n = 0;
    for (int k = 0; k < K; ++k) {
        float s0 = (float)k / (float)K, s1 = (float)(k + 1) / (float)K;
        float t0 = orc_s_to_t(s0, t_near, t_far), t1 = orc_s_to_t(s1, t_near, t_far);
        float tm = (t0 + t1) * 0.5f;
        float x[3], c[3];
        for (int a = 0; a < 3; ++a) x[a] = o[a] + d[a] * tm;
        orc_contract(x, c);
        if (!orc_occupied(c, lv, L, res, bits)) continue;
        if (fld && tau > fld->thr) break;
        if (t0s) {
            ray_idx[base + n] = ray;
            t0s[base + n] = t0;
            t1s[base + n] = t1;
        }
        ++n;
        if (fld) {
            float sg = orc_sigma_f32(x, fld->n_blobs, fld->mu, fld->stdv, fld->peak);
            float dt = t1 - t0;
            tau = tau + sg * dt;
        }
    }
    return n;
}

int orc_march_unbounded(int64_t n_rays, const float* rays_o, const float* rays_d, const float* aabb_min,
                        const float* aabb_max, int res, int n_levels, const uint32_t* bits, int K, float t_near,
                        float t_far, int n_blobs, const float* mu, const float* stdv, const float* peak, float eps,
                        int64_t* counts, const int64_t* offsets, int32_t* ray_idx, float* t0s, float* t1s,
                        int n_threads)
{
    if (n_levels < 1 || n_levels > ORC_MAX_LEVELS || res < 1 || K < 1 || !(t_near > 0.0f) || !(t_far > t_near) ||
        !isfinite(t_far))
        return -1;
    orc_level lv[ORC_MAX_LEVELS];
    orc_levels(aabb_min, aabb_max, res, n_levels, lv);
    orc_march_field fld = {n_blobs, mu, stdv, peak, orc_tau_threshold(eps)};
    const orc_march_field* f = n_blobs > 0 ? &fld : NULL;
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads)
    for (int64_t r = 0; r < n_rays; ++r) {
        int64_t base = offsets ? offsets[r] : 0;
        counts[r] = orc_march_unb_ray(&rays_o[3 * r], &rays_d[3 * r], lv, n_levels, res, bits, K, t_near, t_far, f,
                                      base, (int32_t)r, offsets ? ray_idx : NULL, offsets ? t0s : NULL,
                                      offsets ? t1s : NULL);
    }
    return 0;
}

/* counts[r] = number of samples of ray r.  If `offsets` is non-NULL also write
 * the samples of ray r at [offsets[r], offsets[r]+counts[r]).  n_blobs == 0:
 * no field, no early stop.  Returns 0, or -1 on invalid arguments. */
int orc_march(int64_t n_rays, const float* rays_o, const float* rays_d, const float* aabb_min,
              const float* aabb_max, int res, int n_levels, const uint32_t* bits, float step,
              int max_steps, float t_min, float t_max, int n_blobs, const float* mu,
              const float* stdv, const float* peak, float eps, int64_t* counts,
              const int64_t* offsets, int32_t* ray_idx, float* t0s, float* t1s, int n_threads)
{
    if (n_levels < 1 || n_levels > ORC_MAX_LEVELS || res < 1 || !(step > 0.0f)) return -1;
    orc_level lv[ORC_MAX_LEVELS];
    orc_levels(aabb_min, aabb_max, res, n_levels, lv);
    orc_march_field fld = {n_blobs, mu, stdv, peak, orc_tau_threshold(eps)};
    const orc_march_field* f = n_blobs > 0 ? &fld : NULL;
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads)
    for (int64_t r = 0; r < n_rays; ++r) {
        int64_t base = offsets ? offsets[r] : 0;
        counts[r] = orc_march_ray(&rays_o[3 * r], &rays_d[3 * r], lv, n_levels, res, bits, step,
                                  max_steps, t_min, t_max, f, base, (int32_t)r,
                                  offsets ? ray_idx : NULL, offsets ? t0s : NULL,
                                  offsets ? t1s : NULL);
    }
    return 0;
}

/* Ray/box clip only (for tests): t_near, t_far, hit. */
void orc_ray_clip(int64_t n_rays, const float* rays_o, const float* rays_d, const float* aabb_min,
                  const float* aabb_max, int res, int n_levels, float t_min, float t_max,
                  float* tn_out, float* tf_out, int32_t* hit_out)
{
    orc_level lv[ORC_MAX_LEVELS];
    orc_levels(aabb_min, aabb_max, res, n_levels, lv);
    for (int64_t r = 0; r < n_rays; ++r) {
        float tn = 0.0f, tf = 0.0f;
        hit_out[r] = orc_clip(&rays_o[3 * r], &rays_d[3 * r], &lv[n_levels - 1], t_min, t_max, &tn, &tf);
        tn_out[r] = tn;
        tf_out[r] = tf;
    }
}

/* Level geometry (for tests). out: [L][4][3] = lmin, lmax, scale, width. */
void orc_level_geometry(const float* aabb_min, const float* aabb_max, int res, int n_levels, float* out)
{
    orc_level lv[ORC_MAX_LEVELS];
    orc_levels(aabb_min, aabb_max, res, n_levels, lv);
    for (int l = 0; l < n_levels; ++l)
        for (int a = 0; a < 3; ++a) {
            out[12 * l + a] = lv[l].lmin[a];
            out[12 * l + 3 + a] = lv[l].lmax[a];
            out[12 * l + 6 + a] = lv[l].scale[a];
            out[12 * l + 9 + a] = lv[l].width[a];
        }
}

/* ------------------------------------------------------------------------ */
/* Compositing (Eq. 2 discretised) and its adjoint, FP64                     */
/* ------------------------------------------------------------------------ */

/* Per ray, samples i in order: tau_i = sigma_i (t1_i - t0_i);
 * P_i = sum_{j<i} tau_j; sample i is masked (w = 0, and every later sample too)
 * when eps > 0 and P_i > -ln(eps) (T_i < eps); T_i = exp(-P_i),
 * w_i = T_i * (1 - exp(-tau_i)); T_N = exp(-sum over unmasked tau).
 * rgb = sum w_i c_i + T_N bg, opacity = sum w_i, depth = sum w_i (t0+t1)/2. */
void orc_render_fwd(int64_t n_rays, const int64_t* offsets, const float* t0, const float* t1,
                    const double* sigmas, const double* rgbs, const double* bg, float eps,
                    double* rgb_out, double* opacity_out, double* depth_out, double* trans_out,
                    double* weights_out, int n_threads)
{
    double thr = (double)orc_tau_threshold(eps);
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads)
    for (int64_t r = 0; r < n_rays; ++r) {
        double P = 0.0, acc[3] = {0.0, 0.0, 0.0}, op = 0.0, dep = 0.0;
        int masked = 0;
        for (int64_t i = offsets[r]; i < offsets[r + 1]; ++i) {
            if (!masked && P > thr) masked = 1;
            if (masked) {
                if (weights_out) weights_out[i] = 0.0;
                continue;
            }
            double dt = (double)t1[i] - (double)t0[i];
            double tau = sigmas[i] * dt;
            double T = exp(-P);
            double w = T * -expm1(-tau);
            for (int a = 0; a < 3; ++a) acc[a] += w * rgbs[3 * i + a];
            op += w;
            dep += w * 0.5 * ((double)t0[i] + (double)t1[i]);
            P += tau;
            if (weights_out) weights_out[i] = w;
        }
        double TN = exp(-P);
        for (int a = 0; a < 3; ++a) rgb_out[3 * r + a] = acc[a] + TN * bg[a];
        opacity_out[r] = op;
        depth_out[r] = dep;
        trans_out[r] = TN;
    }
}

/* Gradient of orc_render_fwd for upstream gC = dL/drgb, gA = dL/dopacity,
 * gD = dL/ddepth.  With T_{i+1} = exp(-(P_i + tau_i)), m_i the midpoint,
 * S^c_i = sum_{k>i} w_k c_k and S^m_i = sum_{k>i} w_k m_k (over unmasked k):
 *   dL/dc_i     = w_i gC
 *   dL/dsigma_i = dt_i [ gC.(T_{i+1} c_i - S^c_i - T_N bg) + gA T_N
 *                        + gD (T_{i+1} m_i - S^m_i) ]
 * (from w_k = T_k - T_{k+1}, dT_k/dsigma_i = -dt_i T_k for k > i).  Masked
 * samples receive zero gradient. */
void orc_render_bwd(int64_t n_rays, const int64_t* offsets, const float* t0, const float* t1,
                    const double* sigmas, const double* rgbs, const double* bg, float eps,
                    const double* g_rgb, const double* g_opacity, const double* g_depth,
                    double* g_sigmas, double* g_rgbs, int n_threads)
{
    double thr = (double)orc_tau_threshold(eps);
#pragma omp parallel for schedule(dynamic, 64) num_threads(n_threads)
    for (int64_t r = 0; r < n_rays; ++r) {
        int64_t s = offsets[r], e = offsets[r + 1];
        int64_t n = e - s;
        double* P = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        /* forward: exclusive prefixes and the first masked sample */
        double acc = 0.0;
        int64_t cut = n;
        for (int64_t j = 0; j < n; ++j) {
            if (acc > thr) { cut = j; break; }
            P[j] = acc;
            acc += sigmas[s + j] * ((double)t1[s + j] - (double)t0[s + j]);
        }
        double TN = exp(-acc);
        const double* gC = &g_rgb[3 * r];
        double gA = g_opacity[r], gD = g_depth[r];
        double Sc[3] = {0.0, 0.0, 0.0}, Sm = 0.0;
        for (int64_t j = n - 1; j >= 0; --j) {
            int64_t i = s + j;
            if (j >= cut) {
                g_sigmas[i] = 0.0;
                for (int a = 0; a < 3; ++a) g_rgbs[3 * i + a] = 0.0;
                continue;
            }
            double dt = (double)t1[i] - (double)t0[i];
            double tau = sigmas[i] * dt;
            double Ti = exp(-P[j]);
            double Tn = exp(-(P[j] + tau));
            double w = Ti * -expm1(-tau);
            double m = 0.5 * ((double)t0[i] + (double)t1[i]);
            double g = 0.0;
            for (int a = 0; a < 3; ++a) g += gC[a] * (Tn * rgbs[3 * i + a] - Sc[a] - TN * bg[a]);
            g += gA * TN;
            g += gD * (Tn * m - Sm);
            g_sigmas[i] = dt * g;
            for (int a = 0; a < 3; ++a) g_rgbs[3 * i + a] = w * gC[a];
            for (int a = 0; a < 3; ++a) Sc[a] += w * rgbs[3 * i + a];
            Sm += w * m;
        }
        free(P);
    }
}

/* ------------------------------------------------------------------------ */
/* Estimator update (Eq. 4, EMA form) and its sample points                  */
/* ------------------------------------------------------------------------ */

/* Cell c of level l at integer coords (i0,i1,i2), flat index
 * l*res^3 + (i0*res + i1)*res + i2.  Point per axis:
 * lmin + ((float)i + u) * width, u = 0.5 (centre) or SplitMix64 jitter:
 * stream seed ^ (step << 32), element 3*c + axis, top 24 bits / 2^24. */
void orc_grid_points(const float* aabb_min, const float* aabb_max, int res, int n_levels,
                     uint64_t seed, int64_t step, int jitter, float* xyz_out, int n_threads)
{
    orc_level lv[ORC_MAX_LEVELS];
    orc_levels(aabb_min, aabb_max, res, n_levels, lv);
    int64_t r3 = (int64_t)res * res * res;
    int64_t n = r3 * n_levels;
    uint64_t key = seed ^ ((uint64_t)step << 32);
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int64_t c = 0; c < n; ++c) {
        int l = (int)(c / r3);
        int64_t w = c % r3;
        int64_t i[3] = {w / ((int64_t)res * res), (w / res) % res, w % res};
        for (int a = 0; a < 3; ++a) {
            float u = jitter ? orc_u01(orc_splitmix64_at(key, (uint64_t)(3 * c + a))) : 0.5f;
            float q = (float)i[a] + u;
            xyz_out[3 * c + a] = lv[l].lmin[a] + q * lv[l].width[a];
        }
    }
}

/* ema <- decay*ema + (1-decay)*density (FP32, this operation order);
 * mean = FP64 mean of the updated ema; thr = max(thresh_abs, thresh_frac*mean);
 * bit c = (double)ema_c > thr. */
void orc_update_grid(int64_t n_cells, float* ema, const float* density, float decay,
                     float thresh_frac, float thresh_abs, uint32_t* bits_out, double* mean_out)
{
    float omd = 1.0f - decay;
    for (int64_t c = 0; c < n_cells; ++c) {
        float a = decay * ema[c];
        float b = omd * density[c];
        ema[c] = a + b;
    }
    double sum = 0.0;
    for (int64_t c = 0; c < n_cells; ++c) sum += (double)ema[c];
    double mean = n_cells > 0 ? sum / (double)n_cells : 0.0;
    double thr = (double)thresh_frac * mean;
    if ((double)thresh_abs > thr) thr = (double)thresh_abs;
    memset(bits_out, 0, sizeof(uint32_t) * (size_t)((n_cells + 31) / 32));
    for (int64_t c = 0; c < n_cells; ++c)
        if ((double)ema[c] > thr) bits_out[c >> 5] |= 1u << (c & 31);
    *mean_out = mean;
}

/* ------------------------------------------------------------------------ */
/* Inverse transform sampling from a piecewise-constant PDF (Eq. 1, Eq. 3)   */
/* ------------------------------------------------------------------------ */

/* Per ray: bins [e_j, e_{j+1}], weights w_j >= 0.  W = sum w (sequential FP32).
 * W > 0: F_0 = 0, F_j = (w_0 + ... + w_{j-1}) / W, F_n = 1; else F_j = j/n.
 * u_k = k / n_out (k = 0..n_out); stratified: inner u_k = (k + U_r)/n_out
 * clipped to 1, U_r = SplitMix64(seed, ray) in [0,1).  Bin j = largest
 * j in [0, n-1] with F_j <= u and F_j < 1 (for u < 1 the right-side search, so
 * a zero-weight bin is never entered from inside; u = 1 maps to the end of the
 * last bin with mass); t = e_j + ((u - F_j)/(F_{j+1} - F_j)) (e_{j+1} - e_j),
 * or e_j when F_{j+1} = F_j. */
void orc_sample_pdf(int64_t n_rays, int n_bins, const float* edges, const float* weights,
                    int n_out, int stratified, uint64_t seed, float* out, int n_threads)
{
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int64_t r = 0; r < n_rays; ++r) {
        const float* e = edges + r * (n_bins + 1);
        const float* w = weights + r * n_bins;
        float* F = (float*)malloc(sizeof(float) * (size_t)(n_bins + 1));
        float W = 0.0f;
        for (int j = 0; j < n_bins; ++j) W = W + w[j];
        if (W > 0.0f) {
            float c = 0.0f;
            F[0] = 0.0f;
            for (int j = 1; j < n_bins; ++j) {
                c = c + w[j - 1];
                F[j] = c / W;
            }
            F[n_bins] = 1.0f;
        } else {
            for (int j = 0; j <= n_bins; ++j) F[j] = (float)j / (float)n_bins;
        }
        float U = stratified ? orc_u01(orc_splitmix64_at(seed, (uint64_t)r)) : 0.0f;
        for (int k = 0; k <= n_out; ++k) {
            float u = (float)k / (float)n_out;
            if (stratified && k > 0 && k < n_out) {
                u = ((float)k + U) / (float)n_out;
                if (u > 1.0f) u = 1.0f;
            }
            int j = 0;
            for (int jj = 1; jj < n_bins; ++jj)
                if (F[jj] <= u && F[jj] < 1.0f) j = jj;
            float den = F[j + 1] - F[j];
            float t = e[j];
            if (den > 0.0f) t = e[j] + ((u - F[j]) / den) * (e[j + 1] - e[j]);
            out[r * (n_out + 1) + k] = t;
        }
        free(F);
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
