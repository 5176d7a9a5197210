/*
 * nacc.h -- C ABI of the GB300 (sm_103a) occupancy-grid sampling and
 * differentiable volume-rendering library (the hot path of NerfAcc,
 * arXiv 2305.04966: Algorithm 1 "sampling" and "rendering", Sec. 4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers marked [device] must be CUDA device (or managed) memory that
 *    the caller owns and keeps alive until the work queued on `stream` has
 *    finished.  Pointers marked [host] are read during the call only.
 *  - Arrays are C-contiguous.  "[n][3]" means n rows of 3 floats (x, y, z or
 *    r, g, b).  Floating point is IEEE FP32 unless stated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues kernels on `stream` and returns; the
 *    only call that may synchronise is nacc_march_grid on a capacity
 *    overflow (see there).  No call allocates or frees device memory;
 *    temporary buffers are passed in as `scratch`.
 *  - Every call returns a status (NACC_OK = 0 or a negative NACC_ERR_*).
 *    On error nothing has been enqueued unless stated, and
 *    nacc_last_error() returns a message for the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Calls are thread-safe with respect to each other; work on the same
 *    buffers from different streams must be ordered by the caller.
 *  - Densities must be >= 0 and finite; interval ends t_end >= t_start.
 */
#ifndef NACC_H
#define NACC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NACC_OK 0
#define NACC_ERR_INVALID_ARG (-1) /* bad pointer, size or parameter; nothing enqueued */
#define NACC_ERR_CAPACITY (-2)    /* packed output too small; required size reported */
#define NACC_ERR_CUDA (-3)        /* a CUDA runtime call failed (launch or sync) */
#define NACC_ERR_TIMEOUT (-4)     /* reserved: a bounded device wait expired */
#define NACC_ERR_UNSUPPORTED (-5) /* valid request this library does not implement */

#define NACC_MAX_LEVELS 8

/* Cascaded occupancy grid (Table 1 "Spatial Skipping"; Instant-NGP-style
 * cascade).  Level l covers the level-0 box scaled by 2^l about its centre;
 * each level has res^3 cells.  Cell (i0, i1, i2) of level l has flat index
 *   c = l*res^3 + (i0*res + i1)*res + i2
 * and is occupied iff bit (c & 31) of bits[c >> 5] is set.  A point belongs
 * to the finest level whose closed box contains it, and to the cell
 * floor((x - lmin_l) * res / (lmax_l - lmin_l)) of that level (clamped to
 * [0, res-1]), all in FP32. */
typedef struct nacc_grid {
    float aabb_min[3];    /* level-0 box, aabb_min < aabb_max per axis */
    float aabb_max[3];
    int32_t res;          /* cells per axis per level, 1..1024, res^3 % 32 == 0 */
    int32_t n_levels;     /* 1..NACC_MAX_LEVELS */
    const uint32_t* bits; /* [device] n_levels*res^3/32 words (unused by update/points) */
} nacc_grid;

/* Lattice march parameters (Appendix B: step size, threshold). */
typedef struct nacc_march_params {
    float step;           /* lattice spacing dt > 0 */
    int32_t max_steps;    /* lattice index bound: k < max_steps, 1..2^24 */
    float t_min;          /* near plane: t_near = max(t_min, box entry) */
    float t_max;          /* far plane: t_far = min(t_max, box exit) */
    float early_stop_eps; /* with a field: stop once T < eps (Sec. 4.2, 1e-4); <= 0: never */
    int32_t exact_stops;  /* 0 (default): each early-stop decision is taken from bounds or from the
                             fast density where they prove the exact answer, else exactly; 1: every
                             decision in the exact arithmetic (slow; for validation).  Same result. */
} nacc_march_params;

/* Analytic density field used for early termination inside the march (the
 * "density_fn" of Algorithm 1, here a sum of isotropic Gaussian blobs):
 *   sigma(x) = sum_b peak_b * exp(-|x - mu_b|^2 / (2 std_b^2)).
 * The early-stop decision is defined on it in FP32 with a fixed operation
 * order: x = o + d*tm; per blob in order r2 = (dx*dx + dy*dy) + dz*dz,
 * s = s + peak * e(r2 * coef), coef = -0.5 / (std*std), where e is the
 * exponential defined by its steps (Cody-Waite reduction, degree-7 Taylor
 * polynomial, every operation one rounded FP32 operation; 0 below -86); the
 * depth is the lattice-order FP32 sum of s * (t1 - t0).  The march reaches
 * that decision exactly: from a bound on the ray's depth (sum over blobs of
 * the line integral plus twice the line maximum times dt), from a fast
 * closed-form depth with a proven error bound, or, near the threshold, in
 * the definition's own arithmetic.
 * rgb is only used by the harness field kernel (nacc_harness.h). */
typedef struct nacc_blob_field {
    int32_t n_blobs;    /* 0..1024 */
    const float* mu;    /* [device] [n_blobs][3] */
    const float* std;   /* [device] [n_blobs], > 0 */
    const float* peak;  /* [device] [n_blobs] */
    const float* rgb;   /* [device] [n_blobs][3] (may be NULL for the march) */
} nacc_blob_field;

/* Packed samples (Sec. 4.2 "Sample as Interval", "Packed Tensor"): sample s
 * is the interval [t_starts[s], t_ends[s]] on ray ray_indices[s]; the samples
 * of ray r are s in [offsets[r], offsets[r+1]), in increasing t. */
typedef struct nacc_packed {
    int64_t* offsets;     /* [device] [n_rays+1], written (CSR row pointer) */
    int32_t* ray_indices; /* [device] [capacity] or NULL (then not written) */
    float* t_starts;      /* [device] [capacity] */
    float* t_ends;        /* [device] [capacity] */
    int64_t capacity;     /* elements available in the three sample arrays */
    int64_t* n_samples;   /* [device] 1 element: total sample count, written */
} nacc_packed;

/* Message describing the last error on the calling thread ("" if none).
 * Library plumbing, no passage of the paper. */
const char* nacc_last_error(void);

/* Library version (major*10000 + minor*100 + patch).  Library plumbing. */
int nacc_version(void);

/* Scratch bytes nacc_march_grid needs for n_rays rays (the per-ray counts
 * from which the packed tensor's offsets are built, Sec. 4.2 "Packed
 * Tensor"): per-ray counts, stops and run records (~150 bytes per ray), the
 * grid's block summaries sized for the largest grid (8 levels of 1024^3
 * cells: 32.5 MiB) and a work counter of the early-stop pass.  Pure size
 * arithmetic: no device work, no error status. */
size_t nacc_march_scratch_bytes(int64_t n_rays);

/*
 * Occupancy-grid ray marching into packed samples.
 * Follows: Table 1 "Spatial Skipping" (occupied <=> bit set); Sec. 3.1
 * "Spatial Skipping" (skip empty regions); Sec. 4.2 "Sample as Interval",
 * "Packed Tensor", "No Gradient Filtering" (drop samples with T < 1e-4);
 * Appendix B hyper-parameters (step dt, resolution, threshold).
 *
 * Per ray r (o = rays_o[r], d = rays_d[r], FP32, every operation rounded):
 * [t_near, t_far] = slab clip of the ray against the outermost level's box,
 * intersected with [t_min, t_max]; lattice t0_k = t_near + k*step for
 * k < max_steps while t0_k < t_far; the interval [t0_k, t0_k + step] is
 * emitted iff the midpoint o + d*(t0_k + t1_k)/2 lies in an occupied cell.
 * Empty cells are skipped conservatively: the emitted set is exactly that of
 * the dense march.  With `field` non-NULL and eps > 0, sigma is evaluated at
 * each emitted midpoint and the ray stops at the first occupied k whose
 * accumulated optical depth sum(sigma*(t1-t0)) over the samples before it
 * exceeds -ln(eps) (T < eps).  Directions are used as given (not normalised).
 *
 * rays_o, rays_d: [device] [n_rays][3].  out: see nacc_packed; t_starts,
 * t_ends and ray_indices 16-byte aligned (the samples are written as 128-bit
 * stores).  scratch: [device] >= nacc_march_scratch_bytes(n_rays) bytes,
 * 256-byte aligned.
 * Capacity: if out->capacity >= n_rays*max_steps no overflow is possible and
 * the call never synchronises (CUDA-graph capturable).  Otherwise the call
 * synchronises `stream` after counting; if the total exceeds the capacity it
 * writes offsets and *n_samples but no samples and returns
 * NACC_ERR_CAPACITY (retry with capacity >= *n_samples).
 */
int nacc_march_grid(const nacc_grid* grid, const float* rays_o, const float* rays_d,
                    int64_t n_rays, const nacc_march_params* params,
                    const nacc_blob_field* field, nacc_packed* out, void* scratch,
                    size_t scratch_bytes, void* stream);

/* Scratch bytes nacc_march_unbounded needs for n_rays rays and a lattice of
 * max_steps points (Sec. 3.2 "Handling Unbounded Scenes"; 0 for invalid
 * arguments).  Pure size arithmetic. */
size_t nacc_march_unbounded_scratch_bytes(int64_t n_rays, int32_t max_steps);

/*
 * Lattice marching for unbounded scenes (Sec. 3.2 "Handling Unbounded
 * Scenes": sampling in s-space through a bijection Phi: s -> t).  Per ray,
 * for k = 0..K-1 (K = params->max_steps), FP32 with every operation rounded:
 *   s0 = k / K, s1 = (k+1) / K,  t = 1 / (a * (1 - s) + b * s),
 *   a = 1 / t_near, b = 1 / t_far  (t_near = params->t_min > 0, t_far =
 *   params->t_max finite: the disparity-linear Phi),
 *   tm = (t0 + t1) * 0.5, x = o + d * tm, c = contract(x):
 *   m = max|x_a|; c = x if m <= 1 else x * ((2 - 1/m) * (1/m)),
 * and [t0, t1] is emitted iff the cell of c (finest level whose box holds c,
 * clamped cell, as in nacc_march_grid) is occupied.  The grid covers the
 * contracted cube (e.g. 4 levels around [-0.25, 0.25]^3 reach [-2, 2]^3).
 * There is no ray-box clip.  Early termination as in nacc_march_grid, with
 * the field at x; the early-stop density keeps the blobs whose integral
 * along the ray line exceeds 1e-7 (peak >= 0 expected).  The output is that
 * of testing every lattice point; runs of 32 points whose contracted segment
 * is shown (by interval bounds with margins far above FP32 rounding) to lie
 * within one level and one cell clear of every occupied cell are skipped
 * without testing.  Outputs, scratch and capacity as nacc_march_grid
 * (scratch >= nacc_march_unbounded_scratch_bytes(n_rays, max_steps); it
 * includes 16.25 MiB of "any cell occupied" summaries of the bits over 4^3
 * and 16^3 blocks, rebuilt by every call).
 */
int nacc_march_unbounded(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                         const nacc_march_params* params, const nacc_blob_field* field, nacc_packed* out,
                         void* scratch, size_t scratch_bytes, void* stream);

/*
 * Inverse of the contraction of nacc_march_unbounded (Sec. 3.2), to evaluate
 * the scene at points of the contracted grid (e.g. the cell points of
 * nacc_grid_points for the estimator update).  Per point, FP32 with every
 * operation rounded: m' = max|c_a|; x = c if m' <= 1, else
 *   inv = 1 / (2 - min(m', 2 - 2^-23)),  x_a = c_a * (inv / m').
 * Points with m' >= 2 (outside the contracted cube) map to the image of
 * m' = 2 - 2^-23 (|x| about 8.4e6 m'), not to infinity.
 * c_in, x_out: [device] [n][3] float32 (may alias).  Errors: n < 0, NULL pointers.
 */
int nacc_uncontract_points(int64_t n, const float* c_in, float* x_out, void* stream);

/*
 * Sample points for the estimator update (Eq. 4; Sec. 3.1 "Spatial
 * Skipping": the cached density is refreshed every few steps at points of
 * each cell).  For every cell c of every level (flat index as in nacc_grid):
 *   xyz[c][a] = lmin_l[a] + ((float)i_a + u) * width_l[a],
 *   width_l = (lmax_l - lmin_l)/res,
 * u = 0.5 (jitter == 0, cell centre) or u = (h >> 40) * 2^-24 with
 * h = SplitMix64 output number 3c+a+1 of the stream seeded with
 * seed ^ (step << 32) (jitter != 0).  xyz_out: [device] [n_levels*res^3][3].
 */
int nacc_grid_points(const nacc_grid* grid, uint64_t seed, int64_t step, int32_t jitter,
                     float* xyz_out, void* stream);

/* Scratch bytes nacc_update_grid needs for n_cells cells (the FP64 partial
 * sums of the mean that sets the threshold of Table 1's binarisation).  Pure
 * size arithmetic. */
size_t nacc_update_grid_scratch_bytes(int64_t n_cells);

/*
 * Estimator update F: T^{k-1} -> T^k (Eq. 4) in its EMA form (Sec. 3.1
 * "Spatial Skipping") and binarisation 1[sigma > tau] (Table 1):
 *   ema[c] <- decay*ema[c] + (1-decay)*density[c]   (FP32, this order)
 *   mean   =  FP64 mean of the updated ema over all n_levels*res^3 cells
 *   thr    =  max(thresh_abs, thresh_frac * mean)    (FP64)
 *   bit c of bits_out = ((double)ema[c] > thr)
 * decay = 0 initialises ema from density.  ema: [device] in/out,
 * density: [device], bits_out: [device] n_cells/32 words (may alias
 * grid->bits of a later march).  scratch: [device] >=
 * nacc_update_grid_scratch_bytes(n_cells) bytes, 256-byte aligned.
 */
int nacc_update_grid(const nacc_grid* grid, float* ema, const float* density, float decay,
                     float thresh_frac, float thresh_abs, uint32_t* bits_out, void* scratch,
                     size_t scratch_bytes, void* stream);

/*
 * Estimator update for dynamic scenes (Sec. 4.3 "Dynamic NeRFs": one grid
 * shared by all frames marks the maximum occupancy over the timestamps): as
 * nacc_update_grid with density[c] = max over f < n_frames of
 * densities[f * n_cells + c].  n_frames = 1 is nacc_update_grid.
 */
int nacc_update_grid_frames(const nacc_grid* grid, float* ema, const float* densities, int32_t n_frames,
                            float decay, float thresh_frac, float thresh_abs, uint32_t* bits_out, void* scratch,
                            size_t scratch_bytes, void* stream);

/*
 * Estimator updated by gradient descent through the rendering loss (the
 * Plenoxels variant of Sec. 3.1 "Spatial Skipping"): the grid holds a density
 * per cell.  nacc_grid_density_lookup writes sigma_out[i] = density of the
 * cell of sample i's midpoint -- tm = (t0 + t1) * 0.5, x = o + d * tm, the
 * finest level whose box holds x, clamped cell, the FP32 definition of
 * nacc_march_grid -- or 0 outside every level.  nacc_grid_density_backward
 * adds g_sigma[i] into g_density[cell of i] (atomic FP32 adds: the order of
 * the additions is not fixed).  The sample count is read on the device from
 * *n_samples.  All arrays [device].
 */
int nacc_grid_density_lookup(const nacc_grid* grid, const float* density, const float* rays_o, const float* rays_d,
                             const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                             const int64_t* n_samples, float* sigma_out, void* stream);
int nacc_grid_density_backward(const nacc_grid* grid, const float* rays_o, const float* rays_d,
                               const int32_t* ray_indices, const float* t_starts, const float* t_ends,
                               const int64_t* n_samples, const float* g_sigma, float* g_density, void* stream);

/*
 * One gradient step of that grid (Sec. 3.1 "Spatial Skipping": Plenoxels
 * updates the cached density by gradient descent through the rendering
 * loss): density[c] = max(density[c] - lr * g_density[c], 0) (FP32, rounded
 * in this order), g_density[c] = 0, bit c of bits_out = (density[c] >
 * thresh).  density, g_density: [device] [n_levels*res^3]; bits_out:
 * [device] n_cells/32 words.  Invalid sizes or NULL -> NACC_ERR_INVALID_ARG.
 */
int nacc_update_grid_sgd(const nacc_grid* grid, float* density, float* g_density, float lr, float thresh,
                         uint32_t* bits_out, void* stream);

/*
 * Allocation-free variant of nacc_update_grid (the paper has no counterpart;
 * this is a property of this library's interface).  Same arguments, same
 * arithmetic and same results as nacc_update_grid, but the temporary FP64
 * partial sums live in an array inside the library instead of a caller
 * buffer, so the call performs no device allocation of any kind.  Intended
 * for callers that cannot allocate on the path that refreshes the grid,
 * e.g. code hosted in an application that owns the whole device memory
 * budget and forbids allocations after start-up, or a latency-critical
 * thread that must not pay for the synchronisation an allocation can imply.
 *  - Limit: n_levels*res^3 <= 134,217,728 cells (2^27, e.g. 8 levels of
 *    256^3); larger grids are rejected with NACC_ERR_INVALID_ARG and a
 *    message naming the limit.
 *  - The array (512 KiB + 24 B) is held by every GPU that loads the library,
 *    until the process exits.
 *  - The first call in each CUDA context (per device, and again after a
 *    device reset or a new primary context) looks up the array's device
 *    address in that context; make that first call before any stream
 *    capture in it.
 *  - All calls share the one array and it keeps the last call's contents;
 *    every element a call reads is written earlier in the same call.  Calls
 *    whose GPU work overlaps (e.g. on two streams) race on the array: order
 *    them on one stream.
 */
int nacc_update_grid_noalloc(const nacc_grid* grid, float* ema, const float* density,
                             float decay, float thresh_frac, float thresh_abs,
                             uint32_t* bits_out, void* stream);

/*
 * Inverse transform sampling from a piecewise-constant PDF (Eq. 1), with
 * the CDF read as 1 - T (Eq. 3; Table 1 "PDF Approaches").  Per ray, bins
 * [e_j, e_{j+1}] (j < n_bins) carry weights w_j >= 0 (FP32 throughout):
 *   W = w_0 + ... + w_{n-1} (sequential); if W > 0: F_0 = 0,
 *   F_j = (w_0 + ... + w_{j-1}) / W, F_n = 1; else F_j = j/n (uniform).
 *   u_k = k/n_out for k = 0..n_out; stratified != 0: for 0 < k < n_out,
 *   u_k = min(1, (k + U_r)/n_out), U_r = top 24 bits of SplitMix64 output
 *   r+1 of the stream seeded with `seed`, times 2^-24.
 *   j = largest j in [0, n-1] with F_j <= u_k and F_j < 1;
 *   t_k = e_j + ((u_k - F_j)/(F_{j+1} - F_j)) * (e_{j+1} - e_j), or e_j if
 *   F_{j+1} == F_j.
 * edges: [device] [n_rays][n_bins+1] non-decreasing; weights: [device]
 * [n_rays][n_bins]; edges_out: [device] [n_rays][n_out+1].
 * n_bins 1..4096, n_out 1..4096.
 */
int nacc_sample_pdf(int64_t n_rays, int32_t n_bins, const float* edges, const float* weights,
                    int32_t n_out, int32_t stratified, uint64_t seed, float* edges_out,
                    void* stream);

/*
 * Differentiable volume rendering of packed samples, forward (Eq. 2
 * discretised; Table 1 "PDF Approaches" row; Algorithm 1 "rendering").
 * Per ray r over its samples i (tau_i = sigma_i*(t1_i - t0_i)):
 *   P_i = sum_{j<i} tau_j, T_i = exp(-P_i); sample i is masked when
 *   early_stop_eps > 0 and P_i > -ln(eps) (T_i < eps, Sec. 4.2);
 *   w_i = T_i*(1 - exp(-tau_i)) for unmasked i, else 0;
 *   T_N = exp(-sum of tau_i over unmasked i);
 *   rgb_out = sum w_i c_i + T_N*bg, opacity_out = sum w_i,
 *   depth_out = sum w_i*(t0_i + t1_i)/2, trans_out = T_N.
 * Rays with no samples give rgb = bg, opacity = depth = 0, trans = 1.
 * offsets: [device] [n_rays+1] CSR with offsets[0] = 0 (the total sample
 * count is read on the device from offsets[n_rays]); t_starts, t_ends,
 * sigmas: [device] [S]; rgbs: [device] [S][3], all four 16-byte aligned
 * (groups of four samples move as 128-bit loads); bg: [host] 3 floats;
 * outputs [device]: rgb_out [n_rays][3], opacity_out, depth_out, trans_out
 * [n_rays]; weights_out [S] or NULL.
 */
int nacc_render_fwd(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                    const float* t_ends, const float* sigmas, const float* rgbs, const float* bg,
                    float early_stop_eps, float* rgb_out, float* opacity_out, float* depth_out,
                    float* trans_out, float* weights_out, void* stream);

/*
 * Adjoint of nacc_render_fwd (Algorithm 1: the radiance field receives
 * gradients through rendering).  With g_C = g_rgb[r], g_A = g_opacity[r],
 * g_D = g_depth[r], T_{i+1} = exp(-(P_i + tau_i)), m_i = (t0_i + t1_i)/2,
 * S^c_i = sum_{k>i} w_k c_k, S^m_i = sum_{k>i} w_k m_k (unmasked k):
 *   g_rgbs[i]   = w_i * g_C
 *   g_sigmas[i] = (t1_i - t0_i) * ( g_C . (T_{i+1} c_i - S^c_i - T_N bg)
 *                                 + g_A*T_N + g_D*(T_{i+1} m_i - S^m_i) )
 * and 0 for masked samples.  Per-sample transmittance is recomputed, not
 * saved.  Inputs as nacc_render_fwd plus [device] g_rgb [n_rays][3],
 * g_opacity [n_rays], g_depth [n_rays] (any of the three may be NULL =
 * zero); outputs [device] g_sigmas [S], g_rgbs [S][3].
 */
int nacc_render_bwd(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                    const float* t_ends, const float* sigmas, const float* rgbs, const float* bg,
                    float early_stop_eps, const float* g_rgb, const float* g_opacity,
                    const float* g_depth, float* g_sigmas, float* g_rgbs, void* stream);

/*
 * Checkpointed pair of nacc_render_fwd / nacc_render_bwd (Algorithm 1: the
 * forward rendering, then gradients through it).  Results are bit-identical
 * to the plain pair.  The forward pass also writes, per ray, a 64-byte record
 * of what the adjoint would otherwise recompute in a first sweep over the
 * ray's samples: the optical depth at the start of each 128-position chunk
 * (the chunks the kernels cut a ray into, counted from the ray's first
 * sample rounded down to a multiple of 4), the position of the mask cut
 * (Sec. 4.2) and the kept optical depth (T_N = exp(-depth)).  This is not
 * per-sample transmittance: 16 words per ray, whatever the ray's length.
 * The adjoint reads the record and makes one pass over the samples instead
 * of two.  Rays of more than 14 chunks (1,792 samples) get a record marked
 * as absent, and the adjoint falls back to its own sweep for them.
 * ckpt_out / ckpt: [device] nacc_render_ckpt_bytes(n_rays) bytes, 16-byte
 * aligned, caller-owned; written by nacc_render_fwd_ckpt and read by
 * nacc_render_bwd_ckpt, which must get the same offsets, sample arrays
 * and early_stop_eps (a record whose chunk count exceeds its ray's is
 * ignored; any other mismatch gives wrong gradients, never an access
 * outside the arrays).  Other arguments and errors as the plain pair; NULL
 * or misaligned ckpt -> NACC_ERR_INVALID_ARG.
 */
size_t nacc_render_ckpt_bytes(int64_t n_rays);
int nacc_render_fwd_ckpt(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                         const float* t_ends, const float* sigmas, const float* rgbs, const float* bg,
                         float early_stop_eps, float* rgb_out, float* opacity_out, float* depth_out,
                         float* trans_out, float* weights_out, float* ckpt_out, void* stream);
int nacc_render_bwd_ckpt(int64_t n_rays, const int64_t* offsets, const float* t_starts,
                         const float* t_ends, const float* sigmas, const float* rgbs, const float* bg,
                         float early_stop_eps, const float* g_rgb, const float* g_opacity,
                         const float* g_depth, const float* ckpt, float* g_sigmas, float* g_rgbs,
                         void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NACC_H */
