/*
 * nacc_harness.h -- benchmark / test harness kernels shipped in the same
 * library as nacc.h.  They are NOT the method: they stand in for the user's
 * radiance field (the "density_fn" / "rgb_density_fn" of Algorithm 1 in
 * NerfAcc, arXiv 2305.04966) and for the training loss, so that a full
 * sampling -> rendering -> gradient step can run on synthetic scenes.
 * Conventions (device/host pointers, streams, status codes) as in nacc.h.
 */
#ifndef NACC_HARNESS_H
#define NACC_HARNESS_H

#include <stddef.h>
#include <stdint.h>

#include "nacc.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Analytic blob field at the midpoints of packed samples (Algorithm 1
 * rgb_density_fn): x = rays_o[r] + rays_d[r]*(t0+t1)/2 with r =
 * ray_indices[s]; sigma = sum_b peak_b exp(-|x-mu_b|^2/(2 std_b^2));
 * rgb = sum_b sigma_b rgb_b / sigma (0 where sigma == 0).  The sample count
 * is read on the device from *n_samples, so no host synchronisation is
 * needed.  Writes sigmas [S] and rgbs [S][3] (both [device]).
 */
int nacc_harness_field(const float* rays_o, const float* rays_d, const int32_t* ray_indices,
                       const float* t_starts, const float* t_ends, const int64_t* n_samples,
                       const nacc_blob_field* field, float* sigmas, float* rgbs, void* stream);

/*
 * The same field (harness: Algorithm 1's rgb_density_fn) for a packed sample
 * set given by its CSR offsets
 * [n_rays+1] (no ray_indices needed): one warp per ray evaluates the blobs
 * along the ray in the closed form peak_b 2^(A_b (t - t*_b)^2 + C_b) (t*_b
 * the closest approach, set up once per ray) with the hardware exp2; the
 * relative error is ~1e-5 (FP32 rounding of t - t*_b).  Fields of more than
 * 16 blobs keep, per ray, only the blobs whose integral along the whole ray
 * line exceeds 1e-7 (bound peak_b 2^C_b sqrt(2 pi) std_b / |d|), so each
 * dropped blob changes sigma by at most 1e-7 |d| / (sqrt(2 pi) std_b).  At
 * most 256 blobs; t_starts, t_ends, sigmas, rgbs 16-byte aligned.  Outputs
 * as above.
 */
int nacc_harness_field_rays(const float* rays_o, const float* rays_d, int64_t n_rays, const int64_t* offsets,
                            const float* t_starts, const float* t_ends, const nacc_blob_field* field,
                            float* sigmas, float* rgbs, void* stream);

/* Density of the blob field (harness: Algorithm 1's density_fn, here for the
 * estimator update's cell points) at n points xyz [n][3] -> sigma [n] (both
 * [device]). */
int nacc_harness_field_points(int64_t n, const float* xyz, const nacc_blob_field* field,
                              float* sigma, void* stream);

/*
 * Harness loss (Algorithm 1's training loss, whose gradient rendering
 * back-propagates): mean squared error against a target image and its
 * gradient:
 *   loss = sum (rgb - target)^2 / (3 n),  g_rgb = 2 (rgb - target) / (3 n).
 * rgb, target, g_rgb: [device] [n][3]; loss: [device] 1 float.
 */
int nacc_harness_l2_loss(int64_t n, const float* rgb, const float* target, float* g_rgb,
                         float* loss, void* stream);

/*
 * Library plumbing, no passage of the paper.  Device status of the bounded
 * waits inside the library's kernels (the
 * proposal network's tensor-core kernels and the wait self-test).  Every
 * wait on an mbarrier gives up after 2 s of GPU wall time; the kernel then
 * records the expiry in a device status word and returns instead of hanging.  This call synchronises `stream`, reads and
 * clears that word, and writes NACC_OK or NACC_ERR_TIMEOUT to *status_out
 * [host].  Returns NACC_OK unless a CUDA call failed.
 */
int nacc_device_status(void* stream, int32_t* status_out);

/*
 * Diagnostics (library plumbing): launches one tiny kernel that waits, with
 * the library's
 * bounded-wait routine, on an mbarrier nothing will ever arrive on, giving up
 * after limit_ns nanoseconds (0 < limit_ns <= 1e8).  The expiry is reported
 * through nacc_device_status; the context stays usable.
 */
int nacc_selftest_wait_timeout(int64_t limit_ns, void* stream);

/*
 * Diagnostics (library plumbing): timing of the count phase of
 * nacc_march_grid and nacc_march_unbounded (the run walk and, with a field,
 * the early-stop pass).  While set (by the calling host thread), every
 * nacc_march_grid or nacc_march_unbounded call of that thread records
 * `before` on its stream just before the run-walk kernel and `after` just
 * after the early-stop kernels (or the walk, without a field), so the caller
 * can read their duration with cudaEventElapsedTime.
 * before, after: cudaEvent_t handles created by the caller (NULL, NULL turns
 * the recording off).  The events are not owned by the library.
 */
int nacc_set_march_count_events(void* before, void* after);

#ifdef __cplusplus
}
#endif

#endif /* NACC_HARNESS_H */
