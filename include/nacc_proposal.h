/*
 * nacc_proposal.h -- the learned density proposal of the estimator
 * (NerfAcc, arXiv 2305.04966: Table 1 "PDF Approaches", Sec. 3.2 -- a small
 * network predicts density along the ray; its transmittance defines the PDF
 * that inverse transform sampling, Eq. 1 / nacc_sample_pdf, resamples).
 *
 * Network: encoding e(x) = [x, y, z, then for k = 0..7 and each axis a:
 * sin(2^k pi x_a), cos(2^k pi x_a)] (51 values, zero-padded to 64);
 * h1 = relu(W1 e + b1), h2 = relu(W2 h1 + b2) (width 64), density =
 * softplus(w3 . h2 + b3).  BF16 operands (weights and each layer's input),
 * FP32 accumulation (tcgen05 tensor cores, accumulators in tensor memory),
 * FP32 biases.
 *
 * Parameters: one FP32 array of NACC_MLP_PARAMS values (the master copy):
 * W1 [64][64] (row = output unit) at 0, b1 [64] at 4096, W2 [64][64] at
 * 4160, b2 [64] at 8256, w3 [64] at 8320, b3 at 8384.  The kernels read the
 * BF16 weights from a second array of NACC_MLP_WEIGHTS values: W1 at 0, W2
 * at 4096, w3 at 8192 (bfloat16 bit patterns), written by nacc_mlp_sync or
 * by nacc_mlp_adam.  All pointers are [device], 16-byte aligned; every call
 * is asynchronous on `stream` and returns a nacc status code.
 */
#ifndef NACC_PROPOSAL_H
#define NACC_PROPOSAL_H

#include <stddef.h>
#include <stdint.h>

#include "nacc.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NACC_MLP_PARAMS 8385
#define NACC_MLP_WEIGHTS 8256

/* BF16 copies of the weights of `params` (round to nearest, ties to even):
 * the tensor-core operands of the proposal network (Sec. 3.1 "PDF
 * Approaches").  params [NACC_MLP_PARAMS] FP32, weights [NACC_MLP_WEIGHTS]. */
int nacc_mlp_sync(const float* params, uint16_t* weights, void* stream);

/* Density of the proposal network (Sec. 3.1 "PDF Approaches": a small MLP
 * predicts the densities whose transmittance is the estimator) at n points
 * xyz [n][3] -> sigma [n]. */
int nacc_mlp_forward(int64_t n, const float* xyz, const float* params, const uint16_t* weights,
                     float* sigma, void* stream);

/*
 * Training, fused forward + adjoint over a batch of n points with target
 * densities (the estimator update F of Eq. 4 by gradient descent, as the
 * PDF approaches of Sec. 3.1 update theirs; the target here is the
 * analytic field's density): loss L = (1/n) sum (density - target)^2.  Adds dL/dparams
 * (layout of `params`) into grads [NACC_MLP_PARAMS] and sum (density -
 * target)^2 into *loss_sum (both [device], accumulated: the caller zeroes
 * them, or nacc_mlp_adam does).  The weight gradients are tensor-core
 * products over the batch (BF16 operands, FP32 accumulation).
 */
int nacc_mlp_train_grads(int64_t n, const float* xyz, const float* target, const float* params,
                         const uint16_t* weights, float* grads, float* loss_sum, void* stream);

/*
 * The same network on rows that are already its layer-1 input: the encoding
 * in the operand precision, enc [n][64] BF16 (bit patterns, 16-byte aligned
 * rows; columns 51..63, the encoding's zero padding, are ignored).  Sec. 3.1
 * "PDF Approaches" (the proposal network).  These let a caller (the parity
 * tests) feed both this library and a reference the identical operands;
 * nacc_mlp_forward_encoded -> sigma [n] as nacc_mlp_forward,
 * nacc_mlp_train_grads_encoded accumulates as nacc_mlp_train_grads.
 * Errors: n < 0, NULL pointers, enc misaligned.
 */
int nacc_mlp_forward_encoded(int64_t n, const uint16_t* enc, const float* params, const uint16_t* weights,
                             float* sigma, void* stream);
int nacc_mlp_train_grads_encoded(int64_t n, const uint16_t* enc, const float* target, const float* params,
                                 const uint16_t* weights, float* grads, float* loss_sum, void* stream);

/*
 * The gradient-descent step of that update (Eq. 4 with SGD-type F, Sec. 3.1):
 * one Adam step on the FP32 master parameters (step = 1, 2, ...; bias
 * correction 1 - beta^step), then writes the BF16 weights and zeroes grads.
 * m, v: [device] [NACC_MLP_PARAMS] moment estimates (zero before step 1).
 */
int nacc_mlp_adam(float* params, float* grads, float* m, float* v, int64_t step, float lr, float beta1,
                  float beta2, float eps, uint16_t* weights, void* stream);

/*
 * Density at the midpoints of the bins of rays, the piecewise-constant
 * densities of Sec. 3.1 "PDF Approaches": point (r, j) = o_r + t d_r
 * with t = (edges[r][j] + edges[r][j+1]) / 2 (FP32) -> sigma [n_rays][n_bins];
 * edges [n_rays][n_bins+1].  Same network and precision as nacc_mlp_forward.
 */
int nacc_mlp_forward_rays(int64_t n_rays, int32_t n_bins, const float* rays_o, const float* rays_d,
                          const float* edges, const float* params, const uint16_t* weights, float* sigma,
                          void* stream);

/*
 * Initial bins of the proposal estimator over the bounded range [t_n, t_f]
 * of Sec. 3.1 (Eq. 1): [t_near, t_far] = slab clip of
 * each ray against the box of the grid's level 0 (individually rounded FP32,
 * as in nacc_march_grid), intersected with [t_min, t_max], cut into n_bins
 * equal bins: edges[r][j] = t_near + (t_far - t_near) * (j / n_bins) (each
 * operation rounded), edges[r][n_bins] = t_far.  A ray that misses gets
 * t_near = t_far = max(t_min, 0) (empty bins).  edges [n_rays][n_bins+1].
 */
int nacc_uniform_edges(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                       float t_min, float t_max, int32_t n_bins, float* edges, void* stream);

/*
 * Transmittance weights of densities on a dense bin layout (Eq. 2 /
 * Table 1 "PDF Approaches"): tau_j = sigma_j (e_{j+1} - e_j), P_j = sum_{i<j}
 * tau_i, w_j = exp(-P_j) (1 - exp(-tau_j)) (FP32); trans_out [n_rays] (may
 * be NULL) = exp(-sum tau).  sigmas, weights [n_rays][n_bins].
 */
int nacc_dense_weights(int64_t n_rays, int32_t n_bins, const float* edges, const float* sigmas, float* weights,
                       float* trans_out, void* stream);

/*
 * The bins as packed samples (Sec. 4.2 "Packed Tensor"; nacc_packed layout
 * without ray_indices):
 * offsets[r] = r * n_bins, t_starts[r*n_bins + j] = edges[r][j], t_ends =
 * edges[r][j+1], *n_samples = n_rays * n_bins (all [device]).
 */
int nacc_edges_to_packed(int64_t n_rays, int32_t n_bins, const float* edges, int64_t* offsets, float* t_starts,
                         float* t_ends, int64_t* n_samples, void* stream);

/*
 * Combined estimator (the occupancy grid stacked on the proposal network,
 * Sec. 3.3 "Insights from Unified Formulation", Sec. 4.4 "Combined Sampling"):
 * the occupied range of each ray -- t0 of its first and t1 of its last
 * occupied lattice point, i.e. of the samples nacc_march_grid would emit
 * without a field (same FP32 lattice definition) -- into t_lo, t_hi
 * [n_rays] ([device]).  A ray with no occupied point gets t_lo = t_hi =
 * t_near, or max(t_min, 0) if it misses the grid.  params->early_stop_eps
 * is ignored.  scratch: [device] >= nacc_occupied_range_scratch_bytes(),
 * 256-byte aligned (the grid's block summaries, sized for the largest grid:
 * 32.5 MiB).
 */
size_t nacc_occupied_range_scratch_bytes(void);
int nacc_occupied_range(const nacc_grid* grid, const float* rays_o, const float* rays_d, int64_t n_rays,
                        const nacc_march_params* params, float* t_lo, float* t_hi, void* scratch,
                        size_t scratch_bytes, void* stream);

/*
 * n_bins equal bins of [t_lo[r], t_hi[r]] per ray (the combined estimator's
 * initial bins, Sec. 4.4), the arithmetic of nacc_uniform_edges -> edges
 * [n_rays][n_bins+1].
 */
int nacc_range_edges(int64_t n_rays, const float* t_lo, const float* t_hi, int32_t n_bins, float* edges,
                     void* stream);

/*
 * Unbounded scenes (Sec. 3.2): the proposal density at the contracted bin
 * midpoints, c(o + t d) with t as in nacc_mlp_forward_rays and c the
 * contraction of nacc_march_unbounded (FP32, each operation rounded:
 * m = max|x_a|, x * ((2 - 1/m) * (1/m)) if m > 1).  The network's input
 * domain is the contracted cube [-2, 2]^3.  Arguments as nacc_mlp_forward_rays.
 */
int nacc_mlp_forward_rays_contracted(int64_t n_rays, int32_t n_bins, const float* rays_o, const float* rays_d,
                                     const float* edges, const float* params, const uint16_t* weights,
                                     float* sigma, void* stream);

/*
 * The contraction itself (Sec. 3.2 "Handling Unbounded Scenes") for n
 * points (e.g. the training inputs of the
 * proposal network for unbounded scenes): x_in, c_out [device] [n][3]
 * (may alias).
 */
int nacc_contract_points(int64_t n, const float* x_in, float* c_out, void* stream);

/*
 * Initial bins of the proposal estimator for unbounded scenes (Sec. 3.2
 * "Handling Unbounded Scenes": sampling uniform in s through a bijection
 * Phi): uniform in s, mapped to t by the disparity-linear Phi of
 * nacc_march_unbounded:
 * edges[r][j] = 1 / (a (1 - s_j) + b s_j), s_j = j / n_bins, a = 1/t_near,
 * b = 1/t_far (FP32, each operation rounded), the same row for every ray.
 * edges: [device] [n_rays][n_bins+1].  Requires 0 < t_near < t_far < inf.
 */
int nacc_phi_edges(int64_t n_rays, int32_t n_bins, float t_near, float t_far, float* edges, void* stream);

/* Diagnostics: the FP32 frequency encoding e(x) that the proposal network
 * (Sec. 3.1 "PDF Approaches") reads, for n points -> enc [n][64]. */
int nacc_mlp_encode(int64_t n, const float* xyz, float* enc, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NACC_PROPOSAL_H */
