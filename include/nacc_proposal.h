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

/* BF16 copies of the weights of `params` (round to nearest, ties to even). */
int nacc_mlp_sync(const float* params, uint16_t* weights, void* stream);

/* Density at n points xyz [n][3] -> sigma [n]. */
int nacc_mlp_forward(int64_t n, const float* xyz, const float* params, const uint16_t* weights,
                     float* sigma, void* stream);

/*
 * Training, fused forward + adjoint over a batch of n points with target
 * densities: loss L = (1/n) sum (density - target)^2.  Adds dL/dparams
 * (layout of `params`) into grads [NACC_MLP_PARAMS] and sum (density -
 * target)^2 into *loss_sum (both [device], accumulated: the caller zeroes
 * them, or nacc_mlp_adam does).  The weight gradients are tensor-core
 * products over the batch (BF16 operands, FP32 accumulation).
 */
int nacc_mlp_train_grads(int64_t n, const float* xyz, const float* target, const float* params,
                         const uint16_t* weights, float* grads, float* loss_sum, void* stream);

/*
 * One Adam step on the FP32 master parameters (step = 1, 2, ...; bias
 * correction 1 - beta^step), then writes the BF16 weights and zeroes grads.
 * m, v: [device] [NACC_MLP_PARAMS] moment estimates (zero before step 1).
 */
int nacc_mlp_adam(float* params, float* grads, float* m, float* v, int64_t step, float lr, float beta1,
                  float beta2, float eps, uint16_t* weights, void* stream);

/* Diagnostics: the FP32 encoding e(x) of n points -> enc [n][64]. */
int nacc_mlp_encode(int64_t n, const float* xyz, float* enc, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NACC_PROPOSAL_H */
