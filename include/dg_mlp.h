/*
 * dg_mlp.h -- C ABI of the load-surrogate multilayer perceptron.
 *
 * Not part of the paper's method: a small network that predicts the next
 * lift and drag coefficients of a cylinder from a window of its rigid-body
 * state and force history plus (U*, m*, Re).  It is trained on trajectories
 * that the DG solver generates and is used as the load predictor of the
 * weakly coupled rigid-body step (Algorithm 3), with the DG solve as its
 * fallback and as the judge of its error.
 *
 * Network: depth hidden layers of `width` units with GELU
 * (z Phi(z) = z (1 + erf(z / sqrt 2)) / 2), a linear output layer:
 *     h_0 = x, h_l = GELU(h_{l-1} W_l^T + b_l), y = h_depth W_out^T + b_out.
 * Arithmetic: every matrix product runs on the tensor cores with bfloat16
 * inputs (the weights and the activations, rounded to nearest even) and FP32
 * accumulation; biases, activations, the loss and the optimizer are FP32.
 * Training minimises the mean over batch and outputs of (y - t)^2 with Adam
 * (beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected).
 *
 * Two implementations of the same arithmetic:
 * - chunked (the default when the network fits: inputs and width <= 128,
 *   outputs <= 16, at most 8 layers): one kernel carries chunks of 32 rows
 *   through the forward pass, the loss and the backward pass in shared
 *   memory and leaves per-block gradient sums; a second adds them in block
 *   order and applies Adam (two launches per training step);
 * - layer by layer: one tiled GEMM per product with fused epilogues, and
 *   separate loss, bias-sum, Adam and weight-copy kernels.
 * Both round to bfloat16 at the same points; their FP32 sums run in
 * different orders.  Each is deterministic.
 *
 * Parameters (FP32, this order): for each layer, W row-major [n_out][n_in]
 * then b [n_out].  The library keeps the FP32 master copy, the Adam moments
 * and the bfloat16 copy of the weights on the device.  All calls run on a
 * stream the network creates and synchronise it before returning.
 */
#ifndef DG_MLP_H
#define DG_MLP_H

#include <stdint.h>

#include "dg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_mlp dg_mlp;

/* Create a network on the current device for batches of at most max_batch
 * rows: n_in inputs, depth >= 1 hidden layers of width units, n_out outputs.
 * Weights uniform in +-sqrt(6 / (n_in + n_out)) of their layer from a
 * SplitMix64 stream seeded with `seed`, biases zero, Adam state zero.
 * Errors: DG_EINVAL (a size < 1, width or n_in > 4096, max_batch > 1 << 20),
 * DG_ECUDA.  *out is NULL on failure. */
dg_status dg_mlp_create(int n_in, int width, int depth, int n_out, int max_batch, uint64_t seed, dg_mlp **out);

/* Free the network.  NULL is accepted. */
dg_status dg_mlp_destroy(dg_mlp *m);

/* Message of the last failed call (empty after success). */
const char *dg_mlp_last_error(const dg_mlp *m);

/* Number of parameters (the length of the arrays below). */
int64_t dg_mlp_param_count(const dg_mlp *m);

/* Kernel launches made so far. */
int64_t dg_mlp_kernel_launches(const dg_mlp *m);

/* Copy the FP32 parameters in (resets the Adam moments and step count) or
 * out; host pointer if on_device == 0, device pointer otherwise.
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_mlp_set_params(dg_mlp *m, const float *params, int on_device);
dg_status dg_mlp_get_params(dg_mlp *m, float *params, int on_device);

/* Use the chunked implementation (on != 0) or the layer-by-layer one.
 * Errors: DG_EINVAL, DG_EUNSUPPORTED (on, but the network does not fit the
 * chunked path). */
dg_status dg_mlp_set_fused(dg_mlp *m, int on);

/* 1 if the chunked implementation is in use, else 0 (also for NULL). */
int dg_mlp_is_fused(const dg_mlp *m);

/* y = net(x) for B rows: X device [B][n_in] FP32, Y device [B][n_out] FP32.
 * Errors: DG_EINVAL (null, B < 1 or > max_batch), DG_ECUDA. */
dg_status dg_mlp_forward(dg_mlp *m, const float *X, int B, float *Y);

/* Loss and its gradient with respect to every parameter for targets T
 * (device [B][n_out]); grad device [param_count], loss device [1].
 * Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_mlp_loss_grad(dg_mlp *m, const float *X, const float *T, int B, float *grad, float *loss);

/* nsteps Adam steps of full-batch training on (X, T) with learning rate lr;
 * loss_hist (device [nsteps] FP32, or NULL) receives the loss before each
 * update.  From 8 steps on, one captured step is replayed from a CUDA graph
 * (same kernels and arguments, kept for the next call with the same X, T,
 * B, lr and loss_hist).  Errors: DG_EINVAL, DG_ECUDA. */
dg_status dg_mlp_train(dg_mlp *m, const float *X, const float *T, int B, int nsteps, float lr, float *loss_hist);

#ifdef __cplusplus
}
#endif

#endif /* DG_MLP_H */
