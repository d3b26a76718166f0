/*
 * mvsk_mlp.h — C ABI of the learned warm start of the batched YAND-MVSK solver.
 *
 * The paper starts every solve from x^0 = 1/n (Sec. 5) and accepts any start in
 * Delta(tau), judging the result by its own KKT test.  The warm start maps a
 * request (preference vector lambda, optional target, and a sketch of the
 * panel) to a start: a multilayer perceptron of n_hidden ReLU layers of width
 * d_hidden, x^0 = Pi_Delta(tau)(y / n) of its output y in R^n.  It is trained
 * against solver outputs (y target n w*), by mean-squared error and Adam.
 * The solve itself is unchanged: it runs from x^0 to the requested tolerance.
 *
 * Precision: weights, activations and back-propagated errors are BF16 where
 * they enter a product (tcgen05 tensor-core GEMMs, FP32 accumulation); the
 * pre-activations, gradients, Adam moments and master weights are FP32.
 *
 * Pointers: every array argument is a DEVICE pointer unless marked "host or
 * device".  Row-major throughout.  No call on a network allocates after
 * mvsk_mlp_create; mvsk_mlp_features allocates and frees 544 bytes of device
 * scratch and synchronises the device.
 * Errors: MVSK_EINVAL for bad sizes (B < 1 or B > max_batch, non-positive
 * dimensions, d_in not a multiple of 8), MVSK_ECUDA for CUDA failures or an
 * in-kernel wait that ran out (the GEMMs' bounded mbarrier waits).
 */
#ifndef MVSK_MLP_H
#define MVSK_MLP_H

#include <stdint.h>

#include "mvsk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mvsk_mlp mvsk_mlp; /* opaque; owns its device memory */

/* Width of the request features (mvsk_mlp_features): lambda (4), target and
 * its flag (2), 2 x 32 sketch entries, zero padding. */
#define MVSK_MLP_D_IN 128

/* Network d_in -> d_hidden (n_hidden ReLU layers) -> d_out, weights He-normal
 * from a SplitMix64 / Box-Muller stream of `seed`, biases 0; buffers for
 * batches of up to max_batch rows (a multiple of 8).  d_in, d_hidden and d_out
 * must be multiples of 8; n_hidden >= 1. */
mvsk_status mvsk_mlp_create(int32_t d_in, int32_t d_hidden, int32_t n_hidden, int32_t d_out, int32_t max_batch,
                            uint64_t seed, mvsk_mlp** out);
mvsk_status mvsk_mlp_destroy(mvsk_mlp* mlp);

/* Y (B x d_out, FP32) = network(X) for X (B x d_in, FP32). */
mvsk_status mvsk_mlp_forward(mvsk_mlp* mlp, const float* X, int32_t B, float* Y);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) on the
 * mean-squared error (1/(B d_out)) sum (y - Yt)^2 of the batch (X, Yt);
 * *loss (host) receives the loss before the step.  The gradients of the step
 * stay readable through mvsk_mlp_read(..., what = 2). */
mvsk_status mvsk_mlp_train_step(mvsk_mlp* mlp, const float* X, const float* Yt, int32_t B, float lr, double* loss);

/* Parameters and gradients of layer `layer` (0-based, n_hidden + 1 layers):
 * what = 0 reads W (d_out_l x d_in_l) and b (d_out_l) into host-or-device
 * buffers, 1 writes them (master FP32 copy and its BF16 copies), 2 reads the
 * gradients of the last train step. */
mvsk_status mvsk_mlp_access(mvsk_mlp* mlp, int32_t layer, int32_t what, float* W, float* b);

/* Request features X (B x MVSK_MLP_D_IN, FP32) from the panel's column means
 * mu and scales sigma (n each, FP64; mvsk_column_stats) and the requests'
 * lambda (B x 4) and target (B; NaN = none): lambda as given; (target -
 * mean mu) / std mu and a flag; the projections of the standardised mu and
 * sigma (mean 0, norm 1) on 2 x 32 normal vectors, entry i of vector r being
 * the Box-Muller normal of SplitMix64 outputs 2i, 2i+1 of the stream seeded by
 * output r of the stream `seed` (the Hutchinson probe generator with
 * iteration 0); zeros after. */
mvsk_status mvsk_mlp_features(const double* mu, const double* sigma, int64_t n, int32_t B, const double* lambda,
                              const double* target, uint64_t seed, float* X);

/* Starts W0 (B x n, FP64) = Pi_Delta(tau)(y_b / n) of the network outputs for
 * features X (B x d_in); d_out must equal n. */
mvsk_status mvsk_mlp_warm_start(mvsk_mlp* mlp, const float* X, int32_t B, int64_t n, double tau, double* W0);

#ifdef __cplusplus
}
#endif

#endif /* MVSK_MLP_H */
