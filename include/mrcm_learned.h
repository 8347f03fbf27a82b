/*
 * mrcm_learned.h — C ABI of the learned interface preconditioner.
 *
 * The paper has no learned component and does not say how the interface
 * system (Section 3, Eq. "mrc2") is solved.  On the GMRES path of
 * mrcm_solve_interface (include/mrcm.h) every interface g gets an m x m
 * right-preconditioner block P_g.  Block-Jacobi uses P_g = (M_gg)^{-1}; the
 * learned preconditioner uses P_g = (M_gg)^{-1} (I + Delta_g), where Delta_g
 * is proposed by a small convolutional network from the permeability around
 * the interface.  Delta = 0 is block-Jacobi, and the GMRES falls back to
 * block-Jacobi when the residual stalls (less than 10% reduction over 10
 * steps).
 *
 * Network: input per interface 2 x (2s) x (3s) BF16 values in canonical
 * orientation (rows along the interface, columns across it, the
 * smaller-index subdomain on the left, the window centred on the
 * interface): channel 0 = log10(lambda K)/3 inside the domain, 0 outside;
 * channel 1 = 1 inside, 0 outside.  Three 3x3 convolutions with stride 2,
 * zero padding 1, 32 channels, bias and ReLU; a linear head from the
 * flattened last feature map (nf = 32 x s/4 x 3s/8 values, positions along
 * the interface kept) to m*m outputs (row-major Delta_g).  Activations are stored
 * in BF16 and weights rounded to BF16; all products accumulate in FP32.
 * Parameters are FP32 master weights in the order w1 [32][2][3][3], b1 [32],
 * w2 [32][32][3][3], b2, w3 [32][32][3][3], b3, wh [m*m][nf], bh [m*m]
 * (wh columns in the order channel, row, column of the feature map).
 * Training minimises the mean of w_k (Delta_k - target_k)^2 with Adam, with
 * per-entry weights w_k (default 1; see mrcm_lp_set_loss_weights).
 *
 * Training target of interface g (mrcm_lp_targets): theta (M_gg B_g - I)
 * with theta = 1/2, clipped entrywise to [-2, 2] (near-singular blocks of
 * high-contrast media would otherwise dominate the loss), where B_g is the
 * (g, g) block of the inverse of the
 * interface matrix restricted to g's neighbourhood: the interfaces whose
 * subdomains lie within one subdomain (Chebyshev distance) of g's two
 * subdomains.  Computed in FP64 by Gaussian elimination with partial
 * pivoting.
 *
 * Ownership and errors follow include/mrcm.h: d_* pointers are caller-owned
 * device memory; the network object owns its weights, Adam state and
 * activation buffers for up to max_batch samples (allocated in
 * mrcm_lp_create only); every call returns an mrcm_status.
 */
#ifndef MRCM_LEARNED_H
#define MRCM_LEARNED_H

#include <stdint.h>
#include "mrcm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrcm_lp mrcm_lp;   /* opaque network object */

/* Create a network for subdomain size s (16 or 32) and interface size m
 * (1..8) with buffers for batches of up to max_batch samples.  Convolution
 * weights are He-normal from a seeded generator, biases and the head are
 * zero (the initial network proposes Delta = 0).  Kernels run on
 * cuda_stream. */
mrcm_status mrcm_lp_create(int32_t s, int32_t m, int32_t max_batch, uint64_t seed,
                           void *cuda_stream, mrcm_lp **out);
void mrcm_lp_destroy(mrcm_lp *lp);
const char *mrcm_lp_last_error(const mrcm_lp *lp);
mrcm_status mrcm_lp_set_stream(mrcm_lp *lp, void *cuda_stream);

/* Number of FP32 parameters, and of BF16 input values per sample. */
int64_t mrcm_lp_num_params(const mrcm_lp *lp);
int64_t mrcm_lp_input_size(const mrcm_lp *lp);

/* Copy the FP32 parameters from / to device memory (layout above). */
mrcm_status mrcm_lp_set_params(mrcm_lp *lp, const float *d_params);
mrcm_status mrcm_lp_get_params(mrcm_lp *lp, float *d_params);

/* Per-entry loss weights w_k, k < m*m (device FP32). */
mrcm_status mrcm_lp_set_loss_weights(mrcm_lp *lp, const float *d_weights);

/* Delta for B samples: d_x BF16 [B][2][2s][3s], d_delta FP32 [B][m*m]. */
mrcm_status mrcm_lp_forward(mrcm_lp *lp, const void *d_x, int32_t B, float *d_delta);

/* Loss (FP32 scalar, may be NULL) and its gradient (FP32, num_params
 * values, may be NULL) for B samples with targets d_target [B][m*m]. */
mrcm_status mrcm_lp_gradient(mrcm_lp *lp, const void *d_x, const float *d_target, int32_t B,
                             float *d_grad, float *d_loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the batch; d_loss (may be NULL) receives the batch loss before the step. */
mrcm_status mrcm_lp_train_step(mrcm_lp *lp, const void *d_x, const float *d_target, int32_t B,
                               float lr, float *d_loss);

/* ---- with an MRCM context (GMRES path; every interface the same m, every
 * realisation the same s) ---------------------------------------------- */

/* Interfaces of the context (samples), realisations concatenated. */
int64_t mrcm_lp_num_samples(const mrcm_ctx *ctx);

/* Network inputs of interfaces first .. first+count-1 (canonical order)
 * from device K and lambda [n_real][ny][nx]: d_x BF16 [count][2][2s][3s]. */
mrcm_status mrcm_lp_windows(mrcm_ctx *ctx, const double *d_K, const double *d_lambda,
                            int64_t first, int32_t count, void *d_x);

/* Training targets of every interface after mrcm_build_basis: d_target
 * FP32 [num_samples][m*m].  Synchronises the stream; MRCM_ENOTSPD if a
 * neighbourhood matrix was singular. */
mrcm_status mrcm_lp_targets(mrcm_ctx *ctx, float *d_target);

/* After mrcm_build_basis, for a context set up with precond =
 * MRCM_PRECOND_USER: run the network on every interface and install
 * P_g = (M_gg)^{-1} (I + Delta_g) as the GMRES preconditioner (stream
 * ordered; no synchronisation). */
mrcm_status mrcm_lp_apply(mrcm_ctx *ctx, mrcm_lp *lp, const double *d_K,
                          const double *d_lambda);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_LEARNED_H */
