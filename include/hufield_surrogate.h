/*
 * hufield_surrogate.h -- C ABI of the surrogate network of the generator
 * (sm_103a).  The paper (Zhong & Mao, arXiv 2509.08675) closes (Sec. IV) by
 * naming optimisation loops over the generator's parameters as future work;
 * the plain generator cannot predict the spectrum of a thresholded map
 * without making the field.  This network learns that map, from the eight
 * parameters (p, two semi-axis ratios, rotation, k0, width, suppression
 * exponent s, threshold level t) to the log of the 128 radial S(k) bins of
 * the +-1 map on a 256^2 lattice, from fields the plain generator makes; its
 * input gradient drives inverse design, and every design is re-checked by the
 * plain generator (include/hufield.h).
 *
 * Network (fixed): 8 -> 256 -> 256 -> 256 -> 128, GELU (x Phi(x)) on the
 * hidden layers, linear output.  Mixed precision: the weights, each layer's
 * input activations and the back-propagated dz are BF16; every product sums
 * in FP32; biases, the master weights, Adam's moments and the gradients are
 * FP32.  Precisely (the FP64 reference rounds at the same points):
 *   forward   X0 = bf16(x) (zero-padded to 32 columns), Z_l = X_{l-1} bf16(W_l)^T + b_l,
 *             X_l = bf16(GELU(Z_l)) (l = 1..3), y = X_3 bf16(W_4)^T + b_4
 *   backward  dZ_4 = bf16(dy), dW_l = dZ_l^T X_{l-1}, db_l = sum_rows dZ_l,
 *             dZ_{l-1} = bf16((dZ_l bf16(W_l)) GELU'(Z_{l-1})), dx = dZ_1 bf16(W_1)
 *
 * Parameters: one flat FP32 vector of hufield_mlp_param_count() entries, per
 * layer W_l (row-major [n_out][n_in], the first layer's n_in padded from 8 to
 * 32 with zero columns) then b_l.  wq is a BF16 copy of the same vector
 * (hufield_mlp_cast, or refreshed by hufield_mlp_adam); the GEMMs read the
 * weights there and the biases from params.
 *
 * Conventions: every pointer except those named host_* is a DEVICE pointer
 * owned by the caller, 16-byte aligned (params, wq, grad, m, v: 256-byte
 * aligned).  Calls are asynchronous on `stream` (a cudaStream_t as void*)
 * and return HUFIELD_OK or an error code of include/hufield.h before
 * enqueueing anything on bad arguments.  Nothing here allocates.
 */
#ifndef HUFIELD_SURROGATE_H
#define HUFIELD_SURROGATE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HUFIELD_MLP_IN 8     /* parameters per row */
#define HUFIELD_MLP_OUT 128  /* radial bins per row */

/* Entries of the flat parameter vector (172,928). */
int64_t hufield_mlp_param_count(void);

/* Workspace of hufield_mlp_forward / _backward for `rows` rows (the rows are
 * padded to a multiple of 64): the stored activations a backward call needs.
 * 0 for rows < 1. */
size_t hufield_mlp_workspace_bytes(int64_t rows);

/* Initial parameters: W uniform on [-1/sqrt(fan_in), 1/sqrt(fan_in)] (fan_in
 * the layer's true input width; padding columns 0), b = 0.  Entry i takes
 * word i & 3 of Philox4x32-10 block i >> 2 with counter (j lo, j hi,
 * 0x4D4C5031, 0) and key = seed: u = (x + 1/2) 2^-32, w = (2u - 1) bound. */
int hufield_mlp_init(float *params, uint64_t seed, void *stream);

/* wq = bf16(params), round to nearest even, entry by entry. */
int hufield_mlp_cast(const float *params, uint16_t *wq, void *stream);

/* Encoding of raw parameters theta [rows][8] onto [-1, 1] (x [rows][8]):
 * (p - 4.5)/3.5, log2 r1, log2 r2, 2 rot/pi - 1, (k0 - 0.225)/0.175,
 * (width - 0.055)/0.045, (s - 4)/2, t.  decode is its inverse. */
int hufield_mlp_encode(const float *theta, int64_t rows, float *x, void *stream);
int hufield_mlp_decode(const float *x, int64_t rows, float *theta, void *stream);

/* y [rows][128] = network(x [rows][8]).  Stores the activations backward
 * needs in ws (ws_bytes >= hufield_mlp_workspace_bytes(rows)). */
int hufield_mlp_forward(const float *params, const uint16_t *wq, const float *x, int64_t rows, float *y, void *ws,
                        size_t ws_bytes, void *stream);

/* Back-propagates dy [rows][128] (the loss gradient with respect to y)
 * through the forward call that last used ws with the same rows: grad (flat,
 * param-shaped, overwritten; NULL skips the parameter gradients) and dx
 * [rows][8] (overwritten; NULL skips it). */
int hufield_mlp_backward(const float *params, const uint16_t *wq, const float *dy, int64_t rows, float *grad,
                         float *dx, void *ws, size_t ws_bytes, void *stream);

/* Training loss: with y = mu + sigma y_hat per bin (the log of the predicted
 * mean spectrum; the label standardisation of hufield_mlp_label_stats),
 * loss_sum (one device double, accumulated) += sum over rows and bins of
 * y + S e^{-y}, and dy = sigma (1 - S e^{-y}) / (rows 128): the exponential
 * negative log-likelihood, minimised by y = log E[S], so single-field labels
 * teach the log of the mean spectrum.  y is clamped to [-30, 30] in the
 * exponential. */
int hufield_mlp_deviance(const float *y_hat, const float *S, const float *mu, const float *sigma, int64_t rows,
                         float *dy, double *loss_sum, void *stream);

/* The predicted mean spectrum S [rows][128] = e^{mu + sigma y_hat} (the
 * exponent clamped to [-30, 30]). */
int hufield_mlp_spectrum(const float *y_hat, const float *mu, const float *sigma, int64_t rows, float *S,
                         void *stream);

/* Label standardisation over n rows of S [n][128]: mu_b and sigma_b are the
 * mean and standard deviation of log(S_b + 1e-3) (sigma at least 0.05). */
int hufield_mlp_label_stats(const float *S, int64_t n, float *mu, float *sigma, void *stream);

/* Bin means of n ragged-batch items with 128 radial bins each, as FP32
 * labels: S[i][b] = sums[i 128 + b] / counts[i 128 + b] (0 when empty). */
int hufield_mlp_labels(const double *sums, const int64_t *counts, int64_t n, float *S, void *stream);

/* One Adam step (Kingma & Ba, ICLR 2015; step counts from 1) over n entries
 * with bias correction and decoupled weight decay wd:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= lr (m/(1-b1^step) / (sqrt(v/(1-b2^step)) + eps) + wd p); wq = bf16(p)
 * (wq may be NULL). */
int hufield_mlp_adam(float *params, float *m, float *v, const float *grad, uint16_t *wq, int64_t n, int32_t step,
                     float lr, float beta1, float beta2, float eps, float wd, void *stream);

/* Minibatch by sampling with replacement: row r of the batch copies row
 * idx_r of x_all [n][8] and S_all [n][128], idx_r = (word 0 of Philox4x32-10
 * with counter (r, step lo, step hi, 0x4D4C5032) and key = seed) mod n. */
int hufield_mlp_gather(const float *x_all, const float *S_all, int64_t n, int64_t rows, uint64_t seed, int64_t step,
                       float *x_out, float *S_out, void *stream);

/* One whole training step, enqueued with no host-side per-step arguments so
 * that a CUDA graph of many steps can be replayed: the step counter s lives
 * in the training workspace (hufield_mlp_train_reset sets it).  The step
 * gathers `rows` rows as hufield_mlp_gather with step s and sched->seed,
 * runs forward, the deviance (adding to *loss_sum), backward into grad, and
 * Adam at t = s + 1 with the learning rate
 * lr (f + (1 - f) (1 + cos(pi s / total_steps)) / 2), f = lr_min_frac, and
 * decoupled decay wd; then s += 1.  m, v, grad: param-shaped FP32. */
typedef struct {
    float lr, lr_min_frac, beta1, beta2, eps, wd;
    int64_t total_steps;
    uint64_t seed;
} hufield_mlp_sched;

/* Bytes of the training workspace for `rows` rows per step (0 for rows < 1). */
size_t hufield_mlp_train_workspace_bytes(int64_t rows);
int hufield_mlp_train_reset(void *tws, int64_t step, void *stream);
int hufield_mlp_train_step(float *params, uint16_t *wq, float *m, float *v, float *grad, const float *x_all,
                           const float *S_all, int64_t n, int64_t rows, const float *mu, const float *sigma,
                           const hufield_mlp_sched *sched, double *loss_sum, void *tws, size_t tws_bytes,
                           void *stream);

/* Inverse-design loss per row against a target spectrum T [rows][128]
 * (bin means, all > 0): with y = mu + sigma y_hat,
 * loss_row = sum_{b>=1} (e^{y_b} - T_b)^2 / sum_{b>=1} T_b^2
 *          + lam sum_{b>=1} (y_b - log T_b)^2 / 127,
 * the squared relative L2 error of the predicted spectrum (bin 0, the map's
 * squared mean, is left out) plus a small log-space term; dy its gradient
 * with respect to y_hat (bin 0: 0).  loss_rows may be NULL. */
int hufield_mlp_design_loss(const float *y_hat, const float *T, const float *mu, const float *sigma, int64_t rows,
                            float lam, float *dy, float *loss_rows, void *stream);

/* One Adam step on design inputs x [rows][8] (moments m, v [rows][8]) with
 * gradient dx, then x clamped to [-1, 1]; columns whose bit is set in
 * frozen_mask are left unchanged. */
int hufield_mlp_design_step(float *x, float *m, float *v, const float *dx, int64_t rows, uint32_t frozen_mask,
                            int32_t step, float lr, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HUFIELD_SURROGATE_H */
