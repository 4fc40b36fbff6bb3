/*
 * sp_fno.h -- C ABI of the learned initial guess for the solve of sp.h.
 *
 * A Fourier-layer network (the Fourier neural operator of Li et al., ICLR 2021,
 * Section 4) maps the medium and the right-hand side of one problem to a starting
 * vector u0 for GMRES (sp_solve_x0 in sp.h).  The paper itself has no learned part:
 * the zero-guess preconditioned solve stays the fallback (a guess whose residual
 * exceeds that of zero is dropped) and the measure of the guess (the same explicit
 * true residual decides convergence).  Training data are (medium, source, solution)
 * triples that the solver of sp.h produces.
 *
 * Network (L Fourier layers of width W, M modes per axis, projection width H):
 *   v_0 = P a + p;  h_l = W_l v_l + b_l + K_l v_l;  v_{l+1} = gelu(h_l) (l < L-1),
 *   v_L = h_{L-1};  y = Q2 gelu(Q1 v_L + c1) + c2,
 * with K_l v = real inverse DFT of R_l(k) (DFT of v)(k) over the modes kx = 0..M-1
 * (axis 0) and ky in {0..M-1} U {n-M..n-1} (axis 1), R_l(k) a complex W x W matrix,
 * gelu(x) = x Phi(x).  Loss: mean over the batch of ||y_b - t_b||^2 / ||t_b||^2;
 * optimiser Adam (Kingma and Ba, ICLR 2015, Algorithm 1).
 *
 * Conventions.
 *  - Tensors are float32, batch-major, channel-major, grid flat index j0 + n*j1:
 *    x[b][c][j0 + n*j1].  *_dev pointers are device pointers, *_host host pointers;
 *    the caller owns every buffer it passes, the context its weights, optimiser
 *    state and activations.
 *  - Parameters: one flat float32 vector in this order (row-major; complex entries
 *    as (re, im) pairs): P [W][c_in], p [W]; for each layer R [2M][M][W][W][2]
 *    (first index: ky = 0..M-1, then n-M..n-1), W_l [W][W], b_l [W]; Q1 [H][W],
 *    c1 [H], Q2 [c_out][H], c2 [c_out].  The context keeps an FP32 master copy and
 *    the bfloat16 copy (round to nearest even) that every pass computes with;
 *    products accumulate in FP32.
 *  - Every call is ordered on the stream given to sp_fno_create; only calls that
 *    return a value to a host pointer synchronise it.
 *  - Errors come back as the sp_status codes of sp.h; nothing aborts across the ABI.
 */
#ifndef SP_FNO_GB300_H
#define SP_FNO_GB300_H

#include "sp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sp_fno sp_fno; /* opaque */

typedef struct {
  int n;         /* grid points per axis: a multiple of 64, at most 512 */
  int c_in;      /* input channels, 1..32 */
  int width;     /* W, channels of the Fourier layers, 1..32 */
  int modes;     /* M, kept modes per axis, 1..16, 2M <= n */
  int layers;    /* L, Fourier layers, 1..8 */
  int hidden;    /* H, projection width, 1..128 */
  int c_out;     /* output channels, 1..8 */
  int batch_max; /* largest batch of any call, >= 1 */
  int act_fp32;  /* 0: activations stored as bfloat16; 1: as float32 */
} sp_fno_dims;

typedef struct {
  double lr, beta1, beta2, eps;
} sp_adam;

/* Number of parameters of the network (0 for invalid dims). */
long long sp_fno_param_count(const sp_fno_dims *dims);

/* Allocates the context (weights, Adam moments set to zero, activations for
 * batch_max) and loads params_host (sp_fno_param_count floats).  stream: a
 * cudaStream_t or NULL.  SP_ERR_ARG for dims outside the ranges above,
 * SP_ERR_OOM when device memory runs out. */
sp_status sp_fno_create(const sp_fno_dims *dims, const float *params_host, void *stream,
                        sp_fno **out);
void sp_fno_destroy(sp_fno *f);

/* Replace the weights (FP32 master and bfloat16 copy) and reset Adam (moments and
 * step count).  Synchronous. */
sp_status sp_fno_set_params(sp_fno *f, const float *params_host);
/* Copy the FP32 master weights to the host.  Synchronous. */
sp_status sp_fno_get_params(sp_fno *f, float *params_host);

/* y = network(x) for batch <= batch_max samples: x_dev [batch][c_in][n*n],
 * y_dev [batch][c_out][n*n]. */
sp_status sp_fno_forward(sp_fno *f, int batch, const float *x_dev, float *y_dev);

/* Forward and backward pass without an update: the loss against targets t_dev
 * ([batch][c_out][n*n]) to *loss_host and the gradient (sp_fno_param_count floats)
 * to grad_host; either pointer may be NULL.  y_dev (may be NULL) receives the
 * output.  Synchronous. */
sp_status sp_fno_gradient(sp_fno *f, int batch, const float *x_dev, const float *t_dev,
                          float *y_dev, double *loss_host, float *grad_host);

/* One Adam step on the loss of (x_dev, t_dev).  loss_host may be NULL (then the call
 * does not synchronise); otherwise it receives the loss before the update. */
sp_status sp_fno_train_step(sp_fno *f, int batch, const float *x_dev, const float *t_dev,
                            const sp_adam *opt, double *loss_host);

/* Network input of one problem.  With g = G f (sp_green), the complex scale
 * c = sigma e^{i phi}, sigma = the root mean square of |g| and phi = arg(sum g^2) / 2
 * (0 when that sum vanishes), is written to scale_dev (one complex128), and
 * x[0] = q_scale q, x[1] + i x[2] = g / c (c_in must be 3) to x_dev ([3][N], N = n*n).
 * The solution is complex-linear in g, so the scale removes both the size and the
 * phase of the source (a source e^{i theta} r with r real gives the real field +-r).
 * q_dev: N doubles; g_dev: N complex128. */
sp_status sp_fno_features(sp_fno *f, const double *q_dev, double q_scale, const void *g_dev,
                          float *x_dev, void *scale_dev);
/* Starting vector of one problem from the network output y_dev ([2][N], c_out must
 * be 2): u0 = c (y[0] + i y[1]), complex128. */
sp_status sp_fno_guess(sp_fno *f, const float *y_dev, const void *scale_dev, void *u0_dev);
/* Training target of one problem from a solution u_dev (complex128):
 * t[0] + i t[1] = u / c. */
sp_status sp_fno_target(sp_fno *f, const void *u_dev, const void *scale_dev, float *t_dev);

/* The same three with a prior estimate z of the solution (the network then learns a
 * correction to it; not in the paper: z is the preconditioner applied to g, the
 * first approximation the method itself offers, z = P^{-1} Q g, sp_apply).  Features
 * (c_in must be 5): x[0..2] as sp_fno_features, x[3] + i x[4] = z / c.  Guess:
 * u0 = z + c (y[0] + i y[1]).  Target: t[0] + i t[1] = (u - z) / c.  z_dev: N complex128. */
sp_status sp_fno_features_prior(sp_fno *f, const double *q_dev, double q_scale, const void *g_dev,
                                const void *z_dev, float *x_dev, void *scale_dev);
sp_status sp_fno_guess_prior(sp_fno *f, const float *y_dev, const void *scale_dev, const void *z_dev,
                             void *u0_dev);
sp_status sp_fno_target_prior(sp_fno *f, const void *u_dev, const void *scale_dev, const void *z_dev,
                              float *t_dev);

#ifdef __cplusplus
}
#endif
#endif
