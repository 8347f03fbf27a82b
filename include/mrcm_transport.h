/*
 * mrcm_transport.h — C ABI of the implicit saturation transport and of the
 * sequential implicit (SI) and sequential fully implicit (SFI) time steps
 * that couple it with the MRCM Darcy solve of include/mrcm.h.
 *
 * Transport (Section 4).  The water saturation s obeys Eq. "BL2D",
 * ds/dt + div(f(s) u) = 0, with the fractional flow of quadratic relative
 * permeabilities (Section 5)
 *     f(s) = M s^2 / (M s^2 + (1 - s)^2),   M = mu_o / mu_w.
 * One step from s^n to s^{n+1} is implicit Euler with the velocity frozen
 * (Eq. "BL2D_Newton") and first-order upwind finite volumes
 * (Eqs. "fluxes_impli", "up_fluxes_impli"), on the same grid as the Darcy
 * solve (nx x ny square cells of side h = ly / ny):
 *     H_I(s) = s_I - s_I^n + (dt / h^2) sum_faces h u_out f(s_upwind) = 0
 * (Eq. "BL2D_Newton7").  The upwind side of a face is the cell itself when
 * the outward normal velocity u_out is positive, else the neighbour; an
 * inlet face on the domain boundary carries f(s_in).  Newton's method
 * (Eq. "BL2D_Newton8") starts at s^n and is guarded by the inflection-point
 * trust region of Section 4.1: each new value is clipped to [0, 1], then a
 * cell whose new value lies across the inflection point of f from its old
 * value (f''(new) f''(old) < 0) takes the average of the two.  The loop of
 * a realisation stops once the update norm sqrt(sum_I (s_I^{nu+1} -
 * s_I^nu)^2 h^2) is at most eta.
 *
 * Layout and conventions are those of include/mrcm.h: cell arrays
 * [n_real][ny][nx] FP64 (x fastest); normal face velocities ux
 * [n_real][ny][nx+1] and uy [n_real][ny+1][nx], positive along +x / +y
 * (the arrays mrcm_reconstruct writes).  All d_* pointers are device
 * memory owned by the caller; the transport context owns its workspace,
 * allocated by mrcm_transport_create only.  Calls enqueue work on the
 * context's stream and return; mrcm_transport_get_info synchronises.
 *
 * Errors: every call returns an mrcm_status; the message of the last
 * failing transport call is mrcm_transport_last_error().  Device-side
 * outcomes (Newton or a linear solve hitting its limit, non-finite values)
 * are reported by mrcm_transport_get_info.
 */
#ifndef MRCM_TRANSPORT_H
#define MRCM_TRANSPORT_H

#include <stdint.h>

#include "mrcm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrcm_transport mrcm_transport;   /* opaque, owned by the library */

typedef struct {
  int32_t nx, ny, n_real;  /* grid of every realisation, number of them       */
  double  ly;              /* domain height; h = ly / ny                       */
  double  M;               /* viscosity ratio mu_o / mu_w (> 0)                */
  double  mu_w;            /* water viscosity (> 0); the output mobility is    */
                           /* lambda = s^2 / mu_w + (1 - s)^2 / (M mu_w)       */
                           /* (Eq. "fluxos1")                                  */
  double  s_in;            /* saturation of the water entering at inlet faces  */
  double  eta;             /* Newton stop on the update norm (0: 1e-6, the     */
                           /* paper's tolerance)                               */
  int32_t max_newton;      /* Newton iterations per step (0: 100)              */
  int32_t max_linear;      /* outer iterations per linear solve (0: 4 (tiles   */
                           /* across + tiles along) + 64)                      */
  int32_t plain_newton;    /* 1: no trust region (clip only), for comparison  */
} mrcm_transport_desc;

typedef struct {
  int32_t newton_iters_max;  /* largest Newton count over the realisations    */
  int32_t linear_iters_max;  /* largest outer count of one linear solve       */
  double  update_norm_max;   /* largest final update norm                     */
  double  change_max;        /* max |s_new - s_ref| (0 without d_s_ref)       */
  int32_t flags;             /* 1: Newton limit, 2: linear limit, 4: NaN      */
} mrcm_transport_info;

/* Context for n_real grids of nx x ny cells; allocates the workspace.
 * EINVAL for a bad descriptor, ENOMEM if the workspace does not fit. */
mrcm_status mrcm_transport_create(const mrcm_transport_desc *desc, void *cuda_stream,
                                  mrcm_transport **out);

/* One implicit transport step of every realisation (Section 4): from
 * d_s_old with the frozen face velocities d_ux, d_uy to d_s_new (must not
 * alias d_s_old).  d_lambda (or NULL): receives the total mobility of
 * d_s_new, the input of the next mrcm_factor_local.  d_s_ref (or NULL):
 * reports max |s_new - s_ref| through mrcm_transport_get_info (the SFI
 * outer test).  dt >= 0.  Enqueues one copy and one cooperative kernel. */
mrcm_status mrcm_transport_step(mrcm_transport *t, double dt, const double *d_ux,
                                const double *d_uy, const double *d_s_old, double *d_s_new,
                                double *d_lambda, const double *d_s_ref);

/* Synchronises the stream and reads the last step's outcome; newton_iters
 * (or NULL) receives the Newton count of every realisation.  Returns
 * MRCM_ENOCONV if a realisation or a linear solve hit its limit, MRCM_ENAN
 * for non-finite values. */
mrcm_status mrcm_transport_get_info(mrcm_transport *t, mrcm_transport_info *info,
                                    int32_t *newton_iters);

mrcm_status mrcm_transport_set_stream(mrcm_transport *t, void *cuda_stream);
void        mrcm_transport_destroy(mrcm_transport *t);
const char *mrcm_transport_last_error(void);

/* Sequential implicit step (Section 4): the Darcy solve of ctx (the five
 * calls of include/mrcm.h) with the mobility d_lambda, then the transport
 * step from d_s_old with the velocities it produced.  On return (enqueued)
 * d_p, d_ux, d_uy hold the Darcy solution, d_s_new the new saturation and
 * d_lambda its mobility, ready for the next step. */
mrcm_status mrcm_si_step(mrcm_ctx *ctx, mrcm_transport *t, double dt, const double *d_K,
                         double *d_lambda, const double *d_q, const double *d_s_old,
                         double *d_s_new, double *d_p, double *d_ux, double *d_uy);

/* Sequential fully implicit step (Section 5.4): repeats the Darcy solve
 * with the mobility of the latest saturation iterate and the transport step
 * from d_s_old with its velocities, until the largest change of the
 * saturation between two outer iterations is below tol (the paper uses
 * 1e-4) or max_outer iterations.  d_lambda must hold the mobility of
 * d_s_old on entry; d_s_work is caller scratch of one cell array.  Each
 * outer iteration reads the change back to the host (synchronises).
 * outer_iters (or NULL) receives the outer count; MRCM_ENOCONV if
 * max_outer was reached. */
mrcm_status mrcm_sfi_step(mrcm_ctx *ctx, mrcm_transport *t, double dt, double tol,
                          int32_t max_outer, const double *d_K, double *d_lambda,
                          const double *d_q, const double *d_s_old, double *d_s_new,
                          double *d_s_work, double *d_p, double *d_ux, double *d_uy,
                          int32_t *outer_iters);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_TRANSPORT_H */
