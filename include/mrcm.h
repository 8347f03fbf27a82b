/*
 * mrcm.h — C ABI of the GB300 Multiscale Robin Coupled Method (MRCM) Darcy
 * pressure–velocity solve.
 *
 * The solved problem is the Darcy system of Section 2 (Eq. "Darcy"):
 *     u = -lambda(s) K grad p,  div u = q  in Omega,
 *     p = p_b on the Dirichlet part, u.n = u_b on the Neumann part,
 * on a uniform grid of square cells, decomposed into s x s-cell subdomains.
 * MRCM (Section 3) solves local Robin problems (Eq. "mrc1") with
 * beta = alpha H / kappa (Eq. "beta"), builds a multiscale basis from them,
 * and couples the subdomains through the interface system (Eq. "mrc2"); the
 * solution is the linear combination of the basis (text after Eq. "beta").
 *
 * The five hot-path calls, in calling order:
 *   mrcm_setup            host: tables, workspace (the only allocation)
 *   mrcm_factor_local     (a) assemble + (b) factor every local operator
 *   mrcm_build_basis      (c) multi-RHS local solves, FP64 refinement
 *   mrcm_solve_interface  (d) interface assembly + solve
 *   mrcm_reconstruct      (e) fine pressure and face velocities
 *
 * Conventions shared by every call
 *   Grid: one realisation is nx x ny square cells of side h = ly/ny on
 *   [0, nx h] x [0, ly].  Cell arrays are [n_real][ny][nx] FP64, x fastest.
 *   Face velocities are NORMAL velocities (not integrated fluxes):
 *   ux is [n_real][ny][nx+1] (face i sits at x = i h, positive along +x),
 *   uy is [n_real][ny+1][nx] (face j sits at y = j h, positive along +y).
 *   Subdomains are numbered row-major S = J*Sx + I.  Interfaces of one
 *   realisation are in canonical order: vertical ones (between (I,J) and
 *   (I+1,J)) row-major by (J,I), then horizontal ones (between (I,J) and
 *   (I,J+1)) row-major by (J,I).  The fixed normal n_check points out of the
 *   smaller-index subdomain (Section 3, after Eq. "compatibility"): +x or +y.
 *   Interface unknowns are ordered [U_0..U_{nU-1}, P_0..P_{nP-1}]: flux
 *   coefficients then pressure coefficients.  Interface functions are
 *   polynomials of t in [-1,1] along the interface (+y for vertical, +x for
 *   horizontal interfaces), sampled at face midpoints.
 *   Boundary faces are listed left (ny), right (ny), bottom (nx), top (nx).
 *
 * Ownership: every d_* pointer is DEVICE memory owned by the caller, and the
 * CUDA stream is owned by the caller.  The library owns its workspace, which
 * is allocated in mrcm_setup only and freed by mrcm_destroy; calls 2–5
 * allocate nothing, synchronise nothing (unless an info pointer is passed)
 * and only enqueue kernels on the stream.
 *
 * Errors: every call returns an mrcm_status, never aborts.  Host-side
 * validation failures return MRCM_EINVAL; CUDA launch failures MRCM_ECUDA.
 * Numerical failures detected on the device (non-SPD pivot, NaN, stalled
 * refinement) are accumulated in a device status word and reported by
 * mrcm_get_info (or by mrcm_solve_interface when given an info pointer).
 * mrcm_last_error returns a message for the last failing call.
 */
#ifndef MRCM_H
#define MRCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MRCM_OK = 0,
  MRCM_EINVAL = 1,     /* bad descriptor, argument or calling order        */
  MRCM_ENOMEM = 2,     /* workspace allocation failed in mrcm_setup        */
  MRCM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed      */
  MRCM_ENOTSPD = 4,    /* a local pivot was <= 0 or not finite             */
  MRCM_EIRSTALL = 5,   /* refinement stopped above its tolerance           */
  MRCM_ENOCONV = 6,    /* interface refinement did not converge            */
  MRCM_ENAN = 7,       /* NaN / Inf in inputs or results                   */
  MRCM_ETIMEOUT = 8,   /* a bounded device wait ran out (result invalid)   */
  MRCM_EINCOMPAT = 9   /* pure Neumann: the sources do not balance the     */
                       /* prescribed boundary outflow (no solution)        */
} mrcm_status;

/* Device status flags (bit OR), see mrcm_info.flags. */
#define MRCM_FLAG_NOTSPD      0x1
#define MRCM_FLAG_LOCAL_STALL 0x2
#define MRCM_FLAG_IFACE_STALL 0x4
#define MRCM_FLAG_NAN         0x8
#define MRCM_FLAG_IFACE_PIVOT 0x10
#define MRCM_FLAG_LAYOUT      0x20  /* internal table inconsistency (a bug) */
#define MRCM_FLAG_TIMEOUT     0x80  /* a bounded device wait ran out         */
#define MRCM_FLAG_PRECOND_FALLBACK 0x40  /* informational: the caller-supplied   */
                                         /* preconditioner stalled and GMRES was */
                                         /* rerun with block-Jacobi              */
#define MRCM_FLAG_INCOMPATIBLE 0x200     /* pure Neumann: |sum q h^2 - sum u_b h| */
                                         /* above 1e-10 of the absolute sums      */
#define MRCM_FLAG_LOCAL_REFACTOR 0x100   /* informational: the FP32 refinement of */
                                         /* some subdomains stalled and they     */
                                         /* were re-factored and re-solved in    */
                                         /* FP64 (mrcm_info.local_refactored)    */

typedef enum {
  MRCM_PREC_FP64 = 0,     /* plain path: FP64 factors and solves            */
  MRCM_PREC_FP32_IR = 1   /* FP32 factors/solves, FP64 residual refinement  */
} mrcm_precision;

typedef enum {
  MRCM_BASIS_LEGENDRE = 0,  /* P_k(t), Legendre polynomials                 */
  MRCM_BASIS_MONOMIAL = 1   /* t^k (same spans; for invariance checks)      */
} mrcm_basis_family;

typedef enum {
  MRCM_IFACE_AUTO = 0,    /* direct when every slab has <= 64 unknowns, else GMRES */
  MRCM_IFACE_DIRECT = 1,  /* block cyclic reduction over slabs + refinement  */
  MRCM_IFACE_GMRES = 2    /* restarted FP64 GMRES, right-preconditioned      */
} mrcm_iface_solver;

typedef enum {
  MRCM_PRECOND_BLOCK_JACOBI = 0,  /* P_g = (M_gg)^-1 per interface g          */
  MRCM_PRECOND_USER = 1,          /* blocks from mrcm_set_precond_blocks (the  */
                                  /* learned preconditioner); block-Jacobi    */
                                  /* takes over if the residual stalls        */
  MRCM_PRECOND_NONE = 2,
  MRCM_PRECOND_NEIGHBOURHOOD = 3, /* restricted inverse of each interface's    */
                                  /* neighbourhood: P[N(g), g] = columns g of  */
                                  /* (M_N(g))^-1, FP64, built every solve; N(g) */
                                  /* = interfaces with a subdomain within one  */
                                  /* subdomain of g's two (up to 31; at most   */
                                  /* 160 unknowns)                             */
  MRCM_PRECOND_NEIGHBOURHOOD_SHARED = 4  /* the same with N(g) = interfaces    */
                                         /* sharing a subdomain with g (<= 7)  */
} mrcm_precond;

typedef struct mrcm_ctx mrcm_ctx;   /* opaque, owned by the library */

/* Problem descriptor.  All pointers are HOST pointers; their contents are
 * copied by mrcm_setup and not referenced afterwards. */
typedef struct {
  int32_t nx, ny;            /* cells per realisation                         */
  int32_t n_real;            /* independent realisations solved together      */
  double  ly;                /* domain height; h = ly / ny                    */
  const int32_t *sub_size;   /* [n_real] subdomain edge s in cells (16);      */
                             /* nx and ny must be multiples of s              */
  const int32_t *iface_nU;   /* flux-space size per interface, realisations   */
  const int32_t *iface_nP;   /* concatenated, canonical order; 0 <= n <= s,   */
                             /* nU + nP >= 1; pure Neumann needs nP >= 1      */
  const double  *alpha;      /* NULL: alpha = 1 everywhere; else per face:    */
                             /* realisations concatenated, per interface s    */
                             /* values along the interface; alpha > 0         */
  const int8_t  *bc_type;    /* [2ny+2nx]: 0 = u.n = bc_val (outward normal   */
  const double  *bc_val;     /* velocity), 1 = p = bc_val; shared by all      */
                             /* realisations                                  */
  int32_t pure_neumann;      /* 1: no Dirichlet face; pressure is returned    */
                             /* with zero cell mean per realisation           */
  int32_t basis_family;      /* mrcm_basis_family                             */
  int32_t prec;              /* mrcm_precision                                */
  double  ir_tol;            /* local refinement: stop when ||r||/||b|| <= tol */
  int32_t ir_max;            /* max local refinement sweeps (FP32_IR)         */
  double  iface_tol;         /* interface refinement tolerance (relative)     */
  int32_t iface_ir_max;      /* max interface refinement sweeps after the     */
                             /* first solve                                   */
  int32_t iface_solver;      /* a mrcm_iface_solver value, 0 = auto           */
  int32_t precond;           /* mrcm_precond, GMRES only (0 = block-Jacobi)   */
  int32_t gmres_restart;     /* Krylov steps before a restart, 1..64 (0: 40)  */
  int32_t gmres_max;         /* max GMRES steps in total (0: 5000)            */
  double  gmres_tol;         /* stop at ||f - M x|| <= tol ||f||, the TRUE    */
                             /* residual (0: iface_tol)                       */
  const double *iface_fn;    /* NULL: the functions of basis_family.  Else    */
                             /* per interface (realisations concatenated,     */
                             /* canonical order): nU flux then nP pressure    */
                             /* functions, s face-midpoint values each, along */
                             /* +y (vertical) or +x (horizontal interfaces);  */
                             /* e.g. the physics-based spaces of Section 3    */
  const int8_t *refine;      /* NULL: uniform subdomains.  Else, for every    */
                             /* realisation, (ny/s) x (nx/s) entries (s =     */
                             /* sub_size[r], row-major): a nonzero 32 x 32    */
                             /* block is split into four 16 x 16 subdomains   */
                             /* (a one-level quadtree, Section 3's            */
                             /* decomposition with two sizes).  Interfaces    */
                             /* are then the maximal runs of faces shared by  */
                             /* the same two subdomains (32 or 16 faces: half */
                             /* an edge next to a split block), vertical ones */
                             /* by (first row, x) then horizontal ones by     */
                             /* (y, first column), normal +x / +y, and        */
                             /* beta = alpha H / kappa takes H = the          */
                             /* interface's length.  Such a context solves    */
                             /* step (d) by GMRES (block-Jacobi, the shared   */
                             /* neighbourhood form, or none);                 */
                             /* pure-Neumann problems and gravity are refused */
  int32_t ir_recover;        /* MRCM_PREC_FP32_IR: a subdomain whose local    */
                             /* refinement stalls (relative residual above    */
                             /* 1e3 ir_tol) is re-factored in FP64 and its    */
                             /* columns solved again, inside the same         */
                             /* mrcm_build_basis; at most this many per       */
                             /* factorisation (0: 16; < 0: none).  More       */
                             /* stalls than that give MRCM_EIRSTALL           */
} mrcm_desc;

typedef struct {
  int32_t flags;             /* OR of MRCM_FLAG_*                              */
  int32_t local_sweeps_max;  /* most local refinement sweeps any RHS took      */
  int32_t iface_sweeps;      /* interface refinement sweeps (max over real.)   */
  int32_t gmres_iters;       /* GMRES steps (max over realisations, including  */
                             /* a block-Jacobi rerun); 0 on the direct path    */
  double  local_resid_max;   /* max ||b - A x|| / ||b|| over local solves      */
                             /* (the columns re-solved in FP64 excluded)      */
  double  iface_resid;       /* max over realisations ||f - M x|| / ||f||      */
  int32_t local_refactored;  /* subdomains re-factored in FP64 (ir_recover)    */
} mrcm_info;

/* Validate the descriptor, build subdomain / interface / slab tables, choose
 * the launch shapes and allocate all workspace on the current device.  The
 * stream (a cudaStream_t, NULL = legacy default stream) is used by every
 * later call.  On success *out owns the context; on failure *out is NULL
 * and the return value says why.  Section 3 ("mrc1", "mrc2").
 * With the environment variable MRCM_DEBUG_POISON=1 the floating-point part
 * of the workspace is filled with NaN bytes at allocation (a check that no
 * step reads a value that no earlier step wrote: results must not change). */
mrcm_status mrcm_setup(const mrcm_desc *desc, void *cuda_stream, mrcm_ctx **out);

/* Steps (a)+(b).  d_K, d_lambda: device [n_real][ny][nx] FP64, kappa =
 * lambda*K > 0.  Assembles every subdomain's 5-point Robin operator
 * (two-point fluxes: harmonic mean inside, T_R = kappa/(alpha H/h + 1/2) on
 * interface faces, 2 kappa on Dirichlet faces) and factors all of them in
 * one batched launch.  Re-callable with new lambda (re-factors).  With
 * MRCM_PREC_FP32_IR and at most two 16 x 16-cell subdomains per SM, their
 * FP32 factor is formed inside mrcm_build_basis (each basis CTA factors its
 * subdomain in shared memory); this call then assembles the operators and
 * their Jacobi scaling,
 * which is all that is read from d_K and d_lambda, so the inputs may change
 * once it returns (stream-ordered) as before.  Eq. "mrc1", Eq. "beta". */
mrcm_status mrcm_factor_local(mrcm_ctx *ctx, const double *d_K, const double *d_lambda);

/* Step (c).  d_q: device [n_real][ny][nx] FP64 source density.  Solves every
 * subdomain for one RHS per interface function on each of its interface
 * edges plus one RHS for sources and boundary data; FP32_IR refines each RHS
 * in FP64 until ||r||/||b|| <= ir_tol or ir_max sweeps.  Writes the basis and
 * its interface traces to workspace.  Text after Eq. "beta". */
mrcm_status mrcm_build_basis(mrcm_ctx *ctx, const double *d_q);

/* Gravity (Section 5.4, Eq. "Darcy_wg", the height along +y).  d_w: device
 * [n_real][ny][nx] FP64, the gravity velocity K lambda_g g of every cell, or
 * NULL for none (the default).  The pointer is kept, not copied: the buffer
 * must stay valid, and hold the values, through the mrcm_build_basis and
 * mrcm_reconstruct calls that use it; set it before capturing those calls
 * in a graph.  Its known fluxes enter the particular right-hand side and
 * traces (step c) and the face velocities (step e): on a face normal to y
 * (kappa_l w_r + kappa_r w_l)/(kappa_l + kappa_r), on a Dirichlet face
 * n_y w_c, on a Robin face n_y w_c T_R / (2 kappa_c).  EINVAL for a NULL
 * context. */
mrcm_status mrcm_set_gravity(mrcm_ctx *ctx, const double *d_w);

/* Step (d).  Solves the interface system (Eq. "mrc2"), whose rows are the
 * traces of the basis, for (U_H, P_H).  Direct path: assembles the slab
 * blocks, factors them by block cyclic reduction (FP64, or FP32 with FP64
 * refinement).  GMRES path: restarted FP64 GMRES on the unassembled rows,
 * right-preconditioned by one m x m block per interface, until the true
 * relative residual is <= gmres_tol or gmres_max steps.  info: NULL = fully
 * asynchronous; else the stream is synchronised and *info filled (and the
 * return value reflects device flags). */
mrcm_status mrcm_solve_interface(mrcm_ctx *ctx, mrcm_info *info);

/* Step (e).  Writes p [n_real][ny][nx], ux [n_real][ny][nx+1],
 * uy [n_real][ny+1][nx] (device FP64).  On interface faces ux/uy hold the
 * mean of the two one-sided normal velocities.  d_gamma_u (optional, may be
 * NULL) receives the one-sided outward normal velocities: for every
 * interface in canonical order (realisations concatenated) 2*s values, the
 * smaller-index side first.  Text after Eq. "beta". */
mrcm_status mrcm_reconstruct(mrcm_ctx *ctx, double *d_p, double *d_ux, double *d_uy,
                             double *d_gamma_u);

/* Synchronise the stream and read the device status (see mrcm_info). */
mrcm_status mrcm_get_info(mrcm_ctx *ctx, mrcm_info *info);

/* Replace the stream used by later calls. */
mrcm_status mrcm_set_stream(mrcm_ctx *ctx, void *cuda_stream);

/* Number of kernel launches the last factor/basis/interface/reconstruct
 * sequence enqueued (for launch accounting). */
int32_t mrcm_launch_count(const mrcm_ctx *ctx);

/* Total interface unknowns (sum over realisations) and the length of the
 * d_gamma_u array of mrcm_reconstruct. */
int64_t mrcm_num_interface_unknowns(const mrcm_ctx *ctx);
int64_t mrcm_num_gamma_values(const mrcm_ctx *ctx);

/* Copy the interface solution (U_H, P_H), realisations concatenated in
 * canonical order, to the device buffer d_x (FP64). */
mrcm_status mrcm_copy_interface_solution(mrcm_ctx *ctx, double *d_x);

/* Tile width of the basis kernels (step c): right-hand-side columns per CTA,
 * one of 4, 8, 12, 16 for 16 x 16-cell subdomains and 4, 8 for 32 x 32
 * (also 16 for 32 x 32 with MRCM_PREC_FP32_IR; MRCM_EINVAL otherwise).
 * Results do not depend on it; the time does.  Synchronises the stream; call
 * it before capturing the calls in a CUDA graph. */
mrcm_status mrcm_set_basis_width(mrcm_ctx *ctx, int32_t nc16, int32_t nc32);

/* Autotuner of the tile widths above: factors the problem once (as
 * mrcm_factor_local), times mrcm_build_basis with every candidate width on
 * the caller's inputs (device K, lambda, q as in the calls above; reps timed
 * runs after one warm-up, median, CUDA events on the context's stream),
 * keeps the fastest and writes it to chosen[0..1] (host, may be NULL).
 * Leaves the context factored (call mrcm_build_basis next).  Synchronises;
 * call it before graph capture. */
mrcm_status mrcm_autotune(mrcm_ctx *ctx, const double *d_K, const double *d_lambda,
                          const double *d_q, int32_t reps, int32_t *chosen);

/* 1 if step (d) runs the GMRES path, 0 for the direct path. */
int32_t mrcm_uses_gmres(const mrcm_ctx *ctx);

/* The kernels that run step (d) in this context, fixed at mrcm_setup (the
 * direct paths are chosen by slab size, the cluster path also by whether its
 * shared-memory plan fits; MRCM_NO_CLUSTER=1 in the environment at setup
 * turns the cluster path off).  -1 for a NULL context. */
typedef enum {
  MRCM_PATH_NONE = 0,        /* no interface unknowns (one subdomain)         */
  MRCM_PATH_CLUSTER = 1,     /* one cluster launch per batch: slab block      */
                             /* cyclic reduction and refinement in shared     */
                             /* memory (FP32 factor, slabs <= 64 unknowns)    */
  MRCM_PATH_SLAB = 2,        /* the same reduction over several launches in  */
                             /* global memory (FP64, or FP32 if the cluster   */
                             /* plan does not fit)                            */
  MRCM_PATH_WIDE_SLAB = 3,   /* slabs above 64 unknowns: batched Gauss-Jordan */
                             /* and tensor-core products                      */
  MRCM_PATH_GMRES = 4        /* restarted FP64 GMRES                          */
} mrcm_iface_path;
int32_t mrcm_interface_path(const mrcm_ctx *ctx);

/* Length of the preconditioner-block array: for every interface in
 * canonical order (realisations concatenated) an m x m row-major block,
 * m = nU + nP. */
int64_t mrcm_num_precond_values(const mrcm_ctx *ctx);

/* Preconditioner blocks for precond = MRCM_PRECOND_USER (the learned
 * preconditioner).  d_blocks: device FP64, mrcm_num_precond_values()
 * entries in the layout above; copied (stream-ordered) into the context, so
 * the caller may reuse the buffer after the stream reaches this point.  Each
 * block approximates the inverse of its interface's diagonal block; the
 * GMRES path applies P = blockdiag(blocks) on the right.  EINVAL if the
 * context does not use the GMRES path with precond = MRCM_PRECOND_USER. */
mrcm_status mrcm_set_precond_blocks(mrcm_ctx *ctx, const double *d_blocks);

void mrcm_destroy(mrcm_ctx *ctx);
const char *mrcm_last_error(const mrcm_ctx *ctx);
int32_t mrcm_version(void);

/* Local subdomain solve that allocates nothing.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, e.g. code running inside another runtime's memory pool, or a
 * process whose device footprint must stay fixed after start-up.
 *
 * Solves A x = rhs for nsub independent 16 x 16-cell subdomains (1 <= nsub
 * <= 64), where A is the local two-point operator of Eq. "mrc1": harmonic
 * transmissibilities between cells and, on the 4 x 16 boundary faces, the
 * given face transmissibilities (Robin T_R, 2 kappa for a prescribed
 * pressure, 0 for a prescribed flux).  FP32 block factorisation, FP64
 * refinement to ||D r|| <= 1e-13 ||D rhs|| (D = diag(A)^-1/2), at most 30
 * sweeps.  Device arrays, FP64: d_kappa [nsub][16][16] (x fastest), d_tface
 * [nsub][4][16] (W, E, S, N faces; along +y for W/E, +x for S/N), d_rhs and
 * d_x [nsub][256].  Asynchronous on cuda_stream; numerical failures are not
 * reported (check the output).
 *
 * Its only scratch is a fixed 1 MiB __device__ array in the library, held by
 * every GPU that loads the library until the process exits.  The first call
 * on a device looks up that array's device address, so make it before any
 * stream capture; a call in a new context (after cudaDeviceReset) looks it
 * up again.  Every call reuses the same array and overwrites what it
 * reads, so calls whose kernels overlap on the GPU (e.g. on two streams)
 * race: serialise them.  nsub outside 1..64, or a current device index
 * above 63, returns MRCM_EINVAL (message from mrcm_last_error(NULL)). */
mrcm_status mrcm_local_solve_noalloc(int32_t nsub, const double *d_kappa, const double *d_tface,
                                     const double *d_rhs, double *d_x, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MRCM_H */
