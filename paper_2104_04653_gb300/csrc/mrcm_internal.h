// Internal tables and launch entry points shared by the host orchestrator
// (mrcm_abi.cu) and the kernels (local.cu, iface.cu, recon.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mrcm {

constexpr int kMaxRealisations = 1 << 16;
constexpr int kEdgeW = 0, kEdgeE = 1, kEdgeS = 2, kEdgeN = 3;

// One subdomain (all realisations concatenated).
struct SubInfo {
  int r;             // realisation
  int I, J;          // subdomain coordinates
  int x0, y0;        // first cell (global x, y within the realisation)
  int ncols;         // 1 (sources/BC) + sum over interface edges of nU+nP
  int nrows;         // sum over interface edges of nU+nP (rows of G)
  int edge_iface[4]; // W,E,S,N: global interface id, -1 on the physical boundary
  int edge_col[4];   // first basis column of the edge's functions
  int edge_row[4];   // first row of the edge in G
  // quadtree layouts: an edge next to two half-size subdomains carries two
  // interfaces, the first on faces [0, s/2) (edge_iface, edge_col, edge_row)
  // and this second one on [s/2, s); -1 when the edge has one interface
  int edge_iface2[4];
  int edge_col2[4];
  int edge_row2[4];
  int col_off;       // offset into the column table (ncols entries)
  int s;             // subdomain edge in cells (16 or 32)
  int64_t basis_off; // offset (doubles) of basis [ncols][S*S]
  int64_t g_off;     // offset (doubles) of G [nrows][ncols]
  int64_t coef_off;  // offset (doubles) of the coefficient block (6 S*S + 4 S)
  int64_t w_off;     // offset (elements) of the inverse Schur blocks [S][S][S]
};

// One interface (all realisations concatenated, canonical order).
struct IfaceInfo {
  int r;
  int kind;          // 0 vertical (normal +x), 1 horizontal (normal +y)
  int L, R;          // global subdomain ids, L < R
  int nU, nP;
  int s;             // faces along the interface
  int unk;           // global unknown offset of U_0
  int slab, pos;     // BCR slab index (within realisation), row offset in slab
  int64_t alpha_off; // offset into the per-face alpha array (s values)
  int64_t gam_off;   // offset into the one-sided velocity output (2*s values)
  int64_t tsc_off;   // offset into the congruence scaling blocks (m*m values)
  int fnU, fnP;      // rows of phi_0 and psi_0 in the function table of size s
  int fx, fy;        // its first face: vertical (x line, first row), horizontal
                     // (first column, y line)
  int rowL, rowR;    // first row of its unknowns in the G rows of L and R
  int colL, colR;    // first basis column of its functions in L and R
};

// The interface of face e (0 .. s-1, along +y on W/E, +x on S/N) of edge
// `side` of a subdomain: its id (-1 on the physical boundary), the face's
// index along the interface and the interface's length in faces.
struct FaceIface {
  int g, e, len;
};

// Column c of a subdomain: global unknown it multiplies (-1: particular),
// the edge (0..3) whose Robin data it carries, and the function index.
struct ColInfo {
  int unk;           // global unknown, -1 for the particular column
  int edge;          // 0..3, -1 for the particular column
  int fn;            // function index k
  int is_u;          // 1: flux function phi_k, 0: pressure function psi_k
};

struct RealInfo {
  int s, Sx, Sy;
  int sub0, nsub;
  int iface0, niface;
  int unk0, nunk;
  int pin;           // pinned global unknown (pure Neumann) or -1
  int quad;          // 1: quadtree layout (mrcm_desc.refine), GMRES path only
  int nslab, bmax;   // BCR slabs and padded slab size
  int nlev;          // BCR reduction levels
  int64_t slab_off;  // offset (elements) of this realisation's slab blocks
  int64_t xy_off;    // offset (elements) of this realisation's X/Y blocks
  int64_t vec_off;   // offset (elements) of slab-padded vectors
  double h, H;
};

// One (own interface, neighbour interface) block of a slab's rows, for the
// cluster interface path.  goff indexes pair_goff (m*mn*2 G offsets).
struct PairPlan {
  int p0, m, nU, tsc;      // own interface: first slab position, size, flux size, T offset
  int pn0, mn, tscn, ds;   // neighbour: first position in its slab, size, T offset, slab - own
  int goff;
  int nUn;                 // neighbour's flux size (its T is block lower triangular at nUn)
};

// GMRES interface path (iface_gmres.cu)
constexpr int kGmThreads = 256;
constexpr int kGmKmax = 64;   // largest restart length
constexpr int kGmMmax = 32;   // largest interface size nU + nP

struct GmRow {       // one interface unknown = one row of the interface system
  int64_t gL, gR;    // G offsets of the row's basis-column-1 entry, L and R side
  int cL, cR;        // column-table offsets of basis column 1 on each side
  int nL, nR;        // basis columns on each side (ncols - 1)
};

struct GmBlock {     // one CTA of the GMRES kernel
  int r;             // realisation
  int row0, row1;    // global unknowns [row0, row1) owned by the CTA
  int blk0, nblk;    // the realisation's CTAs
};

struct GmArgs {
  const GmRow *row;
  const GmBlock *blk;
  const double *P;   // preconditioner blocks (m x m per interface, at tsc_off)
  double *Gp;        // G P, same layout as G
  double *V;         // Krylov slots: per realisation (K + 1) x nunk
  double *Wv, *Y;    // work vector and iterate of the preconditioned system
  double *part;      // [CTAs][K + 2] partial sums
  double *resid;     // [n_real] final relative residual
  int *done;         // [n_real]
  int *fallback;     // [n_real] 1: rerun with block-Jacobi
  int *iters;        // [n_real] GMRES steps, accumulated over launches
  int K, maxit;
  int stall;         // 1: stop on a stalled residual and request the rerun
  int gate;          // 1: run only the realisations whose fallback flag is set
  double tol;
  // neighbourhood preconditioner (nb = 1): P has, for every interface g, the
  // column block P[N(g), g] ([n_g][m_g], rows in neighbourhood order) at
  // p_off[g]; G P is stored wide: row i of interface g holds m_g' values for
  // each column block g' of pb(g) (pb_list[pb_off[g] ..], pb_pos = position
  // of the block in the row, gw_w[g] = row length), at gw_off[g] + i gw_w[g];
  // gat lists, for every interface h, the blocks g' with h in N(g') and the
  // P offset of h's first row in them
  int nb;
  double *Pnb;
  const int64_t *p_off;
  double *Gw;
  const int64_t *gw_off;
  const int *gw_w, *pb_off, *pb_list, *pb_pos;
  const int *gat_off, *gat_g;
  const int64_t *gat_o;
};

// learned interface preconditioner (learned.cu)
constexpr int kLpChannels = 32;   // channels of every convolution
constexpr int kLpMaxM = 8;        // largest interface size it serves
constexpr int kLpMaxNb = 64;      // largest neighbourhood (interfaces) of a target
constexpr int kLpMaxLoc = 160;    // largest neighbourhood (unknowns) of a target
constexpr double kLpClip = 2.0;   // entrywise bound of a target

constexpr int kNC16 = 12;     // default basis columns per CTA, s = 16 (4, 8, 12, 16)
constexpr int kNC32 = 8;      // default basis columns per CTA, s = 32 (4, 8; 16 in FP32)

// Direct interface path for slabs above 64 unknowns (iface_big.cu)
constexpr int kBigMaxLev = 20;

struct InvJob {      // in-place inverse of one n x n block
  void *a;           // the block (row-major)
  void *dinv;        // 64 x 64 scratch
  void *cpan;        // n x 64 scratch
  int n, pad;
};

struct GemmJob {     // C = alpha (A1 B1 + A2 B2) (+ C if acc), n x n row-major
  const void *a1, *b1, *a2, *b2;   // a2/b2 may be null
  void *c;
  int n, acc;
  double alpha;
};

struct BigPlan {
  int K, nlev, bmax;             // slabs, levels, largest slab
  int tensor_cores;              // FP32 products on tcgen05 (3 x TF32)
  const void *tc_maps;           // device tensor maps of the raw operands, 4 per GEMM job
  const int *lev_off;            // device [nlev + 1]: first multiplier slot of each level
  void *vec2;                    // second slab-ordered vector
  const InvJob *inv;             // device jobs, level by level, the root last
  const GemmJob *gemm;           // device jobs, two sets per level
  int inv_off[kBigMaxLev + 2];   // host: job ranges per level (nlev + 1 ranges)
  int gemm_off[2 * kBigMaxLev + 1];
};

struct BasisItem {   // one CTA of the basis kernel
  int sub;
  int c0, nc;        // column range
};

// Everything the kernels read, as device pointers (one struct by value).
struct DeviceTables {
  int nx, ny, n_real, nsub, niface, nunk;
  int pure_neumann;
  int smax;          // largest subdomain edge
  double h, inv_h;   // cell size (shared by all realisations)
  const SubInfo *sub;
  const int *sub_by_size;   // subdomain ids: the s = 16 ones first, then s = 32
  int nsub16;               // how many of them have s = 16
  int fuse16;               // FP32: factor the s = 16 subdomains inside the basis kernel
  const IfaceInfo *iface;
  const ColInfo *col;
  const RealInfo *real;
  const int *unk_iface;     // global unknown -> interface id
  const int *unk_slabpos;   // global unknown -> slab*bmax + pos (within realisation)
  const int *pos2unk;       // slab-padded position -> global unknown or -1
  int mmax;                 // largest nU + nP over all interfaces
  // cluster interface path: per slab position (realisations concatenated)
  const int *plan_info;     // p0 << 16 | m << 8 | i, bit 30 P row, bit 29 pinned; -1 padding
  const int *plan_cnt;      // terms of the position's row
  const int *plan_goff;     // [npos][emax] G offset of each term (-1: none)
  const short *plan_xi;     // [npos][emax] position of the term's unknown in slabs k-1..k+1
  const int *plan_fgoff;    // [npos][2] G offsets of the row's source/BC entries
  const int *plan_tsc;      // [npos] offset of the position's interface scaling block
  const PairPlan *pairs;    // per slab, realisations concatenated
  const int *pair_off;      // [n_real * nslab + 1]
  const int *pair_goff;     // G offsets of every pair entry (2 per entry, -1: none)
  int emax;                 // largest number of terms of one interface row
  const double *grav;       // caller's gravity velocity K lambda_g g [R][ny][nx], or null
  const double *fnval;      // function rows of s values: size 16 first, size 32 at fn_off32
  int64_t fn_off32;
                            // interface function k at face midpoint e
  const double *alpha;      // per face
  const int8_t *bc_type;
  const double *bc_val;
};

#ifdef __CUDACC__
// Face e of edge `side` of subdomain sb -> its interface (see FaceIface).
__device__ __forceinline__ FaceIface face_iface(const SubInfo &sb, int side, int e) {
  const int g2 = sb.edge_iface2[side];
  if (g2 < 0) return FaceIface{sb.edge_iface[side], e, sb.s};
  const int hf = sb.s >> 1;
  return e < hf ? FaceIface{sb.edge_iface[side], e, hf} : FaceIface{g2, e - hf, hf};
}

// Value of function row `row` of an interface of `len` faces at face e.
__device__ __forceinline__ double iface_fn_at(const DeviceTables &t, int len, int row, int e) {
  return t.fnval[(len == 16 ? 0 : t.fn_off32) + static_cast<int64_t>(row) * len + e];
}
#endif

// Workspace (device pointers), owned by the context.
struct Workspace {
  double *coef;       // [nsub][6*S*S + 4*S]: tW, tE, tS, tN, d (=1/sqrt(diag)), kappa,
                      // then beta on the four interface edges
  void *W;            // [nsub][S][S][S] inverse Schur blocks, prec-typed
  double *basis;      // basis columns (FP64)
  double *G;          // local interface contributions (FP64)
  void *slabB, *slabA, *slabC;  // [per real][nslab][bmax*bmax], prec-typed
  void *slabI;        // inverses of the eliminated pivot blocks, same layout
  void *X, *Y;        // BCR forward multipliers, prec-typed
  double *tsc;        // per interface m x m congruence scaling T_g (FP64)
  double *f;          // [nunk] interface RHS
  double *x;          // [nunk] interface solution
  double *r;          // [niface] per-interface squared residual norms
  void *vec;          // [per real][nslab*bmax] BCR right-hand side / solution, prec-typed
  double *psum;       // [nsub] per-subdomain pressure sums
  double *gamma_tmp;  // one-sided velocities scratch (if user passes none)
  int *status;        // [8] flags, local sweeps max, iface sweeps, GMRES steps,
                      // stalled subdomains listed for recovery, spare
  double *dstat;      // [2 + n_real] local resid max, iface resid, per real
  double *ifnorm;     // [n_real] ||f|| per realisation
  int *done;          // [n_real + 1] convergence flags
  // refinement-stall recovery (mixed path): a subdomain whose FP32 refinement
  // stalls is listed by the basis kernel, then re-factored in FP64 and its
  // columns solved again by the same call (rec_cap = 0: no recovery)
  int *stall_mark;     // [nsub] 1 once listed; cleared by the factor kernels
  int *stall_list;     // [rec_cap] the listed subdomains (count: status[4])
  double *W64;         // [rec_cap][rec_smax^3] their FP64 inverse Schur blocks
  SubInfo *rec_sub;    // [rec_cap] their SubInfo, w_off pointing into W64
  BasisItem *rec_items;  // [2][rec_cap * rec_maxch]: s = 16, then s = 32 items
  int rec_cap, rec_maxch, rec_smax;
};

// Launch wrappers (return cudaGetLastError()).
cudaError_t launch_factor(const DeviceTables &t, const Workspace &w, int prec,
                          const double *K, const double *lam, cudaStream_t st);
// items: the s = 16 subdomains' CTAs first (nitems16), then the s = 32 ones
cudaError_t launch_basis(const DeviceTables &t, const Workspace &w, int prec,
                         const BasisItem *items, int nitems16, int nitems32, int nc16, int nc32,
                         const double *q, double ir_tol, int ir_max, cudaStream_t st);
// FP64 re-factor and re-solve of the subdomains the mixed basis kernels
// listed (three launches; slots past the listed count return at once)
cudaError_t launch_recover(const DeviceTables &t, const Workspace &w, const double *q,
                           double ir_tol, cudaStream_t st);
constexpr int kRecNC = 8;     // basis columns per CTA of the recovery solves
// pure-Neumann problems: the compatibility check of the sources against the
// boundary outflow (one launch, sets MRCM_FLAG_INCOMPATIBLE)
cudaError_t launch_compat(const DeviceTables &t, const Workspace &w, const double *q,
                          cudaStream_t st);
// test hook: round n stored FP32 values (one subdomain's inverse Schur
// blocks) to `bits` explicit mantissa bits, ties to even
cudaError_t launch_degrade_factor(float *W, int n, int bits, cudaStream_t st);
cudaError_t launch_iface_assemble(const DeviceTables &t, const Workspace &w, int prec,
                                  int64_t slab_elems, const int *pos2unk, int64_t npos,
                                  const int64_t *pos_real_off, cudaStream_t st);
cudaError_t launch_bcr_factor(const DeviceTables &t, const Workspace &w, int prec,
                              const RealInfo *host_real, int *nlaunch, cudaStream_t st);
cudaError_t launch_iface_solve(const DeviceTables &t, const Workspace &w, int prec,
                               const int *pos2unk, double tol, int max_solves, int grid,
                               int max_vec, cudaStream_t st);
cudaError_t launch_reconstruct(const DeviceTables &t, const Workspace &w, double *p,
                               double *ux, double *uy, double *gam, cudaStream_t st);
int iface_solve_grid(int prec, int dev, int max_vec);
// message returned by mrcm_last_error(NULL) (thread-local)
void set_global_error(const char *msg);
// stage_max: the largest per-slab staging footprint (pair plans rounded to
// 16 bytes + 8 bytes per pair entry) over the batch
int iface_cluster_plan(int prec, int nslab, int bmax, int nlev, int mmax, int emax,
                       size_t stage_max, int dev);
cudaError_t launch_iface_cluster(const DeviceTables &t, const Workspace &w, const int *slab_if,
                                 const int *slab_if_off, int nslab, int bmax, int nlev,
                                 double tol, int max_solves, cudaStream_t st);
cudaError_t init_big_attributes();
cudaError_t init_tc_attributes();
size_t tc_gemm_smem();
cudaError_t launch_tc_gemm(const GemmJob *jobs, int njobs, int nmax, int *status,
                           cudaStream_t st);
cudaError_t launch_simt_gemm(const GemmJob *jobs, int njobs, int nmax, cudaStream_t st);
bool tc_encode_raw_maps(const GemmJob &jb, void *out4);
cudaError_t launch_tc_split(const GemmJob *jobs, const void *maps, int njobs, int nmax,
                            int *status, cudaStream_t st);
cudaError_t launch_big_factor(const BigPlan &bp, int prec, int *status, int *nlaunch,
                              cudaStream_t st);
int big_solve_grid(int prec, int dev);
cudaError_t launch_big_solve(const DeviceTables &t, const Workspace &w, const BigPlan &bp, int prec,
                             double tol, int max_solves, int grid, cudaStream_t st);
size_t gmres_smem_bytes(int K);
int gmres_max_blocks(int K, int dev);
cudaError_t launch_gmres_precond(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                                 double *Pbj, bool build_bj, cudaStream_t st);
cudaError_t launch_gmres(const DeviceTables &t, const Workspace &w, const GmArgs &a, int nblk,
                         cudaStream_t st);
cudaError_t init_local_attributes();
// learned preconditioner: window gather, blocks, targets, inference
cudaError_t lp_windows(const DeviceTables &t, const double *K, const double *lam, void *x, int s,
                       int g0, int count, cudaStream_t st);
cudaError_t lp_blocks(const DeviceTables &t, const double *Pbj, const float *delta, double *Puser,
                      int g0, int count, int m, cudaStream_t st);
size_t lp_targets_smem(int nloc, int m);
cudaError_t launch_gmres_nb(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                            const int *nb_off, const int *nb_list, int nloc_max, int mmax,
                            cudaStream_t st);
cudaError_t launch_gmres_bj(const DeviceTables &t, const Workspace &w, const GmArgs &a, double *Pbj,
                            cudaStream_t st);
cudaError_t lp_targets(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                       const int *nb_off, const int *nb_list, int nloc_max, int m, double theta,
                       float *target, int *bad, cudaStream_t st);
cudaError_t init_iface_attributes(int prec, int bmax, int max_vec);

}  // namespace mrcm

// network object of the learned preconditioner (learned.cu)
struct mrcm_lp;
namespace mrcm {
cudaError_t lp_forward(mrcm_lp *lp, const void *x, int B, float *delta);
int lp_s(const mrcm_lp *lp);
int lp_m(const mrcm_lp *lp);
int lp_maxb(const mrcm_lp *lp);
void *lp_xbuf(mrcm_lp *lp);
float *lp_deltabuf(mrcm_lp *lp);
cudaStream_t lp_stream(const mrcm_lp *lp);
}  // namespace mrcm
