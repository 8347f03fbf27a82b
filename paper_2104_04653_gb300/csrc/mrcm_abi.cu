// Host side of the C ABI (include/mrcm.h): descriptor validation, the
// subdomain / interface / slab tables of Section 3, workspace allocation and
// the launch sequence of the five hot-path calls.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"
#include "../../include/mrcm_learned.h"
#include "../../include/mrcm_testing.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <string>
#include <vector>
#include <algorithm>

#include <cuda_runtime.h>

using namespace mrcm;

struct mrcm_ctx {
  mrcm_desc d{};
  int dev = 0;
  cudaStream_t stream = nullptr;
  int prec = 0;
  int state = 0;           // 0 set up, 1 factored, 2 basis, 3 interface solved
  int launches = 0;
  std::string err;
  // host tables
  std::vector<SubInfo> sub;
  std::vector<IfaceInfo> iface;
  std::vector<ColInfo> col;
  std::vector<RealInfo> real;
  std::vector<BasisItem> items;            // s = 16 subdomains' CTAs first
  int nitems16 = 0;
  int nc16 = kNC16, nc32 = kNC32;          // basis tile widths (autotuned)
  int64_t max_items = 0;
  std::vector<int> sub_by_size;
  int nsub16 = 0, smax = 16;
  int64_t coef_elems = 0, w_elems = 0, alpha_elems = 0;
  std::vector<int> unk_iface, unk_slabpos, pos2unk;
  std::vector<int> slab_if, slab_if_off;   // interfaces of every (realisation, slab)
  int mmax = 1, nslab_max = 0, bmax_max = 0, nlev_max = 0;
  int cluster_k = 0;                       // > 0: one-launch cluster interface path
  int rec_cap = 0, rec_maxch = 0;          // refinement-stall recovery slots, items per slot
  int *d_slab_if = nullptr, *d_slab_if_off = nullptr;
  // cluster interface plans (see DeviceTables)
  std::vector<int> plan_info, plan_cnt, plan_goff, plan_fgoff, plan_tsc, pair_off, pair_goff;
  std::vector<short> plan_xi;
  std::vector<PairPlan> pairs;
  int emax = 1;
  bool plans_ok = false;
  std::vector<int64_t> pos_real_off;
  int64_t slab_elems = 0, xy_elems = 0, npos = 0, basis_elems = 0, g_elems = 0, gam_elems = 0;
  int64_t tsc_elems = 0;
  int max_vec = 0;
  int nunk = 0;
  // device
  void *arena = nullptr;
  DeviceTables t{};
  Workspace w{};
  BasisItem *d_items = nullptr;
  int *d_pos2unk = nullptr;
  int64_t *d_pos_real_off = nullptr;
  int solve_grid = 1;
  // GMRES interface path
  bool use_gmres = false;
  // direct path with slabs above 64 unknowns
  bool use_big = false;
  bool quad = false;                       // some realisation has a quadtree layout
  std::vector<int> big_lev_off;
  std::vector<InvJob> big_inv;
  std::vector<GemmJob> big_gemm;
  BigPlan bp{};
  int big_grid = 0;
  int gm_K = 40, gm_maxit = 5000, gm_precond = 0, gm_nblk = 0;
  double gm_tol = 1e-13;
  bool gm_user_set = false;
  std::vector<GmRow> gm_rows;
  std::vector<GmBlock> gm_blocks;
  GmArgs gm{};
  double *gm_Pbj = nullptr, *gm_Pid = nullptr, *gm_Puser = nullptr;
  // learned preconditioner: interface neighbourhoods of the training target
  std::vector<int> nb_off, nb_list;
  int nb_max = 0, nloc_max = 0, m_uniform = 0, s_uniform = 0;
  // caller's interface functions (mrcm_desc::iface_fn): rows per size
  int fn_rows16 = 0, fn_rows32 = 0;
  int *d_nb_off = nullptr, *d_nb_list = nullptr;
  // neighbourhood preconditioner (GmArgs): its neighbourhood lists and host tables
  bool use_nb = false;
  std::vector<int> pnb_off, pnb_list;
  int pnb_max = 0, pnloc_max = 0;
  int *d_pnb_off = nullptr, *d_pnb_list = nullptr;
  std::vector<int64_t> p_off, gw_off, gat_o;
  std::vector<int> gw_w, pb_off, pb_list, pb_pos, gat_off, gat_g;
};

static thread_local std::string g_setup_err;

static int d_nreal(const mrcm_ctx *c) { return c->d.n_real; }

// subdomain sizes present (one launch each for factor, basis, reconstruct)
static int n_sizes(const mrcm_ctx *c) {
  return (c->nsub16 > 0 ? 1 : 0) + (static_cast<int>(c->sub.size()) > c->nsub16 ? 1 : 0);
}

static mrcm_status fail(mrcm_ctx *c, mrcm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  else g_setup_err = buf;
  return s;
}

void mrcm::set_global_error(const char *msg) { g_setup_err = msg; }

static mrcm_status cuda_fail(mrcm_ctx *c, cudaError_t e, const char *where) {
  return fail(c, MRCM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Interface functions at face midpoints t_e = -1 + (2e+1)/s: Legendre
// polynomials by their three-term recurrence, or monomials.
static void fn_table(int family, int s, std::vector<double> &out) {
  out.assign(static_cast<size_t>(s) * s, 0.0);
  for (int e = 0; e < s; ++e) {
    const double tt = -1.0 + (2.0 * e + 1.0) / s;
    double pm1 = 0.0, p = 1.0;
    for (int k = 0; k < s; ++k) {
      if (family == MRCM_BASIS_LEGENDRE) {
        out[static_cast<size_t>(k) * s + e] = p;
        const double pn = ((2.0 * k + 1.0) * tt * p - k * pm1) / (k + 1.0);
        pm1 = p;
        p = pn;
      } else {
        out[static_cast<size_t>(k) * s + e] = std::pow(tt, k);
      }
    }
  }
}

// Quadtree realisation (mrcm_desc.refine): the subdomains (sorted by
// (y0, x0)) and the interface segments in canonical order -- vertical ones
// by (first row, x line), then horizontal ones by (y line, first column);
// L is the subdomain on the -x / -y side.  A segment is a maximal run of
// faces shared by the same two subdomains.
struct QSub {
  int x0, y0, s;
};
struct QSeg {
  int kind, fx, fy, len, L, R;   // L, R: indices into the realisation's subdomains
};

static int64_t refine_entries(const mrcm_desc &d, int r) {
  const int B = d.sub_size[r];
  return static_cast<int64_t>(d.nx / B) * (d.ny / B);
}

static bool is_quad(const mrcm_desc &d, int r, int64_t ref_off) {
  if (!d.refine) return false;
  for (int64_t k = 0; k < refine_entries(d, r); ++k)
    if (d.refine[ref_off + k]) return true;
  return false;
}

static void quad_layout(const mrcm_desc &d, int r, int64_t ref_off, std::vector<QSub> &subs,
                        std::vector<QSeg> &segs) {
  const int B = d.sub_size[r], bx = d.nx / B, by = d.ny / B, q = B / 2;
  subs.clear();
  segs.clear();
  for (int BJ = 0; BJ < by; ++BJ)
    for (int BI = 0; BI < bx; ++BI) {
      if (d.refine[ref_off + static_cast<int64_t>(BJ) * bx + BI]) {
        for (int j = 0; j < 2; ++j)
          for (int i = 0; i < 2; ++i) subs.push_back(QSub{BI * B + i * q, BJ * B + j * q, q});
      } else {
        subs.push_back(QSub{BI * B, BJ * B, B});
      }
    }
  std::sort(subs.begin(), subs.end(), [](const QSub &a, const QSub &b) {
    return a.y0 != b.y0 ? a.y0 < b.y0 : a.x0 < b.x0;
  });
  const int mx = d.nx / q, my = d.ny / q;
  std::vector<int> own(static_cast<size_t>(mx) * my, -1);
  for (size_t k = 0; k < subs.size(); ++k)
    for (int j = subs[k].y0 / q; j < (subs[k].y0 + subs[k].s) / q; ++j)
      for (int i = subs[k].x0 / q; i < (subs[k].x0 + subs[k].s) / q; ++i)
        own[static_cast<size_t>(j) * mx + i] = static_cast<int>(k);
  auto at = [&](int j, int i) { return own[static_cast<size_t>(j) * mx + i]; };
  std::vector<QSeg> vert, horiz;
  for (int i = 1; i < mx; ++i)
    for (int j = 0; j < my;) {
      const int L = at(j, i - 1), R = at(j, i);
      if (L == R) {
        ++j;
        continue;
      }
      int j1 = j;
      while (j1 < my && at(j1, i - 1) == L && at(j1, i) == R) ++j1;
      vert.push_back(QSeg{0, i * q, j * q, (j1 - j) * q, L, R});
      j = j1;
    }
  for (int j = 1; j < my; ++j)
    for (int i = 0; i < mx;) {
      const int L = at(j - 1, i), R = at(j, i);
      if (L == R) {
        ++i;
        continue;
      }
      int i1 = i;
      while (i1 < mx && at(j - 1, i1) == L && at(j, i1) == R) ++i1;
      horiz.push_back(QSeg{1, i * q, j * q, (i1 - i) * q, L, R});
      i = i1;
    }
  auto by_fy_fx = [](const QSeg &a, const QSeg &b) {
    return a.fy != b.fy ? a.fy < b.fy : a.fx < b.fx;
  };
  std::sort(vert.begin(), vert.end(), by_fy_fx);
  std::sort(horiz.begin(), horiz.end(), by_fy_fx);
  segs = vert;
  segs.insert(segs.end(), horiz.begin(), horiz.end());
}

// Interfaces of realisation r and their lengths in faces (canonical order).
static void iface_lengths(const mrcm_desc &d, int r, int64_t ref_off, std::vector<int> &len) {
  len.clear();
  if (is_quad(d, r, ref_off)) {
    std::vector<QSub> subs;
    std::vector<QSeg> segs;
    quad_layout(d, r, ref_off, subs, segs);
    for (const QSeg &sg : segs) len.push_back(sg.len);
    return;
  }
  const int s = d.sub_size[r], sx = d.nx / s, sy = d.ny / s;
  len.assign(static_cast<size_t>(sx - 1) * sy + static_cast<size_t>(sx) * (sy - 1), s);
}

static mrcm_status validate(const mrcm_desc *d) {
  if (!d) return fail(nullptr, MRCM_EINVAL, "descriptor is NULL");
  if (d->nx <= 0 || d->ny <= 0) return fail(nullptr, MRCM_EINVAL, "nx, ny must be positive");
  if (d->n_real <= 0 || d->n_real > kMaxRealisations)
    return fail(nullptr, MRCM_EINVAL, "n_real out of range");
  if (!(d->ly > 0.0) || !std::isfinite(d->ly)) return fail(nullptr, MRCM_EINVAL, "ly must be > 0");
  if (!d->sub_size || !d->iface_nU || !d->iface_nP || !d->bc_type || !d->bc_val)
    return fail(nullptr, MRCM_EINVAL, "sub_size, iface_nU, iface_nP, bc_type, bc_val are required");
  if (d->prec != MRCM_PREC_FP64 && d->prec != MRCM_PREC_FP32_IR)
    return fail(nullptr, MRCM_EINVAL, "unknown precision %d", d->prec);
  if (d->basis_family != MRCM_BASIS_LEGENDRE && d->basis_family != MRCM_BASIS_MONOMIAL)
    return fail(nullptr, MRCM_EINVAL, "unknown basis family %d", d->basis_family);
  if (!(d->ir_tol > 0.0) || !(d->iface_tol > 0.0) || d->ir_max < 0 || d->iface_ir_max < 0)
    return fail(nullptr, MRCM_EINVAL, "tolerances must be > 0 and sweep limits >= 0");
  if (d->ir_max > 1000 || d->iface_ir_max > 1000)
    return fail(nullptr, MRCM_EINVAL, "sweep limits above 1000");
  if (d->iface_solver < MRCM_IFACE_AUTO || d->iface_solver > MRCM_IFACE_GMRES)
    return fail(nullptr, MRCM_EINVAL, "unknown interface solver %d", d->iface_solver);
  if (d->precond < MRCM_PRECOND_BLOCK_JACOBI || d->precond > MRCM_PRECOND_NEIGHBOURHOOD_SHARED)
    return fail(nullptr, MRCM_EINVAL, "unknown preconditioner %d", d->precond);
  if (d->gmres_restart < 0 || d->gmres_restart > kGmKmax)
    return fail(nullptr, MRCM_EINVAL, "gmres_restart must be in 0..%d", kGmKmax);
  if (d->gmres_max < 0 || !(d->gmres_tol >= 0.0))
    return fail(nullptr, MRCM_EINVAL, "gmres_max and gmres_tol must be >= 0");
  for (int r = 0; r < d->n_real; ++r) {
    const int s = d->sub_size[r];
    if (s != 16 && s != 32)
      return fail(nullptr, MRCM_EINVAL, "subdomain size %d not supported (16 or 32)", s);
    if (d->nx % s || d->ny % s)
      return fail(nullptr, MRCM_EINVAL, "grid %dx%d not divisible by subdomain size %d", d->nx,
                  d->ny, s);
  }
  bool any_quad = false;
  if (d->refine) {               // quadtree: only 32 x 32 blocks split, into 16 x 16
    int64_t ro = 0;
    for (int r = 0; r < d->n_real; ++r) {
      if (is_quad(*d, r, ro)) {
        any_quad = true;
        if (d->sub_size[r] != 32)
          return fail(nullptr, MRCM_EINVAL,
                      "refine: realisation %d splits %dx%d subdomains (only 32x32 split)", r,
                      d->sub_size[r], d->sub_size[r]);
      }
      ro += refine_entries(*d, r);
    }
  }
  if (any_quad) {
    if (d->iface_solver == MRCM_IFACE_DIRECT)
      return fail(nullptr, MRCM_EINVAL, "refine: the direct interface solvers need uniform "
                                        "subdomains (use GMRES)");
    if (d->precond != MRCM_PRECOND_BLOCK_JACOBI && d->precond != MRCM_PRECOND_NONE &&
        d->precond != MRCM_PRECOND_NEIGHBOURHOOD_SHARED)
      return fail(nullptr, MRCM_EINVAL, "refine: block-Jacobi, the shared neighbourhood or no "
                                        "preconditioner");
    if (d->pure_neumann)
      return fail(nullptr, MRCM_EINVAL, "refine: pure-Neumann problems need uniform subdomains");
  }
  if (d->iface_fn) {             // every value of the caller's interface functions
    int64_t src = 0, ifc = 0, ro = 0;
    std::vector<int> len;
    for (int r = 0; r < d->n_real; ++r) {
      iface_lengths(*d, r, ro, len);
      if (d->refine) ro += refine_entries(*d, r);
      for (size_t g = 0; g < len.size(); ++g, ++ifc) {
        const int n = std::max(0, d->iface_nU[ifc]) + std::max(0, d->iface_nP[ifc]);
        for (int64_t k = 0; k < static_cast<int64_t>(n) * len[g]; ++k)
          if (!std::isfinite(d->iface_fn[src + k]))
            return fail(nullptr, MRCM_EINVAL, "iface_fn: non-finite value at %lld",
                        static_cast<long long>(src + k));
        src += static_cast<int64_t>(n) * len[g];
      }
    }
  }
  const int nb = 2 * d->nx + 2 * d->ny;
  for (int k = 0; k < nb; ++k) {
    if (d->bc_type[k] != 0 && d->bc_type[k] != 1)
      return fail(nullptr, MRCM_EINVAL, "bc_type[%d] must be 0 or 1", k);
    if (!std::isfinite(d->bc_val[k])) return fail(nullptr, MRCM_EINVAL, "bc_val[%d] not finite", k);
    if (d->pure_neumann && d->bc_type[k] != 0)
      return fail(nullptr, MRCM_EINVAL, "pure_neumann with a Dirichlet face");
  }
  return MRCM_OK;
}

static mrcm_status build_tables(mrcm_ctx *c) {
  const mrcm_desc &d = c->d;
  const double h = d.ly / d.ny;
  int nsub_tot = 0, nif_tot = 0, unk_tot = 0;
  int64_t alpha_off = 0, gam_off = 0, slab_off = 0, xy_off = 0, vec_off = 0;
  int64_t basis_off = 0, g_off = 0, tsc_off = 0, coef_off = 0, w_off = 0;
  int col_off = 0;
  int64_t ref_off = 0;  // this realisation's entries of d.refine
  bool any_quad = false;
  std::vector<int> subs32;
  int nslab_all = 1;   // slabs run along the longer side (the same for every s)
  for (int r = 0; r < d.n_real; ++r) {
    const int sx = d.nx / d.sub_size[r], sy = d.ny / d.sub_size[r];
    nslab_all = std::max(nslab_all, sx >= sy ? sx : sy);
  }
  for (int r = 0; r < d.n_real; ++r) {
    const int S = d.sub_size[r];
    c->smax = std::max(c->smax, S);
    RealInfo ri{};
    ri.s = S;
    ri.Sx = d.nx / S;
    ri.Sy = d.ny / S;
    ri.sub0 = nsub_tot;
    ri.nsub = ri.Sx * ri.Sy;
    ri.iface0 = nif_tot;
    ri.niface = (ri.Sx - 1) * ri.Sy + ri.Sx * (ri.Sy - 1);
    ri.unk0 = unk_tot;
    ri.h = h;
    ri.H = S * h;
    if (d.pure_neumann && ri.nsub < 2)
      return fail(nullptr, MRCM_EINVAL, "pure_neumann needs at least two subdomains");
    if (is_quad(d, r, ref_off)) {
      // quadtree realisation: 32 x 32 blocks, the refined ones as four 16 x 16
      // subdomains; interfaces are the segments of quad_layout
      any_quad = true;
      std::vector<QSub> qs;
      std::vector<QSeg> qg;
      quad_layout(d, r, ref_off, qs, qg);
      ri.quad = 1;
      ri.nsub = static_cast<int>(qs.size());
      ri.niface = static_cast<int>(qg.size());
      for (int g = 0; g < ri.niface; ++g) {
        const QSeg &sg = qg[g];
        IfaceInfo fi{};
        fi.r = r;
        fi.kind = sg.kind;
        fi.L = ri.sub0 + sg.L;
        fi.R = ri.sub0 + sg.R;
        fi.fx = sg.fx;
        fi.fy = sg.fy;
        fi.nU = d.iface_nU[nif_tot + g];
        fi.nP = d.iface_nP[nif_tot + g];
        if (fi.nU < 0 || fi.nP < 0 || fi.nU > sg.len || fi.nP > sg.len || fi.nU + fi.nP < 1)
          return fail(nullptr, MRCM_EINVAL, "interface %d: need 0 <= nU,nP <= %d, nU+nP >= 1",
                      nif_tot + g, sg.len);
        fi.s = sg.len;
        fi.unk = unk_tot;
        unk_tot += fi.nU + fi.nP;
        fi.alpha_off = alpha_off;
        alpha_off += sg.len;
        fi.gam_off = gam_off;
        gam_off += 2 * sg.len;
        fi.tsc_off = tsc_off;
        tsc_off += static_cast<int64_t>(fi.nU + fi.nP) * (fi.nU + fi.nP);
        fi.rowL = fi.rowR = fi.colL = fi.colR = -1;
        if (d.iface_fn) {
          int &rows = sg.len == 16 ? c->fn_rows16 : c->fn_rows32;
          fi.fnU = rows;
          fi.fnP = rows + fi.nU;
          rows += fi.nU + fi.nP;
        } else {
          fi.fnU = fi.fnP = 0;
        }
        c->iface.push_back(fi);
      }
      ri.nunk = unk_tot - ri.unk0;
      ri.pin = -1;
      // the segments on every side of every subdomain, in order along the edge
      std::vector<int> side_seg(qs.size() * 8, -1);
      for (int g = 0; g < ri.niface; ++g) {
        const QSeg &sg = qg[g];
        const int sL = sg.kind == 0 ? kEdgeE : kEdgeN, sR = sg.kind == 0 ? kEdgeW : kEdgeS;
        for (const int k : {sg.L * 8 + sL * 2, sg.R * 8 + sR * 2}) {
          if (side_seg[k] < 0) side_seg[k] = g;
          else if (side_seg[k + 1] < 0) side_seg[k + 1] = g;
          else return fail(nullptr, MRCM_EINVAL, "refine: more than two interfaces on an edge");
        }
      }
      for (size_t k = 0; k < qs.size(); ++k) {
        const int Sk = qs[k].s;
        SubInfo sb{};
        sb.r = r;
        sb.I = qs[k].x0 / 16;
        sb.J = qs[k].y0 / 16;
        sb.x0 = qs[k].x0;
        sb.y0 = qs[k].y0;
        sb.s = Sk;
        const int gid = static_cast<int>(c->sub.size());
        sb.col_off = col_off;
        c->col.push_back(ColInfo{-1, -1, 0, 0});
        int ncol = 1, nrow = 0;
        for (int e = 0; e < 4; ++e) {
          const int a0 = side_seg[k * 8 + e * 2], a1 = side_seg[k * 8 + e * 2 + 1];
          // one interface over the whole edge, or two over its halves
          const bool ok = a0 < 0 ? a1 < 0
                                 : (a1 < 0 ? qg[a0].len == Sk
                                           : qg[a0].len == Sk / 2 && qg[a1].len == Sk / 2);
          if (!ok) return fail(nullptr, MRCM_EINVAL, "refine: unsupported edge layout");
          sb.edge_iface[e] = a0 < 0 ? -1 : ri.iface0 + a0;
          sb.edge_iface2[e] = a1 < 0 ? -1 : ri.iface0 + a1;
          sb.edge_col2[e] = sb.edge_row2[e] = -1;
          for (int half = 0; half < 2; ++half) {
            const int a = half ? a1 : a0;
            if (half) {
              sb.edge_col2[e] = a < 0 ? -1 : ncol;
              sb.edge_row2[e] = a < 0 ? -1 : nrow;
            } else {
              sb.edge_col[e] = ncol;
              sb.edge_row[e] = nrow;
            }
            if (a < 0) continue;
            IfaceInfo &fi = c->iface[ri.iface0 + a];
            if (fi.L == gid) {
              fi.rowL = nrow;
              fi.colL = ncol;
            } else {
              fi.rowR = nrow;
              fi.colR = ncol;
            }
            for (int kk = 0; kk < fi.nU; ++kk)
              c->col.push_back(ColInfo{fi.unk + kk, e, fi.fnU + kk, 1});
            for (int kk = 0; kk < fi.nP; ++kk)
              c->col.push_back(ColInfo{fi.unk + fi.nU + kk, e, fi.fnP + kk, 0});
            ncol += fi.nU + fi.nP;
            nrow += fi.nU + fi.nP;
          }
        }
        sb.ncols = ncol;
        sb.nrows = nrow;
        col_off += ncol;
        sb.basis_off = basis_off;
        basis_off += static_cast<int64_t>(ncol) * Sk * Sk;
        sb.g_off = g_off;
        g_off += static_cast<int64_t>(nrow) * ncol;
        sb.coef_off = coef_off;
        coef_off += 6 * Sk * Sk + 4 * Sk;
        sb.w_off = w_off;
        w_off += static_cast<int64_t>(Sk) * Sk * Sk;
        if (Sk == 16) c->sub_by_size.push_back(gid);
        else subs32.push_back(gid);
        c->sub.push_back(sb);
      }
      // no slab structure: every interface in slab 0 (the direct solvers refuse
      // quadtree layouts; the GMRES path uses no slabs)
      ri.nslab = nslab_all;
      int pos = 0;
      for (int k = 0; k < ri.nslab; ++k) {
        c->slab_if_off.push_back(static_cast<int>(c->slab_if.size()));
        if (k == 0)
          for (int g = 0; g < ri.niface; ++g) {
            c->slab_if.push_back(ri.iface0 + g);
            IfaceInfo &fi = c->iface[ri.iface0 + g];
            fi.slab = 0;
            fi.pos = pos;
            pos += fi.nU + fi.nP;
          }
      }
      ri.bmax = std::max(1, pos);
      ri.nlev = 0;
      ri.slab_off = slab_off;
      ri.xy_off = xy_off;
      ri.vec_off = vec_off;
      c->pos_real_off.push_back(vec_off);
      vec_off += static_cast<int64_t>(ri.nslab) * ri.bmax;
      c->real.push_back(ri);
      nsub_tot += ri.nsub;
      nif_tot += ri.niface;
      ref_off += refine_entries(d, r);
      continue;
    }
    // interfaces in canonical order
    const int nV = (ri.Sx - 1) * ri.Sy;
    for (int g = 0; g < ri.niface; ++g) {
      IfaceInfo fi{};
      fi.r = r;
      int I, J;
      if (g < nV) {
        fi.kind = 0;
        J = g / (ri.Sx - 1);
        I = g % (ri.Sx - 1);
        fi.L = ri.sub0 + J * ri.Sx + I;
        fi.R = fi.L + 1;
      } else {
        fi.kind = 1;
        J = (g - nV) / ri.Sx;
        I = (g - nV) % ri.Sx;
        fi.L = ri.sub0 + J * ri.Sx + I;
        fi.R = fi.L + ri.Sx;
      }
      fi.fx = fi.kind == 0 ? (I + 1) * S : I * S;
      fi.fy = fi.kind == 0 ? J * S : (J + 1) * S;
      fi.nU = d.iface_nU[nif_tot + g];
      fi.nP = d.iface_nP[nif_tot + g];
      if (fi.nU < 0 || fi.nP < 0 || fi.nU > S || fi.nP > S || fi.nU + fi.nP < 1)
        return fail(nullptr, MRCM_EINVAL, "interface %d: need 0 <= nU,nP <= %d, nU+nP >= 1",
                    nif_tot + g, S);
      if (d.pure_neumann && fi.nP < 1)
        return fail(nullptr, MRCM_EINVAL, "pure_neumann needs nP >= 1 on every interface");
      fi.s = S;
      fi.unk = unk_tot;
      unk_tot += fi.nU + fi.nP;
      fi.alpha_off = alpha_off;
      alpha_off += S;
      fi.gam_off = gam_off;
      gam_off += 2 * S;
      fi.tsc_off = tsc_off;
      tsc_off += static_cast<int64_t>(fi.nU + fi.nP) * (fi.nU + fi.nP);
      if (d.iface_fn) {          // own rows: phi_0 .. then psi_0 .. in the size-S section
        int &rows = S == 16 ? c->fn_rows16 : c->fn_rows32;
        fi.fnU = rows;
        fi.fnP = rows + fi.nU;
        rows += fi.nU + fi.nP;
      } else {                   // the family's rows: phi_k = psi_k = row k
        fi.fnU = fi.fnP = 0;
      }
      c->iface.push_back(fi);
    }
    ri.nunk = unk_tot - ri.unk0;
    ri.pin = -1;
    if (d.pure_neumann) {
      const IfaceInfo &f0 = c->iface[ri.iface0];
      ri.pin = f0.unk + f0.nU;   // P_0 of the first interface
    }
    // subdomains
    for (int J = 0; J < ri.Sy; ++J)
      for (int I = 0; I < ri.Sx; ++I) {
        SubInfo sb{};
        sb.r = r;
        sb.I = I;
        sb.J = J;
        sb.x0 = I * S;
        sb.y0 = J * S;
        sb.s = S;
        const int ifW = (I > 0) ? ri.iface0 + J * (ri.Sx - 1) + (I - 1) : -1;
        const int ifE = (I < ri.Sx - 1) ? ri.iface0 + J * (ri.Sx - 1) + I : -1;
        const int ifS = (J > 0) ? ri.iface0 + nV + (J - 1) * ri.Sx + I : -1;
        const int ifN = (J < ri.Sy - 1) ? ri.iface0 + nV + J * ri.Sx + I : -1;
        sb.edge_iface[0] = ifW;
        sb.edge_iface[1] = ifE;
        sb.edge_iface[2] = ifS;
        sb.edge_iface[3] = ifN;
        for (int e = 0; e < 4; ++e) sb.edge_iface2[e] = sb.edge_col2[e] = sb.edge_row2[e] = -1;
        sb.col_off = col_off;
        c->col.push_back(ColInfo{-1, -1, 0, 0});
        int ncol = 1, nrow = 0;
        const int gid_here = static_cast<int>(c->sub.size());
        for (int e = 0; e < 4; ++e) {
          sb.edge_col[e] = ncol;
          sb.edge_row[e] = nrow;
          if (sb.edge_iface[e] < 0) continue;
          IfaceInfo &fi = c->iface[sb.edge_iface[e]];
          if (fi.L == gid_here) {
            fi.rowL = nrow;
            fi.colL = ncol;
          } else {
            fi.rowR = nrow;
            fi.colR = ncol;
          }
          for (int k = 0; k < fi.nU; ++k)
            c->col.push_back(ColInfo{fi.unk + k, e, fi.fnU + k, 1});
          for (int k = 0; k < fi.nP; ++k)
            c->col.push_back(ColInfo{fi.unk + fi.nU + k, e, fi.fnP + k, 0});
          ncol += fi.nU + fi.nP;
          nrow += fi.nU + fi.nP;
        }
        sb.ncols = ncol;
        sb.nrows = nrow;
        col_off += ncol;
        sb.basis_off = basis_off;
        basis_off += static_cast<int64_t>(ncol) * S * S;
        sb.g_off = g_off;
        g_off += static_cast<int64_t>(nrow) * ncol;
        sb.coef_off = coef_off;
        coef_off += 6 * S * S + 4 * S;
        sb.w_off = w_off;
        w_off += static_cast<int64_t>(S) * S * S;
        const int gid = static_cast<int>(c->sub.size());
        if (S == 16) c->sub_by_size.push_back(gid);
        else subs32.push_back(gid);
        c->sub.push_back(sb);
      }
    // slabs: block-tridiagonal grouping of the interfaces
    // Every realisation gets the batch's largest slab count (the direct
    // interface kernels take one slab count per launch); slabs past the
    // realisation's own count are empty: identity rows, no coupling.
    const bool xdir = ri.Sx >= ri.Sy;
    const int nat = xdir ? ri.Sx : ri.Sy;
    ri.nslab = nslab_all;
    std::vector<std::vector<int>> slabs(ri.nslab);
    for (int k = 0; k < nat; ++k) {
      if (xdir) {
        for (int J = 0; J < ri.Sy - 1; ++J) slabs[k].push_back(ri.iface0 + nV + J * ri.Sx + k);
        if (k < ri.Sx - 1)
          for (int J = 0; J < ri.Sy; ++J) slabs[k].push_back(ri.iface0 + J * (ri.Sx - 1) + k);
      } else {
        for (int I = 0; I < ri.Sx - 1; ++I) slabs[k].push_back(ri.iface0 + k * (ri.Sx - 1) + I);
        if (k < ri.Sy - 1)
          for (int I = 0; I < ri.Sx; ++I) slabs[k].push_back(ri.iface0 + nV + k * ri.Sx + I);
      }
    }
    ri.bmax = 1;
    for (int k = 0; k < ri.nslab; ++k) {
      c->slab_if_off.push_back(static_cast<int>(c->slab_if.size()));
      for (int g : slabs[k]) c->slab_if.push_back(g);
    }
    for (int k = 0; k < ri.nslab; ++k) {
      int pos = 0;
      for (int g : slabs[k]) {
        IfaceInfo &fi = c->iface[g];
        fi.slab = k;
        fi.pos = pos;
        pos += fi.nU + fi.nP;
      }
      if (pos > ri.bmax) ri.bmax = pos;
    }
    // a multiple of 4 (positions past the widest slab are padding, identity
    // on the diagonal): the FP32 slab blocks' rows start on 16-byte
    // boundaries, as the tensor-core products' TMA copies require
    ri.bmax = (ri.bmax + 3) & ~3;
    if (ri.bmax > 64) c->use_big = true;
    int nlev = 0;
    while ((1 << nlev) < ri.nslab) ++nlev;
    ri.nlev = nlev;
    ri.slab_off = slab_off;
    slab_off += static_cast<int64_t>(ri.nslab) * ri.bmax * ri.bmax;
    ri.xy_off = xy_off;
    xy_off += static_cast<int64_t>(nlev) * ri.nslab * ri.bmax * ri.bmax;
    ri.vec_off = vec_off;
    c->pos_real_off.push_back(vec_off);
    vec_off += static_cast<int64_t>(ri.nslab) * ri.bmax;
    if (ri.nslab * ri.bmax > c->max_vec) c->max_vec = ri.nslab * ri.bmax;
    c->real.push_back(ri);
    nsub_tot += ri.nsub;
    nif_tot += ri.niface;
    if (d.refine) ref_off += refine_entries(d, r);
  }
  c->slab_if_off.push_back(static_cast<int>(c->slab_if.size()));
  c->nunk = unk_tot;
  c->nsub16 = static_cast<int>(c->sub_by_size.size());
  c->sub_by_size.insert(c->sub_by_size.end(), subs32.begin(), subs32.end());
  c->coef_elems = coef_off;
  c->w_elems = w_off;
  c->alpha_elems = alpha_off;
  c->quad = any_quad;
  if (d.iface_solver == MRCM_IFACE_GMRES || any_quad) c->use_gmres = true;
  if (c->use_gmres) {
    // no slab blocks on the GMRES path
    c->use_big = false;
    slab_off = 0;
    xy_off = 0;
    for (RealInfo &ri : c->real) ri.slab_off = ri.xy_off = 0;
  } else if (c->use_big) {
    // big slabs: one multiplier slot per surviving slab and level (compact)
    const int K = c->real.empty() ? 1 : c->real[0].nslab;
    int nlev = 0;
    while ((1 << nlev) < K) ++nlev;
    c->big_lev_off.assign(1, 0);
    for (int lev = 0, st = 1; lev < nlev; ++lev, st <<= 1)
      c->big_lev_off.push_back(c->big_lev_off.back() + (K + 2 * st - 1) / (2 * st));
    xy_off = 0;
    for (RealInfo &ri : c->real) {
      ri.xy_off = xy_off;
      xy_off += static_cast<int64_t>(c->big_lev_off.back()) * ri.bmax * ri.bmax;
    }
    if (nlev > kBigMaxLev) return fail(nullptr, MRCM_EINVAL, "too many slabs (%d)", K);
  }
  for (const IfaceInfo &fi : c->iface) c->mmax = std::max(c->mmax, fi.nU + fi.nP);
  for (const RealInfo &ri : c->real) {
    c->nslab_max = std::max(c->nslab_max, ri.nslab);
    c->bmax_max = std::max(c->bmax_max, ri.bmax);
    c->nlev_max = std::max(c->nlev_max, ri.nlev);
  }
  c->unk_iface.assign(unk_tot, -1);
  c->unk_slabpos.assign(unk_tot, -1);
  c->pos2unk.assign(vec_off, -1);
  for (size_t g = 0; g < c->iface.size(); ++g) {
    const IfaceInfo &fi = c->iface[g];
    const RealInfo &ri = c->real[fi.r];
    for (int i = 0; i < fi.nU + fi.nP; ++i) {
      const int u = fi.unk + i;
      c->unk_iface[u] = static_cast<int>(g);
      c->unk_slabpos[u] = fi.slab * ri.bmax + fi.pos + i;
      c->pos2unk[ri.vec_off + fi.slab * ri.bmax + fi.pos + i] = u;
    }
  }
  c->slab_elems = slab_off;
  c->xy_elems = xy_off;
  c->npos = vec_off;
  c->basis_elems = basis_off;
  c->g_elems = g_off;
  c->gam_elems = gam_off;
  c->tsc_elems = tsc_off;
  return MRCM_OK;
}

// Per-slab plans of the one-launch cluster interface path: for every slab
// position the G offsets and slab positions of its row's terms, and for
// every (own interface, neighbour interface) block the G offsets of its
// entries.  Everything the kernel would otherwise chase through the tables.
static void build_plans(mrcm_ctx *c) {
  c->emax = 1;
  if (c->use_gmres || c->use_big) {
    c->plans_ok = false;
    return;
  }
  for (const IfaceInfo &fi : c->iface)
    c->emax = std::max(c->emax, c->sub[fi.L].ncols - 1 + c->sub[fi.R].ncols - 1);
  const int E = c->emax;
  const int64_t npos = c->npos;
  if (c->g_elems >= (int64_t(1) << 31) || npos * E >= (int64_t(1) << 31)) {
    c->plans_ok = false;
    return;
  }
  c->plan_info.assign(npos, -1);
  c->plan_cnt.assign(npos, 0);
  c->plan_goff.assign(npos * E, -1);
  c->plan_xi.assign(npos * E, 0);
  c->plan_fgoff.assign(npos * 2, -1);
  c->plan_tsc.assign(npos, 0);
  c->pairs.clear();
  c->pair_off.clear();
  c->pair_goff.clear();
  auto rows_of = [&](const IfaceInfo &fi, int i, int64_t &goffL, int64_t &goffR, const SubInfo *&L,
                     const SubInfo *&R, int &eL, int &eR) {
    L = &c->sub[fi.L];
    R = &c->sub[fi.R];
    eL = fi.kind == 0 ? kEdgeE : kEdgeN;
    eR = fi.kind == 0 ? kEdgeW : kEdgeS;
    goffL = L->g_off + static_cast<int64_t>(L->edge_row[eL] + i) * L->ncols;
    goffR = R->g_off + static_cast<int64_t>(R->edge_row[eR] + i) * R->ncols;
  };
  int slab_base = 0;   // global index of the realisation's first slab
  for (size_t r = 0; r < c->real.size(); ++r) {
    const RealInfo &ri = c->real[r];
    const int b = ri.bmax;
    for (int k = 0; k < ri.nslab; ++k) {
      // rows
      for (int p = 0; p < b; ++p) {
        const int64_t P = ri.vec_off + static_cast<int64_t>(k) * b + p;
        const int u = c->pos2unk[P];
        if (u < 0) continue;
        const IfaceInfo &fi = c->iface[c->unk_iface[u]];
        const int i = u - fi.unk, m = fi.nU + fi.nP;
        const bool pinned = (u == ri.pin);
        c->plan_info[P] = (fi.pos << 16) | (m << 8) | i | (i >= fi.nU ? (1 << 30) : 0) |
                          (pinned ? (1 << 29) : 0);
        c->plan_tsc[P] = static_cast<int>(fi.tsc_off);
        int64_t gL, gR;
        const SubInfo *L, *R;
        int eL, eR;
        rows_of(fi, i, gL, gR, L, R, eL, eR);
        if (pinned) continue;
        c->plan_fgoff[2 * P] = static_cast<int>(gL);
        c->plan_fgoff[2 * P + 1] = static_cast<int>(gR);
        int e = 0;
        for (int side = 0; side < 2; ++side) {
          const SubInfo *S = side == 0 ? L : R;
          const int64_t g0 = side == 0 ? gL : gR;
          for (int cc = 1; cc < S->ncols; ++cc, ++e) {
            const int v = c->col[S->col_off + cc].unk;
            if (v == ri.pin) continue;
            const int sp = c->unk_slabpos[v];
            const int ds = sp / b - k;
            c->plan_goff[P * E + e] = static_cast<int>(g0 + cc);
            c->plan_xi[P * E + e] = static_cast<short>((ds + 1) * b + sp % b);
          }
        }
        c->plan_cnt[P] = e;
      }
      // pairs of this slab
      c->pair_off.push_back(static_cast<int>(c->pairs.size()));
      const int s0 = c->slab_if_off[slab_base + k];
      const int s1 = c->slab_if_off[slab_base + k + 1];
      for (int q = s0; q < s1; ++q) {
        const IfaceInfo &fi = c->iface[c->slab_if[q]];
        const SubInfo &L = c->sub[fi.L], &R = c->sub[fi.R];
        std::vector<int> nb;
        for (int e = 0; e < 4; ++e) {
          if (L.edge_iface[e] >= 0) nb.push_back(L.edge_iface[e]);
          if (R.edge_iface[e] >= 0) nb.push_back(R.edge_iface[e]);
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        const int m = fi.nU + fi.nP;
        for (int gn : nb) {
          const IfaceInfo &fn = c->iface[gn];
          const int mn = fn.nU + fn.nP;
          PairPlan pp;
          pp.p0 = fi.pos;
          pp.m = m;
          pp.nU = fi.nU;
          pp.tsc = static_cast<int>(fi.tsc_off);
          pp.pn0 = fn.pos;
          pp.mn = mn;
          pp.tscn = static_cast<int>(fn.tsc_off);
          pp.ds = fn.slab - fi.slab;
          pp.nUn = fn.nU;
          pp.goff = static_cast<int>(c->pair_goff.size());
          int eLn = -1, eRn = -1;
          for (int e = 0; e < 4; ++e) {
            if (L.edge_iface[e] == gn) eLn = e;
            if (R.edge_iface[e] == gn) eRn = e;
          }
          for (int i = 0; i < m; ++i) {
            int64_t gL, gR;
            const SubInfo *Lp, *Rp;
            int eL, eR;
            rows_of(fi, i, gL, gR, Lp, Rp, eL, eR);
            for (int j = 0; j < mn; ++j) {
              const bool pin = (fi.unk + i == ri.pin) || (fn.unk + j == ri.pin);
              c->pair_goff.push_back(!pin && eLn >= 0 ? static_cast<int>(gL + L.edge_col[eLn] + j) : -1);
              c->pair_goff.push_back(!pin && eRn >= 0 ? static_cast<int>(gR + R.edge_col[eRn] + j) : -1);
            }
          }
          c->pairs.push_back(pp);
        }
      }
    }
    slab_base += ri.nslab;
  }
  c->pair_off.push_back(static_cast<int>(c->pairs.size()));
  // sentinel (in no slab's range): pairs[pa1].goff ends every slab's range
  // of pair_goff, the last slab's included
  PairPlan sentinel = {};
  sentinel.goff = static_cast<int>(c->pair_goff.size());
  c->pairs.push_back(sentinel);
  c->plans_ok = true;
}

// CTAs of the basis kernels: every subdomain's columns in chunks of at most
// nc16 (s = 16, fixed chunks) or nc32 (s = 32, balanced chunks); s = 16
// subdomains first.
static void rebuild_items(mrcm_ctx *c, int nc16, int nc32) {
  c->items.clear();
  std::vector<BasisItem> it32;
  for (size_t g = 0; g < c->sub.size(); ++g) {
    const SubInfo &sb = c->sub[g];
    const int ncol = sb.ncols, gid = static_cast<int>(g);
    // as few CTAs as the width allows, with balanced column counts (no
    // one-column stragglers; each CTA's fixed latency is paid once per item)
    if (sb.s == 16) {
      const int nch = (ncol + nc16 - 1) / nc16;
      for (int k = 0; k < nch; ++k) {
        const int c0 = ncol * k / nch, c1 = ncol * (k + 1) / nch;
        c->items.push_back(BasisItem{gid, c0, c1 - c0});
      }
    } else {
      const int nch = (ncol + nc32 - 1) / nc32;
      for (int k = 0; k < nch; ++k) {
        const int c0 = ncol * k / nch, c1 = ncol * (k + 1) / nch;
        it32.push_back(BasisItem{gid, c0, c1 - c0});
      }
    }
  }
  c->nitems16 = static_cast<int>(c->items.size());
  c->items.insert(c->items.end(), it32.begin(), it32.end());
  c->nc16 = nc16;
  c->nc32 = nc32;
}

// GMRES path: one row descriptor per interface unknown, and the CTA plan of
// the cooperative kernel (each realisation gets CTAs in proportion to its
// unknowns, about 128 rows each, within the co-resident limit cap).
static void build_gmres_rows(mrcm_ctx *c) {
  c->gm_rows.assign(c->nunk, GmRow{});
  for (const IfaceInfo &fi : c->iface) {
    const SubInfo &L = c->sub[fi.L], &R = c->sub[fi.R];
    for (int i = 0; i < fi.nU + fi.nP; ++i) {
      GmRow gr;
      gr.gL = L.g_off + static_cast<int64_t>(fi.rowL + i) * L.ncols + 1;
      gr.gR = R.g_off + static_cast<int64_t>(fi.rowR + i) * R.ncols + 1;
      gr.cL = L.col_off + 1;
      gr.cR = R.col_off + 1;
      gr.nL = L.ncols - 1;
      gr.nR = R.ncols - 1;
      c->gm_rows[fi.unk + i] = gr;
    }
  }
}

// Neighbourhood of interface g: every interface with a subdomain within
// Chebyshev distance 1 of one of g's two subdomains (ascending ids).
static void build_neighbourhoods(mrcm_ctx *c) {
  c->nb_off.assign(1, 0);
  c->nb_list.clear();
  c->nb_max = c->nloc_max = 0;
  std::vector<int> nb;
  for (const IfaceInfo &fi : c->iface) {
    const RealInfo &ri = c->real[fi.r];
    const SubInfo &L = c->sub[fi.L], &R = c->sub[fi.R];
    nb.clear();
    if (ri.quad) {              // no subdomain grid: the interface alone
      const int g = static_cast<int>(&fi - c->iface.data());
      nb.push_back(g);
    } else
    for (int J = std::min(L.J, R.J) - 1; J <= std::max(L.J, R.J) + 1; ++J)
      for (int I = std::min(L.I, R.I) - 1; I <= std::max(L.I, R.I) + 1; ++I) {
        if (I < 0 || J < 0 || I >= ri.Sx || J >= ri.Sy) continue;
        const SubInfo &sb = c->sub[ri.sub0 + J * ri.Sx + I];
        for (int e = 0; e < 4; ++e)
          if (sb.edge_iface[e] >= 0) nb.push_back(sb.edge_iface[e]);
      }
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    int nloc = 0;
    for (int h : nb) nloc += c->iface[h].nU + c->iface[h].nP;
    c->nb_max = std::max(c->nb_max, static_cast<int>(nb.size()));
    c->nloc_max = std::max(c->nloc_max, nloc);
    c->nb_list.insert(c->nb_list.end(), nb.begin(), nb.end());
    c->nb_off.push_back(static_cast<int>(c->nb_list.size()));
  }
  c->m_uniform = c->iface.empty() ? 0 : c->iface[0].nU + c->iface[0].nP;
  for (const IfaceInfo &fi : c->iface)
    if (fi.nU + fi.nP != c->m_uniform) c->m_uniform = 0;
  c->s_uniform = c->real[0].s;
  for (const RealInfo &ri : c->real)
    if (ri.s != c->s_uniform) c->s_uniform = 0;
}

// Neighbourhood lists of the preconditioner: the training-target
// neighbourhoods, or only the interfaces sharing a subdomain with g.
static void build_precond_neighbourhoods(mrcm_ctx *c, bool shared) {
  if (!shared) {
    c->pnb_off = c->nb_off;
    c->pnb_list = c->nb_list;
    c->pnb_max = c->nb_max;
    c->pnloc_max = c->nloc_max;
    return;
  }
  c->pnb_off.assign(1, 0);
  c->pnb_list.clear();
  c->pnb_max = c->pnloc_max = 0;
  std::vector<int> nb;
  for (const IfaceInfo &fi : c->iface) {
    nb.clear();
    for (int side = 0; side < 2; ++side) {
      const SubInfo &sb = c->sub[side ? fi.R : fi.L];
      for (int e = 0; e < 4; ++e) {
        if (sb.edge_iface[e] >= 0) nb.push_back(sb.edge_iface[e]);
        if (sb.edge_iface2[e] >= 0) nb.push_back(sb.edge_iface2[e]);   // quadtree half edges
      }
    }
    std::sort(nb.begin(), nb.end());
    nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    int nloc = 0;
    for (int h : nb) nloc += c->iface[h].nU + c->iface[h].nP;
    c->pnb_max = std::max(c->pnb_max, static_cast<int>(nb.size()));
    c->pnloc_max = std::max(c->pnloc_max, nloc);
    c->pnb_list.insert(c->pnb_list.end(), nb.begin(), nb.end());
    c->pnb_off.push_back(static_cast<int>(c->pnb_list.size()));
  }
}

// Tables of the neighbourhood preconditioner (see GmArgs).  Both relations
// ("a subdomain of h within one subdomain of a subdomain of g", "h and g
// share a subdomain") are symmetric, so the blocks g' with h in N(g') are
// N(h) itself.
static void build_nb_tables(mrcm_ctx *c) {
  const int nif = static_cast<int>(c->iface.size());
  auto msz = [&](int g) { return c->iface[g].nU + c->iface[g].nP; };
  std::vector<int> nb_loc(c->pnb_list.size(), 0);
  c->p_off.assign(nif + 1, 0);
  for (int g = 0; g < nif; ++g) {
    int o = 0;
    for (int j = c->pnb_off[g]; j < c->pnb_off[g + 1]; ++j) {
      nb_loc[j] = o;
      o += msz(c->pnb_list[j]);
    }
    c->p_off[g + 1] = c->p_off[g] + static_cast<int64_t>(o) * msz(g);
  }
  // for every h: the blocks g' holding h, with the P offset of h's first row
  std::vector<std::vector<std::pair<int, int64_t>>> gl(nif);
  for (int g = 0; g < nif; ++g)
    for (int j = c->pnb_off[g]; j < c->pnb_off[g + 1]; ++j)
      gl[c->pnb_list[j]].push_back({g, c->p_off[g] + static_cast<int64_t>(nb_loc[j]) * msz(g)});
  c->gat_off.assign(1, 0);
  c->gat_g.clear();
  c->gat_o.clear();
  for (int h = 0; h < nif; ++h) {
    for (const auto &pr : gl[h]) {
      c->gat_g.push_back(pr.first);
      c->gat_o.push_back(pr.second);
    }
    c->gat_off.push_back(static_cast<int>(c->gat_g.size()));
  }
  // column blocks of the rows of G P: N(h) for every interface h whose
  // unknowns are columns of g's rows (the edge interfaces of g's subdomains)
  c->pb_off.assign(1, 0);
  c->pb_list.clear();
  c->pb_pos.clear();
  c->gw_w.assign(nif, 0);
  c->gw_off.assign(nif + 1, 0);
  std::vector<int> blk;
  for (int g = 0; g < nif; ++g) {
    const IfaceInfo &fi = c->iface[g];
    blk.clear();
    for (int side = 0; side < 2; ++side) {
      const SubInfo &sb = c->sub[side ? fi.R : fi.L];
      for (int e = 0; e < 8; ++e) {
        const int h = e < 4 ? sb.edge_iface[e] : sb.edge_iface2[e - 4];   // quadtree: 2nd halves
        if (h < 0) continue;
        for (int j = c->pnb_off[h]; j < c->pnb_off[h + 1]; ++j) blk.push_back(c->pnb_list[j]);
      }
    }
    std::sort(blk.begin(), blk.end());
    blk.erase(std::unique(blk.begin(), blk.end()), blk.end());
    int w = 0;
    for (int gp : blk) {
      c->pb_list.push_back(gp);
      c->pb_pos.push_back(w);
      w += msz(gp);
    }
    c->pb_off.push_back(static_cast<int>(c->pb_list.size()));
    c->gw_w[g] = w;
    c->gw_off[g + 1] = c->gw_off[g] + static_cast<int64_t>(msz(g)) * w;
  }
}

static bool plan_gmres_blocks(mrcm_ctx *c, int cap) {
  const int R = static_cast<int>(c->real.size());
  if (cap < R) return false;
  std::vector<int64_t> want(R);
  int64_t tot = 0;
  for (int r = 0; r < R; ++r) {
    want[r] = std::max<int64_t>(1, (c->real[r].nunk + 127) / 128);
    tot += want[r];
  }
  std::vector<int> nb(R);
  if (tot <= cap) {
    for (int r = 0; r < R; ++r) nb[r] = static_cast<int>(want[r]);
  } else {
    // scale down, at least one CTA each, never above cap in total
    int64_t used = 0;
    for (int r = 0; r < R; ++r) {
      nb[r] = static_cast<int>(std::max<int64_t>(1, want[r] * (cap - R) / tot));
      used += nb[r];
    }
    for (int r = 0; used < cap && r < R; ++r)
      if (nb[r] < want[r]) {
        ++nb[r];
        ++used;
      }
  }
  c->gm_blocks.clear();
  for (int r = 0; r < R; ++r) {
    const RealInfo &ri = c->real[r];
    const int blk0 = static_cast<int>(c->gm_blocks.size());
    for (int b = 0; b < nb[r]; ++b) {
      GmBlock gb;
      gb.r = r;
      gb.row0 = ri.unk0 + static_cast<int>(static_cast<int64_t>(ri.nunk) * b / nb[r]);
      gb.row1 = ri.unk0 + static_cast<int>(static_cast<int64_t>(ri.nunk) * (b + 1) / nb[r]);
      gb.blk0 = blk0;
      gb.nblk = nb[r];
      c->gm_blocks.push_back(gb);
    }
  }
  c->gm_nblk = static_cast<int>(c->gm_blocks.size());
  return c->gm_nblk <= cap;
}

namespace {
struct Arena {
  size_t off = 0;
  template <typename T>
  size_t take(size_t n) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + n * sizeof(T);
    return o;
  }
};
}  // namespace

extern "C" {

int32_t mrcm_version(void) { return 1; }

const char *mrcm_last_error(const mrcm_ctx *ctx) {
  return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

mrcm_status mrcm_setup(const mrcm_desc *desc, void *cuda_stream, mrcm_ctx **out) {
  if (!out) return fail(nullptr, MRCM_EINVAL, "out is NULL");
  *out = nullptr;
  mrcm_status st = validate(desc);
  if (st != MRCM_OK) return st;
  mrcm_ctx *c = new mrcm_ctx();
  c->d = *desc;
  c->prec = desc->prec;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  st = build_tables(c);
  if (st != MRCM_OK) {
    delete c;
    return st;
  }
  rebuild_items(c, 4, 4);                 // the largest item count any width gives
  c->max_items = static_cast<int64_t>(c->items.size());
  rebuild_items(c, kNC16, kNC32);
  build_plans(c);
  if (c->mmax > kGmMmax) {
    delete c;
    return fail(nullptr, MRCM_EINVAL, "interface size nU + nP = %d above %d", c->mmax, kGmMmax);
  }
  if (c->use_gmres) {
    if (c->mmax > kGmMmax) {
      delete c;
      return fail(nullptr, MRCM_EINVAL, "GMRES path: interface size %d above %d", c->mmax,
                  kGmMmax);
    }
    c->gm_K = desc->gmres_restart > 0 ? desc->gmres_restart : 40;
    c->gm_maxit = desc->gmres_max > 0 ? desc->gmres_max : 5000;
    c->gm_tol = desc->gmres_tol > 0.0 ? desc->gmres_tol : desc->iface_tol;
    c->gm_precond = desc->precond;
    build_gmres_rows(c);
    build_neighbourhoods(c);
    if (c->gm_precond == MRCM_PRECOND_NEIGHBOURHOOD ||
        c->gm_precond == MRCM_PRECOND_NEIGHBOURHOOD_SHARED) {
      build_precond_neighbourhoods(c, c->gm_precond == MRCM_PRECOND_NEIGHBOURHOOD_SHARED);
      if (c->pnb_max > kLpMaxNb || c->pnloc_max > kLpMaxLoc) {
        const int nl = c->pnloc_max;
        delete c;
        return fail(nullptr, MRCM_EINVAL,
                    "neighbourhood preconditioner: neighbourhood of %d unknowns above %d", nl,
                    kLpMaxLoc);
      }
      c->use_nb = true;
      build_nb_tables(c);
    }
  }
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  if (c->use_gmres) {
    const int cap = gmres_max_blocks(c->gm_K, c->dev);
    if (!plan_gmres_blocks(c, cap)) {
      delete c;
      return fail(nullptr, MRCM_EINVAL, "GMRES path: %d realisations exceed the %d co-resident CTAs",
                  d_nreal(c), cap);
    }
  }
  const mrcm_desc &d = c->d;
  const size_t esz = c->prec == MRCM_PREC_FP64 ? sizeof(double) : sizeof(float);
  const int nsub = static_cast<int>(c->sub.size());
  const int nif = static_cast<int>(c->iface.size());
  const int nunk = c->nunk;
  const int nb = 2 * d.nx + 2 * d.ny;
  // interface-function tables for s = 16 (offset 0) and s = 32 (offset 256)
  std::vector<double> fnv, fn32;
  int64_t fn_off32 = 16 * 16;
  if (d.iface_fn) {
    // caller's rows, copied in the order the interfaces took them
    fnv.assign(static_cast<size_t>(c->fn_rows16) * 16, 0.0);
    fn32.assign(static_cast<size_t>(c->fn_rows32) * 32, 0.0);
    int64_t src = 0;
    for (const IfaceInfo &fi : c->iface) {
      const int n = (fi.nU + fi.nP) * fi.s;
      double *dst = (fi.s == 16 ? fnv.data() : fn32.data()) + static_cast<int64_t>(fi.fnU) * fi.s;
      for (int k = 0; k < n; ++k) dst[k] = d.iface_fn[src + k];   // finite (validate)
      src += n;
    }
    fn_off32 = static_cast<int64_t>(c->fn_rows16) * 16;
  } else {
    fn_table(d.basis_family, 16, fnv);
    fn_table(d.basis_family, 32, fn32);
  }
  fnv.insert(fnv.end(), fn32.begin(), fn32.end());
  if (fnv.empty()) fnv.push_back(0.0);
  std::vector<double> alpha(static_cast<size_t>(c->alpha_elems), 1.0);
  if (d.alpha) {
    for (size_t k = 0; k < alpha.size(); ++k) {
      alpha[k] = d.alpha[k];
      if (!(alpha[k] > 0.0) || !std::isfinite(alpha[k])) {
        delete c;
        return fail(nullptr, MRCM_EINVAL, "alpha[%zu] must be positive and finite", k);
      }
    }
  }
  // one arena for tables and workspace
  Arena A;
  const size_t o_sub = A.take<SubInfo>(nsub), o_if = A.take<IfaceInfo>(nif ? nif : 1),
               o_col = A.take<ColInfo>(c->col.size()), o_real = A.take<RealInfo>(c->real.size()),
               o_ui = A.take<int>(nunk ? nunk : 1), o_usp = A.take<int>(nunk ? nunk : 1),
               o_fn = A.take<double>(fnv.size()), o_al = A.take<double>(alpha.size() ? alpha.size() : 1),
               o_bt = A.take<int8_t>(nb), o_bv = A.take<double>(nb),
               o_items = A.take<BasisItem>(c->max_items),
               o_p2u = A.take<int>(c->npos ? c->npos : 1),
               o_pro = A.take<int64_t>(c->pos_real_off.size()),
               o_sif = A.take<int>(c->slab_if.size() ? c->slab_if.size() : 1),
               o_sio = A.take<int>(c->slab_if_off.size()),
               o_pinfo = A.take<int>(c->plan_info.size() + 1),
               o_pcnt = A.take<int>(c->plan_cnt.size() + 1),
               o_pgoff = A.take<int>(c->plan_goff.size() + 1),
               o_pxi = A.take<short>(c->plan_xi.size() + 1),
               o_pfg = A.take<int>(c->plan_fgoff.size() + 1),
               o_ptsc = A.take<int>(c->plan_tsc.size() + 1),
               o_pairs = A.take<PairPlan>(c->pairs.size() + 1),
               o_paoff = A.take<int>(c->pair_off.size() + 1),
               o_pagoff = A.take<int>(c->pair_goff.size() + 1),
               o_sbs = A.take<int>(c->sub_by_size.size()),
               o_coef = A.take<double>(static_cast<size_t>(c->coef_elems)),
               o_W = A.take<char>(static_cast<size_t>(c->w_elems) * esz),
               o_basis = A.take<double>(c->basis_elems), o_G = A.take<double>(c->g_elems ? c->g_elems : 1),
               o_sB = A.take<char>((c->slab_elems ? c->slab_elems : 1) * esz),
               o_sA = A.take<char>((c->slab_elems ? c->slab_elems : 1) * esz),
               o_sC = A.take<char>((c->slab_elems ? c->slab_elems : 1) * esz),
               o_sI = A.take<char>((c->slab_elems && !c->use_big ? c->slab_elems : 1) * esz),
               o_X = A.take<char>((c->xy_elems ? c->xy_elems : 1) * esz),
               o_Y = A.take<char>((c->xy_elems ? c->xy_elems : 1) * esz),
               o_ds = A.take<double>(c->tsc_elems ? c->tsc_elems : 1),
               o_f = A.take<double>(nunk ? nunk : 1), o_x = A.take<double>(nunk ? nunk : 1),
               o_r = A.take<double>(nif ? nif : 1),
               o_vec = A.take<char>((c->npos ? c->npos : 1) * esz),
               o_ps = A.take<double>(nsub), o_gt = A.take<double>(c->gam_elems ? c->gam_elems : 1),
               o_st = A.take<int>(8), o_dst = A.take<double>(2 + 2 * d.n_real),
               o_done = A.take<int>(d.n_real + 1);
  const bool G = c->use_gmres;
  const int64_t Kp = c->gm_K;
  const size_t o_gmrow = A.take<GmRow>(G ? c->gm_rows.size() + 1 : 0),
               o_gmblk = A.take<GmBlock>(G ? c->gm_blocks.size() : 0),
               o_gmGp = A.take<double>(G ? (c->g_elems ? c->g_elems : 1) : 0),
               o_gmPbj = A.take<double>(G ? c->tsc_elems + 1 : 0),
               o_gmPid = A.take<double>(G ? c->tsc_elems + 1 : 0),
               o_gmPus = A.take<double>(G ? c->tsc_elems + 1 : 0),
               o_gmV = A.take<double>(G ? (Kp + 1) * (nunk + 1) : 0),
               o_gmW = A.take<double>(G ? nunk + 1 : 0), o_gmY = A.take<double>(G ? nunk + 1 : 0),
               o_gmpart = A.take<double>(G ? static_cast<int64_t>(c->gm_nblk) * (Kp + 2) : 0),
               o_gmres = A.take<double>(G ? d.n_real : 0),
               o_gmint = A.take<int>(G ? 3 * d.n_real : 0),
               o_nboff = A.take<int>(G ? c->nb_off.size() : 0),
               o_nblist = A.take<int>(G ? c->nb_list.size() + 1 : 0);
  const bool NB = G && c->use_nb;
  const size_t o_pnboff = A.take<int>(NB ? c->pnb_off.size() : 0),
               o_pnblist = A.take<int>(NB ? c->pnb_list.size() + 1 : 0);
  const size_t o_nbP = A.take<double>(NB ? c->p_off.back() + 1 : 0),
               o_nbGw = A.take<double>(NB ? c->gw_off.back() + 1 : 0),
               o_poff = A.take<int64_t>(NB ? c->p_off.size() : 0),
               o_gwoff = A.take<int64_t>(NB ? c->gw_off.size() : 0),
               o_gww = A.take<int>(NB ? c->gw_w.size() : 0),
               o_pboff = A.take<int>(NB ? c->pb_off.size() : 0),
               o_pblist = A.take<int>(NB ? c->pb_list.size() + 1 : 0),
               o_pbpos = A.take<int>(NB ? c->pb_pos.size() + 1 : 0),
               o_gatoff = A.take<int>(NB ? c->gat_off.size() : 0),
               o_gatg = A.take<int>(NB ? c->gat_g.size() + 1 : 0),
               o_gato = A.take<int64_t>(NB ? c->gat_o.size() + 1 : 0);
  // big-slab direct path: second slab vector, inverse scratch, job lists
  const bool BG = c->use_big;
  const int bigK = c->real.empty() ? 1 : c->real[0].nslab;
  const int bigLev = static_cast<int>(c->big_lev_off.size()) - 1;
  int64_t n_inv = 0, n_gemm = 0, inv_slots = 0;
  if (BG) {
    for (int lev = 0, st = 1; lev < bigLev; ++lev, st <<= 1) {
      const int nel = (bigK - st + 2 * st - 1) / (2 * st), nsv = (bigK + 2 * st - 1) / (2 * st);
      n_inv += static_cast<int64_t>(nel) * d.n_real;
      inv_slots = std::max<int64_t>(inv_slots, static_cast<int64_t>(nel) * d.n_real);
      n_gemm += static_cast<int64_t>(5) * nsv * d.n_real;
    }
    n_inv += d.n_real;                                   // the roots
    inv_slots = std::max<int64_t>(inv_slots, d.n_real);
  }
  const int64_t slot_elems = 64 * 64 + static_cast<int64_t>(c->bmax_max) * 64;
  // tensor-core products (FP32 path): 4 tensor maps (128 bytes each) per job,
  // on the raw slab blocks
  const bool TC = BG && c->prec != MRCM_PREC_FP64 && !getenv("MRCM_NO_TENSOR_CORES");
  const size_t o_tcm = A.take<char>(TC ? n_gemm * 4 * 128 : 0);
  const size_t o_vec2 = A.take<char>(BG ? (c->npos ? c->npos : 1) * esz : 0),
               o_iscr = A.take<char>(BG ? inv_slots * slot_elems * esz : 0),
               o_ijob = A.take<InvJob>(BG ? n_inv : 0), o_gjob = A.take<GemmJob>(BG ? n_gemm : 0),
               o_levo = A.take<int>(BG ? c->big_lev_off.size() : 0);
  // refinement-stall recovery (mixed path): FP64 blocks, SubInfo copies and
  // work items of rec_cap subdomains, the list and the per-subdomain marks
  int max_ncols = 1;
  for (const SubInfo &sb : c->sub) max_ncols = std::max(max_ncols, sb.ncols);
  c->rec_cap = (c->prec == MRCM_PREC_FP32_IR && d.ir_recover >= 0)
                   ? std::min(d.ir_recover > 0 ? d.ir_recover : 16, nsub)
                   : 0;
  c->rec_maxch = (max_ncols + kRecNC - 1) / kRecNC;
  const int RC = c->rec_cap;
  const size_t o_rW = A.take<double>(static_cast<int64_t>(RC) * c->smax * c->smax * c->smax),
               o_rsub = A.take<SubInfo>(RC),
               o_ritems = A.take<BasisItem>(static_cast<int64_t>(2) * RC * c->rec_maxch),
               o_rlist = A.take<int>(RC), o_rmark = A.take<int>(RC > 0 ? nsub : 0);
  e = cudaMalloc(&c->arena, A.off);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, MRCM_ENOMEM, "cudaMalloc(%zu bytes): %s", A.off, cudaGetErrorString(e));
  }
  char *base = static_cast<char *>(c->arena);
  // MRCM_DEBUG_POISON: fill the floating-point workspace with 0xFF bytes (NaN
  // in FP32 and FP64) before anything is written.  Every value a step reads
  // must come from an earlier step or from the setup, so results stay the same
  // bit for bit; a read of an unwritten value turns up as a NaN.  "1" fills
  // every buffer below; "0x<mask>" fills buffer i when bit i is set (to find
  // the one at fault).  Integer tables are left alone.
  if (const char *pv = getenv("MRCM_DEBUG_POISON"); pv && pv[0]) {
    const uint64_t mask = (pv[0] == '0' && pv[1] == 'x') ? strtoull(pv, nullptr, 16)
                          : pv[0] == '1'                 ? ~uint64_t(0)
                                                         : 0;
    const size_t cut[] = {o_coef, o_W,      o_basis,  o_G,      o_sB,   o_sA,    o_sC,
                          o_sI,   o_X,      o_Y,      o_ds,     o_f,    o_x,     o_r,
                          o_vec,  o_ps,     o_gt,     o_st,     o_gmGp, o_gmPbj, o_gmPid,
                          o_gmPus, o_gmV,   o_gmW,    o_gmY,    o_gmpart, o_gmres, o_gmint,
                          o_tcm,  o_vec2,   o_iscr,   o_ijob,   o_rW,     o_rsub};
    // spans [cut[k], cut[k+1]) hold floating-point data except those that
    // start at o_st, o_gmint, o_tcm and o_ijob (entries 17, 27, 28 and 31);
    // bit i names the i-th floating-point span: 0 coef .. 16 gt, 17 gmGp ..
    // 25 gmres, 26 vec2, 27 iscr, 28 the recovery's FP64 blocks
    int bit = 0;
    for (size_t k = 0; k + 1 < sizeof(cut) / sizeof(cut[0]); ++k) {
      if (k == 17 || k == 27 || k == 28 || k == 31) continue;
      const size_t a = cut[k], b = cut[k + 1];
      if (((mask >> bit++) & 1) && b > a &&
          (e = cudaMemset(base + a, 0xFF, b - a)) != cudaSuccess) {
        cudaFree(c->arena);
        delete c;
        return cuda_fail(nullptr, e, "mrcm_setup poison fill");
      }
    }
  }
  auto up = [&](size_t off, const void *src, size_t bytes) {
    if (!bytes) return cudaSuccess;
    return cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice);
  };
  // tables
  if ((e = up(o_sub, c->sub.data(), nsub * sizeof(SubInfo))) != cudaSuccess ||
      (e = up(o_if, c->iface.data(), nif * sizeof(IfaceInfo))) != cudaSuccess ||
      (e = up(o_col, c->col.data(), c->col.size() * sizeof(ColInfo))) != cudaSuccess ||
      (e = up(o_real, c->real.data(), c->real.size() * sizeof(RealInfo))) != cudaSuccess ||
      (e = up(o_ui, c->unk_iface.data(), nunk * sizeof(int))) != cudaSuccess ||
      (e = up(o_usp, c->unk_slabpos.data(), nunk * sizeof(int))) != cudaSuccess ||
      (e = up(o_fn, fnv.data(), fnv.size() * sizeof(double))) != cudaSuccess ||
      (e = up(o_al, alpha.data(), alpha.size() * sizeof(double))) != cudaSuccess ||
      (e = up(o_bt, d.bc_type, nb * sizeof(int8_t))) != cudaSuccess ||
      (e = up(o_bv, d.bc_val, nb * sizeof(double))) != cudaSuccess ||
      (e = up(o_items, c->items.data(), c->items.size() * sizeof(BasisItem))) != cudaSuccess ||
      (e = up(o_sbs, c->sub_by_size.data(), c->sub_by_size.size() * sizeof(int))) !=
          cudaSuccess ||
      (e = up(o_p2u, c->pos2unk.data(), c->npos * sizeof(int))) != cudaSuccess ||
      (e = up(o_pro, c->pos_real_off.data(), c->pos_real_off.size() * sizeof(int64_t))) !=
          cudaSuccess ||
      (e = up(o_sif, c->slab_if.data(), c->slab_if.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_sio, c->slab_if_off.data(), c->slab_if_off.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pinfo, c->plan_info.data(), c->plan_info.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pcnt, c->plan_cnt.data(), c->plan_cnt.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pgoff, c->plan_goff.data(), c->plan_goff.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pxi, c->plan_xi.data(), c->plan_xi.size() * sizeof(short))) != cudaSuccess ||
      (e = up(o_pfg, c->plan_fgoff.data(), c->plan_fgoff.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_ptsc, c->plan_tsc.data(), c->plan_tsc.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pairs, c->pairs.data(), c->pairs.size() * sizeof(PairPlan))) != cudaSuccess ||
      (e = up(o_paoff, c->pair_off.data(), c->pair_off.size() * sizeof(int))) != cudaSuccess ||
      (e = up(o_pagoff, c->pair_goff.data(), c->pair_goff.size() * sizeof(int))) != cudaSuccess ||
      (G && (e = up(o_gmrow, c->gm_rows.data(), c->gm_rows.size() * sizeof(GmRow))) !=
                cudaSuccess) ||
      (G && (e = up(o_gmblk, c->gm_blocks.data(), c->gm_blocks.size() * sizeof(GmBlock))) !=
                cudaSuccess) ||
      (G && (e = up(o_nboff, c->nb_off.data(), c->nb_off.size() * sizeof(int))) != cudaSuccess) ||
      (NB && (e = up(o_pnboff, c->pnb_off.data(), c->pnb_off.size() * sizeof(int))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_pnblist, c->pnb_list.data(), c->pnb_list.size() * sizeof(int))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_poff, c->p_off.data(), c->p_off.size() * sizeof(int64_t))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_gwoff, c->gw_off.data(), c->gw_off.size() * sizeof(int64_t))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_gww, c->gw_w.data(), c->gw_w.size() * sizeof(int))) != cudaSuccess) ||
      (NB && (e = up(o_pboff, c->pb_off.data(), c->pb_off.size() * sizeof(int))) != cudaSuccess) ||
      (NB && (e = up(o_pblist, c->pb_list.data(), c->pb_list.size() * sizeof(int))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_pbpos, c->pb_pos.data(), c->pb_pos.size() * sizeof(int))) != cudaSuccess) ||
      (NB && (e = up(o_gatoff, c->gat_off.data(), c->gat_off.size() * sizeof(int))) !=
                 cudaSuccess) ||
      (NB && (e = up(o_gatg, c->gat_g.data(), c->gat_g.size() * sizeof(int))) != cudaSuccess) ||
      (NB && (e = up(o_gato, c->gat_o.data(), c->gat_o.size() * sizeof(int64_t))) !=
                 cudaSuccess) ||
      (G && (e = up(o_nblist, c->nb_list.data(), c->nb_list.size() * sizeof(int))) !=
                cudaSuccess) ||
      (e = cudaMemset(base + o_st, 0, 8 * sizeof(int))) != cudaSuccess ||
      (RC > 0 && (e = cudaMemset(base + o_rmark, 0, nsub * sizeof(int))) != cudaSuccess) ||
      (e = cudaMemset(base + o_dst, 0, (2 + 2 * d.n_real) * sizeof(double))) != cudaSuccess ||
      // slab vectors: positions past a slab's own width pad it to the widest
      // slab of its realisation; no kernel writes them and the block solves
      // multiply them by the zero padding of the slab blocks, so they start
      // (and stay) zero
      (e = cudaMemset(base + o_vec, 0, (c->npos ? c->npos : 1) * esz)) != cudaSuccess) {
    cudaFree(c->arena);
    delete c;
    return cuda_fail(nullptr, e, "mrcm_setup upload");
  }
  DeviceTables &t = c->t;
  t.nx = d.nx;
  t.ny = d.ny;
  t.n_real = d.n_real;
  t.nsub = nsub;
  t.niface = nif;
  t.nunk = nunk;
  t.pure_neumann = d.pure_neumann ? 1 : 0;
  t.smax = c->smax;
  t.h = d.ly / d.ny;
  t.inv_h = d.ny / d.ly;
  t.sub_by_size = reinterpret_cast<const int *>(base + o_sbs);
  t.nsub16 = c->nsub16;
  {
    // FP32, few 16 x 16 subdomains (at most two per SM): a separate factor
    // launch would leave most SMs idle behind one pivot chain per subdomain,
    // so each basis CTA factors its subdomain itself; with more subdomains
    // the separate, throughput-bound factor is cheaper than the repeated
    // chains (one per column chunk)
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->dev);
    t.fuse16 = (c->prec == MRCM_PREC_FP32_IR && c->nsub16 > 0 && c->nsub16 <= 2 * nsm) ? 1 : 0;
  }
  t.sub = reinterpret_cast<const SubInfo *>(base + o_sub);
  t.iface = reinterpret_cast<const IfaceInfo *>(base + o_if);
  t.col = reinterpret_cast<const ColInfo *>(base + o_col);
  t.real = reinterpret_cast<const RealInfo *>(base + o_real);
  t.unk_iface = reinterpret_cast<const int *>(base + o_ui);
  t.unk_slabpos = reinterpret_cast<const int *>(base + o_usp);
  t.fnval = reinterpret_cast<const double *>(base + o_fn);
  t.fn_off32 = fn_off32;
  t.alpha = reinterpret_cast<const double *>(base + o_al);
  t.bc_type = reinterpret_cast<const int8_t *>(base + o_bt);
  t.bc_val = reinterpret_cast<const double *>(base + o_bv);
  c->d_items = reinterpret_cast<BasisItem *>(base + o_items);
  c->d_pos2unk = reinterpret_cast<int *>(base + o_p2u);
  c->d_pos_real_off = reinterpret_cast<int64_t *>(base + o_pro);
  c->d_slab_if = reinterpret_cast<int *>(base + o_sif);
  c->d_slab_if_off = reinterpret_cast<int *>(base + o_sio);
  t.pos2unk = c->d_pos2unk;
  t.mmax = c->mmax;
  t.emax = c->emax;
  t.plan_info = reinterpret_cast<const int *>(base + o_pinfo);
  t.plan_cnt = reinterpret_cast<const int *>(base + o_pcnt);
  t.plan_goff = reinterpret_cast<const int *>(base + o_pgoff);
  t.plan_xi = reinterpret_cast<const short *>(base + o_pxi);
  t.plan_fgoff = reinterpret_cast<const int *>(base + o_pfg);
  t.plan_tsc = reinterpret_cast<const int *>(base + o_ptsc);
  t.pairs = reinterpret_cast<const PairPlan *>(base + o_pairs);
  t.pair_off = reinterpret_cast<const int *>(base + o_paoff);
  t.pair_goff = reinterpret_cast<const int *>(base + o_pagoff);
  Workspace &w = c->w;
  w.coef = reinterpret_cast<double *>(base + o_coef);
  w.W = base + o_W;
  w.basis = reinterpret_cast<double *>(base + o_basis);
  w.G = reinterpret_cast<double *>(base + o_G);
  w.slabB = base + o_sB;
  w.slabA = base + o_sA;
  w.slabC = base + o_sC;
  w.slabI = base + o_sI;
  w.X = base + o_X;
  w.Y = base + o_Y;
  w.tsc = reinterpret_cast<double *>(base + o_ds);
  w.f = reinterpret_cast<double *>(base + o_f);
  w.x = reinterpret_cast<double *>(base + o_x);
  w.r = reinterpret_cast<double *>(base + o_r);
  w.vec = base + o_vec;
  w.psum = reinterpret_cast<double *>(base + o_ps);
  w.gamma_tmp = reinterpret_cast<double *>(base + o_gt);
  w.status = reinterpret_cast<int *>(base + o_st);
  w.dstat = reinterpret_cast<double *>(base + o_dst);
  w.ifnorm = nullptr;
  w.done = reinterpret_cast<int *>(base + o_done);
  w.rec_cap = RC;
  w.rec_maxch = c->rec_maxch;
  w.rec_smax = c->smax;
  w.W64 = RC > 0 ? reinterpret_cast<double *>(base + o_rW) : nullptr;
  w.rec_sub = RC > 0 ? reinterpret_cast<SubInfo *>(base + o_rsub) : nullptr;
  w.rec_items = RC > 0 ? reinterpret_cast<BasisItem *>(base + o_ritems) : nullptr;
  w.stall_list = RC > 0 ? reinterpret_cast<int *>(base + o_rlist) : nullptr;
  w.stall_mark = RC > 0 ? reinterpret_cast<int *>(base + o_rmark) : nullptr;
  if (G) {
    GmArgs &a = c->gm;
    a.row = reinterpret_cast<const GmRow *>(base + o_gmrow);
    a.blk = reinterpret_cast<const GmBlock *>(base + o_gmblk);
    a.Gp = reinterpret_cast<double *>(base + o_gmGp);
    c->gm_Pbj = reinterpret_cast<double *>(base + o_gmPbj);
    c->gm_Pid = reinterpret_cast<double *>(base + o_gmPid);
    c->gm_Puser = reinterpret_cast<double *>(base + o_gmPus);
    a.V = reinterpret_cast<double *>(base + o_gmV);
    a.Wv = reinterpret_cast<double *>(base + o_gmW);
    a.Y = reinterpret_cast<double *>(base + o_gmY);
    a.part = reinterpret_cast<double *>(base + o_gmpart);
    a.resid = reinterpret_cast<double *>(base + o_gmres);
    a.done = reinterpret_cast<int *>(base + o_gmint);
    a.fallback = a.done + d.n_real;
    a.iters = a.fallback + d.n_real;
    c->d_nb_off = reinterpret_cast<int *>(base + o_nboff);
    c->d_nb_list = reinterpret_cast<int *>(base + o_nblist);
    a.nb = 0;
    if (NB) {
      c->d_pnb_off = reinterpret_cast<int *>(base + o_pnboff);
      c->d_pnb_list = reinterpret_cast<int *>(base + o_pnblist);
      a.Pnb = reinterpret_cast<double *>(base + o_nbP);
      a.Gw = reinterpret_cast<double *>(base + o_nbGw);
      a.p_off = reinterpret_cast<const int64_t *>(base + o_poff);
      a.gw_off = reinterpret_cast<const int64_t *>(base + o_gwoff);
      a.gw_w = reinterpret_cast<const int *>(base + o_gww);
      a.pb_off = reinterpret_cast<const int *>(base + o_pboff);
      a.pb_list = reinterpret_cast<const int *>(base + o_pblist);
      a.pb_pos = reinterpret_cast<const int *>(base + o_pbpos);
      a.gat_off = reinterpret_cast<const int *>(base + o_gatoff);
      a.gat_g = reinterpret_cast<const int *>(base + o_gatg);
      a.gat_o = reinterpret_cast<const int64_t *>(base + o_gato);
    }
    a.K = c->gm_K;
    a.maxit = c->gm_maxit;
    a.tol = c->gm_tol;
    // identity blocks (no preconditioner)
    std::vector<double> id(c->tsc_elems + 1, 0.0);
    for (const IfaceInfo &fi : c->iface) {
      const int m = fi.nU + fi.nP;
      for (int k = 0; k < m; ++k) id[fi.tsc_off + k * m + k] = 1.0;
    }
    if ((e = cudaMemcpy(c->gm_Pid, id.data(), id.size() * sizeof(double),
                        cudaMemcpyHostToDevice)) != cudaSuccess) {
      cudaFree(c->arena);
      delete c;
      return cuda_fail(nullptr, e, "mrcm_setup upload");
    }
  }
  if (BG) {
    // jobs: level by level, the eliminated slabs' inverses (in place in the
    // B blocks), then for the survivors X = A_k I_l, Y = C_k I_r and
    // B_k -= X C_l + Y A_r, A_k = -X A_l, C_k = -Y C_r; the roots last
    BigPlan &bp = c->bp;
    bp.K = bigK;
    bp.nlev = bigLev;
    bp.bmax = c->bmax_max;
    bp.tensor_cores = TC ? 1 : 0;
    bp.tc_maps = base + o_tcm;
    const size_t es = esz;
    char *sB = static_cast<char *>(w.slabB), *sA = static_cast<char *>(w.slabA),
         *sC = static_cast<char *>(w.slabC), *sX = static_cast<char *>(w.X),
         *sY = static_cast<char *>(w.Y);
    char *iscr = base + o_iscr;
    auto blk = [&](char *b0, const RealInfo &ri, int k) {
      return static_cast<void *>(b0 + (ri.slab_off + static_cast<int64_t>(k) * ri.bmax * ri.bmax) * es);
    };
    auto xy = [&](char *b0, const RealInfo &ri, int lev, int ki) {
      return static_cast<void *>(b0 + (ri.xy_off + (static_cast<int64_t>(c->big_lev_off[lev]) + ki) *
                                                       ri.bmax * ri.bmax) * es);
    };
    c->big_inv.clear();
    c->big_gemm.clear();
    for (int lev = 0, st = 1; lev <= bigLev; ++lev, st <<= 1) {
      bp.inv_off[lev] = static_cast<int>(c->big_inv.size());
      int slot = 0;
      for (const RealInfo &ri : c->real) {
        if (lev == bigLev) {
          c->big_inv.push_back(InvJob{blk(sB, ri, 0), iscr + slot * slot_elems * es,
                                      iscr + (slot * slot_elems + 4096) * es, ri.bmax, 0});
          ++slot;
          continue;
        }
        for (int k = st; k < bigK; k += 2 * st, ++slot)
          c->big_inv.push_back(InvJob{blk(sB, ri, k), iscr + slot * slot_elems * es,
                                      iscr + (slot * slot_elems + 4096) * es, ri.bmax, 0});
      }
      if (lev == bigLev) break;
      for (int set = 0; set < 2; ++set) {
        bp.gemm_off[2 * lev + set] = static_cast<int>(c->big_gemm.size());
        for (const RealInfo &ri : c->real)
          for (int k = 0, ki = 0; k < bigK; k += 2 * st, ++ki) {
            const bool hl = k - st >= 0, hr = k + st < bigK;
            void *X = xy(sX, ri, lev, ki), *Y = xy(sY, ri, lev, ki);
            if (set == 0) {
              if (hl) c->big_gemm.push_back(GemmJob{blk(sA, ri, k), blk(sB, ri, k - st), nullptr,
                                                    nullptr, X, ri.bmax, 0, 1.0});
              if (hr) c->big_gemm.push_back(GemmJob{blk(sC, ri, k), blk(sB, ri, k + st), nullptr,
                                                    nullptr, Y, ri.bmax, 0, 1.0});
            } else {
              if (hl || hr)
                c->big_gemm.push_back(GemmJob{hl ? X : nullptr, hl ? blk(sC, ri, k - st) : nullptr,
                                              hr ? Y : nullptr, hr ? blk(sA, ri, k + st) : nullptr,
                                              blk(sB, ri, k), ri.bmax, 1, -1.0});
              if (hl) c->big_gemm.push_back(GemmJob{X, blk(sA, ri, k - st), nullptr, nullptr,
                                                    blk(sA, ri, k), ri.bmax, 0, -1.0});
              if (hr) c->big_gemm.push_back(GemmJob{Y, blk(sC, ri, k + st), nullptr, nullptr,
                                                    blk(sC, ri, k), ri.bmax, 0, -1.0});
            }
          }
        bp.gemm_off[2 * lev + set + 1] = static_cast<int>(c->big_gemm.size());
      }
    }
    bp.inv_off[bigLev + 1] = static_cast<int>(c->big_inv.size());
    std::vector<char> maps;
    bool maps_ok = true;
    if (TC) {
      maps.assign(c->big_gemm.size() * 4 * 128, 0);
      for (size_t j = 0; j < c->big_gemm.size(); ++j)
        maps_ok = maps_ok && tc_encode_raw_maps(c->big_gemm[j], maps.data() + j * 4 * 128);
    }
    bp.inv = reinterpret_cast<const InvJob *>(base + o_ijob);
    bp.gemm = reinterpret_cast<const GemmJob *>(base + o_gjob);
    bp.lev_off = reinterpret_cast<const int *>(base + o_levo);
    bp.vec2 = base + o_vec2;
    if (static_cast<int64_t>(c->big_inv.size()) > n_inv ||
        static_cast<int64_t>(c->big_gemm.size()) > n_gemm ||
        (e = up(o_ijob, c->big_inv.data(), c->big_inv.size() * sizeof(InvJob))) != cudaSuccess ||
        (e = up(o_gjob, c->big_gemm.data(), c->big_gemm.size() * sizeof(GemmJob))) != cudaSuccess ||
        (e = up(o_levo, c->big_lev_off.data(), c->big_lev_off.size() * sizeof(int))) !=
            cudaSuccess ||
        !maps_ok || (TC && (e = up(o_tcm, maps.data(), maps.size())) != cudaSuccess)) {
      cudaFree(c->arena);
      delete c;
      return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidValue : e, "big-slab plan");
    }
  }
  int bmax = 1;
  for (const RealInfo &ri : c->real) bmax = ri.bmax > bmax ? ri.bmax : bmax;
  if ((e = init_local_attributes()) != cudaSuccess || (e = init_big_attributes()) != cudaSuccess ||
      (e = init_tc_attributes()) != cudaSuccess ||
      (e = init_iface_attributes(c->prec, bmax, c->use_gmres || BG ? 0 : c->max_vec)) !=
          cudaSuccess) {
    cudaFree(c->arena);
    delete c;
    return cuda_fail(nullptr, e, "kernel attributes");
  }
  c->solve_grid = c->use_gmres || BG ? 0 : iface_solve_grid(c->prec, c->dev, c->max_vec);
  if (BG) c->big_grid = big_solve_grid(c->prec, c->dev);
  if (nunk > 0 && c->plans_ok && !c->use_gmres && !getenv("MRCM_NO_CLUSTER")) {
    // largest staging footprint of a slab's pair plans and pair blocks
    size_t stage_max = 0;
    for (size_t sl = 0; sl + 1 < c->pair_off.size(); ++sl) {
      const int pa0 = c->pair_off[sl], pa1 = c->pair_off[sl + 1];
      const size_t ppb = (static_cast<size_t>(pa1 - pa0) * sizeof(PairPlan) + 15) & ~static_cast<size_t>(15);
      const size_t nst = static_cast<size_t>(c->pairs[pa1].goff - c->pairs[pa0].goff) / 2;
      stage_max = std::max(stage_max, ppb + nst * sizeof(double));
    }
    c->cluster_k = iface_cluster_plan(c->prec, c->nslab_max, c->bmax_max, c->nlev_max, c->mmax,
                                      t.emax, stage_max, c->dev);
  }
  if (nunk > 0 && BG && c->big_grid < 1) {
    cudaFree(c->arena);
    delete c;
    return fail(nullptr, MRCM_ECUDA, "no co-resident grid for the interface solve");
  }
  if (nunk > 0 && !c->use_gmres && !BG && (c->solve_grid < 1 || d.n_real > c->solve_grid)) {
    cudaFree(c->arena);
    delete c;
    return fail(nullptr, MRCM_EINVAL,
                "n_real %d exceeds the %d co-resident interface solvers", d.n_real,
                c->solve_grid);
  }
  *out = c;
  return MRCM_OK;
}

void mrcm_destroy(mrcm_ctx *ctx) {
  if (!ctx) return;
  if (ctx->arena) cudaFree(ctx->arena);
  delete ctx;
}

mrcm_status mrcm_set_stream(mrcm_ctx *ctx, void *cuda_stream) {
  if (!ctx) return MRCM_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return MRCM_OK;
}

mrcm_status mrcm_factor_local(mrcm_ctx *ctx, const double *d_K, const double *d_lambda) {
  if (!ctx) return MRCM_EINVAL;
  if (!d_K || !d_lambda) return fail(ctx, MRCM_EINVAL, "K and lambda must be device pointers");
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->w.status, 0, 8 * sizeof(int), ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset status");
  if ((e = cudaMemsetAsync(ctx->w.dstat, 0, (2 + 2 * ctx->d.n_real) * sizeof(double),
                           ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset status");
  e = launch_factor(ctx->t, ctx->w, ctx->prec, d_K, d_lambda, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "factor_local launch");
  ctx->launches = n_sizes(ctx);
  ctx->state = 1;
  return MRCM_OK;
}

mrcm_status mrcm_build_basis(mrcm_ctx *ctx, const double *d_q) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->state < 1) return fail(ctx, MRCM_EINVAL, "build_basis before factor_local");
  if (!d_q) return fail(ctx, MRCM_EINVAL, "q must be a device pointer");
  cudaError_t e = launch_basis(ctx->t, ctx->w, ctx->prec, ctx->d_items, ctx->nitems16,
                               static_cast<int>(ctx->items.size()) - ctx->nitems16, ctx->nc16,
                               ctx->nc32, d_q, ctx->d.ir_tol, ctx->d.ir_max, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "build_basis launch");
  ctx->launches += n_sizes(ctx);
  if (ctx->d.pure_neumann) {
    if ((e = launch_compat(ctx->t, ctx->w, d_q, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "build_basis compatibility check");
    ctx->launches += 1;
  }
  if (ctx->rec_cap > 0) {
    if ((e = launch_recover(ctx->t, ctx->w, d_q, ctx->d.ir_tol, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "build_basis recovery launch");
    ctx->launches += 1 + n_sizes(ctx);
  }
  ctx->state = 2;
  return MRCM_OK;
}

static mrcm_status read_info(mrcm_ctx *ctx, mrcm_info *info) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  int st[8];
  double ds[2];
  if ((e = cudaMemcpy(st, ctx->w.status, sizeof st, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(ds, ctx->w.dstat, sizeof ds, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(ctx, e, "status read");
  info->flags = st[0];
  info->local_sweeps_max = st[1];
  info->iface_sweeps = st[2];
  info->gmres_iters = st[3];
  info->local_resid_max = ds[0];
  info->iface_resid = ds[1];
  info->local_refactored = std::min(st[4], ctx->rec_cap);
  if (st[0] & MRCM_FLAG_TIMEOUT) return fail(ctx, MRCM_ETIMEOUT, "a bounded device wait ran out");
  if (st[0] & MRCM_FLAG_LAYOUT) return fail(ctx, MRCM_EINVAL, "internal slab layout error");
  if (st[0] & MRCM_FLAG_NAN) return fail(ctx, MRCM_ENAN, "NaN/Inf or non-positive kappa");
  // the earliest step's failure first: a stalled local solve or unbalanced
  // pure-Neumann data spoil the interface system that the later flags judge
  if (st[0] & MRCM_FLAG_NOTSPD) return fail(ctx, MRCM_ENOTSPD, "local pivot <= 0");
  if (st[0] & MRCM_FLAG_INCOMPATIBLE)
    return fail(ctx, MRCM_EINCOMPAT,
                "pure Neumann: the sources do not balance the boundary outflow");
  if (st[0] & MRCM_FLAG_LOCAL_STALL)
    return fail(ctx, MRCM_EIRSTALL, "local refinement stopped at %.3e", ds[0]);
  if (st[0] & MRCM_FLAG_IFACE_PIVOT)
    return fail(ctx, MRCM_ENOTSPD, "interface pivot zero or not finite");
  if (st[0] & MRCM_FLAG_IFACE_STALL)
    return fail(ctx, MRCM_ENOCONV, "interface refinement stopped at %.3e", ds[1]);
  return MRCM_OK;
}

// GMRES path of step (d): preconditioner blocks, G' = G P, the cooperative
// solve; with caller-supplied blocks a second, gated pass reruns the
// stalled realisations with block-Jacobi.
static mrcm_status solve_gmres(mrcm_ctx *ctx) {
  const int R = ctx->d.n_real;
  cudaStream_t st = ctx->stream;
  GmArgs a = ctx->gm;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.done, 0, sizeof(int) * 3 * R, st)) != cudaSuccess)
    return cuda_fail(ctx, e, "reset");
  const int pc = ctx->gm_precond;
  if (pc == MRCM_PRECOND_USER && !ctx->gm_user_set)
    return fail(ctx, MRCM_EINVAL, "precond = MRCM_PRECOND_USER but no blocks were set");
  if (pc == MRCM_PRECOND_NEIGHBOURHOOD || pc == MRCM_PRECOND_NEIGHBOURHOOD_SHARED) {
    a.nb = 1;
    a.stall = 0;
    a.gate = 0;
    if ((e = launch_gmres_nb(ctx->t, ctx->w, a, ctx->d_pnb_off, ctx->d_pnb_list, ctx->pnloc_max,
                             ctx->mmax, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "neighbourhood preconditioner launch");
    ctx->launches += 2;
    if ((e = launch_gmres(ctx->t, ctx->w, a, ctx->gm_nblk, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "GMRES launch");
    ctx->launches += 1;
    return MRCM_OK;
  }
  a.P = pc == MRCM_PRECOND_BLOCK_JACOBI ? ctx->gm_Pbj
        : pc == MRCM_PRECOND_USER       ? ctx->gm_Puser
                                        : ctx->gm_Pid;
  a.stall = pc == MRCM_PRECOND_USER ? 1 : 0;
  a.gate = 0;
  if ((e = launch_gmres_precond(ctx->t, ctx->w, a, ctx->gm_Pbj, pc == MRCM_PRECOND_BLOCK_JACOBI,
                                st)) != cudaSuccess)
    return cuda_fail(ctx, e, "GMRES preconditioner launch");
  ctx->launches += pc == MRCM_PRECOND_BLOCK_JACOBI ? 2 : 1;
  if ((e = launch_gmres(ctx->t, ctx->w, a, ctx->gm_nblk, st)) != cudaSuccess)
    return cuda_fail(ctx, e, "GMRES launch");
  ctx->launches += 1;
  if (pc == MRCM_PRECOND_USER) {
    if ((e = cudaMemsetAsync(a.done, 0, sizeof(int) * R, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "reset");
    a.P = ctx->gm_Pbj;
    a.stall = 0;
    a.gate = 1;
    if ((e = launch_gmres_precond(ctx->t, ctx->w, a, ctx->gm_Pbj, true, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "GMRES preconditioner launch");
    if ((e = launch_gmres(ctx->t, ctx->w, a, ctx->gm_nblk, st)) != cudaSuccess)
      return cuda_fail(ctx, e, "GMRES launch");
    ctx->launches += 3;
  }
  return MRCM_OK;
}

mrcm_status mrcm_solve_interface(mrcm_ctx *ctx, mrcm_info *info) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->state < 2) return fail(ctx, MRCM_EINVAL, "solve_interface before build_basis");
  if (ctx->nunk > 0 && ctx->use_gmres) {
    mrcm_status gs = solve_gmres(ctx);
    if (gs != MRCM_OK) return gs;
  } else if (ctx->nunk > 0 && ctx->use_big) {
    cudaError_t e = launch_iface_assemble(ctx->t, ctx->w, ctx->prec, ctx->slab_elems,
                                          ctx->d_pos2unk, ctx->npos, ctx->d_pos_real_off,
                                          ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "interface assembly launch");
    ctx->launches += 3;
    int nl = 0;
    if ((e = launch_big_factor(ctx->bp, ctx->prec, ctx->w.status, &nl, ctx->stream)) !=
        cudaSuccess)
      return cuda_fail(ctx, e, "interface factor launch");
    ctx->launches += nl;
    if ((e = launch_big_solve(ctx->t, ctx->w, ctx->bp, ctx->prec, ctx->d.iface_tol,
                              1 + ctx->d.iface_ir_max, ctx->big_grid, ctx->stream)) != cudaSuccess)
      return cuda_fail(ctx, e, "interface solve launch");
    ctx->launches += 1;
  } else if (ctx->nunk > 0 && ctx->cluster_k > 0) {
    cudaError_t e = launch_iface_cluster(ctx->t, ctx->w, ctx->d_slab_if, ctx->d_slab_if_off,
                                         ctx->cluster_k, ctx->bmax_max, ctx->nlev_max,
                                         ctx->d.iface_tol, 1 + ctx->d.iface_ir_max, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "interface cluster launch");
    ctx->launches += 1;
  } else if (ctx->nunk > 0) {
    cudaError_t e = launch_iface_assemble(ctx->t, ctx->w, ctx->prec, ctx->slab_elems,
                                          ctx->d_pos2unk, ctx->npos, ctx->d_pos_real_off,
                                          ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "interface assembly launch");
    ctx->launches += 3;
    int nl = 0;
    e = launch_bcr_factor(ctx->t, ctx->w, ctx->prec, ctx->real.data(), &nl, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "interface factor launch");
    ctx->launches += nl;
    const int max_solves = 1 + ctx->d.iface_ir_max;
    if ((e = cudaMemsetAsync(ctx->w.dstat + 2, 0, sizeof(double) * ctx->d.n_real, ctx->stream)) !=
        cudaSuccess)
      return cuda_fail(ctx, e, "reset");
    e = launch_iface_solve(ctx->t, ctx->w, ctx->prec, ctx->d_pos2unk, ctx->d.iface_tol,
                           max_solves, ctx->solve_grid, ctx->max_vec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "interface solve launch");
    ctx->launches += 1;
  }
  ctx->state = 3;
  if (info) return read_info(ctx, info);
  return MRCM_OK;
}

mrcm_status mrcm_set_gravity(mrcm_ctx *ctx, const double *d_w) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->quad && d_w) return fail(ctx, MRCM_EINVAL, "gravity with a quadtree layout");
  ctx->t.grav = d_w;
  return MRCM_OK;
}

mrcm_status mrcm_reconstruct(mrcm_ctx *ctx, double *d_p, double *d_ux, double *d_uy,
                             double *d_gamma_u) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->state < 3) return fail(ctx, MRCM_EINVAL, "reconstruct before solve_interface");
  if (!d_p || !d_ux || !d_uy) return fail(ctx, MRCM_EINVAL, "p, ux, uy must be device pointers");
  cudaError_t e = launch_reconstruct(ctx->t, ctx->w, d_p, d_ux, d_uy, d_gamma_u, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reconstruct launch");
  ctx->launches += n_sizes(ctx) + (ctx->d.pure_neumann ? 2 : 1);
  return MRCM_OK;
}

mrcm_status mrcm_get_info(mrcm_ctx *ctx, mrcm_info *info) {
  if (!ctx || !info) return MRCM_EINVAL;
  return read_info(ctx, info);
}

int32_t mrcm_launch_count(const mrcm_ctx *ctx) { return ctx ? ctx->launches : 0; }

int64_t mrcm_num_interface_unknowns(const mrcm_ctx *ctx) { return ctx ? ctx->nunk : 0; }

int64_t mrcm_num_gamma_values(const mrcm_ctx *ctx) { return ctx ? ctx->gam_elems : 0; }

int32_t mrcm_uses_gmres(const mrcm_ctx *ctx) { return ctx && ctx->use_gmres ? 1 : 0; }

int32_t mrcm_interface_path(const mrcm_ctx *ctx) {
  if (!ctx) return -1;
  if (ctx->nunk == 0) return MRCM_PATH_NONE;
  if (ctx->use_gmres) return MRCM_PATH_GMRES;
  if (ctx->use_big) return MRCM_PATH_WIDE_SLAB;
  if (ctx->cluster_k > 0) return MRCM_PATH_CLUSTER;
  return MRCM_PATH_SLAB;
}

int64_t mrcm_num_precond_values(const mrcm_ctx *ctx) { return ctx ? ctx->tsc_elems : 0; }

mrcm_status mrcm_set_precond_blocks(mrcm_ctx *ctx, const double *d_blocks) {
  if (!ctx) return MRCM_EINVAL;
  if (!ctx->use_gmres || ctx->gm_precond != MRCM_PRECOND_USER)
    return fail(ctx, MRCM_EINVAL, "preconditioner blocks need the GMRES path with MRCM_PRECOND_USER");
  if (ctx->tsc_elems == 0) {
    ctx->gm_user_set = true;
    return MRCM_OK;
  }
  if (!d_blocks) return fail(ctx, MRCM_EINVAL, "d_blocks must be a device pointer");
  cudaError_t e = cudaMemcpyAsync(ctx->gm_Puser, d_blocks, sizeof(double) * ctx->tsc_elems,
                                  cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy preconditioner blocks");
  ctx->gm_user_set = true;
  return MRCM_OK;
}

mrcm_status mrcm_test_degrade_factor(mrcm_ctx *ctx, int32_t sub, int32_t mantissa_bits) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->prec == MRCM_PREC_FP64) return fail(ctx, MRCM_EINVAL, "FP64 context: no FP32 factor");
  if (sub < 0 || sub >= static_cast<int32_t>(ctx->sub.size()))
    return fail(ctx, MRCM_EINVAL, "subdomain %d out of range", sub);
  if (mantissa_bits < 1 || mantissa_bits > 22)
    return fail(ctx, MRCM_EINVAL, "mantissa_bits must be in 1..22");
  const SubInfo &sb = ctx->sub[sub];
  if (sb.s == 16 && ctx->t.fuse16)
    return fail(ctx, MRCM_EINVAL, "the basis kernel forms this subdomain's factor itself");
  float *W = static_cast<float *>(ctx->w.W) + sb.w_off;
  cudaError_t e = launch_degrade_factor(W, sb.s * sb.s * sb.s, mantissa_bits, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "degrade launch");
  return MRCM_OK;
}

mrcm_status mrcm_set_basis_width(mrcm_ctx *ctx, int32_t nc16, int32_t nc32) {
  if (!ctx) return MRCM_EINVAL;
  const bool w32ok = nc32 == 4 || nc32 == 8 || (nc32 == 16 && ctx->prec != MRCM_PREC_FP64);
  if ((nc16 != 4 && nc16 != 8 && nc16 != 12 && nc16 != 16) || !w32ok)
    return fail(ctx, MRCM_EINVAL,
                "basis widths: s = 16 one of 4, 8, 12, 16; s = 32 one of 4, 8 (16 also with "
                "MRCM_PREC_FP32_IR)");
  rebuild_items(ctx, nc16, nc32);
  cudaError_t e = cudaMemcpyAsync(ctx->d_items, ctx->items.data(),
                                  ctx->items.size() * sizeof(BasisItem), cudaMemcpyHostToDevice,
                                  ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "basis item upload");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "stream synchronize");
  return MRCM_OK;
}

mrcm_status mrcm_autotune(mrcm_ctx *ctx, const double *d_K, const double *d_lambda,
                          const double *d_q, int32_t reps, int32_t *chosen) {
  if (!ctx) return MRCM_EINVAL;
  if (!d_K || !d_lambda || !d_q) return fail(ctx, MRCM_EINVAL, "NULL device pointer");
  if (reps < 1 || reps > 100) return fail(ctx, MRCM_EINVAL, "reps must be in 1..100");
  mrcm_status st = mrcm_factor_local(ctx, d_K, d_lambda);
  if (st != MRCM_OK) return st;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return fail(ctx, MRCM_ECUDA, "event create");
  const bool has16 = ctx->nsub16 > 0, has32 = static_cast<int>(ctx->sub.size()) > ctx->nsub16;
  auto time_width = [&](int w16, int w32, float *ms) -> mrcm_status {
    mrcm_status s2 = mrcm_set_basis_width(ctx, w16, w32);
    if (s2 != MRCM_OK) return s2;
    std::vector<float> ts;
    for (int r = 0; r <= reps; ++r) {            // the first run is a warm-up
      cudaEventRecord(a, ctx->stream);
      if ((s2 = mrcm_build_basis(ctx, d_q)) != MRCM_OK) return s2;
      cudaEventRecord(b, ctx->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) return fail(ctx, MRCM_ECUDA, "event sync");
      float t = 0.0f;
      cudaEventElapsedTime(&t, a, b);
      if (r > 0) ts.push_back(t);
    }
    std::sort(ts.begin(), ts.end());
    *ms = ts[ts.size() / 2];
    return MRCM_OK;
  };
  int best16 = ctx->nc16, best32 = ctx->nc32;
  float tbest = 0.0f;
  mrcm_status s2 = MRCM_OK;
  if (has16) {
    tbest = 3.4e38f;
    for (int w16 : {4, 8, 12, 16}) {
      float t;
      if ((s2 = time_width(w16, best32, &t)) != MRCM_OK) break;
      if (t < tbest) { tbest = t; best16 = w16; }
    }
  }
  if (s2 == MRCM_OK && has32) {
    tbest = 3.4e38f;
    for (int w32 : {4, 8, 16}) {
      if (w32 == 16 && ctx->prec == MRCM_PREC_FP64) continue;
      float t;
      if ((s2 = time_width(best16, w32, &t)) != MRCM_OK) break;
      if (t < tbest) { tbest = t; best32 = w32; }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (s2 != MRCM_OK) return s2;
  if ((s2 = mrcm_set_basis_width(ctx, best16, best32)) != MRCM_OK) return s2;
  if (chosen) {
    chosen[0] = best16;
    chosen[1] = best32;
  }
  ctx->state = 1;                                  // factored; the basis is rebuilt by the caller
  return MRCM_OK;
}

int64_t mrcm_lp_num_samples(const mrcm_ctx *ctx) {
  return ctx ? static_cast<int64_t>(ctx->iface.size()) : 0;
}

mrcm_status mrcm_lp_windows(mrcm_ctx *ctx, const double *d_K, const double *d_lambda,
                            int64_t first, int32_t count, void *d_x) {
  if (!ctx) return MRCM_EINVAL;
  if (!d_K || !d_lambda || !d_x) return fail(ctx, MRCM_EINVAL, "NULL device pointer");
  if (!ctx->s_uniform) return fail(ctx, MRCM_EINVAL, "learned preconditioner: mixed subdomain sizes");
  const int64_t nif = static_cast<int64_t>(ctx->iface.size());
  if (first < 0 || count < 0 || first + count > nif)
    return fail(ctx, MRCM_EINVAL, "interface range outside 0..%lld", static_cast<long long>(nif));
  cudaError_t e = lp_windows(ctx->t, d_K, d_lambda, d_x, ctx->s_uniform, static_cast<int>(first),
                             count, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "window launch");
  return MRCM_OK;
}

mrcm_status mrcm_lp_targets(mrcm_ctx *ctx, float *d_target) {
  if (!ctx) return MRCM_EINVAL;
  if (!d_target) return fail(ctx, MRCM_EINVAL, "d_target must be a device pointer");
  if (!ctx->use_gmres) return fail(ctx, MRCM_EINVAL, "targets need the GMRES path");
  if (ctx->state < 2) return fail(ctx, MRCM_EINVAL, "targets before build_basis");
  if (!ctx->m_uniform) return fail(ctx, MRCM_EINVAL, "targets need one interface size m");
  if (ctx->nb_max > kLpMaxNb || ctx->nloc_max > kLpMaxLoc)
    return fail(ctx, MRCM_EINVAL, "neighbourhood of %d unknowns above %d", ctx->nloc_max,
                kLpMaxLoc);
  cudaError_t e = lp_targets(ctx->t, ctx->w, ctx->gm, ctx->d_nb_off, ctx->d_nb_list,
                             ctx->nloc_max, ctx->m_uniform, 0.5, d_target, &ctx->w.status[0],
                             ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "target launch");
  if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "stream synchronize");
  int st0 = 0;
  if ((e = cudaMemcpy(&st0, ctx->w.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(ctx, e, "status read");
  if (st0 & MRCM_FLAG_IFACE_PIVOT) return fail(ctx, MRCM_ENOTSPD, "singular neighbourhood matrix");
  return MRCM_OK;
}

mrcm_status mrcm_lp_apply(mrcm_ctx *ctx, mrcm_lp *lp, const double *d_K, const double *d_lambda) {
  if (!ctx || !lp) return MRCM_EINVAL;
  if (!ctx->use_gmres || ctx->gm_precond != MRCM_PRECOND_USER)
    return fail(ctx, MRCM_EINVAL, "the learned preconditioner needs GMRES with MRCM_PRECOND_USER");
  if (ctx->state < 2) return fail(ctx, MRCM_EINVAL, "lp_apply before build_basis");
  if (ctx->s_uniform != lp_s(lp) || ctx->m_uniform != lp_m(lp))
    return fail(ctx, MRCM_EINVAL, "network (s %d, m %d) does not match the problem", lp_s(lp),
                lp_m(lp));
  if (!d_K || !d_lambda) return fail(ctx, MRCM_EINVAL, "NULL device pointer");
  cudaError_t e;
  if ((e = launch_gmres_bj(ctx->t, ctx->w, ctx->gm, ctx->gm_Pbj, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "block-Jacobi launch");
  ctx->launches += 1;
  const cudaStream_t keep = lp_stream(lp);
  mrcm_lp_set_stream(lp, ctx->stream);
  const int nif = static_cast<int>(ctx->iface.size()), mb = lp_maxb(lp);
  for (int g0 = 0; g0 < nif; g0 += mb) {
    const int cnt = nif - g0 < mb ? nif - g0 : mb;
    if ((e = lp_windows(ctx->t, d_K, d_lambda, lp_xbuf(lp), ctx->s_uniform, g0, cnt,
                        ctx->stream)) != cudaSuccess ||
        (e = lp_forward(lp, lp_xbuf(lp), cnt, lp_deltabuf(lp))) != cudaSuccess ||
        (e = lp_blocks(ctx->t, ctx->gm_Pbj, lp_deltabuf(lp), ctx->gm_Puser, g0, cnt,
                       ctx->m_uniform, ctx->stream)) != cudaSuccess) {
      mrcm_lp_set_stream(lp, keep);
      return cuda_fail(ctx, e, "learned preconditioner launch");
    }
    ctx->launches += 6;
  }
  mrcm_lp_set_stream(lp, keep);
  ctx->gm_user_set = true;
  return MRCM_OK;
}

mrcm_status mrcm_copy_interface_solution(mrcm_ctx *ctx, double *d_x) {
  if (!ctx) return MRCM_EINVAL;
  if (ctx->nunk == 0) return MRCM_OK;
  if (!d_x) return fail(ctx, MRCM_EINVAL, "d_x must be a device pointer");
  if (ctx->state < 3) return fail(ctx, MRCM_EINVAL, "no interface solution yet");
  cudaError_t e = cudaMemcpyAsync(d_x, ctx->w.x, sizeof(double) * ctx->nunk,
                                  cudaMemcpyDeviceToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copy interface solution");
  return MRCM_OK;
}

}  // extern "C"
