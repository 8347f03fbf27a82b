// Step (d) for interface systems too large for the slab reduction: the
// interface system of Eq. "mrc2" solved by restarted FP64 GMRES with right
// preconditioning by m x m blocks, one per interface (block-Jacobi, or
// blocks supplied by the caller, e.g. from the learned preconditioner).
//
// The matrix is never assembled.  Row i of interface g is the sum of the
// two one-sided contributions G_L and G_R that the basis kernel wrote (the
// traces of every basis column of the two adjacent subdomains).  Right
// preconditioning by P = blockdiag(P_g) is folded into those rows once per
// solve, G' = G P, so every GMRES iteration costs a single gather-SpMV.
//
// One cooperative kernel runs the whole iteration for all realisations at
// once.  Each realisation owns a contiguous range of blocks and every block
// a contiguous range of rows.  Orthogonalisation is classical Gram-Schmidt
// applied twice (CGS2): two block-reduced dot-product rounds per step, so
// an Arnoldi step needs three grid-wide barriers.  The small Hessenberg
// least-squares problem is solved redundantly, bit-identically, by every
// block of a realisation, so no block ever waits for a broadcast.
//
// The neighbourhood preconditioner (MRCM_PRECOND_NEIGHBOURHOOD) is not
// block-diagonal: column block g of P is the part of the inverse of the
// interface matrix restricted to g's neighbourhood that belongs to g.  G P
// is then folded into wider rows (the column blocks that reach each row),
// and x = P y gathers over the blocks whose neighbourhood holds the row.
#include "mrcm_internal.h"
#include "iface_common.cuh"
#include "nbsolve.cuh"
#include "../../include/mrcm.h"

#include <algorithm>
#include <cooperative_groups.h>
#include <cstdint>

namespace cg = cooperative_groups;

namespace mrcm {
namespace {

constexpr int kGmWarps = kGmThreads / 32;
constexpr int kGmAcc = (kGmKmax + 1 + kGmWarps - 1) / kGmWarps;

// P_g entry (l, k), with the pinned unknown of a pure-Neumann realisation
// (if it belongs to g) replaced by an identity row and column.
__device__ __forceinline__ double pblk(const double *Pg, int m, int ipin, int l, int k) {
  if (l == ipin || k == ipin) return l == k ? 1.0 : 0.0;
  return Pg[l * m + k];
}

__device__ __forceinline__ int pin_in(const IfaceInfo &fi, int pin) {
  const int m = fi.nU + fi.nP;
  return (pin >= fi.unk && pin < fi.unk + m) ? pin - fi.unk : -1;
}

// ---------------------------------------------------------------------------
// Block-Jacobi blocks: P_g = (M_gg)^{-1}, M_gg the coupling of interface g's
// unknowns with themselves (both sides' traces of g's own basis columns).
// One warp per interface; Gauss-Jordan with partial pivoting in FP64.
constexpr int kBjWarps = 2;

__global__ void __launch_bounds__(32 * kBjWarps) k_gm_bj(DeviceTables t, Workspace w, GmArgs a,
                                                          double *Pout) {
  __shared__ double aug[kBjWarps][kGmMmax][2 * kGmMmax + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = blockIdx.x * kBjWarps + wid;
  if (g >= t.niface) return;
  const IfaceInfo fi = t.iface[g];
  if (a.gate && a.fallback[fi.r] == 0) return;
  const int m = fi.nU + fi.nP;
  const int ipin = pin_in(fi, t.real[fi.r].pin);
  double(*Ab)[2 * kGmMmax + 1] = aug[wid];
  const SubInfo L = t.sub[fi.L], R = t.sub[fi.R];
  if (lane < m) {
    const int i = lane;
    const double *gl = w.G + L.g_off + static_cast<int64_t>(fi.rowL + i) * L.ncols + fi.colL;
    const double *gr = w.G + R.g_off + static_cast<int64_t>(fi.rowR + i) * R.ncols + fi.colR;
    for (int k = 0; k < m; ++k) {
      double v = gl[k] + gr[k];
      if (i == ipin || k == ipin) v = (i == k) ? 1.0 : 0.0;
      Ab[i][k] = v;
      Ab[i][m + k] = (i == k) ? 1.0 : 0.0;
    }
  }
  __syncwarp();
  bool bad = false;
  for (int p = 0; p < m; ++p) {
    // pivot: largest |A(i, p)| over i >= p (ties: smallest i)
    double best = lane >= p && lane < m ? fabs(Ab[lane][p]) : -1.0;
    int bi = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(best > 0.0) || !isfinite(best)) {
      bad = true;
      break;
    }
    if (bi != p)
      for (int k = lane; k < 2 * m; k += 32) {
        const double tmp = Ab[p][k];
        Ab[p][k] = Ab[bi][k];
        Ab[bi][k] = tmp;
      }
    __syncwarp();
    const double ip = 1.0 / Ab[p][p];
    __syncwarp();
    for (int k = lane; k < 2 * m; k += 32) Ab[p][k] *= ip;
    __syncwarp();
    if (lane < m && lane != p) {
      const double f = Ab[lane][p];
      for (int k = 0; k < 2 * m; ++k) Ab[lane][k] -= f * Ab[p][k];
    }
    __syncwarp();
  }
  double *Pg = Pout + fi.tsc_off;
  if (lane < m)
    for (int k = 0; k < m; ++k) Pg[lane * m + k] = bad ? (lane == k ? 1.0 : 0.0) : Ab[lane][m + k];
  if (bad && lane == 0) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
}

// ---------------------------------------------------------------------------
// G' = G P: every basis column block of a subdomain's trace rows times the
// preconditioner block of the interface that column belongs to.  One CTA
// per subdomain; column 0 (sources / boundary data) is not used by G'.
__global__ void __launch_bounds__(128) k_gm_gprime(DeviceTables t, Workspace w, GmArgs a,
                                                    const double *P) {
  const SubInfo sb = t.sub[blockIdx.x];
  if (a.gate && a.fallback[sb.r] == 0) return;
  const int pin = t.real[sb.r].pin;
  const int nc = sb.ncols - 1;
  const double *G = w.G + sb.g_off;
  double *Gp = a.Gp + sb.g_off;
  for (int e = threadIdx.x; e < sb.nrows * nc; e += blockDim.x) {
    const int row = e / nc, c = 1 + e % nc;
    const ColInfo ci = t.col[sb.col_off + c];
    const IfaceInfo fi = t.iface[t.unk_iface[ci.unk]];
    const int m = fi.nU + fi.nP, c0 = fi.L == static_cast<int>(blockIdx.x) ? fi.colL : fi.colR,
              k = c - c0;
    const int ipin = pin_in(fi, pin);
    const double *Pg = P + fi.tsc_off;
    const double *gr = G + static_cast<int64_t>(row) * sb.ncols + c0;
    double acc = 0.0;
    for (int l = 0; l < m; ++l) acc = fma(gr[l], pblk(Pg, m, ipin, l, k), acc);
    Gp[static_cast<int64_t>(row) * sb.ncols + c] = acc;
  }
}

// ---------------------------------------------------------------------------
// Neighbourhood preconditioner (restricted additive Schwarz with one
// subdomain of overlap, Cai and Sarkis 1999, applied on the right): column
// block g of P is the m_g columns of (M_N(g))^{-1} that belong to g, placed
// on the rows of N(g).  One CTA per interface builds its block (FP64
// Gaussian elimination in shared memory, nbsolve.cuh).
__global__ void __launch_bounds__(256) k_gm_nbcols(DeviceTables t, Workspace w, GmArgs a,
                                                   const int *nb_off, const int *nb_list) {
  extern __shared__ __align__(16) double nsm[];
  const int g = blockIdx.x;
  const IfaceInfo fg = t.iface[g];
  const int m = fg.nU + fg.nP;
  const int h0 = nb_off[g], nh = nb_off[g + 1] - h0;
  __shared__ int loc[kLpMaxNb + 1];
  __shared__ int s_n, s_pos, s_piv, s_bad;
  const bool bad = nb_inverse_columns(t, w, a.row, nb_list, h0, nh, g, nsm, nullptr, loc, &s_n,
                                      &s_pos, &s_piv, &s_bad);
  const int n = s_n, ld = n + m;
  double *Pg = a.Pnb + a.p_off[g];
  for (int e = threadIdx.x; e < n * m; e += blockDim.x)
    Pg[e] = bad ? 0.0 : nsm[static_cast<size_t>(e / m) * ld + n + e % m];
  if (bad && threadIdx.x == 0) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
}

// The P entries of interface h's rows in column block g' (null if h is not
// in N(g')): gat lists the blocks holding h, in increasing g'.
__device__ __forceinline__ const double *nb_rows(const GmArgs &a, int h, int gp) {
  for (int j = a.gat_off[h]; j < a.gat_off[h + 1]; ++j)
    if (a.gat_g[j] == gp) return a.Pnb + a.gat_o[j];
  return nullptr;
}

// Wide G P: entry (row i of interface g, column k of block g' in pb(g)) =
// sum over the columns q of the row (both sides, the pinned unknown left
// out) of G[u, q] P[q, (g', k)].  One CTA per interface.
__global__ void __launch_bounds__(128) k_gm_gwide(DeviceTables t, Workspace w, GmArgs a) {
  const int g = blockIdx.x;
  const IfaceInfo fg = t.iface[g];
  const int m = fg.nU + fg.nP, wg = a.gw_w[g];
  const int pin = t.real[fg.r].pin;
  const int b0 = a.pb_off[g], nbk = a.pb_off[g + 1] - b0;
  double *Gw = a.Gw + a.gw_off[g];
  for (int e = threadIdx.x; e < m * wg; e += blockDim.x) {
    const int i = e / wg, col = e % wg;
    int j = nbk - 1;
    while (a.pb_pos[b0 + j] > col) --j;              // block holding this column
    const int gp = a.pb_list[b0 + j], k = col - a.pb_pos[b0 + j];
    const int mp = t.iface[gp].nU + t.iface[gp].nP;
    const int u = fg.unk + i;
    double acc = 0.0;
    if (u != pin) {
      const GmRow R = a.row[u];
      int hlast = -1;
      const double *Ph = nullptr;
      for (int side = 0; side < 2; ++side) {
        const double *gr = w.G + (side ? R.gR : R.gL);
        const ColInfo *cl = t.col + (side ? R.cR : R.cL);
        const int nc = side ? R.nR : R.nL;
        for (int c = 0; c < nc; ++c) {
          const int q = cl[c].unk;
          if (q == pin) continue;
          const int h = t.unk_iface[q];
          if (h != hlast) {
            Ph = nb_rows(a, h, gp);
            hlast = h;
          }
          if (Ph) acc = fma(gr[c], Ph[(q - t.iface[h].unk) * mp + k], acc);
        }
      }
    }
    Gw[static_cast<int64_t>(i) * wg + col] = acc;
  }
}

// ---------------------------------------------------------------------------
// GMRES kernel helpers.

// (M P v)[u] with the neighbourhood preconditioner (wide rows).
__device__ __forceinline__ double gm_apply_nb(const DeviceTables &t, const GmArgs &a, int u,
                                              const double *v, int u0, int pin) {
  if (u == pin) return __ldcg(v + (u - u0));
  const int g = t.unk_iface[u];
  const IfaceInfo fg = t.iface[g];
  const int wg = a.gw_w[g];
  const double *row = a.Gw + a.gw_off[g] + static_cast<int64_t>(u - fg.unk) * wg;
  double s0 = 0.0, s1 = 0.0;
  for (int j = a.pb_off[g]; j < a.pb_off[g + 1]; ++j) {
    const IfaceInfo fp = t.iface[a.pb_list[j]];
    const int mp = fp.nU + fp.nP;
    const double *rj = row + a.pb_pos[j];
    for (int k = 0; k < mp; ++k) {
      const int q = fp.unk + k;
      if (q == pin) continue;
      if (k & 1) s1 = fma(rj[k], __ldcg(v + (q - u0)), s1);
      else s0 = fma(rj[k], __ldcg(v + (q - u0)), s0);
    }
  }
  return s0 + s1;
}

// (P y)[u] with the neighbourhood preconditioner: the blocks g' whose
// neighbourhood holds u's interface h.
__device__ __forceinline__ double gm_prec_nb(const DeviceTables &t, const GmArgs &a, int u,
                                             const double *y, int u0) {
  const int h = t.unk_iface[u];
  const int i = u - t.iface[h].unk;
  double acc = 0.0;
  for (int j = a.gat_off[h]; j < a.gat_off[h + 1]; ++j) {
    const IfaceInfo fp = t.iface[a.gat_g[j]];
    const int mp = fp.nU + fp.nP;
    const double *Pr = a.Pnb + a.gat_o[j] + static_cast<int64_t>(i) * mp;
    for (int k = 0; k < mp; ++k) acc = fma(Pr[k], __ldcg(y + (fp.unk - u0 + k)), acc);
  }
  return acc;
}

// (M P v)[u] for a realisation-local vector v (index = unknown - u0).
__device__ __forceinline__ double gm_apply(const DeviceTables &t, const GmArgs &a, int u,
                                           const double *v, int u0, int pin) {
  if (u == pin) return __ldcg(v + (u - u0));
  const GmRow R = a.row[u];
  double s0 = 0.0, s1 = 0.0;
  const double *gl = a.Gp + R.gL;
  const ColInfo *cl = t.col + R.cL;
  for (int c = 0; c < R.nL; ++c) {
    const int q = cl[c].unk;
    if (q != pin) s0 = fma(gl[c], __ldcg(v + (q - u0)), s0);
  }
  const double *gr = a.Gp + R.gR;
  const ColInfo *cr = t.col + R.cR;
  for (int c = 0; c < R.nR; ++c) {
    const int q = cr[c].unk;
    if (q != pin) s1 = fma(gr[c], __ldcg(v + (q - u0)), s1);
  }
  return s0 + s1;
}

// right-hand side of row u: minus the two sides' source / boundary traces
__device__ __forceinline__ double gm_rhs(const Workspace &w, const GmArgs &a, int u, int pin) {
  if (u == pin) return 0.0;
  const GmRow R = a.row[u];
  return -(w.G[R.gL - 1] + w.G[R.gR - 1]);
}

// sum over the CTA of one value per thread, into out (thread 0 writes)
__device__ __forceinline__ void gm_block_sum(double v, double *scratch, double *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kGmWarps; ++k) s += scratch[k];
    *out = s;
  }
  __syncthreads();
}

// partial dot products of this CTA's rows: out[i] = sum_rows V_i . x for
// i < cnt, the last one scaled by last_scale.  Warp q takes i = q + 8k.
__device__ __forceinline__ void gm_dots(const double *V, int64_t n, int rl0, int rl1,
                                        const double *x, int cnt, double last_scale,
                                        double *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc[kGmAcc];
#pragma unroll
  for (int q = 0; q < kGmAcc; ++q) acc[q] = 0.0;
  for (int u = rl0 + lane; u < rl1; u += 32) {
    const double xu = x[u];
#pragma unroll
    for (int q = 0; q < kGmAcc; ++q) {
      const int i = wid + kGmWarps * q;
      if (i < cnt) acc[q] = fma(V[i * n + u], xu, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kGmAcc; ++q) {
    const int i = wid + kGmWarps * q;
    if (i < cnt) {
      double s = warp_sum(acc[q]);
      if (i == cnt - 1) s *= last_scale;
      if (lane == 0) out[i] = s;
    }
  }
}

// sum of the partials of the realisation's CTAs, in a fixed order so that
// every CTA of the realisation obtains bit-identical values
__device__ __forceinline__ void gm_reduce(const double *part, int stride, int blk0, int nblk,
                                          int cnt, double *out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < cnt; i += kGmWarps) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(part + static_cast<int64_t>(blk0 + b) * stride + i);
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
  __syncthreads();
}

// sum_{i < cnt} h_i V_i[u] with four independent FMA chains
__device__ __forceinline__ double gm_comb(const double *h, const double *V, int64_t n, int u,
                                          int cnt) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = 0;
  for (; i + 3 < cnt; i += 4) {
    a0 = fma(h[i], V[i * n + u], a0);
    a1 = fma(h[i + 1], V[(i + 1) * n + u], a1);
    a2 = fma(h[i + 2], V[(i + 2) * n + u], a2);
    a3 = fma(h[i + 3], V[(i + 3) * n + u], a3);
  }
  for (; i < cnt; ++i) a0 = fma(h[i], V[i * n + u], a0);
  return (a0 + a1) + (a2 + a3);
}

enum { kIter = 0, kUpdate = 1, kDone = 2 };

// NB: the neighbourhood preconditioner (wide rows of G P, x = P y by gather)
template <bool NB>
__global__ void __launch_bounds__(kGmThreads) k_gmres(DeviceTables t, Workspace w, GmArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) double gsm[];
  const int K = a.K;
  double *Rm = gsm;                 // R(i, c) at Rm[c * K + i], upper triangular
  double *cs = Rm + K * K;          // Givens cosines
  double *sn = cs + K;              // Givens sines
  double *gv = sn + K;              // rotated right-hand side [K + 1]
  double *hv = gv + K + 1;          // Hessenberg column [K + 1]
  double *cv = hv + K + 1;          // second-pass dots, then the LS solution [K + 1]
  double *ring = cv + K + 1;        // residual estimates of the last 16 steps
  double *rinv = ring + 16;         // 1 / R(i, i) [K]
  double *scr = rinv + K;           // [kGmWarps + 2]
  const GmBlock B = a.blk[blockIdx.x];
  const RealInfo ri = t.real[B.r];
  const int64_t n = ri.nunk;
  const int u0 = ri.unk0, pin = ri.pin;
  const int rl0 = B.row0 - u0, rl1 = B.row1 - u0;
  double *V = a.V + static_cast<int64_t>(K + 1) * u0;
  double *Wv = a.Wv + u0, *Y = a.Y + u0;
  const int stride = K + 2;
  double *mypart = a.part + static_cast<int64_t>(blockIdx.x) * stride;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool lead = (blockIdx.x == B.blk0) && tid == 0;

  int mode = kUpdate, j = 0, it = 0;
  double beta = 0.0, fn = -1.0;
  bool stalled = false;
  const bool ran = !(a.gate && __ldcg(a.fallback + B.r) == 0);
  if (!ran) {
    mode = kDone;
    if (lead) atomicExch(a.done + B.r, 1);
  }

  // initial residual: Y = 0, r = f
  {
    double s = 0.0;
    if (ran)
      for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) {
        const double f = gm_rhs(w, a, u0 + ul, pin);
        w.f[u0 + ul] = f;
        V[ul] = f;
        Y[ul] = 0.0;
        s = fma(f, f, s);
      }
    gm_block_sum(s, scr, mypart);
  }
  grid.sync();

  for (;;) {
    // ----------------------------------------------------------- phase A
    if (mode != kDone) {
      gm_reduce(a.part, stride, B.blk0, B.nblk, 1, scr + kGmWarps);
      const double nrm2 = scr[kGmWarps];
      if (mode == kUpdate) {
        // the true residual of the current iterate is in slot 0
        beta = sqrt(nrm2);
        if (fn < 0.0) fn = beta;
        const double rel = fn > 0.0 ? beta / fn : 0.0;
        if (!isfinite(rel)) stalled = true;
        if (rel <= a.tol || it >= a.maxit || stalled || fn == 0.0) {
          mode = kDone;
          if (lead) {
            const int tot = atomicAdd(a.iters + B.r, it) + it;
            atomicMax(&w.status[3], tot);
            a.resid[B.r] = rel;
            if (a.stall && !(rel <= a.tol)) {
              a.fallback[B.r] = 1;               // leave for block-Jacobi
            } else {
              atomic_max_pos_double(&w.dstat[1], rel);
              if (!(rel <= a.tol)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_STALL);
              if (a.gate) atomicOr(&w.status[0], MRCM_FLAG_PRECOND_FALLBACK);
            }
            __threadfence();
            atomicExch(a.done + B.r, 1);
          }
        } else {
          j = 0;
          if (tid == 0) gv[0] = beta;
          mode = kIter;
        }
      } else {
        // close Arnoldi step j: last rotation (the earlier ones were applied
        // to the column in phase C), then decide whether to update the iterate
        const double hnext = sqrt(nrm2);
        if (tid == 0) {
          const double hj = hv[j];
          double c = 1.0, s = 0.0, rr = hj;
          if (hnext != 0.0) {
            rr = hypot(hj, hnext);
            c = hj / rr;
            s = hnext / rr;
          }
          cs[j] = c;
          sn[j] = s;
          Rm[j * K + j] = rr;
          gv[j + 1] = -s * gv[j];
          gv[j] = c * gv[j];
        }
        __syncthreads();
        beta = hnext;
        ++j;
        ++it;
        const double est = fabs(gv[j]);
        if (a.stall && it > 10 && est > 0.9 * ring[(it - 10) & 15]) stalled = true;
        if (!isfinite(est)) stalled = true;
        __syncthreads();
        if (tid == 0) ring[it & 15] = est;
        if (est <= a.tol * fn || j == K || it >= a.maxit || stalled || hnext == 0.0) {
          // R z = g by columns (warp 0), then Y += V z
          if (wid == 0) {
            for (int i = lane; i < j; i += 32) {
              cv[i] = gv[i];
              const double d = Rm[i * K + i];
              rinv[i] = d != 0.0 ? 1.0 / d : 0.0;
            }
            __syncwarp();
            for (int c = j - 1; c >= 0; --c) {
              const double zc = cv[c] * rinv[c];
              __syncwarp();
              for (int i = lane; i < c; i += 32) cv[i] = fma(-Rm[c * K + i], zc, cv[i]);
              if (lane == 0) cv[c] = zc;
              __syncwarp();
            }
          }
          __syncthreads();
          for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) Y[ul] += gm_comb(cv, V, n, ul, j);
          mode = kUpdate;
        }
      }
      if (mode == kIter) {
        // w = M P v_j, v_j = slot j / beta (normalised in phase B)
        const double inv = 1.0 / beta;
        const double *vj = V + j * n;
        for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads)
          Wv[ul] = inv * (NB ? gm_apply_nb(t, a, u0 + ul, vj, u0, pin)
                             : gm_apply(t, a, u0 + ul, vj, u0, pin));
        __syncthreads();
        gm_dots(V, n, rl0, rl1, Wv, j + 1, inv, mypart);
      }
    }
    grid.sync();
    // ----------------------------------------------------------- phase B
    {
      int nd = 0;
      for (int r = 0; r < t.n_real; ++r) nd += __ldcg(a.done + r);
      if (nd == t.n_real) break;
    }
    if (mode == kIter) {
      gm_reduce(a.part, stride, B.blk0, B.nblk, j + 1, hv);
      const double inv = 1.0 / beta;
      for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) {
        const double vj = V[j * n + ul] * inv;
        V[j * n + ul] = vj;
        const double c = gm_comb(hv, V, n, ul, j);
        Wv[ul] = Wv[ul] - fma(hv[j], vj, c);
      }
      __syncthreads();
      gm_dots(V, n, rl0, rl1, Wv, j + 1, 1.0, mypart);
    } else if (mode == kUpdate) {
      double s = 0.0;
      for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) {
        const int u = u0 + ul;
        const double r = gm_rhs(w, a, u, pin) -
                         (NB ? gm_apply_nb(t, a, u, Y, u0, pin) : gm_apply(t, a, u, Y, u0, pin));
        V[ul] = r;
        s = fma(r, r, s);
      }
      gm_block_sum(s, scr, mypart);
    }
    grid.sync();
    // ----------------------------------------------------------- phase C
    if (mode == kIter) {
      gm_reduce(a.part, stride, B.blk0, B.nblk, j + 1, cv);
      if (tid <= j) hv[tid] += cv[tid];
      __syncthreads();
      double s = 0.0;
      if (wid == 0) {
        // earlier rotations on the new column, overlapped with the updates
        if (lane == 0) {
          double hprev = hv[0];
          for (int i = 0; i < j; ++i) {
            const double hn = hv[i + 1];
            Rm[j * K + i] = fma(cs[i], hprev, sn[i] * hn);
            hprev = fma(-sn[i], hprev, cs[i] * hn);
          }
          hv[j] = hprev;
        }
      } else {
        for (int ul = rl0 + tid - 32; ul < rl1; ul += kGmThreads - 32) {
          const double wv = Wv[ul] - gm_comb(cv, V, n, ul, j + 1);
          V[(j + 1) * n + ul] = wv;
          s = fma(wv, wv, s);
        }
      }
      gm_block_sum(s, scr, mypart);
    }
    grid.sync();
  }
  // x = P y on this CTA's rows
  if (ran && NB)
    for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) w.x[u0 + ul] = gm_prec_nb(t, a, u0 + ul, Y, u0);
  else if (ran)
    for (int ul = rl0 + tid; ul < rl1; ul += kGmThreads) {
      const int u = u0 + ul;
      const IfaceInfo fi = t.iface[t.unk_iface[u]];
      const int m = fi.nU + fi.nP, i = u - fi.unk, ipin = pin_in(fi, pin);
      const double *Pg = a.P + fi.tsc_off;
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc = fma(pblk(Pg, m, ipin, i, k), __ldcg(Y + (fi.unk - u0 + k)), acc);
      w.x[u] = acc;
    }
}

}  // namespace

size_t gmres_smem_bytes(int K) {
  return sizeof(double) * (static_cast<size_t>(K) * K + 6 * static_cast<size_t>(K) + 19 + kGmWarps + 2);
}

int gmres_max_blocks(int K, int dev) {
  int nsm = 0, per = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = gmres_smem_bytes(K);
  int per_nb = 0;
  if (cudaFuncSetAttribute(k_gmres<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess ||
      cudaFuncSetAttribute(k_gmres<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres<false>, kGmThreads, smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_nb, k_gmres<true>, kGmThreads, smem) !=
          cudaSuccess)
    return 0;
  return nsm * std::min(per, per_nb);
}

cudaError_t launch_gmres_bj(const DeviceTables &t, const Workspace &w, const GmArgs &a, double *Pbj,
                            cudaStream_t st) {
  if (t.niface == 0) return cudaSuccess;
  k_gm_bj<<<(t.niface + kBjWarps - 1) / kBjWarps, 32 * kBjWarps, 0, st>>>(t, w, a, Pbj);
  return cudaGetLastError();
}

cudaError_t launch_gmres_precond(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                                 double *Pbj, bool build_bj, cudaStream_t st) {
  if (build_bj && t.niface > 0) {
    k_gm_bj<<<(t.niface + kBjWarps - 1) / kBjWarps, 32 * kBjWarps, 0, st>>>(t, w, a, Pbj);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_gm_gprime<<<t.nsub, 128, 0, st>>>(t, w, a, a.P);
  return cudaGetLastError();
}

cudaError_t launch_gmres_nb(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                            const int *nb_off, const int *nb_list, int nloc_max, int mmax,
                            cudaStream_t st) {
  if (t.niface == 0) return cudaSuccess;
  const size_t smem = lp_targets_smem(nloc_max, mmax);
  cudaError_t e = cudaFuncSetAttribute(k_gm_nbcols, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_gm_nbcols<<<t.niface, 256, smem, st>>>(t, w, a, nb_off, nb_list);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_gm_gwide<<<t.niface, 128, 0, st>>>(t, w, a);
  return cudaGetLastError();
}

cudaError_t launch_gmres(const DeviceTables &t, const Workspace &w, const GmArgs &a, int nblk,
                         cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk);
  cfg.blockDim = dim3(kGmThreads);
  cfg.dynamicSmemBytes = gmres_smem_bytes(a.K);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return a.nb ? cudaLaunchKernelEx(&cfg, k_gmres<true>, t, w, a)
              : cudaLaunchKernelEx(&cfg, k_gmres<false>, t, w, a);
}

}  // namespace mrcm
