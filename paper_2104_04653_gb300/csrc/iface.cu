// Step (d) of the MRCM solve: the interface system (Eq. "mrc2").
//
// Rows of interface g (between subdomains L < R) are the weak continuity
// conditions of Eq. "compatibility" tested by the interface functions; each
// row is the sum of one contribution from L and one from R, which the basis
// kernel stored as dense rows of G (one G per subdomain, columns = that
// subdomain's basis columns).  The matrix is never formed as a whole:
//
//  * the FP64 residual f - M x is evaluated from G directly;
//  * for the factorisation the unknowns are grouped in slabs (one column of
//    subdomains: its horizontal interfaces and the vertical interfaces on its
//    right; or the transpose when the grid has more subdomain rows than
//    columns), which makes M block tridiagonal over slabs.  With the flux
//    rows negated M is symmetric quasi-definite, so block elimination needs
//    no pivoting; it is done by block cyclic reduction (odd slabs first, then
//    recursively) on the symmetrically scaled matrix, in the working
//    precision, keeping explicit inverses of the eliminated pivots.
//
// FP32_IR refines the FP32 solve with FP64 residuals until the relative
// residual reaches the tolerance.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"
#include "iface_common.cuh"

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace cg = cooperative_groups;

namespace mrcm {
namespace {

constexpr int kBmax = 64;        // largest padded slab handled in shared memory
constexpr int kThreads = 512;

// (1) per-interface congruence scaling (see iface_common.cuh), one warp per
// interface.
__global__ void __launch_bounds__(32) k_iface_prep(DeviceTables t, Workspace w) {
  __shared__ double Sd[kMmax * (kMmax + 1)];
  __shared__ double Xd[kMmax * (kMmax + 1)];
  iface_scale_warp(t, w, blockIdx.x, Sd, Xd, kMmax + 1);
}

// (2) identity on padded slab positions and on the pinned unknown
template <typename T>
__global__ void k_iface_pad(DeviceTables t, Workspace w, const int *pos2unk, int64_t npos,
                            const int64_t *pos_real_off, int nreal) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  int r = 0;
  while (r + 1 < nreal && pos_real_off[r + 1] <= p) ++r;
  const RealInfo ri = t.real[r];
  const int64_t lp = p - pos_real_off[r];
  const int slab = static_cast<int>(lp / ri.bmax), pos = static_cast<int>(lp % ri.bmax);
  const int u = pos2unk[p];
  if (u < 0 || u == ri.pin) {
    T *B = static_cast<T *>(w.slabB) + ri.slab_off +
           static_cast<int64_t>(slab) * ri.bmax * ri.bmax;
    B[pos * ri.bmax + pos] = T(1);
  }
}

// (3) scaled blocks T_g S_{g g'} T_{g'}^T of the block-tridiagonal slab
// matrix; one CTA per interface g, one pass per neighbouring interface g'.
template <typename T>
__global__ void __launch_bounds__(64) k_iface_assemble(DeviceTables t, Workspace w) {
  const int g = blockIdx.x;
  const IfaceInfo fi = t.iface[g];
  const RealInfo ri = t.real[fi.r];
  const int m = fi.nU + fi.nP;
  const SubInfo &L = t.sub[fi.L];
  const SubInfo &R = t.sub[fi.R];
  __shared__ double Tg[kMmax][kMmax + 1], Tn[kMmax][kMmax + 1];
  __shared__ double Sb[kMmax][kMmax + 1], Xb[kMmax][kMmax + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < m * m; e += blockDim.x) Tg[e / m][e % m] = w.tsc[fi.tsc_off + e];
  const int64_t bb = static_cast<int64_t>(ri.bmax) * ri.bmax;
  T *Bs = static_cast<T *>(w.slabB) + ri.slab_off;
  T *As = static_cast<T *>(w.slabA) + ri.slab_off;
  T *Cs = static_cast<T *>(w.slabC) + ri.slab_off;
  // neighbour interfaces: the 4 edges of L then the 4 edges of R (g once)
  for (int k = 0; k < 8; ++k) {
    const int gn = k < 4 ? L.edge_iface[k] : R.edge_iface[k - 4];
    if (gn < 0) continue;
    bool dup = false;
    for (int q = 0; q < k; ++q)
      if ((q < 4 ? L.edge_iface[q] : R.edge_iface[q - 4]) == gn) dup = true;
    if (dup) continue;
    const IfaceInfo fn = t.iface[gn];
    const int mn = fn.nU + fn.nP;
    // edges of L and R carrying gn
    int eL = -1, eR = -1;
    for (int q = 0; q < 4; ++q) {
      if (L.edge_iface[q] == gn) eL = q;
      if (R.edge_iface[q] == gn) eR = q;
    }
    __syncthreads();
    for (int e = tid; e < mn * mn; e += blockDim.x) Tn[e / mn][e % mn] = w.tsc[fn.tsc_off + e];
    for (int e = tid; e < m * mn; e += blockDim.x) {
      const int i = e / mn, j = e % mn;
      const RowRef rr = row_ref(t, w, fi, i);
      double v = 0.0;
      if (eL >= 0) v += rr.gL[L.edge_col[eL] + j];
      if (eR >= 0) v += rr.gR[R.edge_col[eR] + j];
      if (i >= fi.nU) v = -v;                       // symmetrising sign
      if (fi.unk + i == ri.pin || fn.unk + j == ri.pin) v = 0.0;
      Sb[i][j] = v;
    }
    __syncthreads();
    for (int e = tid; e < m * mn; e += blockDim.x) {     // X = T_g S
      const int i = e / mn, j = e % mn;
      double v = 0.0;
      for (int q = 0; q <= i; ++q) v += Tg[i][q] * Sb[q][j];
      Xb[i][j] = v;
    }
    __syncthreads();
    T *blk;
    const int ds = fn.slab - fi.slab;
    if (ds == 0) blk = Bs + fi.slab * bb;
    else if (ds == -1) blk = As + fi.slab * bb;
    else if (ds == 1) blk = Cs + fi.slab * bb;
    else {
      if (tid == 0) atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
      continue;
    }
    for (int e = tid; e < m * mn; e += blockDim.x) {     // Y = X T_gn^T
      const int i = e / mn, j = e % mn;
      double v = 0.0;
      for (int q = 0; q <= j; ++q) v += Xb[i][q] * Tn[j][q];
      blk[static_cast<int64_t>(fi.pos + i) * ri.bmax + fn.pos + j] = static_cast<T>(v);
    }
  }
}

// ------------------------------------------------------------ BCR factor
// Slab blocks live in global memory as compact b x b row-major matrices and
// in shared memory as 64 x 64 tiles (zero outside b x b).  512 threads.
constexpr int kTile = 64;

template <typename T>
__device__ void tile_load(T *dst, const T *src, int b) {
  for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
    const int i = e / kTile, j = e % kTile;
    dst[e] = (i < b && j < b) ? src[i * b + j] : T(0);
  }
}
template <typename T>
__device__ void tile_store(T *dst, const T *src, int b, T scale = T(1)) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    dst[e] = scale * src[i * kTile + j];
  }
}
template <typename T>
__device__ void tile_zero_global(T *dst, int b) {
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) dst[e] = T(0);
}

// C = alpha * A B (+ C if acc), 64 x 64 tiles, k < b.  Thread t owns rows
// 4*(t/32)..+3 and columns 2*(t%32)..+1.
template <typename T>
__device__ void tile_gemm(T *C, const T *A, const T *B, int b, T alpha, bool acc) {
  const int t = threadIdx.x, jp = t & 31, iq = t >> 5;
  const int i0 = 4 * iq, j0 = 2 * jp;
  T c[4][2];
#pragma unroll
  for (int p = 0; p < 4; ++p) c[p][0] = c[p][1] = T(0);
  for (int k = 0; k < b; ++k) {
    const T b0 = B[k * kTile + j0], b1 = B[k * kTile + j0 + 1];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const T a = A[(i0 + p) * kTile + k];
      c[p][0] += a * b0;
      c[p][1] += a * b1;
    }
  }
  __syncthreads();   // C may alias nothing, but callers reuse A/B tiles next
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    T *cr = C + (i0 + p) * kTile + j0;
    cr[0] = acc ? cr[0] + alpha * c[p][0] : alpha * c[p][0];
    cr[1] = acc ? cr[1] + alpha * c[p][1] : alpha * c[p][1];
  }
  __syncthreads();
}

// One reduction level: every surviving slab k = 2*stride*i eliminates its
// odd neighbours l = k - stride and r = k + stride:
//   X = A_k B_l^{-1},  Y = C_k B_r^{-1}
//   B_k -= X C_l + Y A_r,  A_k <- -X A_l,  C_k <- -Y C_r.
// The CTA of k also writes B_r^{-1} (each odd slab has exactly one left
// survivor at its level).  stride = 0: invert the root slab 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bcr_level(DeviceTables t, Workspace w, int stride,
                                                       int lev) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int bad;
  const RealInfo ri = t.real[blockIdx.y];
  const int K = ri.nslab, b = ri.bmax;
  const int64_t bb = static_cast<int64_t>(b) * b;
  T *Bs = static_cast<T *>(w.slabB) + ri.slab_off;
  T *As = static_cast<T *>(w.slabA) + ri.slab_off;
  T *Cs = static_cast<T *>(w.slabC) + ri.slab_off;
  T *Is = static_cast<T *>(w.slabI) + ri.slab_off;
  T *tl = reinterpret_cast<T *>(smraw);
  T *tr = tl + kTile * kTile;
  T *tk = tr + kTile * kTile;
  T *tx = tk + kTile * kTile;
  T *tm = tx + kTile * kTile;
  T *gjs = tm + kTile * kTile;               // Gauss-Jordan scratch (64 + 1024)
  if (threadIdx.x == 0) bad = 0;
  if (stride == 0) {
    if (blockIdx.x != 0) return;
    tile_load(tk, Bs, b);
    __syncthreads();
    gj_inverse_blocked<T, kThreads>(tk, b, kTile, gjs, &bad);
    tile_store(Is, tk, b);
    if (threadIdx.x == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
    return;
  }
  const int k = 2 * stride * blockIdx.x;
  if (k >= K) return;
  const int l = k - stride, r = k + stride;
  T *X = static_cast<T *>(w.X) + ri.xy_off + (static_cast<int64_t>(lev) * K + k) * bb;
  T *Y = static_cast<T *>(w.Y) + ri.xy_off + (static_cast<int64_t>(lev) * K + k) * bb;
  tile_load(tk, Bs + k * bb, b);
  if (l >= 0) tile_load(tl, Bs + l * bb, b);
  if (r < K) tile_load(tr, Bs + r * bb, b);
  __syncthreads();
  if (l >= 0) gj_inverse_blocked<T, kThreads>(tl, b, kTile, gjs, &bad);
  if (r < K) {
    gj_inverse_blocked<T, kThreads>(tr, b, kTile, gjs, &bad);
    tile_store(Is + r * bb, tr, b);
  }
  if (l >= 0) {
    tile_load(tm, As + k * bb, b);
    __syncthreads();
    tile_gemm(tx, tm, tl, b, T(1), false);          // X
    tile_store(X, tx, b);
    tile_load(tm, Cs + l * bb, b);
    __syncthreads();
    tile_gemm(tk, tx, tm, b, T(-1), true);          // B_k -= X C_l
    tile_load(tm, As + l * bb, b);
    __syncthreads();
    tile_gemm(tl, tx, tm, b, T(-1), false);         // -X A_l
    tile_store(As + k * bb, tl, b);
  } else {
    tile_zero_global(X, b);
  }
  if (r < K) {
    tile_load(tm, Cs + k * bb, b);
    __syncthreads();
    tile_gemm(tx, tm, tr, b, T(1), false);          // Y
    tile_store(Y, tx, b);
    tile_load(tm, As + r * bb, b);
    __syncthreads();
    tile_gemm(tk, tx, tm, b, T(-1), true);          // B_k -= Y A_r
    tile_load(tm, Cs + r * bb, b);
    __syncthreads();
    tile_gemm(tr, tx, tm, b, T(-1), false);         // -Y C_r
    tile_store(Cs + k * bb, tr, b);
  } else {
    tile_zero_global(Y, b);
  }
  tile_store(Bs + k * bb, tk, b);
  if (threadIdx.x == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
}

// ------------------------------------------------------------ BCR solve
// y = Shat^{-1} z for one realisation, by one CTA; v holds z on entry and y
// on exit (slab-padded, shared memory), tmp is scratch of the same size.
// One warp per output row: coalesced row reads, shuffle reduction.
template <typename T>
__device__ void bcr_solve_cta(const DeviceTables &t, const Workspace &w, const RealInfo &ri, T *v,
                              T *tmp) {
  const int K = ri.nslab, b = ri.bmax;
  const int64_t bb = static_cast<int64_t>(b) * b;
  const T *As = static_cast<const T *>(w.slabA) + ri.slab_off;
  const T *Cs = static_cast<const T *>(w.slabC) + ri.slab_off;
  const T *Is = static_cast<const T *>(w.slabI) + ri.slab_off;
  const T *X = static_cast<const T *>(w.X) + ri.xy_off;
  const T *Y = static_cast<const T *>(w.Y) + ri.xy_off;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int j0 = lane, j1 = lane + 32;
  // forward: v_k -= X_lev(k) v_{k-s} + Y_lev(k) v_{k+s}, k = 0 mod 2s
  for (int lev = 0, s = 1; lev < ri.nlev; ++lev, s <<= 1) {
    const int nk = (K + 2 * s - 1) / (2 * s);
    for (int o = wid; o < nk * b; o += nw) {
      const int k = (o / b) * 2 * s, i = o % b;
      T acc = T(0);
      if (k - s >= 0) {
        const T *row = X + (static_cast<int64_t>(lev) * K + k) * bb + static_cast<int64_t>(i) * b;
        const T *vl = v + (k - s) * b;
        if (j0 < b) acc += row[j0] * vl[j0];
        if (j1 < b) acc += row[j1] * vl[j1];
      }
      if (k + s < K) {
        const T *row = Y + (static_cast<int64_t>(lev) * K + k) * bb + static_cast<int64_t>(i) * b;
        const T *vr = v + (k + s) * b;
        if (j0 < b) acc += row[j0] * vr[j0];
        if (j1 < b) acc += row[j1] * vr[j1];
      }
      acc = warp_sum(acc);
      if (lane == 0) v[k * b + i] -= acc;
    }
    __syncthreads();
  }
  // root
  for (int i = wid; i < b; i += nw) {
    const T *row = Is + static_cast<int64_t>(i) * b;
    T acc = T(0);
    if (j0 < b) acc += row[j0] * v[j0];
    if (j1 < b) acc += row[j1] * v[j1];
    acc = warp_sum(acc);
    if (lane == 0) tmp[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += blockDim.x) v[i] = tmp[i];
  __syncthreads();
  // backward: x_k = B_k^{-1} (v_k - A_k x_{k-s} - C_k x_{k+s}), k odd multiple of s
  for (int lev = ri.nlev - 1; lev >= 0; --lev) {
    const int s = 1 << lev;
    const int nk = (K - s + 2 * s - 1) / (2 * s);
    for (int o = wid; o < nk * b; o += nw) {
      const int k = s + (o / b) * 2 * s, i = o % b;
      const T *ra = As + k * bb + static_cast<int64_t>(i) * b;
      const T *xl = v + (k - s) * b;
      T acc = T(0);
      if (j0 < b) acc += ra[j0] * xl[j0];
      if (j1 < b) acc += ra[j1] * xl[j1];
      if (k + s < K) {
        const T *rc = Cs + k * bb + static_cast<int64_t>(i) * b;
        const T *xr = v + (k + s) * b;
        if (j0 < b) acc += rc[j0] * xr[j0];
        if (j1 < b) acc += rc[j1] * xr[j1];
      }
      acc = warp_sum(acc);
      if (lane == 0) tmp[k * b + i] = v[k * b + i] - acc;
    }
    __syncthreads();
    for (int o = wid; o < nk * b; o += nw) {
      const int k = s + (o / b) * 2 * s, i = o % b;
      const T *ri_ = Is + k * bb + static_cast<int64_t>(i) * b;
      const T *tk = tmp + k * b;
      T acc = T(0);
      if (j0 < b) acc += ri_[j0] * tk[j0];
      if (j1 < b) acc += ri_[j1] * tk[j1];
      acc = warp_sum(acc);
      if (lane == 0) v[k * b + i] = acc;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ refinement
// Cooperative kernel.  Each sweep:
//   A (all CTAs, one warp per interface): x_g += T_g^T y_g   (previous solve)
//   B (all CTAs, one warp per interface): r_g = f_g - (M x)_g in FP64 from
//     the two G rows of every unknown; z_g = T_g (sign r_g) in the working
//     precision into the slab-ordered vector
//   C (one CTA per realisation): stop test on ||r||/||f||, else y = BCR(z)
// with a grid-wide barrier between phases.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_iface_solve(DeviceTables t, Workspace w,
                                                         const int *pos2unk, double tol,
                                                         int max_solves) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[kThreads / 32];
  __shared__ double s_rel;
  __shared__ double wbuf[kThreads / 32][kMmax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * (kThreads / 32) + wid;
  const int nwarps = gridDim.x * (kThreads / 32);
  T *vec = static_cast<T *>(w.vec);
  int nsolve = 0;
  for (int sweep = 0;; ++sweep) {
    // phase A
    if (sweep > 0) {
      for (int g = gwarp; g < t.niface; g += nwarps) {
        const IfaceInfo fi = t.iface[g];
        const RealInfo &ri = t.real[fi.r];
        if (w.done[fi.r]) continue;
        const int m = fi.nU + fi.nP;
        const T *yv = vec + ri.vec_off + static_cast<int64_t>(fi.slab) * ri.bmax + fi.pos;
        const double *Tg = w.tsc + fi.tsc_off;
        if (lane < m) {
          double d = 0.0;
          for (int q = lane; q < m; ++q) d += Tg[q * m + lane] * static_cast<double>(yv[q]);
          w.x[fi.unk + lane] += d;
        }
      }
      grid.sync();
    }
    // phase B
    for (int g = gwarp; g < t.niface; g += nwarps) {
      const IfaceInfo fi = t.iface[g];
      const RealInfo &ri = t.real[fi.r];
      if (w.done[fi.r]) continue;
      const int m = fi.nU + fi.nP;
      double rv = 0.0;
      if (lane < m && fi.unk + lane != ri.pin) {
        const RowRef rr = row_ref(t, w, fi, lane);
        double sacc = w.f[fi.unk + lane];
        for (int c = 1; c < rr.ncL; ++c) sacc -= rr.gL[c] * w.x[t.col[rr.offL + c].unk];
        for (int c = 1; c < rr.ncR; ++c) sacc -= rr.gR[c] * w.x[t.col[rr.offR + c].unk];
        rv = sacc;
      }
      double sq = rv * rv;
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) w.r[g] = sq;                      // per-interface ||r||^2
      wbuf[wid][lane] = (lane >= fi.nU) ? -rv : rv;      // symmetrising sign
      __syncwarp();
      if (lane < m) {
        const double *Tg = w.tsc + fi.tsc_off;
        double zv = 0.0;
        for (int q = 0; q <= lane; ++q) zv += Tg[lane * m + q] * wbuf[wid][q];
        vec[ri.vec_off + static_cast<int64_t>(fi.slab) * ri.bmax + fi.pos + lane] =
            static_cast<T>(zv);
      }
      __syncwarp();
    }
    grid.sync();
    // phase C
    for (int r = blockIdx.x; r < t.n_real; r += gridDim.x) {
      const RealInfo ri = t.real[r];
      if (w.done[r]) continue;
      double rn = 0.0, fn = 0.0;
      for (int g = ri.iface0 + threadIdx.x; g < ri.iface0 + ri.niface; g += blockDim.x) rn += w.r[g];
      for (int u = ri.unk0 + threadIdx.x; u < ri.unk0 + ri.nunk; u += blockDim.x)
        fn += w.f[u] * w.f[u];
      for (int pass = 0; pass < 2; ++pass) {
        double v = pass == 0 ? rn : fn;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
          double sacc = 0.0;
          for (int k = 0; k < kThreads / 32; ++k) sacc += red[k];
          if (pass == 0) s_rel = sacc;
          else s_rel = sacc > 0.0 ? sqrt(s_rel / sacc) : 0.0;
        }
        __syncthreads();
      }
      const double rel = s_rel;
      const double prev = w.dstat[2 + r];
      __syncthreads();
      if (threadIdx.x == 0) w.dstat[2 + r] = rel;
      const bool stop = (rel <= tol) || (nsolve >= max_solves) || !(rel == rel) ||
                        (nsolve >= 2 && rel > 0.5 * prev);
      if (stop) {
        if (threadIdx.x == 0) {
          w.done[r] = 1;
          atomic_max_pos_double(&w.dstat[1], rel);
          atomicMax(&w.status[2], nsolve > 0 ? nsolve - 1 : 0);
          if (!(rel <= tol)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_STALL);
        }
        continue;
      }
      // y = Shat^{-1} z by block cyclic reduction, in shared memory
      T *v = reinterpret_cast<T *>(smraw);
      T *tmp = v + ri.nslab * ri.bmax;
      const int np = ri.nslab * ri.bmax;
      T *gv = vec + ri.vec_off;
      for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int u = pos2unk[ri.vec_off + p];
        v[p] = (u >= 0 && u != ri.pin) ? gv[p] : T(0);
      }
      __syncthreads();
      bcr_solve_cta(t, w, ri, v, tmp);
      for (int p = threadIdx.x; p < np; p += blockDim.x) gv[p] = v[p];
      __syncthreads();
    }
    ++nsolve;
    grid.sync();
    int all = 1;
    for (int r = 0; r < t.n_real; ++r) all &= w.done[r];
    if (all) break;
  }
}

}  // namespace

cudaError_t launch_iface_assemble(const DeviceTables &t, const Workspace &w, int prec,
                                  int64_t slab_elems, const int *pos2unk, int64_t npos,
                                  const int64_t *pos_real_off, cudaStream_t st) {
  const size_t esz = prec == MRCM_PREC_FP64 ? sizeof(double) : sizeof(float);
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.slabB, 0, slab_elems * esz, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.slabA, 0, slab_elems * esz, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.slabC, 0, slab_elems * esz, st)) != cudaSuccess) return e;
  const int thr = 256;
  const int nb1 = static_cast<int>((npos + thr - 1) / thr);
  k_iface_prep<<<t.niface, 32, 0, st>>>(t, w);
  if (prec == MRCM_PREC_FP64) {
    k_iface_assemble<double><<<t.niface, 64, 0, st>>>(t, w);
    k_iface_pad<double><<<nb1, thr, 0, st>>>(t, w, pos2unk, npos, pos_real_off, t.n_real);
  } else {
    k_iface_assemble<float><<<t.niface, 64, 0, st>>>(t, w);
    k_iface_pad<float><<<nb1, thr, 0, st>>>(t, w, pos2unk, npos, pos_real_off, t.n_real);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t bcr_factor_t(const DeviceTables &t, const Workspace &w, int maxslab, int nlev,
                                int *nlaunch, cudaStream_t st) {
  const size_t smem = (5 * kTile * kTile + 64 + 1024) * sizeof(T);
  for (int lev = 0, stride = 1; lev < nlev; ++lev, stride <<= 1) {
    const int neven = (maxslab + 2 * stride - 1) / (2 * stride);
    k_bcr_level<T><<<dim3(neven, t.n_real), kThreads, smem, st>>>(t, w, stride, lev);
    ++*nlaunch;
  }
  k_bcr_level<T><<<dim3(1, t.n_real), kThreads, smem, st>>>(t, w, 0, 0);
  ++*nlaunch;
  return cudaGetLastError();
}

cudaError_t launch_bcr_factor(const DeviceTables &t, const Workspace &w, int prec,
                              const RealInfo *host_real, int *nlaunch, cudaStream_t st) {
  int maxslab = 0, bmax = 0, nlev = 0;
  for (int r = 0; r < t.n_real; ++r) {
    if (host_real[r].nslab > maxslab) maxslab = host_real[r].nslab;
    if (host_real[r].bmax > bmax) bmax = host_real[r].bmax;
    if (host_real[r].nlev > nlev) nlev = host_real[r].nlev;
  }
  if (bmax > kBmax) return cudaErrorInvalidValue;
  if (prec == MRCM_PREC_FP64) return bcr_factor_t<double>(t, w, maxslab, nlev, nlaunch, st);
  return bcr_factor_t<float>(t, w, maxslab, nlev, nlaunch, st);
}

template <typename T>
static cudaError_t iface_solve_t(const DeviceTables &t, const Workspace &w, const int *pos2unk,
                                 double tol, int max_solves, int grid, size_t vecbytes,
                                 cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 2 * vecbytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_iface_solve<T>, t, w, pos2unk, tol, max_solves);
}

cudaError_t launch_iface_solve(const DeviceTables &t, const Workspace &w, int prec,
                               const int *pos2unk, double tol, int max_solves, int grid,
                               int max_vec, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.x, 0, sizeof(double) * t.nunk, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.dstat + 2, 0, sizeof(double) * t.n_real, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.done, 0, sizeof(int) * (t.n_real + 1), st)) != cudaSuccess) return e;
  if (prec == MRCM_PREC_FP64)
    return iface_solve_t<double>(t, w, pos2unk, tol, max_solves, grid,
                                 sizeof(double) * max_vec, st);
  return iface_solve_t<float>(t, w, pos2unk, tol, max_solves, grid, sizeof(float) * max_vec, st);
}

template <typename T>
static cudaError_t init_iface_t(int bmax, int max_vec) {
  (void)bmax;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_bcr_level<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>((5 * kTile * kTile + 64 + 1024) * sizeof(T)))) !=
      cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_iface_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              2 * max_vec * static_cast<int>(sizeof(T)));
}

cudaError_t init_iface_attributes(int prec, int bmax, int max_vec) {
  if (prec == MRCM_PREC_FP64) return init_iface_t<double>(bmax, max_vec);
  return init_iface_t<float>(bmax, max_vec);
}

// Largest co-resident grid of the cooperative refinement kernel.
int iface_solve_grid(int prec, int dev, int max_vec) {
  int nsm = 0, per = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 2 * static_cast<size_t>(max_vec) *
                      (prec == MRCM_PREC_FP64 ? sizeof(double) : sizeof(float));
  if (prec == MRCM_PREC_FP64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_iface_solve<double>, kThreads, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_iface_solve<float>, kThreads, smem);
  if (per < 1) return 0;
  return nsm;   // one CTA per SM
}

}  // namespace mrcm
