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

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>

namespace cg = cooperative_groups;

namespace mrcm {
namespace {

constexpr int kBmax = 64;        // largest padded slab handled in shared memory
constexpr int kThreads = 512;

__device__ __forceinline__ void atomic_max_pos_double(double *addr, double v) {
  if (!(v >= 0.0)) v = 1e300;
  atomicMax(reinterpret_cast<unsigned long long *>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

// G rows of interface fi on side L and R, and the column of its own unknown i
struct RowRef {
  const double *gL, *gR;   // pointers to the two G rows
  int ncL, ncR;
  int colL, colR;          // column of the row's own unknown (diagonal)
  int offL, offR;          // col table offsets
};

__device__ __forceinline__ RowRef row_ref(const DeviceTables &t, const Workspace &w,
                                          const IfaceInfo &fi, int i) {
  const SubInfo &L = t.sub[fi.L];
  const SubInfo &R = t.sub[fi.R];
  const int eL = fi.kind == 0 ? kEdgeE : kEdgeN;
  const int eR = fi.kind == 0 ? kEdgeW : kEdgeS;
  RowRef rr;
  rr.ncL = L.ncols;
  rr.ncR = R.ncols;
  rr.gL = w.G + L.g_off + static_cast<int64_t>(L.edge_row[eL] + i) * L.ncols;
  rr.gR = w.G + R.g_off + static_cast<int64_t>(R.edge_row[eR] + i) * R.ncols;
  rr.colL = L.edge_col[eL] + i;
  rr.colR = R.edge_col[eR] + i;
  rr.offL = L.col_off;
  rr.offR = R.col_off;
  return rr;
}

// (1) per-interface congruence scaling.  With the flux-continuity (P) rows
// negated the interface matrix is symmetric quasi-definite: S = [-A B; B^T C]
// on every interface block, A and C SPD.  T = blockdiag(L_A^{-1}, L_C^{-1})
// from the Cholesky factors of the interface's own A and C makes the
// diagonal blocks of T S T^T equal to -I and +I, which removes the
// contrast-driven spread of the interface matrix.  Also writes f.
constexpr int kMmax = 32;
__global__ void __launch_bounds__(32) k_iface_prep(DeviceTables t, Workspace w) {
  const int g = blockIdx.x;
  const IfaceInfo fi = t.iface[g];
  const RealInfo &ri = t.real[fi.r];
  const int m = fi.nU + fi.nP;
  __shared__ double Sd[kMmax][kMmax + 1];
  __shared__ double Xd[kMmax][kMmax + 1];
  __shared__ int bad;
  const int i = threadIdx.x;
  if (i == 0) bad = 0;
  if (i < m) {
    const RowRef rr = row_ref(t, w, fi, i);
    const bool pin_i = (fi.unk + i == ri.pin);
    for (int j = 0; j < m; ++j) {
      const bool pin_j = (fi.unk + j == ri.pin);
      double v = rr.gL[rr.colL - i + j] + rr.gR[rr.colR - i + j];
      // A = -M_UU, C = -M_PP (both SPD); U-P coupling not needed here
      const bool same = (i < fi.nU) == (j < fi.nU);
      v = same ? -v : 0.0;
      if (pin_i || pin_j) v = (i == j) ? 1.0 : 0.0;
      Sd[i][j] = v;
    }
    w.f[fi.unk + i] = pin_i ? 0.0 : -(rr.gL[0] + rr.gR[0]);
  }
  __syncwarp();
  // Cholesky of the two diagonal sub-blocks in place (lower), row i per lane
  for (int k = 0; k < m; ++k) {
    const int lo = k < fi.nU ? 0 : fi.nU;      // first index of k's sub-block
    const int hi = k < fi.nU ? fi.nU : m;
    if (i == k) {
      double d = Sd[k][k];
      for (int q = lo; q < k; ++q) d -= Sd[k][q] * Sd[k][q];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      Sd[k][k] = sqrt(d);
    }
    __syncwarp();
    if (i > k && i < hi) {
      double v = Sd[i][k];
      for (int q = lo; q < k; ++q) v -= Sd[i][q] * Sd[k][q];
      Sd[i][k] = v / Sd[k][k];
    }
    __syncwarp();
  }
  // X = L^{-1} (block lower triangular), column j per lane
  if (i < m) {
    const int lo = i < fi.nU ? 0 : fi.nU;
    const int hi = i < fi.nU ? fi.nU : m;
    for (int r = 0; r < m; ++r) Xd[r][i] = 0.0;
    for (int r = lo; r < hi; ++r) {
      if (r < i) continue;
      double v = (r == i) ? 1.0 : 0.0;
      for (int q = i; q < r; ++q) v -= Sd[r][q] * Xd[q][i];
      Xd[r][i] = v / Sd[r][r];
    }
  }
  __syncwarp();
  double *T = w.tsc + fi.tsc_off;
  if (i < m) {
    if (bad) {
      // not quasi-definite: fall back to diagonal scaling
      const RowRef rr = row_ref(t, w, fi, i);
      const double dg = fabs(rr.gL[rr.colL] + rr.gR[rr.colR]);
      for (int j = 0; j < m; ++j) T[i * m + j] = (i == j) ? (dg > 0.0 ? 1.0 / sqrt(dg) : 1.0) : 0.0;
    } else {
      for (int j = 0; j < m; ++j) T[i * m + j] = Xd[i][j];
    }
  }
  if (i == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
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
template <typename T>
__device__ void smem_gj_inverse(T *M, int b, int *bad) {
  // in-place Gauss-Jordan inverse, no pivoting (quasi-definite pivots)
  __shared__ T colk[kBmax], rowk[kBmax];
  __shared__ T piv;
  for (int k = 0; k < b; ++k) {
    for (int i = threadIdx.x; i < b; i += blockDim.x) {
      colk[i] = M[i * b + k];
      rowk[i] = M[k * b + i];
    }
    if (threadIdx.x == 0) {
      piv = M[k * b + k];
      if (!(piv != T(0)) || !isfinite(static_cast<double>(piv))) *bad = 1;
    }
    __syncthreads();
    const T ip = T(1) / piv;
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e / b, j = e % b;
      T nv;
      if (i == k && j == k) nv = ip;
      else if (i == k) nv = rowk[j] * ip;
      else if (j == k) nv = -colk[i] * ip;
      else nv = M[e] - colk[i] * rowk[j] * ip;
      M[e] = nv;
    }
    __syncthreads();
  }
}

// C = beta*C + alpha * A B, all b x b row-major in shared memory; 4x4
// register tiles per thread.
template <typename T>
__device__ void smem_gemm(T *C, const T *A, const T *B, int b, T alpha, bool accumulate) {
  const int nt = (b + 3) / 4;
  for (int tile = threadIdx.x; tile < nt * nt; tile += blockDim.x) {
    const int i0 = (tile / nt) * 4, j0 = (tile % nt) * 4;
    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
    for (int k = 0; k < b; ++k) {
      T av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = (i0 + p < b) ? A[(i0 + p) * b + k] : T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = (j0 + q < b) ? B[k * b + j0 + q] : T(0);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += av[p] * bv[q];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (i0 + p < b && j0 + q < b) {
          T *c = C + (i0 + p) * b + j0 + q;
          *c = accumulate ? *c + alpha * acc[p][q] : alpha * acc[p][q];
        }
      }
  }
}

template <typename T>
__device__ void load_blk(T *dst, const T *src, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}
template <typename T>
__device__ void store_blk(T *dst, const T *src, int n) {
  for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
}

// invert the pivot blocks of the slabs eliminated at this level
// (k = stride*(2i+1)); with stride = 0 inverts slab 0 (the root).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bcr_inv(DeviceTables t, Workspace w, int stride) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T *M = reinterpret_cast<T *>(smraw);
  __shared__ int bad;
  const RealInfo ri = t.real[blockIdx.y];
  const int k = stride == 0 ? (blockIdx.x == 0 ? 0 : ri.nslab) : stride * (2 * blockIdx.x + 1);
  if (k >= ri.nslab) return;
  const int b = ri.bmax;
  const int64_t bb = static_cast<int64_t>(b) * b;
  T *B = static_cast<T *>(w.slabB) + ri.slab_off + k * bb;
  if (threadIdx.x == 0) bad = 0;
  load_blk(M, B, static_cast<int>(bb));
  __syncthreads();
  smem_gj_inverse(M, b, &bad);
  store_blk(B, M, static_cast<int>(bb));
  if (threadIdx.x == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
}

// eliminate the odd neighbours of the surviving slabs k = 2*stride*i
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bcr_update(DeviceTables t, Workspace w, int stride,
                                                        int lev) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const RealInfo ri = t.real[blockIdx.y];
  const int k = 2 * stride * blockIdx.x;
  if (k >= ri.nslab) return;
  const int b = ri.bmax;
  const int bb = b * b;
  T *M1 = reinterpret_cast<T *>(smraw);
  T *M2 = M1 + bb;
  T *M3 = M2 + bb;
  T *M4 = M3 + bb;
  T *Bs = static_cast<T *>(w.slabB) + ri.slab_off;
  T *As = static_cast<T *>(w.slabA) + ri.slab_off;
  T *Cs = static_cast<T *>(w.slabC) + ri.slab_off;
  T *X = static_cast<T *>(w.X) + ri.xy_off + (static_cast<int64_t>(lev) * ri.nslab + k) * bb;
  T *Y = static_cast<T *>(w.Y) + ri.xy_off + (static_cast<int64_t>(lev) * ri.nslab + k) * bb;
  const int l = k - stride, rt = k + stride;
  load_blk(M4, Bs + static_cast<int64_t>(k) * bb, bb);
  if (l >= 0) {
    // X = A_k Binv_l ; B_k -= X C_l ; A_k <- -X A_l
    load_blk(M1, As + static_cast<int64_t>(k) * bb, bb);
    load_blk(M2, Bs + static_cast<int64_t>(l) * bb, bb);
    __syncthreads();
    smem_gemm(M3, M1, M2, b, T(1), false);
    __syncthreads();
    store_blk(X, M3, bb);
    load_blk(M1, Cs + static_cast<int64_t>(l) * bb, bb);
    __syncthreads();
    smem_gemm(M4, M3, M1, b, T(-1), true);
    __syncthreads();
    load_blk(M1, As + static_cast<int64_t>(l) * bb, bb);
    __syncthreads();
    smem_gemm(M2, M3, M1, b, T(-1), false);
    __syncthreads();
    store_blk(As + static_cast<int64_t>(k) * bb, M2, bb);
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < bb; e += blockDim.x) X[e] = T(0);
  }
  if (rt < ri.nslab) {
    // Y = C_k Binv_rt ; B_k -= Y A_rt ; C_k <- -Y C_rt
    load_blk(M1, Cs + static_cast<int64_t>(k) * bb, bb);
    load_blk(M2, Bs + static_cast<int64_t>(rt) * bb, bb);
    __syncthreads();
    smem_gemm(M3, M1, M2, b, T(1), false);
    __syncthreads();
    store_blk(Y, M3, bb);
    load_blk(M1, As + static_cast<int64_t>(rt) * bb, bb);
    __syncthreads();
    smem_gemm(M4, M3, M1, b, T(-1), true);
    __syncthreads();
    load_blk(M1, Cs + static_cast<int64_t>(rt) * bb, bb);
    __syncthreads();
    smem_gemm(M2, M3, M1, b, T(-1), false);
    __syncthreads();
    store_blk(Cs + static_cast<int64_t>(k) * bb, M2, bb);
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < bb; e += blockDim.x) Y[e] = T(0);
  }
  __syncthreads();
  store_blk(Bs + static_cast<int64_t>(k) * bb, M4, bb);
}

// ------------------------------------------------------------ BCR solve
// y = M_scaled^{-1} z for one realisation, by one CTA; z and y are
// slab-padded vectors in shared memory (tmp: scratch of the same size).
template <typename T>
__device__ void bcr_solve_cta(const DeviceTables &t, const Workspace &w, const RealInfo &ri, T *v,
                              T *tmp) {
  const int K = ri.nslab, b = ri.bmax;
  const int64_t bb = static_cast<int64_t>(b) * b;
  const T *Bs = static_cast<const T *>(w.slabB) + ri.slab_off;
  const T *As = static_cast<const T *>(w.slabA) + ri.slab_off;
  const T *Cs = static_cast<const T *>(w.slabC) + ri.slab_off;
  const T *X = static_cast<const T *>(w.X) + ri.xy_off;
  const T *Y = static_cast<const T *>(w.Y) + ri.xy_off;
  // forward: v_k -= X_lev(k) v_{k-stride} + Y_lev(k) v_{k+stride}
  for (int lev = 0, stride = 1; lev < ri.nlev; ++lev, stride <<= 1) {
    const int nk = (K + 2 * stride - 1) / (2 * stride);
    for (int o = threadIdx.x; o < nk * b; o += blockDim.x) {
      const int k = (o / b) * 2 * stride, i = o % b;
      T acc = T(0);
      if (k - stride >= 0) {
        const T *Xk = X + (static_cast<int64_t>(lev) * K + k) * bb + static_cast<int64_t>(i) * b;
        const T *vl = v + (k - stride) * b;
        for (int j = 0; j < b; ++j) acc += Xk[j] * vl[j];
      }
      if (k + stride < K) {
        const T *Yk = Y + (static_cast<int64_t>(lev) * K + k) * bb + static_cast<int64_t>(i) * b;
        const T *vr = v + (k + stride) * b;
        for (int j = 0; j < b; ++j) acc += Yk[j] * vr[j];
      }
      tmp[k * b + i] = v[k * b + i] - acc;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nk * b; o += blockDim.x) {
      const int k = (o / b) * 2 * stride, i = o % b;
      v[k * b + i] = tmp[k * b + i];
    }
    __syncthreads();
  }
  // root
  for (int i = threadIdx.x; i < b; i += blockDim.x) {
    const T *Bi = Bs + static_cast<int64_t>(i) * b;
    T acc = T(0);
    for (int j = 0; j < b; ++j) acc += Bi[j] * v[j];
    tmp[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < b; i += blockDim.x) v[i] = tmp[i];
  __syncthreads();
  // backward: x_k = Binv_k (v_k - A_k x_{k-stride} - C_k x_{k+stride})
  for (int lev = ri.nlev - 1; lev >= 0; --lev) {
    const int stride = 1 << lev;
    const int nk = (K - stride + 2 * stride - 1) / (2 * stride);
    for (int o = threadIdx.x; o < nk * b; o += blockDim.x) {
      const int k = stride + (o / b) * 2 * stride, i = o % b;
      if (k >= K) continue;
      T acc = v[k * b + i];
      const T *Ak = As + k * bb + static_cast<int64_t>(i) * b;
      const T *xl = v + (k - stride) * b;
      for (int j = 0; j < b; ++j) acc -= Ak[j] * xl[j];
      if (k + stride < K) {
        const T *Ck = Cs + k * bb + static_cast<int64_t>(i) * b;
        const T *xr = v + (k + stride) * b;
        for (int j = 0; j < b; ++j) acc -= Ck[j] * xr[j];
      }
      tmp[k * b + i] = acc;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nk * b; o += blockDim.x) {
      const int k = stride + (o / b) * 2 * stride, i = o % b;
      if (k >= K) continue;
      const T *Bk = Bs + k * bb + static_cast<int64_t>(i) * b;
      const T *tk = tmp + k * b;
      T acc = T(0);
      for (int j = 0; j < b; ++j) acc += Bk[j] * tk[j];
      v[k * b + i] = acc;
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
static cudaError_t bcr_factor_t(const DeviceTables &t, const Workspace &w, int maxslab, int bmax,
                                int nlev, int *nlaunch, cudaStream_t st) {
  const size_t bb = static_cast<size_t>(bmax) * bmax * sizeof(T);
  for (int lev = 0, stride = 1; lev < nlev; ++lev, stride <<= 1) {
    const int nodd = (maxslab + 2 * stride - 1 - stride) / (2 * stride);
    if (nodd > 0) {
      k_bcr_inv<T><<<dim3(nodd, t.n_real), kThreads, bb, st>>>(t, w, stride);
      ++*nlaunch;
    }
    const int neven = (maxslab + 2 * stride - 1) / (2 * stride);
    k_bcr_update<T><<<dim3(neven, t.n_real), kThreads, 4 * bb, st>>>(t, w, stride, lev);
    ++*nlaunch;
  }
  k_bcr_inv<T><<<dim3(1, t.n_real), kThreads, bb, st>>>(t, w, 0);
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
  if (prec == MRCM_PREC_FP64) return bcr_factor_t<double>(t, w, maxslab, bmax, nlev, nlaunch, st);
  return bcr_factor_t<float>(t, w, maxslab, bmax, nlev, nlaunch, st);
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
  const int bb = bmax * bmax * static_cast<int>(sizeof(T));
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_bcr_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bb)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_bcr_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                4 * bb)) != cudaSuccess)
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
