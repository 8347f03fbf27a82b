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

__device__ __forceinline__ RowRef row_ref(const DeviceTables &t, const Workspace &w, int u) {
  const int gi = t.unk_iface[u];
  const IfaceInfo fi = t.iface[gi];
  const int i = u - fi.unk;
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

// (1) scaling, right-hand side and padding identity, one thread per padded
// slab position of every realisation.
template <typename T>
__global__ void k_iface_diag(DeviceTables t, Workspace w, const int *pos2unk, int64_t npos,
                             const int64_t *pos_real_off, int nreal) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= npos) return;
  // realisation of this position (npos is small; linear search is fine)
  int r = 0;
  while (r + 1 < nreal && pos_real_off[r + 1] <= p) ++r;
  const RealInfo ri = t.real[r];
  const int64_t lp = p - pos_real_off[r];
  const int slab = static_cast<int>(lp / ri.bmax), pos = static_cast<int>(lp % ri.bmax);
  T *B = static_cast<T *>(w.slabB) + ri.slab_off + static_cast<int64_t>(slab) * ri.bmax * ri.bmax;
  const int u = pos2unk[p];
  if (u < 0 || u == ri.pin) {
    B[pos * ri.bmax + pos] = T(1);
    if (u >= 0) {
      w.dscale[u] = 1.0;
      w.f[u] = 0.0;
    }
    return;
  }
  const RowRef rr = row_ref(t, w, u);
  const double dg = rr.gL[rr.colL] + rr.gR[rr.colR];
  const double ad = fabs(dg);
  w.dscale[u] = ad > 0.0 ? 1.0 / sqrt(ad) : 1.0;
  if (!(ad > 0.0) || !isfinite(ad)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
  w.f[u] = -(rr.gL[0] + rr.gR[0]);
}

// (2) scaled block-tridiagonal slab matrix, one thread per interface row.
template <typename T>
__global__ void k_iface_assemble(DeviceTables t, Workspace w) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= t.nunk) return;
  const IfaceInfo fi = t.iface[t.unk_iface[u]];
  const RealInfo ri = t.real[fi.r];
  if (u == ri.pin) return;
  const RowRef rr = row_ref(t, w, u);
  const int sp = t.unk_slabpos[u];
  const int slab = sp / ri.bmax, row = sp % ri.bmax;
  const double du = w.dscale[u];
  const int64_t bb = static_cast<int64_t>(ri.bmax) * ri.bmax;
  T *Bs = static_cast<T *>(w.slabB) + ri.slab_off;
  T *As = static_cast<T *>(w.slabA) + ri.slab_off;
  T *Cs = static_cast<T *>(w.slabC) + ri.slab_off;
  for (int side = 0; side < 2; ++side) {
    const double *gr = side == 0 ? rr.gL : rr.gR;
    const int nc = side == 0 ? rr.ncL : rr.ncR;
    const int off = side == 0 ? rr.offL : rr.offR;
    for (int c = 1; c < nc; ++c) {
      const int v = t.col[off + c].unk;
      if (v == ri.pin) continue;
      const int vsp = t.unk_slabpos[v];
      const int vs = vsp / ri.bmax, vc = vsp % ri.bmax;
      const double val = gr[c] * du * w.dscale[v];
      T *blk;
      if (vs == slab) blk = Bs + slab * bb;
      else if (vs == slab - 1) blk = As + slab * bb;
      else if (vs == slab + 1) blk = Cs + slab * bb;
      else {
        atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
        continue;
      }
      blk[row * ri.bmax + vc] += static_cast<T>(val);
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
// Cooperative kernel: residual of all realisations by the whole grid, then
// one CTA per realisation checks convergence and applies the BCR solve.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_iface_solve(DeviceTables t, Workspace w,
                                                         const int *pos2unk, double tol,
                                                         int max_solves) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[kThreads / 32];
  __shared__ double s_rel;
  const int nthreads = gridDim.x * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  int nsolve = 0;
  for (int sweep = 0;; ++sweep) {
    // phase 1: r = f - M x (FP64), from the two G rows of every unknown
    for (int u = gtid; u < t.nunk; u += nthreads) {
      const IfaceInfo fi = t.iface[t.unk_iface[u]];
      const RealInfo &ri = t.real[fi.r];
      double s = 0.0;
      if (u != ri.pin) {
        const RowRef rr = row_ref(t, w, u);
        s = w.f[u];
        for (int c = 1; c < rr.ncL; ++c) s -= rr.gL[c] * w.x[t.col[rr.offL + c].unk];
        for (int c = 1; c < rr.ncR; ++c) s -= rr.gR[c] * w.x[t.col[rr.offR + c].unk];
      }
      w.r[u] = s;
    }
    grid.sync();
    // phase 2: per realisation
    for (int r = blockIdx.x; r < t.n_real; r += gridDim.x) {
      const RealInfo ri = t.real[r];
      if (w.done[r]) continue;
      double rn = 0.0, fn = 0.0;
      for (int u = ri.unk0 + threadIdx.x; u < ri.unk0 + ri.nunk; u += blockDim.x) {
        rn += w.r[u] * w.r[u];
        fn += w.f[u] * w.f[u];
      }
      for (int pass = 0; pass < 2; ++pass) {
        double v = pass == 0 ? rn : fn;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
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
                        (nsolve > 2 && rel > 0.5 * prev);
      if (stop) {
        if (threadIdx.x == 0) {
          w.done[r] = 1;
          atomic_max_pos_double(&w.dstat[1], rel);
          atomicMax(&w.status[2], nsolve > 0 ? nsolve - 1 : 0);
          if (!(rel <= tol)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_STALL);
        }
        continue;
      }
      // z = D r (slab padded), y = M_s^{-1} z, x += D y
      T *v = reinterpret_cast<T *>(smraw);
      T *tmp = v + ri.nslab * ri.bmax;
      const int np = ri.nslab * ri.bmax;
      for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int u = pos2unk[ri.vec_off + p];
        v[p] = (u >= 0 && u != ri.pin) ? static_cast<T>(w.dscale[u] * w.r[u]) : T(0);
      }
      __syncthreads();
      bcr_solve_cta(t, w, ri, v, tmp);
      for (int p = threadIdx.x; p < np; p += blockDim.x) {
        const int u = pos2unk[ri.vec_off + p];
        if (u >= 0 && u != ri.pin) w.x[u] += w.dscale[u] * static_cast<double>(v[p]);
      }
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
  const int nb2 = (t.nunk + thr - 1) / thr;
  if (prec == MRCM_PREC_FP64) {
    k_iface_diag<double><<<nb1, thr, 0, st>>>(t, w, pos2unk, npos, pos_real_off, t.n_real);
    k_iface_assemble<double><<<nb2, thr, 0, st>>>(t, w);
  } else {
    k_iface_diag<float><<<nb1, thr, 0, st>>>(t, w, pos2unk, npos, pos_real_off, t.n_real);
    k_iface_assemble<float><<<nb2, thr, 0, st>>>(t, w);
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
