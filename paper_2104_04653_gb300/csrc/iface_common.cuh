// Device helpers shared by the interface kernels (iface.cu and
// iface_cluster.cu): G-row references, the per-interface congruence scaling
// and small reductions.
#pragma once
#include "mrcm_internal.h"
#include "../../include/mrcm.h"

namespace mrcm {
namespace {

constexpr int kMmax = 32;

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
  RowRef rr;
  rr.ncL = L.ncols;
  rr.ncR = R.ncols;
  rr.gL = w.G + L.g_off + static_cast<int64_t>(fi.rowL + i) * L.ncols;
  rr.gR = w.G + R.g_off + static_cast<int64_t>(fi.rowR + i) * R.ncols;
  rr.colL = fi.colL + i;
  rr.colR = fi.colR + i;
  rr.offL = L.col_off;
  rr.offR = R.col_off;
  return rr;
}

// (1) per-interface congruence scaling.  With the flux-continuity (P) rows
// negated the interface matrix is symmetric quasi-definite: S = [-A B; B^T C]
// on every interface block, A and C SPD.  T = blockdiag(L_A^{-1}, L_C^{-1})
// from the Cholesky factors of the interface's own A and C makes the
// diagonal blocks of T S T^T equal to -I and +I, which removes the
// contrast-driven spread of the interface matrix.
//
// iface_scale_core: executed by one full warp.  On entry Sd (m rows, leading
// dimension ld >= m + 1) holds A in [0,nU)^2 and C in [nU,m)^2 (zero
// elsewhere; a pinned unknown has a unit diagonal and a zero row and
// column).  Writes T (m x m, row-major) to Tout; returns nonzero if a pivot
// was not positive (T is then left for the caller to replace).  The
// reciprocal square roots come from rsqrtf plus one FP64 Newton step: no
// FP64 divide or square root, which are very slow on this part; any accurate
// scaling works, the same T is used everywhere.
__device__ __forceinline__ double rsqrt_accurate(double d) {
  double y = static_cast<double>(rsqrtf(static_cast<float>(d)));
  return y * (1.5 - 0.5 * d * y * y);
}
__device__ __forceinline__ float rsqrt_accurate(float d) { return rsqrtf(d); }

template <typename R>
__device__ int iface_scale_core(R *Sd_, R *Xd_, int ld, int m, int nU, R *Tout) {
  const int i = threadIdx.x & 31;
  int bad = 0;
#define Sd(r_, c_) Sd_[(r_) * ld + (c_)]
#define Xd(r_, c_) Xd_[(r_) * ld + (c_)]
  __syncwarp();
  const int dcol = ld - 1;                     // spare column: 1/L_kk
  for (int k = 0; k < m; ++k) {
    const int lo = k < nU ? 0 : nU;            // first index of k's sub-block
    const int hi = k < nU ? nU : m;
    if (i == k) {
      R d = Sd(k, k);
      for (int q = lo; q < k; ++q) d -= Sd(k, q) * Sd(k, q);
      if (!(d > R(0)) || !isfinite(static_cast<double>(d))) {
        bad = 1;
        d = R(1);
      }
      const R y = rsqrt_accurate(d);
      Sd(k, k) = d * y;                        // sqrt(d)
      Sd(k, dcol) = y;                         // 1/sqrt(d)
    }
    __syncwarp();
    if (i > k && i < hi) {
      R v = Sd(i, k);
      for (int q = lo; q < k; ++q) v -= Sd(i, q) * Sd(k, q);
      Sd(i, k) = v * Sd(k, dcol);
    }
    __syncwarp();
  }
  // X = L^{-1} (block lower triangular), column j per lane
  if (i < m) {
    const int lo = i < nU ? 0 : nU;
    const int hi = i < nU ? nU : m;
    for (int r = 0; r < m; ++r) Xd(r, i) = R(0);
    for (int r = lo; r < hi; ++r) {
      if (r < i) continue;
      R v = (r == i) ? R(1) : R(0);
      for (int q = i; q < r; ++q) v -= Sd(r, q) * Xd(q, i);
      Xd(r, i) = v * Sd(r, dcol);
    }
  }
  __syncwarp();
  bad = __any_sync(0xffffffffu, bad);
  if (i < m)
    for (int j = 0; j < m; ++j) Tout[i * m + j] = Xd(i, j);
  __syncwarp();
#undef Sd
#undef Xd
  return bad;
}

// Scaling of interface g from its G rows (multi-kernel path); also writes f.
__device__ void iface_scale_warp(const DeviceTables &t, const Workspace &w, int g, double *Sd_,
                                 double *Xd_, int ld) {
  const IfaceInfo fi = t.iface[g];
  const RealInfo &ri = t.real[fi.r];
  const int m = fi.nU + fi.nP;
  const int i = threadIdx.x & 31;
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
      Sd_[i * ld + j] = v;
    }
    w.f[fi.unk + i] = pin_i ? 0.0 : -(rr.gL[0] + rr.gR[0]);
  }
  double *T = w.tsc + fi.tsc_off;
  const int bad = iface_scale_core(Sd_, Xd_, ld, m, fi.nU, T);
  if (bad) {
    // not quasi-definite: fall back to diagonal scaling
    if (i < m) {
      const RowRef rr = row_ref(t, w, fi, i);
      const double dg = fabs(rr.gL[rr.colL] + rr.gR[rr.colR]);
      const double sc = dg > 0.0 ? static_cast<double>(rsqrtf(static_cast<float>(dg))) : 1.0;
      for (int j = 0; j < m; ++j) T[i * m + j] = (i == j) ? sc : 0.0;
    }
    if (i == 0) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
  }
  __syncwarp();
}

__device__ __forceinline__ float fast_recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_recip(double x) { return 1.0 / x; }

// In-place Gauss-Jordan inverse of the b x b shared matrix M (row stride
// ld, b <= 64), no pivoting, by NT threads, in blocks of 8 pivots: warp 0
// inverts the 8 x 8 pivot block in registers (shuffles) while the others
// copy the pivot column panel; then the pivot row panel is formed and the
// rest of the matrix gets a rank-8 update.  scr: 64 + 2*512 elements of T.
// The pivot rows are written in their own loop: fusing them into the update
// loop was mis-compiled at -O3 (wrong results, correct at -G).
template <typename T, int NT>
__device__ void gj_inverse_blocked(T *M, int b, int ld, T *scr, int *bad) {
  T *Pi = scr, *ColP = scr + 64, *RowP = ColP + 64 * 8;
  const int t = threadIdx.x;
  const int nblk = (b + 7) >> 3;
  for (int K = 0; K < nblk; ++K) {
    const int k0 = 8 * K, kb = (b - k0) < 8 ? (b - k0) : 8;
    if (t < 32) {
      const int r = t >> 3, c = t & 7;   // lane holds (r, c) and (r + 4, c)
      T e0 = (r < kb && c < kb) ? M[(k0 + r) * ld + k0 + c] : T(r == c);
      T e1 = (r + 4 < kb && c < kb) ? M[(k0 + r + 4) * ld + k0 + c] : T(r + 4 == c);
      for (int p = 0; p < kb; ++p) {
        const int src = (p & 3) * 8;
        const T ro = __shfl_sync(0xffffffffu, p < 4 ? e0 : e1, src + c);
        const T pv = __shfl_sync(0xffffffffu, p < 4 ? e0 : e1, src + p);
        const T c0 = __shfl_sync(0xffffffffu, e0, r * 8 + p);
        const T c1 = __shfl_sync(0xffffffffu, e1, r * 8 + p);
        if (t == 0 && (!(pv != T(0)) || !isfinite(static_cast<double>(pv)))) *bad = 1;
        const T ip = fast_recip(pv);
        const T rv = ro * ip;
        T n0 = e0 - c0 * rv, n1 = e1 - c1 * rv;
        n0 = (c == p) ? -c0 * ip : n0;
        n1 = (c == p) ? -c1 * ip : n1;
        n0 = (r == p) ? ((c == p) ? ip : rv) : n0;
        n1 = (r + 4 == p) ? ((c == p) ? ip : rv) : n1;
        e0 = n0;
        e1 = n1;
      }
      Pi[r * 8 + c] = e0;
      Pi[(r + 4) * 8 + c] = e1;
    } else {
      for (int e = t - 32; e < 64 * 8; e += NT - 32) {
        const int i = e >> 3, p = e & 7;
        ColP[e] = (i < b && p < kb) ? M[i * ld + k0 + p] : T(0);
      }
    }
    __syncthreads();
    for (int e = t; e < 8 * 64; e += NT) {
      const int q = e >> 6, j = e & 63;
      T a = T(0);
      if (q < kb && j < b) {
#pragma unroll
        for (int p = 0; p < 8; ++p)
          if (p < kb) a += Pi[q * 8 + p] * M[(k0 + p) * ld + j];
      }
      RowP[e] = a;
    }
    __syncthreads();
    // pivot rows: M[K, :] = RowP, M[K, K] = Pinv
    for (int e = t; e < 8 * 64; e += NT) {
      const int q = e >> 6, j = e & 63;
      if (q < kb && j < b)
        M[(k0 + q) * ld + j] = (j >= k0 && j < k0 + kb) ? Pi[q * 8 + (j - k0)] : RowP[e];
    }
    // other rows: rank-kb update, and -M[i,K] Pinv in the pivot columns
    for (int i0 = 0; i0 < 64; i0 += NT >> 3) {
      const int i = i0 + (t >> 3);
      if (i >= b || (i >= k0 && i < k0 + kb)) continue;
      T cp[8];
#pragma unroll
      for (int p = 0; p < 8; ++p) cp[p] = ColP[i * 8 + p];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int j = (t & 7) + 8 * c;
        if (j >= b) continue;
        T a;
        if (c == K) {
          a = T(0);
#pragma unroll
          for (int p = 0; p < 8; ++p) a -= cp[p] * Pi[p * 8 + (t & 7)];
        } else {
          a = M[i * ld + j];
#pragma unroll
          for (int p = 0; p < 8; ++p) a -= cp[p] * RowP[p * 64 + j];
        }
        M[i * ld + j] = a;
      }
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace
}  // namespace mrcm
