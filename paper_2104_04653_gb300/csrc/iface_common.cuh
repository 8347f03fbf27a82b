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
// Executed by one full warp; Sd, Xd: shared scratch of m rows with leading
// dimension ld (>= m + 1).
__device__ void iface_scale_warp(const DeviceTables &t, const Workspace &w, int g, double *Sd_,
                                 double *Xd_, int ld) {
  const IfaceInfo fi = t.iface[g];
  const RealInfo &ri = t.real[fi.r];
  const int m = fi.nU + fi.nP;
  const int i = threadIdx.x & 31;
  int bad = 0;
#define Sd(r_, c_) Sd_[(r_) * ld + (c_)]
#define Xd(r_, c_) Xd_[(r_) * ld + (c_)]
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
      Sd(i, j) = v;
    }
    w.f[fi.unk + i] = pin_i ? 0.0 : -(rr.gL[0] + rr.gR[0]);
  }
  __syncwarp();
  // Cholesky of the two diagonal sub-blocks in place (lower), row i per lane
  for (int k = 0; k < m; ++k) {
    const int lo = k < fi.nU ? 0 : fi.nU;      // first index of k's sub-block
    const int hi = k < fi.nU ? fi.nU : m;
    if (i == k) {
      double d = Sd(k, k);
      for (int q = lo; q < k; ++q) d -= Sd(k, q) * Sd(k, q);
      if (!(d > 0.0) || !isfinite(d)) {
        bad = 1;
        d = 1.0;
      }
      Sd(k, k) = sqrt(d);
    }
    __syncwarp();
    if (i > k && i < hi) {
      double v = Sd(i, k);
      for (int q = lo; q < k; ++q) v -= Sd(i, q) * Sd(k, q);
      Sd(i, k) = v / Sd(k, k);
    }
    __syncwarp();
  }
  // X = L^{-1} (block lower triangular), column j per lane
  if (i < m) {
    const int lo = i < fi.nU ? 0 : fi.nU;
    const int hi = i < fi.nU ? fi.nU : m;
    for (int r = 0; r < m; ++r) Xd(r, i) = 0.0;
    for (int r = lo; r < hi; ++r) {
      if (r < i) continue;
      double v = (r == i) ? 1.0 : 0.0;
      for (int q = i; q < r; ++q) v -= Sd(r, q) * Xd(q, i);
      Xd(r, i) = v / Sd(r, r);
    }
  }
  __syncwarp();
  bad = __any_sync(0xffffffffu, bad);
  double *T = w.tsc + fi.tsc_off;
  if (i < m) {
    if (bad) {
      // not quasi-definite: fall back to diagonal scaling
      const RowRef rr = row_ref(t, w, fi, i);
      const double dg = fabs(rr.gL[rr.colL] + rr.gR[rr.colR]);
      for (int j = 0; j < m; ++j) T[i * m + j] = (i == j) ? (dg > 0.0 ? 1.0 / sqrt(dg) : 1.0) : 0.0;
    } else {
      for (int j = 0; j < m; ++j) T[i * m + j] = Xd(i, j);
    }
  }
  if (i == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
  __syncwarp();
#undef Sd
#undef Xd
}


template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace
}  // namespace mrcm
