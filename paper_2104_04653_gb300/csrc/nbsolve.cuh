// The interface matrix of Eq. "mrc2" restricted to one interface's
// neighbourhood, and the columns of its inverse that belong to that
// interface, in FP64.  Shared by the learned preconditioner's training
// targets (learned.cu) and the neighbourhood preconditioner of the
// interface GMRES (iface_gmres.cu).
//
// The neighbourhood N(g) of interface g: the interfaces with a subdomain
// within one subdomain (Chebyshev distance) of g's two subdomains, listed in
// increasing index order (nb_list[nb_off[g] ..]).  Its unknowns are ordered
// interface by interface; loc[q] is the first local unknown of the q-th
// neighbour.  A pinned unknown (pure-Neumann realisation) gets an identity
// row and column.
#pragma once

#include "mrcm_internal.h"

namespace mrcm {

// Assemble A = M_N (n x n, leading dimension ld = n + m) with the m unit
// columns of g's unknowns appended, then eliminate with partial pivoting and
// back-substitute: on return (bad = false) A[:, n .. n + m) holds the m
// columns of A^{-1} at g's unknowns.  If mgg is not null the (g, g) block of
// M_N (m x m) is copied there before the elimination.  All threads of the
// CTA take part; loc has room for nh + 1 entries; n and pos_g (g's first
// local unknown) are set by thread 0 and valid for every thread on return.
__device__ inline bool nb_inverse_columns(const DeviceTables &t, const Workspace &w,
                                          const GmRow *grow, const int *nb_list, int h0, int nh,
                                          int g, double *A, double *mgg, int *loc, int *s_n,
                                          int *s_pos, int *s_piv, int *s_bad) {
  const IfaceInfo fg = t.iface[g];
  const int m = fg.nU + fg.nP;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int q = 0; q < nh; ++q) {
      loc[q] = o;
      const IfaceInfo fh = t.iface[nb_list[h0 + q]];
      if (nb_list[h0 + q] == g) *s_pos = o;
      o += fh.nU + fh.nP;
    }
    loc[nh] = o;
    *s_n = o;
    *s_bad = 0;
  }
  __syncthreads();
  const int n = *s_n, ld = n + m, pos_g = *s_pos;
  const int pin = t.real[fg.r].pin;
  for (int e = threadIdx.x; e < n * ld; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  for (int row = threadIdx.x; row < n; row += blockDim.x) {
    int q = 0;
    while (loc[q + 1] <= row) ++q;
    const IfaceInfo fh = t.iface[nb_list[h0 + q]];
    const int u = fh.unk + (row - loc[q]);
    double *Ar = A + static_cast<size_t>(row) * ld;
    if (u == pin) {
      Ar[row] = 1.0;
    } else {
      const GmRow R = grow[u];
      for (int side = 0; side < 2; ++side) {
        const double *gr = w.G + (side ? R.gR : R.gL);
        const ColInfo *cl = t.col + (side ? R.cR : R.cL);
        const int nc = side ? R.nR : R.nL;
        for (int c = 0; c < nc; ++c) {
          const int v = cl[c].unk;
          if (v == pin) continue;
          const int hv = t.unk_iface[v];
          int qq = -1;
          for (int z = 0; z < nh; ++z)
            if (nb_list[h0 + z] == hv) {
              qq = z;
              break;
            }
          if (qq < 0) continue;
          Ar[loc[qq] + (v - t.iface[hv].unk)] += gr[c];
        }
      }
    }
    if (row >= pos_g && row < pos_g + m) Ar[n + row - pos_g] = 1.0;
  }
  __syncthreads();
  if (mgg)
    for (int e = threadIdx.x; e < m * m; e += blockDim.x)
      mgg[e] = A[static_cast<size_t>(pos_g + e / m) * ld + pos_g + e % m];
  // forward elimination with partial pivoting
  for (int p = 0; p < n; ++p) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = p;
      for (int r = p + threadIdx.x; r < n; r += 32) {
        const double v = fabs(A[static_cast<size_t>(r) * ld + p]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        *s_piv = bi;
        if (!(best > 0.0) || !isfinite(best)) *s_bad = 1;
      }
    }
    __syncthreads();
    if (*s_bad) break;
    const int pr = *s_piv;
    if (pr != p)
      for (int c = threadIdx.x; c < ld; c += blockDim.x) {
        const double tmp = A[static_cast<size_t>(p) * ld + c];
        A[static_cast<size_t>(p) * ld + c] = A[static_cast<size_t>(pr) * ld + c];
        A[static_cast<size_t>(pr) * ld + c] = tmp;
      }
    __syncthreads();
    const double ip = 1.0 / A[static_cast<size_t>(p) * ld + p];
    const int rows = n - p - 1, cols = ld - p - 1;
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
      const int r = p + 1 + e / cols, c = p + 1 + e % cols;
      const double f = A[static_cast<size_t>(r) * ld + p] * ip;
      A[static_cast<size_t>(r) * ld + c] -= f * A[static_cast<size_t>(p) * ld + c];
    }
    __syncthreads();
  }
  // back substitution for the m right-hand sides, column-oriented: solve
  // row r, then remove its contribution from every row above in parallel
  if (!*s_bad)
    for (int r = n - 1; r >= 0; --r) {
      if (threadIdx.x < m) {
        double *ar = A + static_cast<size_t>(r) * ld;
        ar[n + threadIdx.x] /= ar[r];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < r * m; e += blockDim.x) {
        const int k = e / m, c = n + e % m;
        A[static_cast<size_t>(k) * ld + c] -=
            A[static_cast<size_t>(k) * ld + r] * A[static_cast<size_t>(r) * ld + c];
      }
      __syncthreads();
    }
  return *s_bad != 0;
}

}  // namespace mrcm
