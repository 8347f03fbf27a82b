// Step (d) of the MRCM solve (Eq. "mrc2") in ONE launch per realisation:
// a thread-block cluster with one CTA per interface slab.
//
// The slabs make the interface matrix block tridiagonal (see iface.cu).  CTA
// k of the cluster owns slab k: it stages its rows of G and its interface
// pairs in shared memory, computes the congruence scaling of its interfaces,
// assembles its scaled diagonal block B_k and couplings A_k, C_k, takes part
// in the block cyclic reduction (odd slabs invert their pivot block,
// surviving slabs read the inverses and couplings of their neighbours
// through distributed shared memory), and keeps its share of the
// factorisation in shared memory for every refinement sweep.  A sweep is:
//   A  x_g += T_g^T y_g            (previous correction; x in FP64 in shared
//                                   memory, written to global memory once)
//   B  r_g = f_g - (M x)_g (FP64), z_g = T_g (sign r_g)
//   C  y = Shat^{-1} z by the cluster's cyclic reduction
// with cluster barriers between the phases; realisations are independent
// clusters, so no grid-wide synchronisation exists.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"
#include "iface_common.cuh"

#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

namespace cg = cooperative_groups;

namespace mrcm {
namespace {

constexpr int kCT = 512;        // threads per CTA
constexpr int kCMaxB = 64;      // largest slab
constexpr int kGjScr = 2 * 64 + 3 * 512;   // Gauss-Jordan scratch (elements): Pi x2, ColP x2, RowP

// FP32 forms of gemm / gemm2 below for b a multiple of 4 (tiles 16-byte
// aligned): four k per step, a 16-byte load of each of the thread's four A
// rows and an 8-byte load of each of the four B rows.  The same products are
// summed in the same order (k ascending) as in the scalar forms.
__device__ __forceinline__ void fma_k4(float (&c)[4][2], const float4 (&a)[4],
                                       const float2 (&bv)[4]) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    c[p][0] = fmaf(a[p].x, bv[0].x, c[p][0]);
    c[p][1] = fmaf(a[p].x, bv[0].y, c[p][1]);
    c[p][0] = fmaf(a[p].y, bv[1].x, c[p][0]);
    c[p][1] = fmaf(a[p].y, bv[1].y, c[p][1]);
    c[p][0] = fmaf(a[p].z, bv[2].x, c[p][0]);
    c[p][1] = fmaf(a[p].z, bv[2].y, c[p][1]);
    c[p][0] = fmaf(a[p].w, bv[3].x, c[p][0]);
    c[p][1] = fmaf(a[p].w, bv[3].y, c[p][1]);
  }
}

__device__ void gemm2_v4(float *C1, float *C2, const float *A, const float *B1, const float *B2,
                         int b, float alpha1, bool acc1, float alpha2, bool acc2, bool two) {
  const int t = threadIdx.x, j0 = 2 * (t & 31), i0 = 4 * (t >> 5);
  if (i0 < b && j0 < b) {   // b % 4 == 0: rows i0..i0+3 and columns j0, j0+1 exist
    float c[4][2] = {}, d[4][2] = {};
    for (int k = 0; k < b; k += 4) {
      float4 a[4];
      float2 bv[4], ev[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = *reinterpret_cast<const float4 *>(A + (i0 + p) * b + k);
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = *reinterpret_cast<const float2 *>(B1 + (k + q) * b + j0);
      fma_k4(c, a, bv);
      if (two) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          ev[q] = *reinterpret_cast<const float2 *>(B2 + (k + q) * b + j0);
        fma_k4(d, a, ev);
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float2 *cr = reinterpret_cast<float2 *>(C1 + (i0 + p) * b + j0);
      float2 o = acc1 ? *cr : make_float2(0.f, 0.f);
      *cr = acc1 ? make_float2(o.x + alpha1 * c[p][0], o.y + alpha1 * c[p][1])
                 : make_float2(alpha1 * c[p][0], alpha1 * c[p][1]);
      if (two) {
        float2 *dr = reinterpret_cast<float2 *>(C2 + (i0 + p) * b + j0);
        float2 od = acc2 ? *dr : make_float2(0.f, 0.f);
        *dr = acc2 ? make_float2(od.x + alpha2 * d[p][0], od.y + alpha2 * d[p][1])
                   : make_float2(alpha2 * d[p][0], alpha2 * d[p][1]);
      }
    }
  }
  __syncthreads();
}

// C = alpha A B (+ C), b x b row-major shared matrices; thread owns rows
// 4*(t/32)..+3, columns 2*(t%32)..+1.  C must not alias A or B.
template <typename T>
__device__ void gemm(T *C, const T *A, const T *B, int b, T alpha, bool acc) {
  if constexpr (std::is_same<T, float>::value) {
    if ((b & 3) == 0) {
      gemm2_v4(C, nullptr, A, B, nullptr, b, alpha, acc, 0.f, false, false);
      return;
    }
  }
  const int t = threadIdx.x, j0 = 2 * (t & 31), i0 = 4 * (t >> 5);
  if (i0 < b && j0 < b) {
    const bool j1ok = j0 + 1 < b;
    T c[4][2] = {};
    for (int k = 0; k < b; ++k) {
      const T b0 = B[k * b + j0];
      const T b1 = j1ok ? B[k * b + j0 + 1] : T(0);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const T a = (i0 + p < b) ? A[(i0 + p) * b + k] : T(0);
        c[p][0] += a * b0;
        c[p][1] += a * b1;
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (i0 + p >= b) continue;
      T *cr = C + (i0 + p) * b + j0;
      cr[0] = acc ? cr[0] + alpha * c[p][0] : alpha * c[p][0];
      if (j1ok) cr[1] = acc ? cr[1] + alpha * c[p][1] : alpha * c[p][1];
    }
  }
  __syncthreads();
}

// dst1 = src1 and dst2 = src2 (n values each, sources may be other CTAs'
// shared memory), both copies in flight together, one barrier
template <typename T>
__device__ void copy_in2(T *dst1, const T *src1, T *dst2, const T *src2, int n) {
  constexpr int U = 4;
  for (int base = threadIdx.x; base < n; base += blockDim.x * U) {
    T v[U], w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      v[u] = e < n ? src1[e] : T(0);
      w[u] = e < n ? src2[e] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < n) {
        dst1[e] = v[u];
        dst2[e] = w[u];
      }
    }
  }
  __syncthreads();
}

// Two products sharing the left operand: C1 = alpha1 A B1 (+ C1 if acc1) and
// C2 = alpha2 A B2 (+ C2 if acc2), one pass over A (same thread layout as gemm)
template <typename T>
__device__ void gemm2(T *C1, T *C2, const T *A, const T *B1, const T *B2, int b, T alpha1,
                      bool acc1, T alpha2, bool acc2) {
  if constexpr (std::is_same<T, float>::value) {
    if ((b & 3) == 0) {
      gemm2_v4(C1, C2, A, B1, B2, b, alpha1, acc1, alpha2, acc2, true);
      return;
    }
  }
  const int t = threadIdx.x, j0 = 2 * (t & 31), i0 = 4 * (t >> 5);
  if (i0 < b && j0 < b) {
    const bool j1ok = j0 + 1 < b;
    T c[4][2] = {}, d[4][2] = {};
    for (int k = 0; k < b; ++k) {
      const T b0 = B1[k * b + j0], e0 = B2[k * b + j0];
      const T b1 = j1ok ? B1[k * b + j0 + 1] : T(0);
      const T e1 = j1ok ? B2[k * b + j0 + 1] : T(0);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const T a = (i0 + p < b) ? A[(i0 + p) * b + k] : T(0);
        c[p][0] += a * b0;
        c[p][1] += a * b1;
        d[p][0] += a * e0;
        d[p][1] += a * e1;
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (i0 + p >= b) continue;
      T *cr = C1 + (i0 + p) * b + j0;
      T *dr = C2 + (i0 + p) * b + j0;
      cr[0] = acc1 ? cr[0] + alpha1 * c[p][0] : alpha1 * c[p][0];
      dr[0] = acc2 ? dr[0] + alpha2 * d[p][0] : alpha2 * d[p][0];
      if (j1ok) {
        cr[1] = acc1 ? cr[1] + alpha1 * c[p][1] : alpha1 * c[p][1];
        dr[1] = acc2 ? dr[1] + alpha2 * d[p][1] : alpha2 * d[p][1];
      }
    }
  }
  __syncthreads();
}

// Two independent products in one pass: C1 = A1 B1 and C2 = A2 B2 (alpha 1,
// no accumulation), each element summed exactly as in gemm.
__device__ void gemm_dual_v4(float *C1, const float *A1, const float *B1, float *C2,
                             const float *A2, const float *B2, int b) {
  const int t = threadIdx.x, j0 = 2 * (t & 31), i0 = 4 * (t >> 5);
  if (i0 < b && j0 < b) {
    float c[4][2] = {}, d[4][2] = {};
    for (int k = 0; k < b; k += 4) {
      float4 a[4], e[4];
      float2 bv[4], ev[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        a[p] = *reinterpret_cast<const float4 *>(A1 + (i0 + p) * b + k);
        e[p] = *reinterpret_cast<const float4 *>(A2 + (i0 + p) * b + k);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        bv[q] = *reinterpret_cast<const float2 *>(B1 + (k + q) * b + j0);
        ev[q] = *reinterpret_cast<const float2 *>(B2 + (k + q) * b + j0);
      }
      fma_k4(c, a, bv);
      fma_k4(d, e, ev);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      *reinterpret_cast<float2 *>(C1 + (i0 + p) * b + j0) = make_float2(c[p][0], c[p][1]);
      *reinterpret_cast<float2 *>(C2 + (i0 + p) * b + j0) = make_float2(d[p][0], d[p][1]);
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void gemm(T *C, const T *A, const T *B, int b, T alpha, bool acc);

template <typename T>
__device__ void gemm_dual(T *C1, const T *A1, const T *B1, T *C2, const T *A2, const T *B2,
                          int b) {
  if constexpr (std::is_same<T, float>::value) {
    if ((b & 3) == 0) {
      gemm_dual_v4(C1, A1, B1, C2, A2, B2, b);
      return;
    }
  }
  gemm(C1, A1, B1, b, T(1), false);
  gemm(C2, A2, B2, b, T(1), false);
}

// dst[0..n) = src[0..n) (src may be another CTA's shared memory): every
// thread issues its eight loads before storing, so a copy costs one
// distributed-shared-memory latency, not eight
template <typename T>
__device__ void copy_in(T *dst, const T *src, int n) {
  constexpr int U = 8;
  for (int base = threadIdx.x; base < n; base += blockDim.x * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      v[u] = e < n ? src[e] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = base + u * blockDim.x;
      if (e < n) dst[e] = v[u];
    }
  }
  __syncthreads();
}

// y = M x for a b x b shared matrix, warp per row
template <typename T>
__device__ void matvec_acc(T *y, const T *M, const T *x, int b, T alpha) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < b; i += nw) {
    T a = T(0);
    for (int j = lane; j < b; j += 32) a += M[i * b + j] * x[j];
    a = warp_sum(a);
    if (lane == 0) y[i] += alpha * a;
  }
}

// The 8 x 8 pivot block at (k0, k0) of M (kb <= 8 rows used, identity
// padding) inverted in registers by one warp (lane holds (r, c) and
// (r + 4, c); shuffles exchange the pivot row and column) into Pi (8 x 8).
template <typename T>
__device__ void gj_pivot_block(const T *M, int ld, int k0, int kb, T *Pi, int *bad) {
  const int lane = threadIdx.x & 31;
  const int r = lane >> 3, c = lane & 7;
  T e0 = (r < kb && c < kb) ? M[(k0 + r) * ld + k0 + c] : T(r == c);
  T e1 = (r + 4 < kb && c < kb) ? M[(k0 + r + 4) * ld + k0 + c] : T(r + 4 == c);
  for (int p = 0; p < kb; ++p) {
    const int src = (p & 3) * 8;
    const T ro = __shfl_sync(0xffffffffu, p < 4 ? e0 : e1, src + c);
    const T pv = __shfl_sync(0xffffffffu, p < 4 ? e0 : e1, src + p);
    const T c0 = __shfl_sync(0xffffffffu, e0, r * 8 + p);
    const T c1 = __shfl_sync(0xffffffffu, e1, r * 8 + p);
    if (lane == 0 && (!(pv != T(0)) || !isfinite(static_cast<double>(pv)))) *bad = 1;
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
}

// Update of rows 0..b-1 of M for the columns j in [c0, c1) that are not in
// the pivot block K (k0, kb): pivot rows take RowP, the others the rank-kb
// update with the column panel CP; columns of block K take -CP Pi.  Threads
// tf .. tf + nt - 1 take part: thread u owns rows (u / 8) + (nt / 8) * n and
// the columns (u % 8) + 8 c of the range.  Same products, same order, as in
// gj_inverse_blocked.
template <typename T>
__device__ void gj_update_cols(T *M, int b, int k0, int kb, const T *CP, const T *Pi,
                               const T *RowP, int c0, int c1, int tf, int nt) {
  const int u = static_cast<int>(threadIdx.x) - tf;
  if (u < 0 || u >= nt) return;
  const int rstep = nt >> 3;
  for (int i = u >> 3; i < b; i += rstep) {
    const bool piv = i >= k0 && i < k0 + kb;
    T cp[8];
    if (!piv) {
#pragma unroll
      for (int p = 0; p < 8; ++p) cp[p] = CP[i * 8 + p];
    }
    for (int j = c0 + (u & 7); j < c1; j += 8) {
      if (j >= b) break;
      const bool kcol = j >= k0 && j < k0 + kb;
      T a;
      if (piv) {
        a = kcol ? Pi[(i - k0) * 8 + (j - k0)] : RowP[(i - k0) * 64 + j];
      } else if (kcol) {
        a = T(0);
#pragma unroll
        for (int p = 0; p < 8; ++p) a -= cp[p] * Pi[p * 8 + (j - k0)];
      } else {
        a = M[i * b + j];
#pragma unroll
        for (int p = 0; p < 8; ++p) a -= cp[p] * RowP[p * 64 + j];
      }
      M[i * b + j] = a;
    }
  }
}

// In-place Gauss-Jordan inverse of the b x b shared matrix M (row stride b,
// b <= 64), no pivoting, in blocks of 8 pivots, by the whole CTA, with one
// block of lookahead: once the columns of block K+1 are updated, warp 0
// inverts the next pivot block while the other warps copy the next column
// panel and update the remaining columns.  Arithmetic per element as in
// gj_inverse_blocked.  scr: kGjScr elements (Pi and ColP double-buffered,
// RowP).
template <typename T>
__device__ void gj_inverse_la(T *M, int b, T *scr, int *bad) {
  T *PiB = scr, *CPB = scr + 128, *RowP = scr + 128 + 1024;
  const int t = threadIdx.x, wid = t >> 5;
  const int nblk = (b + 7) >> 3;
  if (nblk < 1) return;
  // prologue: pivot block 0 (warp 0) and column panel 0 (the other warps)
  if (wid == 0) {
    gj_pivot_block(M, b, 0, b < 8 ? b : 8, PiB, bad);
  } else {
    const int kb = b < 8 ? b : 8;
    for (int e = t - 32; e < 64 * 8; e += kCT - 32) {
      const int i = e >> 3, p = e & 7;
      CPB[e] = (i < b && p < kb) ? M[i * b + p] : T(0);
    }
  }
  __syncthreads();
  for (int K = 0; K < nblk; ++K) {
    const int k0 = 8 * K, kb = (b - k0) < 8 ? (b - k0) : 8;
    const T *Pi = PiB + (K & 1) * 64;
    const T *CP = CPB + (K & 1) * 512;
    // row panel: RowP = Pi M[K rows, :]
    for (int e = t; e < 8 * 64; e += kCT) {
      const int q = e >> 6, j = e & 63;
      T a = T(0);
      if (q < kb && j < b) {
#pragma unroll
        for (int p = 0; p < 8; ++p)
          if (p < kb) a += Pi[q * 8 + p] * M[(k0 + p) * b + j];
      }
      RowP[e] = a;
    }
    __syncthreads();
    if (K + 1 < nblk) {
      const int k1 = k0 + 8, kb1 = (b - k1) < 8 ? (b - k1) : 8;
      // the columns of block K+1, by every thread
      gj_update_cols(M, b, k0, kb, CP, Pi, RowP, k1, k1 + 8, 0, kCT);
      __syncthreads();
      if (wid == 0) {
        gj_pivot_block(M, b, k1, kb1, PiB + ((K + 1) & 1) * 64, bad);
      } else {
        T *CPn = CPB + ((K + 1) & 1) * 512;
        for (int e = t - 32; e < 64 * 8; e += kCT - 32) {
          const int i = e >> 3, p = e & 7;
          CPn[e] = (i < b && p < kb1) ? M[i * b + k1 + p] : T(0);
        }
        gj_update_cols(M, b, k0, kb, CP, Pi, RowP, 0, k1, 32, kCT - 32);
        gj_update_cols(M, b, k0, kb, CP, Pi, RowP, k1 + 8, 64, 32, kCT - 32);
      }
      __syncthreads();
    } else {
      gj_update_cols(M, b, k0, kb, CP, Pi, RowP, 0, 64, 0, kCT);
      __syncthreads();
    }
  }
}

// sum_j M[i][j] x[j] for the row i = threadIdx.x / 8 of the b x b row-major
// shared tile M, by the 8 threads of that row (kCT = 8 kCMaxB threads cover
// every row): each takes every 8th column, in chunks of 8 columns visited in
// an order rotated by the row, so the four rows a warp serves read distinct
// banks; three shuffles add the partial sums.  Every thread of the CTA must
// call it (rows i >= b return 0); every thread of the row gets the sum.
template <typename T>
__device__ __forceinline__ T rowdot8(const T *M, const T *x, int b) {
  const int i = threadIdx.x >> 3, sub = threadIdx.x & 7;
  const int nch = (b + 7) >> 3;
  T a = T(0);
  if (i < b) {
    int cc = i & 3;
    if (cc >= nch) cc = 0;
    for (int c = 0; c < nch; ++c) {
      const int j = 8 * cc + sub;
      if (j < b) a += M[i * b + j] * x[j];
      if (++cc == nch) cc = 0;
    }
  }
  a += __shfl_xor_sync(0xffffffffu, a, 4);
  a += __shfl_xor_sync(0xffffffffu, a, 2);
  a += __shfl_xor_sync(0xffffffffu, a, 1);
  return a;
}
static_assert(kCT == 8 * kCMaxB, "rowdot8 maps 8 threads to each of kCMaxB rows");

template <typename T>
__global__ void __launch_bounds__(kCT, 1)
    k_iface_cluster(DeviceTables t, Workspace w, const int *slab_if, const int *slab_if_off,
                    double tol, int max_solves, int bS, int nlevS) {
  cg::cluster_group cluster = cg::this_cluster();
  const int K = static_cast<int>(cluster.num_blocks());
  const int k = static_cast<int>(cluster.block_rank());
  const int r = blockIdx.x / K;
  const RealInfo ri = t.real[r];
  const int b = ri.bmax, nlev = ri.nlev;
  // tile stride and tile count from the largest slab and level count of
  // the batch, the same for every realisation: the shared-memory layout
  // (and the scratch areas that the plan checks against it) does not
  // shrink with a realisation's own sizes; the stride keeps the FP64 arrays
  // behind the tiles aligned
  const int bb = (bS * bS + 3) & ~3;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kCT / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *tB = reinterpret_cast<T *>(smraw);
  T *tA = tB + bb;
  T *tC = tA + bb;
  T *tW1 = tC + bb;
  T *tW2 = tW1 + bb;
  T *tX = tW2 + bb;             // nlev tiles
  T *tY = tX + nlevS * bb;      // nlev tiles (nlevS reserved)
  T *v = tY + nlevS * bb;       // slab vector (z, then y)
  T *vr1 = v + kCMaxB;
  T *vr2 = vr1 + kCMaxB;
  T *vt = vr2 + kCMaxB;
  T *gjs = vt + kCMaxB;                                   // Gauss-Jordan scratch
  const int E = t.emax, mm = t.mmax;
  double *rl = reinterpret_cast<double *>(gjs + kGjScr);  // FP64 residual of the slab
  double *part = rl + kCMaxB;                             // [2] partial sums
  double *xs = part + 2;                                  // [3 kCMaxB]: x of slabs k-1, k, k+1
  double *fs = xs + 3 * kCMaxB;                           // [kCMaxB] f of the slab rows
  double *Td = fs + kCMaxB;                               // [b][mm] scaling rows (FP64)
  double *rowc = Td + b * mm;                             // [E][b] row coefficients
  short *rowi = reinterpret_cast<short *>(rowc + b * E);  // [E][b] positions in xs
  int *rowcnt = reinterpret_cast<int *>(rowi + ((b * E + 1) & ~1));   // [kCMaxB]
  int *posinf = rowcnt + kCMaxB;   // [kCMaxB] p0 << 16 | m << 8 | i, bit 30 P row, bit 29 pin
  T *Trow = reinterpret_cast<T *>(posinf + kCMaxB);       // [b][mm] scaling rows (working prec.)
  __shared__ int bad;
  __shared__ double red[kCT / 32];
  __shared__ int diagq[kCMaxB];   // pair index of the diagonal block of the interface at p0
  __shared__ int s_goff0, s_goff1; // the slab's range of pair_goff
  const int pa0 = t.pair_off[r * K + k], pa1 = t.pair_off[r * K + k + 1];
  if (tid == 0) {
    bad = 0;
    s_goff0 = t.pairs[pa0].goff;
    s_goff1 = t.pairs[pa1].goff;   // the next slab's first pair, or the sentinel
  }
  const int64_t P0 = ri.vec_off + static_cast<int64_t>(k) * b;   // first slab position

  // ---- the slab's interface rows from the precomputed plans: one gather of G
  for (int p = tid; p < kCMaxB; p += kCT) diagq[p] = -1;
  for (int p = tid; p < b; p += kCT) {
    const int info = t.plan_info[P0 + p];
    posinf[p] = info;
    rowcnt[p] = t.plan_cnt[P0 + p];
    const int f0 = t.plan_fgoff[2 * (P0 + p)], f1 = t.plan_fgoff[2 * (P0 + p) + 1];
    fs[p] = (info >= 0 && f0 >= 0) ? -(w.G[f0] + w.G[f1]) : 0.0;
  }
  // entry-major (term j of row p at j * b + p: the row-per-thread residual
  // reads consecutive words); term positions remapped from [0, 3b) to the
  // three kCMaxB-strided x vectors of xs
  // (eight terms per thread in flight: the offsets, then the values)
  {
    constexpr int U = 8;
    const int n = b * E;
    for (int base = tid; base < n; base += kCT * U) {
      int go[U], xi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * kCT;
        go[u] = e < n ? t.plan_goff[P0 * E + e] : -1;
        xi[u] = e < n ? t.plan_xi[P0 * E + e] : 0;
      }
      double gv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) gv[u] = go[u] >= 0 ? w.G[go[u]] : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = base + u * kCT;
        if (e < n) {
          const int p = e / E, j = e - p * E;
          const int x = xi[u] + (xi[u] >= b ? (xi[u] >= 2 * b ? 2 : 1) : 0) * (kCMaxB - b);
          rowc[j * b + p] = gv[u];
          rowi[j * b + p] = static_cast<short>(x);
        }
      }
    }
  }
  for (int e = tid; e < 3 * kCMaxB; e += kCT) xs[e] = 0.0;
  __syncthreads();
  // ---- the slab's pair plans and the G sums of every pair entry, staged
  // by all threads at once at the end of the tile area (the scaling and the
  // assembly then read no global memory).  The host plan admits the cluster
  // path only where this fits behind both phases' scratch for every slab;
  // otherwise the layout flag is raised and the setup skipped.  The diagonal
  // pairs are found in the same pass.
  const int npair = pa1 - pa0, nst = (s_goff1 - s_goff0) / 2;
  const size_t ppb = (static_cast<size_t>(npair) * sizeof(PairPlan) + 15) & ~static_cast<size_t>(15);
  unsigned char *stage = reinterpret_cast<unsigned char *>(v) - ppb - static_cast<size_t>(nst) * 8;
  PairPlan *pps = reinterpret_cast<PairPlan *>(stage);
  const double *Sst = reinterpret_cast<const double *>(stage + ppb);
  const unsigned char *asm_end = reinterpret_cast<const unsigned char *>(tW1) +
                                 static_cast<size_t>(nw) * 2 * mm * mm * (sizeof(double) + sizeof(T));
  const bool staged = npair >= 0 && nst >= 0 && stage >= asm_end;
  if (!staged && tid == 0) atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
  if (staged) {
    for (int q = pa0 + tid; q < pa1; q += kCT) {
      const PairPlan pp = t.pairs[q];
      pps[q - pa0] = pp;
      if (pp.ds == 0 && pp.pn0 == pp.p0 && pp.p0 >= 0 && pp.p0 < b) diagq[pp.p0] = q;
    }
    {
      constexpr int U = 8;
      double *Sw = reinterpret_cast<double *>(stage + ppb);
      for (int base = tid; base < nst; base += kCT * U) {
        int g0[U], g1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = base + u * kCT;
          g0[u] = e < nst ? t.pair_goff[s_goff0 + 2 * e] : -1;
          g1[u] = e < nst ? t.pair_goff[s_goff0 + 2 * e + 1] : -1;
        }
        double a0[U], a1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          a0[u] = g0[u] >= 0 ? w.G[g0[u]] : 0.0;
          a1[u] = g1[u] >= 0 ? w.G[g1[u]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = base + u * kCT;
          if (e < nst) Sw[e] = a0[u] + a1[u];
        }
      }
    }
  }
  __syncthreads();

  // ---- scaling of this slab's interfaces from their diagonal blocks, one
  // warp per interface, in FP32: any consistent scaling is valid (the same T
  // scales the assembled blocks, the residuals and the corrections), and the
  // FP64 pipe of this part is too slow for a warp-serial Cholesky
  {
    const int ld = mm + 1;
    const int per = 2 * mm * ld + mm * mm;                   // floats per warp
    const size_t area = staged ? static_cast<size_t>(stage - smraw) : 0;
    const int avail = static_cast<int>(area / (sizeof(float) * per));
    const int np = avail < nw ? avail : nw;
    float *scr = reinterpret_cast<float *>(smraw);
    if (np < 1) {
      if (tid == 0) atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
    } else if (wid < np) {
      float *Sd = scr + wid * per, *Xd = Sd + mm * ld, *To = Xd + mm * ld;
      // the slab's interfaces in position order from two ballots over the
      // diagonal-pair table (kCMaxB = 64 entries, -1 where no interface
      // starts); warp wid takes interfaces wid, wid + np, ...
      static_assert(kCMaxB == 64, "two 32-entry ballots cover the table");
      const unsigned m0 = __ballot_sync(0xffffffffu, diagq[lane] >= 0);
      const unsigned m1 = __ballot_sync(0xffffffffu, diagq[lane + 32] >= 0);
      const int n0 = __popc(m0), nif = n0 + __popc(m1);
      for (int n = wid; n < nif; n += np) {
        const int p = n < n0 ? static_cast<int>(__fns(m0, 0, n + 1))
                             : 32 + static_cast<int>(__fns(m1, 0, n - n0 + 1));
        const int q = diagq[p];
        const PairPlan pp = pps[q - pa0];
        const int m = pp.m, nU = pp.nU, p0 = pp.p0;
        const double *Sq = Sst + (pp.goff - s_goff0) / 2;
        // A = -M_UU, C = -M_PP; a pinned unknown gets a unit diagonal
        for (int e = lane; e < m * m; e += 32) {
          const int i = e / m, j = e % m;
          const double val = Sq[e];
          float sv = ((i < nU) == (j < nU)) ? static_cast<float>(-val) : 0.0f;
          if (((posinf[p0 + i] >> 29) & 1) || ((posinf[p0 + j] >> 29) & 1))
            sv = (i == j) ? 1.0f : 0.0f;
          Sd[i * ld + j] = sv;
        }
        const int bd = iface_scale_core(Sd, Xd, ld, m, nU, To);
        if (lane < m) {
          for (int j = 0; j < mm; ++j) {
            float tv = j < m ? To[lane * m + j] : 0.0f;
            if (bd && j < m) tv = (lane == j) ? 1.0f : 0.0f;
            Td[(p0 + lane) * mm + j] = static_cast<double>(tv);
            Trow[(p0 + lane) * mm + j] = static_cast<T>(tv);
          }
        }
        if (bd && lane == 0) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
        __syncwarp();
      }
    }
  }
  cluster.sync();   // every slab's Trow complete (read by its neighbours below)

  // ---- assemble the scaled slab blocks: T_g S_{g g'} T_{g'}^T, one warp
  // per (own, neighbour) interface pair, S from the precomputed G offsets
  for (int e = tid; e < 3 * bb; e += kCT) tB[e] = T(0);
  __syncthreads();
  {
    double *scr = reinterpret_cast<double *>(tW1) + wid * 2 * mm * mm;
    T *scrT = reinterpret_cast<T *>(reinterpret_cast<double *>(tW1) + nw * 2 * mm * mm) +
              wid * 2 * mm * mm;
    // the scratch of all warps ends before v (batch-wide sizes only, so the
    // test has the same outcome in every CTA; the host plan ensures it)
    const bool fits = reinterpret_cast<const unsigned char *>(
                          reinterpret_cast<T *>(reinterpret_cast<double *>(tW1) + nw * 2 * mm * mm) +
                          nw * 2 * mm * mm) <= reinterpret_cast<const unsigned char *>(v);
    if (!fits && tid == 0) atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
    for (int q = pa0 + wid; fits && staged && q < pa1; q += nw) {
      const PairPlan pp = pps[q - pa0];
      const int m = pp.m, mn = pp.mn;
      double *Sb = scr, *Xb = scr + mm * mm;
      const double *Sq = Sst + (pp.goff - s_goff0) / 2;
      for (int e = lane; e < m * mn; e += 32) {
        const int i = e / mn;
        Sb[e] = (i >= pp.nU) ? -Sq[e] : Sq[e];             // symmetrising sign
      }
      __syncwarp();
      T *blk = pp.ds == 0 ? tB : (pp.ds == -1 ? tA : tC);
      if (pp.ds < -1 || pp.ds > 1) {
        if (lane == 0) atomicOr(&w.status[0], MRCM_FLAG_LAYOUT);
        continue;
      }
      const bool own = pp.ds == 0;
      const bool diag = own && pp.pn0 == pp.p0;
      // X = T_g S in FP64 (rounding S or X T^T's left factor to the working
      // precision first costs a refinement sweep); the diagonal block, whose
      // T S T^T = [-I *; * I] cancels, also takes Y = X T^T in FP64, the
      // other blocks in the working precision.  Off the diagonal X and the
      // neighbour's T are rounded once per entry (a conversion from FP64
      // runs on the slow FP64 pipe of this part, so none sits in the inner
      // product loop).
      T *XT = scrT, *TnT = scrT + mm * mm;
      {
        // T_g and T_n are block lower triangular, blockdiag(L_A^-1, L_C^-1):
        // row i of T_g has nonzeros in [lo(i), i], lo = 0 for a flux row and
        // nU for a pressure row (the skipped terms are exact zeros)
        const double *Tg = Td + pp.p0 * mm;
        for (int e = lane; e < m * mn; e += 32) {
          const int i = e / mn, j = e % mn;
          double a = 0.0;
          for (int qq = i < pp.nU ? 0 : pp.nU; qq <= i; ++qq) a += Tg[i * mm + qq] * Sb[qq * mn + j];
          if (diag)
            Xb[e] = a;
          else
            XT[e] = static_cast<T>(a);
        }
        if (!own) {   // the neighbour slab's scaling rows, from its shared memory
          const T *rT = cluster.map_shared_rank(Trow, k + pp.ds) + pp.pn0 * mm;
          for (int e = lane; e < mn * mn; e += 32) TnT[e] = rT[(e / mn) * mm + e % mn];
        }
      }
      __syncwarp();
      if (diag) {
        const double *Tn = Td + pp.pn0 * mm;
        for (int e = lane; e < m * mn; e += 32) {
          const int i = e / mn, j = e % mn;
          double a = 0.0;
          for (int qq = j < pp.nUn ? 0 : pp.nUn; qq <= j; ++qq) a += Xb[i * mn + qq] * Tn[j * mm + qq];
          blk[(pp.p0 + i) * b + pp.pn0 + j] = static_cast<T>(a);
        }
      } else {
        const T *Tn = own ? Trow + pp.pn0 * mm : TnT;
        const int ldn = own ? mm : mn;
        for (int e = lane; e < m * mn; e += 32) {
          const int i = e / mn, j = e % mn;
          T a = T(0);
          for (int qq = j < pp.nUn ? 0 : pp.nUn; qq <= j; ++qq) a += XT[i * mn + qq] * Tn[j * ldn + qq];
          blk[(pp.p0 + i) * b + pp.pn0 + j] = a;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // padded positions and the pinned unknown: identity (after the blocks,
  // whose pinned row and column are zero)
  for (int p = tid; p < b; p += kCT) {
    const int info = posinf[p];
    if (info < 0 || ((info >> 29) & 1)) tB[p * b + p] = T(1);
  }
  __syncthreads();
  cluster.sync();

  // ---- block cyclic reduction
  for (int lev = 0; lev < nlev; ++lev) {
    const int s = 1 << lev;
    if (k % (2 * s) == s) gj_inverse_la(tB, b, gjs, &bad);
    cluster.sync();
    if (k % (2 * s) == 0) {
      const int l = k - s, rt = k + s;
      T *X = tX + lev * bb;
      T *Y = tY + lev * bb;
      if (l >= 0 && rt < K) {
        // both neighbours: their inverses in one copy pass, X and Y in one
        // product pass, then the two fused updates
        copy_in2(tW1, cluster.map_shared_rank(tB, l), tW2, cluster.map_shared_rank(tB, rt), b * b);
        gemm_dual(X, tA, tW1, Y, tC, tW2, b);                      // X = A_k B_l^{-1}, Y = C_k B_r^{-1}
        copy_in2(tW1, cluster.map_shared_rank(tC, l), tW2, cluster.map_shared_rank(tA, l), b * b);
        gemm2(tB, tA, X, tW1, tW2, b, T(-1), true, T(-1), false);  // B_k -= X C_l, A_k = -X A_l
        copy_in2(tW1, cluster.map_shared_rank(tA, rt), tW2, cluster.map_shared_rank(tC, rt), b * b);
        gemm2(tB, tC, Y, tW1, tW2, b, T(-1), true, T(-1), false);  // B_k -= Y A_r, C_k = -Y C_r
      } else if (l >= 0) {                                         // left neighbour only
        copy_in(tW1, cluster.map_shared_rank(tB, l), b * b);         // B_l^{-1}
        gemm(X, tA, tW1, b, T(1), false);                          // X = A_k B_l^{-1}
        copy_in2(tW1, cluster.map_shared_rank(tC, l), tW2, cluster.map_shared_rank(tA, l), b * b);
        gemm2(tB, tA, X, tW1, tW2, b, T(-1), true, T(-1), false);  // B_k -= X C_l, A_k = -X A_l
        for (int e = tid; e < b * b; e += kCT) Y[e] = T(0);
      } else if (rt < K) {                                         // right neighbour only
        for (int e = tid; e < b * b; e += kCT) X[e] = T(0);
        copy_in(tW1, cluster.map_shared_rank(tB, rt), b * b);        // B_r^{-1}
        gemm(Y, tC, tW1, b, T(1), false);                          // Y = C_k B_r^{-1}
        copy_in2(tW1, cluster.map_shared_rank(tA, rt), tW2, cluster.map_shared_rank(tC, rt), b * b);
        gemm2(tB, tC, Y, tW1, tW2, b, T(-1), true, T(-1), false);  // B_k -= Y A_r, C_k = -Y C_r
      } else {
        for (int e = tid; e < b * b; e += kCT) X[e] = T(0);
        for (int e = tid; e < b * b; e += kCT) Y[e] = T(0);
      }
    }
    cluster.sync();
  }
  if (k == 0) gj_inverse_la(tB, b, gjs, &bad);
  if (tid == 0 && bad) atomicOr(&w.status[0], MRCM_FLAG_IFACE_PIVOT);
  cluster.sync();

  // ---- refinement: x of this slab and of its two neighbours (xs, FP64),
  // the residual rows (rowc/rowi), f and the scaling rows are all in shared
  // memory from here on; global memory is written once at the end.
  // ||f||^2 of the realisation (every CTA sums the K partials in the same order)
  if (tid < 32) {
    double a = 0.0;
    for (int q = tid; q < b; q += 32) a += fs[q] * fs[q];
    a = warp_sum(a);
    if (tid == 0) part[1] = a;
  }
  cluster.sync();
  double fnorm2 = 0.0;
  if (tid < 32) {
    double a = tid < K ? *cluster.map_shared_rank(part + 1, tid) : 0.0;
    fnorm2 = warp_sum(a);
  }
  fnorm2 = __shfl_sync(0xffffffffu, fnorm2, 0);   // lanes of warp 0; others below
  __shared__ double s_f2, s_r2;
  if (tid == 0) s_f2 = fnorm2;
  __syncthreads();
  fnorm2 = s_f2;
  const double tol2 = tol * tol;

  double prev2 = 1e300, rn2 = 0.0;
  int nsolve = 0;
  for (;;) {
    // A: x += T^T y (working precision correction added in FP64)
    if (nsolve > 0) {
      for (int pos = tid; pos < b; pos += kCT) {
        const int pi_ = posinf[pos];
        if (pi_ < 0) continue;
        const int p0 = (pi_ >> 16) & 255, m = (pi_ >> 8) & 255, i = pi_ & 255;
        T d = T(0);
        for (int q = i; q < m; ++q) d += Trow[(p0 + q) * mm + i] * v[p0 + q];
        xs[kCMaxB + pos] += static_cast<double>(d);
      }
      cluster.sync();
    }
    // neighbours' x (all zero before the first solve)
    if (nsolve > 0) {
      if (k > 0)
        for (int p = tid; p < b; p += kCT) xs[p] = cluster.map_shared_rank(xs, k - 1)[kCMaxB + p];
      if (k + 1 < K)
        for (int p = tid; p < b; p += kCT)
          xs[2 * kCMaxB + p] = cluster.map_shared_rank(xs, k + 1)[kCMaxB + p];
    }
    __syncthreads();
    // B: FP64 residual, one thread per row with four independent chains (no
    // FP64 warp reductions: every FP64 warp instruction costs the FP64 pipe
    // ~19 clocks on this part).  Before the first solve x = 0, so r = f: no
    // products.
    double rsq = 0.0;
    if (nsolve == 0) {
      if (tid < b) {
        const double rv = rowcnt[tid] > 0 ? fs[tid] : 0.0;
        rl[tid] = ((posinf[tid] >> 30) & 1) ? -rv : rv;
        rsq = rv * rv;
      }
    } else if (tid < b) {
      const int pos = tid, cnt = rowcnt[pos];
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      const double *rc = rowc + pos;
      const short *ri_ = rowi + pos;
      int e = 0;
      for (; e + 3 < cnt; e += 4) {
        const int x0 = ri_[e * b], x1 = ri_[(e + 1) * b], x2 = ri_[(e + 2) * b],
                  x3 = ri_[(e + 3) * b];
        a0 = fma(rc[e * b], xs[x0], a0);
        a1 = fma(rc[(e + 1) * b], xs[x1], a1);
        a2 = fma(rc[(e + 2) * b], xs[x2], a2);
        a3 = fma(rc[(e + 3) * b], xs[x3], a3);
      }
      for (; e < cnt; ++e) a0 = fma(rc[e * b], xs[ri_[e * b]], a0);
      const double rv = cnt > 0 ? fs[pos] - ((a0 + a1) + (a2 + a3)) : 0.0;
      rl[pos] = ((posinf[pos] >> 30) & 1) ? -rv : rv;
      rsq = rv * rv;
    }
    if (tid < ((b + 31) & ~31)) {
      rsq = warp_sum(rsq);
      if (lane == 0) red[wid] = rsq;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0;
      for (int q = 0; q < (b + 31) / 32; ++q) a += red[q];
      part[0] = a;
    }
    // z = T (sign r) in the working precision
    for (int pos = tid; pos < b; pos += kCT) {
      const int pi_ = posinf[pos];
      T z = T(0);
      if (pi_ >= 0 && rowcnt[pos] > 0) {
        const int p0 = (pi_ >> 16) & 255, i = pi_ & 255;
        for (int q = 0; q <= i; ++q) z += Trow[pos * mm + q] * static_cast<T>(rl[p0 + q]);
      }
      v[pos] = z;
    }
    cluster.sync();
    if (tid < 32) {
      double a = tid < K ? *cluster.map_shared_rank(part, tid) : 0.0;
      a = warp_sum(a);
      if (tid == 0) s_r2 = a;
    }
    __syncthreads();
    rn2 = s_r2;
    const bool stop = (rn2 <= tol2 * fnorm2) || (nsolve >= max_solves) || !(rn2 == rn2) ||
                      (nsolve >= 2 && rn2 > 0.25 * prev2);
    prev2 = rn2;
    if (stop) break;
    // C: y = Shat^{-1} z, cluster-wide cyclic reduction (8 threads per row)
    for (int lev = 0; lev < nlev; ++lev) {
      const int s = 1 << lev;
      if (k % (2 * s) == 0) {
        const int l = k - s, rt = k + s;
        for (int p = tid; p < b; p += kCT) {
          vr1[p] = l >= 0 ? cluster.map_shared_rank(v, l)[p] : T(0);
          vr2[p] = rt < K ? cluster.map_shared_rank(v, rt)[p] : T(0);
        }
        __syncthreads();
        T acc = T(0);
        if (l >= 0) acc += rowdot8(tX + lev * bb, vr1, b);
        if (rt < K) acc += rowdot8(tY + lev * bb, vr2, b);
        if ((tid & 7) == 0 && (tid >> 3) < b) v[tid >> 3] -= acc;
      }
      cluster.sync();
    }
    if (k == 0) {
      for (int p = tid; p < b; p += kCT) vr1[p] = v[p];
      __syncthreads();
      const T y = rowdot8(tB, vr1, b);
      if ((tid & 7) == 0 && (tid >> 3) < b) v[tid >> 3] = y;
    }
    cluster.sync();
    for (int lev = nlev - 1; lev >= 0; --lev) {
      const int s = 1 << lev;
      if (k % (2 * s) == s) {
        const int l = k - s, rt = k + s;
        for (int p = tid; p < b; p += kCT) {
          vr1[p] = cluster.map_shared_rank(v, l)[p];
          vr2[p] = rt < K ? cluster.map_shared_rank(v, rt)[p] : T(0);
        }
        __syncthreads();
        T acc = rowdot8(tA, vr1, b);
        if (rt < K) acc += rowdot8(tC, vr2, b);
        if ((tid & 7) == 0 && (tid >> 3) < b) vt[tid >> 3] = v[tid >> 3] - acc;
        __syncthreads();
        const T y = rowdot8(tB, vt, b);
        if ((tid & 7) == 0 && (tid >> 3) < b) v[tid >> 3] = y;
      }
      cluster.sync();
    }
    ++nsolve;
  }
  // the interface solution of this slab, for reconstruction
  for (int pos = tid; pos < b; pos += kCT) {
    const int u = t.pos2unk[P0 + pos];
    if (u >= 0) w.x[u] = xs[kCMaxB + pos];
  }
  if (k == 0 && tid == 0) {
    const double rel = fnorm2 > 0.0 ? sqrt(rn2 / fnorm2) : 0.0;
    w.done[r] = 1;
    w.dstat[2 + r] = rel;
    atomic_max_pos_double(&w.dstat[1], rel);
    atomicMax(&w.status[2], nsolve > 0 ? nsolve - 1 : 0);
    if (!(rel <= tol)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_STALL);
  }
}

template <typename T>
size_t cluster_smem(int bmax, int nlev, int emax, int mmax) {
  const size_t bb = (static_cast<size_t>(bmax) * bmax + 3) & ~static_cast<size_t>(3);
  size_t n = (5 + 2 * static_cast<size_t>(nlev)) * bb * sizeof(T) +
             (4 * kCMaxB + kGjScr) * sizeof(T);
  n = (n + 7) & ~static_cast<size_t>(7);
  n += (kCMaxB + 2 + 3 * kCMaxB + kCMaxB) * sizeof(double);      // rl, part, xs, fs
  n += static_cast<size_t>(bmax) * mmax * sizeof(double);         // Td
  n += static_cast<size_t>(bmax) * emax * sizeof(double);         // rowc
  n += ((static_cast<size_t>(bmax) * emax + 1) & ~static_cast<size_t>(1)) * sizeof(short);
  n += 2 * kCMaxB * sizeof(int);                                  // rowcnt, posinf
  n += static_cast<size_t>(bmax) * mmax * sizeof(T);              // Trow
  return n + 64;
}

}  // namespace

// Can the one-launch cluster path run this problem?  Returns the cluster
// size (0: no).
int iface_cluster_plan(int prec, int nslab, int bmax, int nlev, int mmax, int emax,
                       size_t stage_max, int dev) {
  if (prec != MRCM_PREC_FP32_IR) return 0;
  if (nslab < 1 || nslab > 16 || bmax > kCMaxB || 3 * kCMaxB > 32767) return 0;
  const size_t smem = cluster_smem<float>(bmax, nlev, emax, mmax);
  // per-warp assembly scratch must fit behind the first three tiles
  const size_t scr = static_cast<size_t>(kCT / 32) * 2 * mmax * mmax * (sizeof(double) + sizeof(float));
  const size_t behind = (2 + 2 * static_cast<size_t>(nlev)) *
                        ((static_cast<size_t>(bmax) * bmax + 3) & ~static_cast<size_t>(3)) *
                        sizeof(float);
  // the scaling scratch of at least one warp must fit in the tile area
  const size_t tiles = (5 + 2 * static_cast<size_t>(nlev)) *
                       ((static_cast<size_t>(bmax) * bmax + 3) & ~static_cast<size_t>(3)) *
                       sizeof(float);
  if (2 * static_cast<size_t>(mmax) * (mmax + 1) * sizeof(double) > tiles) return 0;
  if (scr > behind) return 0;
  // every slab's staged pair plans and pair blocks fit behind the assembly
  // scratch, and one warp's scaling scratch fits in front of them
  if (scr + stage_max > behind) return 0;
  const size_t per = (2 * static_cast<size_t>(mmax) * (mmax + 1) + static_cast<size_t>(mmax) * mmax) *
                     sizeof(float);
  if (stage_max + per > tiles) return 0;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > static_cast<size_t>(optin)) return 0;
  if (cudaFuncSetAttribute(k_iface_cluster<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(smem)) != cudaSuccess)
    return 0;
  if (nslab > 8 &&
      cudaFuncSetAttribute(k_iface_cluster<float>,
                           cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nslab);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nslab;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_iface_cluster<float>, &cfg) != cudaSuccess)
    return 0;
  cudaGetLastError();
  return nclusters > 0 ? nslab : 0;
}

cudaError_t launch_iface_cluster(const DeviceTables &t, const Workspace &w, const int *slab_if,
                                 const int *slab_if_off, int nslab, int bmax, int nlev,
                                 double tol, int max_solves, cudaStream_t st) {
  const size_t smem = cluster_smem<float>(bmax, nlev, t.emax, t.mmax);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nslab * t.n_real);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nslab;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_iface_cluster<float>, t, w, slab_if, slab_if_off, tol,
                            max_solves, bmax, nlev);
}

}  // namespace mrcm
