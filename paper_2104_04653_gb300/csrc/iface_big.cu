// Step (d), direct path for slabs larger than one CTA's tiles (b > 64): the
// same block cyclic reduction over slabs as iface.cu (Eq. "mrc2", slab
// ordering, congruence scaling, FP64 refinement), with every dense block
// operation spread over the GPU:
//
//  * inverses of the eliminated pivot blocks by batched blocked Gauss-Jordan
//    (no pivoting: the scaled slab blocks are symmetric quasi-definite), one
//    panel of 64 pivots at a time: k_gj_panel inverts the 64 x 64 diagonal
//    tile and forms the pivot row panel, k_gj_trail applies the rank-64
//    update to every other tile and forms the new pivot column panel (for
//    FP32 blocks k_gj_rowpanel_vec and k_gj_trail_vec, 16-byte accesses);
//  * the six block products of every surviving slab per level by a batched
//    128 x 128-tile SIMT GEMM over job descriptors (k_bgemm), two products
//    accumulated in one job for B_k -= X C_l + Y A_r;
//  * the refinement loop in one cooperative kernel (k_big_solve): FP64
//    residual from G, scaling, stop test, then the reduction solve with one
//    warp per block row and grid barriers between levels.
#include "mrcm_internal.h"
#include "iface_common.cuh"
#include "../../include/mrcm.h"

#include <cooperative_groups.h>
#include <cstdint>

namespace cg = cooperative_groups;

namespace mrcm {
namespace {

constexpr int kGjNb = 64;       // panel width of the blocked Gauss-Jordan
constexpr int kGjThreads = 256;

// ---------------------------------------------------------------- inverse
// Panel step p of the in-place Gauss-Jordan inverse of every matrix of the
// batch, in three launches:
//   k_gj_panel (one CTA per matrix): D = A[p.., p..]^{-1} into job.dinv;
//   k_gj_rowpanel (one CTA per matrix and 64-column tile): the old pivot
//     column panel rows of that tile into job.cpan, and the pivot row panel
//     R = D A[p.., tile] back into the matrix (D itself for the panel tile);
//   k_gj_trail (below): the rank-64 update of every other row tile.
constexpr size_t kGjPanelElems = kGjNb * kGjNb + 64 + 2 * 512;
constexpr size_t kGjTrailElems = 2 * kGjNb * kGjNb;

template <typename T>
__global__ void __launch_bounds__(kGjThreads) k_gj_panel(const InvJob *jobs, int p,
                                                         int *status) {
  extern __shared__ __align__(16) unsigned char gsmraw[];
  T *D = reinterpret_cast<T *>(gsmraw);
  T *scr = D + kGjNb * kGjNb;
  __shared__ int bad;
  const InvJob jb = jobs[blockIdx.x];
  const int n = jb.n;
  if (p >= n) return;
  const T *A = static_cast<const T *>(jb.a);
  T *Dout = static_cast<T *>(jb.dinv);
  const int w = n - p < kGjNb ? n - p : kGjNb;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
#pragma unroll 4
  for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) {
    const int i = e / kGjNb, j = e % kGjNb;
    D[e] = (i < w && j < w) ? A[static_cast<int64_t>(p + i) * n + p + j] : T(i == j);
  }
  __syncthreads();
  gj_inverse_blocked<T, kGjThreads>(D, kGjNb, kGjNb, scr, &bad);
  __syncthreads();
#pragma unroll 4
  for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) Dout[e] = D[e];
  if (t == 0 && bad) atomicOr(status, MRCM_FLAG_IFACE_PIVOT);
}

template <typename T>
__global__ void __launch_bounds__(kGjThreads) k_gj_rowpanel(const InvJob *jobs, int p) {
  extern __shared__ __align__(16) unsigned char gsmraw[];
  T *D = reinterpret_cast<T *>(gsmraw);
  T *tile = D + kGjNb * kGjNb;
  const InvJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (p >= n) return;
  const int nt = (n + kGjNb - 1) / kGjNb;
  if (static_cast<int>(blockIdx.x) >= nt) return;
  const int j0 = blockIdx.x * kGjNb;
  T *A = static_cast<T *>(jb.a);
  const T *Dv = static_cast<const T *>(jb.dinv);
  T *Cp = static_cast<T *>(jb.cpan);
  const int w = n - p < kGjNb ? n - p : kGjNb;
  const int wj = n - j0 < kGjNb ? n - j0 : kGjNb;
  const int t = threadIdx.x;
  if (j0 == p) {
    // the panel tile: rows [p, p+w) become D
#pragma unroll 4
    for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) {
      const int i = e / kGjNb, j = e % kGjNb;
      if (i < w && j < w) A[static_cast<int64_t>(p + i) * n + p + j] = Dv[e];
    }
    return;
  }
  // old column panel of the rows of this tile (rows j0 .. j0+wj)
#pragma unroll 4
  for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) {
    const int i = e / kGjNb, c = e % kGjNb;
    if (i < wj && c < w) Cp[static_cast<int64_t>(j0 + i) * w + c] =
        A[static_cast<int64_t>(j0 + i) * n + p + c];
  }
#pragma unroll 4
  for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) {
    D[e] = Dv[e];
    const int c = e / kGjNb, j = e % kGjNb;
    tile[e] = (c < w && j < wj) ? A[static_cast<int64_t>(p + c) * n + j0 + j] : T(0);
  }
  __syncthreads();
  // R = D tile: thread owns 4 rows x 4 columns
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int c = 0; c < w; ++c) {
    T da[4], tb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) da[a] = D[(tr + a) * kGjNb + c];
#pragma unroll
    for (int b = 0; b < 4; ++b) tb[b] = tile[c * kGjNb + tc + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += da[a] * tb[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (tr + a >= w) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (tc + b < wj) A[static_cast<int64_t>(p + tr + a) * n + j0 + tc + b] = acc[a][b];
  }
}

// k_gj_rowpanel for FP32 blocks with 16-byte accesses (the alignment
// argument of k_gj_trail_vec below): D is held with rows padded to 68 floats;
// the products are summed in the same order as k_gj_rowpanel.
constexpr int kGjDLd = kGjNb + 4;
constexpr size_t kGjRowVecBytes = (kGjNb * kGjDLd + kGjNb * kGjNb) * sizeof(float);

__global__ void __launch_bounds__(kGjThreads, 4) k_gj_rowpanel_vec(const InvJob *jobs, int p) {
  extern __shared__ __align__(16) unsigned char gsmraw[];
  float *D = reinterpret_cast<float *>(gsmraw);   // [row][kGjDLd]
  float *tile = D + kGjNb * kGjDLd;               // [c][col]
  const InvJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (p >= n) return;
  const int nt = (n + kGjNb - 1) / kGjNb;
  if (static_cast<int>(blockIdx.x) >= nt) return;
  const int j0 = blockIdx.x * kGjNb;
  float *A = static_cast<float *>(jb.a);
  const float *Dv = static_cast<const float *>(jb.dinv);
  float *Cp = static_cast<float *>(jb.cpan);
  const int w = n - p < kGjNb ? n - p : kGjNb;
  const int wj = n - j0 < kGjNb ? n - j0 : kGjNb;
  const int t = threadIdx.x;
  const int q = (t % 16) * 4, a0 = t / 16;   // staging: columns q..q+3 of rows a0 + 16 k
  if (j0 == p) {
    // the panel tile: rows [p, p+w) become D
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int i = a0 + 16 * k;
      if (i < w && q < w)
        *reinterpret_cast<float4 *>(A + static_cast<int64_t>(p + i) * n + p + q) =
            *reinterpret_cast<const float4 *>(Dv + i * kGjNb + q);
    }
    return;
  }
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  {
    float4 cv[4], dv[4], tv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = a0 + 16 * k;
      // old column panel of the rows of this tile (rows j0 .. j0+wj)
      cv[k] = (a < wj && q < w)
                  ? *reinterpret_cast<const float4 *>(A + static_cast<int64_t>(j0 + a) * n + p + q)
                  : z4;
      dv[k] = *reinterpret_cast<const float4 *>(Dv + a * kGjNb + q);
      tv[k] = (a < w && q < wj)
                  ? *reinterpret_cast<const float4 *>(A + static_cast<int64_t>(p + a) * n + j0 + q)
                  : z4;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = a0 + 16 * k;
      if (a < wj && q < w) *reinterpret_cast<float4 *>(Cp + static_cast<int64_t>(j0 + a) * w + q) = cv[k];
      *reinterpret_cast<float4 *>(D + a * kGjDLd + q) = dv[k];
      *reinterpret_cast<float4 *>(tile + a * kGjNb + q) = tv[k];
    }
  }
  __syncthreads();
  // R = D tile: thread owns 4 rows x 4 columns
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int c = 0; c < w; c += 4) {
    float4 da[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) da[a] = *reinterpret_cast<const float4 *>(D + (tr + a) * kGjDLd + c);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float4 tb = *reinterpret_cast<const float4 *>(tile + (c + cc) * kGjNb + tc);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float x = cc == 0 ? da[a].x : cc == 1 ? da[a].y : cc == 2 ? da[a].z : da[a].w;
        acc[a][0] += x * tb.x;
        acc[a][1] += x * tb.y;
        acc[a][2] += x * tb.z;
        acc[a][3] += x * tb.w;
      }
    }
  }
  if (tc >= wj) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (tr + a >= w) continue;
    *reinterpret_cast<float4 *>(A + static_cast<int64_t>(p + tr + a) * n + j0 + tc) =
        make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
  }
}

// Rank-w update of panel step p: for rows i outside the panel,
//   A[i, j] -= Cp[i, :] R[:, j]   (j outside the panel columns)
//   A[i, panel] = -Cp[i, :] D
// One CTA per (64 x 64 output tile, matrix).
template <typename T>
__global__ void __launch_bounds__(kGjThreads) k_gj_trail(const InvJob *jobs, int p) {
  extern __shared__ __align__(16) unsigned char gsmraw[];
  T *Cs = reinterpret_cast<T *>(gsmraw);   // [row][c]
  T *Rs = Cs + kGjNb * kGjNb;              // [c][col]
  const InvJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (p >= n) return;
  const int nt = (n + kGjNb - 1) / kGjNb;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;
  const int i0 = ti * kGjNb, j0 = tj * kGjNb;
  if (i0 == p) return;                          // the pivot rows are final
  T *A = static_cast<T *>(jb.a);
  const T *Dv = static_cast<const T *>(jb.dinv);
  const T *Cp = static_cast<const T *>(jb.cpan);
  const int w = n - p < kGjNb ? n - p : kGjNb;
  const int hi = n - i0 < kGjNb ? n - i0 : kGjNb, wj = n - j0 < kGjNb ? n - j0 : kGjNb;
  const bool pcol = (j0 == p);
  const int t = threadIdx.x;
  for (int e = t; e < kGjNb * kGjNb; e += kGjThreads) {
    const int a = e / kGjNb, b = e % kGjNb;
    Cs[e] = (a < hi && b < w) ? Cp[static_cast<int64_t>(i0 + a) * w + b] : T(0);
    T r = T(0);
    if (a < w && b < wj) r = pcol ? Dv[a * kGjNb + b] : A[static_cast<int64_t>(p + a) * n + j0 + b];
    Rs[e] = r;
  }
  __syncthreads();
  // thread: 4 rows x 4 columns
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int c = 0; c < w; ++c) {
    T ca[4], rb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ca[a] = Cs[(tr + a) * kGjNb + c];
#pragma unroll
    for (int b = 0; b < 4; ++b) rb[b] = Rs[c * kGjNb + tc + b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += ca[a] * rb[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (tr + a >= hi) continue;
    T *row = A + static_cast<int64_t>(i0 + tr + a) * n + j0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (tc + b >= wj) continue;
      row[tc + b] = pcol ? -acc[a][b] : row[tc + b] - acc[a][b];
    }
  }
}

// The same rank-w update for FP32 blocks, with 16-byte accesses throughout.
// Every FP32 slab block has n a multiple of 4 (the slab size is rounded up
// when the layout is planned) and p, i0, j0 are multiples of 64, so w, hi,
// wj are multiples of 4 and every row segment read or written here starts on
// a 16-byte boundary of the 256-byte aligned workspace.  The column panel
// rows are padded to 68 floats in shared memory (the two row groups of a
// warp fall in different banks); the thread's 4 x 4 output values are read
// ahead of the products.  Per output value the products are summed in the
// same order as k_gj_trail, so both give identical results.
constexpr int kGjCsLd = kGjNb + 4;
constexpr size_t kGjTrailVecBytes = (kGjNb * kGjCsLd + kGjNb * kGjNb) * sizeof(float);

__global__ void __launch_bounds__(kGjThreads, 4) k_gj_trail_vec(const InvJob *jobs, int p) {
  extern __shared__ __align__(16) unsigned char gsmraw[];
  float *Cs = reinterpret_cast<float *>(gsmraw);   // [row][kGjCsLd]
  float *Rs = Cs + kGjNb * kGjCsLd;                // [c][col]
  const InvJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  if (p >= n) return;
  const int nt = (n + kGjNb - 1) / kGjNb;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;
  const int i0 = ti * kGjNb, j0 = tj * kGjNb;
  if (i0 == p) return;                          // the pivot rows are final
  float *A = static_cast<float *>(jb.a);
  const float *Dv = static_cast<const float *>(jb.dinv);
  const float *Cp = static_cast<const float *>(jb.cpan);
  const int w = n - p < kGjNb ? n - p : kGjNb;
  const int hi = n - i0 < kGjNb ? n - i0 : kGjNb, wj = n - j0 < kGjNb ? n - j0 : kGjNb;
  const bool pcol = (j0 == p);
  const int t = threadIdx.x;
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 old[4];
  if (!pcol) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
      old[a] = (tr + a < hi && tc < wj)
                   ? *reinterpret_cast<const float4 *>(A + static_cast<int64_t>(i0 + tr + a) * n + j0 + tc)
                   : z4;
  }
  {
    // staging: thread t copies columns q .. q+3 of rows a0 + 16 k
    const int q = (t % 16) * 4, a0 = t / 16;
    float4 cv[4], rv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = a0 + 16 * k;
      cv[k] = (a < hi && q < w)
                  ? *reinterpret_cast<const float4 *>(Cp + static_cast<int64_t>(i0 + a) * w + q)
                  : z4;
      rv[k] = (a < w && q < wj)
                  ? *reinterpret_cast<const float4 *>(pcol ? Dv + a * kGjNb + q
                                                           : A + static_cast<int64_t>(p + a) * n + j0 + q)
                  : z4;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = a0 + 16 * k;
      *reinterpret_cast<float4 *>(Cs + a * kGjCsLd + q) = cv[k];
      *reinterpret_cast<float4 *>(Rs + a * kGjNb + q) = rv[k];
    }
  }
  __syncthreads();
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int c = 0; c < w; c += 4) {
    float4 ca[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ca[a] = *reinterpret_cast<const float4 *>(Cs + (tr + a) * kGjCsLd + c);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const float4 rb = *reinterpret_cast<const float4 *>(Rs + (c + cc) * kGjNb + tc);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const float x = cc == 0 ? ca[a].x : cc == 1 ? ca[a].y : cc == 2 ? ca[a].z : ca[a].w;
        acc[a][0] += x * rb.x;
        acc[a][1] += x * rb.y;
        acc[a][2] += x * rb.z;
        acc[a][3] += x * rb.w;
      }
    }
  }
  if (tc >= wj) return;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    if (tr + a >= hi) continue;
    const float4 r = pcol ? make_float4(-acc[a][0], -acc[a][1], -acc[a][2], -acc[a][3])
                          : make_float4(old[a].x - acc[a][0], old[a].y - acc[a][1],
                                        old[a].z - acc[a][2], old[a].w - acc[a][3]);
    *reinterpret_cast<float4 *>(A + static_cast<int64_t>(i0 + tr + a) * n + j0 + tc) = r;
  }
}

// ---------------------------------------------------------------- GEMM
// C = alpha (A1 B1 + A2 B2) (+ C if acc), all n x n row-major.  128 x 128
// output tile per CTA and 256 threads; each thread owns the 8 x 8 outputs
// at rows {4ty.., 64+4ty..} and columns {4tx.., 64+4tx..}, read from
// shared memory as 4-wide vectors (conflict-free).  k-steps of 8 are
// double-buffered: the next step's operands are loaded into registers
// while the current one is multiplied.
constexpr int kBM = 128, kBK = 8;

template <typename T>
struct Vec4 {
  static __device__ __forceinline__ void ld(const T *p, T v[4]) {
    v[0] = p[0];
    v[1] = p[1];
    v[2] = p[2];
    v[3] = p[3];
  }
};
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void ld(const float *p, float v[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void ld(const double *p, double v[4]) {
    const double2 q0 = *reinterpret_cast<const double2 *>(p);
    const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
  }
};

template <typename T>
__global__ void __launch_bounds__(256) k_bgemm(const GemmJob *jobs) {
  __shared__ __align__(16) T As[2][kBK][kBM];
  __shared__ __align__(16) T Bs[2][kBK][kBM];
  const GemmJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  const int nt = (n + kBM - 1) / kBM;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;
  const int i0 = ti * kBM, j0 = tj * kBM;
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  const int ar = t >> 1, ak = (t & 1) * 4;          // loader: A rows, 4 k each
  const int bk = t >> 5, bc = (t & 31) * 4;         // loader: B k, 4 columns each
  const T *A1 = static_cast<const T *>(jb.a1), *A2 = static_cast<const T *>(jb.a2);
  const T *B1 = static_cast<const T *>(jb.b1), *B2 = static_cast<const T *>(jb.b2);
  const int nk = (n + kBK - 1) / kBK;
  const int np = (A1 && B1 ? 1 : 0) + (A2 && B2 ? 1 : 0);
  const int first = (A1 && B1) ? 0 : 1;
  const int total = np * nk;
  T ra[4], rb[4];
  auto load = [&](int step) {
    const int prod = first + step / nk, k0 = (step % nk) * kBK;
    const T *Ap = prod == 0 ? A1 : A2, *Bp = prod == 0 ? B1 : B2;
    const int gi = i0 + ar;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gk = k0 + ak + q;
      ra[q] = (gi < n && gk < n) ? Ap[static_cast<int64_t>(gi) * n + gk] : T(0);
    }
    const int gk = k0 + bk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gj = j0 + bc + q;
      rb[q] = (gk < n && gj < n) ? Bp[static_cast<int64_t>(gk) * n + gj] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) As[buf][ak + q][ar] = ra[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) Bs[buf][bk][bc + q] = rb[q];
  };
  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
  if (total > 0) {
    load(0);
    store(0);
    __syncthreads();
  }
  for (int step = 0; step < total; ++step) {
    const int buf = step & 1;
    if (step + 1 < total) load(step + 1);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      T a[8], b[8];
      Vec4<T>::ld(&As[buf][kk][ty * 4], a);
      Vec4<T>::ld(&As[buf][kk][64 + ty * 4], a + 4);
      Vec4<T>::ld(&Bs[buf][kk][tx * 4], b);
      Vec4<T>::ld(&Bs[buf][kk][64 + tx * 4], b + 4);
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[q][r] += a[q] * b[r];
    }
    if (step + 1 < total) store(buf ^ 1);
    __syncthreads();
  }
  T *C = static_cast<T *>(jb.c);
  const T alpha = static_cast<T>(jb.alpha);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int gi = i0 + (q < 4 ? ty * 4 + q : 64 + ty * 4 + q - 4);
    if (gi >= n) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int gj = j0 + (r < 4 ? tx * 4 + r : 64 + tx * 4 + r - 4);
      if (gj >= n) continue;
      const int64_t o = static_cast<int64_t>(gi) * n + gj;
      C[o] = jb.acc ? C[o] + alpha * acc[q][r] : alpha * acc[q][r];
    }
  }
}

// ---------------------------------------------------------------- solve
// warp-level dot product of a matrix row with a vector (length n)
template <typename T>
__device__ __forceinline__ T row_dot(const T *row, const T *x, int n) {
  const int lane = threadIdx.x & 31;
  T acc = T(0);
  for (int j = lane; j < n; j += 32) acc += row[j] * x[j];
  return warp_sum(acc);
}

// The FP32 form: the solve streams the stored blocks once per sweep, one row
// per warp, so the bandwidth it reaches is set by the row bytes each warp
// keeps in flight.  Every lane issues all 16 of its loads of a 512-float
// chunk (16 coalesced 128-byte requests per warp) before the first product,
// then sums them in the same order as the loop above (element lane + 32 i,
// i ascending), so both forms give identical results: the interface
// refinement's stop test sees the same residuals.
template <>
__device__ __forceinline__ float row_dot<float>(const float *row, const float *x, int n) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (int base = 0; base < n; base += 512) {
    float rv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int j = base + lane + 32 * i;
      rv[i] = j < n ? __ldcs(row + j) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int j = base + lane + 32 * i;
      if (j < n) acc = fmaf(rv[i], x[j], acc);
    }
  }
  return warp_sum(acc);
}

constexpr int kBsCols = 4 * kMmax + 1;   // columns of a subdomain (uniform layouts)

// Refinement with the big-slab reduction solve, all realisations in one
// cooperative launch.  Each sweep: x += T^T y; r = f - M x (FP64), z = T
// (sign r); stop test per realisation; y = Shat^{-1} z by cyclic reduction
// (forward levels, root, backward levels), one warp per block row.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_big_solve(DeviceTables t, Workspace w, BigPlan bp,
                                                   double tol, int max_solves) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double red[8];
  __shared__ double s_rel;
  __shared__ double wbuf[8][kMmax];
  __shared__ double xg[8][2 * kBsCols];   // per warp: x of the two subdomains' columns
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * 8 + wid;
  const int nwarps = gridDim.x * 8;
  T *vec = static_cast<T *>(w.vec);
  T *tmp = static_cast<T *>(bp.vec2);
  const int K = bp.K, R = t.n_real, B = bp.bmax;
  int nsolve = 0;
  for (int sweep = 0;; ++sweep) {
    // A: x += T^T y
    if (sweep > 0) {
      for (int g = gwarp; g < t.niface; g += nwarps) {
        const IfaceInfo fi = t.iface[g];
        if (__ldcg(w.done + fi.r)) continue;
        const RealInfo &ri = t.real[fi.r];
        const int m = fi.nU + fi.nP;
        const T *yv = vec + ri.vec_off + static_cast<int64_t>(fi.slab) * ri.bmax + fi.pos;
        const double *Tg = w.tsc + fi.tsc_off;
        if (lane < m) {
          double d = 0.0;
          for (int q = lane; q < m; ++q) d += Tg[q * m + lane] * static_cast<double>(__ldcg(yv + q));
          w.x[fi.unk + lane] += d;
        }
      }
      grid.sync();
    }
    // B: FP64 residual, scaled into the slab vector.  The rows of an
    // interface share the column lists of its two subdomains: the warp first
    // gathers those columns' x into shared memory (independent loads, 32 at
    // a time), then each lane (one unknown) sums its two contiguous G rows
    // against them in four independent chains.
    for (int g = gwarp; g < t.niface; g += nwarps) {
      const IfaceInfo fi = t.iface[g];
      if (__ldcg(w.done + fi.r)) continue;
      const RealInfo &ri = t.real[fi.r];
      const int m = fi.nU + fi.nP;
      const int ncL = t.sub[fi.L].ncols, ncR = t.sub[fi.R].ncols;
      const int offL = t.sub[fi.L].col_off, offR = t.sub[fi.R].col_off;
      const bool staged = ncL <= kBsCols && ncR <= kBsCols;
      double *xl = xg[wid], *xr = xl + kBsCols;
      if (staged) {
        for (int c = 1 + lane; c < ncL; c += 32) xl[c] = __ldcg(w.x + t.col[offL + c].unk);
        for (int c = 1 + lane; c < ncR; c += 32) xr[c] = __ldcg(w.x + t.col[offR + c].unk);
      }
      __syncwarp();
      double rv = 0.0;
      if (lane < m && fi.unk + lane != ri.pin) {
        const RowRef rr = row_ref(t, w, fi, lane);
        if (staged) {
          double s0 = w.f[fi.unk + lane], s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int c = 1;
          for (; c + 3 < ncL; c += 4) {
            s0 -= rr.gL[c] * xl[c];
            s1 -= rr.gL[c + 1] * xl[c + 1];
            s2 -= rr.gL[c + 2] * xl[c + 2];
            s3 -= rr.gL[c + 3] * xl[c + 3];
          }
          for (; c < ncL; ++c) s0 -= rr.gL[c] * xl[c];
          for (c = 1; c + 3 < ncR; c += 4) {
            s0 -= rr.gR[c] * xr[c];
            s1 -= rr.gR[c + 1] * xr[c + 1];
            s2 -= rr.gR[c + 2] * xr[c + 2];
            s3 -= rr.gR[c + 3] * xr[c + 3];
          }
          for (; c < ncR; ++c) s0 -= rr.gR[c] * xr[c];
          rv = (s0 + s1) + (s2 + s3);
        } else {
          double sacc = w.f[fi.unk + lane];
          for (int c = 1; c < ncL; ++c) sacc -= rr.gL[c] * __ldcg(w.x + t.col[offL + c].unk);
          for (int c = 1; c < ncR; ++c) sacc -= rr.gR[c] * __ldcg(w.x + t.col[offR + c].unk);
          rv = sacc;
        }
      }
      double sq = rv * rv;
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) w.r[g] = sq;
      wbuf[wid][lane] = (lane >= fi.nU) ? -rv : rv;
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
    // C: stop test, one CTA per realisation
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
      if (__ldcg(w.done + r)) continue;
      const RealInfo ri = t.real[r];
      double rn = 0.0, fn = 0.0;
      for (int g = ri.iface0 + threadIdx.x; g < ri.iface0 + ri.niface; g += blockDim.x)
        rn += __ldcg(w.r + g);
      for (int u = ri.unk0 + threadIdx.x; u < ri.unk0 + ri.nunk; u += blockDim.x)
        fn += w.f[u] * w.f[u];
      for (int pass = 0; pass < 2; ++pass) {
        double v = pass == 0 ? rn : fn;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
          double sacc = 0.0;
          for (int k = 0; k < 8; ++k) sacc += red[k];
          if (pass == 0) s_rel = sacc;
          else s_rel = sacc > 0.0 ? sqrt(s_rel / sacc) : 0.0;
        }
        __syncthreads();
      }
      const double rel = s_rel;
      const double prev = w.dstat[2 + r];
      __syncthreads();
      if (threadIdx.x == 0) {
        w.dstat[2 + r] = rel;
        const bool stop = (rel <= tol) || (nsolve >= max_solves) || !(rel == rel) ||
                          (nsolve >= 2 && rel > 0.5 * prev);
        if (stop) {
          atomic_max_pos_double(&w.dstat[1], rel);
          atomicMax(&w.status[2], nsolve > 0 ? nsolve - 1 : 0);
          if (!(rel <= tol)) atomicOr(&w.status[0], MRCM_FLAG_IFACE_STALL);
          __threadfence();
          atomicExch(w.done + r, 1);
        }
      }
    }
    grid.sync();
    {
      int all = 1;
      for (int r = 0; r < R; ++r) all &= __ldcg(w.done + r);
      if (all) break;
    }
    // D: y = Shat^{-1} z.  Forward: v_k -= X v_{k-s} + Y v_{k+s} (survivors)
    for (int lev = 0, s = 1; lev < bp.nlev; ++lev, s <<= 1) {
      const int nsv = (K + 2 * s - 1) / (2 * s);
      const int64_t items = static_cast<int64_t>(R) * nsv * B;
      for (int64_t q = gwarp; q < items; q += nwarps) {
        const int r = static_cast<int>(q / (static_cast<int64_t>(nsv) * B));
        const int rem = static_cast<int>(q % (static_cast<int64_t>(nsv) * B));
        const int ki = rem / B, i = rem % B;
        if (__ldcg(w.done + r)) continue;
        const RealInfo &ri = t.real[r];
        const int b = ri.bmax;
        if (i >= b) continue;
        const int k = ki * 2 * s;
        const int64_t bb = static_cast<int64_t>(b) * b;
        const T *Xs = static_cast<const T *>(w.X) + ri.xy_off +
                      (static_cast<int64_t>(bp.lev_off[lev]) + ki) * bb;
        const T *Ys = static_cast<const T *>(w.Y) + ri.xy_off +
                      (static_cast<int64_t>(bp.lev_off[lev]) + ki) * bb;
        T *v = vec + ri.vec_off;
        T acc = T(0);
        if (k - s >= 0) acc += row_dot(Xs + static_cast<int64_t>(i) * b, v + (k - s) * b, b);
        if (k + s < K) acc += row_dot(Ys + static_cast<int64_t>(i) * b, v + (k + s) * b, b);
        if (lane == 0) v[k * b + i] -= acc;
      }
      grid.sync();
    }
    // root: slab 0 (its block holds the inverse)
    for (int64_t q = gwarp; q < static_cast<int64_t>(R) * B; q += nwarps) {
      const int r = static_cast<int>(q / B), i = static_cast<int>(q % B);
      if (__ldcg(w.done + r)) continue;
      const RealInfo &ri = t.real[r];
      const int b = ri.bmax;
      if (i >= b) continue;
      const T *I0 = static_cast<const T *>(w.slabB) + ri.slab_off;
      const T acc = row_dot(I0 + static_cast<int64_t>(i) * b, vec + ri.vec_off, b);
      if (lane == 0) tmp[ri.vec_off + i] = acc;
    }
    grid.sync();
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
         q < static_cast<int64_t>(R) * B; q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const int r = static_cast<int>(q / B), i = static_cast<int>(q % B);
      if (__ldcg(w.done + r) || i >= t.real[r].bmax) continue;
      vec[t.real[r].vec_off + i] = tmp[t.real[r].vec_off + i];
    }
    grid.sync();
    // backward: y_k = B_k^{-1} (v_k - A_k y_{k-s} - C_k y_{k+s}), eliminated k
    for (int lev = bp.nlev - 1; lev >= 0; --lev) {
      const int s = 1 << lev;
      const int nel = (K - s + 2 * s - 1) / (2 * s);
      const int64_t items = static_cast<int64_t>(R) * nel * B;
      for (int64_t q = gwarp; q < items; q += nwarps) {
        const int r = static_cast<int>(q / (static_cast<int64_t>(nel) * B));
        const int rem = static_cast<int>(q % (static_cast<int64_t>(nel) * B));
        const int ki = rem / B, i = rem % B;
        if (__ldcg(w.done + r)) continue;
        const RealInfo &ri = t.real[r];
        const int b = ri.bmax;
        if (i >= b) continue;
        const int k = s + ki * 2 * s;
        const int64_t bb = static_cast<int64_t>(b) * b;
        const T *As = static_cast<const T *>(w.slabA) + ri.slab_off + k * bb;
        const T *Cs = static_cast<const T *>(w.slabC) + ri.slab_off + k * bb;
        T *v = vec + ri.vec_off;
        T acc = row_dot(As + static_cast<int64_t>(i) * b, v + (k - s) * b, b);
        if (k + s < K) acc += row_dot(Cs + static_cast<int64_t>(i) * b, v + (k + s) * b, b);
        if (lane == 0) tmp[ri.vec_off + k * b + i] = v[k * b + i] - acc;
      }
      grid.sync();
      for (int64_t q = gwarp; q < items; q += nwarps) {
        const int r = static_cast<int>(q / (static_cast<int64_t>(nel) * B));
        const int rem = static_cast<int>(q % (static_cast<int64_t>(nel) * B));
        const int ki = rem / B, i = rem % B;
        if (__ldcg(w.done + r)) continue;
        const RealInfo &ri = t.real[r];
        const int b = ri.bmax;
        if (i >= b) continue;
        const int k = s + ki * 2 * s;
        const int64_t bb = static_cast<int64_t>(b) * b;
        const T *Is = static_cast<const T *>(w.slabB) + ri.slab_off + k * bb;
        const T acc = row_dot(Is + static_cast<int64_t>(i) * b, tmp + ri.vec_off + k * b, b);
        if (lane == 0) vec[ri.vec_off + k * b + i] = acc;
      }
      grid.sync();
    }
    ++nsolve;
  }
}

}  // namespace

// ------------------------------------------------------------ host launch
template <typename T>
static cudaError_t big_factor_t(const BigPlan &bp, int *status, int *nlaunch, cudaStream_t st) {
  for (int lev = 0; lev <= bp.nlev; ++lev) {
    // inverses of this level's eliminated slabs (the root at lev == nlev)
    const int i0 = bp.inv_off[lev], ni = bp.inv_off[lev + 1] - i0;
    if (ni > 0) {
      const int tiles = (bp.bmax + kGjNb - 1) / kGjNb;
      for (int p = 0; p < bp.bmax; p += kGjNb) {
        k_gj_panel<T><<<ni, kGjThreads, kGjPanelElems * sizeof(T), st>>>(bp.inv + i0, p, status);
        if constexpr (sizeof(T) == sizeof(float)) {
          k_gj_rowpanel_vec<<<dim3(tiles, ni), kGjThreads, kGjRowVecBytes, st>>>(bp.inv + i0, p);
          k_gj_trail_vec<<<dim3(tiles * tiles, ni), kGjThreads, kGjTrailVecBytes, st>>>(
              bp.inv + i0, p);
        } else {
          k_gj_rowpanel<T><<<dim3(tiles, ni), kGjThreads, kGjTrailElems * sizeof(T), st>>>(
              bp.inv + i0, p);
          k_gj_trail<T><<<dim3(tiles * tiles, ni), kGjThreads, kGjTrailElems * sizeof(T), st>>>(
              bp.inv + i0, p);
        }
        *nlaunch += 3;
      }
    }
    if (lev == bp.nlev) break;
    const int tiles = (bp.bmax + kBM - 1) / kBM;
    for (int set = 0; set < 2; ++set) {
      const int g0 = bp.gemm_off[2 * lev + set], ng = bp.gemm_off[2 * lev + set + 1] - g0;
      if (ng == 0) continue;
      if (sizeof(T) == sizeof(float) && bp.tensor_cores) {
        cudaError_t e = launch_tc_split(bp.gemm + g0,
                                        static_cast<const char *>(bp.tc_maps) + g0 * 4 * 128, ng,
                                        bp.bmax, status, st);
        if (e != cudaSuccess) return e;
      } else {
        k_bgemm<T><<<dim3(tiles * tiles, ng), 256, 0, st>>>(bp.gemm + g0);
      }
      ++*nlaunch;
    }
  }
  return cudaGetLastError();
}

cudaError_t init_big_attributes() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_gj_panel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kGjPanelElems * sizeof(float)))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gj_panel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kGjPanelElems * sizeof(double)))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gj_trail_vec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kGjTrailVecBytes))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gj_rowpanel_vec, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kGjRowVecBytes))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k_gj_rowpanel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kGjTrailElems * sizeof(double)))) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_gj_trail<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kGjTrailElems * sizeof(double)));
}

cudaError_t launch_big_factor(const BigPlan &bp, int prec, int *status, int *nlaunch,
                              cudaStream_t st) {
  if (prec == MRCM_PREC_FP64) return big_factor_t<double>(bp, status, nlaunch, st);
  return big_factor_t<float>(bp, status, nlaunch, st);
}

cudaError_t launch_simt_gemm(const GemmJob *jobs, int njobs, int nmax, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  const int tiles = (nmax + kBM - 1) / kBM;
  k_bgemm<float><<<dim3(tiles * tiles, njobs), 256, 0, st>>>(jobs);
  return cudaGetLastError();
}

int big_solve_grid(int prec, int dev) {
  int nsm = 0, per = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (prec == MRCM_PREC_FP64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_big_solve<double>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_big_solve<float>, 256, 0);
  return nsm * (per < 4 ? per : 4);
}

cudaError_t launch_big_solve(const DeviceTables &t, const Workspace &w, const BigPlan &bp, int prec,
                             double tol, int max_solves, int grid, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(w.x, 0, sizeof(double) * t.nunk, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.dstat + 2, 0, sizeof(double) * t.n_real, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(w.done, 0, sizeof(int) * (t.n_real + 1), st)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (prec == MRCM_PREC_FP64)
    return cudaLaunchKernelEx(&cfg, k_big_solve<double>, t, w, bp, tol, max_solves);
  return cudaLaunchKernelEx(&cfg, k_big_solve<float>, t, w, bp, tol, max_solves);
}

}  // namespace mrcm
