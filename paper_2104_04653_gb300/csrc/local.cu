// Steps (a)+(b) and (c) of the MRCM solve: per-subdomain assembly of the
// local Robin operator (Eq. "mrc1" with beta of Eq. "beta"), its batched
// factorisation, and the multi-RHS basis solves with FP64 refinement.
//
// The local operator of an s x s subdomain, with cells ordered row by row,
// is block tridiagonal: diagonal blocks D_j (one grid row, tridiagonal) and
// diagonal couplings E_j between rows j and j+1.  After symmetric Jacobi
// scaling (unit diagonal) it is factored as a block LDL^T whose pivots are
// the Schur complements S_j = D_j - E_{j-1} S_{j-1}^{-1} E_{j-1}; the kernel
// keeps their explicit inverses W_j = S_j^{-1}, so every step of a solve is
// a dense s x s matrix times a block of right-hand sides, with no
// sequential dependence inside a grid row.
//
// With FP32 factors and few 16 x 16 subdomains (at most two per SM; the
// setup decides, DeviceTables::fuse16) the factor launch only assembles the
// coefficients and each basis CTA forms its own subdomain's W_j in shared
// memory: the chain is one warp's work per subdomain, so a separate launch
// would leave most SMs idle, while with many subdomains the separate,
// throughput-bound factor launch is cheaper than one chain per column chunk.
#include "mrcm_internal.h"
#include "fpconv.cuh"
#include "../../include/mrcm.h"
#include "../../include/mrcm_testing.h"

#include <cstdint>
#include <cuda_runtime.h>
#include <type_traits>

namespace mrcm {
namespace {

constexpr int kS = 16;      // subdomain edge of the shared-memory-resident kernels
// per-subdomain coefficient block (at SubInfo::coef_off): tW tE tS tN d
// kappa [S*S each], then beta on the interface faces [4][S]
constexpr int kCoefStride = 6 * kS * kS + 4 * kS;
static_assert(kCoefStride % 2 == 0, "coefficient blocks are staged as 16-byte vectors");

__device__ __forceinline__ void atomic_max_pos_double(double *addr, double v) {
  // valid for v >= 0: IEEE order of non-negative doubles matches their bits
  if (!(v >= 0.0)) v = 1e300;
  atomicMax(reinterpret_cast<unsigned long long *>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}


// Face transmissibilities (two-point fluxes on square cells): harmonic mean
// between cells, kappa/(alpha H/h + 1/2) on a Robin face, 2 kappa on a
// Dirichlet face, 0 on a Neumann face.
//
// Harmonic-mean transmissibility of an interior face (square cells).  It is
// bitwise symmetric in its arguments (2 k1 k2 = 2 (k1 k2) exactly, sum and
// product commute), so one evaluation serves both cells of the face.
__device__ __forceinline__ double harmonic_face_T(double k1, double k2) {
  return 2.0 * k1 * k2 / (k1 + k2);
}

// Jacobi scaling 1/sqrt(A_cc) of a cell.  Any consistent positive scaling is
// valid (the same d scales the factor, the residuals and the corrections),
// but the factor takes the scaled diagonal as exactly 1, so d must be close
// to the exact value: the FP32 factor takes one Newton-Raphson step for
// x^(-1/2), y (3 - x y^2) / 2, in FP64 from the FP32 estimate (relative error
// squares, ~1e-14), four FP64 operations instead of a divide and a square
// root.  The FP64 path, which has no refinement, takes the exact value, and
// so does any diagonal outside FP32's normal range.
template <typename T>
__device__ __forceinline__ double jacobi_scale(double diag) {
  if constexpr (std::is_same<T, float>::value) {
    const float f = static_cast<float>(diag);
    if (f > 1e-30f && f < 1e30f) {
      const double y = static_cast<double>(rsqrtf(f));
      return y * fma(-0.5 * diag, y * y, 1.5);
    }
  }
  return 1.0 / sqrt(diag);
}

// A face of cell (a, b) on the subdomain edge ``side``: Robin on an
// interface edge, Dirichlet / Neumann on the physical boundary.
template <int S>
__device__ __forceinline__ double edge_face_T(const DeviceTables &t, const SubInfo &sb, double kc,
                                              int a, int b, int side) {
  if (sb.edge_iface[side] >= 0) {
    // H / h is the length of the face's interface (S without refinement)
    const FaceIface fi = face_iface(sb, side, (side < 2) ? b : a);
    const double al = t.alpha[t.iface[fi.g].alpha_off + fi.e];
    return kc / (al * static_cast<double>(fi.len) + 0.5);
  }
  const int gi = sb.x0 + a, gj = sb.y0 + b;
  int k;
  if (side == kEdgeW) k = gj;
  else if (side == kEdgeE) k = t.ny + gj;
  else if (side == kEdgeS) k = 2 * t.ny + gi;
  else k = 2 * t.ny + t.nx + gi;
  return (t.bc_type[k] == 1) ? 2.0 * kc : 0.0;
}

// ---------------------------------------------------------------------------
// (a)+(b).  Stage 1 (one thread per cell): FP64 transmissibilities, Jacobi
// scaling and the scaled couplings.  Stage 2 (one warp per subdomain): the
// block LDL^T recursion S_j = D_j - E_{j-1} W_{j-1} E_{j-1} and the
// Gauss-Jordan inverses W_j = S_j^{-1} in registers.  Lane l holds column
// c = l % S and rows HL (l / S) .. + RPL - 1 of the current block (HL = 32/S
// lanes per column, RPL = S / HL rows per lane); pivots are exchanged with
// warp shuffles, so the S^2-step pivot chain has no block-wide barrier.
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Stage 2 for one subdomain, executed by one whole warp.  offx[cell]: scaled
// coupling of (a,b) to (a+1,b); ecp[cell]: to (a,b+1).  Writes W_j to Wg.
// The S x S working matrix is spread over the warp as a 4 x 8 grid of lanes,
// lane (rb, cb) = (lane / 8, lane % 8) holding rows LR rb .. LR rb + LR - 1 and
// columns LC cb .. LC cb + LC - 1 (LR = S / 4, LC = S / 8).  Gauss-Jordan runs
// two pivots at a time: the 2 x 2 pivot block lies in one lane, is inverted
// in closed form, and the block update (pivot rows Pi R_K., pivot columns
// -R_.K Pi, the rest R - R_.K Pi R_K.) is applied in one pass, which halves the
// dependent chain of shuffles and reciprocals.  A 2 x 2 block of an SPD
// matrix has a00 > 0 and det > 0 exactly when both sequential pivots are
// positive, which is the test here.  FP32 only; FP64 takes the single-pivot
// form above.
// One pivot at a time, lane = column (S / 32 lanes per column): the form
// used in FP64, where the pair update's extra products cost more on the
// slow FP64 pipe than the shorter chain saves.
template <typename T, int S>
__device__ __forceinline__ bool schur_inverses_single(int lane, const T *offx, const T *ecp,
                                                      T *Wg) {
  constexpr int N = S * S, HL = 32 / S, RPL = S / HL;
  static_assert(HL * S == 32, "S must divide 32 lanes");
  const int c = lane % S, h = lane / S;
  T R[RPL];
  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < S; ++j) {
    const T ec = j > 0 ? ecp[(j - 1) * S + c] : T(0);
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int r = RPL * h + q;
      T v = T(0);
      if (r == c) v = T(1);
      else if (r - c == 1) v = offx[j * S + c];
      else if (c - r == 1) v = offx[j * S + r];
      if (j > 0) v -= ecp[(j - 1) * S + r] * ec * R[q];
      R[q] = v;
    }
#pragma unroll
    for (int p = 0; p < S; ++p) {
      const int src = (p / RPL) * S;
      const T rowv = shfl(R[p % RPL], src + c);
      const T piv = shfl(R[p % RPL], src + p);
      T colv[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) colv[q] = shfl(R[q], h * S + p);
      if (!(piv > T(0))) bad = true;
      const T ip = recip(piv);
      const T rv = rowv * ip;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int r = RPL * h + q;
        T nv = R[q] - colv[q] * rv;
        nv = (c == p) ? -colv[q] * ip : nv;
        nv = (r == p) ? ((c == p) ? ip : rv) : nv;
        R[q] = nv;
      }
    }
#pragma unroll
    for (int q = 0; q < RPL; ++q) Wg[j * N + (RPL * h + q) * S + c] = R[q];
  }
  return bad;
}

template <typename T, int S>
__device__ __forceinline__ bool schur_inverses(int lane, const T *offx, const T *ecp, T *Wg) {
  if constexpr (!std::is_same<T, float>::value) {
    return schur_inverses_single<T, S>(lane, offx, ecp, Wg);
  }
  constexpr int N = S * S, LR = S / 4, LC = S / 8;
  static_assert(LR * 4 == S && LC * 8 == S && LR % 2 == 0 && LC % 2 == 0,
                "S must be a multiple of 16 so that pivot pairs stay inside a lane block");
  const int rb = lane >> 3, cb = lane & 7;
  T R[LR][LC];
#pragma unroll
  for (int q = 0; q < LR; ++q)
#pragma unroll
    for (int w = 0; w < LC; ++w) R[q][w] = T(0);
  bool bad = false;
#pragma unroll 1
  for (int j = 0; j < S; ++j) {
    // Schur complement S_j = A_jj - E W_{j-1} E (E diagonal), Jacobi-scaled
    T ec[LC];
#pragma unroll
    for (int w = 0; w < LC; ++w) ec[w] = j > 0 ? ecp[(j - 1) * S + LC * cb + w] : T(0);
#pragma unroll
    for (int q = 0; q < LR; ++q) {
      const int r = LR * rb + q;
      const T er = j > 0 ? ecp[(j - 1) * S + r] : T(0);
#pragma unroll
      for (int w = 0; w < LC; ++w) {
        const int c = LC * cb + w;
        T v = T(0);
        if (r == c) v = T(1);
        else if (r - c == 1) v = offx[j * S + c];
        else if (c - r == 1) v = offx[j * S + r];
        if (j > 0) v -= er * ec[w] * R[q][w];
        R[q][w] = v;
      }
    }
#pragma unroll
    for (int p = 0; p < S; p += 2) {
      const int prb = p / LR, pq = p % LR, pcb = p / LC, pw = p % LC;
      const int lpiv = prb * 8 + pcb;
      const T a00 = shfl(R[pq][pw], lpiv), a01 = shfl(R[pq][pw + 1], lpiv);
      const T a10 = shfl(R[pq + 1][pw], lpiv), a11 = shfl(R[pq + 1][pw + 1], lpiv);
      T rw0[LC], rw1[LC], cl0[LR], cl1[LR];
#pragma unroll
      for (int w = 0; w < LC; ++w) {   // the pivot rows at this lane's columns
        rw0[w] = shfl(R[pq][w], prb * 8 + cb);
        rw1[w] = shfl(R[pq + 1][w], prb * 8 + cb);
      }
#pragma unroll
      for (int q = 0; q < LR; ++q) {   // this lane's rows at the pivot columns
        cl0[q] = shfl(R[q][pw], rb * 8 + pcb);
        cl1[q] = shfl(R[q][pw + 1], rb * 8 + pcb);
      }
      const T det = a00 * a11 - a01 * a10;
      if (!(a00 > T(0)) || !(det > T(0))) bad = true;
      const T idet = recip(det);
      const T p00 = a11 * idet, p01 = -a01 * idet, p10 = -a10 * idet, p11 = a00 * idet;
      T rp0[LC], rp1[LC];
#pragma unroll
      for (int w = 0; w < LC; ++w) {   // new pivot rows Pi R_K.
        rp0[w] = p00 * rw0[w] + p01 * rw1[w];
        rp1[w] = p10 * rw0[w] + p11 * rw1[w];
      }
#pragma unroll
      for (int q = 0; q < LR; ++q) {
#pragma unroll
        for (int w = 0; w < LC; ++w) {
          T nv = R[q][w] - (cl0[q] * rp0[w] + cl1[q] * rp1[w]);
          if (w == pw || w == pw + 1) {            // possibly a pivot column
            const T pc = (w == pw) ? -(cl0[q] * p00 + cl1[q] * p10)
                                   : -(cl0[q] * p01 + cl1[q] * p11);
            nv = (cb == pcb) ? pc : nv;
          }
          if (q == pq || q == pq + 1) {            // possibly a pivot row
            T prv = (q == pq) ? rp0[w] : rp1[w];
            if (w == pw || w == pw + 1) {
              const T pb = (q == pq) ? ((w == pw) ? p00 : p01) : ((w == pw) ? p10 : p11);
              prv = (cb == pcb) ? pb : prv;
            }
            nv = (rb == prb) ? prv : nv;
          }
          R[q][w] = nv;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < LR; ++q)
#pragma unroll
      for (int w = 0; w < LC; ++w) Wg[j * N + (LR * rb + q) * S + LC * cb + w] = R[q][w];
  }
  return bad;
}

// Twisted form of the chain above (FP32, the fused basis path): the block
// rows are eliminated from both ends at once and meet at the middle block
// M = S / 2.  Warp 0 (half 0) forms W_j = (A_jj - E_{j-1} W_{j-1} E_{j-1})^-1
// for j = 0 .. M-1 as before; warp 1 (half 1) forms W_j = (A_jj - E_j W_{j+1}
// E_j)^-1 for j = S-1 down to M+1; warp 0 then inverts the middle block
// A_MM - E_{M-1} W_{M-1} E_{M-1} - E_M W_{M+1} E_M, with W_{M+1} read from
// shared memory after a 64-thread named barrier (id 2; warp 1 reaches it
// once its chain is written).  The dependent chain is M + 1 block inverses
// instead of S.  E_j = diag(ecp[j S ..]) couples block rows j and j + 1.
template <int S>
__device__ __forceinline__ bool schur_inverses_twisted(int half, int lane, const float *offx,
                                                       const float *ecp, float *Wg) {
  using T = float;
  constexpr int N = S * S, LR = S / 4, LC = S / 8, M = S / 2;
  static_assert(LR * 4 == S && LC * 8 == S && LR % 2 == 0 && LC % 2 == 0,
                "S must be a multiple of 16 so that pivot pairs stay inside a lane block");
  const int rb = lane >> 3, cb = lane & 7;
  T R[LR][LC];
#pragma unroll
  for (int q = 0; q < LR; ++q)
#pragma unroll
    for (int w = 0; w < LC; ++w) R[q][w] = T(0);
  bool bad = false;
  const int nsteps = half == 0 ? M + 1 : S - 1 - M;
#pragma unroll 1
  for (int k = 0; k < nsteps; ++k) {
    const int j = half == 0 ? k : S - 1 - k;
    const bool mid = half == 0 && j == M;
    if (mid) asm volatile("bar.sync 2, 64;" ::: "memory");   // W_{M+1} is in Wg
    const bool has = half == 0 ? j > 0 : j < S - 1;        // a previous block of this chain
    const int je = half == 0 ? j - 1 : j;                   // its coupling row of ecp
    T ec[LC];
#pragma unroll
    for (int w = 0; w < LC; ++w) ec[w] = has ? ecp[je * S + LC * cb + w] : T(0);
#pragma unroll
    for (int q = 0; q < LR; ++q) {
      const int r = LR * rb + q;
      const T er = has ? ecp[je * S + r] : T(0);
#pragma unroll
      for (int w = 0; w < LC; ++w) {
        const int c = LC * cb + w;
        T v = T(0);
        if (r == c) v = T(1);
        else if (r - c == 1) v = offx[j * S + c];
        else if (c - r == 1) v = offx[j * S + r];
        if (has) v -= er * ec[w] * R[q][w];
        if (mid) v -= ecp[M * S + r] * ecp[M * S + c] * Wg[(M + 1) * N + r * S + c];
        R[q][w] = v;
      }
    }
#pragma unroll
    for (int p = 0; p < S; p += 2) {
      const int prb = p / LR, pq = p % LR, pcb = p / LC, pw = p % LC;
      const int lpiv = prb * 8 + pcb;
      const T a00 = shfl(R[pq][pw], lpiv), a01 = shfl(R[pq][pw + 1], lpiv);
      const T a10 = shfl(R[pq + 1][pw], lpiv), a11 = shfl(R[pq + 1][pw + 1], lpiv);
      T rw0[LC], rw1[LC], cl0[LR], cl1[LR];
#pragma unroll
      for (int w = 0; w < LC; ++w) {
        rw0[w] = shfl(R[pq][w], prb * 8 + cb);
        rw1[w] = shfl(R[pq + 1][w], prb * 8 + cb);
      }
#pragma unroll
      for (int q = 0; q < LR; ++q) {
        cl0[q] = shfl(R[q][pw], rb * 8 + pcb);
        cl1[q] = shfl(R[q][pw + 1], rb * 8 + pcb);
      }
      const T det = a00 * a11 - a01 * a10;
      if (!(a00 > T(0)) || !(det > T(0))) bad = true;
      const T idet = recip(det);
      const T p00 = a11 * idet, p01 = -a01 * idet, p10 = -a10 * idet, p11 = a00 * idet;
      T rp0[LC], rp1[LC];
#pragma unroll
      for (int w = 0; w < LC; ++w) {
        rp0[w] = p00 * rw0[w] + p01 * rw1[w];
        rp1[w] = p10 * rw0[w] + p11 * rw1[w];
      }
#pragma unroll
      for (int q = 0; q < LR; ++q) {
#pragma unroll
        for (int w = 0; w < LC; ++w) {
          T nv = R[q][w] - (cl0[q] * rp0[w] + cl1[q] * rp1[w]);
          if (w == pw || w == pw + 1) {
            const T pc = (w == pw) ? -(cl0[q] * p00 + cl1[q] * p10)
                                   : -(cl0[q] * p01 + cl1[q] * p11);
            nv = (cb == pcb) ? pc : nv;
          }
          if (q == pq || q == pq + 1) {
            T prv = (q == pq) ? rp0[w] : rp1[w];
            if (w == pw || w == pw + 1) {
              const T pb = (q == pq) ? ((w == pw) ? p00 : p01) : ((w == pw) ? p10 : p11);
              prv = (cb == pcb) ? pb : prv;
            }
            nv = (rb == prb) ? prv : nv;
          }
          R[q][w] = nv;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < LR; ++q)
#pragma unroll
      for (int w = 0; w < LC; ++w) Wg[j * N + (LR * rb + q) * S + LC * cb + w] = R[q][w];
  }
  if (half == 1) asm volatile("bar.sync 2, 64;" ::: "memory");   // this chain is written
  return bad;
}

// beta = alpha H / kappa on the interface faces of cell (a, b) (Eq. "beta")
template <int S>
__device__ __forceinline__ void write_beta(const DeviceTables &t, const SubInfo &sb, double kc,
                                           int a, int b, double *coef) {
  constexpr int N = S * S;
  const bool onface[4] = {a == 0, a == S - 1, b == 0, b == S - 1};
#pragma unroll
  for (int side = 0; side < 4; ++side) {
    if (!onface[side] || sb.edge_iface[side] < 0) continue;
    const int e = (side < 2) ? b : a;
    const FaceIface fi = face_iface(sb, side, e);   // H = the interface's length
    const double H = fi.len * t.h;
    const double al = t.alpha[t.iface[fi.g].alpha_off + fi.e];
    coef[6 * N + side * S + e] = al * H / kc;
  }
}

// One column's (or one CTA's) final relative refinement residual.  Up to
// 1e3 tol it enters the maximum in dstat[0]; above, the subdomain is listed
// (once) for the FP64 recovery, or, with no slot left or no recovery, the
// stall is flagged (MRCM_EIRSTALL) and enters the maximum.
__device__ __forceinline__ void report_local_resid(const Workspace &w, int g, double rel,
                                                   double tol) {
  if (rel <= 1e3 * tol) {
    atomic_max_pos_double(&w.dstat[0], rel);
    return;
  }
  if (w.rec_cap > 0) {
    if (atomicExch(&w.stall_mark[g], 1) != 0) return;   // listed or flagged already
    const int slot = atomicAdd(&w.status[4], 1);
    if (slot < w.rec_cap) {
      w.stall_list[slot] = g;
      return;
    }
  }
  atomicOr(&w.status[0], MRCM_FLAG_LOCAL_STALL);
  atomic_max_pos_double(&w.dstat[0], rel);
}

// s = 16: one CTA of 256 threads per subdomain.  CHAIN = false: stage 1 only
// (coefficients and Jacobi scale); the FP32 basis kernel then factors each
// subdomain itself (k_basis with FUSED).
template <typename T, bool CHAIN = true>
__global__ void __launch_bounds__(kS *kS) k_factor(DeviceTables t, Workspace w, const double *K,
                                                   const double *lam) {
  constexpr int S = kS, N = S * S;
  const int g = t.sub_by_size[blockIdx.x];
  const SubInfo sb = t.sub[g];
  const int tid = threadIdx.x;
  const int a = tid % S, b = tid / S;
  if (tid == 0 && w.rec_cap > 0) w.stall_mark[g] = 0;   // a new factorisation
  __shared__ double kap[N];
  __shared__ double dsc[N];
  __shared__ double tfE[N], tfN[N];   // E and N face transmissibilities
  __shared__ T offx[N];   // scaled coupling of cell (a,b) to (a+1,b)
  __shared__ T ecp[N];    // scaled coupling of cell (a,b) to (a,b+1)

  const int64_t cell = (static_cast<int64_t>(sb.r) * t.ny + sb.y0 + b) * t.nx + sb.x0 + a;
  const double kc = K[cell] * lam[cell];
  if (!(kc > 0.0) || !isfinite(kc)) atomicOr(&w.status[0], MRCM_FLAG_NAN);
  kap[tid] = kc;
  __syncthreads();
  // each interior face once: a cell computes its E and N faces, and takes W
  // and S from the neighbouring cells (the same values, see harmonic_face_T)
  double T4[4];
  T4[1] = a < S - 1 ? harmonic_face_T(kc, kap[tid + 1]) : edge_face_T<S>(t, sb, kc, a, b, kEdgeE);
  T4[3] = b < S - 1 ? harmonic_face_T(kc, kap[tid + S]) : edge_face_T<S>(t, sb, kc, a, b, kEdgeN);
  tfE[tid] = T4[1];
  tfN[tid] = T4[3];
  __syncthreads();
  T4[0] = a > 0 ? tfE[tid - 1] : edge_face_T<S>(t, sb, kc, a, b, kEdgeW);
  T4[2] = b > 0 ? tfN[tid - S] : edge_face_T<S>(t, sb, kc, a, b, kEdgeS);
  const double d = jacobi_scale<T>(T4[0] + T4[1] + T4[2] + T4[3]);
  double *coef = w.coef + sb.coef_off;
#pragma unroll
  for (int k = 0; k < 4; ++k) coef[k * N + tid] = T4[k];
  coef[4 * N + tid] = d;
  coef[5 * N + tid] = kc;
  write_beta<S>(t, sb, kc, a, b, coef);
  dsc[tid] = d;
  if constexpr (!CHAIN) return;
  __syncthreads();
  offx[tid] = static_cast<T>(a < S - 1 ? -T4[1] * d * dsc[tid + 1] : 0.0);
  ecp[tid] = static_cast<T>(b < S - 1 ? -T4[3] * d * dsc[tid + S] : 0.0);
  __syncthreads();
  T *Wg = static_cast<T *>(w.W) + sb.w_off;
  bool bad;
  if constexpr (std::is_same<T, float>::value) {
    // FP32: the twisted chain on warps 0 and 1 (the basis kernel's FP32
    // block solve expects that form)
    if (tid >= 64) return;
    bad = schur_inverses_twisted<S>(tid >> 5, tid & 31, offx, ecp, Wg);
  } else {
    if (tid >= 32) return;
    bad = schur_inverses<T, S>(tid, offx, ecp, Wg);
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(&w.status[0], MRCM_FLAG_NOTSPD);
}

// s = 32: one WARP per subdomain (kFW subdomains per CTA), stage 1 with
// N / 32 cells per lane, so that every resident warp works in stage 2.
constexpr int kFW = 4;

template <typename T, int S>
struct FactorWarpSmem {
  double dsc[S * S];
  T offx[S * S];
  T ecp[S * S];
};

template <typename T, int S>
__global__ void __launch_bounds__(32 * kFW) k_factor_warp(DeviceTables t, Workspace w,
                                                          const double *K, const double *lam,
                                                          int first, int count) {
  constexpr int N = S * S, CPL = N / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int idx = blockIdx.x * kFW + wid;
  if (idx >= count) return;     // whole warp; no CTA-wide barrier follows
  FactorWarpSmem<T, S> &sm = reinterpret_cast<FactorWarpSmem<T, S> *>(smraw)[wid];
  const int g = t.sub_by_size[first + idx];
  const SubInfo sb = t.sub[g];
  if (lane == 0 && w.rec_cap > 0) w.stall_mark[g] = 0;  // a new factorisation
  double *coef = w.coef + sb.coef_off;
  const int64_t row0 = static_cast<int64_t>(sb.r) * t.ny + sb.y0;
  auto kappa = [&](int a, int b) {
    const int64_t cc = (row0 + b) * t.nx + sb.x0 + a;
    return K[cc] * lam[cc];
  };
  bool nan = false;
  // lane a walks column a row by row (cell = lane + 32 k, S = 32): kappa is
  // read once per cell, one row ahead; the E neighbour's kappa and the W
  // face come from the next / previous lane, the S face from the previous
  // row (each interior face evaluated once, see harmonic_face_T)
  static_assert(S == 32, "one lane per column");
  double kc_next = kappa(lane, 0), tS = 0.0;
  for (int k = 0; k < CPL; ++k) {
    const int cell = lane + 32 * k, a = lane, b = k;
    const double kc = kc_next;
    if (k + 1 < CPL) kc_next = kappa(a, b + 1);
    if (!(kc > 0.0) || !isfinite(kc)) nan = true;
    const double kE = __shfl_down_sync(0xffffffffu, kc, 1);
    double T4[4];
    T4[1] = a < S - 1 ? harmonic_face_T(kc, kE) : edge_face_T<S>(t, sb, kc, a, b, kEdgeE);
    const double tW = __shfl_up_sync(0xffffffffu, T4[1], 1);
    T4[0] = a > 0 ? tW : edge_face_T<S>(t, sb, kc, a, b, kEdgeW);
    T4[3] = b < S - 1 ? harmonic_face_T(kc, kc_next) : edge_face_T<S>(t, sb, kc, a, b, kEdgeN);
    T4[2] = b > 0 ? tS : edge_face_T<S>(t, sb, kc, a, b, kEdgeS);
    tS = T4[3];
    const double d = jacobi_scale<T>(T4[0] + T4[1] + T4[2] + T4[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) coef[q * N + cell] = T4[q];
    coef[4 * N + cell] = d;
    coef[5 * N + cell] = kc;
    write_beta<S>(t, sb, kc, a, b, coef);
    sm.dsc[cell] = d;
  }
  if (__any_sync(0xffffffffu, nan) && lane == 0) atomicOr(&w.status[0], MRCM_FLAG_NAN);
  __syncwarp();
  for (int k = 0; k < CPL; ++k) {
    const int cell = lane + 32 * k, a = cell % S, b = cell / S;
    const double d = sm.dsc[cell];
    sm.offx[cell] = static_cast<T>(a < S - 1 ? -coef[N + cell] * d * sm.dsc[cell + 1] : 0.0);
    sm.ecp[cell] = static_cast<T>(b < S - 1 ? -coef[3 * N + cell] * d * sm.dsc[cell + S] : 0.0);
  }
  __syncwarp();
  T *Wg = static_cast<T *>(w.W) + sb.w_off;
  const bool bad = schur_inverses<T, S>(lane, sm.offx, sm.ecp, Wg);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&w.status[0], MRCM_FLAG_NOTSPD);
}


// Right-hand side of one basis column at cell (a, b), FP64: the particular
// column carries the sources q h^2 and the physical boundary data (2 kappa
// p_b on a Dirichlet face, -u_b h on a Neumann face); a basis column carries
// Gravity (Eq. "Darcy_wg", height along +y, w = K lambda_g g per cell): the
// known part of a cell's outward flux through its S (n_y = -1) and N
// (n_y = +1) faces.  Inside the subdomain the face pressure is eliminated
// between the two half-cell fluxes 2 kappa (p_c - p_f)/h + n_y w_c, which
// leaves (kappa_c w_n + kappa_n w_c)/(kappa_c + kappa_n); a Robin face keeps
// n_y w_c T_R / (2 kappa_c) (p_f eliminated with -beta u + p_f = g); a
// Dirichlet face n_y w_c; a Neumann face nothing (its flux is given).
template <int S>
__device__ __forceinline__ double gravity_outflow(const DeviceTables &t, const SubInfo &sb,
                                                  const double *coef, int a, int b) {
  constexpr int N = S * S;
  const int tid = b * S + a, gi = sb.x0 + a, gj = sb.y0 + b;
  const double *wr = t.grav + static_cast<int64_t>(sb.r) * t.ny * t.nx;
  const double wc = wr[static_cast<int64_t>(gj) * t.nx + gi], kc = coef[5 * N + tid];
  double out = 0.0;
  for (int side = kEdgeS; side <= kEdgeN; ++side) {
    const double ny = side == kEdgeN ? 1.0 : -1.0;
    const bool edge = side == kEdgeN ? b == S - 1 : b == 0;
    if (!edge) {
      const int dn = side == kEdgeN ? S : -S, gjn = side == kEdgeN ? gj + 1 : gj - 1;
      const double kn = coef[5 * N + tid + dn], wn = wr[static_cast<int64_t>(gjn) * t.nx + gi];
      out += ny * (kc * wn + kn * wc) / (kc + kn);
    } else if (sb.edge_iface[side] >= 0) {
      out += ny * wc * coef[side * N + tid] / (2.0 * kc);
    } else {
      const int k = side == kEdgeS ? 2 * t.ny + gi : 2 * t.ny + t.nx + gi;
      if (t.bc_type[k] == 1) out += ny * wc;
    }
  }
  return out;
}

// T_R g on its own edge, g = -beta sigma phi_k(e) for a flux function and
// psi_k(e) for a pressure function (Eq. "mrc1").  With gravity the
// particular column also carries minus the known gravity outflow.
template <int S>
__device__ __forceinline__ double rhs_value(const DeviceTables &t, const SubInfo &sb,
                                            const double *coef, const double *q,
                                            const ColInfo &ci, int a, int b) {
  constexpr int N = S * S;
  const int tid = b * S + a;
  const int gi = sb.x0 + a, gj = sb.y0 + b;
  const double h = t.h;
  double val = 0.0;
  if (ci.unk < 0) {
    const int64_t cell = (static_cast<int64_t>(sb.r) * t.ny + gj) * t.nx + gi;
    val = q[cell] * h * h;
    const bool onface[4] = {a == 0, a == S - 1, b == 0, b == S - 1};
#pragma unroll
    for (int side = 0; side < 4; ++side) {
      if (!onface[side] || sb.edge_iface[side] >= 0) continue;
      int k;
      if (side == kEdgeW) k = gj;
      else if (side == kEdgeE) k = t.ny + gj;
      else if (side == kEdgeS) k = 2 * t.ny + gi;
      else k = 2 * t.ny + t.nx + gi;
      if (t.bc_type[k] == 1) val += coef[side * N + tid] * t.bc_val[k];
      else val -= t.bc_val[k] * h;
    }
    if (t.grav) val -= h * gravity_outflow<S>(t, sb, coef, a, b);
  } else {
    const int side = ci.edge;
    const bool adj = (side == kEdgeW && a == 0) || (side == kEdgeE && a == S - 1) ||
                     (side == kEdgeS && b == 0) || (side == kEdgeN && b == S - 1);
    const int e = (side < 2) ? b : a;
    const FaceIface fi = face_iface(sb, side, e);
    // the column's data lives on the faces of its own interface only
    if (adj && fi.g == t.unk_iface[ci.unk]) {
      const double fv = iface_fn_at(t, fi.len, ci.fn, fi.e);
      double gval;
      if (ci.is_u) {
        const double beta = coef[6 * N + side * S + e];
        const double sigma = (side == kEdgeE || side == kEdgeN) ? 1.0 : -1.0;
        gval = -beta * sigma * fv;
      } else {
        gval = fv;
      }
      val = coef[side * N + tid] * gval;
    }
  }
  return val;
}

// One-sided traces of the finished columns on every interface edge face,
//   u(e) = T_R (p_c - g_e)/h,  p_face(e) = g_e + beta_e u(e),
// then this side's share of the rows of G (Eq. "mrc2"):
//   U rows: sigma * sum_e h phi_k(e) p_face(e)    (pressure continuity)
//   P rows: sum_e h psi_k(e) u(e)                 (flux continuity)
// x: column c of the CTA at x + c S^2 (FP64).  All threads of the CTA.
template <int S, int NCMAX>
__device__ __forceinline__ void traces_and_rows(const DeviceTables &t, const Workspace &w,
                                                const SubInfo &sb, const double *coef,
                                                const ColInfo *col, const double *x, int c0,
                                                int nc, double (*su)[S][NCMAX],
                                                double (*sp)[S][NCMAX]) {
  constexpr int N = S * S;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const double h = t.h, inv_h = t.inv_h;
  for (int q = tid; q < 4 * S * nc; q += nthr) {
    const int side = q / (S * nc), e = (q / nc) % S, c = q % nc;
    if (sb.edge_iface[side] < 0) continue;
    const FaceIface fe = face_iface(sb, side, e);
    int la, lb;
    if (side == kEdgeW) { la = 0; lb = e; }
    else if (side == kEdgeE) { la = S - 1; lb = e; }
    else if (side == kEdgeS) { la = e; lb = 0; }
    else { la = e; lb = S - 1; }
    const int cl = lb * S + la;
    const double TR = coef[side * N + cl];
    const double beta = coef[6 * N + side * S + e];
    const ColInfo ci = col[c];
    double ge = 0.0;
    if (ci.edge == side && fe.g == t.unk_iface[ci.unk]) {
      const double fv = iface_fn_at(t, fe.len, ci.fn, fe.e);
      const double sigma = (side == kEdgeE || side == kEdgeN) ? 1.0 : -1.0;
      ge = ci.is_u ? -beta * sigma * fv : fv;
    }
    double u = TR * inv_h * (x[c * N + cl] - ge);
    if (t.grav && ci.unk < 0 && side >= kEdgeS) {   // the particular column's gravity part
      const double wc = t.grav[(static_cast<int64_t>(sb.r) * t.ny + sb.y0 + lb) * t.nx + sb.x0 + la];
      u += (side == kEdgeN ? 1.0 : -1.0) * wc * TR / (2.0 * coef[5 * N + cl]);
    }
    su[side][e][c] = u;
    sp[side][e][c] = ge + beta * u;
  }
  __syncthreads();
  double *G = w.G + sb.g_off;
  const int nrow = sb.nrows;
  for (int pr = tid; pr < nrow * nc; pr += nthr) {
    const int row = pr / nc, c = pr % nc;
    // the interface (segment) whose rows hold this row: edge side, half hf
    int side = 0, hf = 0;
    for (int q = 0; q < 8; ++q) {
      const int sd = q >> 1, hh = q & 1;
      const int g = hh ? sb.edge_iface2[sd] : sb.edge_iface[sd];
      if (g < 0) continue;
      const int r0 = hh ? sb.edge_row2[sd] : sb.edge_row[sd];
      if (row >= r0 && row < r0 + t.iface[g].nU + t.iface[g].nP) {
        side = sd;
        hf = hh;
        break;
      }
    }
    const IfaceInfo &fr = t.iface[hf ? sb.edge_iface2[side] : sb.edge_iface[side]];
    const int nU = fr.nU, len = fr.s, e0 = hf ? len : 0;
    const int k = row - (hf ? sb.edge_row2[side] : sb.edge_row[side]);
    const bool urow = k < nU;
    const double *fn = t.fnval + (len == 16 ? 0 : t.fn_off32) +
                       static_cast<int64_t>(urow ? fr.fnU + k : fr.fnP + k - nU) * len;
    double acc = 0.0;
    if (urow) {
      for (int e = 0; e < len; ++e) acc += fn[e] * sp[side][e0 + e][c];
      acc *= (side == kEdgeE || side == kEdgeN) ? h : -h;
    } else {
      for (int e = 0; e < len; ++e) acc += fn[e] * su[side][e0 + e][c];
      acc *= h;
    }
    G[static_cast<int64_t>(row) * sb.ncols + c0 + c] = acc;
  }
}

// ---------------------------------------------------------------------------
// (c): one CTA per (subdomain, block of up to NC <= 16 basis columns; NC is
// the tile width the autotuner chooses).
template <typename T, int NC>
struct BasisSmem {
  T Ws[kS * kS * kS];       // W_j, j = 0..S-1 (symmetric)
  T ec[kS * kS];            // scaled row couplings e_j[a]
  T offx[kS * kS];          // scaled in-row couplings (fused factor only)
  T z[NC * kS * kS];       // scaled residual (input of the solve)
  T v[NC * kS * kS];       // forward values, then the solution
  double coef[kCoefStride]; // tW tE tS tN d kappa, edge beta
  double su[4][kS][NC];    // one-sided velocity traces on the four edges
  double sp[4][kS][NC];    // face-pressure traces
  double x[NC * kS * kS];  // FP64 iterate
  double bb[NC * kS * kS]; // FP64 right-hand sides
  float redf[NC][kS * kS / 32];
  float bnf[NC];
  float rnf[NC];
  float rel2;
  ColInfo col[NC];
};

template <typename T, int NC>
__device__ void block_solve(BasisSmem<T, NC> &sm, int nc) {
  // y = L^{-T} D^{-1} L^{-1} z for the block LDL^T of the scaled operator.
  // Column c is carried by the 16 threads (a, c), all in one warp (c = tid /
  // 16), and its steps touch only its own z and v: a warp barrier orders the
  // steps; one CTA barrier at the end publishes v to the other warps.
  constexpr int S = kS, N = S * S;
  const int tid = threadIdx.x;
  const int a = tid % S, c = tid / S;
  const bool act = c < nc;
  // forward: v_j = W_j (z_j - e_{j-1} * v_{j-1})
  for (int j = 0; j < S; ++j) {
    if (act) {
      const T *Wj = sm.Ws + j * N;
      const T *zj = sm.z + c * N + j * S;
      T acc = T(0);
      if (j == 0) {
#pragma unroll
        for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * zj[bq];
      } else {
        const T *vp = sm.v + c * N + (j - 1) * S;
        const T *ep = sm.ec + (j - 1) * S;
#pragma unroll
        for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * (zj[bq] - ep[bq] * vp[bq]);
      }
      sm.v[c * N + j * S + a] = acc;
    }
    __syncwarp();
  }
  // backward: y_j = v_j - W_j (e_j * y_{j+1})
  for (int j = S - 2; j >= 0; --j) {
    if (act) {
      const T *Wj = sm.Ws + j * N;
      const T *yn = sm.v + c * N + (j + 1) * S;
      const T *ep = sm.ec + j * S;
      T acc = T(0);
#pragma unroll
      for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * (ep[bq] * yn[bq]);
      sm.v[c * N + j * S + a] -= acc;
    }
    __syncwarp();
  }
  __syncthreads();
}

// The same solve on the twisted factor (schur_inverses_twisted): one warp
// per column (columns c, c + 8, ...), lanes 0-15 (row a = lane) walking the
// block rows 0 .. M-1 down and lanes 16-31 the rows S-1 .. M+1 up, in
// lock step; the middle row M joins them, then both halves substitute back
// towards their ends.  17 dependent block steps instead of 31 at S = 16.
//   forward:  v_j = W_j (z_j - E_{j-1} v_{j-1})  (top),
//             v_j = W_j (z_j - E_j v_{j+1})      (bottom),
//             v_M = W_M (z_M - E_{M-1} v_{M-1} - E_M v_{M+1});
//   backward: y_j = v_j - W_j E_j y_{j+1}        (top, j = M-1 .. 0),
//             y_j = v_j - W_j E_{j-1} y_{j-1}    (bottom, j = M+1 .. S-1).
template <typename T, int NC>
__device__ void block_solve_twisted(BasisSmem<T, NC> &sm, int nc) {
  constexpr int S = kS, N = S * S, M = S / 2;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int a = lane & (S - 1);
  const bool bot = lane >= S;
  static_assert(2 * S == 32 && kS * kS / 32 == 8, "a half warp per block row, 8 warps");
  for (int c = wid; c < nc; c += 8) {
    T *v = sm.v + c * N;
    const T *z = sm.z + c * N;
    for (int k = 0; k < M; ++k) {
      const int j = bot ? S - 1 - k : k;
      if (!bot || j > M) {
        const T *Wj = sm.Ws + j * N;
        const T *zj = z + j * S;
        T acc = T(0);
        if (k == 0) {
#pragma unroll
          for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * zj[bq];
        } else {
          const T *vp = v + (bot ? j + 1 : j - 1) * S;
          const T *ep = sm.ec + (bot ? j : j - 1) * S;
#pragma unroll
          for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * (zj[bq] - ep[bq] * vp[bq]);
        }
        v[j * S + a] = acc;
      }
      __syncwarp();
    }
    if (!bot) {
      const T *Wm = sm.Ws + M * N;
      const T *zm = z + M * S, *vt = v + (M - 1) * S, *vb = v + (M + 1) * S;
      const T *et = sm.ec + (M - 1) * S, *eb = sm.ec + M * S;
      T acc = T(0);
#pragma unroll
      for (int bq = 0; bq < S; ++bq)
        acc += Wm[bq * S + a] * (zm[bq] - et[bq] * vt[bq] - eb[bq] * vb[bq]);
      v[M * S + a] = acc;
    }
    __syncwarp();
    for (int k = 0; k < M; ++k) {
      const int j = bot ? M + 1 + k : M - 1 - k;
      if (!bot || j < S) {
        const T *Wj = sm.Ws + j * N;
        const T *yn = v + (bot ? j - 1 : j + 1) * S;
        const T *ep = sm.ec + (bot ? j - 1 : j) * S;
        T acc = T(0);
#pragma unroll
        for (int bq = 0; bq < S; ++bq) acc += Wj[bq * S + a] * (ep[bq] * yn[bq]);
        v[j * S + a] -= acc;
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// per-column sum over the CTA of val[c] (c < nc) into out[c]
template <typename T, int NC>
__device__ void column_sums(BasisSmem<T, NC> &sm, const float *val, int nc, float *out) {
  constexpr int NW = kS * kS / 32;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (c < nc) {
      float s = val[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sm.redf[c][wid] = s;
    }
  }
  __syncthreads();
  if (tid < nc) {
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < NW; ++k) s += sm.redf[tid][k];
    out[tid] = s;
  }
  __syncthreads();
}

// FUSED: the inverse Schur blocks are computed here (warp 0, into shared
// memory) from the coefficients instead of read from global memory: the
// FP32 factor of one subdomain costs one warp's pivot chain per column
// chunk, and saves a launch and the W round trip.
template <typename T, int NC, bool FUSED = false>
__global__ void __launch_bounds__(kS *kS) k_basis(DeviceTables t, Workspace w,
                                                  const BasisItem *items, const double *q,
                                                  double tol, int ir_max) {
  constexpr int S = kS, N = S * S;
  extern __shared__ __align__(16) unsigned char smraw[];
  BasisSmem<T, NC> &sm = *reinterpret_cast<BasisSmem<T, NC> *>(smraw);
  const BasisItem it = items[blockIdx.x];
  if (it.nc == 0) return;   // an unused slot of the recovery launch (whole CTA)
  const int g = it.sub;
  const SubInfo sb = t.sub[g];
  const int nc = it.nc;
  const int tid = threadIdx.x;
  const int a = tid % S, b = tid / S;

  // stage W_j, the coefficients and the column descriptors: 16-byte loads,
  // all of a thread's loads issued before its stores (both arrays start on a
  // 16-byte boundary: offsets are multiples of S^3 elements and of the even
  // coefficient stride)
  {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int NW = S * N * static_cast<int>(sizeof(T)) / 16 / N;   // vectors per thread
    const V *wsrc = reinterpret_cast<const V *>(static_cast<const T *>(w.W) + sb.w_off);
    V *wdst = reinterpret_cast<V *>(sm.Ws);
    constexpr int NCV = kCoefStride / 2, NCT = (NCV + N - 1) / N;
    const double2 *csrc = reinterpret_cast<const double2 *>(w.coef + sb.coef_off);
    double2 *cdst = reinterpret_cast<double2 *>(sm.coef);
    V wv[NW];
    double2 cv[NCT];
    if constexpr (!FUSED) {
#pragma unroll
      for (int k = 0; k < NW; ++k) wv[k] = wsrc[tid + k * N];
    }
#pragma unroll
    for (int k = 0; k < NCT; ++k)
      if (tid + k * N < NCV) cv[k] = csrc[tid + k * N];
    if (tid < nc) sm.col[tid] = t.col[sb.col_off + it.c0 + tid];
    if constexpr (!FUSED) {
#pragma unroll
      for (int k = 0; k < NW; ++k) wdst[tid + k * N] = wv[k];
    }
#pragma unroll
    for (int k = 0; k < NCT; ++k)
      if (tid + k * N < NCV) cdst[tid + k * N] = cv[k];
  }
  __syncthreads();
  const double *tWs = sm.coef, *tEs = sm.coef + N, *tSs = sm.coef + 2 * N,
               *tNs = sm.coef + 3 * N, *ds = sm.coef + 4 * N, *ks = sm.coef + 5 * N;
  if (b < S - 1) sm.ec[tid] = static_cast<T>(-tNs[tid] * ds[tid] * ds[tid + S]);
  else sm.ec[tid] = T(0);
  // right-hand sides of cell ``cell`` for every column (FP64), the zero
  // iterate and the scaled residual z = D b
  auto rhs_cell = [&](int cell) {
    const double dc = ds[cell];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c >= nc) continue;
      const double val = rhs_value<S>(t, sb, sm.coef, q, sm.col[c], cell % S, cell / S);
      sm.bb[c * N + cell] = val;
      sm.x[c * N + cell] = 0.0;
      sm.z[c * N + cell] = static_cast<T>(dc * val);
    }
  };
  if constexpr (FUSED) {
    // the scaled couplings exactly as the factor kernel forms them; then the
    // Schur-block chain of this subdomain in warp 0 while the other warps
    // set up the right-hand sides of all cells
    sm.offx[tid] = a < S - 1 ? static_cast<T>(-tEs[tid] * ds[tid] * ds[tid + 1]) : T(0);
    __syncthreads();
    if constexpr (std::is_same<T, float>::value) {
      // the twisted chain on warps 0 and 1, the right-hand sides on the rest
      if (tid < 64) {
        const bool bad = schur_inverses_twisted<S>(tid >> 5, tid & 31, sm.offx, sm.ec, sm.Ws);
        if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0)
          atomicOr(&w.status[0], MRCM_FLAG_NOTSPD);
      } else {
        for (int cell = tid - 64; cell < N; cell += N - 64) rhs_cell(cell);
      }
    } else {
      if (tid < 32) {
        const bool bad = schur_inverses<T, S>(tid, sm.offx, sm.ec, sm.Ws);
        if (__any_sync(0xffffffffu, bad) && tid == 0) atomicOr(&w.status[0], MRCM_FLAG_NOTSPD);
      } else {
        for (int cell = tid - 32; cell < N; cell += N - 32) rhs_cell(cell);
      }
    }
    __syncthreads();
  } else {
    rhs_cell(tid);
  }

  const double myT[4] = {tWs[tid], tEs[tid], tSs[tid], tNs[tid]};
  const double dsl = ds[tid];
  const float dsf = static_cast<float>(dsl);
  const double mydiag = myT[0] + myT[1] + myT[2] + myT[3];
  float bnl[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float zv = c < nc ? static_cast<float>(sm.z[c * N + tid]) : 0.0f;
    bnl[c] = zv * zv;
  }
  column_sums(sm, bnl, nc, sm.bnf);

  // refinement loop: z holds D r in the working precision.  Convergence is
  // tested on the Jacobi-scaled residual, ||D r|| <= tol ||D b|| per column,
  // with squared norms (no division on the FP64 pipe).
  const float tol2 = static_cast<float>(tol) * static_cast<float>(tol);
  int sweep = 0;
  float prev2 = 3e38f, rel2 = 0.0f;
  for (;;) {
    if constexpr (std::is_same<T, float>::value) block_solve_twisted(sm, nc);
    else block_solve(sm, nc);
    for (int c = 0; c < nc; ++c) {
      if (sizeof(T) == sizeof(float))
        sm.x[c * N + tid] += f32_to_f64(dsf * static_cast<float>(sm.v[c * N + tid]));
      else
        sm.x[c * N + tid] += dsl * static_cast<double>(sm.v[c * N + tid]);
    }
    __syncthreads();
    if (sweep >= ir_max) break;
    // FP64 residual r = b - A x (five FP64 FMAs per cell and column)
    float rn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      rn[c] = 0.0f;
      if (c >= nc) continue;
      const double *xc = sm.x + c * N;
      double r = fma(-mydiag, xc[tid], sm.bb[c * N + tid]);
      if (a > 0) r = fma(myT[0], xc[tid - 1], r);
      if (a < S - 1) r = fma(myT[1], xc[tid + 1], r);
      if (b > 0) r = fma(myT[2], xc[tid - S], r);
      if (b < S - 1) r = fma(myT[3], xc[tid + S], r);
      T zv;
      if (sizeof(T) == sizeof(float)) zv = static_cast<T>(f64_to_f32(r) * dsf);
      else zv = static_cast<T>(dsl * r);
      sm.z[c * N + tid] = zv;
      rn[c] = static_cast<float>(zv) * static_cast<float>(zv);
    }
    column_sums(sm, rn, nc, sm.rnf);
    if (tid < 32) {
      float rr = 0.0f;
      if (tid < nc) rr = sm.bnf[tid] > 0.0f ? sm.rnf[tid] / sm.bnf[tid] : 0.0f;
      if (rr != rr) rr = 3e38f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, o));
      if (tid == 0) sm.rel2 = rr;
    }
    __syncthreads();
    rel2 = sm.rel2;
    ++sweep;
    if (rel2 <= tol2) break;
    if (sweep > 2 && rel2 > 0.25f * prev2) break;  // stalled
    prev2 = rel2;
  }
  if (tid == 0 && ir_max > 0) {
    atomicMax(&w.status[1], sweep);
    report_local_resid(w, g, sqrt(static_cast<double>(rel2)), tol);
  }

  // basis columns (FP64)
  double *bas = w.basis + sb.basis_off;
  for (int c = 0; c < nc; ++c) bas[static_cast<int64_t>(it.c0 + c) * N + tid] = sm.x[c * N + tid];

  traces_and_rows<S, NC>(t, w, sb, sm.coef, sm.col, sm.x, it.c0, nc, sm.su, sm.sp);
}

// ---------------------------------------------------------------------------
// (c) for s = 32.  The S inverse Schur blocks (S^3 values) do not fit in
// shared memory next to the right-hand sides, so W_j is streamed through a
// double buffer, one block per solve step (prefetched during the step
// before), and the FP64 iterate lives in the basis array itself: each
// thread owns one cell of every column of the CTA.  Each 32-term row of a
// W_j product is split over kKS threads and summed with shuffles.
constexpr int kS32 = 32;
// NC columns per CTA (4 or 8), KS = 32 / NC threads per W row, W rows padded to
// 32 + KS floats so the split reads are bank-conflict free
template <int NC>
struct Split32 {
  static constexpr int KS = kS32 / NC;
  static constexpr int Wst = kS32 + KS;
  static_assert(KS * kS32 * NC == kS32 * kS32, "one thread per (split, row, column)");
};

template <typename T, int NC>
struct BasisSmem32 {
  T Wb[2][kS32 * Split32<NC>::Wst];
  T ec[kS32 * kS32];
  T z[NC * kS32 * kS32];
  T v[NC * kS32 * kS32];
  double su[4][kS32][NC];
  double sp[4][kS32][NC];
  float redf[NC][kS32 * kS32 / 32];
  float bnf[NC];
  float rnf[NC];
  float rel2;
  ColInfo col[NC];
};

template <typename T, int NC>
__device__ void block_solve32(BasisSmem32<T, NC> &sm, const T *Wg, int nc) {
  constexpr int S = kS32, N = S * S, NSTEP = 2 * S - 1;
  constexpr int kKS = Split32<NC>::KS, kWst = Split32<NC>::Wst;
  const int tid = threadIdx.x;
  const int ks = tid % kKS, o = tid / kKS, a = o % S, c = o / S;
  const bool act = c < nc;            // uniform over a warp (c = tid / 128)
  const int wrow = (tid / S) * kWst + tid % S;
  // W_j of step kk (forward j = kk, backward j = 2S - 2 - kk); this thread's
  // element is loaded two steps ahead (a step is about one L2 round trip)
  auto wstep = [&](int kk) {
    const int jj = kk < S ? kk : 2 * S - 2 - kk;
    return Wg[static_cast<int64_t>(jj) * N + tid];
  };
  sm.Wb[0][wrow] = Wg[tid];
  T w1 = NSTEP > 1 ? wstep(1) : T(0);
  __syncthreads();
  int buf = 0;
  for (int k = 0; k < NSTEP; ++k) {
    const int j = k < S ? k : 2 * S - 2 - k;
    const T nextw = w1;
    if (k + 2 < NSTEP) w1 = wstep(k + 2);
    const T *Wj = sm.Wb[buf] + a * kWst;
    T acc = T(0);
    if (act) {
      if (k < S) {
        // forward: v_j = W_j (z_j - e_{j-1} v_{j-1})
        const T *zj = sm.z + c * N + j * S;
        if (j == 0) {
#pragma unroll
          for (int q = 0; q < S / kKS; ++q) {
            const int bq = ks + kKS * q;
            acc += Wj[bq] * zj[bq];
          }
        } else {
          const T *vp = sm.v + c * N + (j - 1) * S;
          const T *ep = sm.ec + (j - 1) * S;
#pragma unroll
          for (int q = 0; q < S / kKS; ++q) {
            const int bq = ks + kKS * q;
            acc += Wj[bq] * (zj[bq] - ep[bq] * vp[bq]);
          }
        }
      } else {
        // backward: y_j = v_j - W_j (e_j y_{j+1})
        const T *yn = sm.v + c * N + (j + 1) * S;
        const T *ep = sm.ec + j * S;
#pragma unroll
        for (int q = 0; q < S / kKS; ++q) {
          const int bq = ks + kKS * q;
          acc += Wj[bq] * (ep[bq] * yn[bq]);
        }
      }
    }
#pragma unroll
    for (int m = 1; m < kKS; m <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, m);
    if (act && ks == 0) {
      if (k < S) sm.v[c * N + j * S + a] = acc;
      else sm.v[c * N + j * S + a] -= acc;
    }
    if (k + 1 < NSTEP) sm.Wb[buf ^ 1][wrow] = nextw;
    __syncthreads();
    buf ^= 1;
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(kS32 *kS32, 1) k_basis32(DeviceTables t, Workspace w,
                                                           const BasisItem *items,
                                                           const double *q, double tol,
                                                           int ir_max) {
  constexpr int S = kS32, N = S * S, NW = N / 32;
  extern __shared__ __align__(16) unsigned char smraw[];
  BasisSmem32<T, NC> &sm = *reinterpret_cast<BasisSmem32<T, NC> *>(smraw);
  const BasisItem it = items[blockIdx.x];
  if (it.nc == 0) return;   // an unused slot of the recovery launch (whole CTA)
  const SubInfo sb = t.sub[it.sub];
  const int nc = it.nc;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int a = tid % S, b = tid / S;
  const T *Wg = static_cast<const T *>(w.W) + sb.w_off;
  const double *coef = w.coef + sb.coef_off;
  double *X = w.basis + sb.basis_off + static_cast<int64_t>(it.c0) * N;
  if (tid < nc) sm.col[tid] = t.col[sb.col_off + it.c0 + tid];
  const double myT[4] = {coef[tid], coef[N + tid], coef[2 * N + tid], coef[3 * N + tid]};
  const double dsl = coef[4 * N + tid];
  const float dsf = static_cast<float>(dsl);
  const double mydiag = myT[0] + myT[1] + myT[2] + myT[3];
  sm.ec[tid] = b < S - 1 ? static_cast<T>(-myT[3] * dsl * coef[4 * N + tid + S]) : T(0);
  __syncthreads();

  auto col_sums = [&](const float *val, float *out) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (c < nc) {
        float s2 = val[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        if (lane == 0) sm.redf[c][wid] = s2;
      }
    }
    __syncthreads();
    if (tid < nc) {
      float s2 = 0.0f;
      for (int k = 0; k < NW; ++k) s2 += sm.redf[tid][k];
      out[tid] = s2;
    }
    __syncthreads();
  };

  double bb[NC];
  float bnl[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    bb[c] = 0.0;
    bnl[c] = 0.0f;
    if (c >= nc) continue;
    const double val = rhs_value<S>(t, sb, coef, q, sm.col[c], a, b);
    bb[c] = val;
    X[c * N + tid] = 0.0;
    const T zv = static_cast<T>(dsl * val);
    sm.z[c * N + tid] = zv;
    bnl[c] = static_cast<float>(zv) * static_cast<float>(zv);
  }
  col_sums(bnl, sm.bnf);

  const float tol2 = static_cast<float>(tol) * static_cast<float>(tol);
  int sweep = 0;
  float prev2 = 3e38f, rel2 = 0.0f;
  for (;;) {
    block_solve32(sm, Wg, nc);
    for (int c = 0; c < nc; ++c) {
      if (sizeof(T) == sizeof(float))
        X[c * N + tid] += f32_to_f64(dsf * static_cast<float>(sm.v[c * N + tid]));
      else
        X[c * N + tid] += dsl * static_cast<double>(sm.v[c * N + tid]);
    }
    __syncthreads();
    if (sweep >= ir_max) break;
    // FP64 residual r = b - A x, the neighbours' x from the basis array
    float rn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      rn[c] = 0.0f;
      if (c >= nc) continue;
      const double *xc = X + c * N;
      double r = fma(-mydiag, xc[tid], bb[c]);
      if (a > 0) r = fma(myT[0], xc[tid - 1], r);
      if (a < S - 1) r = fma(myT[1], xc[tid + 1], r);
      if (b > 0) r = fma(myT[2], xc[tid - S], r);
      if (b < S - 1) r = fma(myT[3], xc[tid + S], r);
      T zv;
      if (sizeof(T) == sizeof(float)) zv = static_cast<T>(f64_to_f32(r) * dsf);
      else zv = static_cast<T>(dsl * r);
      sm.z[c * N + tid] = zv;
      rn[c] = static_cast<float>(zv) * static_cast<float>(zv);
    }
    col_sums(rn, sm.rnf);
    if (tid < 32) {
      float rr = 0.0f;
      if (tid < nc) rr = sm.bnf[tid] > 0.0f ? sm.rnf[tid] / sm.bnf[tid] : 0.0f;
      if (rr != rr) rr = 3e38f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, o));
      if (tid == 0) sm.rel2 = rr;
    }
    __syncthreads();
    rel2 = sm.rel2;
    ++sweep;
    if (rel2 <= tol2) break;
    if (sweep > 2 && rel2 > 0.25f * prev2) break;  // stalled
    prev2 = rel2;
  }
  if (tid == 0 && ir_max > 0) {
    atomicMax(&w.status[1], sweep);
    report_local_resid(w, it.sub, sqrt(static_cast<double>(rel2)), tol);
  }
  traces_and_rows<S, NC>(t, w, sb, coef, sm.col, X, it.c0, nc, sm.su, sm.sp);
}

// ---------------------------------------------------------------------------
// (c) for s = 32 on the mixed path: one warp per basis column.
//
// The columns of a subdomain are independent right-hand sides, and the block
// solve's 63 dependent steps (forward j = 0..31, backward j = 30..0) only
// couple the 32 cells of one grid row of one column.  So each warp carries
// one column: lane a holds z and v of cell (a, j) for every block row j in
// registers, a step is the 32 x 32 product W_j in, with `in` broadcast by
// shuffles, and no step waits for another warp.  All 32 inverse Schur blocks
// (128 KB, FP32) stay resident in shared memory, copied asynchronously while
// the right-hand sides are formed.  Lane a reads row a of W_j with a
// diagonal skew (column (k + a) mod 32 at inner step k), which keeps the 32
// lanes on 32 banks.  The FP64 residual takes the lane's own iterate values
// of rows j-1, j, j+1 and its neighbours' by shuffles.  Each column stops on
// its own test, so the result does not depend on how columns are grouped
// into CTAs.
template <int NW>
struct Basis32W {
  float W[kS32 * kS32 * kS32];   // W_j, j = 0..31, row-major [j][a][q]
  float ec[kS32 * kS32];         // scaled row couplings e_j[a]
  float z[NW][kS32 * kS32];      // each warp's scaled residual, [j][a]
  double diag[kS32 * kS32];      // FP64 diagonal tW + tE + tS + tN of every cell
  float dsf[kS32 * kS32];        // the Jacobi scale d in FP32
  ColInfo col[NW];
};

template <int NW>
__global__ void __launch_bounds__(32 * NW, 1) k_basis32w(DeviceTables t, Workspace w,
                                                         const BasisItem *items, const double *q,
                                                         double tol, int ir_max) {
  constexpr int S = kS32, N = S * S;
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smraw[];
  Basis32W<NW> &sm = *reinterpret_cast<Basis32W<NW> *>(smraw);
  const BasisItem it = items[blockIdx.x];
  const SubInfo sb = t.sub[it.sub];
  const int nc = it.nc;
  const int tid = threadIdx.x, lane = tid & 31, c = tid >> 5;
  const float *Wg = static_cast<const float *>(w.W) + sb.w_off;
  const double *coef = w.coef + sb.coef_off;   // tW tE tS tN d: read through L1
  double *X = w.basis + sb.basis_off + static_cast<int64_t>(it.c0) * N;
  // W (16-byte chunks; w_off is a multiple of S^3 floats) in flight while the
  // right-hand sides are set up
  {
    const unsigned sdst = static_cast<unsigned>(__cvta_generic_to_shared(sm.W));
    for (int k = tid; k < N * S / 4; k += 32 * NW)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst + 16u * k),
                   "l"(Wg + 4 * k)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  if (tid < nc) sm.col[tid] = t.col[sb.col_off + it.c0 + tid];
  // per-cell constants of every sweep, formed once per CTA (the FP64 pipe
  // bounds this kernel)
  for (int k = tid; k < N; k += 32 * NW) {
    sm.ec[k] = k / S < S - 1
                   ? static_cast<float>(-coef[3 * N + k] * coef[4 * N + k] * coef[4 * N + k + S])
                   : 0.0f;
    sm.diag[k] = coef[k] + coef[N + k] + coef[2 * N + k] + coef[3 * N + k];
    sm.dsf[k] = static_cast<float>(coef[4 * N + k]);
  }
  __syncthreads();
  const bool act = c < nc;
  ColInfo ci{};
  if (act) ci = sm.col[c];
  float *zc = sm.z[c];
  double *Xc = X + static_cast<int64_t>(c) * N;
  // right-hand side and scaled initial residual z = D b of this column
  float bn = 0.0f;
  if (act)
    for (int j = 0; j < S; ++j) {
      const int k = j * S + lane;
      const float zv = static_cast<float>(coef[4 * N + k] * rhs_value<S>(t, sb, coef, q, ci, lane, j));
      zc[k] = zv;
      bn = fmaf(zv, zv, bn);
      Xc[k] = 0.0;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bn += __shfl_xor_sync(FULL, bn, o);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();

  const float tol2 = static_cast<float>(tol) * static_cast<float>(tol);
  int sweep = 0;
  float prev2 = 3e38f, rel2 = 0.0f;
  while (act) {
    // forward: v_j = W_j (z_j - e_{j-1} v_{j-1}), in place over z (each lane
    // reads and writes only its own entry; the exchange is by shuffles)
    float vp = 0.0f;
#pragma unroll 4
    for (int j = 0; j < S; ++j) {
      const float in = j == 0 ? zc[lane] : zc[j * S + lane] - sm.ec[(j - 1) * S + lane] * vp;
      const float *Wa = sm.W + j * N + lane * S;
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int k = 0; k < S; k += 2) {
        const int q0 = (k + lane) & (S - 1), q1 = (k + 1 + lane) & (S - 1);
        a0 = fmaf(Wa[q0], __shfl_sync(FULL, in, q0), a0);
        a1 = fmaf(Wa[q1], __shfl_sync(FULL, in, q1), a1);
      }
      vp = a0 + a1;
      zc[j * S + lane] = vp;
    }
    // backward: y_j = v_j - W_j (e_j y_{j+1}), y_31 = v_31; then x += D y
    // (the correction in FP32, accumulated in FP64)
    Xc[(S - 1) * S + lane] += f32_to_f64(sm.dsf[(S - 1) * S + lane] * vp);
#pragma unroll 4
    for (int j = S - 2; j >= 0; --j) {
      const float tq = sm.ec[j * S + lane] * vp;
      const float *Wa = sm.W + j * N + lane * S;
      float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
      for (int k = 0; k < S; k += 2) {
        const int q0 = (k + lane) & (S - 1), q1 = (k + 1 + lane) & (S - 1);
        a0 = fmaf(Wa[q0], __shfl_sync(FULL, tq, q0), a0);
        a1 = fmaf(Wa[q1], __shfl_sync(FULL, tq, q1), a1);
      }
      vp = zc[j * S + lane] - (a0 + a1);
      Xc[j * S + lane] += f32_to_f64(sm.dsf[j * S + lane] * vp);
    }
    if (sweep >= ir_max) break;
    // FP64 residual r = b - A x over rows j-1, j, j+1 of this lane's cells
    float rn = 0.0f;
    double xm = 0.0, xc = Xc[lane];
    for (int j = 0; j < S; ++j) {
      const double xp = j < S - 1 ? Xc[(j + 1) * S + lane] : 0.0;
      const double xl = __shfl_up_sync(FULL, xc, 1), xr = __shfl_down_sync(FULL, xc, 1);
      const int k = j * S + lane;
      const double tW = coef[k], tE = coef[N + k], tS = coef[2 * N + k], tN = coef[3 * N + k];
      const double diag = sm.diag[k];
      double r = fma(-diag, xc, rhs_value<S>(t, sb, coef, q, ci, lane, j));
      if (lane > 0) r = fma(tW, xl, r);
      if (lane < S - 1) r = fma(tE, xr, r);
      if (j > 0) r = fma(tS, xm, r);
      if (j < S - 1) r = fma(tN, xp, r);
      const float zv = f64_to_f32(r) * sm.dsf[k];
      zc[k] = zv;
      rn = fmaf(zv, zv, rn);
      xm = xc;
      xc = xp;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rn += __shfl_xor_sync(FULL, rn, o);
    rel2 = bn > 0.0f ? rn / bn : 0.0f;
    if (rel2 != rel2) rel2 = 3e38f;
    ++sweep;
    if (rel2 <= tol2) break;
    if (sweep > 2 && rel2 > 0.25f * prev2) break;  // stalled
    prev2 = rel2;
    __syncwarp();
  }
  if (act && lane == 0 && ir_max > 0) {
    atomicMax(&w.status[1], sweep);
    report_local_resid(w, it.sub, sqrt(static_cast<double>(rel2)), tol);
  }
  __syncthreads();                 // every column done; W's space now holds the traces
  double(*su)[S][NW] = reinterpret_cast<double(*)[S][NW]>(sm.W);
  double(*sp)[S][NW] = reinterpret_cast<double(*)[S][NW]>(sm.W + 2 * 4 * S * NW);
  traces_and_rows<S, NW>(t, w, sb, coef, sm.col, X, it.c0, nc, su, sp);
}
static_assert(2 * 2 * 4 * kS32 * 16 <= kS32 * kS32 * kS32, "the traces fit in W's space");

// ---------------------------------------------------------------------------
// Refinement-stall recovery.  One warp per slot of the list the mixed basis
// kernels wrote: it lays out the slot's work items for the FP64 basis kernels
// (the unused slots' items are empty, so those CTAs return at once), copies
// the subdomain's SubInfo with w_off pointing into the FP64 scratch, and forms
// the FP64 inverse Schur blocks from the coefficients stage 1 of the factor
// stored (the scaled couplings exactly as the factor kernels form them).
template <int S>
__device__ bool refactor_fp64(int lane, const double *coef, double *offx, double *ecp,
                              double *W) {
  constexpr int N = S * S;
  const double *tE = coef + N, *tN = coef + 3 * N, *d = coef + 4 * N;
  for (int cell = lane; cell < N; cell += 32) {
    const int a = cell % S, b = cell / S;
    offx[cell] = a < S - 1 ? -tE[cell] * d[cell] * d[cell + 1] : 0.0;
    ecp[cell] = b < S - 1 ? -tN[cell] * d[cell] * d[cell + S] : 0.0;
  }
  __syncwarp();
  return schur_inverses<double, S>(lane, offx, ecp, W);
}

__global__ void __launch_bounds__(32) k_refactor64(DeviceTables t, Workspace w) {
  __shared__ double offx[kS32 * kS32], ecp[kS32 * kS32];
  const int slot = blockIdx.x, lane = threadIdx.x;
  const int nlisted = w.status[4];
  const int listed = nlisted < w.rec_cap ? nlisted : w.rec_cap;
  if (slot == 0 && lane == 0 && nlisted > 0) atomicOr(&w.status[0], MRCM_FLAG_LOCAL_REFACTOR);
  BasisItem *it16 = w.rec_items + static_cast<int64_t>(slot) * w.rec_maxch;
  BasisItem *it32 = it16 + static_cast<int64_t>(w.rec_cap) * w.rec_maxch;
  int g = -1, s = 0, ncol = 0, nch = 0;
  if (slot < listed) {
    g = w.stall_list[slot];
    s = t.sub[g].s;
    ncol = t.sub[g].ncols;
    nch = (ncol + kRecNC - 1) / kRecNC;   // <= rec_maxch (the largest ncols)
  }
  for (int k = lane; k < w.rec_maxch; k += 32) {
    BasisItem e{slot, 0, 0};
    if (k < nch) {
      e.c0 = ncol * k / nch;
      e.nc = ncol * (k + 1) / nch - e.c0;
    }
    it16[k] = s == 16 ? e : BasisItem{slot, 0, 0};
    it32[k] = s == 32 ? e : BasisItem{slot, 0, 0};
  }
  if (slot >= listed) return;
  SubInfo sb = t.sub[g];
  sb.w_off = static_cast<int64_t>(slot) * w.rec_smax * w.rec_smax * w.rec_smax;
  if (lane == 0) w.rec_sub[slot] = sb;
  const double *coef = w.coef + sb.coef_off;
  const bool bad = s == 16 ? refactor_fp64<kS>(lane, coef, offx, ecp, w.W64 + sb.w_off)
                           : refactor_fp64<kS32>(lane, coef, offx, ecp, w.W64 + sb.w_off);
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&w.status[0], MRCM_FLAG_NOTSPD);
}

// Pure-Neumann problems have a solution only when the sources balance the
// prescribed boundary outflow: the cell balances summed over the domain give
// sum_c q_c h^2 = sum_f u_f h (u_f the outward normal velocity of boundary
// face f).  One CTA per realisation sums both in FP64 (a fixed order: the
// result does not depend on timing) and raises MRCM_FLAG_INCOMPATIBLE when
// they differ by more than 1e-10 of the sum of their absolute values.
constexpr int kCompatThreads = 512;
__global__ void __launch_bounds__(kCompatThreads) k_compat(DeviceTables t, Workspace w,
                                                           const double *q) {
  const int r = blockIdx.x, tid = threadIdx.x;
  const int64_t n = static_cast<int64_t>(t.nx) * t.ny;
  const double *qr = q + static_cast<int64_t>(r) * n;
  double sq = 0.0, aq = 0.0, sb = 0.0, ab = 0.0;
  for (int64_t k = tid; k < n; k += kCompatThreads) {
    const double v = qr[k];
    sq += v;
    aq += fabs(v);
  }
  for (int k = tid; k < 2 * (t.nx + t.ny); k += kCompatThreads) {
    const double v = t.bc_val[k];
    sb += v;
    ab += fabs(v);
  }
  __shared__ double part[4][kCompatThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    aq += __shfl_xor_sync(0xffffffffu, aq, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    ab += __shfl_xor_sync(0xffffffffu, ab, o);
  }
  if ((tid & 31) == 0) {
    part[0][tid >> 5] = sq;
    part[1][tid >> 5] = aq;
    part[2][tid >> 5] = sb;
    part[3][tid >> 5] = ab;
  }
  __syncthreads();
  if (tid == 0) {
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < kCompatThreads / 32; ++k)
      for (int j = 0; j < 4; ++j) s4[j] += part[j][k];
    const double h = t.h;
    const double imbalance = s4[0] * h * h - s4[2] * h, scale = s4[1] * h * h + s4[3] * h;
    if (!(fabs(imbalance) <= 1e-10 * scale)) atomicOr(&w.status[0], MRCM_FLAG_INCOMPATIBLE);
  }
}

// Test hook: W[k] rounded to `bits` explicit mantissa bits, ties to even
// (bits = 7: the precision of bfloat16).
__global__ void k_degrade_factor(float *W, int n, int bits) {
  const unsigned shift = 23u - static_cast<unsigned>(bits);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    unsigned u = __float_as_uint(W[k]);
    u += ((1u << shift) >> 1) - 1u + ((u >> shift) & 1u);
    W[k] = __uint_as_float(u & ~((1u << shift) - 1u));
  }
}

}  // namespace

cudaError_t launch_recover(const DeviceTables &t, const Workspace &w, const double *q,
                           double ir_tol, cudaStream_t st) {
  if (w.rec_cap <= 0) return cudaSuccess;
  k_refactor64<<<w.rec_cap, 32, 0, st>>>(t, w);
  DeviceTables tr = t;
  tr.sub = w.rec_sub;
  Workspace wr = w;
  wr.W = w.W64;
  const int n = w.rec_cap * w.rec_maxch;
  if (t.nsub16 > 0)
    k_basis<double, kRecNC, false><<<n, kS * kS, sizeof(BasisSmem<double, kRecNC>), st>>>(
        tr, wr, w.rec_items, q, ir_tol, 0);
  if (t.nsub > t.nsub16)
    k_basis32<double, kRecNC><<<n, kS32 * kS32, sizeof(BasisSmem32<double, kRecNC>), st>>>(
        tr, wr, w.rec_items + n, q, ir_tol, 0);
  return cudaGetLastError();
}

cudaError_t launch_compat(const DeviceTables &t, const Workspace &w, const double *q,
                          cudaStream_t st) {
  k_compat<<<t.n_real, kCompatThreads, 0, st>>>(t, w, q);
  return cudaGetLastError();
}

cudaError_t launch_degrade_factor(float *W, int n, int bits, cudaStream_t st) {
  k_degrade_factor<<<(n + 255) / 256, 256, 0, st>>>(W, n, bits);
  return cudaGetLastError();
}

cudaError_t launch_factor(const DeviceTables &t, const Workspace &w, int prec, const double *K,
                          const double *lam, cudaStream_t st) {
  const int n16 = t.nsub16, n32 = t.nsub - t.nsub16;
  if (n16 > 0) {
    if (prec == MRCM_PREC_FP64)
      k_factor<double><<<n16, kS * kS, 0, st>>>(t, w, K, lam);
    else if (t.fuse16)   // coefficients only: the basis kernel factors each subdomain
      k_factor<float, false><<<n16, kS * kS, 0, st>>>(t, w, K, lam);
    else
      k_factor<float, true><<<n16, kS * kS, 0, st>>>(t, w, K, lam);
  }
  if (n32 > 0) {
    const int grid = (n32 + kFW - 1) / kFW;
    if (prec == MRCM_PREC_FP64)
      k_factor_warp<double, 32><<<grid, 32 * kFW, kFW * sizeof(FactorWarpSmem<double, 32>), st>>>(
          t, w, K, lam, n16, n32);
    else
      k_factor_warp<float, 32><<<grid, 32 * kFW, kFW * sizeof(FactorWarpSmem<float, 32>), st>>>(
          t, w, K, lam, n16, n32);
  }
  return cudaGetLastError();
}

template <typename T, int NC>
static cudaError_t basis16(const DeviceTables &t, const Workspace &w, const BasisItem *items, int n,
                           const double *q, double tol, int ir_max, cudaStream_t st) {
  if (std::is_same<T, float>::value && t.fuse16)   // the factor is fused in
    k_basis<T, NC, true><<<n, kS * kS, sizeof(BasisSmem<T, NC>), st>>>(t, w, items, q, tol, ir_max);
  else
    k_basis<T, NC, false><<<n, kS * kS, sizeof(BasisSmem<T, NC>), st>>>(t, w, items, q, tol, ir_max);
  return cudaGetLastError();
}
template <typename T, int NC>
static cudaError_t basis32(const DeviceTables &t, const Workspace &w, const BasisItem *items, int n,
                           const double *q, double tol, int ir_max, cudaStream_t st) {
  k_basis32<T, NC><<<n, kS32 * kS32, sizeof(BasisSmem32<T, NC>), st>>>(t, w, items, q, tol,
                                                                       ir_max);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_basis_t(const DeviceTables &t, const Workspace &w,
                                  const BasisItem *items, int n16, int n32, int nc16, int nc32,
                                  const double *q, double tol, int ir_max, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (n16 > 0) {
    switch (nc16) {
      case 4: e = basis16<T, 4>(t, w, items, n16, q, tol, ir_max, st); break;
      case 8: e = basis16<T, 8>(t, w, items, n16, q, tol, ir_max, st); break;
      case 12: e = basis16<T, 12>(t, w, items, n16, q, tol, ir_max, st); break;
      case 16: e = basis16<T, 16>(t, w, items, n16, q, tol, ir_max, st); break;
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  if (n32 > 0) {
    if constexpr (std::is_same<T, float>::value) {   // mixed path: one warp per column
      switch (nc32) {
        case 4: k_basis32w<4><<<n32, 128, sizeof(Basis32W<4>), st>>>(t, w, items + n16, q, tol, ir_max); break;
        case 8: k_basis32w<8><<<n32, 256, sizeof(Basis32W<8>), st>>>(t, w, items + n16, q, tol, ir_max); break;
        case 16: k_basis32w<16><<<n32, 512, sizeof(Basis32W<16>), st>>>(t, w, items + n16, q, tol, ir_max); break;
        default: return cudaErrorInvalidValue;
      }
      e = cudaGetLastError();
    } else {
      switch (nc32) {
        case 4: e = basis32<T, 4>(t, w, items + n16, n32, q, tol, ir_max, st); break;
        case 8: e = basis32<T, 8>(t, w, items + n16, n32, q, tol, ir_max, st); break;
        default: return cudaErrorInvalidValue;
      }
    }
  }
  return e;
}

template <typename K, typename S>
static cudaError_t smem_attr(K kern) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(sizeof(S)));
}

cudaError_t init_local_attributes() {
  cudaError_t e;
  if ((e = smem_attr<decltype(&k_basis<float, 4, true>), BasisSmem<float, 4>>(
               k_basis<float, 4, true>)) ||
      (e = smem_attr<decltype(&k_basis<float, 4, false>), BasisSmem<float, 4>>(
               k_basis<float, 4, false>)) ||
      (e = smem_attr<decltype(&k_basis<float, 8, true>), BasisSmem<float, 8>>(
               k_basis<float, 8, true>)) ||
      (e = smem_attr<decltype(&k_basis<float, 8, false>), BasisSmem<float, 8>>(
               k_basis<float, 8, false>)) ||
      (e = smem_attr<decltype(&k_basis<float, 12, true>), BasisSmem<float, 12>>(
               k_basis<float, 12, true>)) ||
      (e = smem_attr<decltype(&k_basis<float, 12, false>), BasisSmem<float, 12>>(
               k_basis<float, 12, false>)) ||
      (e = smem_attr<decltype(&k_basis<float, 16, true>), BasisSmem<float, 16>>(
               k_basis<float, 16, true>)) ||
      (e = smem_attr<decltype(&k_basis<float, 16, false>), BasisSmem<float, 16>>(
               k_basis<float, 16, false>)) ||
      (e = smem_attr<decltype(&k_basis<double, 4>), BasisSmem<double, 4>>(k_basis<double, 4>)) ||
      (e = smem_attr<decltype(&k_basis<double, 8>), BasisSmem<double, 8>>(k_basis<double, 8>)) ||
      (e = smem_attr<decltype(&k_basis<double, 12>), BasisSmem<double, 12>>(k_basis<double, 12>)) ||
      (e = smem_attr<decltype(&k_basis<double, 16>), BasisSmem<double, 16>>(k_basis<double, 16>)) ||
      (e = smem_attr<decltype(&k_basis32w<4>), Basis32W<4>>(k_basis32w<4>)) ||
      (e = smem_attr<decltype(&k_basis32w<8>), Basis32W<8>>(k_basis32w<8>)) ||
      (e = smem_attr<decltype(&k_basis32w<16>), Basis32W<16>>(k_basis32w<16>)) ||
      (e = smem_attr<decltype(&k_basis32<double, 4>), BasisSmem32<double, 4>>(k_basis32<double, 4>)) ||
      (e = smem_attr<decltype(&k_basis32<double, 8>), BasisSmem32<double, 8>>(k_basis32<double, 8>)))
    return e;
  if ((e = cudaFuncSetAttribute(k_factor_warp<float, 32>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(kFW * sizeof(FactorWarpSmem<float, 32>)))) !=
      cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_factor_warp<double, 32>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kFW * sizeof(FactorWarpSmem<double, 32>)));
}

cudaError_t launch_basis(const DeviceTables &t, const Workspace &w, int prec,
                         const BasisItem *items, int nitems16, int nitems32, int nc16, int nc32,
                         const double *q, double ir_tol, int ir_max, cudaStream_t st) {
  if (prec == MRCM_PREC_FP64)
    return launch_basis_t<double>(t, w, items, nitems16, nitems32, nc16, nc32, q, ir_tol, 0, st);
  return launch_basis_t<float>(t, w, items, nitems16, nitems32, nc16, nc32, q, ir_tol, ir_max,
                               st);
}


namespace {
__global__ void k_fp_convert_check(uint64_t start, uint64_t count, unsigned long long *bad) {
  for (uint64_t i = start + blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
       i < start + count; i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const float f = __uint_as_float(static_cast<unsigned>(i));
    const double a = static_cast<double>(f), b = f32_to_f64(f);
    if (!((f != f) ? (b != b) : (__double_as_longlong(a) == __double_as_longlong(b))))
      atomicAdd(&bad[0], 1ull);
    uint64_t h = i * 0x9E3779B97F4A7C15ull;
    h ^= h >> 31;
    const double dv[4] = {__longlong_as_double(static_cast<long long>(h)),
                          static_cast<double>(f) * (1.0 + ldexp(1.0, -24) * static_cast<double>((i >> 3) & 3)),
                          ldexp(static_cast<double>(f), -static_cast<int>(i & 127) - 40),
                          ldexp(static_cast<double>(f), static_cast<int>(i & 127))};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float x = static_cast<float>(dv[k]), y = f64_to_f32(dv[k]);
      if (!((dv[k] != dv[k]) ? (y != y) : (__float_as_uint(x) == __float_as_uint(y))))
        atomicAdd(&bad[1], 1ull);
    }
  }
}
}  // namespace

}  // namespace mrcm

extern "C" mrcm_status mrcm_test_fp_convert(uint64_t start, uint64_t count, uint64_t *d_mismatch,
                                            void *cuda_stream) {
  if (!d_mismatch || count > (1ull << 32)) return MRCM_EINVAL;
  if (count == 0) return MRCM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  mrcm::k_fp_convert_check<<<152 * 16, 256, 0, st>>>(
      start, count, reinterpret_cast<unsigned long long *>(d_mismatch));
  if (cudaGetLastError() != cudaSuccess) return MRCM_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MRCM_OK : MRCM_ECUDA;
}
