// Step (e) of the MRCM solve: fine-scale pressure as the linear combination
// of the multiscale basis with the interface coefficients (text after
// Eq. "beta"), and face normal velocities from it: two-point fluxes inside a
// subdomain, the Robin flux T_R (p_c - g)/h on each side of an interface
// face (g = -beta sigma U_H + P_H, Eq. "mrc1"), reported as the mean of the
// two one-sided values, and the boundary data or Dirichlet flux on physical
// faces.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"

#include <cstdint>
#include <cuda_runtime.h>

namespace mrcm {
namespace {

// Pressure and face velocities of cell k of a subdomain of size S (pc its
// pressure; p holds the subdomain's pressures in shared memory).
template <int S>
__device__ __forceinline__ void recon_cell(const DeviceTables &t, const Workspace &w,
                                           const SubInfo &sb, double *P, double *UX, double *UY,
                                           double *GAM, const double *p, int k, double pc) {
  constexpr int N = S * S;
  const int a = k % S, b = k / S;
  const double *coef = w.coef + sb.coef_off;
  const double tW = coef[k], tE = coef[N + k], tS = coef[2 * N + k], tN = coef[3 * N + k];
  const double inv_h = t.inv_h;   // a product, not an FP64 division (slow here)
  const int gi = sb.x0 + a, gj = sb.y0 + b;
  const int nx = t.nx, ny = t.ny;
  const int64_t cell = (static_cast<int64_t>(sb.r) * ny + gj) * nx + gi;
  P[cell] = pc;
  double *ux = UX + static_cast<int64_t>(sb.r) * ny * (nx + 1);
  double *uy = UY + static_cast<int64_t>(sb.r) * (ny + 1) * nx;
  if (a < S - 1) ux[static_cast<int64_t>(gj) * (nx + 1) + gi + 1] = tE * (pc - p[k + 1]) * inv_h;
  if (b < S - 1) {
    double v = tN * (pc - p[k + S]) * inv_h;
    if (t.grav) {     // gravity flux of the face (the half-cell elimination)
      const double *wr = t.grav + static_cast<int64_t>(sb.r) * ny * nx;
      const double k0 = coef[5 * N + k], k1 = coef[5 * N + k + S];
      const double w0 = wr[static_cast<int64_t>(gj) * nx + gi], w1 = wr[static_cast<int64_t>(gj + 1) * nx + gi];
      v += (k0 * w1 + k1 * w0) / (k0 + k1);
    }
    uy[static_cast<int64_t>(gj + 1) * nx + gi] = v;
  }
  const bool onface[4] = {a == 0, a == S - 1, b == 0, b == S - 1};
  const double Tf[4] = {tW, tE, tS, tN};
#pragma unroll
  for (int side = 0; side < 4; ++side) {
    if (!onface[side]) continue;
    const int e = side < 2 ? b : a;
    const double sgn = (side == kEdgeE || side == kEdgeN) ? 1.0 : -1.0;  // outward along +x/+y
    double un;  // outward normal velocity
    if (sb.edge_iface[side] >= 0) {
      const FaceIface fe = face_iface(sb, side, e);
      const IfaceInfo fi = t.iface[fe.g];
      const double beta = coef[6 * N + side * S + e];
      double UH = 0.0, PH = 0.0;
      for (int q = 0; q < fi.nU; ++q) UH += w.x[fi.unk + q] * iface_fn_at(t, fe.len, fi.fnU + q, fe.e);
      for (int q = 0; q < fi.nP; ++q)
        PH += w.x[fi.unk + fi.nU + q] * iface_fn_at(t, fe.len, fi.fnP + q, fe.e);
      const double gval = -beta * sgn * UH + PH;
      un = Tf[side] * (pc - gval) * inv_h;
      if (t.grav && side >= kEdgeS)
        un += sgn * t.grav[(static_cast<int64_t>(sb.r) * ny + gj) * nx + gi] * Tf[side] /
              (2.0 * coef[5 * N + k]);
      GAM[fi.gam_off + (sgn > 0 ? 0 : fe.len) + fe.e] = un;
      continue;
    }
    int kb;
    if (side == kEdgeW) kb = gj;
    else if (side == kEdgeE) kb = ny + gj;
    else if (side == kEdgeS) kb = 2 * ny + gi;
    else kb = 2 * ny + nx + gi;
    un = t.bc_type[kb] == 1 ? Tf[side] * (pc - t.bc_val[kb]) * inv_h : t.bc_val[kb];
    if (t.grav && t.bc_type[kb] == 1 && side >= kEdgeS)
      un += sgn * t.grav[(static_cast<int64_t>(sb.r) * ny + gj) * nx + gi];
    if (side == kEdgeW) ux[static_cast<int64_t>(gj) * (nx + 1)] = -un;
    else if (side == kEdgeE) ux[static_cast<int64_t>(gj) * (nx + 1) + nx] = un;
    else if (side == kEdgeS) uy[gi] = -un;
    else uy[static_cast<int64_t>(ny) * nx + gi] = un;
  }
}

// One CTA of kReconThreads threads per subdomain of size S (ids from first
// on); thread tid owns cells tid + i kReconThreads (i < CPT).
constexpr int kReconThreads = 256;

template <int S>
__global__ void __launch_bounds__(kReconThreads, 3) k_recon_cells(DeviceTables t, Workspace w,
                                                                  double *P, double *UX,
                                                                  double *UY, double *GAM,
                                                                  int first) {
  constexpr int N = S * S, NT = kReconThreads, CPT = N / NT;
  static_assert(CPT * NT == N, "whole cells per thread");
  const int g = t.sub_by_size[first + blockIdx.x];
  const SubInfo sb = t.sub[g];
  const int tid = threadIdx.x;
  __shared__ double p[N];
  __shared__ double coefc[1 + 8 * S];
  __shared__ double red[N / 32];
  for (int c = tid; c < sb.ncols; c += NT) {
    const int u = t.col[sb.col_off + c].unk;
    coefc[c] = u < 0 ? 1.0 : w.x[u];
  }
  __syncthreads();
  // p = sum_c x_c basis_c: per cell four independent sums over the columns,
  // the thread's cells interleaved, so that 4 CPT basis loads are in flight
  // at once (every cell sums in the same order whatever CPT is)
  const double *bas = w.basis + sb.basis_off;
  double p0[CPT], p1[CPT], p2[CPT], p3[CPT];
#pragma unroll
  for (int i = 0; i < CPT; ++i) p0[i] = p1[i] = p2[i] = p3[i] = 0.0;
  int c = 0;
  for (; c + 3 < sb.ncols; c += 4) {
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
      const int k = tid + i * NT;
      p0[i] += coefc[c] * bas[static_cast<int64_t>(c) * N + k];
      p1[i] += coefc[c + 1] * bas[static_cast<int64_t>(c + 1) * N + k];
      p2[i] += coefc[c + 2] * bas[static_cast<int64_t>(c + 2) * N + k];
      p3[i] += coefc[c + 3] * bas[static_cast<int64_t>(c + 3) * N + k];
    }
  }
  for (; c < sb.ncols; ++c)
#pragma unroll
    for (int i = 0; i < CPT; ++i) p0[i] += coefc[c] * bas[static_cast<int64_t>(c) * N + tid + i * NT];
  double pc[CPT];
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    pc[i] = (p0[i] + p1[i]) + (p2[i] + p3[i]);
    p[tid + i * NT] = pc[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < CPT; ++i) recon_cell<S>(t, w, sb, P, UX, UY, GAM, p, tid + i * NT, pc[i]);
  // per-subdomain pressure sum (deterministic order) for the mean shift:
  // each warp sums 32 consecutive cells, the partials are added in cell order
#pragma unroll
  for (int i = 0; i < CPT; ++i) {
    double s = pc[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[(tid + i * NT) >> 5] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int k = 0; k < N / 32; ++k) acc += red[k];
    w.psum[g] = acc;
  }
}

__global__ void k_recon_mean(DeviceTables t, Workspace w, double *pmean) {
  const RealInfo ri = t.real[blockIdx.x];
  __shared__ double red[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < ri.nsub; k += blockDim.x) s += w.psum[ri.sub0 + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) acc += red[k];
    pmean[blockIdx.x] = acc / (static_cast<double>(t.nx) * t.ny);
  }
}

// interface faces: mean of the one-sided velocities (n_check-oriented);
// pure Neumann: shift p to zero cell mean.
__global__ void k_recon_final(DeviceTables t, Workspace w, double *P, double *UX, double *UY,
                              const double *GAM, const double *pmean, int64_t ncells,
                              int64_t nfaces) {
  const int SM = t.smax;   // faces enumerated as (interface, e < smax)
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < nfaces;
       k += stride) {
    const int gi = static_cast<int>(k / SM), e = static_cast<int>(k % SM);
    const IfaceInfo fi = t.iface[gi];
    const int S = fi.s;
    if (e >= S) continue;
    const double v = 0.5 * (GAM[fi.gam_off + e] - GAM[fi.gam_off + S + e]);
    if (fi.kind == 0) {
      const int i = fi.fx, j = fi.fy + e;
      UX[(static_cast<int64_t>(fi.r) * t.ny + j) * (t.nx + 1) + i] = v;
    } else {
      const int i = fi.fx + e, j = fi.fy;
      UY[(static_cast<int64_t>(fi.r) * (t.ny + 1) + j) * t.nx + i] = v;
    }
  }
  if (t.pure_neumann) {
    const int64_t per = static_cast<int64_t>(t.nx) * t.ny;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < ncells;
         k += stride)
      P[k] -= pmean[k / per];
  }
}

}  // namespace

cudaError_t launch_reconstruct(const DeviceTables &t, const Workspace &w, double *p, double *ux,
                               double *uy, double *gam, cudaStream_t st) {
  double *G = gam ? gam : w.gamma_tmp;
  if (t.nsub16 > 0)
    k_recon_cells<16><<<t.nsub16, kReconThreads, 0, st>>>(t, w, p, ux, uy, G, 0);
  if (t.nsub > t.nsub16)
    k_recon_cells<32><<<t.nsub - t.nsub16, kReconThreads, 0, st>>>(t, w, p, ux, uy, G, t.nsub16);
  double *pmean = w.dstat + 2 + t.n_real;
  if (t.pure_neumann) k_recon_mean<<<t.n_real, 256, 0, st>>>(t, w, pmean);
  const int64_t ncells = static_cast<int64_t>(t.n_real) * t.nx * t.ny;
  const int64_t nfaces = static_cast<int64_t>(t.niface) * t.smax;
  const int64_t work = nfaces > ncells ? nfaces : ncells;
  int blocks = static_cast<int>((work + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_recon_final<<<blocks, 256, 0, st>>>(t, w, p, ux, uy, G, pmean, ncells, nfaces);
  return cudaGetLastError();
}

}  // namespace mrcm
