// Learned interface preconditioner (no counterpart in the paper): a small
// convolutional network that reads the permeability around each interface
// and proposes a correction Delta_g of the interface's block-Jacobi block,
// P_g = (M_gg)^{-1} (I + Delta_g), for the right-preconditioned interface
// GMRES of Eq. "mrc2".  Zero output is exactly block-Jacobi.
//
// Network (per interface): input 2 x 2s x 3s (log10(kappa)/3 and an inside
// mask, canonical orientation), three 3x3 stride-2 convolutions with 32
// channels, bias and ReLU, and a linear head from the flattened last
// feature map (32 x s/4 x 3s/8) to m*m.
// Storage: BF16 activations and BF16-rounded weights; every product is
// accumulated in FP32; FP32 master weights and Adam state.  Training
// target: theta (M_gg B_g - I) clipped entrywise to [-2, 2], B_g the (g, g)
// block of the inverse of the interface matrix restricted to g's
// neighbourhood (interfaces within one subdomain), theta = 1/2, computed
// here in FP64.
#include "mrcm_internal.h"
#include "iface_common.cuh"
#include "nbsolve.cuh"
#include "../../include/mrcm.h"
#include "../../include/mrcm_learned.h"

#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

namespace mrcm {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kCh = kLpChannels;

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// ---------------------------------------------------------------- inputs
__global__ void k_lp_window(DeviceTables t, const double *K, const double *lam, bf16 *x, int s,
                            int g0) {
  const int H = 2 * s, W = 3 * s, HW = H * W;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= HW) return;
  const int g = g0 + blockIdx.y;
  const IfaceInfo fi = t.iface[g];
  const SubInfo L = t.sub[fi.L];
  const int a = pix / W, c = pix % W;
  int xx, yy;
  if (fi.kind == 0) {
    yy = L.y0 - s / 2 + a;
    xx = L.x0 - s / 2 + c;
  } else {
    xx = L.x0 - s / 2 + a;
    yy = L.y0 - s / 2 + c;
  }
  const bool in = xx >= 0 && xx < t.nx && yy >= 0 && yy < t.ny;
  float v = 0.0f;
  if (in) {
    const int64_t cell = (static_cast<int64_t>(fi.r) * t.ny + yy) * t.nx + xx;
    v = static_cast<float>(log10(K[cell] * lam[cell]) / 3.0);
  }
  bf16 *xs = x + static_cast<int64_t>(blockIdx.y) * 2 * HW;
  xs[pix] = __float2bfloat16_rn(v);
  xs[HW + pix] = __float2bfloat16_rn(in ? 1.0f : 0.0f);
}

// ---------------------------------------------------------------- forward
// 3x3 convolution, stride 2, zero padding 1, bias, ReLU.  One thread per
// output position computes all 32 output channels; weights (BF16-rounded,
// FP32 in shared memory, [ci][tap][co]) are read as float4 broadcasts.
template <int CIN>
__global__ void __launch_bounds__(256) k_conv_fwd(const bf16 *in, const float *w, const float *b,
                                                  bf16 *out, int H, int W) {
  __shared__ __align__(16) float ws[CIN * 9 * kCh];
  for (int e = threadIdx.x; e < CIN * 9 * kCh; e += blockDim.x) {
    const int co = e % kCh, k = e / kCh;
    ws[e] = bfr(w[co * CIN * 9 + k]);
  }
  __syncthreads();
  const int Ho = H / 2, Wo = W / 2;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= Ho * Wo) return;
  const int i = pix / Wo, j = pix % Wo;
  const bf16 *x = in + static_cast<int64_t>(blockIdx.y) * CIN * H * W;
  float acc[kCh];
#pragma unroll
  for (int co = 0; co < kCh; ++co) acc[co] = b[co];
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int y = 2 * i + ky - 1;
      if (y < 0 || y >= H) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int xx = 2 * j + kx - 1;
        if (xx < 0 || xx >= W) continue;
        const float a = bf(x[(static_cast<int64_t>(ci) * H + y) * W + xx]);
        const float4 *wr = reinterpret_cast<const float4 *>(ws + (ci * 9 + ky * 3 + kx) * kCh);
#pragma unroll
        for (int q = 0; q < kCh / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q] = fmaf(wv.x, a, acc[4 * q]);
          acc[4 * q + 1] = fmaf(wv.y, a, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wv.z, a, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wv.w, a, acc[4 * q + 3]);
        }
      }
    }
  }
  bf16 *o = out + static_cast<int64_t>(blockIdx.y) * kCh * Ho * Wo;
#pragma unroll
  for (int co = 0; co < kCh; ++co)
    o[static_cast<int64_t>(co) * Ho * Wo + pix] = __float2bfloat16_rn(fmaxf(acc[co], 0.0f));
}

// linear head on the flattened last feature map (nf values per sample):
// one warp per (sample, output), lanes striding over the features
__global__ void k_head_fwd(const bf16 *a3, const float *wh, const float *bh, float *delta, int B,
                           int nf, int mm) {
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (wg >= B * mm) return;
  const int bidx = wg / mm, k = wg % mm;
  const bf16 *a = a3 + static_cast<int64_t>(bidx) * nf;
  const float *w = wh + static_cast<int64_t>(k) * nf;
  float v = 0.0f;
  for (int j = lane; j < nf; j += 32) v = fmaf(bfr(w[j]), bf(a[j]), v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) delta[bidx * mm + k] = v + bh[k];
}

// ---------------------------------------------------------------- backward
// loss = mean w_k (delta_k - target_k)^2 and dd = d loss / d delta
__global__ void k_head_loss(const float *delta, const float *target, const float *wk, float *dd,
                            float *loss, int B, int mm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const float inv_n = 1.0f / (static_cast<float>(B) * mm);
  float l2 = 0.0f;
  if (e < B * mm) {
    const int k = e % mm;
    const float diff = delta[e] - target[e];
    dd[e] = 2.0f * wk[k] * diff * inv_n;
    l2 = wk[k] * diff * diff * inv_n;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l2);
}

// head gradients: gwh[k][j] = sum_b dd[b][k] a3[b][j], gbh[k] = sum_b dd[b][k]
__global__ void k_head_wgrad(const bf16 *a3, const float *dd, float *gwh, float *gbh, int B,
                             int nf, int mm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < mm * nf) {
    const int k = e / nf, j = e % nf;
    float acc = 0.0f;
    for (int bidx = 0; bidx < B; ++bidx)
      acc = fmaf(dd[bidx * mm + k], bf(a3[static_cast<int64_t>(bidx) * nf + j]), acc);
    gwh[e] = acc;
  }
  if (e < mm) {
    float acc = 0.0f;
    for (int bidx = 0; bidx < B; ++bidx) acc += dd[bidx * mm + e];
    gbh[e] = acc;
  }
}

// dZ3[b][j] = sum_k dd[b][k] wh[k][j] where a3[b][j] > 0
__global__ void k_head_dgrad(const bf16 *a3, const float *wh, const float *dd, float *dz3, int B,
                             int nf, int mm) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= static_cast<int64_t>(B) * nf) return;
  const int bidx = static_cast<int>(e / nf), j = static_cast<int>(e % nf);
  float acc = 0.0f;
  for (int k = 0; k < mm; ++k)
    acc = fmaf(dd[bidx * mm + k], bfr(wh[static_cast<int64_t>(k) * nf + j]), acc);
  dz3[e] = bf(a3[e]) > 0.0f ? acc : 0.0f;
}

// weight and bias gradients of one convolution: thread (ci, tap, group of
// CG output channels); each CTA loops over samples and adds its partial
// sums once.  dZ is staged through shared memory in chunks of positions.
constexpr int kPch = 64;

template <int CIN, int CG>
__global__ void __launch_bounds__(CIN * 9 * (kCh / CG)) k_conv_wgrad(const bf16 *ain,
                                                                      const float *dz, float *gw,
                                                                      float *gb, int B, int H,
                                                                      int W) {
  constexpr int NG = kCh / CG;
  __shared__ float dzs[kCh][kPch];
  const int t = threadIdx.x;
  const int cog = t % NG, k = t / NG, ci = k / 9, tap = k % 9, ky = tap / 3, kx = tap % 3;
  const int Ho = H / 2, Wo = W / 2, np = Ho * Wo;
  float acc[CG], accb[CG];
#pragma unroll
  for (int q = 0; q < CG; ++q) acc[q] = accb[q] = 0.0f;
  for (int bidx = blockIdx.x; bidx < B; bidx += gridDim.x) {
    const float *d = dz + static_cast<int64_t>(bidx) * kCh * np;
    const bf16 *x = ain + (static_cast<int64_t>(bidx) * CIN + ci) * H * W;
    for (int p0 = 0; p0 < np; p0 += kPch) {
      const int cnt = np - p0 < kPch ? np - p0 : kPch;
      __syncthreads();
      for (int e = t; e < kCh * kPch; e += blockDim.x) {
        const int co = e / kPch, pp = e % kPch;
        dzs[co][pp] = pp < cnt ? d[static_cast<int64_t>(co) * np + p0 + pp] : 0.0f;
      }
      __syncthreads();
      for (int pp = 0; pp < cnt; ++pp) {
        const int pix = p0 + pp, i = pix / Wo, j = pix % Wo;
        const int y = 2 * i + ky - 1, xx = 2 * j + kx - 1;
        const float a = (y >= 0 && y < H && xx >= 0 && xx < W) ? bf(x[y * W + xx]) : 0.0f;
#pragma unroll
        for (int q = 0; q < CG; ++q) {
          const float dv = dzs[cog * CG + q][pp];
          acc[q] = fmaf(dv, a, acc[q]);
          accb[q] += dv;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < CG; ++q) {
    const int co = cog * CG + q;
    atomicAdd(&gw[(co * CIN + ci) * 9 + tap], acc[q]);
    if (k == 0) atomicAdd(&gb[co], accb[q]);
  }
}

// input gradient of one convolution (transposed convolution), times the
// ReLU mask of that input: thread per input position, all CIN channels
template <int CIN>
__global__ void __launch_bounds__(256) k_conv_dgrad(const float *dz, const float *w,
                                                    const bf16 *aprev, float *dzprev, int H,
                                                    int W) {
  __shared__ __align__(16) float ws[9 * kCh * CIN];     // [tap][co][ci]
  for (int e = threadIdx.x; e < 9 * kCh * CIN; e += blockDim.x) {
    const int ci = e % CIN, co = (e / CIN) % kCh, tap = e / (CIN * kCh);
    ws[e] = bfr(w[(co * CIN + ci) * 9 + tap]);
  }
  __syncthreads();
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= H * W) return;
  const int y = pix / W, xx = pix % W;
  const int Ho = H / 2, Wo = W / 2;
  const float *d = dz + static_cast<int64_t>(blockIdx.y) * kCh * Ho * Wo;
  float acc[CIN];
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
#pragma unroll
  for (int ky = 0; ky < 3; ++ky) {
    const int ty = y + 1 - ky;
    if (ty < 0 || (ty & 1)) continue;
    const int i = ty >> 1;
    if (i >= Ho) continue;
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const int tx = xx + 1 - kx;
      if (tx < 0 || (tx & 1)) continue;
      const int j = tx >> 1;
      if (j >= Wo) continue;
      for (int co = 0; co < kCh; ++co) {
        const float dv = d[(static_cast<int64_t>(co) * Ho + i) * Wo + j];
        const float4 *wr = reinterpret_cast<const float4 *>(ws + ((ky * 3 + kx) * kCh + co) * CIN);
#pragma unroll
        for (int q = 0; q < CIN / 4; ++q) {
          const float4 wv = wr[q];
          acc[4 * q] = fmaf(wv.x, dv, acc[4 * q]);
          acc[4 * q + 1] = fmaf(wv.y, dv, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wv.z, dv, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wv.w, dv, acc[4 * q + 3]);
        }
      }
    }
  }
  const bf16 *ap = aprev + static_cast<int64_t>(blockIdx.y) * CIN * H * W;
  float *o = dzprev + static_cast<int64_t>(blockIdx.y) * CIN * H * W;
#pragma unroll
  for (int ci = 0; ci < CIN; ++ci) {
    const int64_t e = static_cast<int64_t>(ci) * H * W + pix;
    o[e] = bf(ap[e]) > 0.0f ? acc[ci] : 0.0f;
  }
}

// Adam (Kingma and Ba 2015) on the FP32 master weights
__global__ void k_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------- blocks for the GMRES
// P_g = Pbj_g (I + Delta_g) for interfaces g0 .. g0 + count - 1
__global__ void k_lp_blocks(DeviceTables t, const double *Pbj, const float *delta, double *Puser,
                            int g0, int count, int m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count * m * m) return;
  const int gl = e / (m * m), i = (e / m) % m, k = e % m;
  const IfaceInfo fi = t.iface[g0 + gl];
  const double *Pb = Pbj + fi.tsc_off;
  const float *D = delta + static_cast<int64_t>(gl) * m * m;
  double acc = Pb[i * m + k];
  for (int l = 0; l < m; ++l) acc = fma(Pb[i * m + l], static_cast<double>(D[l * m + k]), acc);
  Puser[fi.tsc_off + i * m + k] = acc;
}

// ------------------------------------------------- training targets (FP64)
// One CTA per interface g: dense interface matrix of g's neighbourhood,
// Gaussian elimination with partial pivoting on [A | E_g] for the m columns
// of the (g, g) block of A^{-1}, then theta (M_gg B_g - I).
__global__ void __launch_bounds__(256) k_lp_targets(DeviceTables t, Workspace w, GmArgs a,
                                                    const int *nb_off, const int *nb_list,
                                                    int nloc_max, double theta, float *target,
                                                    int *bad_out) {
  extern __shared__ __align__(16) double lsm[];
  const int g = blockIdx.x;
  const IfaceInfo fg = t.iface[g];
  const int m = fg.nU + fg.nP;
  const int h0 = nb_off[g], nh = nb_off[g + 1] - h0;
  __shared__ int loc[kLpMaxNb + 1];     // local offset of each neighbourhood interface
  __shared__ int s_n, s_pos, s_piv, s_bad;
  // A: [n][n + m], then the [m][m] copy of the diagonal block; n is known
  // only inside the helper, so the copy goes to the end of the largest A
  double *A = lsm;
  double *Mgg = lsm + static_cast<size_t>(nloc_max) * (nloc_max + m);
  nb_inverse_columns(t, w, a.row, nb_list, h0, nh, g, A, Mgg, loc, &s_n, &s_pos, &s_piv, &s_bad);
  const int n = s_n, ld = n + m, pos_g = s_pos;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, k = e % m;
    double v = 0.0;
    if (!s_bad) {
      for (int l = 0; l < m; ++l) v += Mgg[i * m + l] * A[static_cast<size_t>(pos_g + l) * ld + n + k];
      v = theta * (v - (i == k ? 1.0 : 0.0));
      v = fmin(fmax(v, -kLpClip), kLpClip);
    }
    target[static_cast<int64_t>(g) * m * m + e] = static_cast<float>(v);
  }
  if (s_bad && threadIdx.x == 0) atomicOr(bad_out, MRCM_FLAG_IFACE_PIVOT);
}

}  // namespace

// ------------------------------------------------------------ host network
struct LpBuffers {
  int s, m, maxb, H, W;
  float *params, *grad, *am, *av;      // FP32 master weights, gradient, Adam state
  bf16 *x, *a1, *a2, *a3;              // activations
  float *dz1, *dz2, *dz3, *dd, *delta, *loss, *wk;
  int64_t nparam;
  int64_t off_w[3], off_b[3], off_wh, off_bh;
  int step;
  cudaStream_t stream;
};

}  // namespace mrcm

struct mrcm_lp {
  mrcm::LpBuffers b{};
  void *arena = nullptr;
  std::string err;
};

namespace mrcm {

static int64_t lp_in_count(const LpBuffers &b) { return 2LL * b.H * b.W; }

cudaError_t lp_forward(mrcm_lp *lp, const void *x, int B, float *delta) {
  LpBuffers &b = lp->b;
  const bf16 *X = static_cast<const bf16 *>(x);
  const int H = b.H, W = b.W;
  cudaStream_t st = b.stream;
  const float *P = b.params;
  k_conv_fwd<2><<<dim3((H / 2 * W / 2 + 255) / 256, B), 256, 0, st>>>(X, P + b.off_w[0],
                                                                      P + b.off_b[0], b.a1, H, W);
  k_conv_fwd<kCh><<<dim3((H / 4 * W / 4 + 255) / 256, B), 256, 0, st>>>(
      b.a1, P + b.off_w[1], P + b.off_b[1], b.a2, H / 2, W / 2);
  k_conv_fwd<kCh><<<dim3((H / 8 * W / 8 + 255) / 256, B), 256, 0, st>>>(
      b.a2, P + b.off_w[2], P + b.off_b[2], b.a3, H / 4, W / 4);
  const int mm = b.m * b.m, nf = kCh * (H / 8) * (W / 8);
  k_head_fwd<<<(B * mm + 7) / 8, 256, 0, st>>>(b.a3, P + b.off_wh, P + b.off_bh, delta, B, nf, mm);
  return cudaGetLastError();
}

cudaError_t lp_backward(mrcm_lp *lp, const void *x, const float *target, int B) {
  LpBuffers &b = lp->b;
  const bf16 *X = static_cast<const bf16 *>(x);
  const int H = b.H, W = b.W;
  cudaStream_t st = b.stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(b.grad, 0, sizeof(float) * b.nparam, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b.loss, 0, sizeof(float), st)) != cudaSuccess) return e;
  const float *P = b.params;
  float *G = b.grad;
  const int mm = b.m * b.m, nf = kCh * (H / 8) * (W / 8);
  k_head_loss<<<(B * mm + 255) / 256, 256, 0, st>>>(b.delta, target, b.wk, b.dd, b.loss, B, mm);
  k_head_wgrad<<<(mm * nf + 255) / 256, 256, 0, st>>>(b.a3, b.dd, G + b.off_wh, G + b.off_bh,
                                                      B, nf, mm);
  k_head_dgrad<<<static_cast<int>((static_cast<int64_t>(B) * nf + 255) / 256), 256, 0, st>>>(
      b.a3, P + b.off_wh, b.dd, b.dz3, B, nf, mm);
  const int gridw = B < 304 ? B : 304;
  k_conv_wgrad<kCh, kCh><<<gridw, kCh * 9, 0, st>>>(b.a2, b.dz3, G + b.off_w[2], G + b.off_b[2],
                                                    B, H / 4, W / 4);
  k_conv_dgrad<kCh><<<dim3((H / 4 * W / 4 + 255) / 256, B), 256, 0, st>>>(
      b.dz3, P + b.off_w[2], b.a2, b.dz2, H / 4, W / 4);
  k_conv_wgrad<kCh, kCh><<<gridw, kCh * 9, 0, st>>>(b.a1, b.dz2, G + b.off_w[1], G + b.off_b[1],
                                                    B, H / 2, W / 2);
  k_conv_dgrad<kCh><<<dim3((H / 2 * W / 2 + 255) / 256, B), 256, 0, st>>>(
      b.dz2, P + b.off_w[1], b.a1, b.dz1, H / 2, W / 2);
  k_conv_wgrad<2, 4><<<gridw, 2 * 9 * (kCh / 4), 0, st>>>(X, b.dz1, G + b.off_w[0],
                                                          G + b.off_b[0], B, H, W);
  return cudaGetLastError();
}

cudaError_t lp_windows(const DeviceTables &t, const double *K, const double *lam, void *x, int s,
                       int g0, int count, cudaStream_t st) {
  const int HW = 6 * s * s;
  if (count <= 0) return cudaSuccess;
  k_lp_window<<<dim3((HW + 255) / 256, count), 256, 0, st>>>(t, K, lam, static_cast<bf16 *>(x), s,
                                                             g0);
  return cudaGetLastError();
}

cudaError_t lp_blocks(const DeviceTables &t, const double *Pbj, const float *delta, double *Puser,
                      int g0, int count, int m, cudaStream_t st) {
  const int n = count * m * m;
  if (n <= 0) return cudaSuccess;
  k_lp_blocks<<<(n + 255) / 256, 256, 0, st>>>(t, Pbj, delta, Puser, g0, count, m);
  return cudaGetLastError();
}

size_t lp_targets_smem(int nloc, int m) {
  return sizeof(double) * (static_cast<size_t>(nloc) * (nloc + m) + static_cast<size_t>(m) * m);
}

cudaError_t lp_targets(const DeviceTables &t, const Workspace &w, const GmArgs &a,
                       const int *nb_off, const int *nb_list, int nloc_max, int m, double theta,
                       float *target, int *bad, cudaStream_t st) {
  const size_t smem = lp_targets_smem(nloc_max, m);
  cudaError_t e = cudaFuncSetAttribute(k_lp_targets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if (t.niface == 0) return cudaSuccess;
  k_lp_targets<<<t.niface, 256, smem, st>>>(t, w, a, nb_off, nb_list, nloc_max, theta, target,
                                            bad);
  return cudaGetLastError();
}

int lp_s(const mrcm_lp *lp) { return lp->b.s; }
int lp_m(const mrcm_lp *lp) { return lp->b.m; }
int lp_maxb(const mrcm_lp *lp) { return lp->b.maxb; }
void *lp_xbuf(mrcm_lp *lp) { return lp->b.x; }
float *lp_deltabuf(mrcm_lp *lp) { return lp->b.delta; }
cudaStream_t lp_stream(const mrcm_lp *lp) { return lp->b.stream; }

}  // namespace mrcm

using namespace mrcm;

static thread_local std::string g_lp_err;

static mrcm_status lp_fail(mrcm_lp *lp, mrcm_status s, const char *msg) {
  if (lp) lp->err = msg;
  else g_lp_err = msg;
  return s;
}

extern "C" {

mrcm_status mrcm_lp_create(int32_t s, int32_t m, int32_t max_batch, uint64_t seed,
                           void *cuda_stream, mrcm_lp **out) {
  if (!out) return lp_fail(nullptr, MRCM_EINVAL, "out is NULL");
  *out = nullptr;
  if (s != 16 && s != 32) return lp_fail(nullptr, MRCM_EINVAL, "s must be 16 or 32");
  if (m < 1 || m > kLpMaxM) return lp_fail(nullptr, MRCM_EINVAL, "m out of range");
  if (max_batch < 1 || max_batch > (1 << 20)) return lp_fail(nullptr, MRCM_EINVAL, "max_batch out of range");
  mrcm_lp *lp = new mrcm_lp();
  LpBuffers &b = lp->b;
  b.s = s;
  b.m = m;
  b.maxb = max_batch;
  b.H = 2 * s;
  b.W = 3 * s;
  b.stream = static_cast<cudaStream_t>(cuda_stream);
  // parameter layout: w1 b1 w2 b2 w3 b3 wh bh
  int64_t o = 0;
  const int cin[3] = {2, kCh, kCh};
  for (int l = 0; l < 3; ++l) {
    b.off_w[l] = o;
    o += static_cast<int64_t>(kCh) * cin[l] * 9;
    b.off_b[l] = o;
    o += kCh;
  }
  b.off_wh = o;
  o += static_cast<int64_t>(m) * m * kCh * (b.H / 8) * (b.W / 8);
  b.off_bh = o;
  o += static_cast<int64_t>(m) * m;
  b.nparam = o;
  const int64_t B = max_batch, HW = static_cast<int64_t>(b.H) * b.W;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t r = (off + 255) & ~size_t(255);
    off = r + bytes;
    return r;
  };
  const size_t o_p = take(4 * o), o_g = take(4 * o), o_m = take(4 * o), o_v = take(4 * o),
               o_x = take(2 * B * 2 * HW), o_a1 = take(2 * B * kCh * HW / 4),
               o_a2 = take(2 * B * kCh * HW / 16), o_a3 = take(2 * B * kCh * HW / 64),
               o_d1 = take(4 * B * kCh * HW / 4), o_d2 = take(4 * B * kCh * HW / 16),
               o_d3 = take(4 * B * kCh * HW / 64), o_f = take(4 * B * m * m),
               o_de = take(4 * B * m * m), o_l = take(4), o_wk = take(4 * m * m);
  if (cudaMalloc(&lp->arena, off) != cudaSuccess) {
    delete lp;
    return lp_fail(nullptr, MRCM_ENOMEM, "cudaMalloc failed for the network");
  }
  char *base = static_cast<char *>(lp->arena);
  b.params = reinterpret_cast<float *>(base + o_p);
  b.grad = reinterpret_cast<float *>(base + o_g);
  b.am = reinterpret_cast<float *>(base + o_m);
  b.av = reinterpret_cast<float *>(base + o_v);
  b.x = reinterpret_cast<bf16 *>(base + o_x);
  b.a1 = reinterpret_cast<bf16 *>(base + o_a1);
  b.a2 = reinterpret_cast<bf16 *>(base + o_a2);
  b.a3 = reinterpret_cast<bf16 *>(base + o_a3);
  b.dz1 = reinterpret_cast<float *>(base + o_d1);
  b.dz2 = reinterpret_cast<float *>(base + o_d2);
  b.dz3 = reinterpret_cast<float *>(base + o_d3);
  b.dd = reinterpret_cast<float *>(base + o_f);
  b.delta = reinterpret_cast<float *>(base + o_de);
  b.loss = reinterpret_cast<float *>(base + o_l);
  b.wk = reinterpret_cast<float *>(base + o_wk);
  // He-normal convolution weights from a seeded generator (Box-Muller on a
  // 64-bit LCG, host side), zero biases and head: the initial network
  // proposes Delta = 0, i.e. block-Jacobi
  std::vector<float> h(o, 0.0f);
  uint64_t st = seed * 6364136223846793005ULL + 1442695040888963407ULL;
  auto unif = [&]() {
    st = st * 6364136223846793005ULL + 1442695040888963407ULL;
    return (static_cast<double>(st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < 3; ++l) {
    const double sd = std::sqrt(2.0 / (cin[l] * 9));
    for (int64_t k = 0; k < static_cast<int64_t>(kCh) * cin[l] * 9; ++k) {
      const double u1 = unif(), u2 = unif();
      h[b.off_w[l] + k] = static_cast<float>(sd * std::sqrt(-2.0 * std::log(u1)) *
                                             std::cos(6.283185307179586 * u2));
    }
  }
  const std::vector<float> ones(static_cast<size_t>(m) * m, 1.0f);
  if (cudaMemcpy(b.params, h.data(), 4 * o, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b.wk, ones.data(), 4 * ones.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b.am, 0, 4 * o) != cudaSuccess || cudaMemset(b.av, 0, 4 * o) != cudaSuccess) {
    cudaFree(lp->arena);
    delete lp;
    return lp_fail(nullptr, MRCM_ECUDA, "network upload failed");
  }
  b.step = 0;
  *out = lp;
  return MRCM_OK;
}

void mrcm_lp_destroy(mrcm_lp *lp) {
  if (!lp) return;
  if (lp->arena) cudaFree(lp->arena);
  delete lp;
}

const char *mrcm_lp_last_error(const mrcm_lp *lp) { return lp ? lp->err.c_str() : g_lp_err.c_str(); }

int64_t mrcm_lp_num_params(const mrcm_lp *lp) { return lp ? lp->b.nparam : 0; }

int64_t mrcm_lp_input_size(const mrcm_lp *lp) { return lp ? lp_in_count(lp->b) : 0; }

mrcm_status mrcm_lp_set_stream(mrcm_lp *lp, void *cuda_stream) {
  if (!lp) return MRCM_EINVAL;
  lp->b.stream = static_cast<cudaStream_t>(cuda_stream);
  return MRCM_OK;
}

mrcm_status mrcm_lp_set_params(mrcm_lp *lp, const float *d_params) {
  if (!lp || !d_params) return lp_fail(lp, MRCM_EINVAL, "NULL argument");
  if (cudaMemcpyAsync(lp->b.params, d_params, 4 * lp->b.nparam, cudaMemcpyDeviceToDevice,
                      lp->b.stream) != cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "copy failed");
  return MRCM_OK;
}

mrcm_status mrcm_lp_set_loss_weights(mrcm_lp *lp, const float *d_weights) {
  if (!lp || !d_weights) return lp_fail(lp, MRCM_EINVAL, "NULL argument");
  if (cudaMemcpyAsync(lp->b.wk, d_weights, 4 * lp->b.m * lp->b.m, cudaMemcpyDeviceToDevice,
                      lp->b.stream) != cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "copy failed");
  return MRCM_OK;
}

mrcm_status mrcm_lp_get_params(mrcm_lp *lp, float *d_params) {
  if (!lp || !d_params) return lp_fail(lp, MRCM_EINVAL, "NULL argument");
  if (cudaMemcpyAsync(d_params, lp->b.params, 4 * lp->b.nparam, cudaMemcpyDeviceToDevice,
                      lp->b.stream) != cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "copy failed");
  return MRCM_OK;
}

mrcm_status mrcm_lp_forward(mrcm_lp *lp, const void *d_x, int32_t B, float *d_delta) {
  if (!lp || !d_x || !d_delta) return lp_fail(lp, MRCM_EINVAL, "NULL argument");
  if (B < 1 || B > lp->b.maxb) return lp_fail(lp, MRCM_EINVAL, "batch outside 1..max_batch");
  if (lp_forward(lp, d_x, B, d_delta) != cudaSuccess) return lp_fail(lp, MRCM_ECUDA, "launch failed");
  return MRCM_OK;
}

mrcm_status mrcm_lp_gradient(mrcm_lp *lp, const void *d_x, const float *d_target, int32_t B,
                             float *d_grad, float *d_loss) {
  if (!lp || !d_x || !d_target) return lp_fail(lp, MRCM_EINVAL, "NULL argument");
  if (B < 1 || B > lp->b.maxb) return lp_fail(lp, MRCM_EINVAL, "batch outside 1..max_batch");
  LpBuffers &b = lp->b;
  if (lp_forward(lp, d_x, B, b.delta) != cudaSuccess ||
      lp_backward(lp, d_x, d_target, B) != cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "launch failed");
  if (d_grad && cudaMemcpyAsync(d_grad, b.grad, 4 * b.nparam, cudaMemcpyDeviceToDevice,
                                b.stream) != cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "copy failed");
  if (d_loss && cudaMemcpyAsync(d_loss, b.loss, 4, cudaMemcpyDeviceToDevice, b.stream) !=
                    cudaSuccess)
    return lp_fail(lp, MRCM_ECUDA, "copy failed");
  return MRCM_OK;
}

mrcm_status mrcm_lp_train_step(mrcm_lp *lp, const void *d_x, const float *d_target, int32_t B,
                               float lr, float *d_loss) {
  mrcm_status s = mrcm_lp_gradient(lp, d_x, d_target, B, nullptr, d_loss);
  if (s != MRCM_OK) return s;
  LpBuffers &b = lp->b;
  ++b.step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, static_cast<float>(b.step));
  const float c2 = 1.0f - std::pow(b2, static_cast<float>(b.step));
  const int n = static_cast<int>(b.nparam);
  k_adam<<<(n + 255) / 256, 256, 0, b.stream>>>(b.params, b.grad, b.am, b.av, n, lr, b1, b2,
                                                 1e-8f, c1, c2);
  if (cudaGetLastError() != cudaSuccess) return lp_fail(lp, MRCM_ECUDA, "launch failed");
  return MRCM_OK;
}

}  // extern "C"
