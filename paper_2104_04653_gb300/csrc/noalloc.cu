// mrcm_local_solve_noalloc: the local subdomain solve without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// owned by another runtime (a framework allocator that must see every byte),
// or a process that has to keep its device footprint fixed after start-up.
// This entry point gives them the local solve (assembly, FP32 block
// factorisation, FP64 refinement) with its only scratch memory, the inverse
// Schur blocks of the factorisation, in a file-scope __device__ array of fixed
// size.  Every GPU that loads the library holds that array (kNoAllocMaxSub
// subdomains x 16 KB = 1 MiB) until the process exits.
//
// It is a variant of the factor kernel of local.cu: the same block LDL^T with
// explicit Gauss-Jordan inverses of the 16 x 16 Schur blocks, here written to
// the static array, followed in the same kernel by the refined solve.
#include "../../include/mrcm.h"
#include "mrcm_internal.h"

#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

namespace {

constexpr int kS = 16, kN = kS * kS;
constexpr int kNoAllocMaxSub = 64;
constexpr int kMaxDevices = 64;

// The scratch: inverse Schur blocks W_j (FP32), per subdomain kS x kN.
// Host code must not pass the symbol itself to a kernel (it is a host-side
// stand-in, not a device address); it takes the address from
// cudaGetSymbolAddress once per device.
static __device__ __align__(256) float g_noalloc_W[kNoAllocMaxSub * kS * kN];

// Per device: the array's device address and the context it was looked up
// in.  A device reset (cudaDeviceReset) destroys the primary context and the
// module with it; the next context may place the array elsewhere, so the
// address is looked up again whenever the current context differs.
float *g_sym[kMaxDevices] = {};
CUcontext g_sym_ctx[kMaxDevices] = {};
std::mutex g_sym_mu;

// The current driver context, through the runtime's driver entry point (the
// library does not link the driver library); null if unavailable.
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 get = nullptr;
  if (!get) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return nullptr;
    get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  }
  CUcontext ctx = nullptr;
  return get(&ctx) == CUDA_SUCCESS ? ctx : nullptr;
}

__device__ __forceinline__ float shflf(float v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// One CTA (256 threads) per subdomain.
//   kappa [nsub][16][16]   cell kappa = lambda K (x fastest)
//   tface [nsub][4][16]    transmissibility of the W, E, S, N boundary faces
//                          (along +y for W/E, +x for S/N)
//   rhs, x [nsub][256]     FP64 right-hand side and solution
__global__ void __launch_bounds__(kN) k_local_noalloc(const double *kappa, const double *tface,
                                                      const double *rhs, double *x, float *Wscr,
                                                      double tol, int ir_max) {
  const int g = blockIdx.x, tid = threadIdx.x, a = tid % kS, b = tid / kS;
  __shared__ double kap[kN], ds[kN], bb[kN], xs[kN];
  __shared__ float offx[kN], ecp[kN], Ws[kS * kN], z[kN], v[kN];
  __shared__ float red[kN / 32];
  __shared__ float s_r2, s_b2;
  kap[tid] = kappa[static_cast<int64_t>(g) * kN + tid];
  __syncthreads();
  const double kc = kap[tid];
  double T4[4];
  const int na[4] = {a - 1, a + 1, a, a}, nb[4] = {b, b, b - 1, b + 1};
#pragma unroll
  for (int side = 0; side < 4; ++side) {
    if (na[side] >= 0 && na[side] < kS && nb[side] >= 0 && nb[side] < kS) {
      const double kn = kap[nb[side] * kS + na[side]];
      T4[side] = 2.0 * kc * kn / (kc + kn);
    } else {
      const int e = side < 2 ? b : a;
      T4[side] = tface[(static_cast<int64_t>(g) * 4 + side) * kS + e];
    }
  }
  const double diag = T4[0] + T4[1] + T4[2] + T4[3];
  ds[tid] = 1.0 / sqrt(diag);
  __syncthreads();
  offx[tid] = static_cast<float>(a < kS - 1 ? -T4[1] * ds[tid] * ds[tid + 1] : 0.0);
  ecp[tid] = static_cast<float>(b < kS - 1 ? -T4[3] * ds[tid] * ds[tid + kS] : 0.0);
  __syncthreads();
  float *W = Wscr + static_cast<int64_t>(g) * kS * kN;
  if (tid < 32) {
    // block LDL^T of the scaled operator, Schur blocks inverted in registers
    const int c = tid & 15, h = tid >> 4;
    float R[8];
    for (int j = 0; j < kS; ++j) {
      const float ec = j > 0 ? ecp[(j - 1) * kS + c] : 0.0f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int r = 8 * h + q;
        float val = 0.0f;
        if (r == c) val = 1.0f;
        else if (r - c == 1) val = offx[j * kS + c];
        else if (c - r == 1) val = offx[j * kS + r];
        if (j > 0) val -= ecp[(j - 1) * kS + r] * ec * R[q];
        R[q] = val;
      }
#pragma unroll
      for (int p = 0; p < kS; ++p) {
        const int src = (p >> 3) << 4;
        const float rowv = shflf(R[p & 7], src + c);
        const float piv = shflf(R[p & 7], src + p);
        float colv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) colv[q] = shflf(R[q], (h << 4) + p);
        const float ip = __fdividef(1.0f, piv);
        const float rv = rowv * ip;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int r = 8 * h + q;
          float nv = R[q] - colv[q] * rv;
          nv = (c == p) ? -colv[q] * ip : nv;
          nv = (r == p) ? ((c == p) ? ip : rv) : nv;
          R[q] = nv;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) W[j * kN + (8 * h + q) * kS + c] = R[q];
    }
  }
  __syncthreads();                       // W (global scratch) complete for this CTA
  for (int k = tid; k < kS * kN; k += kN) Ws[k] = W[k];
  const double bl = rhs[static_cast<int64_t>(g) * kN + tid];
  bb[tid] = bl;
  xs[tid] = 0.0;
  const float dsf = static_cast<float>(ds[tid]);
  const float zb = static_cast<float>(bl) * dsf;
  z[tid] = zb;
  {
    float s = zb * zb;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
  }
  __syncthreads();
  if (tid == 0) {
    float s = 0.0f;
    for (int k = 0; k < kN / 32; ++k) s += red[k];
    s_b2 = s;
  }
  const float tol2 = static_cast<float>(tol) * static_cast<float>(tol);
  for (int sweep = 0;; ++sweep) {
    __syncthreads();
    // forward: v_j = W_j (z_j - e_{j-1} v_{j-1}), 16 threads per block row
    for (int j = 0; j < kS; ++j) {
      if (tid < kS) {
        float acc = 0.0f;
        for (int q = 0; q < kS; ++q) {
          const float in = j == 0 ? z[q] : z[j * kS + q] - ecp[(j - 1) * kS + q] * v[(j - 1) * kS + q];
          acc += Ws[j * kN + q * kS + tid] * in;
        }
        v[j * kS + tid] = acc;
      }
      __syncthreads();
    }
    // backward: y_j = v_j - W_j (e_j y_{j+1})
    for (int j = kS - 2; j >= 0; --j) {
      if (tid < kS) {
        float acc = 0.0f;
        for (int q = 0; q < kS; ++q) acc += Ws[j * kN + q * kS + tid] * (ecp[j * kS + q] * v[(j + 1) * kS + q]);
        v[j * kS + tid] -= acc;
      }
      __syncthreads();
    }
    xs[tid] += static_cast<double>(dsf * v[tid]);
    __syncthreads();
    if (sweep >= ir_max) break;
    double r = fma(-diag, xs[tid], bb[tid]);
    if (a > 0) r = fma(T4[0], xs[tid - 1], r);
    if (a < kS - 1) r = fma(T4[1], xs[tid + 1], r);
    if (b > 0) r = fma(T4[2], xs[tid - kS], r);
    if (b < kS - 1) r = fma(T4[3], xs[tid + kS], r);
    const float zr = static_cast<float>(r) * dsf;
    z[tid] = zr;
    float s = zr * zr;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((tid & 31) == 0) red[tid >> 5] = s;
    __syncthreads();
    if (tid == 0) {
      float acc = 0.0f;
      for (int k = 0; k < kN / 32; ++k) acc += red[k];
      s_r2 = acc;
    }
    __syncthreads();
    if (!(s_r2 > tol2 * s_b2)) break;    // converged (or NaN: stop)
  }
  x[static_cast<int64_t>(g) * kN + tid] = xs[tid];
}

}  // namespace

extern "C" mrcm_status mrcm_local_solve_noalloc(int32_t nsub, const double *d_kappa,
                                                const double *d_tface, const double *d_rhs,
                                                double *d_x, void *cuda_stream) {
  char msg[256];
  if (nsub < 1 || nsub > kNoAllocMaxSub) {
    snprintf(msg, sizeof msg,
             "mrcm_local_solve_noalloc: nsub=%d outside 1..%d (fixed scratch size)", nsub,
             kNoAllocMaxSub);
    mrcm::set_global_error(msg);
    return MRCM_EINVAL;
  }
  if (!d_kappa || !d_tface || !d_rhs || !d_x) {
    mrcm::set_global_error("mrcm_local_solve_noalloc: NULL device pointer");
    return MRCM_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "mrcm_local_solve_noalloc: cudaGetDevice: %s",
             cudaGetErrorString(e));
    mrcm::set_global_error(msg);
    return MRCM_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    snprintf(msg, sizeof msg,
             "mrcm_local_solve_noalloc: device index %d outside 0..%d (per-device table size)",
             dev, kMaxDevices - 1);
    mrcm::set_global_error(msg);
    return MRCM_EINVAL;
  }
  float *W = nullptr;
  {
    // first call on this device (or in a new context after a device reset):
    // look up the device address of the scratch array; this must happen
    // before any stream capture of this entry point
    std::lock_guard<std::mutex> lk(g_sym_mu);
    const CUcontext ctx = current_context();
    if (!g_sym[dev] || !ctx || ctx != g_sym_ctx[dev]) {
      void *ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_W);
      if (e != cudaSuccess || !ptr) {
        snprintf(msg, sizeof msg, "mrcm_local_solve_noalloc: cudaGetSymbolAddress: %s",
                 cudaGetErrorString(e));
        mrcm::set_global_error(msg);
        return MRCM_ECUDA;
      }
      g_sym[dev] = static_cast<float *>(ptr);
      g_sym_ctx[dev] = current_context();
    }
    W = g_sym[dev];
  }
  k_local_noalloc<<<nsub, kN, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      d_kappa, d_tface, d_rhs, d_x, W, 1e-13, 30);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "mrcm_local_solve_noalloc: launch: %s", cudaGetErrorString(e));
    mrcm::set_global_error(msg);
    return MRCM_ECUDA;
  }
  return MRCM_OK;
}
