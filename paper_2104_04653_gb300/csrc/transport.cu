// Implicit saturation transport (Section 4) and the sequential implicit /
// sequential fully implicit time steps built on it.
//
// One implicit Euler step of Eq. "BL2D" with the velocity frozen
// (Eq. "BL2D_Newton"), finite volumes with first-order upwind fluxes
// (Eqs. "fluxes_impli", "up_fluxes_impli"):
//     H_I(s) = s_I - s_I^n + (dt / h^2) sum_faces h u_out f(s_upwind) = 0,
// solved by Newton's method (Eq. "BL2D_Newton8") guarded by the
// inflection-point trust region of Section 4.1: every new value is kept in
// [0, 1], and a cell whose new value lies across the inflection point of f
// from its old one (f''(new) f''(old) < 0) takes the average of the two.
// The loop stops once ||s^{nu+1} - s^nu||_L2 <= eta.
//
// GB300 design.  The whole Newton loop of a step is ONE cooperative kernel
// (grid-wide barriers between phases; every realisation of the batch in the
// same launch, each stopping on its own test).  The linear system H' d = -H
// is the upwind Jacobian: a cell couples only to the neighbours it receives
// water from, so with the velocity of a potential flow the matrix is
// triangular in the order of the flow.  The solve exploits that:
//   * the grid is cut into 16 x 16-cell tiles, one CTA per tile at a time;
//   * a tile is solved exactly in shared memory by Jacobi sweeps on its own
//     cells, the values across its edges held fixed: on a flow that is
//     acyclic inside the tile the sweeps stop changing, bit for bit, after
//     at most the longest upwind path through the tile;
//   * outer block-Jacobi iterations exchange the tile edges through global
//     memory until no value changes (or the change is below 1e-15 of the
//     largest value, for flows with cycles), so the outer count is the
//     number of tile crossings along the longest upwind path.
// All arithmetic is FP64.  Reductions that decide a branch are exact (max
// of non-negative doubles through their integer bit patterns) or in a fixed
// order (the update norms), so every run takes the same path.
#include "../../include/mrcm.h"
#include "../../include/mrcm_transport.h"
#include "mrcm_internal.h"

#include <algorithm>
#include <cmath>
#include <cooperative_groups.h>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace cg = cooperative_groups;

namespace {

constexpr int kT = 16;                   // tile edge (cells)
constexpr int kThreads = kT * kT;        // one thread per cell of the tile
constexpr int kInnerCap = kT * kT + 1;   // sweeps: longest acyclic path + 1
constexpr double kCycleTol = 1e-15;      // outer stop for flows with cycles

// flags of the transport status word
constexpr int kFlagNewton = 0x1;         // a realisation hit max_newton
constexpr int kFlagLinear = 0x2;         // a linear solve hit its cap
constexpr int kFlagNan = 0x4;            // non-finite residual or update

struct TArgs {
  int nx, ny, R, tx, ty, ntiles;         // grid, tiles per realisation row/col
  double h, dt, M, f_in, eta, mu_w, mu_o;
  int max_newton, max_linear, trust_region;
  const double *ux, *uy, *s_old, *s_ref;
  double *s, *lambda;
  double *idiag, *cw, *ce, *cs, *cn, *rhs, *dA, *dB;
  double *fv, *fd;                       // f and f' of every cell (phase A0)
  double *tile_nrm2;                     // [R * tiles per realisation]
  // reductions as bit patterns of non-negative doubles: [0..2] max change
  // and [3..5] max |d| of the linear iterations (three rotating slots: a
  // slot is cleared two grid barriers after its last read), [6] max |s - ref|
  unsigned long long *red;
  int *done, *iters;                     // per realisation
  double *last_norm;                     // per realisation
  int *status;                           // [0] flags, [1] largest linear count
};

// f(s) = M s^2 / (M s^2 + (1 - s)^2) and f'(s) = 2 M s (1 - s) / den^2 by
// the quotient rule (Section 5), sharing one division (FP64 division is
// slow on this part: 442 clocks measured).
__device__ __forceinline__ void tf01(double s, double M, double &f, double &d) {
  const double den = M * s * s + (1.0 - s) * (1.0 - s);
  const double inv = 1.0 / den;
  f = M * s * s * inv;
  d = 2.0 * M * s * (1.0 - s) * inv * inv;
}
// f''(s) = (g' den - 2 g den') / den^3 with g = 2 M s (1 - s): den > 0, so
// the numerator carries its sign, which is all the trust region needs.
__device__ __forceinline__ double tf2_num(double s, double M) {
  const double den = M * s * s + (1.0 - s) * (1.0 - s);
  const double g = 2.0 * M * s * (1.0 - s);
  const double gp = 2.0 * M * (1.0 - 2.0 * s);
  const double denp = 2.0 * M * s - 2.0 * (1.0 - s);
  return gp * den - 2.0 * g * denp;
}

__device__ __forceinline__ unsigned long long dbits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}

// max over the CTA of a non-negative double, into *dst by its bit pattern
__device__ void block_max_to(double v, unsigned long long *dst, double *red8) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red8[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red8[0];
    for (int k = 1; k < kThreads / 32; ++k) m = fmax(m, red8[k]);
    if (m > 0.0) atomicMax(dst, dbits(m));
  }
  __syncthreads();
}

// fixed-order CTA sum (tree over lanes, then warps in order)
__device__ double block_sum(double v, double *red8) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red8[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < kThreads / 32; ++k) s += red8[k];
  __syncthreads();
  return s;   // valid in thread 0
}

struct Cell {
  bool in;          // inside the grid
  int r, i, j;      // realisation, column, row
  int64_t c;        // index into [R][ny][nx]
};

__device__ __forceinline__ Cell tile_cell(const TArgs &a, int t) {
  const int per = a.tx * a.ty;
  Cell q;
  q.r = t / per;
  const int tt = t - q.r * per, ti = tt % a.tx, tj = tt / a.tx;
  q.i = ti * kT + (threadIdx.x % kT);
  q.j = tj * kT + (threadIdx.x / kT);
  q.in = q.i < a.nx && q.j < a.ny;
  q.c = (static_cast<int64_t>(q.r) * a.ny + q.j) * a.nx + q.i;
  return q;
}

// outward normal velocities of cell (i, j) of realisation r: W, E, S, N
__device__ __forceinline__ void outward(const TArgs &a, const Cell &q, double u[4]) {
  const int64_t xr = static_cast<int64_t>(q.r) * a.ny * (a.nx + 1);
  const int64_t yr = static_cast<int64_t>(q.r) * (a.ny + 1) * a.nx;
  u[0] = -a.ux[xr + static_cast<int64_t>(q.j) * (a.nx + 1) + q.i];
  u[1] = a.ux[xr + static_cast<int64_t>(q.j) * (a.nx + 1) + q.i + 1];
  u[2] = -a.uy[yr + static_cast<int64_t>(q.j) * a.nx + q.i];
  u[3] = a.uy[yr + static_cast<int64_t>(q.j + 1) * a.nx + q.i];
}

// Phase A: H and the Jacobian of one cell; rhs = -H, the linear iterate 0.
__device__ void assemble_cell(const TArgs &a, const Cell &q) {
  double u[4];
  outward(a, q, u);
  const double sI = a.s[q.c];
  const double fI = a.fv[q.c], dI = a.fd[q.c];
  const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
  const double c = a.dt / a.h;
  double out = 0.0, diag = 1.0, cpl[4];
  for (int k = 0; k < 4; ++k) {
    const int ni = q.i + di[k], nj = q.j + dj[k];
    const bool inside = ni >= 0 && ni < a.nx && nj >= 0 && nj < a.ny;
    const int64_t nc = q.c + dj[k] * static_cast<int64_t>(a.nx) + di[k];
    const double fJ = inside ? a.fv[nc] : a.f_in;
    out += (u[k] > 0.0 ? u[k] * fI : u[k] * fJ) * a.h;
    if (u[k] > 0.0) diag += c * u[k] * dI;
    cpl[k] = (u[k] <= 0.0 && inside) ? c * u[k] * a.fd[nc] : 0.0;
  }
  const double H = sI - a.s_old[q.c] + a.dt / (a.h * a.h) * out;
  a.rhs[q.c] = -H;
  a.idiag[q.c] = 1.0 / diag;     // the sweeps multiply (diag >= 1)
  a.cw[q.c] = cpl[0];
  a.ce[q.c] = cpl[1];
  a.cs[q.c] = cpl[2];
  a.cn[q.c] = cpl[3];
  a.dA[q.c] = 0.0;
  if (!isfinite(H)) atomicOr(&a.status[0], kFlagNan);
}

// Phase B, one tile: exact Jacobi sweeps on the tile's cells with the
// values across its edges taken from src; result to dst.  Returns (in
// thread 0 through shared memory) nothing; block maxima go to red.
__device__ void solve_tile(const TArgs &a, int t, const double *src, double *dst, int slot,
                           double *sd, double *red8) {
  const Cell q = tile_cell(a, t);
  const int lx = threadIdx.x % kT + 1, ly = threadIdx.x / kT + 1;
  constexpr int W = kT + 2;
  // halo ring and interior from src (previous outer iterate); outside: 0
  for (int e = threadIdx.x; e < W * W; e += kThreads) {
    const int hx = e % W, hy = e / W;
    const int per = a.tx * a.ty, tt = t - q.r * per;
    const int gi = (tt % a.tx) * kT + hx - 1, gj = (tt / a.tx) * kT + hy - 1;
    double v = 0.0;
    if (gi >= 0 && gi < a.nx && gj >= 0 && gj < a.ny)
      v = src[(static_cast<int64_t>(q.r) * a.ny + gj) * a.nx + gi];
    sd[e] = v;
  }
  double idg = 1.0, cw = 0.0, ce = 0.0, cs = 0.0, cn = 0.0, b = 0.0, old = 0.0;
  if (q.in) {
    idg = a.idiag[q.c];
    cw = a.cw[q.c];
    ce = a.ce[q.c];
    cs = a.cs[q.c];
    cn = a.cn[q.c];
    b = a.rhs[q.c];
  }
  __syncthreads();
  old = sd[ly * W + lx];
  for (int sweep = 0; sweep < kInnerCap; ++sweep) {
    double v = old;
    if (q.in)
      v = (b - cw * sd[ly * W + lx - 1] - ce * sd[ly * W + lx + 1] - cs * sd[(ly - 1) * W + lx] -
           cn * sd[(ly + 1) * W + lx]) * idg;
    const int changed = q.in && v != sd[ly * W + lx];
    __syncthreads();
    if (q.in) sd[ly * W + lx] = v;
    if (!__syncthreads_or(changed)) break;
  }
  double chg = 0.0, mag = 0.0;
  if (q.in) {
    const double v = sd[ly * W + lx];
    dst[q.c] = v;
    chg = fabs(v - old);
    mag = fabs(v);
  }
  block_max_to(chg, &a.red[slot], red8);
  block_max_to(mag, &a.red[3 + slot], red8);
}

__global__ void __launch_bounds__(kThreads) k_transport(TArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sd[(kT + 2) * (kT + 2)];
  __shared__ double red8[kThreads / 32];
  const int T = a.ntiles, per = a.tx * a.ty;
  int all_done = 0;
  for (int it = 1; it <= a.max_newton && !all_done; ++it) {
    // A0: f and f' of every cell (one division each)
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
      const Cell q = tile_cell(a, t);
      if (q.in && !a.done[q.r]) tf01(a.s[q.c], a.M, a.fv[q.c], a.fd[q.c]);
    }
    grid.sync();
    // A: residual and Jacobian
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
      const Cell q = tile_cell(a, t);
      if (q.in && !a.done[q.r]) assemble_cell(a, q);
    }
    if (blockIdx.x == 0 && threadIdx.x < 6) a.red[threadIdx.x] = 0ull;
    grid.sync();
    // B: outer block-Jacobi iterations of exact tile solves
    double *src = a.dA, *dst = a.dB;
    int k = 0;
    for (; k < a.max_linear; ++k) {
      // slot k % 3 collects this iteration; slot (k + 1) % 3, read last
      // before the previous barrier but one, is cleared for the next
      const int slot = k % 3, next = (k + 1) % 3;
      for (int t = blockIdx.x; t < T; t += gridDim.x)
        if (!a.done[t / per]) solve_tile(a, t, src, dst, slot, sd, red8);
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.red[next] = 0ull;
        a.red[3 + next] = 0ull;
      }
      grid.sync();
      const double chg = __longlong_as_double(static_cast<long long>(a.red[slot]));
      const double mag = __longlong_as_double(static_cast<long long>(a.red[3 + slot]));
      double *tmp = src;
      src = dst;
      dst = tmp;
      if (chg == 0.0 || chg <= kCycleTol * mag) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (k >= a.max_linear) atomicOr(&a.status[0], kFlagLinear);
      atomicMax(&a.status[1], k + 1);
    }
    // C: trust-region update, per-tile update norms
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
      const Cell q = tile_cell(a, t);
      if (a.done[q.r]) continue;
      double d2 = 0.0;
      if (q.in) {
        const double so = a.s[q.c];
        double nv = fmin(fmax(so + src[q.c], 0.0), 1.0);
        if (a.trust_region && tf2_num(nv, a.M) * tf2_num(so, a.M) < 0.0) nv = 0.5 * (nv + so);
        if (!isfinite(nv)) atomicOr(&a.status[0], kFlagNan);
        a.s[q.c] = nv;
        d2 = (nv - so) * (nv - so) * a.h * a.h;
      }
      const double sum = block_sum(d2, red8);
      if (threadIdx.x == 0) a.tile_nrm2[t] = sum;
    }
    grid.sync();
    // D: one warp per realisation sums its tiles in a fixed order
    const int lane = threadIdx.x & 31, wglob = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    for (int r = wglob; r < a.R; r += gridDim.x * (kThreads / 32)) {
      if (a.done[r]) continue;
      double v = 0.0;
      for (int t = lane; t < per; t += 32) v += a.tile_nrm2[static_cast<int64_t>(r) * per + t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) {
        const double nrm = sqrt(v);
        a.last_norm[r] = nrm;
        a.iters[r] = it;
        if (nrm <= a.eta) a.done[r] = 1;
      }
    }
    grid.sync();
    all_done = 1;
    for (int r = 0; r < a.R; ++r) all_done &= a.done[r];
  }
  if (!all_done && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.status[0], kFlagNewton);
  // outputs: total mobility lambda = s^2/mu_w + (1-s)^2/mu_o; change vs ref
  double chg = 0.0;
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const Cell q = tile_cell(a, t);
    if (!q.in) continue;
    const double sv = a.s[q.c];
    if (a.lambda) a.lambda[q.c] = sv * sv / a.mu_w + (1.0 - sv) * (1.0 - sv) / a.mu_o;
    if (a.s_ref) chg = fmax(chg, fabs(sv - a.s_ref[q.c]));
  }
  if (a.s_ref) block_max_to(chg, &a.red[6], red8);
}

__global__ void k_copy(const double *src, double *dst, int64_t n) {
  for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
       k += static_cast<int64_t>(gridDim.x) * blockDim.x)
    dst[k] = src[k];
}

thread_local std::string g_terr;

mrcm_status terr(mrcm_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_terr = buf;
  return s;
}

}  // namespace

struct mrcm_transport {
  mrcm_transport_desc d{};
  cudaStream_t stream = nullptr;
  int dev = 0, grid = 0, tx = 0, ty = 0, ntiles = 0;
  int64_t ncell = 0;
  char *arena = nullptr;
  TArgs a{};
  bool stepped = false;
};

extern "C" {

const char *mrcm_transport_last_error(void) { return g_terr.c_str(); }

mrcm_status mrcm_transport_create(const mrcm_transport_desc *desc, void *cuda_stream,
                                  mrcm_transport **out) {
  if (!out) return terr(MRCM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!desc) return terr(MRCM_EINVAL, "descriptor is NULL");
  const mrcm_transport_desc &d = *desc;
  if (d.nx < 1 || d.ny < 1 || d.n_real < 1 || d.n_real > mrcm::kMaxRealisations)
    return terr(MRCM_EINVAL, "grid %d x %d x %d", d.nx, d.ny, d.n_real);
  if (static_cast<int64_t>(d.nx) * d.ny > (int64_t{1} << 28))
    return terr(MRCM_EINVAL, "grid of %lld cells above 2^28", static_cast<long long>(d.nx) * d.ny);
  if (!(d.ly > 0.0) || !(d.M > 0.0) || !(d.mu_w > 0.0) || !(d.s_in >= 0.0 && d.s_in <= 1.0) ||
      !(d.eta >= 0.0) || d.max_newton < 0 || d.max_newton > 100000 || d.max_linear < 0 ||
      d.max_linear > 1000000)
    return terr(MRCM_EINVAL, "invalid transport parameters");
  mrcm_transport *t = new mrcm_transport();
  t->d = d;
  if (t->d.eta == 0.0) t->d.eta = 1e-6;
  if (t->d.max_newton == 0) t->d.max_newton = 100;
  t->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&t->dev);
  if (e != cudaSuccess) {
    delete t;
    return terr(MRCM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  }
  t->tx = (d.nx + kT - 1) / kT;
  t->ty = (d.ny + kT - 1) / kT;
  t->ntiles = t->tx * t->ty * d.n_real;
  if (t->d.max_linear == 0) t->d.max_linear = 4 * (t->tx + t->ty) + 64;
  t->ncell = static_cast<int64_t>(d.nx) * d.ny * d.n_real;
  int nsm = 0, per = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, t->dev);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_transport, kThreads, 0)) !=
          cudaSuccess ||
      per < 1) {
    delete t;
    return terr(MRCM_ECUDA, "occupancy of the transport kernel: %s", cudaGetErrorString(e));
  }
  t->grid = std::min(t->ntiles, nsm * per);
  // workspace: 10 cell arrays, tile norms, reductions and per-realisation
  // state, each rounded up to 256 bytes
  const int64_t nc = t->ncell, R = d.n_real;
  auto rnd = [](size_t n) { return (n + 255) & ~static_cast<size_t>(255); };
  const size_t sizes[16] = {8 * static_cast<size_t>(nc), 8 * static_cast<size_t>(nc),
                            8 * static_cast<size_t>(nc), 8 * static_cast<size_t>(nc),
                            8 * static_cast<size_t>(nc), 8 * static_cast<size_t>(nc),
                            8 * static_cast<size_t>(nc), 8 * static_cast<size_t>(nc),
                            8 * static_cast<size_t>(nc), 8 * static_cast<size_t>(nc),
                            8 * static_cast<size_t>(t->ntiles), 8 * static_cast<size_t>(R),
                            8 * 8, 4 * static_cast<size_t>(R), 4 * static_cast<size_t>(R), 16};
  size_t bytes = 0;
  for (size_t z : sizes) bytes += rnd(z);
  if ((e = cudaMalloc(&t->arena, bytes)) != cudaSuccess) {
    delete t;
    return terr(MRCM_ENOMEM, "transport workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  char *p = t->arena;
  int taken = 0;
  auto take = [&](size_t n) {
    char *q = p;
    p += rnd(n);
    ++taken;
    return q;
  };
  TArgs &a = t->a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.R = d.n_real;
  a.tx = t->tx;
  a.ty = t->ty;
  a.ntiles = t->ntiles;
  a.h = d.ly / d.ny;
  a.M = d.M;
  a.mu_w = d.mu_w;
  a.mu_o = d.M * d.mu_w;
  a.f_in = d.M * d.s_in * d.s_in / (d.M * d.s_in * d.s_in + (1.0 - d.s_in) * (1.0 - d.s_in));
  a.eta = t->d.eta;
  a.max_newton = t->d.max_newton;
  a.max_linear = t->d.max_linear;
  a.trust_region = d.plain_newton ? 0 : 1;
  a.idiag = reinterpret_cast<double *>(take(nc * 8));
  a.cw = reinterpret_cast<double *>(take(nc * 8));
  a.ce = reinterpret_cast<double *>(take(nc * 8));
  a.cs = reinterpret_cast<double *>(take(nc * 8));
  a.cn = reinterpret_cast<double *>(take(nc * 8));
  a.rhs = reinterpret_cast<double *>(take(nc * 8));
  a.dA = reinterpret_cast<double *>(take(nc * 8));
  a.dB = reinterpret_cast<double *>(take(nc * 8));
  a.fv = reinterpret_cast<double *>(take(nc * 8));
  a.fd = reinterpret_cast<double *>(take(nc * 8));
  a.tile_nrm2 = reinterpret_cast<double *>(take(t->ntiles * 8));
  a.last_norm = reinterpret_cast<double *>(take(R * 8));
  a.red = reinterpret_cast<unsigned long long *>(take(8 * 8));
  a.done = reinterpret_cast<int *>(take(R * 4));
  a.iters = reinterpret_cast<int *>(take(R * 4));
  a.status = reinterpret_cast<int *>(take(16));
  if (taken != 16 || p != t->arena + bytes) {       // the takes above match sizes[]
    cudaFree(t->arena);
    delete t;
    return terr(MRCM_ECUDA, "transport workspace layout mismatch");
  }
  if ((e = cudaMemset(t->arena, 0, bytes)) != cudaSuccess) {
    cudaFree(t->arena);
    delete t;
    return terr(MRCM_ECUDA, "transport workspace clear: %s", cudaGetErrorString(e));
  }
  *out = t;
  return MRCM_OK;
}

mrcm_status mrcm_transport_step(mrcm_transport *t, double dt, const double *d_ux,
                                const double *d_uy, const double *d_s_old, double *d_s_new,
                                double *d_lambda, const double *d_s_ref) {
  if (!t) return terr(MRCM_EINVAL, "NULL transport context");
  if (!d_ux || !d_uy || !d_s_old || !d_s_new)
    return terr(MRCM_EINVAL, "NULL velocity or saturation pointer");
  if (d_s_new == d_s_old) return terr(MRCM_EINVAL, "s_new must not alias s_old");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return terr(MRCM_EINVAL, "dt = %g", dt);
  TArgs a = t->a;
  a.dt = dt;
  a.ux = d_ux;
  a.uy = d_uy;
  a.s_old = d_s_old;
  a.s_ref = d_s_ref;
  a.s = d_s_new;
  a.lambda = d_lambda;
  cudaError_t e;
  const int R = t->d.n_real;
  // per-step state: done flags, iteration counts, reductions, status
  if ((e = cudaMemsetAsync(a.done, 0, sizeof(int) * R, t->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.iters, 0, sizeof(int) * R, t->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.red, 0, sizeof(unsigned long long) * 8, t->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(a.status, 0, 16, t->stream)) != cudaSuccess)
    return terr(MRCM_ECUDA, "transport reset: %s", cudaGetErrorString(e));
  // the Newton loop starts from s^n (Section 4: s^{n+1,0} = s^n)
  const int cb = static_cast<int>(std::min<int64_t>((t->ncell + 255) / 256, 4096));
  k_copy<<<cb, 256, 0, t->stream>>>(d_s_old, d_s_new, t->ncell);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return terr(MRCM_ECUDA, "transport copy: %s", cudaGetErrorString(e));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(t->grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = t->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if ((e = cudaLaunchKernelEx(&cfg, k_transport, a)) != cudaSuccess)
    return terr(MRCM_ECUDA, "transport launch: %s", cudaGetErrorString(e));
  t->stepped = true;
  return MRCM_OK;
}

mrcm_status mrcm_transport_get_info(mrcm_transport *t, mrcm_transport_info *info,
                                    int32_t *newton_iters) {
  if (!t || !info) return terr(MRCM_EINVAL, "NULL argument");
  *info = mrcm_transport_info{};
  if (!t->stepped) return MRCM_OK;
  const int R = t->d.n_real;
  std::vector<int> it(R);
  std::vector<double> nrm(R);
  int st[2] = {0, 0};
  unsigned long long chg = 0;
  cudaError_t e;
  if ((e = cudaStreamSynchronize(t->stream)) != cudaSuccess ||
      (e = cudaMemcpy(it.data(), t->a.iters, sizeof(int) * R, cudaMemcpyDeviceToHost)) !=
          cudaSuccess ||
      (e = cudaMemcpy(nrm.data(), t->a.last_norm, sizeof(double) * R, cudaMemcpyDeviceToHost)) !=
          cudaSuccess ||
      (e = cudaMemcpy(st, t->a.status, sizeof st, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&chg, t->a.red + 6, sizeof chg, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return terr(MRCM_ECUDA, "transport info: %s", cudaGetErrorString(e));
  for (int r = 0; r < R; ++r) {
    info->newton_iters_max = std::max(info->newton_iters_max, it[r]);
    info->update_norm_max = std::max(info->update_norm_max, nrm[r]);
    if (newton_iters) newton_iters[r] = it[r];
  }
  info->linear_iters_max = st[1];
  info->flags = st[0];
  double c;
  static_assert(sizeof c == sizeof chg, "bit pattern");
  memcpy(&c, &chg, sizeof c);
  info->change_max = c;
  if (st[0] & kFlagNan) return terr(MRCM_ENAN, "transport: non-finite residual or update");
  if (st[0] & kFlagNewton)
    return terr(MRCM_ENOCONV, "transport: Newton stopped at %d iterations, update norm %.3e",
                t->d.max_newton, info->update_norm_max);
  if (st[0] & kFlagLinear)
    return terr(MRCM_ENOCONV, "transport: a linear solve stopped at %d outer iterations",
                t->d.max_linear);
  return MRCM_OK;
}

mrcm_status mrcm_transport_set_stream(mrcm_transport *t, void *cuda_stream) {
  if (!t) return terr(MRCM_EINVAL, "NULL transport context");
  t->stream = static_cast<cudaStream_t>(cuda_stream);
  return MRCM_OK;
}

void mrcm_transport_destroy(mrcm_transport *t) {
  if (!t) return;
  if (t->arena) cudaFree(t->arena);
  delete t;
}

// The Darcy solve of one SI / SFI iteration: the five calls of mrcm.h.
static mrcm_status darcy(mrcm_ctx *ctx, const double *d_K, const double *d_lambda,
                         const double *d_q, double *d_p, double *d_ux, double *d_uy) {
  mrcm_status st;
  if ((st = mrcm_factor_local(ctx, d_K, d_lambda)) != MRCM_OK ||
      (st = mrcm_build_basis(ctx, d_q)) != MRCM_OK ||
      (st = mrcm_solve_interface(ctx, nullptr)) != MRCM_OK ||
      (st = mrcm_reconstruct(ctx, d_p, d_ux, d_uy, nullptr)) != MRCM_OK)
    return terr(st, "Darcy solve: %s", mrcm_last_error(ctx));
  return MRCM_OK;
}

mrcm_status mrcm_si_step(mrcm_ctx *ctx, mrcm_transport *t, double dt, const double *d_K,
                         double *d_lambda, const double *d_q, const double *d_s_old,
                         double *d_s_new, double *d_p, double *d_ux, double *d_uy) {
  if (!ctx || !t) return terr(MRCM_EINVAL, "NULL context");
  mrcm_status st = darcy(ctx, d_K, d_lambda, d_q, d_p, d_ux, d_uy);
  if (st != MRCM_OK) return st;
  return mrcm_transport_step(t, dt, d_ux, d_uy, d_s_old, d_s_new, d_lambda, nullptr);
}

mrcm_status mrcm_sfi_step(mrcm_ctx *ctx, mrcm_transport *t, double dt, double tol,
                          int32_t max_outer, const double *d_K, double *d_lambda,
                          const double *d_q, const double *d_s_old, double *d_s_new,
                          double *d_s_work, double *d_p, double *d_ux, double *d_uy,
                          int32_t *outer_iters) {
  if (!ctx || !t) return terr(MRCM_EINVAL, "NULL context");
  if (!d_s_work || d_s_work == d_s_new || d_s_work == d_s_old)
    return terr(MRCM_EINVAL, "d_s_work must be a separate cell array");
  if (max_outer < 1 || !(tol >= 0.0)) return terr(MRCM_EINVAL, "max_outer / tol");
  if (outer_iters) *outer_iters = 0;
  cudaError_t e;
  const size_t bytes = sizeof(double) * static_cast<size_t>(t->ncell);
  // the first iterate is s^n (its mobility is the caller's d_lambda)
  if ((e = cudaMemcpyAsync(d_s_new, d_s_old, bytes, cudaMemcpyDeviceToDevice, t->stream)) !=
      cudaSuccess)
    return terr(MRCM_ECUDA, "SFI copy: %s", cudaGetErrorString(e));
  for (int k = 1; k <= max_outer; ++k) {
    mrcm_status st = darcy(ctx, d_K, d_lambda, d_q, d_p, d_ux, d_uy);
    if (st != MRCM_OK) return st;
    if ((e = cudaMemcpyAsync(d_s_work, d_s_new, bytes, cudaMemcpyDeviceToDevice, t->stream)) !=
        cudaSuccess)
      return terr(MRCM_ECUDA, "SFI copy: %s", cudaGetErrorString(e));
    if ((st = mrcm_transport_step(t, dt, d_ux, d_uy, d_s_old, d_s_new, d_lambda, d_s_work)) !=
        MRCM_OK)
      return st;
    mrcm_transport_info info;
    if ((st = mrcm_transport_get_info(t, &info, nullptr)) != MRCM_OK) return st;
    if (outer_iters) *outer_iters = k;
    if (info.change_max < tol) return MRCM_OK;
  }
  return terr(MRCM_ENOCONV, "SFI: %d outer iterations without the change falling below %g",
              max_outer, tol);
}

}  // extern "C"
