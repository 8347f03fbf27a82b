// Batched n x n GEMM on the 5th-generation tensor cores (tcgen05) with
// FP32-level accuracy: every FP32 operand is split into a TF32 head and a
// TF32 tail (x = hi + lo, hi = x rounded to TF32), and
//   A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory (the dropped A_lo B_lo term is
// 2^-22 relative).  Used by the large-slab interface factor (the same job
// descriptors as the SIMT kernel).
//
// Per CTA: one 128 x 128 output tile, 256 threads.  K advances in chunks of
// 32: all threads load the chunk of A (128 rows) and B (128 columns),
// split it and store the four operand tiles in shared memory in the
// 128-byte-swizzled K-major layout; one thread issues 4 x 3 MMAs
// (M = 128, N = 128, K = 8 each) and commits them to an mbarrier that every
// thread waits on (bounded) before the buffers are reused.  The accumulator
// (128 lanes x 128 FP32 columns of TMEM) is read back with tcgen05.ld, two
// warps per 32-lane quarter.
#include "mrcm_internal.h"
#include "../../include/mrcm.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include <vector>

namespace mrcm {
namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = 32;     // tile and K chunk
constexpr int kTcTileBytes = kTcM * kTcK * 4;         // 16 KB per operand tile
constexpr unsigned kTcWaitLimit = 1u << 26;           // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) in a 128-row x 32-element K-major tile
// with the 128-byte swizzle (16-byte chunk index XOR row mod 8)
__device__ __forceinline__ uint32_t sw128(int row, int k) {
  return static_cast<uint32_t>(row * 128 + ((((k >> 2) ^ (row & 7)) & 7) << 4) + ((k & 3) << 2));
}

// shared-memory matrix descriptor: 128B swizzle, K-major, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFF);          // start address
  d |= static_cast<uint64_t>(1) << 16;                        // leading byte offset (unused)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;                // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                        // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                        // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, FP32 accumulate, A and B K-major,
// M = 128, N = 128
__device__ __forceinline__ uint32_t idesc_tf32() {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format: F32
  d |= 2u << 7;                    // A format: TF32
  d |= 2u << 10;                   // B format: TF32
  d |= static_cast<uint32_t>(kTcN >> 3) << 17;
  d |= static_cast<uint32_t>(kTcM >> 4) << 24;
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

// wait for the phase with the given parity; false if the limit ran out
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          unsigned limit = kTcWaitLimit) {
  for (unsigned it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity));
    if (ok) return true;
  }
  return false;
}

// The tensor-core kernels' bounded wait on an mbarrier that nothing
// completes (its one expected arrival never comes): the wait gives up after
// ``limit`` tries and the timeout flag is raised, as in the GEMM kernels.
__global__ void k_wait_probe(int *status, unsigned limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(smem_u32(&bar), 1);
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar), 0, limit);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(status, MRCM_FLAG_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)));
  }
}

__global__ void __launch_bounds__(256) k_tc_gemm(const GemmJob *jobs, int *status) {
  extern __shared__ __align__(1024) unsigned char tcsm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  // the four operand tiles, 1024-byte aligned
  const uint32_t raw = smem_u32(tcsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *sm = tcsm + (base - raw);
  const uint32_t tAh = base, tAl = base + kTcTileBytes, tBh = base + 2 * kTcTileBytes,
                 tBl = base + 3 * kTcTileBytes;

  const GemmJob jb = jobs[blockIdx.y];
  const int n = jb.n;
  const int nt = (n + kTcM - 1) / kTcM;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;                       // whole CTA, before any barrier
  const int i0 = ti * kTcM, j0 = tj * kTcN;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const uint32_t bar_a = smem_u32(&bar);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    mbar_init(bar_a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  const float *A1 = static_cast<const float *>(jb.a1), *A2 = static_cast<const float *>(jb.a2);
  const float *B1 = static_cast<const float *>(jb.b1), *B2 = static_cast<const float *>(jb.b2);
  const int nk = (n + kTcK - 1) / kTcK;
  const int np = (A1 && B1 ? 1 : 0) + (A2 && B2 ? 1 : 0);
  const int first = (A1 && B1) ? 0 : 1;
  const int total = np * nk;
  const uint32_t idesc = idesc_tf32();
  uint32_t parity = 0;
  bool fail = false;
  for (int step = 0; step < total; ++step) {
    const int prod = first + step / nk, k0 = (step % nk) * kTcK;
    const float *Ap = prod == 0 ? A1 : A2, *Bp = prod == 0 ? B1 : B2;
    // A chunk: 128 rows x 32 k (16 per thread); B chunk: 32 k x 128 columns,
    // stored transposed (row = output column, K-major)
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int e = t + 256 * q;
      const int r = e >> 5, k = e & 31;
      const int gi = i0 + r, gk = k0 + k;
      const float v = (gi < n && gk < n) ? Ap[static_cast<int64_t>(gi) * n + gk] : 0.0f;
      const float hi = tf32_round(v);
      const uint32_t o = sw128(r, k);
      *reinterpret_cast<float *>(sm + o) = hi;
      *reinterpret_cast<float *>(sm + kTcTileBytes + o) = v - hi;
    }
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int e = t + 256 * q;
      const int k = e >> 7, c = e & 127;
      const int gk = k0 + k, gj = j0 + c;
      const float v = (gk < n && gj < n) ? Bp[static_cast<int64_t>(gk) * n + gj] : 0.0f;
      const float hi = tf32_round(v);
      const uint32_t o = sw128(c, k);
      *reinterpret_cast<float *>(sm + 2 * kTcTileBytes + o) = hi;
      *reinterpret_cast<float *>(sm + 3 * kTcTileBytes + o) = v - hi;
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t off = kk * 32;        // 8 TF32 = 32 bytes along K
        const uint64_t ah = sdesc(tAh + off), al = sdesc(tAl + off);
        const uint64_t bh = sdesc(tBh + off), bl = sdesc(tBl + off);
        mma_tf32(tmem, ah, bh, idesc, (step | kk) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              bar_a));
    }
    if (!mbar_wait(bar_a, parity)) fail = true;
    if (__syncthreads_or(fail)) {
      // give the MMAs in flight one more bounded wait before TMEM is freed
      mbar_wait(bar_a, parity);
      fail = true;
      break;
    }
    parity ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (fail) {
    if (t == 0) atomicOr(status, MRCM_FLAG_TIMEOUT);
  } else if (total > 0) {
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31, columns 64 (w / 4) .. + 63
    const int quarter = warp & 3, half = warp >> 2;
    const int row = i0 + 32 * quarter + lane;
    float *C = static_cast<float *>(jb.c);
    const float alpha = static_cast<float>(jb.alpha);
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      const int col0 = 64 * half + 32 * cb;
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + col0;
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
        float *cr = C + static_cast<int64_t>(row) * n;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int gj = j0 + col0 + q;
          if (gj < n) {
            const float a = alpha * __uint_as_float(v[q]);
            cr[gj] = jb.acc ? cr[gj] + a : a;
          }
        }
      }
    }
  } else {
    // no product: C = 0 (or unchanged when accumulating)
    float *C = static_cast<float *>(jb.c);
    if (!jb.acc)
      for (int e = t; e < kTcM * kTcN; e += 256) {
        const int r = i0 + e / kTcN, c = j0 + e % kTcN;
        if (r < n && c < n) C[static_cast<int64_t>(r) * n + c] = 0.0f;
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

// ---------------------------------------------------------------------------
// Pipelined form.  A packing pass writes every product's operands as TF32
// head and tail planes with rows padded to a multiple of 32 (zeros): A as
// [n][ldp] (K contiguous), B transposed to [n][ldp] (row = output column,
// K contiguous).  The GEMM kernel then streams 32-wide K chunks of the four
// planes with TMA (cp.async.bulk.tensor, 128-byte swizzle, the MMA layout)
// through a 3-stage ring: one thread issues the copies (full barriers with
// transaction counts), one thread issues the MMAs and commits each stage
// back to its empty barrier, and a final commit releases the epilogue.
constexpr int kTcStages = 3;
constexpr int kTcStageBytes = 4 * kTcTileBytes;       // A_hi A_lo B_hi B_lo

// plane p (0 A_hi, 1 A_lo, 2 B_hi, 3 B_lo) of product q of job slot j
__device__ __forceinline__ float *pack_plane(float *base, int64_t plane_elems, int slot, int q,
                                             int p) {
  return base + ((static_cast<int64_t>(slot) * 2 + q) * 4 + p) * plane_elems;
}

// grid: (32 x 32 tiles of [n][ldp], jobs of the chunk, product); 32 x 8 threads
__global__ void __launch_bounds__(256) k_tc_pack(const GemmJob *jobs, float *base,
                                                 int64_t plane_elems) {
  __shared__ float tb[32][33];
  const GemmJob jb = jobs[blockIdx.y];
  const int q = blockIdx.z;
  const float *A = static_cast<const float *>(q == 0 ? jb.a1 : jb.a2);
  const float *B = static_cast<const float *>(q == 0 ? jb.b1 : jb.b2);
  if (!A || !B) return;
  const int n = jb.n, ldp = (n + kTcK - 1) / kTcK * kTcK;
  const int tk = ldp / 32, tr = (n + 31) / 32;
  if (static_cast<int>(blockIdx.x) >= tk * tr) return;
  const int r0 = (blockIdx.x / tk) * 32, k0 = (blockIdx.x % tk) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float *ahi = pack_plane(base, plane_elems, blockIdx.y, q, 0);
  float *alo = pack_plane(base, plane_elems, blockIdx.y, q, 1);
  float *bhi = pack_plane(base, plane_elems, blockIdx.y, q, 2);
  float *blo = pack_plane(base, plane_elems, blockIdx.y, q, 3);
  for (int rr = ty; rr < 32; rr += 8) {
    const int r = r0 + rr, k = k0 + tx;
    if (r >= n) continue;
    const float v = k < n ? A[static_cast<int64_t>(r) * n + k] : 0.0f;
    const float hi = tf32_round(v);
    ahi[static_cast<int64_t>(r) * ldp + k] = hi;
    alo[static_cast<int64_t>(r) * ldp + k] = v - hi;
  }
  // B^T: tile rows k0.., columns r0.. of B become rows r0.., columns k0..
  for (int kk = ty; kk < 32; kk += 8) {
    const int k = k0 + kk, c = r0 + tx;
    tb[kk][tx] = (k < n && c < n) ? B[static_cast<int64_t>(k) * n + c] : 0.0f;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = r0 + cc, k = k0 + tx;
    if (c >= n) continue;
    const float v = tb[tx][cc];
    const float hi = tf32_round(v);
    bhi[static_cast<int64_t>(c) * ldp + k] = hi;
    blo[static_cast<int64_t>(c) * ldp + k] = v - hi;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__global__ void __launch_bounds__(256) k_tc_gemm_tma(const GemmJob *jobs, const CUtensorMap *maps,
                                                     int *status) {
  extern __shared__ __align__(1024) unsigned char tcsm[];
  __shared__ uint64_t full[kTcStages], empty[kTcStages], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const uint32_t raw = smem_u32(tcsm);
  const uint32_t base = (raw + 1023u) & ~1023u;

  const GemmJob jb = jobs[blockIdx.y];
  const CUtensorMap *mp = maps + static_cast<int64_t>(blockIdx.y) * 8;
  const int n = jb.n;
  const int nt = (n + kTcM - 1) / kTcM;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;
  const int i0 = ti * kTcM, j0 = tj * kTcN;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nk = (n + kTcK - 1) / kTcK;
  const bool has1 = jb.a1 && jb.b1, has2 = jb.a2 && jb.b2;
  const int first = has1 ? 0 : 1;
  const int total = ((has1 ? 1 : 0) + (has2 ? 1 : 0)) * nk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 32) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (t == 0) {
    // producer
    for (int step = 0; step < total; ++step) {
      const int s = step % kTcStages;
      if (step >= kTcStages && !mbar_wait(smem_u32(&empty[s]), ((step / kTcStages) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      const int q = first + step / nk, k0 = (step % nk) * kTcK;
      const uint32_t st = base + s * kTcStageBytes, fb = smem_u32(&full[s]);
      mbar_expect_tx(fb, kTcStageBytes);
      tma_load_2d(st, mp + q * 4 + 0, k0, i0, fb);
      tma_load_2d(st + kTcTileBytes, mp + q * 4 + 1, k0, i0, fb);
      tma_load_2d(st + 2 * kTcTileBytes, mp + q * 4 + 2, k0, j0, fb);
      tma_load_2d(st + 3 * kTcTileBytes, mp + q * 4 + 3, k0, j0, fb);
    }
  } else if (t == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32();
    for (int step = 0; step < total; ++step) {
      const int s = step % kTcStages;
      if (!mbar_wait(smem_u32(&full[s]), (step / kTcStages) & 1)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t st = base + s * kTcStageBytes;
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const uint32_t off = kk * 32;
        const uint64_t ah = sdesc(st + off), al = sdesc(st + kTcTileBytes + off);
        const uint64_t bh = sdesc(st + 2 * kTcTileBytes + off),
                       bl = sdesc(st + 3 * kTcTileBytes + off);
        mma_tf32(tmem, ah, bh, idesc, (step | kk) ? 1u : 0u);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      tc_commit(smem_u32(&empty[s]));
    }
    tc_commit(smem_u32(&done));
  }
  __syncwarp();
  bool ok = mbar_wait(smem_u32(&done), 0);
  __syncthreads();
  ok = ok && !s_fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!ok) {
    if (t == 0) atomicOr(status, MRCM_FLAG_TIMEOUT);
    mbar_wait(smem_u32(&done), 0);
  } else if (total > 0) {
    const int quarter = warp & 3, half = warp >> 2;
    const int row = i0 + 32 * quarter + lane;
    float *C = static_cast<float *>(jb.c);
    const float alpha = static_cast<float>(jb.alpha);
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
      const int col0 = 64 * half + 32 * cb;
      const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + col0;
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < n) {
        float *cr = C + static_cast<int64_t>(row) * n;
#pragma unroll
        for (int qq = 0; qq < 32; ++qq) {
          const int gj = j0 + col0 + qq;
          if (gj < n) {
            const float a = alpha * __uint_as_float(v[qq]);
            cr[gj] = jb.acc ? cr[gj] + a : a;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem));
}

}  // namespace

size_t tc_gemm_smem() { return 4 * kTcTileBytes + 1024; }
size_t tc_tma_smem() { return static_cast<size_t>(kTcStages) * kTcStageBytes + 1024; }

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(tc_gemm_smem()));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tc_tma_smem()));
}

int tc_pack_ldp(int n) { return (n + kTcK - 1) / kTcK * kTcK; }

// Tensor maps of one job's packed planes (8 per job: product x plane), all
// [n][ldp] FP32 with 32 x 128 boxes and the 128-byte swizzle.
bool tc_encode_maps(void *plane_base, int64_t plane_elems, int slot, int n, void *out8) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int ldp = tc_pack_ldp(n);
  CUtensorMap *m = static_cast<CUtensorMap *>(out8);
  for (int q = 0; q < 2; ++q)
    for (int p = 0; p < 4; ++p) {
      float *pl = static_cast<float *>(plane_base) +
                  ((static_cast<int64_t>(slot) * 2 + q) * 4 + p) * plane_elems;
      const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(ldp), static_cast<cuuint64_t>(n)};
      const cuuint64_t gstr[1] = {static_cast<cuuint64_t>(ldp) * 4};
      const cuuint32_t box[2] = {kTcK, kTcM};
      const cuuint32_t es[2] = {1, 1};
      if (enc(&m[q * 4 + p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl, gdim, gstr, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
          CUDA_SUCCESS)
        return false;
    }
  return true;
}

// one chunk of jobs (<= slots): pack, then the pipelined GEMM
cudaError_t launch_tc_chunk(const GemmJob *jobs, const void *maps, int njobs, int nmax,
                            void *plane_base, int64_t plane_elems, int *status, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  const int ldp = tc_pack_ldp(nmax), t32 = (nmax + 31) / 32 * (ldp / 32);
  k_tc_pack<<<dim3(t32, njobs, 2), 256, 0, st>>>(jobs, static_cast<float *>(plane_base),
                                                 plane_elems);
  const int tiles = (nmax + kTcM - 1) / kTcM;
  k_tc_gemm_tma<<<dim3(tiles * tiles, njobs), 256, tc_tma_smem(), st>>>(
      jobs, static_cast<const CUtensorMap *>(maps), status);
  return cudaGetLastError();
}

__device__ GemmJob g_test_job;

cudaError_t launch_tc_gemm(const GemmJob *jobs, int njobs, int nmax, int *status,
                           cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  const int tiles = (nmax + kTcM - 1) / kTcM;
  k_tc_gemm<<<dim3(tiles * tiles, njobs), 256, tc_gemm_smem(), st>>>(jobs, status);
  return cudaGetLastError();
}

}  // namespace mrcm

// test hook (include/mrcm_testing.h)
extern "C" mrcm_status mrcm_test_gemm(int32_t impl, int32_t n, const float *d_a1,
                                      const float *d_b1, const float *d_a2, const float *d_b2,
                                      float *d_c, double alpha, int32_t acc, int32_t *d_status,
                                      void *cuda_stream) {
  using namespace mrcm;
  if (n < 1 || !d_a1 || !d_b1 || !d_c || !d_status || impl < 0 || impl > 2) return MRCM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  GemmJob j{d_a1, d_b1, d_a2, d_b2, d_c, n, acc ? 1 : 0, alpha};
  GemmJob *dj = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void **>(&dj), g_test_job) != cudaSuccess ||
      cudaMemcpyAsync(dj, &j, sizeof j, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MRCM_ECUDA;
  cudaError_t e;
  if (impl == 2) {
    // scratch planes and maps for one job (allocated per call: a test hook)
    const int64_t pe = static_cast<int64_t>(n) * tc_pack_ldp(n);
    void *planes = nullptr, *dmaps = nullptr;
    CUtensorMap hm[8];
    if ((e = init_tc_attributes()) != cudaSuccess ||
        cudaMalloc(&planes, sizeof(float) * pe * 8) != cudaSuccess ||
        cudaMalloc(&dmaps, sizeof hm) != cudaSuccess)
      return MRCM_ECUDA;
    bool okm = tc_encode_maps(planes, pe, 0, n, hm);
    if (okm && cudaMemcpyAsync(dmaps, hm, sizeof hm, cudaMemcpyHostToDevice, st) == cudaSuccess)
      e = launch_tc_chunk(dj, dmaps, 1, n, planes, pe, d_status, st);
    else
      e = cudaErrorInvalidValue;
    cudaStreamSynchronize(st);
    cudaFree(planes);
    cudaFree(dmaps);
  } else if (impl == 1) {
    if ((e = init_tc_attributes()) != cudaSuccess) return MRCM_ECUDA;
    e = launch_tc_gemm(dj, 1, n, d_status, st);
  } else {
    e = launch_simt_gemm(dj, 1, n, st);
  }
  if (e != cudaSuccess) return MRCM_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MRCM_OK : MRCM_ECUDA;
}

extern "C" mrcm_status mrcm_test_wait_timeout(uint32_t limit, int32_t *d_status,
                                              void *cuda_stream) {
  using namespace mrcm;
  if (!d_status || limit < 1 || limit > kTcWaitLimit) return MRCM_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_wait_probe<<<1, 32, 0, st>>>(d_status, limit);
  if (cudaGetLastError() != cudaSuccess) return MRCM_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? MRCM_OK : MRCM_ECUDA;
}
