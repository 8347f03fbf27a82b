// Batched n x n GEMM on the 5th-generation tensor cores (tcgen05) with
// FP32-level accuracy: every FP32 operand is split into a TF32 head and a
// TF32 tail (x = hi + lo, hi = x rounded to TF32), and
//   A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi
// is accumulated in FP32 in tensor memory (the dropped A_lo B_lo term is
// 2^-22 relative).  Used by the large-slab interface factor (the same job
// descriptors as the SIMT kernel).
//
// Simple form (k_tc_gemm, the test hook's reference for the pipelined one):
// one 128 x 128 output tile per CTA, 256 threads.  K advances in chunks of
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
#include <cstring>
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
// Pipelined form on the raw FP32 matrices (row strides a multiple of 16
// bytes), in two rings.  Raw ring (3 x 32 KB): per 32-wide K chunk one thread
// issues two TMA copies (cp.async.bulk.tensor), the 128 x 32 chunk of A in
// the 128-byte-swizzled K-major layout the MMA reads and the 32 x 128
// row-major chunk of B.  Four splitter warps read a raw stage into registers
// and release it at once (the copies run up to three chunks ahead, whatever
// the MMAs are doing), then write the TF32 head and tail tiles into the
// split ring (2 x 64 KB): A at the same offsets, B transposed to K-major
// (16-byte stores, conflict-free under the swizzle).  One thread issues the
// MMAs of a split stage and commits it back to the splitters.  Every
// mbarrier wait is bounded.
constexpr int kTsRaw = 3, kTsSplit = 2;
constexpr int kTsRawBytes = 2 * kTcTileBytes;         // A (swizzled), B (row-major)
constexpr int kTsSplitBytes = 4 * kTcTileBytes;       // A_hi A_lo B_hi B_lo
constexpr int kTsSplitters = 128;                      // warps 4..7

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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

__global__ void __launch_bounds__(256) k_tc_gemm_split(const GemmJob *jobs,
                                                       const CUtensorMap *maps, int *status) {
  extern __shared__ __align__(1024) unsigned char tcsm[];
  __shared__ uint64_t rfull[kTsRaw], rempty[kTsRaw], hfull[kTsSplit], hempty[kTsSplit], done;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const uint32_t raw = smem_u32(tcsm);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char *sm = tcsm + (base - raw);
  const uint32_t hbase = base + kTsRaw * kTsRawBytes;     // split ring after the raw ring
  unsigned char *hsm = sm + kTsRaw * kTsRawBytes;

  const GemmJob jb = jobs[blockIdx.y];
  const CUtensorMap *mp = maps + static_cast<int64_t>(blockIdx.y) * 4;
  const int n = jb.n;
  const int nt = (n + kTcM - 1) / kTcM;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  if (ti >= nt) return;                       // whole CTA, before any barrier
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
    for (int s = 0; s < kTsRaw; ++s) {
      mbar_init(smem_u32(&rfull[s]), 1);
      mbar_init(smem_u32(&rempty[s]), kTsSplitters);
    }
    for (int s = 0; s < kTsSplit; ++s) {
      mbar_init(smem_u32(&hfull[s]), kTsSplitters);
      mbar_init(smem_u32(&hempty[s]), 1);
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
    // producer: raw chunks of A and B into the raw ring
    for (int step = 0; step < total; ++step) {
      const int s = step % kTsRaw;
      if (step >= kTsRaw && !mbar_wait(smem_u32(&rempty[s]), ((step / kTsRaw) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      const int q = first + step / nk, k0 = (step % nk) * kTcK;
      const uint32_t st = base + s * kTsRawBytes, fb = smem_u32(&rfull[s]);
      mbar_expect_tx(fb, kTsRawBytes);
      tma_load_2d(st, mp + 2 * q, k0, i0, fb);
      tma_load_2d(st + kTcTileBytes, mp + 2 * q + 1, j0, k0, fb);
    }
  } else if (t == 32) {
    // MMA issuer
    const uint32_t idesc = idesc_tf32();
    for (int step = 0; step < total; ++step) {
      const int h = step % kTsSplit;
      if (!mbar_wait(smem_u32(&hfull[h]), (step / kTsSplit) & 1)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t st = hbase + h * kTsSplitBytes;
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
      tc_commit(smem_u32(&hempty[h]));
    }
    tc_commit(smem_u32(&done));
  } else if (warp >= 4) {
    // splitters: raw stage -> registers (then released) -> head and tail tiles
    const int u = t - 128;
    for (int step = 0; step < total; ++step) {
      const int s = step % kTsRaw, h = step % kTsSplit;
      if (!mbar_wait(smem_u32(&rfull[s]), (step / kTsRaw) & 1)) {
        s_fail = 1;
        break;
      }
      const unsigned char *rs = sm + s * kTsRawBytes;
      float4 av[kTcTileBytes / 16 / kTsSplitters];
#pragma unroll
      for (int q = 0; q < kTcTileBytes / 16 / kTsSplitters; ++q)
        av[q] = reinterpret_cast<const float4 *>(rs)[u + kTsSplitters * q];
      float bv[kTcK];
      const float *braw = reinterpret_cast<const float *>(rs + kTcTileBytes);
#pragma unroll
      for (int k = 0; k < kTcK; ++k) bv[k] = braw[k * kTcN + u];
      mbar_arrive(smem_u32(&rempty[s]));
      if (step >= kTsSplit && !mbar_wait(smem_u32(&hempty[h]), ((step / kTsSplit) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      unsigned char *hs = hsm + h * kTsSplitBytes;
#pragma unroll
      for (int q = 0; q < kTcTileBytes / 16 / kTsSplitters; ++q) {
        const float4 v = av[q];
        const float4 hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z),
                                      tf32_round(v.w));
        const int e = u + kTsSplitters * q;
        reinterpret_cast<float4 *>(hs)[e] = hi;
        reinterpret_cast<float4 *>(hs + kTcTileBytes)[e] =
            make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
      }
#pragma unroll
      for (int c = 0; c < kTcK / 4; ++c) {
        const float4 v = make_float4(bv[4 * c], bv[4 * c + 1], bv[4 * c + 2], bv[4 * c + 3]);
        const float4 hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z),
                                      tf32_round(v.w));
        const uint32_t o = sw128(u, 4 * c);
        *reinterpret_cast<float4 *>(hs + 2 * kTcTileBytes + o) = hi;
        *reinterpret_cast<float4 *>(hs + 3 * kTcTileBytes + o) =
            make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&hfull[h]));
    }
  }
  __syncwarp();
  bool ok = mbar_wait(smem_u32(&done), 0);
  __syncthreads();
  ok = ok && !s_fail;
  asm volatile("tcgen05.fence::after_thread_sync;");
  float *C = static_cast<float *>(jb.c);
  if (!ok) {
    if (t == 0) atomicOr(status, MRCM_FLAG_TIMEOUT);
    mbar_wait(smem_u32(&done), 0);
  } else if (total > 0) {
    // epilogue: warp w holds output rows 32 (w % 4) .. + 31 (its TMEM lane
    // quarter), columns 64 (w / 4) .. + 63 in two 32-column blocks; each
    // block goes through a padded 32 x 33 shared buffer (the split ring is
    // idle now), so that every global load and store covers a 128-byte row
    // segment instead of one word in each of 32 rows
    const int quarter = warp & 3, half = warp >> 2;
    const float alpha = static_cast<float>(jb.alpha);
    float *buf = reinterpret_cast<float *>(hsm) + warp * 32 * 33;
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
#pragma unroll
      for (int qq = 0; qq < 32; ++qq) buf[lane * 33 + qq] = __uint_as_float(v[qq]);
      __syncwarp();
      const int gj = j0 + col0 + lane;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int gi = i0 + 32 * quarter + r;
        if (gi < n && gj < n) {
          float *cp = C + static_cast<int64_t>(gi) * n + gj;
          const float a = alpha * buf[r * 33 + lane];
          *cp = jb.acc ? *cp + a : a;
        }
      }
      __syncwarp();
    }
  } else if (!jb.acc) {
    // no product: C = 0 (unchanged when accumulating)
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

}  // namespace

size_t tc_gemm_smem() { return 4 * kTcTileBytes + 1024; }
size_t tc_split_smem() {
  return static_cast<size_t>(kTsRaw) * kTsRawBytes + static_cast<size_t>(kTsSplit) * kTsSplitBytes +
         1024;
}

cudaError_t init_tc_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(tc_gemm_smem()));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_tc_gemm_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(tc_split_smem()));
}

// Tensor maps of one job's raw operands (4 per job: A1, B1, A2, B2; zero
// for an absent product): n x n FP32 row-major.  A: 32 x 128 boxes (K, row)
// with the 128-byte swizzle; B: 128 x 32 boxes (column, K), no swizzle.
// False when the encoder refuses (e.g. a row stride that is not a multiple
// of 16 bytes) or is unavailable.
bool tc_encode_raw_maps(const GemmJob &jb, void *out4) {
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
  if (jb.n % 4 != 0) return false;
  CUtensorMap *m = static_cast<CUtensorMap *>(out4);
  const cuuint64_t gdim[2] = {static_cast<cuuint64_t>(jb.n), static_cast<cuuint64_t>(jb.n)};
  const cuuint64_t gstr[1] = {static_cast<cuuint64_t>(jb.n) * 4};
  const cuuint32_t es[2] = {1, 1};
  const void *ops[4] = {jb.a1, jb.b1, jb.a2, jb.b2};
  for (int k = 0; k < 4; ++k) {
    if (!ops[k]) continue;
    const bool isA = (k % 2) == 0;
    const cuuint32_t box[2] = {isA ? static_cast<cuuint32_t>(kTcK) : static_cast<cuuint32_t>(kTcN),
                               isA ? static_cast<cuuint32_t>(kTcM) : static_cast<cuuint32_t>(kTcK)};
    if (enc(&m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ops[k]), gdim, gstr, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            isA ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// all jobs of a set in one launch: (output tiles of the largest job, jobs)
cudaError_t launch_tc_split(const GemmJob *jobs, const void *maps, int njobs, int nmax,
                            int *status, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  const int tiles = (nmax + kTcM - 1) / kTcM;
  k_tc_gemm_split<<<dim3(tiles * tiles, njobs), 256, tc_split_smem(), st>>>(
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
    // tensor maps of the caller's matrices (n a multiple of 4)
    void *dmaps = nullptr;
    CUtensorMap hm[4];
    memset(hm, 0, sizeof hm);
    if (n % 4 != 0) return MRCM_EINVAL;
    if ((e = init_tc_attributes()) != cudaSuccess || cudaMalloc(&dmaps, sizeof hm) != cudaSuccess)
      return MRCM_ECUDA;
    if (tc_encode_raw_maps(j, hm) &&
        cudaMemcpyAsync(dmaps, hm, sizeof hm, cudaMemcpyHostToDevice, st) == cudaSuccess)
      e = launch_tc_split(dj, dmaps, 1, n, d_status, st);
    else
      e = cudaErrorInvalidValue;
    cudaStreamSynchronize(st);
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
