// Conversions between binary32 and binary64 on the integer pipe.
//
// On GB300 the hardware conversions between float and double issue on the
// FP64 pipe, at about the DFMA rate (1.9 per clock per SM measured, against
// 1.6 for DFMA).  The FP32 refinement loops of the local solves convert twice
// per cell, column and sweep (the FP64 residual to FP32 for the block solve,
// the FP32 correction to FP64 for the iterate), next to the residual's five
// DFMA and the iterate's DADD, and that pipe bounds them.  These helpers form
// the same results from the IEEE 754 binary32 and binary64 encodings (sign,
// biased exponent, trailing significand; round to nearest, ties to even) with
// integer operations, which leave the FP64 pipe to the arithmetic.  They give
// bit for bit the hardware conversions' results for every finite input and
// for infinities; a NaN gives a NaN.
#pragma once

#include <cstdint>

namespace mrcm {

// binary32 -> binary64 (exact)
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned hi, lo;
  if (e - 1u < 254u) {                 // normal: rebias 127 -> 1023
    hi = s | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  } else if (e == 0xffu) {             // infinity (m = 0) or NaN (m != 0)
    hi = s | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else if (m == 0u) {                // signed zero
    hi = s;
    lo = 0u;
  } else {                             // subnormal m 2^-149 = 1.f 2^(p-149)
    const int p = 31 - __clz(m);
    const uint64_t fr = (static_cast<uint64_t>(m) << (52 - p)) & 0xfffffffffffffull;
    const uint64_t b = (static_cast<uint64_t>(s) << 32) |
                       (static_cast<uint64_t>(p + 874) << 52) | fr;
    return __longlong_as_double(static_cast<long long>(b));
  }
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// binary64 -> binary32, round to nearest, ties to even
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(d));
  const unsigned lo = static_cast<unsigned>(__double2loint(d));
  const unsigned s = hi & 0x80000000u, e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {               // result exponent 1..254 before rounding
    // 23 kept significand bits, 29 dropped; a carry out of the significand
    // moves into the exponent (up to infinity), as rounding requires
    unsigned m = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rb = lo & 0x1fffffffu;
    m += (rb > 0x10000000u || (rb == 0x10000000u && (m & 1u))) ? 1u : 0u;
    return __uint_as_float(s | m);
  }
  if (e == 0x7ffu) return __uint_as_float(((hi & 0xfffffu) | lo) ? 0x7fffffffu : (s | 0x7f800000u));
  if (e > 1150u) return __uint_as_float(s | 0x7f800000u);   // beyond the float range
  // subnormal or zero result: |d| 2^149 rounded to an integer, ties to even
  const int sh = 926 - static_cast<int>(e);                  // >= 30
  if (sh >= 54) return __uint_as_float(s);                    // below half the least subnormal
  const uint64_t m53 = (static_cast<uint64_t>((hi & 0xfffffu) | 0x100000u) << 32) | lo;
  uint64_t q = m53 >> sh;
  const uint64_t rem = m53 & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(s | static_cast<unsigned>(q));
}

}  // namespace mrcm
