// FP64 <-> FP32 conversions on the integer pipe.
//
// On this GPU the FP64 pipe retires about one warp instruction per 16 SM
// cycles, and a cvt between FP64 and FP32 occupies it like an add.  The
// refinement's streaming kernels (residual, solution update) are bound by
// that pipe, so their conversions are done here with integer operations on
// the IEEE-754 bit fields instead:
//
//   binary64: sign | 11-bit exponent (bias 1023) | 52-bit fraction
//   binary32: sign |  8-bit exponent (bias  127) | 23-bit fraction
//
// A normal number keeps its sign and fraction; the exponent is re-biased by
// 1023 - 127 = 896 and the fraction is cut to (or padded from) 23 bits.

#pragma once
#include <stdint.h>

namespace bt {

// FP64 -> FP32, rounded toward zero (relative error below 2^-23).  Values
// below FP32's normal range become signed zero; values above it, infinities
// and NaNs become a signed infinity.
__device__ __forceinline__ float f64_to_f32_rz(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v);
  const uint32_t lo = (uint32_t)__double2loint(v);
  const uint32_t a = hi & 0x7fffffffu;  // exponent and top 20 fraction bits
  // (a:lo) << 3 keeps the exponent's low 9 bits above 23 fraction bits; the
  // re-bias wraps correctly modulo 2^32 for exponents 897..1150.
  uint32_t f = __funnelshift_l(lo, a, 3) - (896u << 23);
  f = a < (897u << 20) ? 0u : f;
  f = a >= (1151u << 20) ? 0x7f800000u : f;
  return __uint_as_float(f | (hi & 0x80000000u));
}

// FP32 -> FP64, exact for zero, normal numbers, infinities and NaNs.
// Subnormal inputs (below 1.2e-38 in magnitude) become signed zero.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + (896u << 20);
  uint32_t lo = a << 29;
  if (a < 0x00800000u) {
    hi = 0u;
    lo = 0u;
  } else if (a >= 0x7f800000u) {
    hi = 0x7ff00000u | ((a >> 3) & 0x000fffffu);
  }
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

}  // namespace bt
