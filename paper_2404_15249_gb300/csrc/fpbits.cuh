// Exact conversions between FP64 and FP32 values by integer operations on their bit
// patterns.  On this GPU every FP64 operation, conversions included, runs on the FP64
// pipe at a small fraction of the FP32 rate, which bounds the kernels that only convert
// grids between the two formats; these helpers keep normal numbers on the integer pipe and
// fall back to the hardware conversion for zero, subnormals, infinities, NaN and values
// outside the FP32 exponent range, where they give the same results.
#pragma once
#include <cstdint>
#include <cstring>

#ifndef __CUDACC__                 // plain C++ (the host-side test of these conversions)
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace kfbi {

__host__ __device__ __forceinline__ uint64_t fpb_bits(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}
__host__ __device__ __forceinline__ double fpb_double(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ uint32_t fpb_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float fpb_float(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

// (double)f, exact: a normal FP32 value's exponent is rebiased (127 -> 1023) and its 23
// fraction bits move to the top of the 52; anything else takes the hardware conversion
__host__ __device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = fpb_bits(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const uint64_t s = (uint64_t)(u >> 31) << 63;
  return fpb_double(s | ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)(u & 0x7fffffu) << 29));
}

// (hi, lo) with hi = (float)v (round to nearest, ties to even) and lo = (float)(v - hi), the
// FP32 pair that carries v to about 48 bits.  For v whose hi and lo are both normal FP32
// numbers: hi by rounding the 52-bit fraction to 23 bits on the integer pattern (a carry
// out of the fraction moves into the exponent, as it should); v - hi is exact in FP64
// (at most half an FP32 unit of v), so it is the integer remainder of the significand at
// v's exponent, converted to FP32 by the integer-to-float conversion and scaled by a power
// of two.  Otherwise the hardware conversions give the pair.
__host__ __device__ __forceinline__ void f64_to_f32_pair(double v, float& hi, float& lo) {
  const uint64_t u = fpb_bits(v);
  if ((u << 1) == 0ull) {                                // +-0: (+-0, +0)
    hi = fpb_float((uint32_t)(u >> 32) & 0x80000000u);
    lo = 0.f;
    return;
  }
  const int e = (int)((u >> 52) & 0x7ffu);               // biased FP64 exponent
  // hi normal needs 1023 - 126 <= e <= 1023 + 127 (allowing for a rounding carry), and the
  // remainder's scale 2^(e - 1075) must keep lo normal: e - 1075 >= -126 + ... (checked as
  // e >= 1023 - 126 + 29 + 24 so that any nonzero remainder is a normal FP32 value)
  if (e < 1023 - 126 + 53 || e > 1023 + 126) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
    return;
  }
  const uint64_t mag = u & 0x7fffffffffffffffull;
  // rounding to nearest even at bit 29 of the pattern (exponent and fraction together)
  const uint64_t half = (1ull << 28) - 1ull + ((mag >> 29) & 1ull);
  const uint64_t r = (mag + half) >> 29;                 // the FP64 pattern >> 29, rounded
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  // rebias: the top 11 exponent bits of r hold e (or e + 1 after a carry); FP32 exponent
  // = that - 1023 + 127
  const uint32_t fpat = (uint32_t)(r - ((uint64_t)(1023 - 127) << 23));
  hi = fpb_float(sign | fpat);
  // remainder: significand of v minus hi's significand scaled to v's exponent (both with
  // the hidden bit), in units of 2^(e - 1075)
  const int64_t sig_v = (int64_t)((mag & 0xfffffffffffffull) | (1ull << 52));
  const int ehi = (int)(r >> 23);                        // e or e + 1
  const int64_t sig_hi = (int64_t)(((r & 0x7fffffull) | (1ull << 23)) << 29) << (ehi - e);
  int64_t rem = sig_v - sig_hi;                          // |rem| <= 2^28
  if (u >> 63) rem = -rem;                               // v - hi for negative v (+0 if equal)
  // lo = rem * 2^(e - 1075), rem exact in FP32 when |rem| < 2^24, else rounded once
  const float remf = (float)(int32_t)rem;
  const int sc = e - 1075 + 127;                         // FP32 biased exponent of 2^(e-1075)
  lo = remf * fpb_float((uint32_t)sc << 23);
}

}  // namespace kfbi
