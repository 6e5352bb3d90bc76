// Floating-point format conversions done on the integer pipes (GB300 issues FP64
// arithmetic, conversions included, at a small fraction of its FP32 and integer rates).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gw {

// From the IEEE bit fields: float -> double is exact; double -> float rounds to nearest
// even.  Subnormal inputs and results are flushed to zero.
__device__ __forceinline__ double f2d(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t E = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  if (E == 0) return __longlong_as_double((long long)sign);
  const unsigned long long Ed = E == 0xFFu ? 0x7FFull : (unsigned long long)(E + 896u);  // rebias 127 -> 1023
  return __longlong_as_double((long long)(sign | (Ed << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ float d2f(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(u >> 63) << 31;
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (uint32_t)((u & 0xFFFFFFFFFFFFFull) != 0));
  const int Ef = E - 896;  // rebias 1023 -> 127
  if (Ef <= 0) return __uint_as_float(sign);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  // round the 52-bit fraction to 23 bits, ties to even; a carry out bumps the exponent
  const unsigned long long up = ((m >> 28) & 1ull) & (((m & 0xFFFFFFFull) != 0) | ((m >> 29) & 1ull));
  uint32_t bits = ((uint32_t)Ef << 23) + (uint32_t)((m >> 29) + up);
  if (bits >= 0x7F800000u) bits = 0x7F800000u;
  return __uint_as_float(sign | bits);
}

}  // namespace gw
