// Exact base-2^7 digits of FP64 / FP32 values for products on the BF16 tensor cores
// (an Ozaki-type splitting): after a power-of-two scaling, every value is a sum of
// signed digits d_s 2^-7(s+1) that BF16 holds exactly, so the products of two digits
// are exact and sums of them are exact while they stay within 2^24 of their unit.
// Integer arithmetic on the bit fields only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

namespace gw {

__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
__device__ __forceinline__ int exp_field(float x) { return (int)((__float_as_uint(x) >> 23) & 0xFF); }

// round(x 2^(56 - e)) for |x| < 2^e as a 64-bit integer, from the bits of x: the
// significand shifted by its exponent relative to 2^(e - 56), rounded half up when
// shifted right.  |result| < 2^56; subnormal x gives 0.
__device__ __forceinline__ long long shift_round(long long m, int sh) {
  if (sh >= 0) return m << sh;
  if (sh > -63) return (m + (1ll << (-sh - 1))) >> (-sh);
  return 0;
}
__device__ __forceinline__ long long fixed56(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long r = shift_round((long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull), E - 1019 - e);  // <= 3
  return (u >> 63) ? -r : r;
}
__device__ __forceinline__ long long fixed56(float x, int e) {
  const uint32_t u = __float_as_uint(x);
  const int E = (int)((u >> 23) & 0xFF);
  if (E == 0) return 0;
  const long long r = shift_round((long long)((u & 0x7FFFFFu) | 0x800000u), E - 94 - e);  // <= 32
  return (u >> 31) ? -r : r;
}

// Signed base-2^7 digits of one scaled entry: m = round(v 2^56) for |v| < 1, then
// digit s = round(m / 2^(49 - 7 s)) taken from the top, so that v = sum_s d_s 2^-7(s+1)
// up to 2^-57 with |d_0| <= 128 and |d_s| <= 64 after it; every d_s 2^-7(s+1) is exact
// in BF16 (at most 8 significant bits).
__device__ __forceinline__ int next_digit(long long& m, int s) {
  const int sh = 49 - 7 * s;
  const long long d = sh > 0 ? (m + (1ll << (sh - 1))) >> sh : m;
  m -= d << sh;
  return (int)d;
}
// bits of d 2^-7(s+1) in BF16 (exact)
__device__ __forceinline__ uint32_t digit_bf16(int d, int s) {
  const float sc = __int_as_float((127 - 7 * (s + 1)) << 23);
  return __float_as_uint((float)d * sc) >> 16;
}


// -x by flipping the sign bit (an integer operation: negating a double is an FP64
// instruction, which this chip issues at a small fraction of its other rates).
__device__ __forceinline__ double dneg(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// S 2^e as a double for a 64-bit integer S, from the bit fields: normalise, round the
// 64-bit magnitude to 53 bits (ties to even), add e to the exponent.  |e| and |S| keep
// the result a normal double in every use here.
__device__ __forceinline__ double i2d_scaled(long long S, int e) {
  if (S == 0) return 0.0;
  const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
  unsigned long long m = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll((long long)m);
  m <<= lz;                     // leading one at bit 63
  int ex = 63 - lz + e;         // value = 1.xxx 2^ex
  const unsigned long long rest = m & 0x7FFull;  // the 11 bits below the 53 kept
  unsigned long long mant = m >> 11;             // 53 bits with the leading one
  if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) ++mant;
  if (mant >> 53) { mant >>= 1; ++ex; }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(ex + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// Host forms of exp_field and fixed56 with the device's rules (scale exponent from the
// exponent field, rounding half up at 2^-56 of the scale).
inline int host_exp_field(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return (int)((u >> 52) & 0x7FF);
}
inline long long host_fixed56(double x, int e) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = E - 1019 - e;
  long long r = sh >= 0 ? (m << sh) : (sh > -63 ? (m + (1ll << (-sh - 1))) >> (-sh) : 0);
  return (u >> 63) ? -r : r;
}
}  // namespace gw
