// Digits of the exact-integer split products (oz_gemm.cuh, oz_deriv.cu):
// each value x of a row with exponent E (|x| < 2^E over the row) is rounded to
// the integer X = round(|x| 2^{8S - E}) and written as balanced base-256
// digits alpha_0 in [0, 256], alpha_s in [-128, 127] (s >= 1), then given the
// sign of x, so |alpha_s| <= 128 and every digit is exact in bf16.  Integer
// work on the bit patterns only (FP64 arithmetic runs at 1/64 of the FP32
// rate on this chip).
#pragma once

#include <climits>

#include "sky_internal.cuh"

namespace sky {
namespace ozdig {

__device__ __forceinline__ int exp_of(double x) {   // e with |x| < 2^e, INT_MIN for 0
  const int ef = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return ef == 0 ? INT_MIN : ef - 1022;
}
__device__ __forceinline__ int exp_of(float x) {
  const int ef = (int)((__float_as_uint(x) >> 23) & 0xFF);
  return ef == 0 ? INT_MIN : ef - 126;
}

// |x| 2^{8S - E} rounded to an integer (denormals and zero give 0).
template <int S>
__device__ __forceinline__ unsigned long long fixed_of(double x, int E) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7FF);
  if (ef == 0) return 0ull;
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = ef - 1075 + 8 * S - E;
  if (sh >= 0) return sh < 11 ? mant << sh : 0ull;   // |x| < 2^E keeps sh < 0 for S <= 6
  const int r = -sh;
  if (r >= 64) return 0ull;
  return (mant + (1ull << (r - 1))) >> r;
}
template <int S>
__device__ __forceinline__ unsigned long long fixed_of(float x, int E) {
  const unsigned bits = __float_as_uint(x);
  const int ef = (int)((bits >> 23) & 0xFF);
  if (ef == 0) return 0ull;
  const unsigned long long mant = (bits & 0x7FFFFFu) | 0x800000u;
  const int sh = ef - 150 + 8 * S - E;
  if (sh >= 0) return sh < 40 ? mant << sh : 0ull;
  const int r = -sh;
  if (r >= 64) return 0ull;
  return (mant + (1ull << (r - 1))) >> r;
}
__device__ __forceinline__ bool sign_of(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool sign_of(float x) { return (int)__float_as_uint(x) < 0; }

// Balanced base-256 digits of x relative to 2^E, as bf16 bit patterns.
__device__ __forceinline__ unsigned short bf16_of_int(int d) {   // |d| <= 256: exact
  const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}
template <int S, typename R>
__device__ __forceinline__ void digits(R x, int E, unsigned short* out) {
  long long X = (long long)fixed_of<S>(x, E);
  const bool neg = sign_of(x);
  int d[S];
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    int v = (int)(X & 255);
    X >>= 8;
    if (v >= 128) { v -= 256; ++X; }
    d[s] = v;
  }
  d[0] = (int)X;
#pragma unroll
  for (int s = 0; s < S; ++s) out[s] = bf16_of_int(neg ? -d[s] : d[s]);
}
__device__ __forceinline__ unsigned short neg_bf16(unsigned short h) { return h ^ 0x8000u; }
__device__ __forceinline__ unsigned pack2(unsigned short lo, unsigned short hi) {
  return (unsigned)lo | ((unsigned)hi << 16);
}

}  // namespace ozdig
}  // namespace sky
