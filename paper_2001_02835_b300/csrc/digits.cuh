// Digit slicing of the split form: an error-free split of each spectrum value
// into S balanced base-256 digits stored as BF16 (in the spirit of Ozaki et
// al.; see split.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace digits {

// exact int -> float for |d| < 2^22 without a conversion instruction
// (1.5 * 2^23 + d has d in its low mantissa bits)
__device__ __forceinline__ float small_int_to_float(int d) {
  return __int_as_float(0x4B400000 + d) - 12582912.0f;
}

template <int S>
__device__ __forceinline__ void to_digits(double x, int e, float (&s)[S]) {
  constexpr int W = 8 * S - 1;
  const long long bits = __double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (bexp != 0) {
    const unsigned long long mant = ((unsigned long long)bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1075 + e - W - bexp;
    if (sh <= 0) X = mant << (-sh);
    else if (sh < 64) X = (mant + (1ull << (sh - 1))) >> sh;
  }
  const float sign = bits < 0 ? -1.f : 1.f;
#pragma unroll
  for (int i = S - 1; i >= 1; --i) {
    int d = (int)(X & 255ull);
    X >>= 8;
    if (d > 128) { d -= 256; X += 1; }
    s[i] = sign * small_int_to_float(d) * __int_as_float((127 - 8 * i) << 23);
  }
  s[0] = sign * small_int_to_float((int)X);
}

// digits of a double-float value x = hi + lo (|x| < 2^e) in FP32 arithmetic:
// with v = x 2^-e (|v| < 1) and sigma_i = 1.5 * 2^(16 - 8i), t = (v + sigma_i) -
// sigma_i rounds v to the nearest multiple of 2^(-7-8i) exactly, v - t is
// exact, and t * 2^7 = d_i 2^(-8i) is the stored slice value.  Digits 0..2
// come from hi alone (|lo| < 2^-25 lies below their grid); lo joins the
// residual before digit 3, so |d_i| <= 128 for i < 3 and <= 192 after.
template <int S>
__device__ __forceinline__ void to_digits(dfl x, int e, float (&s)[S]) {
  float f1, f2;
  pow2_pair(-e, f1, f2);
  float v = (x.h * f1) * f2;
  const float lo = (x.l * f1) * f2;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    if (i == 3) v = __fadd_rn(v, lo);
    const float sig = __int_as_float(((143 - 8 * i) << 23) | 0x400000);
    const float t = __fsub_rn(__fadd_rn(v, sig), sig);   // rounding to the digit grid
    v = __fsub_rn(v, t);
    s[i] = t * 128.f;
  }
}

// smallest e with |x| < 2^e for every part, from the exponent field
// (a subnormal part has |x| < 2^-1022, resp. 2^-126; only a row of exact zeros gets -100000)
__device__ __forceinline__ int exp_bound(double2 v) {
  const int a = (int)((__double_as_longlong(v.x) >> 52) & 0x7FF), b = (int)((__double_as_longlong(v.y) >> 52) & 0x7FF);
  const int m = max(a, b);
  if (m != 0) return m - 1022;
  return ((__double_as_longlong(v.x) | __double_as_longlong(v.y)) << 1) ? -1022 : -100000;
}
__device__ __forceinline__ int exp_bound(float4 v) {
  // |hi + lo| < 2^(exponent(hi) + 1) since |lo| <= ulp(hi)/2
  const int a = (int)((__float_as_uint(v.x) >> 23) & 0xFF), b = (int)((__float_as_uint(v.z) >> 23) & 0xFF);
  const int m = max(a, b);
  if (m != 0) return m - 126;
  return ((__float_as_uint(v.x) | __float_as_uint(v.z)) << 1) ? -126 : -100000;
}
__device__ __forceinline__ double2 conj_of(double2 v) { return make_double2(v.x, -v.y); }
__device__ __forceinline__ float4 conj_of(float4 v) { return make_float4(v.x, v.y, -v.z, -v.w); }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float4 zero_of(float4) { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <int S>
__device__ __forceinline__ void digits_re_im(double2 v, int e, float (&re)[S], float (&im)[S]) {
  to_digits<S>(v.x, e, re);
  to_digits<S>(v.y, e, im);
}
template <int S>
__device__ __forceinline__ void digits_re_im(float4 v, int e, float (&re)[S], float (&im)[S]) {
  to_digits<S>(dfl{v.x, v.y}, e, re);
  to_digits<S>(dfl{v.z, v.w}, e, im);
}

}  // namespace digits
