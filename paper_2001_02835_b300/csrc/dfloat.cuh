// Double-float ("double-word") arithmetic on FP32 pairs for the transforms of
// the split form.  A value is hi + lo with |lo| <= ulp(hi)/2 (about 48
// significant bits).  Sums use Knuth's TwoSum and Dekker's FastTwoSum,
// products the FMA residual a*b - fl(a*b); see Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017).  Conversions to and from FP64 work on the bit
// patterns with integer operations, because the FP64 pipe of B300 runs at
// about 1/58 of the FP32 rate.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct dfl {
  float h, l;
};
struct cdf {
  dfl re, im;
};

// The steps whose rounding the error-free transformations rely on are written
// with __fadd_rn / __fsub_rn / __fmul_rn, which the compiler never contracts
// into an FMA: TwoSum needs s = fl(a + b) exactly, and the FMA residual of a
// product needs p = fl(a * b), whatever the surrounding expressions are.
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dfl df_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfl{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  df_two_sum(a.h, b.h, s, e);
  e += a.l + b.l;
  return df_fast(s, e);
}
__device__ __forceinline__ dfl df_neg(dfl a) { return dfl{-a.h, -a.l}; }
__device__ __forceinline__ dfl df_sub(dfl a, dfl b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ dfl df_scale(dfl a, float p2) { return dfl{a.h * p2, a.l * p2}; }

__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return cdf{df_add(a.re, b.re), df_add(a.im, b.im)}; }

// Sum whose result is only fed to another df_add: the exact TwoSum of the high
// parts is kept, but the final FastTwoSum renormalisation is skipped (|lo| may
// then exceed ulp(hi)/2 by a few units; the next df_add renormalises).
__device__ __forceinline__ dfl df_add_lazy(dfl a, dfl b) {
  float s, e;
  df_two_sum(a.h, b.h, s, e);
  return dfl{s, e + (a.l + b.l)};
}
__device__ __forceinline__ cdf cdf_add_lazy(cdf a, cdf b) {
  return cdf{df_add_lazy(a.re, b.re), df_add_lazy(a.im, b.im)};
}
__device__ __forceinline__ cdf cdf_sub_lazy(cdf a, cdf b) {
  return cdf{df_add_lazy(a.re, dfl{-b.re.h, -b.re.l}), df_add_lazy(a.im, dfl{-b.im.h, -b.im.l})};
}
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return cdf{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }

// a * w with w = (c, s) given as double-float pairs (a twiddle factor), without
// the final renormalisation: (hi, lo) is the exact sum of the high products
// plus the rounded residuals and cross terms, so |lo| may exceed ulp(hi)/2 when
// the high products cancel.  For results that only feed further sums.
__device__ __forceinline__ cdf cdf_mul_lazy(cdf a, dfl c, dfl s) {
  // re = a.re c - a.im s
  float p1 = __fmul_rn(a.re.h, c.h), e1 = fmaf(a.re.h, c.h, -p1);
  float p2 = __fmul_rn(a.im.h, s.h), e2 = fmaf(a.im.h, s.h, -p2);
  float sr, e3;
  df_two_sum(p1, -p2, sr, e3);
  float lo = (e1 - e2) + e3;
  lo = fmaf(a.re.h, c.l, lo);
  lo = fmaf(a.re.l, c.h, lo);
  lo = fmaf(-a.im.h, s.l, lo);
  lo = fmaf(-a.im.l, s.h, lo);
  // im = a.re s + a.im c
  float q1 = __fmul_rn(a.re.h, s.h), f1 = fmaf(a.re.h, s.h, -q1);
  float q2 = __fmul_rn(a.im.h, c.h), f2 = fmaf(a.im.h, c.h, -q2);
  float si, f3;
  df_two_sum(q1, q2, si, f3);
  float lo2 = (f1 + f2) + f3;
  lo2 = fmaf(a.re.h, s.l, lo2);
  lo2 = fmaf(a.re.l, s.h, lo2);
  lo2 = fmaf(a.im.h, c.l, lo2);
  lo2 = fmaf(a.im.l, c.h, lo2);
  return cdf{dfl{sr, lo}, dfl{si, lo2}};
}
__device__ __forceinline__ cdf cdf_mul(cdf a, dfl c, dfl s) {
  const cdf r = cdf_mul_lazy(a, c, s);
  return cdf{df_fast(r.re.h, r.re.l), df_fast(r.im.h, r.im.l)};
}

// ---- sums on a common grid (inside one radix-4 butterfly of the transforms) ----
// The high parts of a butterfly's inputs are first rounded to one grid u, a power
// of two, and the remainders join the low parts (exact: h = g + (h - g)).  With
// every input below 2^(E+1) in magnitude and u = 2^(E-21), any sum of up to four
// high parts is a multiple of u of at most 2^(E+3) = 2^24 u, so a single FP32
// addition forms it exactly; only the low parts round.  A sum then costs two
// additions instead of the eight to eleven of TwoSum-based double-float.  The
// price is that a value's error is bounded relative to the butterfly's largest
// input (about 2^-45 of it per step) rather than to the value itself.
//
// K = 1.5 * 2^(E+2) is the rounding constant: for |h| < 2^(E+1) = K/3, h + K
// lies in [2^(E+2), 2^(E+3)], whose spacing is u, so fl(h + K) - K is h rounded
// to the grid (the subtraction is exact by Sterbenz's lemma).  amax is the
// largest |hi| of the butterfly's inputs; its exponent field gives E.  Zero or
// subnormal amax gives a grid at the bottom of the FP32 range.
__device__ __forceinline__ float grid_magic(float amax) {
  unsigned ex = (__float_as_uint(amax) & 0x7F800000u) + (2u << 23);
  ex = min(ex, 254u << 23);
  return __uint_as_float(ex | 0x00400000u);
}
__device__ __forceinline__ dfl df_regrid(dfl a, float K) {
  const float g = __fsub_rn(__fadd_rn(a.h, K), K);
  return dfl{g, __fadd_rn(__fsub_rn(a.h, g), a.l)};
}
__device__ __forceinline__ cdf cdf_regrid(cdf a, float K) { return cdf{df_regrid(a.re, K), df_regrid(a.im, K)}; }
__device__ __forceinline__ float cdf_amax(cdf a) { return fmaxf(fabsf(a.re.h), fabsf(a.im.h)); }
// sums of two values on the same grid: the high part is exact, the low part rounds
__device__ __forceinline__ cdf cg_add(cdf a, cdf b) {
  return cdf{dfl{__fadd_rn(a.re.h, b.re.h), __fadd_rn(a.re.l, b.re.l)},
             dfl{__fadd_rn(a.im.h, b.im.h), __fadd_rn(a.im.l, b.im.l)}};
}
__device__ __forceinline__ cdf cg_sub(cdf a, cdf b) {
  return cdf{dfl{__fsub_rn(a.re.h, b.re.h), __fsub_rn(a.re.l, b.re.l)},
             dfl{__fsub_rn(a.im.h, b.im.h), __fsub_rn(a.im.l, b.im.l)}};
}
// multiplication by i and by -i (exact)
__device__ __forceinline__ cdf cdf_mul_i(cdf a) { return cdf{df_neg(a.im), a.re}; }
__device__ __forceinline__ cdf cdf_mul_mi(cdf a) { return cdf{a.im, df_neg(a.re)}; }

// 2^k as a float for -252 <= k <= 254 (two factors keep it exact)
__device__ __forceinline__ void pow2_pair(int k, float& f1, float& f2) {
  const int k1 = k / 2, k2 = k - k1;
  f1 = __int_as_float((max(-126, min(127, k1)) + 127) << 23);
  f2 = __int_as_float((max(-126, min(127, k2)) + 127) << 23);
}

// FP64 -> double-float: hi keeps the top 24 significant bits, lo the next 29
// bits rounded to 24.  Zero and FP64 denormals map to 0.
__device__ __forceinline__ dfl df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return dfl{0.f, 0.f};
  const int fe = e - 1023 + 127;
  if (fe < 1 || fe > 254) {  // outside the FP32 exponent range: saturate through the slow path
    const float h = __double2float_rz(x);
    return dfl{h, 0.f};
  }
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  const float h = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)(m >> 29));
  float f1, f2;
  pow2_pair(e - 1075, f1, f2);
  float l = (float)(unsigned)(m & 0x1FFFFFFFull) * f1 * f2;
  if (sign) l = -l;
  return dfl{h, l};
}

// float -> FP64 by bit assembly, subnormal floats normalised with a leading-zero
// count; integer operations only (no FP64-pipe conversion).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xFF;
  const unsigned m = u & 0x7FFFFF;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  unsigned long long bits;
  if (ef == 0) {
    // m 2^-149 with the leading one at bit p: exponent p - 149, fraction m << (52 - p)
    const int p = 31 - __clz(m | 1u);
    bits = m ? (sign | ((unsigned long long)(p - 149 + 1023) << 52) |
                (((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFull))
             : sign;
  } else if (ef == 255) {
    bits = sign | 0x7FF0000000000000ull | ((unsigned long long)m << 29);
  } else {
    bits = sign | ((unsigned long long)(ef - 127 + 1023) << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}
// normal floats and zeros, the common case: the FP64 word is the float's sign, its exponent
// rebiased (+896 in the 11-bit field) and its fraction shifted up by 29 bits
__device__ __forceinline__ bool f2d_fast_ok(float f) {
  const unsigned a = __float_as_uint(f) & 0x7FFFFFFFu;
  return a == 0u || (a >> 23) - 1u < 254u;
}
__device__ __forceinline__ double f2d_fast(float f) {
  const unsigned u = __float_as_uint(f), a = u & 0x7FFFFFFFu;
  const unsigned hi = (u & 0x80000000u) | (a ? (a >> 3) + (896u << 20) : 0u);
  return __hiloint2double((int)hi, (int)(a << 29));
}
__device__ __forceinline__ double df_to_double(dfl a) {
  // one uniform branch: the whole warp takes the short path unless a subnormal, infinite or
  // NaN part is present
  if (__all_sync(__activemask(), f2d_fast_ok(a.h) && f2d_fast_ok(a.l))) return f2d_fast(a.h) + f2d_fast(a.l);
  return f2d(a.h) + f2d(a.l);
}

// round(x * 2^sh) for x = hi + lo as a signed 64-bit integer (|result| < 2^63)
__device__ __forceinline__ long long f_scaled_int(float f, int sh_base) {
  const unsigned u = __float_as_uint(f);
  const int ef = (int)((u >> 23) & 0xFF);
  if (ef == 0) return 0;
  const long long m = (long long)((u & 0x7FFFFF) | 0x800000);
  const int sh = ef - 150 + sh_base;
  long long v;
  if (sh >= 0) v = m << sh;
  else if (sh > -63) v = (m + (1LL << (-sh - 1))) >> (-sh);
  else v = 0;
  return (u >> 31) ? -v : v;
}
