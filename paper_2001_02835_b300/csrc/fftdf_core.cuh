// Shared pieces of the double-float order transforms (split form, Sec. 2
// FFT-CONV Steps 2 and 4): twiddles, bit reversal, float4 <-> complex
// double-float, and the forward transform of a strip of entries in shared
// memory.
//
// The radix-2^2 butterflies form their sums on a common grid (dfloat.cuh):
// the inputs' high parts are rounded to the grid of the butterfly's largest
// input, after which every sum of high parts is one exact FP32 addition.  The
// last step of a transform uses TwoSum-based double-float sums instead, so
// that its outputs are normalised (|lo| <= ulp(hi)/2), as the slicer expects.
// The stages are unrolled at compile time: the span, the twiddle step and,
// where a thread meets one twiddle set per stage, the twiddles themselves are
// fixed before the stage's loop, and a twiddle equal to +-i is applied as a
// swap of real and imaginary parts.
#pragma once
#include "dfloat.cuh"
#include "fft_twiddle.cuh"

namespace fftdf {

__device__ __forceinline__ void tw(int n, int M, bool inverse, dfl& c, dfl& s) {
  const float4 t = c_twiddle_f4[n * (NSPT_FFT_MAX_LEN / M)];
  c = dfl{t.x, t.y};
  s = inverse ? dfl{-t.z, -t.w} : dfl{t.z, t.w};
}

template <int M>
__device__ __forceinline__ int bitrev(int i) {
  constexpr int LOG = (M <= 1) ? 0 : (31 - __builtin_clz(M));
  return (int)(__brev((unsigned)i) >> (32 - LOG));
}

__device__ __forceinline__ cdf ld(const float4* p) {
  const float4 v = *p;
  return cdf{dfl{v.x, v.y}, dfl{v.z, v.w}};
}
__device__ __forceinline__ void st(float4* p, cdf a) { *p = make_float4(a.re.h, a.re.l, a.im.h, a.im.l); }

template <int X>
constexpr int ilog2() { return X <= 1 ? 0 : 1 + ilog2<X / 2>(); }

// The three twiddles of one radix-4 butterfly: w^(2j), w^j, w^(3j) (forward) or
// their conjugates (inverse), with j = n * step; mul_i: w^(2j) is i (or -i).
template <int M, bool INV>
struct Tw3 {
  dfl c2, s2, c1, s1, c3, s3;
  bool any, mul_i;
  __device__ __forceinline__ void load(int j) {
    any = j != 0;
    mul_i = 2 * j == M / 4;
    if (any) {
      if (!mul_i) tw(2 * j, M, INV, c2, s2);
      tw(j, M, INV, c1, s1);
      tw(3 * j, M, INV, c3, s3);
    }
  }
  // a *= w^(2j), b *= w^j, c *= w^(3j)
  __device__ __forceinline__ void apply(cdf& a, cdf& b, cdf& c) const {
    if (!any) return;
    a = mul_i ? (INV ? cdf_mul_mi(a) : cdf_mul_i(a)) : cdf_mul_lazy(a, c2, s2);
    b = cdf_mul_lazy(b, c1, s1);
    c = cdf_mul_lazy(c, c3, s3);
  }
};

__device__ __forceinline__ float cdf_amax4(cdf a, cdf b, cdf c, cdf d) {
  return fmaxf(fmaxf(cdf_amax(a), cdf_amax(b)), fmaxf(cdf_amax(c), cdf_amax(d)));
}

// DIF radix-2^2 butterfly of rows (p, p+q, p+2q, p+3q), sums on a common grid,
// before the step's twiddles: x0 <- (x0 + x2) + (x1 + x3), x1 <- (x0 + x2) - (x1 + x3),
// x2 <- (x0 - x2) + i (x1 - x3), x3 <- (x0 - x2) - i (x1 - x3).
__device__ __forceinline__ void dif4_grid(cdf& x0, cdf& x1, cdf& x2, cdf& x3) {
  const float K = grid_magic(cdf_amax4(x0, x1, x2, x3));
  x0 = cdf_regrid(x0, K); x1 = cdf_regrid(x1, K); x2 = cdf_regrid(x2, K); x3 = cdf_regrid(x3, K);
  const cdf s0 = cg_add(x0, x2), s1 = cg_add(x1, x3), d0 = cg_sub(x0, x2), d1 = cg_sub(x1, x3);
  const cdf id1 = cdf_mul_i(d1);
  x0 = cg_add(s0, s1); x1 = cg_sub(s0, s1); x2 = cg_add(d0, id1); x3 = cg_sub(d0, id1);
}

// The same butterfly with x2 = x3 = 0 (first step of the zero-padded input).
__device__ __forceinline__ void dif4_pruned_grid(cdf x0, cdf x1, cdf& o0, cdf& o1, cdf& o2, cdf& o3) {
  const float K = grid_magic(fmaxf(cdf_amax(x0), cdf_amax(x1)));
  x0 = cdf_regrid(x0, K); x1 = cdf_regrid(x1, K);
  const cdf ix1 = cdf_mul_i(x1);
  o0 = cg_add(x0, x1); o1 = cg_sub(x0, x1); o2 = cg_add(x0, ix1); o3 = cg_sub(x0, ix1);
}

// DIF radix-2 butterfly on a common grid, before its twiddle: x0 <- x0 + x1, x1 <- x0 - x1.
__device__ __forceinline__ void dif2_grid(cdf& x0, cdf& x1) {
  const float K = grid_magic(fmaxf(cdf_amax(x0), cdf_amax(x1)));
  x0 = cdf_regrid(x0, K); x1 = cdf_regrid(x1, K);
  const cdf s = cg_add(x0, x1);
  x1 = cg_sub(x0, x1);
  x0 = s;
}

// One DIF radix-2^2 step over spans (H, H/2), H >= 4, sums on a common grid:
// for the group of size 2H at g * 2H and n < H/2, with x_m = row g*2H + n + m*H/2,
//   o0 = (x0 + x2) + (x1 + x3),           o1 = ((x0 + x2) - (x1 + x3)) w^(2j),
//   o2 = ((x0 - x2) + i (x1 - x3)) w^j,   o3 = ((x0 - x2) - i (x1 - x3)) w^(3j),
// j = n * M / (2H), written back in place.
template <int M, int EB, int H>
__device__ __forceinline__ void dif4_stage(float4* sm) {
  constexpr int Q4 = H / 2, LQ = ilog2<Q4>(), TS = M / (2 * H);
  const int e = threadIdx.x, y = threadIdx.y;
  // with Q4 <= 8 every butterfly of this thread has n = y mod Q4: one twiddle set
  Tw3<M, false> t;
  if (Q4 <= 8) t.load((y & (Q4 - 1)) * TS);
#pragma unroll
  for (int u = y; u < M / 4; u += 8) {
    const int g = u >> LQ, n = u & (Q4 - 1);
    const int base = g * 2 * H + n;
    cdf x0 = ld(&sm[base * EB + e]), x1 = ld(&sm[(base + Q4) * EB + e]);
    cdf x2 = ld(&sm[(base + 2 * Q4) * EB + e]), x3 = ld(&sm[(base + 3 * Q4) * EB + e]);
    dif4_grid(x0, x1, x2, x3);
    if (Q4 > 8) t.load(n * TS);
    t.apply(x1, x2, x3);
    st(&sm[base * EB + e], x0);
    st(&sm[(base + Q4) * EB + e], x1);
    st(&sm[(base + 2 * Q4) * EB + e], x2);
    st(&sm[(base + 3 * Q4) * EB + e], x3);
  }
}

// The last DIF radix-2^2 step (spans 2, 1; no twiddles) with normalised outputs.
template <int M, int EB>
__device__ __forceinline__ void dif4_last(float4* sm) {
  const int e = threadIdx.x, y = threadIdx.y;
#pragma unroll
  for (int u = y; u < M / 4; u += 8) {
    const int base = 4 * u;
    const cdf x0 = ld(&sm[base * EB + e]), x1 = ld(&sm[(base + 1) * EB + e]);
    const cdf x2 = ld(&sm[(base + 2) * EB + e]), x3 = ld(&sm[(base + 3) * EB + e]);
    // first-layer sums feed only the second layer, which renormalises
    const cdf s0 = cdf_add_lazy(x0, x2), s1 = cdf_add_lazy(x1, x3);
    const cdf d0 = cdf_sub_lazy(x0, x2), d1 = cdf_sub_lazy(x1, x3);
    const cdf id1 = cdf_mul_i(d1);
    st(&sm[base * EB + e], cdf_add(s0, s1));
    st(&sm[(base + 1) * EB + e], cdf_sub(s0, s1));
    st(&sm[(base + 2) * EB + e], cdf_add(d0, id1));
    st(&sm[(base + 3) * EB + e], cdf_sub(d0, id1));
  }
}

// The last DIF radix-2 step (span 1, twiddles 1) with normalised outputs.
template <int M, int EB>
__device__ __forceinline__ void dif2_last(float4* sm) {
  const int e = threadIdx.x, y = threadIdx.y;
#pragma unroll
  for (int bf = y; bf < M / 2; bf += 8) {
    const int i0 = 2 * bf, i1 = i0 + 1;
    const cdf u = ld(&sm[i0 * EB + e]), v = ld(&sm[i1 * EB + e]);
    st(&sm[i0 * EB + e], cdf_add(u, v));
    st(&sm[i1 * EB + e], cdf_sub(u, v));
  }
}

// DIF steps from span H down to span 1, each followed by a barrier.
template <int M, int EB, int H>
__device__ __forceinline__ void dif_stages(float4* sm) {
  if constexpr (H >= 4) {
    dif4_stage<M, EB, H>(sm);
    __syncthreads();
    dif_stages<M, EB, H / 4>(sm);
  } else if constexpr (H == 2) {
    dif4_last<M, EB>(sm);
    __syncthreads();
  } else if constexpr (H == 1) {
    dif2_last<M, EB>(sm);
    __syncthreads();
  }
}

// Forward DIF transform (radix 2^2 steps, first step pruned: the upper half of
// the zero-padded input is zero) of this CTA's EB entries, thread (e, y) =
// (threadIdx.x, threadIdx.y) owning column e of sm [M][EB].  src points at
// order 0 of column e's entry (orders E apart); row k is read only for k <= T
// and valid, and scaled by 2^(log2s + k log2r).  On return (after a barrier)
// sm row i holds mode bitrev(i).
template <int M, int EB>
__device__ __forceinline__ void fwd_to_smem(float4* sm, const double2* __restrict__ src, long long E, bool valid,
                                            int T, int log2s, int log2r) {
  const int e = threadIdx.x, y = threadIdx.y;
  auto raw_in = [&](int k) -> double2 {
    return (k <= T && valid) ? src[(long long)k * E] : make_double2(0.0, 0.0);
  };
  auto conv_in = [&](double2 x, int k) -> cdf {
    cdf v = cdf{df_from_double(x.x), df_from_double(x.y)};
    if (log2s != 0 || log2r != 0) {
      float f1, f2;
      pow2_pair(log2s + k * log2r, f1, f2);
      v = cdf{df_scale(df_scale(v.re, f1), f2), df_scale(df_scale(v.im, f1), f2)};
    }
    return v;
  };
  if constexpr (M >= 4) {
    // first two DIF stages at once (radix 2^2), upper half of the input zero:
    // X[n] = x0 + x1, X[n + M/4] = (x0 - x1) w^2n, X[n + M/2] = (x0 + i x1) w^n,
    // X[n + 3M/4] = (x0 - i x1) w^3n, with x0 = x[n], x1 = x[n + M/4], n < M/4
    // every input of this thread is requested before the first butterfly
    constexpr int NIT = (M / 4 + 7) / 8;
    double2 r0[NIT], r1[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int n = y + 8 * it;
      r0[it] = (n < M / 4) ? raw_in(n) : make_double2(0.0, 0.0);
      r1[it] = (n < M / 4) ? raw_in(n + M / 4) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
      const int n = y + 8 * it;
      if (n >= M / 4) break;
      cdf x0 = conv_in(r0[it], n), x1 = conv_in(r1[it], n + M / 4);
      cdf o0, o1, o2, o3;
      if constexpr (M == 4) {
        // the only step: normalised double-float sums
        const cdf ix1 = cdf_mul_i(x1);
        o0 = cdf_add(x0, x1); o1 = cdf_sub(x0, x1); o2 = cdf_add(x0, ix1); o3 = cdf_sub(x0, ix1);
      } else {
        dif4_pruned_grid(x0, x1, o0, o1, o2, o3);
        Tw3<M, false> t;
        t.load(n);
        t.apply(o1, o2, o3);
      }
      st(&sm[n * EB + e], o0);
      st(&sm[(n + M / 4) * EB + e], o1);
      st(&sm[(n + M / 2) * EB + e], o2);
      st(&sm[(n + 3 * M / 4) * EB + e], o3);
    }
    __syncthreads();
    dif_stages<M, EB, M / 8>(sm);
  } else {
    // M = 2: one stage, x[1] = 0
    if (y == 0) {
      const cdf v = conv_in(raw_in(0), 0);
      st(&sm[0 * EB + e], v);
      st(&sm[1 * EB + e], v);
    }
    __syncthreads();
  }
}

// ---- register-resident forward transform (M = 64, 128) ----
// Eight threads share a column of M rows.  The DIF steps of spans M/2 .. 8 only
// combine rows that are equal modulo 8, so thread y first runs them on its own
// rows y + 8a (a < M/8) in registers; one exchange through shared memory then
// gives it M/64 groups of 8 consecutive rows, on which it runs the steps of
// spans 4, 2 and 1, again in registers.  Shared memory is written and read
// once per row instead of once per step.
template <int M>
struct RegFft {
  static_assert(M == 64 || M == 128, "register path covers M = 64 and 128");
  static constexpr int A = M / 8;     // rows per thread
  static constexpr int GPT = M / 64;  // groups of 8 consecutive rows per thread after the exchange
};

// On return z[t][j] holds row 8m + j (mode bitrev(8m + j)) of column e, m = y * GPT + t;
// the exchange leaves sm in use until a barrier.
template <int M, int EB>
__device__ __forceinline__ void fwd_regs(float4* sm, const double2* __restrict__ src, long long E, bool valid,
                                         int T, int log2s, int log2r, cdf (&z)[RegFft<M>::GPT][8]) {
  constexpr int A = RegFft<M>::A, GPT = RegFft<M>::GPT;
  const int e = threadIdx.x, y = threadIdx.y;
  // rows y + 8a with a < A/2 are the nonzero inputs; all are requested first
  double2 r[A / 2];
#pragma unroll
  for (int a = 0; a < A / 2; ++a) {
    const int k = y + 8 * a;
    r[a] = (k <= T && valid) ? src[(long long)k * E] : make_double2(0.0, 0.0);
  }
  auto conv_in = [&](double2 v, int k) -> cdf {
    cdf c = cdf{df_from_double(v.x), df_from_double(v.y)};
    if (log2s != 0 || log2r != 0) {
      float f1, f2;
      pow2_pair(log2s + k * log2r, f1, f2);
      c = cdf{df_scale(df_scale(c.re, f1), f2), df_scale(df_scale(c.im, f1), f2)};
    }
    return c;
  };
  cdf x[A];  // x[a] = row y + 8a
  // spans (M/2, M/4), pruned: rows n and n + M/4 in, rows n + {0, 1, 2, 3} M/4 out, n = y + 8a
#pragma unroll
  for (int a = 0; a < A / 4; ++a) {
    const int n = y + 8 * a;
    dif4_pruned_grid(conv_in(r[a], n), conv_in(r[a + A / 4], n + M / 4), x[a], x[a + A / 4], x[a + A / 2],
                     x[a + 3 * A / 4]);
    Tw3<M, false> t;
    t.load(n);
    t.apply(x[a + A / 4], x[a + A / 2], x[a + 3 * A / 4]);
  }
  if constexpr (M == 128) {
    // spans (16, 8): rows 32g + y + {0, 8, 16, 24} = x[4g .. 4g + 3], twiddle index 4y
    Tw3<M, false> t;
    t.load(4 * y);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      dif4_grid(x[4 * g], x[4 * g + 1], x[4 * g + 2], x[4 * g + 3]);
      t.apply(x[4 * g + 1], x[4 * g + 2], x[4 * g + 3]);
    }
  } else {
    // span 8: rows 16g + y and 16g + y + 8 = x[2g], x[2g + 1], twiddle w^(4y)
    dfl c, s;
    if (y != 0) tw(4 * y, M, false, c, s);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      dif2_grid(x[2 * g], x[2 * g + 1]);
      if (y != 0) x[2 * g + 1] = cdf_mul_lazy(x[2 * g + 1], c, s);
    }
  }
  // exchange: rows y + 8a out, groups of 8 consecutive rows in
#pragma unroll
  for (int a = 0; a < A; ++a) st(&sm[(y + 8 * a) * EB + e], x[a]);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < GPT; ++t)
#pragma unroll
    for (int j = 0; j < 8; ++j) z[t][j] = ld(&sm[(8 * (y * GPT + t) + j) * EB + e]);
  // spans (4, 2): butterflies p = 0 (no twiddles) and p = 1 (w^(2j) = i, w^j, w^(3j), j = M/8);
  // span 1 (twiddles 1) with normalised outputs
  Tw3<M, false> t;
  t.load(M / 8);
#pragma unroll
  for (int g = 0; g < GPT; ++g) {
    dif4_grid(z[g][0], z[g][2], z[g][4], z[g][6]);
    dif4_grid(z[g][1], z[g][3], z[g][5], z[g][7]);
    t.apply(z[g][3], z[g][5], z[g][7]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const cdf u = z[g][2 * k], v = z[g][2 * k + 1];
      z[g][2 * k] = cdf_add(u, v);
      z[g][2 * k + 1] = cdf_sub(u, v);
    }
  }
}

}  // namespace fftdf
