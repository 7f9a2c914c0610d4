// Shared pieces of the double-float order transforms (split form, Sec. 2
// FFT-CONV Steps 2 and 4): twiddles, bit reversal, float4 <-> complex
// double-float, and the forward transform of a strip of entries in shared
// memory.
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
  auto load_in = [&](int k) -> cdf { return conv_in(raw_in(k), k); };
  int h;  // span of the next radix-2 stage still to do
  if (M >= 4) {
    // first two DIF stages at once (radix 2^2), upper half of the input zero:
    // X[n] = x0 + x1, X[n + M/4] = (x0 - x1) w^2n, X[n + M/2] = (x0 + i x1) w^n,
    // X[n + 3M/4] = (x0 - i x1) w^3n, with x0 = x[n], x1 = x[n + M/4], n < M/4
    // every input of this thread is requested before the first butterfly
    constexpr int NIT = M >= 4 ? (M / 4 + 7) / 8 : 1;
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
      const cdf x0 = conv_in(r0[it], n), x1 = conv_in(r1[it], n + M / 4);
      const cdf ix1 = cdf{df_neg(x1.im), x1.re};
      cdf o0 = cdf_add(x0, x1), o1 = cdf_sub(x0, x1), o2 = cdf_add(x0, ix1), o3 = cdf_sub(x0, ix1);
      if (n != 0) {
        dfl c, s;
        tw(2 * n, M, false, c, s); o1 = cdf_mul_lazy(o1, c, s);
        tw(n, M, false, c, s);     o2 = cdf_mul_lazy(o2, c, s);
        tw(3 * n, M, false, c, s); o3 = cdf_mul_lazy(o3, c, s);
      }
      st(&sm[n * EB + e], o0);
      st(&sm[(n + M / 4) * EB + e], o1);
      st(&sm[(n + M / 2) * EB + e], o2);
      st(&sm[(n + 3 * M / 4) * EB + e], o3);
    }
    h = M / 8;  // span of the next stage
  } else {
    // M = 2: one stage, x[1] = 0
    for (int k = y; k < 1; k += 8) {
      const cdf v = load_in(0);
      st(&sm[0 * EB + e], v);
      st(&sm[1 * EB + e], v);
    }
    h = 0;
  }
  __syncthreads();
  // remaining DIF stages: radix 2^2 steps over spans (h, h/2) while two are left
#pragma unroll 1
  for (; h >= 2; h >>= 2) {
    const int q4 = h / 2;   // quarter of the group of size L = 2h
    const int tstep = M / (2 * h);
    for (int u = y; u < M / 4; u += 8) {
      const int g = u >> (__ffs(q4) - 1), n = u & (q4 - 1);  // q4 is a power of two
      const int base = g * 2 * h + n;
      const cdf x0 = ld(&sm[base * EB + e]), x1 = ld(&sm[(base + q4) * EB + e]);
      const cdf x2 = ld(&sm[(base + 2 * q4) * EB + e]), x3 = ld(&sm[(base + 3 * q4) * EB + e]);
      // first-layer sums feed only the second layer, which renormalises
      const cdf s0 = cdf_add_lazy(x0, x2), s1 = cdf_add_lazy(x1, x3);
      const cdf d0 = cdf_sub_lazy(x0, x2), d1 = cdf_sub_lazy(x1, x3);
      const cdf id1 = cdf{df_neg(d1.im), d1.re};
      cdf o0 = cdf_add(s0, s1), o1 = cdf_sub(s0, s1), o2 = cdf_add(d0, id1), o3 = cdf_sub(d0, id1);
      if (n != 0) {
        dfl c, s;
        tw(2 * n * tstep, M, false, c, s); o1 = cdf_mul_lazy(o1, c, s);
        tw(n * tstep, M, false, c, s);     o2 = cdf_mul_lazy(o2, c, s);
        tw(3 * n * tstep, M, false, c, s); o3 = cdf_mul_lazy(o3, c, s);
      }
      st(&sm[base * EB + e], o0);
      st(&sm[(base + q4) * EB + e], o1);
      st(&sm[(base + 2 * q4) * EB + e], o2);
      st(&sm[(base + 3 * q4) * EB + e], o3);
    }
    __syncthreads();
  }
  if (h == 1) {  // one radix-2 stage of span 1 left (twiddles all 1)
    for (int bf = y; bf < M / 2; bf += 8) {
      const int i0 = 2 * bf, i1 = i0 + 1;
      const cdf u = ld(&sm[i0 * EB + e]), v = ld(&sm[i1 * EB + e]);
      st(&sm[i0 * EB + e], cdf_add(u, v));
      st(&sm[i1 * EB + e], cdf_sub(u, v));
    }
    __syncthreads();
  }
}

}  // namespace fftdf
