// Order-axis FFT and inverse FFT in double-float arithmetic, for the split
// form (Sec. 2, FFT-CONV Steps 1-2 and 4-5).
//
// Same structure as the FP64 transforms (fft64.cu): a CTA stages a strip of
// EB consecutive entries of one batch element for all orders in shared memory
// and runs radix-2 butterflies there -- decimation in frequency for the
// forward transform (first stage pruned: the upper half of the zero-padded
// input is zero), decimation in time for the inverse (last stage pruned to the
// kept orders 0..T).  Arithmetic is double-float (about 48 significant bits),
// so the FP64 pipe is used only for the final hi + lo of each output of the
// inverse transform.  Spectra are float4 (re_hi, re_lo, im_hi, im_lo) per
// entry, 16 bytes like complex128.  Twiddles (cos, sin) come from the same
// extended-precision host table as the FP64 transforms, split into float pairs.
#include "common.cuh"
#include "dfloat.cuh"
#include "fft_twiddle.cuh"
#include "prof.cuh"
#include "zgemm64.cuh"

namespace {

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

// in: FP64 series, batch element b at in + b*in_stride*E, orders 0..T read
//     (row k pre-scaled by 2^(log2s + k*log2r));  out: [batch][M][E] float4
template <int M, int EB>
__global__ void __launch_bounds__(EB * 8)
fft_fwd_df_kernel(const double2* __restrict__ in, long long in_stride, float4* __restrict__ out, int E, int T,
                  int log2s, int log2r) {
  extern __shared__ float4 sm[];  // [M][EB]
  const int e = threadIdx.x, y = threadIdx.y, b = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB;
  const bool valid = (e0 + e) < E;
  const double2* src = in + (long long)b * in_stride * E + e0 + e;
  for (int k = y; k < M / 2; k += 8) {
    cdf v = cdf{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
    if (k <= T && valid) {
      const double2 x = src[(long long)k * E];
      v = cdf{df_from_double(x.x), df_from_double(x.y)};
      if (log2s != 0 || log2r != 0) {
        float f1, f2;
        pow2_pair(log2s + k * log2r, f1, f2);
        v = cdf{df_scale(df_scale(v.re, f1), f2), df_scale(df_scale(v.im, f1), f2)};
      }
    }
    st(&sm[k * EB + e], v);
    if (k == 0) {
      st(&sm[(k + M / 2) * EB + e], v);
    } else {
      dfl c, s;
      tw(k, M, false, c, s);
      st(&sm[(k + M / 2) * EB + e], cdf_mul(v, c, s));
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int h = M / 4; h >= 1; h >>= 1) {
    const int tstep = M / (2 * h);
    for (int bf = y; bf < M / 2; bf += 8) {
      const int g = bf / h, j = bf % h;
      const int i0 = g * 2 * h + j, i1 = i0 + h;
      const cdf u = ld(&sm[i0 * EB + e]), v = ld(&sm[i1 * EB + e]);
      st(&sm[i0 * EB + e], cdf_add(u, v));
      const cdf d = cdf_sub(u, v);
      if (j == 0) {
        st(&sm[i1 * EB + e], d);
      } else {
        dfl c, s;
        tw(j * tstep, M, false, c, s);
        st(&sm[i1 * EB + e], cdf_mul(d, c, s));
      }
    }
    __syncthreads();
  }
  if (!valid) return;
  float4* dst = out + (long long)b * M * E + e0 + e;
  for (int i = y; i < M; i += 8) dst[(long long)bitrev<M>(i) * E] = sm[i * EB + e];
}

// in: [batch][M][E] float4 spectrum; out: FP64 orders 0..T at out + b*out_stride*E,
// row k scaled by 2^(log2u - k*log2r) / M
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast(p, e);
}

// post: extra real double-float factor (1/n of Horner); add_identity: + 1 on the
// diagonal of order 0 (entry e is (e / N, e % N)); orders below kmin are not stored
template <int M, int EB>
__global__ void __launch_bounds__(EB * 8)
fft_inv_df_kernel(const float4* __restrict__ in, double2* __restrict__ out, long long out_stride, int E, int T,
                  int log2u, int log2r, float post_h, float post_l, int add_identity, int N, int kmin) {
  extern __shared__ float4 sm[];
  const int e = threadIdx.x, y = threadIdx.y, b = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB;
  const bool valid = (e0 + e) < E;
  const float4* src = in + (long long)b * M * E + e0 + e;
  for (int p = y; p < M; p += 8)
    sm[bitrev<M>(p) * EB + e] = valid ? src[(long long)p * E] : make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
#pragma unroll 1
  for (int h = 1; h <= M / 4; h <<= 1) {
    const int tstep = M / (2 * h);
    for (int bf = y; bf < M / 2; bf += 8) {
      const int g = bf / h, j = bf % h;
      const int i0 = g * 2 * h + j, i1 = i0 + h;
      const cdf u = ld(&sm[i0 * EB + e]);
      cdf v = ld(&sm[i1 * EB + e]);
      if (j != 0) {
        dfl c, s;
        tw(j * tstep, M, true, c, s);
        v = cdf_mul(v, c, s);
      }
      st(&sm[i0 * EB + e], cdf_add(u, v));
      st(&sm[i1 * EB + e], cdf_sub(u, v));
    }
    __syncthreads();
  }
  if (!valid) return;
  double2* dst = out + (long long)b * out_stride * E + e0 + e;
  constexpr int LOGM = 31 - __builtin_clz(M);
  const long long ent = e0 + e;
  const bool diag = add_identity && (ent / N) == (ent % N);
  const bool scaled = !(post_h == 1.f && post_l == 0.f);
  for (int k = y; k <= T; k += 8) {
    if (k < kmin) continue;
    const cdf u = ld(&sm[k * EB + e]);
    cdf v = ld(&sm[(k + M / 2) * EB + e]);
    if (k != 0) {
      dfl c, s;
      tw(k, M, true, c, s);
      v = cdf_mul(v, c, s);
    }
    cdf r = cdf_add(u, v);
    float f1, f2;
    pow2_pair(log2u - k * log2r - LOGM, f1, f2);
    r = cdf{df_scale(df_scale(r.re, f1), f2), df_scale(df_scale(r.im, f1), f2)};
    if (scaled) r = cdf{df_mul(r.re, dfl{post_h, post_l}), df_mul(r.im, dfl{post_h, post_l})};
    if (diag && k == 0) r.re = df_add(r.re, dfl{1.f, 0.f});
    dst[(long long)k * E] = make_double2(df_to_double(r.re), df_to_double(r.im));
  }
}

template <int M>
constexpr int strip_entries() { return M <= 128 ? 32 : (M == 256 ? 16 : 8); }

template <int M>
cudaError_t launch_fwd(const double2* in, long long ins, float4* out, int E, int T, int batch, int ls, int lr,
                       cudaStream_t st) {
  constexpr int EB = strip_entries<M>();
  const size_t smem = (size_t)M * EB * sizeof(float4);
  auto kern = fft_fwd_df_kernel<M, EB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((E + EB - 1) / EB, batch), block(EB, 8);
  kern<<<grid, block, smem, st>>>(in, ins, out, E, T, ls, lr);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_inv(const float4* in, double2* out, long long outs, int E, int T, int batch, int lu, int lr,
                       float ph, float pl, int addi, int N, int kmin, cudaStream_t st) {
  constexpr int EB = strip_entries<M>();
  const size_t smem = (size_t)M * EB * sizeof(float4);
  auto kern = fft_inv_df_kernel<M, EB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((E + EB - 1) / EB, batch), block(EB, 8);
  kern<<<grid, block, smem, st>>>(in, out, outs, E, T, lu, lr, ph, pl, addi, N, kmin);
  return cudaGetLastError();
}

}  // namespace

cudaError_t nspt_fft_fwd_df(const double2* in, long long in_stride, float4* out, int E, int t, int batch, int M,
                            int log2s, int log2r, cudaStream_t st) {
  if (2 * (t + 1) > M) return cudaErrorInvalidValue;
  ProfScope ps(NSPT_STAGE_FFT_FWD, st);
  switch (M) {
#define NSPT_CASE(m) case m: return launch_fwd<m>(in, in_stride, out, E, t, batch, log2s, log2r, st);
    NSPT_CASE(2) NSPT_CASE(4) NSPT_CASE(8) NSPT_CASE(16) NSPT_CASE(32) NSPT_CASE(64) NSPT_CASE(128)
    NSPT_CASE(256) NSPT_CASE(512)
#undef NSPT_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t nspt_fft_inv_df(const float4* in, double2* out, long long out_stride, int E, int t, int batch, int M,
                            int log2u, int log2r, cudaStream_t st, double post, int add_identity, int N, int kmin) {
  if (2 * (t + 1) > M) return cudaErrorInvalidValue;
  if (add_identity && N < 1) return cudaErrorInvalidValue;
  const float ph = (float)post, pl = (float)(post - (double)ph);
  ProfScope ps(NSPT_STAGE_FFT_INV, st);
  switch (M) {
#define NSPT_CASE(m) case m: return launch_inv<m>(in, out, out_stride, E, t, batch, log2u, log2r, ph, pl, add_identity, (N > 0 ? N : 1), kmin, st);
    NSPT_CASE(2) NSPT_CASE(4) NSPT_CASE(8) NSPT_CASE(16) NSPT_CASE(32) NSPT_CASE(64) NSPT_CASE(128)
    NSPT_CASE(256) NSPT_CASE(512)
#undef NSPT_CASE
    default: return cudaErrorInvalidValue;
  }
}
