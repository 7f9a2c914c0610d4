// Order-axis FFT and inverse FFT in double-float arithmetic, for the split
// form (Sec. 2, FFT-CONV Steps 1-2 and 4-5).
//
// Same structure as the FP64 transforms (fft64.cu): a CTA stages a strip of
// EB consecutive entries of one batch element for all orders in shared memory
// and runs radix-2^2 butterflies there -- decimation in frequency for the
// forward transform (first step pruned: the upper half of the zero-padded
// input is zero; the body is in fftdf_core.cuh), decimation in time for the
// inverse (last stage pruned to the kept orders 0..T).  Every thread requests
// all of its inputs before the first butterfly.  The forward transform can
// write the spectra transposed (blocks of 8 x EB/8 entries) for the right
// operand of a product.  Arithmetic is double-float (about 48 significant bits),
// so the FP64 pipe is used only for the final hi + lo of each output of the
// inverse transform.  Spectra are float4 (re_hi, re_lo, im_hi, im_lo) per
// entry, 16 bytes like complex128.  Twiddles (cos, sin) come from the same
// extended-precision host table as the FP64 transforms, split into float pairs.
#include "common.cuh"
#include "dfloat.cuh"
#include "fft_twiddle.cuh"
#include "fftdf_core.cuh"
#include "prof.cuh"
#include "zgemm64.cuh"

namespace {

using fftdf::tw;
using fftdf::bitrev;
using fftdf::ld;
using fftdf::st;

// in: FP64 series, batch element b at in + b*in_stride*E, orders 0..T read
//     (row k pre-scaled by 2^(log2s + k*log2r));  out: [batch][M][E] float4.
// TOUT: every spectrum matrix is written transposed (out entry (l, j) holds
// mode p of input entry (j, l), E = N*N).  A CTA then takes a block of 8 rows
// x EB/8 columns instead of a strip, so that its loads are EB/8 consecutive
// entries of each row and its stores 8 consecutive entries (128 bytes) of
// each transposed row.
template <int M, int EB, bool TOUT>
__global__ void __launch_bounds__(EB * 8)
fft_fwd_df_kernel(const double2* __restrict__ in, long long in_stride, float4* __restrict__ out, int E, int T,
                  int log2s, int log2r, int N, const int* __restrict__ dlr) {
  if (dlr) log2r *= *dlr;  // rescale exponent fitted on the device
  extern __shared__ float4 sm[];  // [M][EB]
  constexpr int CB = EB / 8;      // columns per block (TOUT)
  const int e = threadIdx.x, y = threadIdx.y, b = blockIdx.y;
  long long e0 = (long long)blockIdx.x * EB;
  bool valid = (e0 + e) < E;
  int j0 = 0, l0 = 0;
  const double2* src = in + (long long)b * in_stride * E + e0 + e;
  if (TOUT) {
    const int nlb = (N + CB - 1) / CB;
    j0 = (blockIdx.x / nlb) * 8;
    l0 = (blockIdx.x % nlb) * CB;
    const int j = j0 + e / CB, l = l0 + e % CB;   // loaded entry of this thread
    valid = j < N && l < N;
    src = in + (long long)b * in_stride * E + (long long)j * N + l;
  }
  fftdf::fwd_to_smem<M, EB>(sm, src, E, valid, T, log2s, log2r);
  if (TOUT) {
    // this thread stores smem column c = entry (j0 + e % 8, l0 + e / 8) at (l, j)
    const int jj = e % 8, ll = e / 8, c = jj * CB + ll;
    if (j0 + jj >= N || l0 + ll >= N) return;
    float4* dst = out + (long long)b * M * E + (long long)(l0 + ll) * N + j0 + jj;
    for (int i = y; i < M; i += 8) dst[(long long)bitrev<M>(i) * E] = sm[i * EB + c];
    return;
  }
  if (!valid) return;
  float4* dst = out + (long long)b * M * E + e0 + e;
  for (int i = y; i < M; i += 8) dst[(long long)bitrev<M>(i) * E] = sm[i * EB + e];
}

// in: [batch][M][E] float4 spectrum; out: FP64 orders 0..T at out + b*out_stride*E,
// row k scaled by 2^(log2u - k*log2r) / M
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_fast(p, e);
}

// post: extra real double-float factor on the result; add_identity: + 1 on the
// diagonal of order 0 (entry e is (e / N, e % N)); orders below kmin are not stored
template <int M, int EB>
__global__ void __launch_bounds__(EB * 8)
fft_inv_df_kernel(const float4* __restrict__ in, double2* __restrict__ out, long long out_stride, int E, int T,
                  int log2u, int log2r, float post_h, float post_l, int add_identity, int N, int kmin,
                  const int* __restrict__ dlr) {
  if (dlr) log2r *= *dlr;  // rescale exponent fitted on the device
  extern __shared__ float4 sm[];
  const int e = threadIdx.x, y = threadIdx.y, b = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB;
  const bool valid = (e0 + e) < E;
  const float4* src = in + (long long)b * M * E + e0 + e;
  // loads in groups of up to 16 per thread, all in flight before their stores
  constexpr int NL = (M + 7) / 8, G = NL < 16 ? NL : 16;
#pragma unroll 1
  for (int g0 = 0; g0 < NL; g0 += G) {
    float4 v[G];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int p = y + 8 * (g0 + i);
      v[i] = (valid && p < M) ? src[(long long)p * E] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int p = y + 8 * (g0 + i);
      if (p < M) sm[bitrev<M>(p) * EB + e] = v[i];
    }
  }
  __syncthreads();
  // DIT stages of spans 1 .. M/4: radix 2^2 steps over spans (h, 2h) while two are left
  int h = 1;
#pragma unroll 1
  for (; 2 * h <= M / 4; h <<= 2) {
    const int tstep = M / (4 * h);  // w_L^-m = conj(w_M^(m M / L)), L = 4h
    for (int u = y; u < M / 4; u += 8) {
      const int g = u >> (__ffs(h) - 1), n = u & (h - 1);  // h is a power of two
      const int base = g * 4 * h + n;
      cdf a = ld(&sm[base * EB + e]), bq = ld(&sm[(base + h) * EB + e]);
      cdf c = ld(&sm[(base + 2 * h) * EB + e]), d = ld(&sm[(base + 3 * h) * EB + e]);
      if (n != 0) {
        dfl cw, sw;
        tw(2 * n * tstep, M, true, cw, sw); bq = cdf_mul_lazy(bq, cw, sw);
        tw(n * tstep, M, true, cw, sw);     c = cdf_mul_lazy(c, cw, sw);
        tw(3 * n * tstep, M, true, cw, sw); d = cdf_mul_lazy(d, cw, sw);
      }
      // first-layer sums feed only the second layer, which renormalises
      const cdf apb = cdf_add_lazy(a, bq), amb = cdf_sub_lazy(a, bq);
      const cdf cpd = cdf_add_lazy(c, d), cmd = cdf_sub_lazy(c, d);
      const cdf mi = cdf{cmd.im, df_neg(cmd.re)};  // (-i)(c - d)
      st(&sm[base * EB + e], cdf_add(apb, cpd));
      st(&sm[(base + h) * EB + e], cdf_add(amb, mi));
      st(&sm[(base + 2 * h) * EB + e], cdf_sub(apb, cpd));
      st(&sm[(base + 3 * h) * EB + e], cdf_sub(amb, mi));
    }
    __syncthreads();
  }
  if (h <= M / 4) {  // one radix-2 DIT stage of span h left
    const int tstep = M / (2 * h);
    for (int bf = y; bf < M / 2; bf += 8) {
      const int g = bf >> (__ffs(h) - 1), j = bf & (h - 1);
      const int i0 = g * 2 * h + j, i1 = i0 + h;
      const cdf u = ld(&sm[i0 * EB + e]);
      cdf v = ld(&sm[i1 * EB + e]);
      if (j != 0) {
        dfl c, s;
        tw(j * tstep, M, true, c, s);
        v = cdf_mul_lazy(v, c, s);
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
      v = cdf_mul_lazy(v, c, s);
    }
    cdf r = cdf_add_lazy(u, v);  // converted to FP64 as hi + lo, exact either way
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
                       int tout_n, cudaStream_t st) {
  constexpr int EB = strip_entries<M>();
  const size_t smem = (size_t)M * EB * sizeof(float4);
  auto kern = tout_n ? fft_fwd_df_kernel<M, EB, true> : fft_fwd_df_kernel<M, EB, false>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const long long blocks = tout_n ? (long long)((tout_n + 7) / 8) * ((tout_n + EB / 8 - 1) / (EB / 8))
                                  : ((long long)E + EB - 1) / EB;
  dim3 grid((unsigned)blocks, batch), block(EB, 8);
  kern<<<grid, block, smem, st>>>(in, ins, out, E, T, ls, lr, tout_n, nspt_dev_log2r());
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
  kern<<<grid, block, smem, st>>>(in, out, outs, E, T, lu, lr, ph, pl, addi, N, kmin, nspt_dev_log2r());
  return cudaGetLastError();
}

}  // namespace

cudaError_t nspt_fft_fwd_df(const double2* in, long long in_stride, float4* out, int E, int t, int batch, int M,
                            int log2s, int log2r, cudaStream_t st, int transpose_n) {
  if (2 * (t + 1) > M) return cudaErrorInvalidValue;
  if (transpose_n && (long long)transpose_n * transpose_n != E) return cudaErrorInvalidValue;
  ProfScope ps(NSPT_STAGE_FFT_FWD, st);
  switch (M) {
#define NSPT_CASE(m) case m: return launch_fwd<m>(in, in_stride, out, E, t, batch, log2s, log2r, transpose_n, st);
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
