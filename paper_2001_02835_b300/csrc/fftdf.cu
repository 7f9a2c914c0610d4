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
  if constexpr (M == 64 || M == 128) {
    constexpr int GPT = fftdf::RegFft<M>::GPT;
    cdf z[GPT][8];
    fftdf::fwd_regs<M, EB>(sm, src, E, valid, T, log2s, log2r, z);
    if (!TOUT) {
      if (!valid) return;
      float4* dst = out + (long long)b * M * E + e0 + e;
#pragma unroll
      for (int t = 0; t < GPT; ++t)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int i = 8 * (y * GPT + t) + j;
          st(&dst[(long long)bitrev<M>(i) * E], z[t][j]);
        }
      return;
    }
    // transposed output straight from the registers: this thread's entry (j, l) =
    // (j0 + e / CB, l0 + e % CB) goes to (l, j), so for one mode a warp writes CB runs of 8
    // consecutive j (128 bytes each)
    if (!valid) return;
    float4* dst = out + (long long)b * M * E + (long long)(l0 + e % CB) * N + j0 + e / CB;
#pragma unroll
    for (int t = 0; t < GPT; ++t)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = 8 * (y * GPT + t) + j;
        st(&dst[(long long)bitrev<M>(i) * E], z[t][j]);
      }
    return;
  } else {
    fftdf::fwd_to_smem<M, EB>(sm, src, E, valid, T, log2s, log2r);
  }
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

// DIT radix-2^2 butterfly (after the step's twiddles), sums on a common grid:
// a <- (a + b) + (c + d), b <- (a - b) - i (c - d), c <- (a + b) - (c + d), d <- (a - b) + i (c - d).
__device__ __forceinline__ void dit4_grid(cdf& a, cdf& b, cdf& c, cdf& d) {
  const float K = grid_magic(fftdf::cdf_amax4(a, b, c, d));
  a = cdf_regrid(a, K); b = cdf_regrid(b, K); c = cdf_regrid(c, K); d = cdf_regrid(d, K);
  const cdf apb = cg_add(a, b), amb = cg_sub(a, b), cpd = cg_add(c, d);
  const cdf mi = cdf_mul_mi(cg_sub(c, d));  // (-i)(c - d)
  a = cg_add(apb, cpd); b = cg_add(amb, mi); c = cg_sub(apb, cpd); d = cg_sub(amb, mi);
}

// One DIT radix-2^2 step over spans (H, 2H), sums on a common grid: for the
// group of size 4H at g * 4H and n < H, with x_m = row g*4H + n + m*H and
// j = n * M / (4H), the inputs x1, x2, x3 are first multiplied by w^-2j, w^-j,
// w^-3j, then
//   o0 = (x0 + x1) + (x2 + x3),   o1 = (x0 - x1) - i (x2 - x3),
//   o2 = (x0 + x1) - (x2 + x3),   o3 = (x0 - x1) + i (x2 - x3).
template <int M, int EB, int H>
__device__ __forceinline__ void dit4_stage(float4* sm) {
  constexpr int LH = fftdf::ilog2<H>(), TS = M / (4 * H);
  const int e = threadIdx.x, y = threadIdx.y;
  // with H <= 8 every butterfly of this thread has n = y mod H: one twiddle set
  fftdf::Tw3<M, true> t;
  if (H <= 8) t.load((y & (H - 1)) * TS);
#pragma unroll
  for (int u = y; u < M / 4; u += 8) {
    const int g = u >> LH, n = u & (H - 1);
    const int base = g * 4 * H + n;
    cdf a = ld(&sm[base * EB + e]), bq = ld(&sm[(base + H) * EB + e]);
    cdf c = ld(&sm[(base + 2 * H) * EB + e]), d = ld(&sm[(base + 3 * H) * EB + e]);
    if (H > 8) t.load(n * TS);
    t.apply(bq, c, d);
    dit4_grid(a, bq, c, d);
    st(&sm[base * EB + e], a);
    st(&sm[(base + H) * EB + e], bq);
    st(&sm[(base + 2 * H) * EB + e], c);
    st(&sm[(base + 3 * H) * EB + e], d);
  }
}

// One DIT radix-2 step of span H (normalised double-float sums).
template <int M, int EB, int H>
__device__ __forceinline__ void dit2_stage(float4* sm) {
  constexpr int LH = fftdf::ilog2<H>(), TS = M / (2 * H);
  const int e = threadIdx.x, y = threadIdx.y;
#pragma unroll
  for (int bf = y; bf < M / 2; bf += 8) {
    const int g = bf >> LH, j = bf & (H - 1);
    const int i0 = g * 2 * H + j, i1 = i0 + H;
    const cdf u = ld(&sm[i0 * EB + e]);
    cdf v = ld(&sm[i1 * EB + e]);
    if (j != 0) {
      dfl c, s;
      tw(j * TS, M, true, c, s);
      v = cdf_mul_lazy(v, c, s);
    }
    st(&sm[i0 * EB + e], cdf_add(u, v));
    st(&sm[i1 * EB + e], cdf_sub(u, v));
  }
}

// DIT steps of spans H, 4H, ... while two are left below M/2, then one radix-2
// step if one is; the last stage (span M/2) is fused into the output.
template <int M, int EB, int H>
__device__ __forceinline__ void dit_stages(float4* sm) {
  if constexpr (2 * H <= M / 4) {
    dit4_stage<M, EB, H>(sm);
    __syncthreads();
    dit_stages<M, EB, 4 * H>(sm);
  } else if constexpr (H <= M / 4) {
    dit2_stage<M, EB, H>(sm);
    __syncthreads();
  }
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
  constexpr int LOGM = 31 - __builtin_clz(M);
  const long long ent = e0 + e;
  const bool diag = add_identity && (ent / N) == (ent % N);
  const bool scaled = !(post_h == 1.f && post_l == 0.f);
  double2* dst = out + (long long)b * out_stride * E + e0 + e;
  // order k: scaled by 2^(log2u - k log2r) / M and by post, + 1 on the diagonal of order 0
  auto put = [&](int k, cdf r) {
    float f1, f2;
    pow2_pair(log2u - k * log2r - LOGM, f1, f2);
    r = cdf{df_scale(df_scale(r.re, f1), f2), df_scale(df_scale(r.im, f1), f2)};
    if (scaled) r = cdf{df_mul(r.re, dfl{post_h, post_l}), df_mul(r.im, dfl{post_h, post_l})};
    if (diag && k == 0) r.re = df_add(r.re, dfl{1.f, 0.f});
    dst[(long long)k * E] = make_double2(df_to_double(r.re), df_to_double(r.im));  // hi + lo in FP64
  };
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
  dit_stages<M, EB, 1>(sm);
  if (!valid) return;
  for (int k = y; k <= T; k += 8) {
    if (k < kmin) continue;
    const cdf u = ld(&sm[k * EB + e]);
    cdf v = ld(&sm[(k + M / 2) * EB + e]);
    if (k != 0) {
      dfl c, s;
      tw(k, M, true, c, s);
      v = cdf_mul_lazy(v, c, s);
    }
    put(k, cdf_add_lazy(u, v));
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
