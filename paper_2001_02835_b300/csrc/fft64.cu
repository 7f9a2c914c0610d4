// Order-axis FFT and inverse FFT of polynomial-matrix series, FP64 form
// (Sec. 2, FFT-CONV Steps 1-2 and 4-5).
//
// Layout: a series batch is [batch][T+1][E] complex128 with E = N*N entries of
// one coefficient matrix; the spectrum is [batch][M][E].  The transform runs
// along the order axis, whose stride is E: a CTA takes EB consecutive entries
// of one batch element and all orders, so every global row access is one
// contiguous, vectorised run of EB*16 bytes.  The strip is staged in shared
// memory ([M][EB]) and transformed there with radix-2 butterflies.
//
// Forward (Steps 1-2): decimation in frequency, natural-order input, first
// stage pruned because the upper half of the zero-padded input is zero,
// bit-reversed output written to its natural mode index p.
// Inverse (Steps 4-5): decimation in time, bit-reversed load, last stage
// pruned to the kept orders k = 0..T, scaled by 1/M.
// Twiddles w^n = exp(2 pi i n / Mmax) come from a host table computed in long
// double (w = exp(+2 pi i/M) forward as in Step 2; conjugate for Step 4).
#include "common.cuh"
#include "fft_twiddle.cuh"
#include "zgemm64.cuh"
#include "prof.cuh"

namespace {

__device__ __forceinline__ double2 tw_fwd(int n, int M) {
  // w_M^n = w_Mmax^(n * Mmax / M)
  return c_twiddle[n * (NSPT_FFT_MAX_LEN / M)];
}

template <int M>
__device__ __forceinline__ int bitrev(int i) {
  constexpr int LOG = (M <= 1) ? 0 : (31 - __builtin_clz(M));
  return (int)(__brev((unsigned)i) >> (32 - LOG));
}

// in:  [batch][T+1][E]  (rows scaled by scale_k = 2^(log2s + k*log2r))
// out: [batch][M][E]
template <int M, int EB>
__global__ void __launch_bounds__(EB * 8)
fft_fwd64_kernel(const double2* __restrict__ in, long long in_stride, double2* __restrict__ out, int E,
                 int T, int log2s, int log2r, const int* __restrict__ dlr) {
  if (dlr) log2r *= *dlr;  // rescale exponent fitted on the device
  extern __shared__ double2 sm[];  // [M][EB]
  const int e = threadIdx.x;       // entry within strip
  const int y = threadIdx.y;       // 0..7
  const int b = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB;
  const bool valid = (e0 + e) < E;
  const double2* src = in + (long long)b * in_stride * E + e0 + e;
  for (int k = y; k < M / 2; k += 8) {
    double2 v = make_double2(0.0, 0.0);
    if (k <= T && valid) {
      v = src[(long long)k * E];
      if (log2s != 0 || log2r != 0) {
        const double s = ldexp(1.0, log2s + k * log2r);
        v = cscale(v, s);
      }
    }
    // first DIF stage with a zero upper half: x[j] stays, x[j+M/2] = x[j] w^j
    sm[k * EB + e] = v;
    sm[(k + M / 2) * EB + e] = (k == 0) ? v : cmul(v, tw_fwd(k, M));
  }
  __syncthreads();
#pragma unroll 1
  for (int h = M / 4; h >= 1; h >>= 1) {
    const int tstep = M / (2 * h);
    for (int bf = y; bf < M / 2; bf += 8) {
      const int g = bf >> (__ffs(h) - 1), j = bf & (h - 1);  // h is a power of two
      const int i0 = g * 2 * h + j, i1 = i0 + h;
      const double2 u = sm[i0 * EB + e], v = sm[i1 * EB + e];
      sm[i0 * EB + e] = cadd(u, v);
      const double2 d = csub(u, v);
      sm[i1 * EB + e] = (j == 0) ? d : cmul(d, tw_fwd(j * tstep, M));
    }
    __syncthreads();
  }
  if (!valid) return;
  double2* dst = out + (long long)b * M * E + e0 + e;
  for (int i = y; i < M; i += 8) dst[(long long)bitrev<M>(i) * E] = sm[i * EB + e];
}

__device__ __forceinline__ double2 load_spec(const double2* p) { return *p; }
// double-float spectrum (re_hi, re_lo, im_hi, im_lo) from the tensor-core GEMM
__device__ __forceinline__ double2 load_spec(const float4* p) {
  const float4 v = *p;
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// in:  [batch][M][E] spectrum; out: [batch][T+1][E], row k scaled by
// 2^(log2u - k*log2r) / M.
template <int M, int EB, typename InT>
__global__ void __launch_bounds__(EB * 8)
fft_inv64_kernel(const InT* __restrict__ in, double2* __restrict__ out, long long out_stride, int E,
                 int N, int T, int log2u, int log2r, double post, int add_identity, int kmin,
                 const int* __restrict__ dlr) {
  if (dlr) log2r *= *dlr;  // rescale exponent fitted on the device
  extern __shared__ double2 sm[];
  const int e = threadIdx.x;
  const int y = threadIdx.y;
  const int b = blockIdx.y;
  const long long e0 = (long long)blockIdx.x * EB;
  const bool valid = (e0 + e) < E;
  const InT* src = in + (long long)b * M * E + e0 + e;
  for (int p = y; p < M; p += 8)
    sm[bitrev<M>(p) * EB + e] = valid ? load_spec(src + (long long)p * E) : make_double2(0.0, 0.0);
  __syncthreads();
#pragma unroll 1
  for (int h = 1; h <= M / 4; h <<= 1) {
    const int tstep = M / (2 * h);
    for (int bf = y; bf < M / 2; bf += 8) {
      const int g = bf >> (__ffs(h) - 1), j = bf & (h - 1);  // h is a power of two
      const int i0 = g * 2 * h + j, i1 = i0 + h;
      const double2 u = sm[i0 * EB + e];
      double2 v = sm[i1 * EB + e];
      if (j != 0) v = cmul(v, cconj(tw_fwd(j * tstep, M)));
      sm[i0 * EB + e] = cadd(u, v);
      sm[i1 * EB + e] = csub(u, v);
    }
    __syncthreads();
  }
  if (!valid) return;
  double2* dst = out + (long long)b * out_stride * E + e0 + e;
  const long long ent = e0 + e;
  const bool diag = add_identity && (ent / N) == (ent % N);
  for (int k = y; k <= T; k += 8) {
    if (k < kmin) continue;
    const double2 u = sm[k * EB + e];
    double2 v = sm[(k + M / 2) * EB + e];
    if (k != 0) v = cmul(v, cconj(tw_fwd(k, M)));
    const double s = post * ldexp(1.0, log2u - k * log2r) / (double)M;
    double2 r = cscale(cadd(u, v), s);
    if (diag && k == 0) r.x += 1.0;
    dst[(long long)k * E] = r;
  }
}

template <int M>
constexpr int strip_entries() { return M <= 128 ? 32 : (M == 256 ? 16 : 8); }

template <int M>
cudaError_t launch_fwd(const double2* in, long long ins, double2* out, int E, int T, int batch, int ls, int lr,
                       cudaStream_t st) {
  constexpr int EB = strip_entries<M>();
  const size_t smem = (size_t)M * EB * sizeof(double2);
  auto kern = fft_fwd64_kernel<M, EB>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((E + EB - 1) / EB, batch), block(EB, 8);
  kern<<<grid, block, smem, st>>>(in, ins, out, E, T, ls, lr, nspt_dev_log2r());
  return cudaGetLastError();
}

template <int M, typename InT>
cudaError_t launch_inv(const InT* in, double2* out, long long outs, int E, int N, int T, int batch, int lu,
                       int lr, double post, int addi, int kmin, cudaStream_t st) {
  constexpr int EB = strip_entries<M>();
  const size_t smem = (size_t)M * EB * sizeof(double2);
  auto kern = fft_inv64_kernel<M, EB, InT>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  dim3 grid((E + EB - 1) / EB, batch), block(EB, 8);
  kern<<<grid, block, smem, st>>>(in, out, outs, E, N, T, lu, lr, post, addi, kmin, nspt_dev_log2r());
  return cudaGetLastError();
}

}  // namespace

// Host entry points used by the planner (api.cu).
cudaError_t nspt_fft_fwd64(const double2* in, long long in_stride, double2* out, int E, int t, int batch,
                           int M, int log2s, int log2r, cudaStream_t st) {
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

cudaError_t nspt_fft_inv64(const double2* in, double2* out, long long out_stride, int E, int N, int t,
                           int batch, int M, int log2u, int log2r, double post, int add_identity,
                           cudaStream_t st, int kmin) {
  if (2 * (t + 1) > M) return cudaErrorInvalidValue;
  ProfScope ps(NSPT_STAGE_FFT_INV, st);
  switch (M) {
#define NSPT_CASE(m) case m: return launch_inv<m, double2>(in, out, out_stride, E, N, t, batch, log2u, log2r, post, add_identity, kmin, st);
    NSPT_CASE(2) NSPT_CASE(4) NSPT_CASE(8) NSPT_CASE(16) NSPT_CASE(32) NSPT_CASE(64) NSPT_CASE(128)
    NSPT_CASE(256) NSPT_CASE(512)
#undef NSPT_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t nspt_fft_inv64_df(const float4* in, double2* out, long long out_stride, int E, int N, int t, int batch,
                              int M, int log2u, int log2r, cudaStream_t st) {
  if (2 * (t + 1) > M) return cudaErrorInvalidValue;
  ProfScope ps(NSPT_STAGE_FFT_INV, st);
  switch (M) {
#define NSPT_CASE(m) case m: return launch_inv<m, float4>(in, out, out_stride, E, N, t, batch, log2u, log2r, 1.0, 0, 0, st);
    NSPT_CASE(2) NSPT_CASE(4) NSPT_CASE(8) NSPT_CASE(16) NSPT_CASE(32) NSPT_CASE(64) NSPT_CASE(128)
    NSPT_CASE(256) NSPT_CASE(512)
#undef NSPT_CASE
    default: return cudaErrorInvalidValue;
  }
}
