// Parameters of the FP64 complex GEMM families (see zgemm64.cu).
#pragma once
#include <cuda_runtime.h>

enum { ZG_MODE = 0, ZG_CONV = 1, ZG_CORR_A = 2, ZG_CORR_B = 3 };

struct ZgemmParams {
  const double2* A;   // batch element b starts at A + b*sA*N*N
  const double2* B;   // ... B + b*sB*N*N
  double2* C;         // ... C + b*sC*N*N; output q at + q*N*N
  int N;
  int kind;           // ZG_*
  int nmat;           // output matrices per batch element (modes M, or T+1)
  long long sA, sB, sC;  // batch strides in matrices
  int T;              // truncation order (CORR kinds)
  int opA, opB;       // 0 = as stored, 1 = conjugate transpose
  int revA, revB;     // MODE: read mode (nmat - p) mod nmat
  double2 alpha;      // C = alpha * sum (+ C if accumulate)
  int accumulate;
};

cudaError_t nspt_zgemm64(const ZgemmParams& P, int batch, cudaStream_t st);
// Forward order FFT (Steps 1-2): series b starts at in + b*in_stride*E and its
// orders 0..t are read (t+1 <= M/2); the spectrum goes to out + b*M*E.
// Row k is pre-scaled by 2^(log2s + k*log2r).
cudaError_t nspt_fft_fwd64(const double2* in, long long in_stride, double2* out, int E, int t, int batch,
                           int M, int log2s, int log2r, cudaStream_t st);
// Inverse order FFT (Steps 4-5): spectrum b at in + b*M*E; orders 0..t written to
// out + b*out_stride*E, scaled by post * 2^(log2u - k*log2r) / M; when
// add_identity, the N x N identity is added to order 0 (E = N*N).  Orders
// below kmin are not stored.
cudaError_t nspt_fft_inv64(const double2* in, double2* out, long long out_stride, int E, int N, int t,
                           int batch, int M, int log2u, int log2r, double post, int add_identity,
                           cudaStream_t st, int kmin = 0);
// Inverse order FFT of a double-float spectrum (float4 = re_hi, re_lo, im_hi, im_lo).
cudaError_t nspt_fft_inv64_df(const float4* in, double2* out, long long out_stride, int E, int N, int t, int batch,
                              int M, int log2u, int log2r, cudaStream_t st);
// Double-float order FFTs of the split form (fftdf.cu): FP64 series in,
// float4 (re_hi, re_lo, im_hi, im_lo) spectrum out, and back.  transpose_n = N
// writes every spectrum matrix transposed (E = N*N); 0 keeps the layout.
cudaError_t nspt_fft_fwd_df(const double2* in, long long in_stride, float4* out, int E, int t, int batch, int M,
                            int log2s, int log2r, cudaStream_t st, int transpose_n = 0);
cudaError_t nspt_fft_inv_df(const float4* in, double2* out, long long out_stride, int E, int t, int batch, int M,
                            int log2u, int log2r, cudaStream_t st, double post = 1.0, int add_identity = 0,
                            int N = 0, int kmin = 0);
