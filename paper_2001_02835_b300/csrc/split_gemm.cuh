#pragma once
#include <cuda_runtime.h>

struct SplitGemmArgs {
  const void* slicesA;  // bf16 [Q][S][2][N][Kp]  rows of A~_q (K-major)
  const void* slicesB;  // bf16 [Q][S][3][N][Kp]  rows of (B~_q)^T (K-major): re, im, -re
  const int* expA;      // [Q][N] row exponents of A~_q
  const int* expB;      // [Q][N] row exponents of (B~_q)^T
  float4* C;            // [Q][N][N] double-float (re_hi, re_lo, im_hi, im_lo)
  int N, Kp, Q, S;
  int num_sms;
  int* err;             // device error word (0 = ok)
  int bn;               // output tile width (32 or 48; 0 = default 48)
  double2 alpha;        // C = alpha * A B (+ C) when use_alpha / accumulate
  int use_alpha, accumulate;
  long long ldc_q = 0;  // float4 entries from C_q to C_{q+1} (0: N * N, consecutive matrices)
};

// problems per grouped launch (their tensor maps travel in the kernel parameters)
#define NSPT_SPLIT_MAX_PROBLEMS 64

int nspt_split_gemm_init();
int nspt_split_gemm(const SplitGemmArgs& a, cudaStream_t st);
// one persistent launch over the tiles of `count` problems (same S); err of a[0] is used
int nspt_split_gemm_batch(const SplitGemmArgs* a, int count, int S, int bn, int num_sms, cudaStream_t st);
// 3M variant (three real products per complex product; plain products, S <= 6): both operands'
// slices with planes (re, im, re + im), tile 128 x 32 (split_gemm3m.cu)
int nspt_split_gemm3m_init();
int nspt_split_gemm3m(const SplitGemmArgs& a, cudaStream_t st);
// variant with the left operand in tensor memory (tile 128 x 40), selected by bn = 40
int nspt_split_gemm_ta_init();
int nspt_split_gemm_ta_batch(const SplitGemmArgs* a, int count, int S, int num_sms, cudaStream_t st);
// budget of the tensor GEMMs' abortable waits (ns; < 0: give up at once)
long long nspt_split_wait_budget();
void nspt_split_set_wait_budget(long long ns);
