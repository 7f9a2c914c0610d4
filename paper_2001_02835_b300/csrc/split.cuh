// Split-precision form of the product path (tensor-core mode GEMMs).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <functional>

#include "../../include/nspt.h"

int nspt_split_init();
// row pitch of the digit slices: N rounded up to 8 BF16 values (16 bytes)
inline int nspt_split_kpad(int N) { return (N + 7) & ~7; }
int nspt_split_num_sms();
// untuned tile width (complex columns) of the tensor-core GEMMs for products of size <= nmax
int nspt_split_default_bn(int nmax);
// runs chain(i, stream) for i < count on the library's side streams, forked from and joined
// back to st (on st itself when the side streams are missing)
int nspt_split_fork_join(int count, cudaStream_t st, const std::function<int(int, cudaStream_t)>& chain);
// cm: complex products as 4 real products (the embedding, every entry point) or 3 (3M: products only)
size_t nspt_split_ws_mul(int N, int T, int batch, int M, int slices, int cm = 4);
size_t nspt_split_ws_bwd(int N, int T, int batch, int M, int slices);
int nspt_split_mul(int N, int T, int batch, int M, int slices, int log2r, bool rescale_auto, const double2* A,
                   const double2* B, double2* C, void* ws, cudaStream_t st, int cm = 4);
// naive form (Eq. 5) with split-precision pair GEMMs (every order sliced from FP64; no transforms);
// log2r / rescale_auto: the slices of order k stand for 2^(k log2r) times the order (exponent shift),
// undone on the FP64 output, so that the double-float accumulator stays in the FP32 range
size_t nspt_split_ws_naive(int N, int T, int batch, int slices);
int nspt_split_mul_naive(int N, int T, int batch, int slices, int log2r, bool rescale_auto, const double2* A,
                         const double2* B, double2* C, void* ws, cudaStream_t st);
// backward of the naive form with the split pair GEMMs (same workspace as the product)
int nspt_split_bwd_naive(int N, int T, int batch, int slices, int log2r, const double2* A, const double2* B,
                         const double2* G, double2* gA, double2* gB, void* ws, cudaStream_t st);
int nspt_split_bwd(int N, int T, int batch, int M, int slices, int log2r, const double2* A, const double2* B,
                   const double2* G, double2* gA, double2* gB, void* ws, cudaStream_t st);
// mode: NSPT_LMODE_* (tek.cuh); Yin: i X for NSPT_LMODE_UPDATE; log2r: every order transform of the
// step scales order k by 2^(k log2r) and its inverse undoes it (exact, and the same result in exact
// arithmetic: the ring map X_k -> r^k X_k commutes with every product and sum of the step)
int nspt_split_langevin(int N, int T, int batch, int M, int slices, double2* U, const double2* eta, double2* F,
                        int flux, double eps, void* ws, cudaStream_t st, int mode = 0, const double2* Yin = nullptr,
                        int log2r = 0);
// slices of Q planes of X (see slice_kernel): out bf16 [Q][S][2][N][Kp], exps [Q][N]
int nspt_split_slice(int S, const double2* X, long long bstride, int M, int rev, int trans, int conj, int N, int Q,
                     int P, void* out, int* exps, cudaStream_t st);
// sum3 (with P = 3): the third plane holds re + im at the row exponent + 1 (3M operands; row form,
// N <= 512, trans = 0 only, else NSPT_ERR_UNSUPPORTED)
int nspt_split_slice_df(int S, const float4* X, long long bstride, int M, int rev, int trans, int conj, int N, int Q,
                        int P, void* out, int* exps, cudaStream_t st, int sum3 = 0);
int nspt_split_gemm_stage(const void* slA, const void* slB, const int* expA, const int* expB, void* C, int N, int Q,
                          int S, int* err, cudaStream_t st);
int nspt_split_read_error(void* ws, int* host_err, cudaStream_t st);
// fit of the per-order rescale exponent on the device: with y_k = log2 max|A_k| + log2 max|B_k|
// over the orders where both are nonzero (A, B: `batch` series [T+1][N][N]), the integer log2r
// minimising the spread of y_k + 2 k log2r (smallest |log2r| among equals), among those that lift
// no order of A or B above max(1, its largest order) and, with float_range, keep the scale factors
// within 2^+-120 (the FP32 range of the double-float transforms).  scratch: 2 (T+1) ints of device
// memory; the exponent is written to *out (device memory) on `st`; nothing is read back.
int nspt_split_fit_rescale_dev(const double2* A, const double2* B, int N, int T, int batch, int* scratch, int* out,
                               cudaStream_t st, bool float_range = true);
size_t nspt_split_ws_grouped(const nspt_polymat_desc* d, int count, int S);
int nspt_split_mul_grouped(const nspt_polymat_desc* d, int count, int S, int log2r, void* ws, cudaStream_t st);
int nspt_split_autotune_grouped(const nspt_polymat_desc* d, int count, int S, void* ws, const char* cache_path,
                                int* chosen, cudaStream_t st);
size_t nspt_split_ws_langevin(int N, int T, int nb, int M, int S);
