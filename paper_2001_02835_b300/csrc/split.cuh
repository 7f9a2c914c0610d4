// Split-precision form of the product path (tensor-core mode GEMMs).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

int nspt_split_init();
size_t nspt_split_ws_mul(int N, int T, int batch, int M, int slices);
size_t nspt_split_ws_bwd(int N, int T, int batch, int M, int slices);
int nspt_split_mul(int N, int T, int batch, int M, int slices, int log2r, bool rescale_auto, const double2* A,
                   const double2* B, double2* C, void* ws, cudaStream_t st);
int nspt_split_bwd(int N, int T, int batch, int M, int slices, int log2r, const double2* A, const double2* B,
                   const double2* G, double2* gA, double2* gB, void* ws, cudaStream_t st);
int nspt_split_langevin(int N, int T, int batch, int M, int slices, double2* U, const double2* eta, double2* F,
                        int flux, double eps, void* ws, cudaStream_t st);
