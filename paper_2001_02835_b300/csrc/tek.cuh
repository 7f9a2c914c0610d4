#pragma once
#include <cuda_runtime.h>
#include <algorithm>
// S, F, Y: [nseries][T+1][N][N]; eta: [nseries][N][N]; imtr_ws: nseries*(T+1) doubles.
cudaError_t nspt_tek_drift(const double2* S, double* imtr_ws, const double2* eta, double2* F, double2* Y,
                           int N, int T, long long nseries, double eps, cudaStream_t st);
