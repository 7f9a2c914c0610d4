#pragma once
#include <cuda_runtime.h>
#include <algorithm>
// S, F, Y: [nseries][T+1][N][N]; eta: [nseries][N][N]; imtr_ws: nseries*(T+1) doubles.
cudaError_t nspt_tek_drift(const double2* S, double* imtr_ws, const double2* eta, double2* F, double2* Y,
                           int N, int T, long long nseries, double eps, cudaStream_t st);
// molecular dynamics helpers: P, F, Y [nseries][T+1][E]; eta [nseries][E]
cudaError_t nspt_md_refresh(double2* P, const double2* eta, int T, long long E, long long nseries, cudaStream_t st);
cudaError_t nspt_md_kick(double2* P, const double2* F, double a, int T, long long E, long long nseries, cudaStream_t st);
cudaError_t nspt_md_y(double2* Y, const double2* P, double eps, int T, long long E, long long nseries, cudaStream_t st);
// phases of one Langevin / MD evaluation
enum { NSPT_LMODE_STEP = 0, NSPT_LMODE_DRIFT = 1, NSPT_LMODE_UPDATE = 2 };
