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

// exp_star(Y) (Y^(0) = 0) by Paterson-Stockmeyer in the truncated ring:
// Y^2 .. Y^s, then Horner in Y^s, Q_j = B_j + Y^s Q_{j+1}, B_j = sum_{i<s} Y^i / (js+i)!.
// Block size s <= NSPT_PS_MAX_BLOCK minimising the mode-GEMM count when every
// product runs at its own truncation (Y^k starts at order k).
constexpr int NSPT_PS_MAX_BLOCK = 8;
inline int nspt_pow2_at_least(int x) {
  int m = 1;
  while (m < x) m <<= 1;
  return m;
}
inline long long nspt_ps_cost(int T, int s) {
  long long c = 0;
  for (int k = 2; k <= s; ++k) c += nspt_pow2_at_least(2 * (T - k + 1));
  for (int j = T / s - 1; j >= 0; --j) c += nspt_pow2_at_least(2 * (T - s * (j + 1) + 1));
  return c;
}
inline int nspt_ps_block(int T) {
  int best = 1;
  for (int s = 2; s <= NSPT_PS_MAX_BLOCK && s <= T; ++s)
    if (nspt_ps_cost(T, s) < nspt_ps_cost(T, best)) best = s;
  return best;
}
// Truncation to read the left operand of a Paterson-Stockmeyer product at: the largest
// truncation among the products of the same phase that share its transform length, so that
// one transform of the operand serves them all.  Powers: Y^k = Y * Y^(k-1) to order T - k
// (k = 2..s); Horner: Y^s Q_{j+1} to order T - s (j + 1) (j = T/s - 1 .. 0).
inline int nspt_ps_power_ta(int T, int s, int k) {
  const int M = nspt_pow2_at_least(2 * (T - k + 1));
  int ta = T - k;
  for (int k2 = 2; k2 <= s; ++k2)
    if (nspt_pow2_at_least(2 * (T - k2 + 1)) == M && T - k2 > ta) ta = T - k2;
  return ta;
}
inline int nspt_ps_horner_ta(int T, int s, int j) {
  const int M = nspt_pow2_at_least(2 * (T - s * (j + 1) + 1));
  int ta = T - s * (j + 1);
  for (int j2 = T / s - 1; j2 >= 0; --j2)
    if (nspt_pow2_at_least(2 * (T - s * (j2 + 1) + 1)) == M && T - s * (j2 + 1) > ta) ta = T - s * (j2 + 1);
  return ta;
}
// temporary link-series slots (units of batch x (T+1) x N^2 entries) of a step's workspace:
// 18 for the staple pipeline, reused by exp_star for 4 per power Y^2..Y^s plus 4 for the
// Horner product
inline int nspt_tmp_series(int T) {
  const int ps = 4 * (nspt_ps_block(T) > 1 ? nspt_ps_block(T) : 1);
  return ps > 18 ? ps : 18;
}
// terms of one block: P[i] = Y^i (i >= 1; P[0] unused), c[i] its coefficient, c[0] that of 1
struct PsTerms {
  const double2* P[NSPT_PS_MAX_BLOCK];
  double c[NSPT_PS_MAX_BLOCK];
};
// Q^(k) = c_0 delta_{k0} 1 + sum_{i=1}^{m} c_i (Y^i)^(k) + prod^(k - shift) (k >= shift), k = 0..tq
cudaError_t nspt_ps_combine(double2* Q, const PsTerms& t, int m, const double2* prod, int shift, int tq, int T, int N,
                            long long nseries, cudaStream_t st);

// Wilson loops: t[b][k][ch] = zc sum_{l<=k} <L1^(l), L2^(k-l)>_ch, the sum over chunk ch
// of the entries (summed over ch: zc Tr[(L1 * L2^+)^(k)]) for series L1, L2 [batch][T+1][E];
// and W[b][a][c][k] = scale sum_p sum_ch (tr[p][a][c][b][k][ch] + conj(tr[p][c][a][b][k][ch]))
// from tr [nplanes][amax][amax][batch][T+1][NSPT_TRACE_CHUNKS]
constexpr int NSPT_TRACE_CHUNKS = 64;
cudaError_t nspt_trace_corr(const double2* L1, const double2* L2, double2* t, double2 zc, int T, long long E,
                            int batch, cudaStream_t st);
cudaError_t nspt_wilson_combine(const double2* tr, double2* W, int nplanes, int amax, int batch, int T, double scale,
                                cudaStream_t st);

// unitarity projection: Y[m] = X[m]^H for nmat N x N matrices (Y must not overlap X);
// order 0 of each of nseries series [T+1][N][N]: X^(0) = c 1 (set != 0) or X^(0) += c 1
cudaError_t nspt_series_dagger(const double2* X, double2* Y, int N, long long nmat, cudaStream_t st);
cudaError_t nspt_series_order0_identity(double2* X, int T, int N, long long nseries, double c, int set,
                                        cudaStream_t st);
// U(1) phase removal: Y_j = (j + 1) V_(j+1) (Y_T = 0); out[m] = sum_i Im X[m]_ii for nmat
// matrices; V_k <- sum_j V_j s_(k-j) in place with s = exp(-i a / N), a_k = t_(k-1) / k for
// t [nseries][T+1] (t_k = Im Tr(V^+ * V')_k), sr [nseries][T+1] scratch
cudaError_t nspt_series_derivative(const double2* V, double2* Y, int T, int N, long long nseries, cudaStream_t st);
cudaError_t nspt_series_imag_trace(const double2* X, double* out, int N, long long nmat, cudaStream_t st);
cudaError_t nspt_series_remove_phase(double2* V, const double* a, double2* sr, int T, int N, long long nseries,
                                     cudaStream_t st);
