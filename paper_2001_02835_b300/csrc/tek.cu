// Elementwise kernels of the TEK Langevin step and MD integrator (Eqs. 2-3 in
// rescaled time), of exp_star by Paterson-Stockmeyer (block combination), and
// of the Wilson-loop measurement (trace of the last product as a correlation),
// and of the unitarity projection (series dagger, order-0 identity terms).
//
// From the staple series S_mu (Eq. 3, plus sign on the second term) of every
// link of every stream:
//   F^(k) = i [S^(k) - S^(k)^H - Tr(S^(k) - S^(k)^H)/N]            (drift)
//   X^(0) = 0, X^(1) = eps F^(1) + sqrt(2 eps) eta, X^(k>=2) = eps F^(k)
//   Y = i X                                         (argument of exp_star)
// With s = sum_i Im S_ii, Tr(S - S^H) = 2 i s, so F = i (S - S^H) + (2 s/N) 1.
// A 32x32 tile of S and its mirror tile are staged in shared memory so that
// both the direct and the transposed reads are coalesced.
#include "common.cuh"
#include "tek.cuh"
#include "prof.cuh"

namespace {

// one warp per matrix: out[m] = sum_i Im S_m[i][i]
__global__ void imag_trace_kernel(const double2* __restrict__ S, double* __restrict__ out, int N, long long nmat) {
  const long long m = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (m >= nmat) return;
  const double2* Sm = S + m * N * N;
  double acc = 0.0;
  for (int i = lane; i < N; i += 32) acc += Sm[(long long)i * N + i].y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[m] = acc;
}

// grid: (tiles_j, tiles_i, nmat); block (32, 8)
__global__ void drift_kernel(const double2* __restrict__ S, const double* __restrict__ imtr,
                             const double2* __restrict__ eta, double2* __restrict__ F,
                             double2* __restrict__ Y, int N, int T, double eps, double noise_amp) {
  __shared__ double2 tA[32][33];   // S[i0+r][j0+c]
  __shared__ double2 tB[32][33];   // S[j0+r][i0+c]
  const long long m = blockIdx.z;  // matrix index = series*(T+1) + k
  const int k = (int)(m % (T + 1));
  const long long series = m / (T + 1);
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const double2* Sm = S + m * N * N;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = threadIdx.x;
    tA[r][c] = (i0 + r < N && j0 + c < N) ? Sm[(long long)(i0 + r) * N + j0 + c] : make_double2(0, 0);
    tB[r][c] = (j0 + r < N && i0 + c < N) ? Sm[(long long)(j0 + r) * N + i0 + c] : make_double2(0, 0);
  }
  __syncthreads();
  const double diag = 2.0 * imtr[m] / (double)N;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = threadIdx.x;
    const int i = i0 + r, j = j0 + c;
    if (i >= N || j >= N) continue;
    const double2 a = tA[r][c];       // S_ij
    const double2 bt = tB[c][r];      // S_ji
    // D = S_ij - conj(S_ji);  F = i D + diag * delta_ij
    const double dr = a.x - bt.x, di = a.y + bt.y;
    double2 f = make_double2(-di, dr);
    if (i == j) f.x += diag;
    const long long off = m * N * N + (long long)i * N + j;
    if (F) F[off] = f;
    // X = eps F (+ noise at order 1), X^(0) = 0; Y = i X
    double2 x = make_double2(eps * f.x, eps * f.y);
    if (k == 0) x = make_double2(0.0, 0.0);
    if (k == 1 && eta) {
      const double2 e = eta[series * N * N + (long long)i * N + j];
      x.x += noise_amp * e.x;
      x.y += noise_amp * e.y;
    }
    Y[off] = make_double2(-x.y, x.x);
  }
}

}  // namespace

cudaError_t nspt_tek_drift(const double2* S, double* imtr_ws, const double2* eta, double2* F, double2* Y,
                           int N, int T, long long nseries, double eps, cudaStream_t st) {
  const long long nmat = nseries * (T + 1);
  if (nmat == 0) return cudaSuccess;
  const int wpb = 8;
  ProfScope ps(NSPT_STAGE_TEK, st, 1 + (int)((nmat + 65534) / 65535));
  imag_trace_kernel<<<(unsigned)((nmat + wpb - 1) / wpb), wpb * 32, 0, st>>>(S, imtr_ws, N, nmat);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int tiles = (N + 31) / 32;
  if (nmat > 65535) {
    // chunk over matrices (grid z limit)
    for (long long m0 = 0; m0 < nmat; m0 += 65535 / (T + 1) * (T + 1)) {
      const long long chunk = std::min<long long>(65535 / (T + 1) * (T + 1), nmat - m0);
      const long long s0 = m0 / (T + 1);
      dim3 grid(tiles, tiles, (unsigned)chunk);
      drift_kernel<<<grid, dim3(32, 8), 0, st>>>(S + m0 * N * N, imtr_ws + m0, eta + s0 * N * N,
                                                 F ? F + m0 * N * N : nullptr, Y + m0 * N * N, N, T, eps,
                                                 sqrt(2.0 * eps));
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  dim3 grid(tiles, tiles, (unsigned)nmat);
  drift_kernel<<<grid, dim3(32, 8), 0, st>>>(S, imtr_ws, eta, F, Y, N, T, eps, sqrt(2.0 * eps));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Molecular dynamics (leapfrog, Eq. 3 with beta absorbed): momentum series with
// no order g^0, so order 0 of the drift is dropped.
// ---------------------------------------------------------------------------
namespace {

// P[s][0] = 0, P[s][1] = eta[s], P[s][k>=2] = 0
__global__ void md_refresh_kernel(double2* P, const double2* eta, int T, long long E, long long nseries) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = nseries * (T + 1) * E;
  if (i >= n) return;
  const long long e = i % E, k = (i / E) % (T + 1), s = i / (E * (T + 1));
  P[i] = (k == 1) ? eta[s * E + e] : make_double2(0.0, 0.0);
}

// P^(k) += a F^(k) for k >= 1; P^(0) = 0
__global__ void md_kick_kernel(double2* P, const double2* F, double a, int T, long long E, long long nseries) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = nseries * (T + 1) * E;
  if (i >= n) return;
  const long long k = (i / E) % (T + 1);
  if (k == 0) { P[i] = make_double2(0.0, 0.0); return; }
  const double2 f = F[i];
  P[i] = make_double2(fma(a, f.x, P[i].x), fma(a, f.y, P[i].y));
}

// Y = i eps P, Y^(0) = 0
__global__ void md_y_kernel(double2* Y, const double2* P, double eps, int T, long long E, long long nseries) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = nseries * (T + 1) * E;
  if (i >= n) return;
  const long long k = (i / E) % (T + 1);
  const double2 p = P[i];
  Y[i] = (k == 0) ? make_double2(0.0, 0.0) : make_double2(-eps * p.y, eps * p.x);
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

// Q^(k) = c_0 delta_{k0} 1 + sum_{i=1}^{m} c_i (Y^i)^(k) + prod^(k - shift) [k >= shift], k = 0..tq;
// series of T1 orders, nseries of them
__global__ void ps_combine_kernel(double2* __restrict__ Q, PsTerms t, int m, const double2* __restrict__ prod,
                                  int shift, int tq, int T1, int N, long long E, long long nseries) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = nseries * (tq + 1) * E;
  if (i >= n) return;
  const long long e = i % E, k = (i / E) % (tq + 1), sr = i / (E * (tq + 1));
  const long long idx = (sr * T1 + k) * E + e;
  double2 v = make_double2((k == 0 && e / N == e % N) ? t.c[0] : 0.0, 0.0);
  for (int j = 1; j <= m; ++j) {
    const double2 p = t.P[j][idx];
    v.x = fma(t.c[j], p.x, v.x);
    v.y = fma(t.c[j], p.y, v.y);
  }
  if (prod && k >= shift) {
    const double2 p = prod[(sr * T1 + k - shift) * E + e];
    v.x += p.x;
    v.y += p.y;
  }
  Q[idx] = v;
}

}  // namespace

cudaError_t nspt_ps_combine(double2* Q, const PsTerms& t, int m, const double2* prod, int shift, int tq, int T, int N,
                            long long nseries, cudaStream_t st) {
  if (m < 0 || m >= NSPT_PS_MAX_BLOCK || tq < 0 || tq > T) return cudaErrorInvalidValue;
  const long long E = (long long)N * N;
  ProfScope ps(NSPT_STAGE_TEK, st);
  ps_combine_kernel<<<blocks_for(nseries * (tq + 1) * E), 256, 0, st>>>(Q, t, m, prod, shift, tq, T + 1, N, E,
                                                                       nseries);
  return cudaGetLastError();
}

cudaError_t nspt_md_refresh(double2* P, const double2* eta, int T, long long E, long long nseries, cudaStream_t st) {
  ProfScope ps(NSPT_STAGE_TEK, st);
  md_refresh_kernel<<<blocks_for(nseries * (T + 1) * E), 256, 0, st>>>(P, eta, T, E, nseries);
  return cudaGetLastError();
}
cudaError_t nspt_md_kick(double2* P, const double2* F, double a, int T, long long E, long long nseries, cudaStream_t st) {
  ProfScope ps(NSPT_STAGE_TEK, st);
  md_kick_kernel<<<blocks_for(nseries * (T + 1) * E), 256, 0, st>>>(P, F, a, T, E, nseries);
  return cudaGetLastError();
}
cudaError_t nspt_md_y(double2* Y, const double2* P, double eps, int T, long long E, long long nseries, cudaStream_t st) {
  ProfScope ps(NSPT_STAGE_TEK, st);
  md_y_kernel<<<blocks_for(nseries * (T + 1) * E), 256, 0, st>>>(Y, P, eps, T, E, nseries);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Wilson loops: trace of the last star product without forming it,
// Tr[(L1 * L2^+)^(k)] = sum_{l <= k} sum_ij L1^(l)_ij conj(L2^(k-l)_ij).
// ---------------------------------------------------------------------------
namespace {

// grid (T+1, NSPT_TRACE_CHUNKS, batch), 256 threads: the partial sums
// t[b][k][ch] = zc * sum_{l<=k} sum_{e in chunk ch} L1^(l)_e conj(L2^(k-l)_e)
__global__ void __launch_bounds__(256) trace_corr_kernel(const double2* __restrict__ L1,
                                                         const double2* __restrict__ L2, double2* __restrict__ t,
                                                         double2 zc, int T, long long E) {
  const int k = blockIdx.x, ch = blockIdx.y, b = blockIdx.z;
  const long long csz = (E + NSPT_TRACE_CHUNKS - 1) / NSPT_TRACE_CHUNKS;
  const long long e0 = ch * csz, e1 = min(E, e0 + csz);
  const long long base = (long long)b * (T + 1) * E;
  double sr = 0.0, si = 0.0;
  for (int l = 0; l <= k; ++l) {
    const double2* x = L1 + base + (long long)l * E;
    const double2* y = L2 + base + (long long)(k - l) * E;
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const double2 u = x[e], v = y[e];
      sr = fma(u.x, v.x, fma(u.y, v.y, sr));   // Re(u conj(v))
      si = fma(u.y, v.x, fma(-u.x, v.y, si));  // Im(u conj(v))
    }
  }
  __shared__ double red[2][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = sr; red[1][threadIdx.x >> 5] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ar = 0.0, ai = 0.0;
    for (int w = 0; w < 8; ++w) { ar += red[0][w]; ai += red[1][w]; }
    t[((long long)b * (T + 1) + k) * NSPT_TRACE_CHUNKS + ch] =
        make_double2(zc.x * ar - zc.y * ai, zc.x * ai + zc.y * ar);
  }
}

// W[b][a][c][k] = scale * sum_p sum_ch (tr[p][a][c][b][k][ch] + conj(tr[p][c][a][b][k][ch]))
__global__ void wilson_combine_kernel(const double2* __restrict__ tr, double2* __restrict__ W, int nplanes, int amax,
                                      int batch, int T1, double scale) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = (long long)batch * amax * amax * T1;
  if (i >= n) return;
  const int k = (int)(i % T1);
  const int c = (int)((i / T1) % amax), a = (int)((i / ((long long)T1 * amax)) % amax);
  const int b = (int)(i / ((long long)T1 * amax * amax));
  double re = 0.0, im = 0.0;
  for (int p = 0; p < nplanes; ++p) {
    const double2* x = tr + (((((long long)p * amax + a) * amax + c) * batch + b) * T1 + k) * NSPT_TRACE_CHUNKS;
    const double2* y = tr + (((((long long)p * amax + c) * amax + a) * batch + b) * T1 + k) * NSPT_TRACE_CHUNKS;
    for (int ch = 0; ch < NSPT_TRACE_CHUNKS; ++ch) {
      re += x[ch].x + y[ch].x;
      im += x[ch].y - y[ch].y;
    }
  }
  W[i] = make_double2(scale * re, scale * im);
}

}  // namespace

cudaError_t nspt_trace_corr(const double2* L1, const double2* L2, double2* t, double2 zc, int T, long long E,
                            int batch, cudaStream_t st) {
  ProfScope ps(NSPT_STAGE_TEK, st);
  trace_corr_kernel<<<dim3(T + 1, NSPT_TRACE_CHUNKS, batch), 256, 0, st>>>(L1, L2, t, zc, T, E);
  return cudaGetLastError();
}

cudaError_t nspt_wilson_combine(const double2* tr, double2* W, int nplanes, int amax, int batch, int T, double scale,
                                cudaStream_t st) {
  ProfScope ps(NSPT_STAGE_TEK, st);
  const long long n = (long long)batch * amax * amax * (T + 1);
  wilson_combine_kernel<<<blocks_for(n), 256, 0, st>>>(tr, W, nplanes, amax, batch, T + 1, scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Unitarity projection helpers: the series dagger (U^+)^(k) = (U^(k))^H of every
// coefficient, and order-0 identity terms.
// ---------------------------------------------------------------------------
namespace {

// grid (ceil(N/32), ceil(N/32), min(nmat, 65535)), block (32, 8): one 32 x 32 tile of each
// matrix (matrices z, z + gridDim.z, ...) through shared memory, rows read and written
// coalesced
__global__ void __launch_bounds__(256) dagger_kernel(const double2* __restrict__ X, double2* __restrict__ Y, int N,
                                                     long long nmat) {
  __shared__ double2 tile[32][33];
  const long long E = (long long)N * N;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (long long m = blockIdx.z; m < nmat; m += gridDim.z) {
    const double2* Xm = X + m * E;
    double2* Ym = Y + m * E;
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int i = by + r, j = bx + threadIdx.x;
      if (i < N && j < N) tile[r][threadIdx.x] = Xm[(long long)i * N + j];
    }
    __syncthreads();
    // Y[j][i] = conj(X[i][j]): row j = bx + r of Y, column i = by + threadIdx.x
    for (int r = threadIdx.y; r < 32; r += 8) {
      const int j = bx + r, i = by + threadIdx.x;
      if (i < N && j < N) {
        const double2 v = tile[threadIdx.x][r];
        Ym[(long long)j * N + i] = make_double2(v.x, -v.y);
      }
    }
    __syncthreads();
  }
}

// order 0 of every series: X[s][0] = c 1 (set) or X[s][0] += c 1 (add)
__global__ void order0_identity_kernel(double2* X, int T1, int N, long long nseries, double c, int set) {
  const long long E = (long long)N * N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseries * E) return;
  const long long s = i / E, e = i % E;
  double2* x = X + s * T1 * E + e;
  const bool diag = (e / N) == (e % N);
  if (set) *x = make_double2(diag ? c : 0.0, 0.0);
  else if (diag) x->x += c;
}

}  // namespace

cudaError_t nspt_series_dagger(const double2* X, double2* Y, int N, long long nmat, cudaStream_t st) {
  if (nmat <= 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  const unsigned nt = (unsigned)((N + 31) / 32);
  dim3 grid(nt, nt, (unsigned)std::min<long long>(nmat, 65535));
  dagger_kernel<<<grid, dim3(32, 8), 0, st>>>(X, Y, N, nmat);
  return cudaGetLastError();
}

cudaError_t nspt_series_order0_identity(double2* X, int T, int N, long long nseries, double c, int set,
                                        cudaStream_t st) {
  if (nseries <= 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  order0_identity_kernel<<<blocks_for(nseries * (long long)N * N), 256, 0, st>>>(X, T + 1, N, nseries, c, set);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// U(1) phase removal after the unitarity projection: the derivative series, Im Tr
// per order, the phase series exp(-i a / N), and the scalar-series product
// W_k = sum_j V_j s_(k-j).
// ---------------------------------------------------------------------------
namespace {

// derivative series Y_j = (j + 1) V_(j+1), j < T, Y_T = 0, of every series
__global__ void deriv_series_kernel(const double2* __restrict__ V, double2* __restrict__ Y, int T, int N,
                                    long long nseries) {
  const long long E = (long long)N * N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseries * (T + 1) * E) return;
  const long long e = i % E, j = (i / E) % (T + 1), q = i / ((T + 1) * E);
  const double2* v = V + q * (T + 1) * E + e;
  Y[i] = (j < T) ? make_double2((j + 1) * v[(j + 1) * E].x, (j + 1) * v[(j + 1) * E].y) : make_double2(0.0, 0.0);
}

// one thread per series: the phase a_k = t_(k-1) / k (t = Im Tr(V^+ * V') per order, so that
// a' = t), and s_0 = 1, s_k = (1/k) sum_{j=1}^{k} j b_j s_(k-j) with b_j = -i a_j / N (the
// coefficients of exp(b), from (exp b)' = b' exp b); j b_j = -i t_(j-1) / N
__global__ void phase_series_kernel(const double* __restrict__ t, double2* __restrict__ sr, int T, int N,
                                    long long nseries) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nseries) return;
  const double* tq = t + q * (T + 1);
  double2* s = sr + q * (T + 1);
  s[0] = make_double2(1.0, 0.0);
  for (int k = 1; k <= T; ++k) {
    double re = 0.0, im = 0.0;
    for (int j = 1; j <= k; ++j) {
      // j b_j s_(k-j) = (-i x)(u + i v) = x v - i x u, x = j a_j / N = t_(j-1) / N
      const double x = tq[j - 1] / N;
      const double2 u = s[k - j];
      re += x * u.y;
      im -= x * u.x;
    }
    s[k] = make_double2(re / k, im / k);
  }
}

// in place, one thread per entry of every series: V_k <- sum_{j<=k} V_j s_(k-j), k = T..1
// (descending, so every V_j read is still the input); order 0 is unchanged since s_0 = 1
__global__ void scalar_series_mul_kernel(double2* __restrict__ V, const double2* __restrict__ sr, int T, int N,
                                         long long nseries) {
  const long long E = (long long)N * N;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nseries * E) return;
  const long long q = i / E, e = i % E;
  double2* v = V + q * (T + 1) * E + e;
  const double2* s = sr + q * (T + 1);
  for (int k = T; k >= 1; --k) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j <= k; ++j) {
      const double2 x = v[(long long)j * E], y = s[k - j];
      re += x.x * y.x - x.y * y.y;
      im += x.x * y.y + x.y * y.x;
    }
    v[(long long)k * E] = make_double2(re, im);
  }
}

}  // namespace

cudaError_t nspt_series_derivative(const double2* V, double2* Y, int T, int N, long long nseries, cudaStream_t st) {
  if (nseries <= 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  deriv_series_kernel<<<blocks_for(nseries * (T + 1) * (long long)N * N), 256, 0, st>>>(V, Y, T, N, nseries);
  return cudaGetLastError();
}

cudaError_t nspt_series_imag_trace(const double2* X, double* out, int N, long long nmat, cudaStream_t st) {
  if (nmat <= 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  imag_trace_kernel<<<(unsigned)((nmat + 7) / 8), 256, 0, st>>>(X, out, N, nmat);
  return cudaGetLastError();
}

cudaError_t nspt_series_remove_phase(double2* V, const double* t, double2* sr, int T, int N, long long nseries,
                                     cudaStream_t st) {
  if (nseries <= 0 || T < 1) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  phase_series_kernel<<<(unsigned)((nseries + 127) / 128), 128, 0, st>>>(t, sr, T, N, nseries);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scalar_series_mul_kernel<<<blocks_for(nseries * (long long)N * N), 256, 0, st>>>(V, sr, T, N, nseries);
  return cudaGetLastError();
}
