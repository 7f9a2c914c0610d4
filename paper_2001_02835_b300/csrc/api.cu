// C ABI, planner and orchestration of the NSPT polynomial-matrix library.
//
// Every entry point validates its arguments on the host, carves the caller's
// workspace, and enqueues kernels on the caller's stream.  No device memory is
// allocated; nothing is synchronised or read back except where a declaration
// says so (the automatic per-order rescale, the tile autotuner, the status
// read).  The host-buffer product creates its two copy streams and its events
// once per device.  The FFT-CONV orchestration follows Sec. 2 Steps 1-5; the
// Langevin step and the MD integrator follow Eqs. 1-3 (see include/nspt.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "zgemm64.cuh"
#include "tek.cuh"
#include "split.cuh"
#include "prof.cuh"
#include "split_gemm.cuh"
#include <algorithm>

namespace {
thread_local cudaError_t g_last_cuda = cudaSuccess;
thread_local const int* g_dev_log2r = nullptr;

int next_pow2(int x) {
  int m = 1;
  while (m < x) m <<= 1;
  return m;
}

struct Plan {
  int N, T, batch;
  long long E;
  int algo, prec, M, slices, log2r;
  bool rescale_auto;
  int cm;  // split form: real products per complex product (4, or 3 for 3M)
};

// allow_3m: the entry point takes complex_mode = 3 (the plain product)
// plan of the Wilson loops (no workspace-query constant of its own)
constexpr int kPlanWilson = 100;

// op: the NSPT_OP_* call the plan is for (kPlanWilson: the Wilson loops; -1: a plan used inside
// another entry point).  The product (NSPT_OP_MUL) alone takes the 3M variant; the entry points
// whose products all go through the product call (the product, its backward, the unitarity
// projection and the Wilson loops) take the naive form of the split products
int make_plan(int N, int T, int batch, const nspt_opts* o, Plan* p, int op = -1) {
  const bool product = op == NSPT_OP_MUL;
  const bool naive_split_ok = product || op == NSPT_OP_MUL_BACKWARD || op == NSPT_OP_UNITARIZE ||
                              op == kPlanWilson;
  nspt_opts d;
  nspt_opts_default(&d);
  if (!o) o = &d;
  if (N < 1 || T < 0 || batch < 1 || N > 4096 || T > 255) return NSPT_ERR_ARG;
  p->N = N; p->T = T; p->batch = batch; p->E = (long long)N * N;
  p->algo = o->algo;
  p->prec = o->prec;
  if (p->prec != NSPT_PREC_FP64 && p->prec != NSPT_PREC_SPLIT) return NSPT_ERR_ARG;
  // auto: naive below T = 3, where the transforms cost more than the few pair products save;
  // the split form's naive products exist for nspt_polymat_mul only
  if (p->algo == NSPT_ALGO_AUTO)
    p->algo = (T >= 3 || (p->prec == NSPT_PREC_SPLIT && !naive_split_ok)) ? NSPT_ALGO_FFT : NSPT_ALGO_NAIVE;
  if (p->algo != NSPT_ALGO_NAIVE && p->algo != NSPT_ALGO_FFT) return NSPT_ERR_ARG;
  p->M = o->fft_len ? o->fft_len : next_pow2(2 * (T + 1));
  if (ilog2_exact(p->M) < 0 || p->M < 2 * (T + 1) || p->M > 512) return NSPT_ERR_ARG;
  p->slices = o->slices ? o->slices : 6;
  if (p->slices < 2 || p->slices > 8) return NSPT_ERR_ARG;
  p->cm = 4;
  if (o->complex_mode == 3) {
    // 3M: split-form FFT-CONV products with S <= 6 and row-form slicing (N <= 512)
    if (!product || p->prec != NSPT_PREC_SPLIT || p->algo != NSPT_ALGO_FFT || p->slices > 6 || N > 512)
      return NSPT_ERR_UNSUPPORTED;
    p->cm = 3;
  } else if (o->complex_mode != 0 && o->complex_mode != 4) {
    return NSPT_ERR_UNSUPPORTED;
  }
  p->rescale_auto = (o->rescale_log2r == NSPT_RESCALE_AUTO);
  p->log2r = p->rescale_auto ? 0 : o->rescale_log2r;
  if (!p->rescale_auto && (p->log2r < -60 || p->log2r > 60)) return NSPT_ERR_ARG;
  if (p->prec == NSPT_PREC_SPLIT && p->algo == NSPT_ALGO_NAIVE && !naive_split_ok) return NSPT_ERR_UNSUPPORTED;
  // the split form's slicers hold up to 8 spectrum rows of N entries in shared memory
  if (p->prec == NSPT_PREC_SPLIT && N > 1024) return NSPT_ERR_UNSUPPORTED;
  return NSPT_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  if (!a || !b) return false;
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

// --------------------------------------------------------------------------
// FP64 building blocks
// --------------------------------------------------------------------------
ZgemmParams zg(int kind, const double2* A, long long sA, const double2* B, long long sB, double2* C,
               long long sC, int N, int nmat, int T) {
  ZgemmParams P;
  memset(&P, 0, sizeof(P));
  P.A = A; P.B = B; P.C = C; P.sA = sA; P.sB = sB; P.sC = sC;
  P.N = N; P.kind = kind; P.nmat = nmat; P.T = T;
  P.alpha = make_double2(1.0, 0.0);
  return P;
}

__global__ void add_identity_kernel(double2* X, long long stride_mats, int N, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count * N) return;
  const long long s = i / N;
  const int d = (int)(i % N);
  X[s * stride_mats * N * N + (long long)d * N + d].x += 1.0;
}

cudaError_t add_identity(double2* X, long long stride_mats, int N, long long count, cudaStream_t st) {
  const long long n = count * N;
  if (n == 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  add_identity_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, stride_mats, N, count);
  return cudaGetLastError();
}

#define TRY(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { g_last_cuda = _e; return NSPT_ERR_CUDA; } } while (0)

// --- forward product, FP64 ---
size_t ws_mul(const Plan& p) {
  if (p.algo == NSPT_ALGO_NAIVE)
    return p.prec == NSPT_PREC_SPLIT ? nspt_split_ws_naive(p.N, p.T, p.batch, p.slices) : 0;
  const size_t spec = (size_t)p.batch * p.M * p.E * sizeof(double2);
  if (p.prec == NSPT_PREC_FP64) return 3 * ((spec + 255) & ~(size_t)255) + 2 * 513 * sizeof(int);  // + fit scratch
  return nspt_split_ws_mul(p.N, p.T, p.batch, p.M, p.slices, p.cm);
}

int mul_fp64(const Plan& p, const double2* A, const double2* B, double2* C, void* ws, cudaStream_t st) {
  const int N = p.N, T = p.T, b = p.batch, M = p.M;
  if (p.algo == NSPT_ALGO_NAIVE) {
    ZgemmParams P = zg(ZG_CONV, A, T + 1, B, T + 1, C, T + 1, N, T + 1, T);
    TRY(nspt_zgemm64(P, b, st));
    return NSPT_OK;
  }
  WsCarver w(ws, SIZE_MAX);
  double2* At = w.take<double2>((size_t)b * M * p.E);
  double2* Bt = w.take<double2>((size_t)b * M * p.E);
  double2* Ct = w.take<double2>((size_t)b * M * p.E);
  int* fit = w.take<int>(2 * 513);
  // per-order rescale A_k, B_k -> r^k A_k, r^k B_k, undone on C (exact; as in the split form)
  int lr = p.log2r;
  int* dlr = nullptr;  // fitted exponent in device memory (the last word of the fit scratch)
  if (p.rescale_auto) {
    dlr = fit + 2 * 513 - 1;
    const int rc = nspt_split_fit_rescale_dev(A, B, N, T, b, fit, dlr, st, false);
    if (rc) return rc;
    lr = 1;
  }
  NsptDevLog2r scope(dlr);
  TRY(nspt_fft_fwd64(A, T + 1, At, (int)p.E, T, b, M, 0, lr, st));
  TRY(nspt_fft_fwd64(B, T + 1, Bt, (int)p.E, T, b, M, 0, lr, st));
  ZgemmParams P = zg(ZG_MODE, At, M, Bt, M, Ct, M, N, M, T);
  TRY(nspt_zgemm64(P, b, st));
  TRY(nspt_fft_inv64(Ct, C, T + 1, (int)p.E, N, T, b, M, 0, lr, 1.0, 0, st));
  return NSPT_OK;
}

// --- backward, FP64 ---
size_t ws_bwd(const Plan& p) {
  if (p.algo == NSPT_ALGO_NAIVE)
    return p.prec == NSPT_PREC_SPLIT ? nspt_split_ws_naive(p.N, p.T, p.batch, p.slices) : 0;
  const size_t spec = (size_t)p.batch * p.M * p.E * sizeof(double2);
  if (p.prec == NSPT_PREC_FP64) return 4 * ((spec + 255) & ~(size_t)255);
  return nspt_split_ws_bwd(p.N, p.T, p.batch, p.M, p.slices);
}

int bwd_fp64(const Plan& p, const double2* A, const double2* B, const double2* G, double2* gA, double2* gB,
             void* ws, cudaStream_t st) {
  const int N = p.N, T = p.T, b = p.batch, M = p.M;
  if (p.algo == NSPT_ALGO_NAIVE) {
    if (gA) {
      ZgemmParams P = zg(ZG_CORR_A, G, T + 1, B, T + 1, gA, T + 1, N, T + 1, T);
      P.opB = 1;
      TRY(nspt_zgemm64(P, b, st));
    }
    if (gB) {
      ZgemmParams P = zg(ZG_CORR_B, A, T + 1, G, T + 1, gB, T + 1, N, T + 1, T);
      P.opA = 1;
      TRY(nspt_zgemm64(P, b, st));
    }
    return NSPT_OK;
  }
  WsCarver w(ws, SIZE_MAX);
  double2* At = w.take<double2>((size_t)b * M * p.E);
  double2* Bt = w.take<double2>((size_t)b * M * p.E);
  double2* Gt = w.take<double2>((size_t)b * M * p.E);
  double2* Xt = w.take<double2>((size_t)b * M * p.E);
  TRY(nspt_fft_fwd64(G, T + 1, Gt, (int)p.E, T, b, M, 0, 0, st));
  if (gA) {
    TRY(nspt_fft_fwd64(B, T + 1, Bt, (int)p.E, T, b, M, 0, 0, st));
    ZgemmParams P = zg(ZG_MODE, Gt, M, Bt, M, Xt, M, N, M, T);
    P.opB = 1;
    TRY(nspt_zgemm64(P, b, st));
    TRY(nspt_fft_inv64(Xt, gA, T + 1, (int)p.E, N, T, b, M, 0, 0, 1.0, 0, st));
  }
  if (gB) {
    TRY(nspt_fft_fwd64(A, T + 1, At, (int)p.E, T, b, M, 0, 0, st));
    ZgemmParams P = zg(ZG_MODE, At, M, Gt, M, Xt, M, N, M, T);
    P.opA = 1;
    TRY(nspt_zgemm64(P, b, st));
    TRY(nspt_fft_inv64(Xt, gB, T + 1, (int)p.E, N, T, b, M, 0, 0, 1.0, 0, st));
  }
  return NSPT_OK;
}

// --------------------------------------------------------------------------
// Langevin step (Eqs. 1-3).  The engine hides the naive / FFT choice behind
// "operands" (a series for the naive form, a spectrum for the FFT form) and
// "accumulators" (a series / a spectrum summed over terms).
// --------------------------------------------------------------------------
const int kPairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
int pair_index(int a, int b) {  // a < b
  for (int i = 0; i < 6; ++i)
    if (kPairs[i][0] == a && kPairs[i][1] == b) return i;
  return -1;
}
int ordered_index(int mu, int nu) { return mu * 3 + (nu < mu ? nu : nu - 1); }  // 0..11

size_t ws_langevin_core(const Plan& p) {
  if (p.prec == NSPT_PREC_SPLIT) return nspt_split_ws_langevin(p.N, p.T, p.batch, p.M, p.slices);
  const long long E = p.E;
  const long long T1 = p.T + 1, M = p.M;
  size_t mats;
  if (p.algo == NSPT_ALGO_FFT) {
    // spectra: U(4) PQ(18) Acc(18) In(4); series: tmp S(4) Y(4) R(8); exp spectra Y,R,C (12)
    mats = (size_t)(4 + 18 + 18 + 4 + 12) * M + (size_t)(nspt_tmp_series(p.T) + 4 + 4 + 8) * T1;
  } else {
    // series: P1(6) Q(12) inner(4) S(4) Y(4) R(8) U0(4)
    mats = (size_t)(6 + 12 + 4 + 4 + 4 + 8 + 4) * T1;
  }
  // + up to 255 bytes of alignment per carved buffer (at most 16 buffers)
  return (size_t)p.batch * mats * E * sizeof(double2) + (size_t)p.batch * 4 * T1 * sizeof(double) + 16 * 256;
}

// a TEK step's workspace: the pipeline's, then the scratch of the per-order rescale fit
constexpr size_t kFitScratch = 2 * 513 * sizeof(int);
size_t ws_langevin(const Plan& p) { return ((ws_langevin_core(p) + 255) & ~(size_t)255) + kFitScratch; }
void* fit_scratch(const Plan& p, void* ws) { return (char*)ws + ((ws_langevin_core(p) + 255) & ~(size_t)255); }

// exponent of the per-order rescale of a TEK step's order transforms (FFT forms only): fixed, or
// with NSPT_RESCALE_AUTO fitted on the device to the per-order maxima of A and B; then *lr = 1
// and *dlr points at the fitted exponent, which the caller hands to the transforms through an
// NsptDevLog2r scope
int tek_log2r(const Plan& p, const double2* A, const double2* B, void* ws, cudaStream_t st, int* lr,
              const int** dlr) {
  *lr = 0;
  *dlr = nullptr;
  if (p.algo != NSPT_ALGO_FFT) return NSPT_OK;
  if (!p.rescale_auto) { *lr = p.log2r; return NSPT_OK; }
  int* scratch = (int*)fit_scratch(p, ws);
  int* out = scratch + 2 * 513 - 1;
  const int rc = nspt_split_fit_rescale_dev(A, B, p.N, p.T, p.batch * 4, scratch, out, st, p.prec == NSPT_PREC_SPLIT);
  if (rc) return rc;
  *lr = 1;
  *dlr = out;
  return NSPT_OK;
}

// mode: NSPT_LMODE_STEP (drift, increment, update), NSPT_LMODE_DRIFT (drift F only),
// NSPT_LMODE_UPDATE (U <- exp_star(Yin) U with the caller's Yin = i X, X^(0) = 0)
int langevin_fp64(const Plan& p, double2* U, const double2* eta, double2* F, int flux, double eps, void* ws,
                  cudaStream_t st, int mode = NSPT_LMODE_STEP, const double2* Yin = nullptr, int lr = 0) {
  const int N = p.N, T = p.T, nb = p.batch;
  const long long E = p.E, T1 = T + 1;
  int L = (int)llround(sqrt((double)N));
  // twist phases z[mu][nu] = exp(2 pi i flux eps_{mu nu} / L), computed on the host
  double2 z[4][4];
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      const double sgn = (mu < nu) ? 1.0 : -1.0;
      const double ang = 2.0 * M_PI * flux * sgn / L;
      z[mu][nu] = (mu == nu) ? make_double2(0, 0) : make_double2(cos(ang), sin(ang));
    }
  WsCarver w(ws, ws_langevin_core(p));
  if (p.algo == NSPT_ALGO_FFT) {
    const int M = p.M;
    double2* specU = w.take<double2>((size_t)nb * 4 * M * E);
    double2* specPQ = w.take<double2>((size_t)nb * 18 * M * E);
    double2* specAcc = w.take<double2>((size_t)nb * 18 * M * E);
    double2* specIn = w.take<double2>((size_t)nb * 4 * M * E);
    double2* serTmp = w.take<double2>((size_t)nb * nspt_tmp_series(T) * T1 * E);
    double2* serS = w.take<double2>((size_t)nb * 4 * T1 * E);
    double2* serY = w.take<double2>((size_t)nb * 4 * T1 * E);
    double2* serR[2] = {w.take<double2>((size_t)nb * 4 * T1 * E), w.take<double2>((size_t)nb * 4 * T1 * E)};
    double2* spY = w.take<double2>((size_t)nb * 4 * M * E);
    double2* spR = w.take<double2>((size_t)nb * 4 * M * E);
    double2* spC = w.take<double2>((size_t)nb * 4 * M * E);
    double* imtr = w.take<double>((size_t)nb * 4 * T1);
    if (!w.fits()) return NSPT_ERR_WORKSPACE;  // the carve outgrew ws_langevin_core: a sizing bug
    const long long sm = (long long)M;  // matrices per spectrum
    // 1. spectra of the four links
    TRY(nspt_fft_fwd64(U, T1, specU, (int)E, T, nb * 4, M, 0, lr, st));
    auto specOf = [&](double2* base, int slot) { return base + (long long)slot * M * E; };
    if (mode != NSPT_LMODE_UPDATE) {
    // 2. P1(mu,nu) = U_nu * U_mu^+ (mu<nu), Q(mu,nu) = U_mu * U_nu (mu != nu)
    for (int i = 0; i < 6; ++i) {
      const int mu = kPairs[i][0], nu = kPairs[i][1];
      ZgemmParams P = zg(ZG_MODE, specOf(specU, nu), 4 * sm, specOf(specU, mu), 4 * sm, specOf(specAcc, i),
                         18 * sm, N, M, T);
      P.opB = 1; P.revB = 1;
      TRY(nspt_zgemm64(P, nb, st));
    }
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = 0; nu < 4; ++nu) {
        if (mu == nu) continue;
        ZgemmParams P = zg(ZG_MODE, specOf(specU, mu), 4 * sm, specOf(specU, nu), 4 * sm,
                           specOf(specAcc, 6 + ordered_index(mu, nu)), 18 * sm, N, M, T);
        TRY(nspt_zgemm64(P, nb, st));
      }
    // truncate (Step 5) and return to the frequency domain
    TRY(nspt_fft_inv64(specAcc, serTmp, T1, (int)E, N, T, nb * 18, M, 0, lr, 1.0, 0, st));
    TRY(nspt_fft_fwd64(serTmp, T1, specPQ, (int)E, T, nb * 18, M, 0, lr, st));
    // 3. inner_mu = sum_nu z P1(mu,nu) U_nu^+ + conj(z) P2(mu,nu) U_nu,  P2(mu,nu) = Q(mu,nu)^+
    for (int mu = 0; mu < 4; ++mu) {
      bool first = true;
      for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        {
          const int pi = (mu < nu) ? pair_index(mu, nu) : pair_index(nu, mu);
          ZgemmParams P = zg(ZG_MODE, specOf(specPQ, pi), 18 * sm, specOf(specU, nu), 4 * sm, specOf(specIn, mu),
                             4 * sm, N, M, T);
          if (mu > nu) { P.opA = 1; P.revA = 1; }
          P.opB = 1; P.revB = 1;
          P.alpha = z[mu][nu];
          P.accumulate = first ? 0 : 1;
          first = false;
          TRY(nspt_zgemm64(P, nb, st));
        }
        {
          ZgemmParams P = zg(ZG_MODE, specOf(specPQ, 6 + ordered_index(mu, nu)), 18 * sm, specOf(specU, nu), 4 * sm,
                             specOf(specIn, mu), 4 * sm, N, M, T);
          P.opA = 1; P.revA = 1;
          P.alpha = make_double2(z[mu][nu].x, -z[mu][nu].y);
          P.accumulate = 1;
          TRY(nspt_zgemm64(P, nb, st));
        }
      }
    }
    // truncate inner_mu and return it to the frequency domain (in place in specIn)
    TRY(nspt_fft_inv64(specIn, serTmp, T1, (int)E, N, T, nb * 4, M, 0, lr, 1.0, 0, st));
    TRY(nspt_fft_fwd64(serTmp, T1, specIn, (int)E, T, nb * 4, M, 0, lr, st));
    // 4. S_mu = U_mu * inner_mu
    for (int mu = 0; mu < 4; ++mu) {
      ZgemmParams P = zg(ZG_MODE, specOf(specU, mu), 4 * sm, specOf(specIn, mu), 4 * sm, specOf(specAcc, mu), 4 * sm,
                         N, M, T);
      TRY(nspt_zgemm64(P, nb, st));
    }
    TRY(nspt_fft_inv64(specAcc, serS, T1, (int)E, N, T, nb * 4, M, 0, lr, 1.0, 0, st));
    // 5. drift and the Langevin increment Y = i X
    TRY(nspt_tek_drift(serS, imtr, eta, F, serY, N, T, (long long)nb * 4, eps, st));
    }
    if (mode == NSPT_LMODE_DRIFT) return NSPT_OK;
    const double2* Ysrc = (mode == NSPT_LMODE_UPDATE) ? Yin : serY;
    // 6. exp_star(Y) by Paterson-Stockmeyer in the truncated ring (Y^(0) = 0, so Y^k
    //    starts at order k and every product runs at its own truncation on
    //    order-shifted series): Y^2 .. Y^s, then Q_j = B_j + Y^s Q_{j+1} for
    //    j = r-1 .. 0 with B_j = sum_{i<s} Y^i / (js+i)!, Q_j needed to order T - s j
    const long long ns = (long long)nb * 4, ser4 = ns * T1 * E;
    // c^(0..t) = (a * b)^(0..t) for series a (read to order ta >= t) and b (read to order t);
    // consecutive products with the same left operand and transform length transform it once,
    // read to the largest truncation of the run (ta + t < Mt keeps the product wrap-free)
    const double2* a_done = nullptr;
    int a_Mt = 0, a_t = -1;
    auto star_t = [&](const double2* a, int ta, const double2* b, double2* c, int t) -> int {
      const int Mt = next_pow2(2 * (t + 1));
      if (ta < t || 2 * (ta + 1) > Mt) ta = t;
      if (!(a == a_done && Mt == a_Mt && t <= a_t && a_t + t < Mt)) {
        TRY(nspt_fft_fwd64(a, T1, spY, (int)E, ta, nb * 4, Mt, 0, lr, st));
        a_done = a; a_Mt = Mt; a_t = ta;
      }
      TRY(nspt_fft_fwd64(b, T1, spR, (int)E, t, nb * 4, Mt, 0, lr, st));
      ZgemmParams P = zg(ZG_MODE, spY, Mt, spR, Mt, spC, Mt, N, Mt, t);
      TRY(nspt_zgemm64(P, nb * 4, st));
      TRY(nspt_fft_inv64(spC, c, T1, (int)E, N, t, nb * 4, Mt, 0, lr, 1.0, 0, st));
      return NSPT_OK;
    };
    const int sb = nspt_ps_block(T), r = T / sb;
    const double2* Yp[NSPT_PS_MAX_BLOCK + 1] = {nullptr, Ysrc};
    int rc;
    for (int k = 2; k <= sb; ++k) {
      double2* Pk = serTmp + (k - 2) * ser4;
      TRY(cudaMemsetAsync(Pk, 0, (size_t)ser4 * sizeof(double2), st));  // orders below k stay 0
      if ((rc = star_t(Ysrc + E, nspt_ps_power_ta(T, sb, k), Yp[k - 1] + (k - 1) * E, Pk + k * E, T - k))) return rc;
      Yp[k] = Pk;
    }
    double2* prod = serTmp + (sb - 1) * ser4;  // the slot after the powers Y^2..Y^s
    auto block = [&](int j) {
      PsTerms tm{};
      double f = 1.0;  // 1 / (j s)!
      for (int n = 2; n <= j * sb; ++n) f /= n;
      for (int i = 0; i < sb; ++i) {
        if (i > 0) f /= (j * sb + i);
        tm.c[i] = (j * sb + i <= T) ? f : 0.0;
        if (i > 0) tm.P[i] = Yp[i];
      }
      return tm;
    };
    int cur = 0;
    TRY(nspt_ps_combine(serR[0], block(r), sb - 1, nullptr, sb, T - sb * r, T, N, ns, st));
    for (int j = r - 1; j >= 0; --j) {
      const int t = T - sb * (j + 1);
      if ((rc = star_t(Yp[sb] + sb * E, nspt_ps_horner_ta(T, sb, j), serR[cur], prod, t))) return rc;  // (Y^s Q_{j+1}) from order s
      TRY(nspt_ps_combine(serR[cur ^ 1], block(j), sb - 1, prod, sb, T - sb * j, T, N, ns, st));
      cur ^= 1;
    }
    // 7. U <- exp_star(i X) * U  (spectrum of the old U is still in specU);
    //    order 0 is exactly U^(0) since X^(0) = 0, so it is not rewritten
    TRY(nspt_fft_fwd64(serR[cur], T1, spR, (int)E, T, nb * 4, M, 0, lr, st));
    ZgemmParams P = zg(ZG_MODE, spR, M, specU, M, spC, M, N, M, T);
    TRY(nspt_zgemm64(P, nb * 4, st));
    TRY(nspt_fft_inv64(spC, U, T1, (int)E, N, T, nb * 4, M, 0, lr, 1.0, 0, st, /*kmin=*/1));
    return NSPT_OK;
  }
  // ---------------- naive form ----------------
  double2* serP1 = w.take<double2>((size_t)nb * 6 * T1 * E);
  double2* serQ = w.take<double2>((size_t)nb * 12 * T1 * E);
  double2* serIn = w.take<double2>((size_t)nb * 4 * T1 * E);
  double2* serS = w.take<double2>((size_t)nb * 4 * T1 * E);
  double2* serY = w.take<double2>((size_t)nb * 4 * T1 * E);
  double2* serR[2] = {w.take<double2>((size_t)nb * 4 * T1 * E), w.take<double2>((size_t)nb * 4 * T1 * E)};
  double2* serU0 = w.take<double2>((size_t)nb * 4 * T1 * E);
  double* imtr = w.take<double>((size_t)nb * 4 * T1);
  if (!w.fits()) return NSPT_ERR_WORKSPACE;  // the carve outgrew ws_langevin_core: a sizing bug
  auto link = [&](const double2* base, int mu) { return base + (long long)mu * T1 * E; };
  auto wlink = [&](double2* base, int mu) { return base + (long long)mu * T1 * E; };
  if (mode != NSPT_LMODE_UPDATE) {
  for (int i = 0; i < 6; ++i) {
    const int mu = kPairs[i][0], nu = kPairs[i][1];
    ZgemmParams P = zg(ZG_CONV, link(U, nu), 4 * T1, link(U, mu), 4 * T1, serP1 + (long long)i * T1 * E, 6 * T1, N,
                       T + 1, T);
    P.opB = 1;
    TRY(nspt_zgemm64(P, nb, st));
  }
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      if (mu == nu) continue;
      ZgemmParams P = zg(ZG_CONV, link(U, mu), 4 * T1, link(U, nu), 4 * T1,
                         serQ + (long long)ordered_index(mu, nu) * T1 * E, 12 * T1, N, T + 1, T);
      TRY(nspt_zgemm64(P, nb, st));
    }
  for (int mu = 0; mu < 4; ++mu) {
    bool first = true;
    for (int nu = 0; nu < 4; ++nu) {
      if (nu == mu) continue;
      {
        const int pi = (mu < nu) ? pair_index(mu, nu) : pair_index(nu, mu);
        ZgemmParams P = zg(ZG_CONV, serP1 + (long long)pi * T1 * E, 6 * T1, link(U, nu), 4 * T1, wlink(serIn, mu),
                           4 * T1, N, T + 1, T);
        if (mu > nu) P.opA = 1;
        P.opB = 1;
        P.alpha = z[mu][nu];
        P.accumulate = first ? 0 : 1;
        first = false;
        TRY(nspt_zgemm64(P, nb, st));
      }
      {
        ZgemmParams P = zg(ZG_CONV, serQ + (long long)ordered_index(mu, nu) * T1 * E, 12 * T1, link(U, nu), 4 * T1,
                           wlink(serIn, mu), 4 * T1, N, T + 1, T);
        P.opA = 1;
        P.alpha = make_double2(z[mu][nu].x, -z[mu][nu].y);
        P.accumulate = 1;
        TRY(nspt_zgemm64(P, nb, st));
      }
    }
  }
  {
    ZgemmParams P = zg(ZG_CONV, U, T1, serIn, T1, serS, T1, N, T + 1, T);
    TRY(nspt_zgemm64(P, nb * 4, st));
  }
  TRY(nspt_tek_drift(serS, imtr, eta, F, serY, N, T, (long long)nb * 4, eps, st));
  }
  if (mode == NSPT_LMODE_DRIFT) return NSPT_OK;
  const double2* Ysrc = (mode == NSPT_LMODE_UPDATE) ? Yin : serY;
  TRY(cudaMemsetAsync(serR[0], 0, (size_t)nb * 4 * T1 * E * sizeof(double2), st));
  TRY(cudaMemsetAsync(serR[1], 0, (size_t)nb * 4 * T1 * E * sizeof(double2), st));
  TRY(add_identity(serR[0], T1, N, (long long)nb * 4, st));
  int cur = 0;
  for (int n = T; n >= 1; --n) {
    const int t = T - n + 1;
    ZgemmParams P = zg(ZG_CONV, Ysrc, T1, serR[cur], T1, serR[cur ^ 1], T1, N, t + 1, t);
    P.alpha = make_double2(1.0 / n, 0.0);
    TRY(nspt_zgemm64(P, nb * 4, st));
    TRY(add_identity(serR[cur ^ 1], T1, N, (long long)nb * 4, st));
    cur ^= 1;
  }
  TRY(cudaMemcpyAsync(serU0, U, (size_t)nb * 4 * T1 * E * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  ZgemmParams P = zg(ZG_CONV, serR[cur], T1, serU0, T1, U, T1, N, T + 1, T);
  TRY(nspt_zgemm64(P, nb * 4, st));
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// Molecular dynamics: leapfrog with momentum refresh (Eq. 3, the paper's
// integrator), built from the drift-only and update-only phases above.
// ---------------------------------------------------------------------------
size_t ws_md(const Plan& p) {
  const size_t ser = ((size_t)p.batch * 4 * (p.T + 1) * p.E * sizeof(double2) + 255) & ~(size_t)255;
  return ((ws_langevin(p) + 255) & ~(size_t)255) + 2 * ser;
}

int md_phase(const Plan& p, double2* U, double2* F, const double2* Y, int flux, void* lws, cudaStream_t st, int mode) {
  int lr = 0;
  const int* dlr = nullptr;
  // the force phase multiplies links only; the link update also powers of the increment Y
  const int rc = tek_log2r(p, U, mode == NSPT_LMODE_UPDATE ? Y : U, lws, st, &lr, &dlr);
  if (rc) return rc;
  NsptDevLog2r scope(dlr);
  if (p.prec == NSPT_PREC_SPLIT)
    return nspt_split_langevin(p.N, p.T, p.batch, p.M, p.slices, U, nullptr, F, flux, 0.0, lws, st, mode, Y, lr);
  return langevin_fp64(p, U, nullptr, F, flux, 0.0, lws, st, mode, Y, lr);
}

int md_run(const Plan& p, double2* U, double2* P, const double2* eta, int flux, double eps, int nsteps, void* ws,
           cudaStream_t st) {
  const long long E = p.E, ns = (long long)p.batch * 4;
  const int T = p.T;
  WsCarver w(ws, SIZE_MAX);
  void* lws = w.take<char>(ws_langevin(p));
  double2* F = w.take<double2>((size_t)ns * (T + 1) * E);
  double2* Y = w.take<double2>((size_t)ns * (T + 1) * E);
  int rc;
  if (eta) TRY(nspt_md_refresh(P, eta, T, E, ns, st));
  if (nsteps <= 0) return NSPT_OK;
  // force phase: F(U) and the momentum kicks; link phase: U <- exp_star(i eps P) U
  auto force = [&]() -> int {
    ProfScope ps(NSPT_STAGE_MD_FORCE, st, 0);
    return md_phase(p, U, F, nullptr, flux, lws, st, NSPT_LMODE_DRIFT);
  };
  if ((rc = force())) return rc;
  for (int s = 0; s < nsteps; ++s) {
    {
      ProfScope ps(NSPT_STAGE_MD_FORCE, st, 0);
      TRY(nspt_md_kick(P, F, 0.5 * eps, T, E, ns, st));   // P_half = P + eps/2 F(U)
    }
    {
      ProfScope ps(NSPT_STAGE_MD_LINK, st, 0);
      TRY(nspt_md_y(Y, P, eps, T, E, ns, st));            // Y = i eps P_half
      if ((rc = md_phase(p, U, F, Y, flux, lws, st, NSPT_LMODE_UPDATE))) return rc;  // U <- exp_star(Y) U
    }
    if ((rc = force())) return rc;                          // F(U')
    ProfScope ps(NSPT_STAGE_MD_FORCE, st, 0);
    TRY(nspt_md_kick(P, F, 0.5 * eps, T, E, ns, st));     // P' = P_half + eps/2 F(U')
  }
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// Wilson loops of the TEK links (the NSPT measurement): powers of the links,
// two products per plane and extent pair, and the trace of the last product
// as a correlation of the two factors.
// ---------------------------------------------------------------------------
constexpr int kWilsonMaxExtent = 8;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t ws_wilson(const Plan& p, int amax) {
  const size_t ser = (size_t)p.batch * (p.T + 1) * p.E * sizeof(double2);
  const size_t tr = (size_t)6 * amax * amax * p.batch * (p.T + 1) * NSPT_TRACE_CHUNKS * sizeof(double2);
  return al256((size_t)4 * amax * ser) + al256(2 * ser) + al256(tr) + al256(ws_mul(p));
}

int mul_plan(const Plan& p, const double2* A, const double2* B, double2* C, void* ws, cudaStream_t st) {
  if (p.prec == NSPT_PREC_FP64) return mul_fp64(p, A, B, C, ws, st);
  if (p.algo == NSPT_ALGO_NAIVE)
    return nspt_split_mul_naive(p.N, p.T, p.batch, p.slices, p.log2r, p.rescale_auto, A, B, C, ws, st);
  return nspt_split_mul(p.N, p.T, p.batch, p.M, p.slices, p.log2r, p.rescale_auto, A, B, C, ws, st, p.cm);
}

int wilson_run(const Plan& p, const double2* U, int flux, int amax, double2* W, void* ws, cudaStream_t st) {
  const int N = p.N, T = p.T, batch = p.batch;
  const long long E = p.E, T1 = T + 1, ser = (long long)batch * T1 * E;
  const int L = (int)llround(sqrt((double)N));
  char* base = (char*)ws;
  double2* Pw = (double2*)base;                                  // [4][amax][batch][T+1][E]
  base += al256((size_t)4 * amax * ser * sizeof(double2));
  double2* L1 = (double2*)base;
  double2* L2 = L1 + ser;
  base += al256((size_t)2 * ser * sizeof(double2));
  double2* tr = (double2*)base;                                  // [6][amax][amax][batch][T+1][chunks]
  base += al256((size_t)6 * amax * amax * batch * T1 * NSPT_TRACE_CHUNKS * sizeof(double2));
  void* mws = base;
  auto pw = [&](int mu, int a) { return Pw + ((long long)mu * amax + (a - 1)) * ser; };
  int rc;
  for (int mu = 0; mu < 4; ++mu) {
    // U_mu of every batch element into one contiguous batch
    TRY(cudaMemcpy2DAsync(pw(mu, 1), (size_t)T1 * E * sizeof(double2), U + (long long)mu * T1 * E,
                          (size_t)4 * T1 * E * sizeof(double2), (size_t)T1 * E * sizeof(double2), batch,
                          cudaMemcpyDeviceToDevice, st));
    for (int a = 2; a <= amax; ++a)
      if ((rc = mul_plan(p, pw(mu, a - 1), pw(mu, 1), pw(mu, a), mws, st))) return rc;
  }
  int pl = 0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = mu + 1; nu < 4; ++nu, ++pl)
      for (int a = 1; a <= amax; ++a)
        for (int c = 1; c <= amax; ++c) {
          // z_{mu nu}^(ac) Tr[(U_mu^a U_nu^c) * (U_nu^c U_mu^a)^+]
          if ((rc = mul_plan(p, pw(mu, a), pw(nu, c), L1, mws, st))) return rc;
          if ((rc = mul_plan(p, pw(nu, c), pw(mu, a), L2, mws, st))) return rc;
          const double ang = 2.0 * M_PI * flux * a * c / L;
          TRY(nspt_trace_corr(L1, L2,
                              tr + (((long long)pl * amax + (a - 1)) * amax + (c - 1)) * batch * T1 * NSPT_TRACE_CHUNKS,
                              make_double2(cos(ang), sin(ang)), T, E, batch, st));
        }
  // the (nu, mu) planes are the conjugates of the (mu, nu) planes with the extents swapped
  TRY(nspt_wilson_combine(tr, W, 6, amax, batch, T, 1.0 / (12.0 * N), st));
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// Unitarity projection: V = U * (U^+ U)^(-1/2) in the truncated ring (the polar
// factor), order 0 kept.  D = U^+ U - 1 with D^(0) := 0, the binomial series
// S = sum_{n<=T} c_n D^n (c_n = binom(-1/2, n)) by Horner,
// S_n = c_n 1 + D * S_{n+1}, then V = U * S; every product in the form of opts.
// ---------------------------------------------------------------------------
size_t ws_unitarize(const Plan& p) {
  const size_t ser = (size_t)p.batch * (p.T + 1) * p.E * sizeof(double2);
  const size_t ph = (size_t)p.batch * (p.T + 1);  // phase a_k (double) and exp series (double2)
  return 3 * al256(ser) + al256(ph * sizeof(double)) + al256(ph * sizeof(double2)) + al256(ws_mul(p));
}

double binom_minus_half(int n) {  // (-1)^n (2n)! / (4^n (n!)^2), by the ratio c_n / c_{n-1}
  double c = 1.0;
  for (int k = 1; k <= n; ++k) c *= -(2.0 * k - 1.0) / (2.0 * k);
  return c;
}

int unitarize_run(const Plan& p, double2* U, int special, void* ws, cudaStream_t st) {
  const int N = p.N, T = p.T, nb = p.batch;
  const long long E = p.E, T1 = T + 1, ser = (long long)nb * T1 * E;
  char* base = (char*)ws;
  double2* D = (double2*)base;
  base += al256(ser * sizeof(double2));
  double2* S[2] = {(double2*)base, (double2*)(base + al256(ser * sizeof(double2)))};
  base += 2 * al256(ser * sizeof(double2));
  double* phase = (double*)base;
  base += al256((size_t)nb * T1 * sizeof(double));
  double2* phs = (double2*)base;
  base += al256((size_t)nb * T1 * sizeof(double2));
  void* mws = base;
  int rc;
  // D = U^+ * U - 1, with D^(0) = 0 (order 0 is unitary); U^+ goes through S[0]
  TRY(nspt_series_dagger(U, S[0], N, (long long)nb * T1, st));
  if ((rc = mul_plan(p, S[0], U, D, mws, st))) return rc;
  TRY(nspt_series_order0_identity(D, T, N, nb, 0.0, 1, st));
  // S_T = c_T 1, S_n = c_n 1 + D * S_{n+1} (order 0 of D * S is zero in exact arithmetic: set)
  TRY(cudaMemsetAsync(S[0], 0, (size_t)ser * sizeof(double2), st));
  TRY(nspt_series_order0_identity(S[0], T, N, nb, binom_minus_half(T), 1, st));
  int cur = 0;
  for (int n = T - 1; n >= 0; --n) {
    if ((rc = mul_plan(p, D, S[cur], S[cur ^ 1], mws, st))) return rc;
    TRY(nspt_series_order0_identity(S[cur ^ 1], T, N, nb, binom_minus_half(n), 1, st));
    cur ^= 1;
  }
  // V = U * S into D (free again), orders 1..T copied back; order 0 of U is kept as it is
  if ((rc = mul_plan(p, U, S[cur], D, mws, st))) return rc;
  if (T >= 1)
    TRY(cudaMemcpy2DAsync(U + E, (size_t)T1 * E * sizeof(double2), D + E, (size_t)T1 * E * sizeof(double2),
                          (size_t)T * E * sizeof(double2), nb, cudaMemcpyDeviceToDevice, st));
  if (!special || T < 1) return NSPT_OK;
  // U(1) phase a(g) = Im Tr log(U0^+ U(g)) of the unitary series now in U, from Jacobi's
  // formula: d/dg log det U = Tr(U^-1 U') = Tr(U^+ * U') (U unitary through order T), so
  // a_k = Im Tr(U^+ * U')_(k-1) / k -- one product; then U <- U * exp(-i a / N) (scalar
  // series), so that det U = det U0 through order T
  TRY(nspt_series_dagger(U, S[0], N, (long long)nb * T1, st));
  TRY(nspt_series_derivative(U, S[1], T, N, nb, st));
  if ((rc = mul_plan(p, S[0], S[1], D, mws, st))) return rc;
  TRY(nspt_series_imag_trace(D, phase, N, (long long)nb * T1, st));
  TRY(nspt_series_remove_phase(U, phase, phs, T, N, nb, st));
  return NSPT_OK;
}

std::mutex g_init_mu;
int g_init_dev[64] = {0};

// ---------------------------------------------------------------------------
// Products of host-resident series: one batch element at a time through two
// device slots, with the host-to-device copies of element i+1, the product of
// element i (caller's stream) and the device-to-host copy of element i-1 on
// three streams.  Streams and events are created once per device.
// ---------------------------------------------------------------------------
constexpr int kHostSlots = 2;  // device slots (a third measured no faster: the copies are PCIe-bound)

struct HostPipe {
  bool ready = false;
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, ev_in[kHostSlots] = {}, ev_comp[kHostSlots] = {}, ev_out[kHostSlots] = {};
  // chaining state: the slots of the previous call (same workspace, stream and element size)
  const void* ws = nullptr;
  cudaStream_t st = nullptr;
  size_t bytes = 0;
  bool used[kHostSlots] = {};
  int next = 0;
  std::mutex mu;  // one enqueue at a time per device
};
HostPipe g_pipe[64];
std::mutex g_pipe_mu;

int host_pipe(HostPipe** hp) {
  int dev = 0;
  TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return NSPT_ERR_DEVICE;
  std::lock_guard<std::mutex> lk(g_pipe_mu);
  HostPipe& h = g_pipe[dev];
  if (!h.ready) {
    TRY(cudaStreamCreateWithFlags(&h.in, cudaStreamNonBlocking));
    TRY(cudaStreamCreateWithFlags(&h.out, cudaStreamNonBlocking));
    TRY(cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming));
    for (int s = 0; s < kHostSlots; ++s) {
      TRY(cudaEventCreateWithFlags(&h.ev_in[s], cudaEventDisableTiming));
      TRY(cudaEventCreateWithFlags(&h.ev_comp[s], cudaEventDisableTiming));
      TRY(cudaEventCreateWithFlags(&h.ev_out[s], cudaEventDisableTiming));
    }
    h.ready = true;
  }
  *hp = &h;
  return NSPT_OK;
}

size_t ws_host(const Plan& pc) {
  const size_t ser = (size_t)(pc.T + 1) * pc.E * sizeof(double2);
  return 3 * kHostSlots * al256(ser) + al256(ws_mul(pc));
}

int host_run(const Plan& pc, int batch, const double2* A, const double2* B, double2* C, void* ws, HostPipe& hp,
             cudaStream_t st) {
  const size_t bytes = (size_t)(pc.T + 1) * pc.E * sizeof(double2);
  const long long ser = (long long)(pc.T + 1) * pc.E;
  char* base = (char*)ws;
  double2* d[kHostSlots][3];
  for (int s = 0; s < kHostSlots; ++s)
    for (int j = 0; j < 3; ++j) d[s][j] = (double2*)(base + (3 * s + j) * al256(bytes));
  void* mws = base + 3 * kHostSlots * al256(bytes);
  std::lock_guard<std::mutex> lk(hp.mu);
  if (!(hp.ws == ws && hp.st == st && hp.bytes == bytes)) {
    // not a continuation of the previous call: everything already queued on the caller's
    // stream (earlier users of this workspace) comes first
    TRY(cudaEventRecord(hp.start, st));
    TRY(cudaStreamWaitEvent(hp.in, hp.start, 0));
    TRY(cudaStreamWaitEvent(hp.out, hp.start, 0));
    for (int k = 0; k < kHostSlots; ++k) hp.used[k] = false;
    hp.next = 0;
  }
  hp.ws = ws;
  hp.st = st;
  hp.bytes = bytes;
  int rc, s = 0;
  for (int i = 0; i < batch; ++i) {
    s = hp.next;
    hp.next = (hp.next + 1) % kHostSlots;
    if (hp.used[s]) TRY(cudaStreamWaitEvent(hp.in, hp.ev_comp[s], 0));  // slot's A, B consumed
    TRY(cudaMemcpyAsync(d[s][0], A + i * ser, bytes, cudaMemcpyHostToDevice, hp.in));
    TRY(cudaMemcpyAsync(d[s][1], B + i * ser, bytes, cudaMemcpyHostToDevice, hp.in));
    TRY(cudaEventRecord(hp.ev_in[s], hp.in));
    TRY(cudaStreamWaitEvent(st, hp.ev_in[s], 0));
    if (hp.used[s]) TRY(cudaStreamWaitEvent(st, hp.ev_out[s], 0));      // slot's C copied out
    hp.used[s] = true;
    if ((rc = mul_plan(pc, d[s][0], d[s][1], d[s][2], mws, st))) { hp.ws = nullptr; return rc; }
    TRY(cudaEventRecord(hp.ev_comp[s], st));
    TRY(cudaStreamWaitEvent(hp.out, hp.ev_comp[s], 0));
    TRY(cudaMemcpyAsync(C + i * ser, d[s][2], bytes, cudaMemcpyDeviceToHost, hp.out));
    TRY(cudaEventRecord(hp.ev_out[s], hp.out));
  }
  // the caller's stream continues after the last copy out (the copies out are in order)
  TRY(cudaStreamWaitEvent(st, hp.ev_out[s], 0));
  return NSPT_OK;
}

}  // namespace

void nspt_set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }
const int* nspt_dev_log2r() { return g_dev_log2r; }
NsptDevLog2r::NsptDevLog2r(const int* p) : prev_(g_dev_log2r) { g_dev_log2r = p; }
NsptDevLog2r::~NsptDevLog2r() { g_dev_log2r = prev_; }

extern "C" {

void nspt_opts_default(nspt_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->algo = NSPT_ALGO_AUTO;
  o->prec = NSPT_PREC_FP64;
  o->rescale_log2r = 0;
}

int nspt_init(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { g_last_cuda = e; return NSPT_ERR_CUDA; }
  if (dev < 0 || dev >= 64) return NSPT_ERR_DEVICE;
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (g_init_dev[dev] == 1) return NSPT_OK;
  if (g_init_dev[dev] == -1) return NSPT_ERR_DEVICE;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) { g_last_cuda = e; return NSPT_ERR_CUDA; }
  if (!(prop.major == 10 && prop.minor == 3)) { g_init_dev[dev] = -1; return NSPT_ERR_DEVICE; }
  int rc = nspt_split_init();
  if (rc != NSPT_OK) return rc;
  g_init_dev[dev] = 1;
  return NSPT_OK;
}

size_t nspt_workspace_size(int op, int N, int T, int batch, const nspt_opts* opts) {
  Plan p;
  if (make_plan(N, T, batch, opts, &p, op) != NSPT_OK) return 0;
  switch (op) {
    case NSPT_OP_MUL: return ws_mul(p);
    case NSPT_OP_MUL_BACKWARD: return ws_bwd(p);
    case NSPT_OP_LANGEVIN: return ws_langevin(p);
    case NSPT_OP_MD: return ws_md(p);
    case NSPT_OP_UNITARIZE: return ws_unitarize(p);
    default: return 0;
  }
}

static int check_ws(const nspt_opts* o, size_t need) {
  if (need == 0) return NSPT_OK;
  if (!o || !o->workspace || o->workspace_bytes < need) return NSPT_ERR_WORKSPACE;
  if (((uintptr_t)o->workspace) & 255) return NSPT_ERR_WORKSPACE;
  return NSPT_OK;
}

int nspt_polymat_mul(const void* A, const void* B, void* C, int N, int T, int batch, const nspt_opts* opts,
                     void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p, NSPT_OP_MUL);
  if (rc) return rc;
  if (!A || !B || !C) return NSPT_ERR_ARG;
  const size_t bytes = (size_t)batch * (T + 1) * p.E * sizeof(double2);
  if (overlaps(C, bytes, A, bytes) || overlaps(C, bytes, B, bytes)) return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_mul(p)))) return rc;
  if ((rc = nspt_init())) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  {
    const void* ptrs[3] = {A, B, C};
    if ((rc = nspt_check_ptrs(st, true, ptrs, 3))) return rc;
  }
  return mul_plan(p, (const double2*)A, (const double2*)B, (double2*)C, opts ? opts->workspace : nullptr, st);
}

int nspt_polymat_mul_backward(const void* A, const void* B, const void* gC, void* gA, void* gB, int N, int T,
                              int batch, const nspt_opts* opts, void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p, NSPT_OP_MUL_BACKWARD);
  if (rc) return rc;
  if (!A || !B || !gC) return NSPT_ERR_ARG;
  if (!gA && !gB) return NSPT_OK;
  const size_t bytes = (size_t)batch * (T + 1) * p.E * sizeof(double2);
  const void* ins[3] = {A, B, gC};
  for (int i = 0; i < 3; ++i)
    if (overlaps(gA, bytes, ins[i], bytes) || overlaps(gB, bytes, ins[i], bytes)) return NSPT_ERR_ALIAS;
  if (overlaps(gA, bytes, gB, bytes)) return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_bwd(p)))) return rc;
  if ((rc = nspt_init())) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  {
    const void* ptrs[5] = {A, B, gC, gA, gB};
    if ((rc = nspt_check_ptrs(st, true, ptrs, 5))) return rc;
  }
  if (p.prec == NSPT_PREC_FP64)
    return bwd_fp64(p, (const double2*)A, (const double2*)B, (const double2*)gC, (double2*)gA, (double2*)gB,
                    opts ? opts->workspace : nullptr, st);
  if (p.algo == NSPT_ALGO_NAIVE)
    return nspt_split_bwd_naive(p.N, p.T, p.batch, p.slices, p.log2r, (const double2*)A, (const double2*)B,
                                (const double2*)gC, (double2*)gA, (double2*)gB, opts->workspace, st);
  return nspt_split_bwd(p.N, p.T, p.batch, p.M, p.slices, p.log2r, (const double2*)A, (const double2*)B,
                        (const double2*)gC, (double2*)gA, (double2*)gB, opts->workspace, st);
}

int nspt_tek_unitarize(void* U, int N, int T, int batch, int special, const nspt_opts* opts, void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p, NSPT_OP_UNITARIZE);
  if (rc) return rc;
  if (!U) return NSPT_ERR_ARG;
  if ((rc = check_ws(opts, ws_unitarize(p)))) return rc;
  if ((rc = nspt_init())) return rc;
  {
    const void* ptrs[1] = {U};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 1))) return rc;
  }
  if (special != 0 && special != 1) return NSPT_ERR_ARG;
  return unitarize_run(p, (double2*)U, special, opts ? opts->workspace : nullptr, (cudaStream_t)stream);
}

int nspt_tek_langevin_step(void* U, const void* eta, void* F, int N, int T, int batch, int flux, double eps,
                           const nspt_opts* opts, void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p);
  if (rc) return rc;
  if (!U || !eta) return NSPT_ERR_ARG;
  const int L = (int)llround(sqrt((double)N));
  if (L * L != N || flux <= 0) return NSPT_ERR_ARG;
  int a = flux % L, bb = L;
  while (a) { int t = bb % a; bb = a; a = t; }
  if (bb != 1) return NSPT_ERR_ARG;
  if (!(eps > 0.0) || !std::isfinite(eps)) return NSPT_ERR_ARG;
  const size_t ubytes = (size_t)batch * 4 * (T + 1) * p.E * sizeof(double2);
  const size_t ebytes = (size_t)batch * 4 * p.E * sizeof(double2);
  if (overlaps(U, ubytes, eta, ebytes) || overlaps(F, ubytes, U, ubytes) || overlaps(F, ubytes, eta, ebytes))
    return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_langevin(p)))) return rc;
  if ((rc = nspt_init())) return rc;
  {
    const void* ptrs[3] = {U, eta, F};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 3))) return rc;
  }
  int lr = 0;
  const int* dlr = nullptr;
  if ((rc = tek_log2r(p, (const double2*)U, (const double2*)U, opts ? opts->workspace : nullptr, (cudaStream_t)stream,
                      &lr, &dlr)))
    return rc;
  NsptDevLog2r scope(dlr);
  if (p.prec != NSPT_PREC_FP64) {
    return nspt_split_langevin(p.N, p.T, p.batch, p.M, p.slices, (double2*)U, (const double2*)eta, (double2*)F, flux,
                               eps, opts->workspace, (cudaStream_t)stream, NSPT_LMODE_STEP, nullptr, lr);
  }
  return langevin_fp64(p, (double2*)U, (const double2*)eta, (double2*)F, flux, eps, opts ? opts->workspace : nullptr,
                       (cudaStream_t)stream, NSPT_LMODE_STEP, nullptr, lr);
}

static int check_group(const nspt_polymat_desc* d, int count, const nspt_opts* o, Plan* first) {
  if (!d || count < 1 || count > NSPT_SPLIT_MAX_PROBLEMS) return NSPT_ERR_ARG;
  if (o && o->fft_len != 0) return NSPT_ERR_ARG;
  for (int i = 0; i < count; ++i) {
    Plan p;
    int rc = make_plan(d[i].N, d[i].T, d[i].batch, o, &p);
    if (rc) return rc;
    if (p.algo != NSPT_ALGO_FFT && p.prec == NSPT_PREC_SPLIT) return NSPT_ERR_UNSUPPORTED;
    if (!d[i].A || !d[i].B || !d[i].C) return NSPT_ERR_ARG;
    const size_t bytes = (size_t)d[i].batch * (d[i].T + 1) * p.E * sizeof(double2);
    for (int j = 0; j < count; ++j) {
      const size_t bj = (size_t)d[j].batch * (d[j].T + 1) * (size_t)d[j].N * d[j].N * sizeof(double2);
      if (overlaps(d[i].C, bytes, d[j].A, bj) || overlaps(d[i].C, bytes, d[j].B, bj)) return NSPT_ERR_ALIAS;
      if (j != i && overlaps(d[i].C, bytes, d[j].C, bj)) return NSPT_ERR_ALIAS;
    }
    if (i == 0) *first = p;
  }
  return NSPT_OK;
}

size_t nspt_workspace_size_grouped(const nspt_polymat_desc* d, int count, const nspt_opts* o) {
  Plan p;
  if (check_group(d, count, o, &p)) return 0;
  if (p.prec == NSPT_PREC_SPLIT) return nspt_split_ws_grouped(d, count, p.slices);
  size_t mx = 0;
  for (int i = 0; i < count; ++i) {
    Plan q;
    make_plan(d[i].N, d[i].T, d[i].batch, o, &q);
    mx = std::max(mx, ws_mul(q));
  }
  return mx;
}

int nspt_polymat_mul_grouped(const nspt_polymat_desc* d, int count, const nspt_opts* o, void* stream) {
  Plan p;
  int rc = check_group(d, count, o, &p);
  if (rc) return rc;
  if ((rc = check_ws(o, nspt_workspace_size_grouped(d, count, o)))) return rc;
  if ((rc = nspt_init())) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < count; ++i) {
    const void* ptrs[3] = {d[i].A, d[i].B, d[i].C};
    if ((rc = nspt_check_ptrs(st, true, ptrs, 3))) return rc;
  }
  if (p.prec == NSPT_PREC_SPLIT) {
    if (p.rescale_auto) return NSPT_ERR_UNSUPPORTED;
    return nspt_split_mul_grouped(d, count, p.slices, p.log2r, o->workspace, st);
  }
  for (int i = 0; i < count; ++i) {
    Plan q;
    make_plan(d[i].N, d[i].T, d[i].batch, o, &q);
    rc = mul_fp64(q, (const double2*)d[i].A, (const double2*)d[i].B, (double2*)d[i].C, o ? o->workspace : nullptr,
                  st);
    if (rc) return rc;
  }
  return NSPT_OK;
}

int nspt_autotune_grouped(const nspt_polymat_desc* d, int count, const nspt_opts* o, const char* cache_path,
                          int* chosen_bn, void* stream) {
  Plan p;
  int rc = check_group(d, count, o, &p);
  if (rc) return rc;
  if (!chosen_bn || p.prec != NSPT_PREC_SPLIT) return NSPT_ERR_ARG;
  if ((rc = check_ws(o, nspt_workspace_size_grouped(d, count, o)))) return rc;
  if ((rc = nspt_init())) return rc;
  for (int i = 0; i < count; ++i) {
    const void* ptrs[3] = {d[i].A, d[i].B, d[i].C};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 3))) return rc;
  }
  return nspt_split_autotune_grouped(d, count, p.slices, o->workspace, cache_path, chosen_bn, (cudaStream_t)stream);
}

int nspt_tek_md_trajectory(void* U, void* P, const void* eta_refresh, int N, int T, int batch, int flux, double eps,
                           int nsteps, const nspt_opts* opts, void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p);
  if (rc) return rc;
  if (!U || !P || nsteps < 0) return NSPT_ERR_ARG;
  const int L = (int)llround(sqrt((double)N));
  if (L * L != N || flux <= 0) return NSPT_ERR_ARG;
  int a = flux % L, bb = L;
  while (a) { int t = bb % a; bb = a; a = t; }
  if (bb != 1) return NSPT_ERR_ARG;
  if (!(eps > 0.0) || !std::isfinite(eps)) return NSPT_ERR_ARG;
  const size_t ubytes = (size_t)batch * 4 * (T + 1) * p.E * sizeof(double2);
  const size_t ebytes = (size_t)batch * 4 * p.E * sizeof(double2);
  if (overlaps(U, ubytes, P, ubytes) || overlaps(U, ubytes, eta_refresh, ebytes) ||
      overlaps(P, ubytes, eta_refresh, ebytes))
    return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_md(p)))) return rc;
  if ((rc = nspt_init())) return rc;
  {
    const void* ptrs[3] = {U, P, eta_refresh};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 3))) return rc;
  }
  return md_run(p, (double2*)U, (double2*)P, (const double2*)eta_refresh, flux, eps, nsteps, opts->workspace,
                (cudaStream_t)stream);
}

size_t nspt_workspace_size_wilson(int N, int T, int batch, int amax, const nspt_opts* opts) {
  Plan p;
  if (make_plan(N, T, batch, opts, &p, kPlanWilson) || amax < 1 || amax > kWilsonMaxExtent) return 0;
  return ws_wilson(p, amax);
}

int nspt_tek_wilson_loops(const void* U, int N, int T, int batch, int flux, int amax, void* W, const nspt_opts* opts,
                          void* stream) {
  Plan p;
  int rc = make_plan(N, T, batch, opts, &p, kPlanWilson);
  if (rc) return rc;
  if (!U || !W || amax < 1 || amax > kWilsonMaxExtent) return NSPT_ERR_ARG;
  const int L = (int)llround(sqrt((double)N));
  if (L * L != N || flux <= 0) return NSPT_ERR_ARG;
  int a = flux % L, bb = L;
  while (a) { int t = bb % a; bb = a; a = t; }
  if (bb != 1) return NSPT_ERR_ARG;
  const size_t ubytes = (size_t)batch * 4 * (T + 1) * p.E * sizeof(double2);
  const size_t wbytes = (size_t)batch * amax * amax * (T + 1) * sizeof(double2);
  if (overlaps(U, ubytes, W, wbytes)) return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_wilson(p, amax)))) return rc;
  if ((rc = nspt_init())) return rc;
  {
    const void* ptrs[2] = {U, W};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 2))) return rc;
  }
  return wilson_run(p, (const double2*)U, flux, amax, (double2*)W, opts->workspace, (cudaStream_t)stream);
}

size_t nspt_workspace_size_host(int N, int T, int batch, const nspt_opts* opts) {
  Plan pc;
  if (batch < 1 || make_plan(N, T, 1, opts, &pc, NSPT_OP_MUL)) return 0;
  return ws_host(pc);
}

int nspt_polymat_mul_host(const void* A, const void* B, void* C, int N, int T, int batch, const nspt_opts* opts,
                          void* stream) {
  Plan p, pc;
  int rc = make_plan(N, T, batch, opts, &p, NSPT_OP_MUL);
  if (rc) return rc;
  if ((rc = make_plan(N, T, 1, opts, &pc, NSPT_OP_MUL))) return rc;
  if (!A || !B || !C) return NSPT_ERR_ARG;
  const size_t bytes = (size_t)batch * (T + 1) * p.E * sizeof(double2);
  if (overlaps(C, bytes, A, bytes) || overlaps(C, bytes, B, bytes)) return NSPT_ERR_ALIAS;
  if ((rc = check_ws(opts, ws_host(pc)))) return rc;
  if ((rc = nspt_init())) return rc;
  {
    const void* hptrs[3] = {A, B, C};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, false, hptrs, 3))) return rc;
    const void* dptrs[1] = {opts->workspace};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, dptrs, 1))) return rc;
  }
  HostPipe* hp = nullptr;
  if ((rc = host_pipe(&hp))) return rc;
  return host_run(pc, batch, (const double2*)A, (const double2*)B, (double2*)C, opts->workspace, *hp,
                  (cudaStream_t)stream);
}

int nspt_debug_wait_budget(long long ns) {
  nspt_split_set_wait_budget(ns);
  return NSPT_OK;
}

int nspt_order_fft(const void* A, void* At, int N, int T, int batch, int M, void* stream) {
  if (!A || !At || N < 1 || T < 0 || batch < 1) return NSPT_ERR_ARG;
  if (ilog2_exact(M) < 0 || M < 2 * (T + 1) || M > 512) return NSPT_ERR_ARG;
  const long long E = (long long)N * N;
  if (overlaps(A, (size_t)batch * (T + 1) * E * 16, At, (size_t)batch * M * E * 16)) return NSPT_ERR_ALIAS;
  int rc = nspt_init();
  if (rc) return rc;
  cudaError_t e = nspt_fft_fwd64((const double2*)A, T + 1, (double2*)At, (int)E, T, batch, M, 0, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) { g_last_cuda = e; return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

int nspt_order_ifft(const void* Ct, void* C, int N, int T, int batch, int M, void* stream) {
  if (!Ct || !C || N < 1 || T < 0 || batch < 1) return NSPT_ERR_ARG;
  if (ilog2_exact(M) < 0 || M < 2 * (T + 1) || M > 512) return NSPT_ERR_ARG;
  const long long E = (long long)N * N;
  if (overlaps(C, (size_t)batch * (T + 1) * E * 16, Ct, (size_t)batch * M * E * 16)) return NSPT_ERR_ALIAS;
  int rc = nspt_init();
  if (rc) return rc;
  cudaError_t e = nspt_fft_inv64((const double2*)Ct, (double2*)C, T + 1, (int)E, N, T, batch, M, 0, 0, 1.0, 0,
                                 (cudaStream_t)stream);
  if (e != cudaSuccess) { g_last_cuda = e; return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

const char* nspt_status_string(int s) {
  switch (s) {
    case NSPT_OK: return "ok";
    case NSPT_ERR_ARG: return "invalid argument";
    case NSPT_ERR_ALIAS: return "output overlaps an input";
    case NSPT_ERR_UNSUPPORTED: return "unsupported option combination";
    case NSPT_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case NSPT_ERR_CUDA: return "CUDA error";
    case NSPT_ERR_TIMEOUT: return "device-side wait timed out";
    case NSPT_ERR_DEVICE: return "device is not sm_103 (B300)";
    default: return "unknown status";
  }
}

const char* nspt_last_error(void) { return cudaGetErrorString(g_last_cuda); }

int nspt_device_status(const nspt_opts* opts, void* stream) {
  if (!opts || !opts->workspace) return NSPT_ERR_ARG;
  int err = 0;
  int rc = nspt_split_read_error(opts->workspace, &err, (cudaStream_t)stream);
  if (rc) return rc;
  return err ? NSPT_ERR_TIMEOUT : NSPT_OK;
}

int nspt_split_slices(const void* X, void* slices, int* exps, int N, int Q, int S, int trans, int conj, int right,
                      void* stream) {
  if (!X || !slices || !exps || N < 1 || N > 1024 || Q < 1 || Q > 65535 || S < 2 || S > 8) return NSPT_ERR_ARG;
  int rc = nspt_init();
  if (rc) return rc;
  return nspt_split_slice(S, (const double2*)X, Q, Q, 0, trans ? 1 : 0, conj ? 1 : 0, N, Q, right ? 3 : 2, slices,
                          exps, (cudaStream_t)stream);
}

int nspt_split_mode_gemm(const void* slA, const void* slB, const int* expA, const int* expB, void* Ct, int N, int Q,
                         int S, int* err, void* stream) {
  if (!slA || !slB || !expA || !expB || !Ct || !err || N < 1 || N > 1024 || Q < 1 || S < 2 || S > 8)
    return NSPT_ERR_ARG;
  int rc = nspt_init();
  if (rc) return rc;
  return nspt_split_gemm_stage(slA, slB, expA, expB, Ct, N, Q, S, err, (cudaStream_t)stream);
}

}  // extern "C"
