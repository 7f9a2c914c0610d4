// Naive form (Eq. 5) of the split products and its backward: every order sliced once from FP64,
// one tensor-core GEMM (split_gemm.cu) per pair of orders, double-float accumulators, FP64 out.
// The slicers, the side streams and the tile-width rule come from split.cu.
#include <algorithm>
#include <functional>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "dfloat.cuh"
#include "prof.cuh"
#include "split.cuh"
#include "split_gemm.cuh"

#define TRYC(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { nspt_set_last_cuda_error(_e); return NSPT_ERR_CUDA; } } while (0)
#define TRYS(x) do { int _r = (x); if (_r != NSPT_OK) return _r; } while (0)

// ---------------------------------------------------------------------------
// Naive form (Eq. 5) on the tensor cores: C_k = sum_{l=0}^{k} A_l B_{k-l} as
// (T+1)(T+2)/2 split-precision GEMMs per batch element, one for each pair
// (l, j = k - l), accumulated in double-float.  Every order is sliced once,
// straight from FP64 (A_l by rows, B_j by columns); each GEMM carries its
// own operands' row and column exponents, so an order is not limited by the
// size of the others as in a mode product, and no order transform is run.
//
// Schedule.  The pairs with l - j = d form one batched GEMM over j with
// consecutive slices of A and of B and an output every second order
// (k = 2j + d).  Set i holds the differences d = -i and d = i + 1 (d = 0 and 1
// for i = 0) of every batch element: they write orders of opposite parity, so
// no output is written twice within a set.  Set i has about T + 1 - i GEMMs
// per batch element, so sets i and T - i are launched together, into two
// accumulators (sets 0 .. T/2 into the first, whose set 0 writes every order
// once; the others into a zeroed second one), summed on the way out: about
// T/2 + 1 launches of T + 2 GEMMs per batch element each, instead of T + 1
// launches whose last ones fill a fraction of the SMs.
// ---------------------------------------------------------------------------
namespace {

struct NaiveWs {
  int* err;
  __nv_bfloat16 *slA, *slB;
  int *expA, *expB;
  float4 *Ct, *Ct2;   // the two accumulators (Ct2 unused at T = 0)
};

NaiveWs carve_naive(void* ws, int N, int T, int batch, int S, size_t* total) {
  WsCarver w(ws, SIZE_MAX);
  NaiveWs s;
  const long long Q = (long long)batch * (T + 1);
  s.err = w.take<int>(64);
  s.slA = w.take<__nv_bfloat16>((size_t)Q * S * 2 * N * nspt_split_kpad(N));
  s.slB = w.take<__nv_bfloat16>((size_t)Q * S * 3 * N * nspt_split_kpad(N));
  s.expA = w.take<int>((size_t)Q * N);
  s.expB = w.take<int>((size_t)Q * N);
  s.Ct = w.take<float4>((size_t)Q * N * N);
  s.Ct2 = T > 0 ? w.take<float4>((size_t)Q * N * N) : nullptr;
  if (total) *total = w.off;
  return s;
}

// e_r += (m k + c) log2r on the rows of slot k (k = 0..T) of the two slice sets (m, c per set;
// count = batch (T+1) N rows each): the slices then stand for exactly 2^((m k + c) log2r) times
// their orders.  Products: m = 1, c = 0 for both operands, so every A_l B_{k-l} comes out scaled
// by 2^(k log2r).  A zero row keeps zero digits whatever its exponent.
__global__ void naive_shift_exps_kernel(int* expA, int* expB, int N, int T1, long long count, int mA, int cA,
                                        int mB, int cB, int log2r, const int* dlr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int k = (int)((i / N) % T1);
  const int lr = dlr ? *dlr : log2r;
  expA[i] += (mA * k + cA) * lr;
  expB[i] += (mB * k + cB) * lr;
}

// C_k = 2^(sgn k log2r) (hi + lo) in FP64 of the sum of the two accumulators (Ct2 may be null),
// for count = batch (T+1) E entries (products: sgn = -1)
__global__ void naive_out_kernel(const float4* __restrict__ Ct, const float4* __restrict__ Ct2,
                                 double2* __restrict__ C, long long E, int T1, long long count, int sgn,
                                 int log2r, const int* dlr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int k = (int)((i / E) % T1);
  const int sh = sgn * k * (dlr ? *dlr : log2r);
  const float4 a = Ct[i];
  cdf v{dfl{a.x, a.y}, dfl{a.z, a.w}};
  if (Ct2) {
    const float4 b = Ct2[i];
    v = cdf_add(v, cdf{dfl{b.x, b.y}, dfl{b.z, b.w}});
  }
  double re = df_to_double(v.re), im = df_to_double(v.im);
  if (sh != 0) { re = scalbn(re, sh); im = scalbn(im, sh); }
  C[i] = make_double2(re, im);
}

int naive_shift(const NaiveWs& w, int N, int T, int batch, int mA, int cA, int mB, int cB, int log2r,
                const int* dlr, cudaStream_t st) {
  const long long rows = (long long)batch * (T + 1) * N;
  ProfScope ps(NSPT_STAGE_OTHER, st);
  naive_shift_exps_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(w.expA, w.expB, N, T + 1, rows, mA, cA,
                                                                         mB, cB, log2r, dlr);
  TRYC(cudaGetLastError());
  return NSPT_OK;
}

int naive_out(const NaiveWs& w, double2* C, int N, int T, int batch, int sgn, int log2r, const int* dlr,
              cudaStream_t st) {
  const long long E = (long long)N * N, cnt = (long long)batch * (T + 1) * E;
  ProfScope ps(NSPT_STAGE_OTHER, st);
  naive_out_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(w.Ct, w.Ct2, C, E, T + 1, cnt, sgn, log2r, dlr);
  TRYC(cudaGetLastError());
  return NSPT_OK;
}

// One batched GEMM of a pair schedule, the same for every batch element: cnt pair products whose
// left and right slices start at slots l0 and r0 (both rising by one) and whose outputs start at
// order o0 (rising by two), written into accumulator acc (0 or 1) plainly or added to it.
struct PairGroup { int launch, acc, l0, r0, o0, cnt, plain; };

// the product's schedule above: launch i holds set i (accumulator 0, plain for i = 0) and set
// T - i (accumulator 1, zeroed first)
std::vector<PairGroup> product_schedule(int T) {
  std::vector<PairGroup> g;
  auto add_set = [&](int launch, int i, int acc, bool plain) {
    const int ds[2] = {i == 0 ? 0 : -i, i + 1};
    for (int d : ds) {
      if (d > T) continue;
      const int j0 = std::max(0, -d);
      const int cnt = (T - d) / 2 - j0 + 1;  // j = j0 .. floor((T - d) / 2)
      if (cnt >= 1) g.push_back(PairGroup{launch, acc, j0 + d, j0, 2 * j0 + d, cnt, plain ? 1 : 0});
    }
  };
  for (int i = 0; 2 * i <= T; ++i) {
    add_set(i, i, 0, i == 0);
    if (T - i > i) add_set(i, T - i, 1, false);
  }
  return g;
}

// enqueues a schedule's launches in order, each group expanded over the batch, at most
// NSPT_SPLIT_MAX_PROBLEMS problems per launch
int run_pair_schedule(const NaiveWs& w, const std::vector<PairGroup>& sched, int N, int T, int batch, int S,
                      cudaStream_t st) {
  const int T1 = T + 1, Kp = nspt_split_kpad(N);
  const long long sa = (long long)S * 2 * N * Kp, sb = (long long)S * 3 * N * Kp, E = (long long)N * N;
  std::vector<SplitGemmArgs> probs;
  for (size_t gi = 0; gi < sched.size();) {
    probs.clear();
    const int launch = sched[gi].launch;
    for (; gi < sched.size() && sched[gi].launch == launch; ++gi) {
      const PairGroup& g = sched[gi];
      if (g.acc == 1 && !w.Ct2) return NSPT_ERR_ARG;
      for (int b = 0; b < batch; ++b) {
        const long long base = (long long)b * T1;
        SplitGemmArgs a;
        a.slicesA = w.slA + (base + g.l0) * sa;
        a.slicesB = w.slB + (base + g.r0) * sb;
        a.expA = w.expA + (base + g.l0) * N;
        a.expB = w.expB + (base + g.r0) * N;
        a.C = (g.acc == 0 ? w.Ct : w.Ct2) + (base + g.o0) * E;
        a.ldc_q = 2 * E;
        a.N = N; a.Kp = Kp; a.Q = g.cnt; a.S = S; a.num_sms = nspt_split_num_sms(); a.err = w.err;
        a.bn = nspt_split_default_bn(N);
        a.alpha = make_double2(1.0, 0.0); a.use_alpha = 0; a.accumulate = !g.plain;
        probs.push_back(a);
      }
    }
    for (size_t o = 0; o < probs.size(); o += NSPT_SPLIT_MAX_PROBLEMS) {
      const int n = (int)std::min<size_t>(NSPT_SPLIT_MAX_PROBLEMS, probs.size() - o);
      TRYS(nspt_split_gemm_batch(probs.data() + o, n, S, nspt_split_default_bn(N), nspt_split_num_sms(),
                                 st));
    }
  }
  return NSPT_OK;
}

int naive_gemms(const NaiveWs& w, int N, int T, int batch, int S, cudaStream_t st) {
  if (T > 0) TRYC(cudaMemsetAsync(w.Ct2, 0, (size_t)batch * (T + 1) * N * N * sizeof(float4), st));
  return run_pair_schedule(w, product_schedule(T), N, T, batch, S, st);
}

// The backward's schedule.  gA_j = sum_k gC_k (B_{k-j})^H and gB_j = sum_k (A_{k-j})^H gC_k
// are sums over the pairs (k, m = k - j).  Group s (0..2T) holds the pairs with k + m = s,
// max(ceil(s/2), s - T) <= k <= min(s, T): its output j = 2k - s runs over every second order,
// and the operand indexed by m is sliced in reversed order (slot T - m), so both operands' slots
// rise by one with k (left_rev: the left operand is the m-indexed one).  Groups of one parity
// write one parity of j.  Accumulator 0 takes the groups s <= T, accumulator 1 the groups
// s > T (both zeroed first); in each, the even groups in ascending size go with the odd groups
// in descending size, one such pair per accumulator per launch, so that the launches hold
// about T + 2 GEMMs per batch element each.
std::vector<PairGroup> corr_schedule(int T, bool left_rev) {
  struct Grp { int s, k0, cnt; };
  std::vector<std::vector<Grp>> lists[2];
  for (int a = 0; a < 2; ++a) {
    std::vector<Grp> ev, od;
    for (int s = (a == 0 ? 0 : T + 1); s <= (a == 0 ? T : 2 * T); ++s) {
      Grp g;
      g.s = s;
      g.k0 = std::max((s + 1) / 2, s - T);
      g.cnt = std::min(s, T) - g.k0 + 1;
      if (g.cnt >= 1) (s % 2 ? od : ev).push_back(g);
    }
    auto smaller = [](const Grp& x, const Grp& y) { return x.cnt < y.cnt || (x.cnt == y.cnt && x.s < y.s); };
    std::sort(ev.begin(), ev.end(), smaller);
    std::sort(od.begin(), od.end(), smaller);
    for (size_t i = 0; i < std::max(ev.size(), od.size()); ++i) {
      std::vector<Grp> l;
      if (i < ev.size()) l.push_back(ev[i]);
      if (i < od.size()) l.push_back(od[od.size() - 1 - i]);
      lists[a].push_back(l);
    }
  }
  std::vector<PairGroup> out;
  for (size_t li = 0; li < std::max(lists[0].size(), lists[1].size()); ++li)
    for (int a = 0; a < 2; ++a) {
      if (li >= lists[a].size()) continue;
      for (const Grp& g : lists[a][li]) {
        const int up = g.k0, down = T - g.s + g.k0;   // slots of the k- and m-indexed operands
        out.push_back(PairGroup{(int)li, a, left_rev ? down : up, left_rev ? up : down, 2 * g.k0 - g.s, g.cnt, 0});
      }
    }
  return out;
}

int corr_gemms(const NaiveWs& w, int N, int T, int batch, int S, bool left_rev, cudaStream_t st) {
  const size_t bytes = (size_t)batch * (T + 1) * N * N * sizeof(float4);
  TRYC(cudaMemsetAsync(w.Ct, 0, bytes, st));
  if (w.Ct2) TRYC(cudaMemsetAsync(w.Ct2, 0, bytes, st));
  return run_pair_schedule(w, corr_schedule(T, left_rev), N, T, batch, S, st);
}

}  // namespace

int nspt_debug_pair_schedule(int T, int kind, int* out, int cap) {
  if (T < 0 || T > 255 || kind < 0 || kind > 2 || cap < 0 || (cap > 0 && !out)) return NSPT_ERR_ARG;
  const std::vector<PairGroup> g = kind == 0 ? product_schedule(T) : corr_schedule(T, kind == 2);
  for (size_t i = 0; i < g.size() && (int)(7 * i + 7) <= cap; ++i) {
    const int v[7] = {g[i].launch, g[i].acc, g[i].l0, g[i].r0, g[i].o0, g[i].cnt, g[i].plain};
    for (int c = 0; c < 7; ++c) out[7 * i + c] = v[c];
  }
  return (int)g.size();
}

size_t nspt_split_ws_naive(int N, int T, int batch, int S) {
  size_t total = 0;
  carve_naive(nullptr, N, T, batch, S, &total);
  return total;
}

int nspt_split_mul_naive(int N, int T, int batch, int S, int log2r, bool rescale_auto, const double2* A,
                         const double2* B, double2* C, void* ws, cudaStream_t st) {
  NaiveWs w = carve_naive(ws, N, T, batch, S, nullptr);
  const int T1 = T + 1, Q = batch * T1;
  // fitted rescale into a spare word of the status block (the per-order maxima go to the
  // accumulator, which the first GEMM launch overwrites)
  int* dlr = nullptr;
  if (rescale_auto) {
    dlr = w.err + 16;
    TRYS(nspt_split_fit_rescale_dev(A, B, N, T, batch, reinterpret_cast<int*>(w.Ct), dlr, st));
  }
  TRYC(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // a2: slices of every order, the two operands on side streams
  TRYS(nspt_split_fork_join(2, st, [&](int i, cudaStream_t s) -> int {
    if (i == 0) return nspt_split_slice(S, A, T1, T1, 0, 0, 0, N, Q, 2, w.slA, w.expA, s);
    return nspt_split_slice(S, B, T1, T1, 0, 1, 0, N, Q, 3, w.slB, w.expB, s);
  }));
  if (rescale_auto || log2r != 0) TRYS(naive_shift(w, N, T, batch, 1, 0, 1, 0, log2r, dlr, st));
  // a3 (Eq. 5): the pair GEMMs, accumulated in double-float
  TRYS(naive_gemms(w, N, T, batch, S, st));
  return naive_out(w, C, N, T, batch, -1, log2r, dlr, st);
}

int nspt_split_bwd_naive(int N, int T, int batch, int S, int log2r, const double2* A, const double2* B,
                         const double2* G, double2* gA, double2* gB, void* ws, cudaStream_t st) {
  NaiveWs w = carve_naive(ws, N, T, batch, S, nullptr);
  const int T1 = T + 1, Q = batch * T1;
  TRYC(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // with the rescale, gC_k stands for 2^(-k log2r) gC_k and A_m, B_m for 2^(m log2r) A_m, B_m
  // (exponent shifts), so the order-j outputs come out scaled by 2^(-j log2r)
  if (gA) {
    // left: rows of gC_k (slots k); right: rows of (B_m^H)^T = conj(B_m) (slots T - m)
    TRYS(nspt_split_fork_join(2, st, [&](int i, cudaStream_t s) -> int {
      if (i == 0) return nspt_split_slice(S, G, T1, T1, 0, 0, 0, N, Q, 2, w.slA, w.expA, s);
      return nspt_split_slice(S, B, T1, T1, 2, 0, 1, N, Q, 3, w.slB, w.expB, s);
    }));
    if (log2r) TRYS(naive_shift(w, N, T, batch, -1, 0, -1, T, log2r, nullptr, st));
    TRYS(corr_gemms(w, N, T, batch, S, false, st));
    TRYS(naive_out(w, gA, N, T, batch, 1, log2r, nullptr, st));
  }
  if (gB) {
    // left: rows of A_m^H = conjugated columns of A_m (slots T - m); right: rows of gC_k^T =
    // columns of gC_k (slots k)
    TRYS(nspt_split_fork_join(2, st, [&](int i, cudaStream_t s) -> int {
      if (i == 0) return nspt_split_slice(S, A, T1, T1, 2, 1, 1, N, Q, 2, w.slA, w.expA, s);
      return nspt_split_slice(S, G, T1, T1, 0, 1, 0, N, Q, 3, w.slB, w.expB, s);
    }));
    if (log2r) TRYS(naive_shift(w, N, T, batch, -1, T, -1, 0, log2r, nullptr, st));
    TRYS(corr_gemms(w, N, T, batch, S, true, st));
    TRYS(naive_out(w, gB, N, T, batch, 1, log2r, nullptr, st));
  }
  return NSPT_OK;
}

