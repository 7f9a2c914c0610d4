// Split-precision product path (Sec. 2 Steps 1-5 with Step 3 on the tensor
// cores): FP64 series -> double-float spectra (fftdf.cu; the right operand's
// spectra written transposed) -> BF16 digit slices -> tensor-core mode GEMMs
// with exact FP32 digit groups -> double-float spectrum -> inverse transform
// to FP64.  Also the backward, the grouped launch with its tile autotuner,
// and the split-form Langevin step / MD phases.
//
// Slicing (an error-free split in the spirit of Ozaki et al.): each row r of
// an operand gets e_r with |x| < 2^e_r for all of its real and imaginary
// parts, and x 2^-e_r is cut into S balanced base-256 digits d_0..d_{S-1}
// (|d_i| <= 128 for the leading digits), so x = 2^(e_r - 7) sum_i d_i 2^(-8i)
// up to 2^(e_r - 8S); digit i is stored as the BF16 value d_i * 2^(-8i)
// (exact).  The digits of FP64 values come from the bit pattern, those of
// double-float values from FP32 rounding steps (digits.cuh); no FP64
// arithmetic is used, since on B300 the FP64 pipe is about 1/58 of FP32.
#include <algorithm>
#include <cmath>
#include <functional>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "prof.cuh"
#include "split.cuh"
#include "split_gemm.cuh"
#include "zgemm64.cuh"
#include "dfloat.cuh"
#include "digits.cuh"
#include "tek.cuh"

namespace {

int g_num_sms = 0;

using namespace digits;

// grid (ceil(N/RB), Q); block 256.  Output row r of plane q is row r of the
// source matrix (trans = 0) or its column r (trans = 1), conjugated if conj;
// P = 2 planes per digit (re, im) for a left operand, P = 3 (re, im, -re) for a
// right operand of the tensor-core GEMM;
// the source of plane q = b*M + p is mode p (rev = 0), (M - p) mod M (rev = 1) or
// M - 1 - p (rev = 2, this kernel only: order series stored from the last order down)
// of batch element b.
constexpr int RB = 8;  // output rows per CTA

// four floats as four round-to-nearest bf16 values in one 8-byte word
__device__ __forceinline__ uint2 pack_bf16x4(float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// Shared-memory layout of slice_kernel: the rows of the output block, row rr at rr * ldr (ldr
// odd and >= N rounded up to 4), entry k of a row at slice_swz(k) = k ^ ((k >> 3) & 3).  Both
// staging patterns (a warp writing 32 consecutive entries of one row; a quarter warp writing one
// entry of each of 8 rows) and the digit stage (a lane reading 4 adjacent entries) then touch 8
// distinct 16-byte bank groups per quarter warp.
__host__ __device__ constexpr int slice_ldr(int N) { return ((N + 3) & ~3) + 1; }
__device__ __forceinline__ int slice_swz(int k) { return k ^ ((k >> 3) & 3); }

// RBK output rows per CTA: 8 for row sources, 16 for column sources (trans), whose staging then
// reads 256-byte runs of 16 consecutive entries
template <int S, typename InT, int RBK>
__global__ void __launch_bounds__(256, 3)
slice_kernel(const InT* __restrict__ X, long long bstride, int M, int rev, int trans, int conj, int N, int Kp,
             int P, __nv_bfloat16* __restrict__ out, int* __restrict__ exps) {
  extern __shared__ __align__(16) unsigned char tile_raw[];
  InT* tile = reinterpret_cast<InT*>(tile_raw);
  const int q = blockIdx.y;
  const int b = q / M, p = q % M;
  const int sp = rev == 2 ? M - 1 - p : (rev ? (M - p) % M : p);
  const InT* Xm = X + ((long long)b * bstride + sp) * N * N;
  const int r0 = blockIdx.x * RBK;
  const int nr = min(RBK, N - r0);
  const int ldr = slice_ldr(N);
  if (!trans) {
    // one warp per source row: coalesced row reads, four loads in flight per thread
    for (int rr = threadIdx.x >> 5; rr < nr; rr += blockDim.x >> 5) {
      const InT* src = Xm + (long long)(r0 + rr) * N;
      InT* dst = tile + rr * ldr;
      int k = threadIdx.x & 31;
      for (; k + 96 < N; k += 128) {
        const InT x0 = src[k], x1 = src[k + 32], x2 = src[k + 64], x3 = src[k + 96];
        dst[slice_swz(k)] = x0; dst[slice_swz(k + 32)] = x1; dst[slice_swz(k + 64)] = x2; dst[slice_swz(k + 96)] = x3;
      }
      for (; k < N; k += 32) dst[slice_swz(k)] = src[k];
    }
  } else {
    // RBK consecutive entries of every source row: one 128- or 256-byte run per row
    const int rr = threadIdx.x % RBK;
    constexpr int STEP = 256 / RBK;
    if (rr < nr) {
      const InT* src = Xm + r0 + rr;
      InT* dst = tile + rr * ldr;
      int k = threadIdx.x / RBK;
      for (; k + 3 * STEP < N; k += 4 * STEP) {
        const InT x0 = src[(long long)k * N], x1 = src[(long long)(k + STEP) * N];
        const InT x2 = src[(long long)(k + 2 * STEP) * N], x3 = src[(long long)(k + 3 * STEP) * N];
        dst[slice_swz(k)] = x0; dst[slice_swz(k + STEP)] = x1;
        dst[slice_swz(k + 2 * STEP)] = x2; dst[slice_swz(k + 3 * STEP)] = x3;
      }
      for (; k < N; k += STEP) dst[slice_swz(k)] = src[(long long)k * N];
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long plane = (long long)N * Kp;
  for (int rr = warp; rr < nr; rr += blockDim.x / 32) {
    const InT* row = tile + rr * ldr;
    auto elem = [&](int k) -> InT {
      const InT v = row[slice_swz(k)];
      return conj ? conj_of(v) : v;
    };
    int mx = -100000;
    for (int k = lane; k < N; k += 32) mx = max(mx, exp_bound(elem(k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int e = (mx == -100000) ? -1000 : mx;  // |x| < 2^e for every part of the row
    const int r = r0 + rr;
    if (lane == 0) exps[(long long)q * N + r] = e;
    __nv_bfloat16* orow = out + (long long)q * S * P * plane + (long long)r * Kp;
    // four adjacent entries per lane; lanes 2j and 2j + 1 hold entries 8j..8j+7 of a chunk and
    // trade halves (one shuffle per word), so that every plane leaves in 16-byte stores: the even
    // lane stores the re (and -re: sign bits flipped, exact) digits of the eight entries, the odd
    // lane the im digits.  Every lane runs every chunk, so the shuffles see the whole warp.  (Held
    // to three CTAs per SM by the launch bounds: 80 registers, a few bytes of spills.)
    const bool odd = lane & 1;
    const int k8 = 8 * (lane >> 1);
    for (int k0 = 0; k0 < N; k0 += 128) {
      const int k = k0 + 4 * lane;
      const bool act = k0 + k8 < N;   // the pair's eight entries start inside the row (and Kp)
      float re[4][S], im[4][S];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const InT v = (k + c < N) ? elem(k + c) : zero_of(row[0]);
        digits_re_im<S>(v, e, re[c], im[c]);
      }
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const uint2 pr = pack_bf16x4(re[0][i], re[1][i], re[2][i], re[3][i]);
        const uint2 pi = pack_bf16x4(im[0][i], im[1][i], im[2][i], im[3][i]);
        const uint2 send = odd ? pr : pi;
        const unsigned gx = __shfl_xor_sync(0xffffffffu, send.x, 1), gy = __shfl_xor_sync(0xffffffffu, send.y, 1);
        if (!act) continue;
        __nv_bfloat16* o = orow + (long long)P * i * plane + k0 + k8;
        if (!odd) {
          const uint4 w = make_uint4(pr.x, pr.y, gx, gy);
          *reinterpret_cast<uint4*>(o) = w;
          if (P == 3)
            *reinterpret_cast<uint4*>(o + 2 * plane) =
                make_uint4(w.x ^ 0x80008000u, w.y ^ 0x80008000u, w.z ^ 0x80008000u, w.w ^ 0x80008000u);
        } else {
          *reinterpret_cast<uint4*>(o + plane) = make_uint4(gx, gy, pi.x, pi.y);
        }
      }
    }
  }
}

// Row form without shared memory (trans = 0, double-float spectra): one warp
// per output row; every lane loads its NQ quads of four adjacent entries up
// front (all loads in flight at once), the row exponent is a warp max over the
// registers, and the digits are produced one digit index at a time for the
// four entries, each leaving as one 8-byte bf16x4 store per plane (256
// contiguous bytes per warp store).  Same output as slice_kernel.  With sum3
// (P = 3) the third plane holds the digits of re + im (the 3M product's
// operand) at the row exponent e + 1 instead of -re: |re + im| < 2^(e+1).

// W consecutive bf16 values as one 8-byte (W = 4) or 16-byte (W = 8) store
template <int W>
__device__ __forceinline__ void store_bf16(__nv_bfloat16* o, const float (&d)[W]) {
  if constexpr (W == 4) {
    *reinterpret_cast<uint2*>(o) = pack_bf16x4(d[0], d[1], d[2], d[3]);
  } else {
    static_assert(W == 8, "4 or 8 entries per store");
    const uint2 a = pack_bf16x4(d[0], d[1], d[2], d[3]), b = pack_bf16x4(d[4], d[5], d[6], d[7]);
    *reinterpret_cast<uint4*>(o) = make_uint4(a.x, a.y, b.x, b.y);
  }
}

// W adjacent entries per lane and chunk (4: 8-byte stores, 8: 16-byte stores); NQ chunks of
// LPR W entries per row, LPR lanes per row: 32, or 16 with two rows per warp (TWO, for rows of at
// most 16 W entries, which then keep every lane busy)
template <int S, int NQ, int W, bool SUM3, bool TWO = false>
__global__ void __launch_bounds__(256, NQ * W <= 8 ? 4 : 2)
slice_rows_kernel(const float4* __restrict__ X, long long bstride, int M, int rev, int conj, int N, int Kp, int P,
                  __nv_bfloat16* __restrict__ out, int* __restrict__ exps) {
  constexpr bool sum3 = SUM3;
  constexpr int LPR = TWO ? 16 : 32, RPW = 32 / LPR;
  const int q = blockIdx.y;
  const int b = q / M, p = q % M;
  const int sp = rev ? (M - p) % M : p;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ln = lane % LPR, r0 = (blockIdx.x * RB + warp) * RPW;
  const int r = r0 + lane / LPR;
  if (r0 >= N) return;                 // every row of the warp is past the end
  const bool rv = r < N;               // (TWO) the warp's second row may be past the end
  const float4* src = X + ((long long)b * bstride + sp) * N * N + (long long)(rv ? r : r0) * N;
  float4 v[NQ][W];
#pragma unroll
  for (int t = 0; t < NQ; ++t) {
    const int k = W * ln + LPR * W * t;
#pragma unroll
    for (int c = 0; c < W; ++c) v[t][c] = (rv && k + c < N) ? src[k + c] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int mx = -100000;
#pragma unroll
  for (int t = 0; t < NQ; ++t)
#pragma unroll
    for (int c = 0; c < W; ++c) mx = max(mx, exp_bound(v[t][c]));
#pragma unroll
  for (int o = LPR / 2; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (!rv) return;                     // no shuffles below
  const int e = (mx == -100000) ? -1000 : mx;  // |x| < 2^e for every part of the row
  if (ln == 0) exps[(long long)q * N + r] = e;
  const long long plane = (long long)N * Kp;
  __nv_bfloat16* orow = out + (long long)q * S * P * plane + (long long)r * Kp;
  float f1, f2, g1, g2;
  pow2_pair(-e, f1, f2);
  pow2_pair(-e - 1, g1, g2);
#pragma unroll
  for (int t = 0; t < NQ; ++t) {
    const int k = W * ln + LPR * W * t;
    if (k >= N) break;
    // residuals of x 2^-e (|.| < 1) for the real and imaginary parts of the W entries,
    // and (3M) of (re + im) 2^-(e+1)
    float vr[W], vi[W], lr[W], li[W], vs[W], ls[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      const float4 x = v[t][c];
      const float sg = conj ? -1.f : 1.f;
      vr[c] = (x.x * f1) * f2;
      lr[c] = (x.y * f1) * f2;
      vi[c] = sg * ((x.z * f1) * f2);
      li[c] = sg * ((x.w * f1) * f2);
      if (sum3) {
        const dfl su = df_add(dfl{x.x, x.y}, dfl{sg * x.z, sg * x.w});
        vs[c] = (su.h * g1) * g2;
        ls[c] = (su.l * g1) * g2;
      } else {
        vs[c] = 0.f;
        ls[c] = 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      // digit i: t = v rounded to a multiple of 2^(-7-8i); lo joins before digit 3 (see to_digits)
      const float sig = __int_as_float(((143 - 8 * i) << 23) | 0x400000);
      float dr[W], di[W], ds[W];
#pragma unroll
      for (int c = 0; c < W; ++c) {
        if (i == 3) { vr[c] = vr[c] + lr[c]; vi[c] = vi[c] + li[c]; vs[c] = vs[c] + ls[c]; }
        const float tr = (vr[c] + sig) - sig, ti = (vi[c] + sig) - sig, ts = (vs[c] + sig) - sig;
        vr[c] = vr[c] - tr;
        vi[c] = vi[c] - ti;
        vs[c] = vs[c] - ts;
        dr[c] = tr * 128.f;
        di[c] = ti * 128.f;
        ds[c] = ts * 128.f;
      }
      __nv_bfloat16* o = orow + (long long)P * i * plane + k;
      if (P == 3 && !sum3) {
#pragma unroll
        for (int c = 0; c < W; ++c) ds[c] = -dr[c];
      }
      store_bf16<W>(o, dr);
      store_bf16<W>(o + plane, di);
      if (P == 3) store_bf16<W>(o + 2 * plane, ds);
    }
  }
}

template <int S, int NQ, int W, bool TWO = false>
int launch_slice_rows(const float4* X, long long bstride, int M, int rev, int conj, int N, int Kp, int Q, int P,
                      int sum3, __nv_bfloat16* out, int* exps, cudaStream_t st) {
  constexpr int rows = RB * (TWO ? 2 : 1);   // rows per CTA
  dim3 grid((N + rows - 1) / rows, Q);
  ProfScope ps(NSPT_STAGE_SLICE, st);
  if (sum3) {
    if constexpr (S <= 6) {
      slice_rows_kernel<S, NQ, W, true, TWO><<<grid, 256, 0, st>>>(X, bstride, M, rev, conj, N, Kp, P, out, exps);
    } else {
      return NSPT_ERR_UNSUPPORTED;
    }
  } else {
    slice_rows_kernel<S, NQ, W, false, TWO><<<grid, 256, 0, st>>>(X, bstride, M, rev, conj, N, Kp, P, out, exps);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

template <int S, typename InT>
int launch_slice(const InT* X, long long bstride, int M, int rev, int trans, int conj, int N, int Kp, int Q, int P,
                 int sum3, __nv_bfloat16* out, int* exps, cudaStream_t st) {
  if (rev < 0 || rev > 2) return NSPT_ERR_ARG;
  if constexpr (std::is_same<InT, float4>::value) {
    if (!trans && N <= 512) {
      if (rev == 2) return NSPT_ERR_UNSUPPORTED;   // the row form takes rev = 0, 1
      // two rows per warp up to 16 W entries a row
      if (N <= 64) return launch_slice_rows<S, 1, 4, true>(X, bstride, M, rev, conj, N, Kp, Q, P, sum3, out, exps, st);
      if (N <= 128) return launch_slice_rows<S, 1, 8, true>(X, bstride, M, rev, conj, N, Kp, Q, P, sum3, out, exps, st);
      if (N <= 256) return launch_slice_rows<S, 1, 8>(X, bstride, M, rev, conj, N, Kp, Q, P, sum3, out, exps, st);
      return launch_slice_rows<S, 2, 8>(X, bstride, M, rev, conj, N, Kp, Q, P, sum3, out, exps, st);
    }
  }
  if (sum3) return NSPT_ERR_UNSUPPORTED;  // the (re + im) plane: row form only
  // column sources: 16 rows per CTA while the tile stays within 200 KB of shared memory (32 rows,
  // one CTA per SM at N = 225, measured slower)
  const bool wide = trans && (size_t)16 * slice_ldr(N) * sizeof(InT) <= (size_t)200 * 1024;
  const int rbk = wide ? 16 : RB;
  auto kern = wide ? slice_kernel<S, InT, 16> : slice_kernel<S, InT, RB>;
  const size_t smem = (size_t)rbk * slice_ldr(N) * sizeof(InT);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  dim3 grid((N + rbk - 1) / rbk, Q);
  ProfScope ps(NSPT_STAGE_SLICE, st);
  kern<<<grid, 256, smem, st>>>(X, bstride, M, rev, trans, conj, N, Kp, P, out, exps);
  e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

int kpad(int N) { return nspt_split_kpad(N); }

struct SplitWs {
  float4 *At, *Bt;
  __nv_bfloat16 *slA, *slB;
  int *expA, *expB, *err;
  float4* Ct;
};

// cm = 3: the left operand's slices carry a third plane (re + im) as well
SplitWs carve(void* ws, int N, int batch, int M, int S, size_t* total, int cm = 4) {
  WsCarver w(ws, SIZE_MAX);
  SplitWs s;
  const long long E = (long long)N * N, Q = (long long)batch * M;
  s.err = w.take<int>(64);
  s.At = w.take<float4>((size_t)Q * E);
  s.Bt = w.take<float4>((size_t)Q * E);
  s.slA = w.take<__nv_bfloat16>((size_t)Q * S * (cm == 3 ? 3 : 2) * N * kpad(N));
  s.slB = w.take<__nv_bfloat16>((size_t)Q * S * 3 * N * kpad(N));
  s.expA = w.take<int>((size_t)Q * N);
  s.expB = w.take<int>((size_t)Q * N);
  s.Ct = s.At;  // A~ is dead once sliced
  if (total) *total = w.off;
  return s;
}

// ---------------- tile-width table filled by the autotuner ----------------
std::mutex g_tune_mu;
std::map<std::string, int> g_tuned_bn;

std::string signature(int S, const std::vector<std::pair<int, int>>& nq) {
  std::string sig = "S" + std::to_string(S);
  for (auto& x : nq) sig += ";" + std::to_string(x.first) + "x" + std::to_string(x.second);
  return sig;
}

// untuned default for products of size at most nmax: 32 complex columns per tile up to N = 128
// (where 48 would pad 121..128 columns to 144), else 48.  Measured at SU(121): the split Langevin
// step 36.9 -> 35.2 ms, the 40-step MD trajectory at O(g^15) 110.6 -> 108.5 ms, a lone O(g^15)
// product of batch 4 2% slower (fewer tiles than two waves); the autotuner overrides it per
// signature
int default_bn(int nmax) { return nmax <= 128 ? 32 : 48; }

int choose_bn(const std::string& sig, int nmax) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned_bn.find(sig);
  return it == g_tuned_bn.end() ? default_bn(nmax) : it->second;
}

SplitGemmArgs gemm_args(const SplitWs& w, int N, int Q, int S) {
  SplitGemmArgs a;
  a.slicesA = w.slA; a.slicesB = w.slB; a.expA = w.expA; a.expB = w.expB; a.C = w.Ct;
  a.N = N; a.Kp = kpad(N); a.Q = Q; a.S = S; a.num_sms = g_num_sms; a.err = w.err; a.bn = 0;
  a.alpha = make_double2(1.0, 0.0); a.use_alpha = 0; a.accumulate = 0;
  return a;
}

int gemm(const SplitWs& w, int N, int Q, int S, cudaStream_t st) {
  SplitGemmArgs a = gemm_args(w, N, Q, S);
  a.bn = choose_bn(signature(S, {{N, Q}}), N);
  return nspt_split_gemm(a, st);
}

#define TRYC(x) do { cudaError_t _e = (x); if (_e != cudaSuccess) { nspt_set_last_cuda_error(_e); return NSPT_ERR_CUDA; } } while (0)
#define TRYS(x) do { int _r = (x); if (_r != NSPT_OK) return _r; } while (0)

}  // namespace

template <typename InT>
int slice_any(int S, const InT* X, long long bstride, int M, int rev, int trans, int conj, int N, int Q, int P,
              void* out, int* exps, cudaStream_t st, int sum3 = 0) {
  __nv_bfloat16* o = (__nv_bfloat16*)out;
  switch (S) {
#define NSPT_CASE(s) case s: return launch_slice<s, InT>(X, bstride, M, rev, trans, conj, N, kpad(N), Q, P, sum3, o, exps, st);
    NSPT_CASE(2) NSPT_CASE(3) NSPT_CASE(4) NSPT_CASE(5) NSPT_CASE(6) NSPT_CASE(7) NSPT_CASE(8)
#undef NSPT_CASE
    default: return NSPT_ERR_ARG;
  }
}

int nspt_split_slice(int S, const double2* X, long long bstride, int M, int rev, int trans, int conj, int N, int Q,
                     int P, void* out, int* exps, cudaStream_t st) {
  return slice_any<double2>(S, X, bstride, M, rev, trans, conj, N, Q, P, out, exps, st);
}

int nspt_split_slice_df(int S, const float4* X, long long bstride, int M, int rev, int trans, int conj, int N, int Q,
                        int P, void* out, int* exps, cudaStream_t st, int sum3) {
  return slice_any<float4>(S, X, bstride, M, rev, trans, conj, N, Q, P, out, exps, st, sum3);
}

// Library-owned side streams of a device: the independent per-product chains of a grouped call
// (transforms and slicing before the one GEMM launch, inverse transforms after it) run on them,
// forked from and joined back to the caller's stream by events, so that the small launches of
// different products overlap.  Under graph capture the fork and join become graph edges.  Made in
// nspt_init (never inside a capture); a mutex orders the enqueue of concurrent calls.
constexpr int kSideStreams = 4;
struct SideStreams {
  std::mutex mu;
  bool ok = false;
  cudaStream_t s[kSideStreams];
  cudaEvent_t fork, join[kSideStreams];
};
SideStreams g_side[64];

SideStreams* side_streams() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  return g_side[dev].ok ? &g_side[dev] : nullptr;
}

// enqueues chain(i, stream) for i < count, spread over the side streams between a fork from and a
// join back to st; without side streams the chains run on st
template <typename F>
int fork_join(int count, cudaStream_t st, F chain) {
  SideStreams* ss = side_streams();
  if (!ss) {
    for (int i = 0; i < count; ++i) TRYS(chain(i, st));
    return NSPT_OK;
  }
  std::lock_guard<std::mutex> lk(ss->mu);
  const int k = std::min(count, kSideStreams);
  TRYC(cudaEventRecord(ss->fork, st));
  for (int j = 0; j < k; ++j) TRYC(cudaStreamWaitEvent(ss->s[j], ss->fork, 0));
  int rc = NSPT_OK;
  for (int i = 0; i < count && rc == NSPT_OK; ++i) rc = chain(i, ss->s[i % k]);
  // join even after a failed enqueue, so that st never runs ahead of work already queued
  for (int j = 0; j < k; ++j) {
    TRYC(cudaEventRecord(ss->join[j], ss->s[j]));
    TRYC(cudaStreamWaitEvent(st, ss->join[j], 0));
  }
  return rc;
}

int nspt_split_init() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (dev >= 0 && dev < 64) {
    SideStreams& ss = g_side[dev];
    std::lock_guard<std::mutex> lk(ss.mu);
    if (!ss.ok) {
      bool good = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess;
      for (int j = 0; j < kSideStreams && good; ++j)
        good = cudaStreamCreateWithFlags(&ss.s[j], cudaStreamNonBlocking) == cudaSuccess &&
               cudaEventCreateWithFlags(&ss.join[j], cudaEventDisableTiming) == cudaSuccess;
      ss.ok = good;   // on failure the grouped calls run their chains on the caller's stream
    }
  }
  return nspt_split_gemm_init();
}

size_t nspt_split_ws_mul(int N, int T, int batch, int M, int S, int cm) {
  size_t total = 0;
  carve(nullptr, N, batch, M, S, &total, cm);
  return total;
}

size_t nspt_split_ws_bwd(int N, int T, int batch, int M, int S) {
  // G~ spectrum in addition to the product workspace
  return nspt_split_ws_mul(N, T, batch, M, S) + (((size_t)batch * M * N * N * sizeof(double2) + 255) & ~(size_t)255);
}

namespace {

// per order k: the largest FP64 exponent field over the real and imaginary parts of
// every entry of A_k (out[k]) and of B_k (out[T + 1 + k]) across the batch (0 = all zero)
__global__ void order_maxexp_kernel(const double2* __restrict__ A, const double2* __restrict__ B, int* out, long long E,
                                    int T, int batch) {
  const int k = blockIdx.y;
  int ma = 0, mb = 0;
  for (int b = 0; b < batch; ++b) {
    const double2* a = A + ((long long)b * (T + 1) + k) * E;
    const double2* bb = B + ((long long)b * (T + 1) + k) * E;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < E; i += (long long)gridDim.x * blockDim.x) {
      const double2 x = a[i], y = bb[i];
      ma = max(ma, max((int)((__double_as_longlong(x.x) >> 52) & 0x7FF), (int)((__double_as_longlong(x.y) >> 52) & 0x7FF)));
      mb = max(mb, max((int)((__double_as_longlong(y.x) >> 52) & 0x7FF), (int)((__double_as_longlong(y.y) >> 52) & 0x7FF)));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
    mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out + k, ma);
    atomicMax(out + T + 1 + k, mb);
  }
}

}  // namespace

namespace {

// One block of 128 threads: candidate c (c <= 120) is log2r = 0, 1, -1, 2, -2, ... (c odd:
// (c + 1) / 2, c even: -c / 2).  Its spread max_k - min_k of y_k + 2 k log2r over the orders
// where both operands are nonzero, or +inf when it is not allowed; the smallest spread wins,
// the earliest candidate (smallest |log2r|) among equal spreads.  h: exponent fields of the
// per-order maxima of A (h[k]) and B (h[T + 1 + k]), 0 for an all-zero order.
__global__ void __launch_bounds__(128) fit_log2r_kernel(const int* __restrict__ h, int T, int float_range,
                                                        int* __restrict__ out) {
  __shared__ double spread[128];
  __shared__ int maxes[2];
  const int c = threadIdx.x;
  if (c == 0) {
    int ma = -100000, mb = -100000;
    for (int k = 0; k <= T; ++k) {
      if (h[k] != 0) ma = max(ma, h[k] - 1023);
      if (h[T + 1 + k] != 0) mb = max(mb, h[T + 1 + k] - 1023);
    }
    maxes[0] = ma;
    maxes[1] = mb;
  }
  __syncthreads();
  const int lr = (c % 2) ? (c + 1) / 2 : -(c / 2);
  const int capA = max(maxes[0], 0), capB = max(maxes[1], 0);
  bool ok = c <= 120 && !(float_range && abs(lr) * T > 120);
  double lo = 1e300, hi = -1e300;
  int ny = 0;
  for (int k = 0; k <= T; ++k) {
    const int a = h[k], b = h[T + 1 + k];
    if (a != 0 && a - 1023 + k * lr > capA) ok = false;
    if (b != 0 && b - 1023 + k * lr > capB) ok = false;
    if (a != 0 && b != 0) {
      const double v = (double)(a - 1023) + (double)(b - 1023) + 2.0 * k * lr;
      lo = fmin(lo, v);
      hi = fmax(hi, v);
      ++ny;
    }
  }
  spread[c] = ok ? hi - lo : 1e300;
  __syncthreads();
  if (c == 0) {
    int best_c = -1;
    double best = 1e300;
    if (ny >= 2)
      for (int i = 0; i <= 120; ++i)
        if (spread[i] < best - 1e-9) { best = spread[i]; best_c = i; }
    *out = best_c < 0 ? 0 : ((best_c % 2) ? (best_c + 1) / 2 : -(best_c / 2));
  }
}

}  // namespace

int nspt_split_fit_rescale_dev(const double2* A, const double2* B, int N, int T, int batch, int* scratch, int* out,
                               cudaStream_t st, bool float_range) {
  TRYC(cudaMemsetAsync(scratch, 0, sizeof(int) * 2 * (T + 1), st));
  const long long E = (long long)N * N;
  dim3 grid((unsigned)std::min<long long>((E + 255) / 256, 64), T + 1);
  {
    ProfScope ps(NSPT_STAGE_OTHER, st);
    order_maxexp_kernel<<<grid, 256, 0, st>>>(A, B, scratch, E, T, batch);
  }
  TRYC(cudaGetLastError());
  {
    ProfScope ps(NSPT_STAGE_OTHER, st);
    fit_log2r_kernel<<<1, 128, 0, st>>>(scratch, T, float_range ? 1 : 0, out);
  }
  TRYC(cudaGetLastError());
  return NSPT_OK;
}

int nspt_split_mul(int N, int T, int batch, int M, int S, int log2r, bool rescale_auto, const double2* A,
                   const double2* B, double2* C, void* ws, cudaStream_t st, int cm) {
  const int E = N * N, Q = batch * M;
  if (cm == 3 && (S > 6 || N > 512)) return NSPT_ERR_UNSUPPORTED;
  SplitWs w = carve(ws, N, batch, M, S, nullptr, cm);
  // fitted rescale: on the device, into a spare word of the status block (the maxima go to expA,
  // which the slicer overwrites later; the exponent must outlive it for the inverse transform)
  int* dlr = nullptr;
  if (rescale_auto) {
    dlr = w.err + 16;
    TRYS(nspt_split_fit_rescale_dev(A, B, N, T, batch, w.expA, dlr, st));
    log2r = 1;
  }
  NsptDevLog2r scope(dlr);
  TRYC(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // a0 + a1: per-order rescale A_k -> 2^(k log2r) A_k fused into the forward transform
  // (B's spectra are written transposed, so that both operands are sliced by rows)
  // a2: slices of A~_q (rows) and of B~_q^T (rows of the transposed spectra); the two operands'
  // chains run on side streams, so that one operand's transform overlaps the other's slicing
  // (3M: both operands' slices carry planes (re, im, re + im))
  TRYS(fork_join(2, st, [&](int i, cudaStream_t s) -> int {
    if (i == 0) {
      TRYC(nspt_fft_fwd_df(A, T + 1, w.At, E, T, batch, M, 0, log2r, s));
      TRYS(nspt_split_slice_df(S, w.At, M, M, 0, 0, 0, N, Q, cm == 3 ? 3 : 2, w.slA, w.expA, s, cm == 3));
    } else {
      TRYC(nspt_fft_fwd_df(B, T + 1, w.Bt, E, T, batch, M, 0, log2r, s, N));
      TRYS(nspt_split_slice_df(S, w.Bt, M, M, 0, 0, 0, N, Q, 3, w.slB, w.expB, s, cm == 3));
    }
    return NSPT_OK;
  }));
  // a3: mode GEMMs on the tensor cores
  if (cm == 3) {
    TRYS(nspt_split_gemm3m(gemm_args(w, N, Q, S), st));
  } else {
    TRYS(gemm(w, N, Q, S, st));
  }
  // a4: inverse transform, truncation, unscale 2^(-k log2r)
  TRYC(nspt_fft_inv_df(w.Ct, C, T + 1, E, T, batch, M, 0, log2r, st));
  return NSPT_OK;
}

int nspt_split_bwd(int N, int T, int batch, int M, int S, int log2r, const double2* A, const double2* B,
                   const double2* G, double2* gA, double2* gB, void* ws, cudaStream_t st) {
  const int E = N * N, Q = batch * M;
  size_t off = 0;
  SplitWs w = carve(ws, N, batch, M, S, &off);
  float4* Gt = reinterpret_cast<float4*>((char*)ws + off);
  TRYC(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // with A' = r^k A, B' = r^k B, G' = r^-k G the correlations come out scaled by r^-j
  TRYC(nspt_fft_fwd_df(G, T + 1, Gt, E, T, batch, M, 0, -log2r, st));
  if (gA) {
    // gA~_p = G~_p (B~_p)^H
    TRYC(nspt_fft_fwd_df(B, T + 1, w.Bt, E, T, batch, M, 0, log2r, st));
    TRYS(nspt_split_slice_df(S, Gt, M, M, 0, 0, 0, N, Q, 2, w.slA, w.expA, st));
    TRYS(nspt_split_slice_df(S, w.Bt, M, M, 0, 0, 1, N, Q, 3, w.slB, w.expB, st));
    TRYS(gemm(w, N, Q, S, st));
    TRYC(nspt_fft_inv_df(w.Ct, gA, T + 1, E, T, batch, M, 0, -log2r, st));
  }
  if (gB) {
    // gB~_p = (A~_p)^H G~_p
    TRYC(nspt_fft_fwd_df(A, T + 1, w.Bt, E, T, batch, M, 0, log2r, st, N));   // A~ transposed
    TRYS(nspt_split_slice_df(S, w.Bt, M, M, 0, 0, 1, N, Q, 2, w.slA, w.expA, st));
    TRYS(nspt_split_slice_df(S, Gt, M, M, 0, 1, 0, N, Q, 3, w.slB, w.expB, st));
    TRYS(gemm(w, N, Q, S, st));
    TRYC(nspt_fft_inv_df(w.Ct, gB, T + 1, E, T, batch, M, 0, -log2r, st));
  }
  return NSPT_OK;
}

int nspt_split_gemm_stage(const void* slA, const void* slB, const int* expA, const int* expB, void* C, int N, int Q,
                          int S, int* err, cudaStream_t st) {
  SplitGemmArgs a;
  a.slicesA = slA; a.slicesB = slB; a.expA = expA; a.expB = expB; a.C = (float4*)C;
  a.N = N; a.Kp = kpad(N); a.Q = Q; a.S = S; a.num_sms = g_num_sms; a.err = err; a.bn = 0;
  a.alpha = make_double2(1.0, 0.0); a.use_alpha = 0; a.accumulate = 0;
  return nspt_split_gemm(a, st);
}

int nspt_split_num_sms() { return g_num_sms; }
int nspt_split_default_bn(int nmax) { return default_bn(nmax); }
int nspt_split_fork_join(int count, cudaStream_t st, const std::function<int(int, cudaStream_t)>& chain) {
  return fork_join(count, st, chain);
}

int nspt_split_read_error(void* ws, int* host_err, cudaStream_t st) {
  if (!ws) return NSPT_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(host_err, ws, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// Grouped products: independent products of uneven (N, T) whose mode GEMMs
// run in one persistent tensor-core launch.
// ---------------------------------------------------------------------------
namespace {

int pow2_at_least(int x) {
  int m = 1;
  while (m < x) m <<= 1;
  return m;
}

struct GroupLayout {
  int* err;
  std::vector<SplitWs> ws;
  size_t total;
};

GroupLayout carve_group(void* base, const nspt_polymat_desc* d, int count, int S) {
  GroupLayout g;
  WsCarver w(base, SIZE_MAX);
  g.err = w.take<int>(64);
  for (int i = 0; i < count; ++i) {
    const int N = d[i].N, M = pow2_at_least(2 * (d[i].T + 1));
    const long long E = (long long)N * N, Q = (long long)d[i].batch * M;
    SplitWs s;
    s.err = g.err;
    s.At = w.take<float4>((size_t)Q * E);
    s.Bt = w.take<float4>((size_t)Q * E);
    s.slA = w.take<__nv_bfloat16>((size_t)Q * S * 2 * N * kpad(N));
    s.slB = w.take<__nv_bfloat16>((size_t)Q * S * 3 * N * kpad(N));
    s.expA = w.take<int>((size_t)Q * N);
    s.expB = w.take<int>((size_t)Q * N);
    s.Ct = s.At;
    g.ws.push_back(s);
  }
  g.total = w.off;
  return g;
}

std::string group_signature(const nspt_polymat_desc* d, int count, int S) {
  std::vector<std::pair<int, int>> nq;
  for (int i = 0; i < count; ++i) nq.push_back({d[i].N, d[i].batch * pow2_at_least(2 * (d[i].T + 1))});
  return signature(S, nq);
}

int group_prepare(const nspt_polymat_desc* d, int count, int S, int log2r, const GroupLayout& g,
                  std::vector<SplitGemmArgs>& args, cudaStream_t st) {
  TRYC(cudaMemsetAsync(g.err, 0, sizeof(int), st));
  args.clear();
  for (int i = 0; i < count; ++i) {
    const int N = d[i].N, M = pow2_at_least(2 * (d[i].T + 1));
    args.push_back(gemm_args(g.ws[i], N, d[i].batch * M, S));
  }
  // every product's transforms and slicing: independent chains (own workspace regions)
  return fork_join(count, st, [&](int i, cudaStream_t s) -> int {
    const int N = d[i].N, T = d[i].T, b = d[i].batch, M = pow2_at_least(2 * (T + 1));
    const int E = N * N, Q = b * M;
    const SplitWs& w = g.ws[i];
    TRYC(nspt_fft_fwd_df((const double2*)d[i].A, T + 1, w.At, E, T, b, M, 0, log2r, s));
    TRYC(nspt_fft_fwd_df((const double2*)d[i].B, T + 1, w.Bt, E, T, b, M, 0, log2r, s, N));
    TRYS(nspt_split_slice_df(S, w.At, M, M, 0, 0, 0, N, Q, 2, w.slA, w.expA, s));
    TRYS(nspt_split_slice_df(S, w.Bt, M, M, 0, 0, 0, N, Q, 3, w.slB, w.expB, s));
    return NSPT_OK;
  });
}

}  // namespace

size_t nspt_split_ws_grouped(const nspt_polymat_desc* d, int count, int S) {
  return carve_group(nullptr, d, count, S).total;
}

int nspt_split_mul_grouped(const nspt_polymat_desc* d, int count, int S, int log2r, void* ws, cudaStream_t st) {
  GroupLayout g = carve_group(ws, d, count, S);
  std::vector<SplitGemmArgs> args;
  TRYS(group_prepare(d, count, S, log2r, g, args, st));
  int nmax = 1;
  for (int i = 0; i < count; ++i) nmax = std::max(nmax, d[i].N);
  TRYS(nspt_split_gemm_batch(args.data(), count, S, choose_bn(group_signature(d, count, S), nmax), g_num_sms, st));
  return fork_join(count, st, [&](int i, cudaStream_t s) -> int {
    const int N = d[i].N, T = d[i].T, M = pow2_at_least(2 * (T + 1));
    TRYC(nspt_fft_inv_df(g.ws[i].Ct, (double2*)d[i].C, T + 1, N * N, T, d[i].batch, M, 0, log2r, s));
    return NSPT_OK;
  });
}

int nspt_split_autotune_grouped(const nspt_polymat_desc* d, int count, int S, void* ws, const char* cache_path,
                                int* chosen, cudaStream_t st) {
  const std::string sig = group_signature(d, count, S);
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char key[8192];
      int bn = 0;
      while (fscanf(f, "%8191s %d", key, &bn) == 2) {
        if (sig == key && (bn == 32 || bn == 40 || bn == 48)) {
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tuned_bn[sig] = bn;
        }
      }
      fclose(f);
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_bn.find(sig);
    if (it != g_tuned_bn.end()) { *chosen = it->second; return NSPT_OK; }
  }
  GroupLayout g = carve_group(ws, d, count, S);
  std::vector<SplitGemmArgs> args;
  TRYS(group_prepare(d, count, S, 0, g, args, st));
  const int cands[3] = {32, 40, 48};  // 40: left operand held in tensor memory
  float best = 1e30f;
  int best_bn = 48;
  cudaEvent_t e0, e1;
  TRYC(cudaEventCreate(&e0));
  TRYC(cudaEventCreate(&e1));
  for (int bn : cands) {
    int rc = nspt_split_gemm_batch(args.data(), count, S, bn, g_num_sms, st);  // warm-up
    for (int r = 0; r < 3 && rc == NSPT_OK; ++r) {
      if (r == 0) cudaEventRecord(e0, st);
      rc = nspt_split_gemm_batch(args.data(), count, S, bn, g_num_sms, st);
    }
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || rc != NSPT_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc ? rc : NSPT_ERR_CUDA;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_bn = bn; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_bn[sig] = best_bn;
  }
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s %d\n", sig.c_str(), best_bn);
      fclose(f);
    }
  }
  *chosen = best_bn;
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// Langevin step of the TEK model in the split form (Eqs. 1-3): the same
// sequence of star products as the FP64 form, with double-float spectra,
// digit slices and tensor-core mode GEMMs.  Spectra of daggered series come
// from the spectra of the series themselves: FFT(X^+)_p = (X~_{(M-p) mod M})^H,
// realised by the slicer's reversal, transposition and conjugation.
// ---------------------------------------------------------------------------
namespace {

struct SpecRef {
  const float4* p;  // batch element b, mode m at p + (b * bs + m) * N^2
  long long bs;
  int dag;          // use (X~_{(M-p) mod M})^H
  int tr = 0;       // the stored matrices are the transposed spectra X~^T
};

struct Job {
  SpecRef a, b;
  float4* c;        // [nb][M] output spectrum
  double2 alpha;
  int use_alpha, accumulate;
};

const int kPairsS[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
int pair_idx(int a, int b) {
  for (int i = 0; i < 6; ++i)
    if (kPairsS[i][0] == a && kPairsS[i][1] == b) return i;
  return -1;
}
int ord_idx(int mu, int nu) { return mu * 3 + (nu < mu ? nu : nu - 1); }

constexpr int kMaxJobs = 18;

// X[s][0] += identity for every series s (stride in matrices)
__global__ void identity_order0_kernel(double2* X, long long stride_mats, int N, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count * N) return;
  const long long s = i / N;
  const int d = (int)(i % N);
  X[s * stride_mats * N * N + (long long)d * N + d].x += 1.0;
}

cudaError_t set_identity_order0(double2* X, long long stride_mats, int N, long long count, cudaStream_t st) {
  const long long n = count * N;
  if (n == 0) return cudaSuccess;
  ProfScope ps(NSPT_STAGE_TEK, st);
  identity_order0_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, stride_mats, N, count);
  return cudaGetLastError();
}

struct LangevinWs {
  int* err;
  float4 *specU, *specUT, *specAcc, *specPQ, *specIn, *spY, *spR, *spC;  // specUT: transposed link spectra
  double2 *serTmp, *serS, *serY, *serR[2];
  double* imtr;
  __nv_bfloat16 *slA[kMaxJobs], *slB[kMaxJobs];
  int *expA[kMaxJobs], *expB[kMaxJobs];
  // slices of the link spectra, kept for a whole force evaluation: left operand U_x (lkA[x]),
  // right operands U_x^+ (lkB[x]) and U_x (lkB[4 + x], from the transposed spectra)
  __nv_bfloat16 *lkA[4], *lkB[8];
  int *lkEA[4], *lkEB[8];
  size_t total;
};

// which link slices of a force evaluation are already made (host side, reset per call)
struct LinkCache {
  const LangevinWs* w;
  long long specE, bs;
  bool okA[4], okB[8];
};

LangevinWs carve_langevin(void* base, int N, int T, int nb, int M, int S) {
  LangevinWs w;
  WsCarver c(base, SIZE_MAX);
  const long long E = (long long)N * N, T1 = T + 1;
  const long long spec = (long long)nb * M * E, ser = (long long)nb * T1 * E;
  w.err = c.take<int>(64);
  w.specU = c.take<float4>(4 * spec);
  w.specUT = c.take<float4>(4 * spec);
  w.specAcc = c.take<float4>(18 * spec);
  w.specPQ = c.take<float4>(18 * spec);
  w.specIn = c.take<float4>(4 * spec);
  w.spY = c.take<float4>(4 * spec);
  w.spR = c.take<float4>(4 * spec);
  w.spC = c.take<float4>(4 * spec);
  w.serTmp = c.take<double2>((long long)nspt_tmp_series(T) * ser);
  w.serS = c.take<double2>(4 * ser);
  w.serY = c.take<double2>(4 * ser);
  w.serR[0] = c.take<double2>(4 * ser);
  w.serR[1] = c.take<double2>(4 * ser);
  w.imtr = c.take<double>(4 * nb * T1);
  // per-job slices sized for Q = nb * M modes, one contiguous pool per kind; the
  // exp_star product (one job of up to 4 nb M modes) uses the first four slots of each pool
  const size_t Q = (size_t)nb * M;
  const size_t sa = Q * S * 2 * N * kpad(N), sb = Q * S * 3 * N * kpad(N), se = Q * N;
  __nv_bfloat16* poolA = c.take<__nv_bfloat16>(kMaxJobs * sa);
  __nv_bfloat16* poolB = c.take<__nv_bfloat16>(kMaxJobs * sb);
  int* poolEA = c.take<int>(kMaxJobs * se);
  int* poolEB = c.take<int>(kMaxJobs * se);
  for (int j = 0; j < kMaxJobs; ++j) {
    w.slA[j] = base ? poolA + j * sa : nullptr;
    w.slB[j] = base ? poolB + j * sb : nullptr;
    w.expA[j] = base ? poolEA + j * se : nullptr;
    w.expB[j] = base ? poolEB + j * se : nullptr;
  }
  __nv_bfloat16* lkPoolA = c.take<__nv_bfloat16>(4 * sa);
  __nv_bfloat16* lkPoolB = c.take<__nv_bfloat16>(8 * sb);
  int* lkPoolEA = c.take<int>(4 * se);
  int* lkPoolEB = c.take<int>(8 * se);
  for (int x = 0; x < 8; ++x) {
    if (x < 4) {
      w.lkA[x] = base ? lkPoolA + x * sa : nullptr;
      w.lkEA[x] = base ? lkPoolEA + x * se : nullptr;
    }
    w.lkB[x] = base ? lkPoolB + x * sb : nullptr;
    w.lkEB[x] = base ? lkPoolEB + x * se : nullptr;
  }
  w.total = c.off;
  return w;
}

// Link operand of a job: the index of its cached slices (left: x for U_x; right: x for U_x^+, 4 + x
// for U_x from the transposed spectra), or -1
int link_slot(const LinkCache* lc, const SpecRef& r, bool right) {
  if (!lc || r.bs != lc->bs) return -1;
  for (int x = 0; x < 4; ++x) {
    if (!right && r.p == lc->w->specU + x * lc->specE && !r.dag && !r.tr) return x;
    if (right && r.p == lc->w->specU + x * lc->specE && r.dag && !r.tr) return x;
    if (right && r.p == lc->w->specUT + x * lc->specE && !r.dag && r.tr) return 4 + x;
  }
  return -1;
}

int run_jobs(const LangevinWs& w, const Job* jobs, int count, int N, int nb, int M, int S, cudaStream_t st,
             __nv_bfloat16* slA_big = nullptr, __nv_bfloat16* slB_big = nullptr, int* eA_big = nullptr,
             int* eB_big = nullptr, LinkCache* lc = nullptr, bool a_ready = false) {
  std::vector<SplitGemmArgs> args;
  std::vector<std::pair<int, int>> sig;
  std::vector<char> slice_a(count, 1), slice_b(count, 1);
  for (int j = 0; j < count; ++j) {
    const Job& J = jobs[j];
    __nv_bfloat16* sa = slA_big ? slA_big : w.slA[j];
    __nv_bfloat16* sb = slB_big ? slB_big : w.slB[j];
    int* ea = eA_big ? eA_big : w.expA[j];
    int* eb = eB_big ? eB_big : w.expB[j];
    // a link operand is sliced once per force evaluation (by the first job that takes it) and
    // its slices reused
    const int xa = link_slot(lc, J.a, false), xb = link_slot(lc, J.b, true);
    if (xa >= 0) { sa = w.lkA[xa]; ea = w.lkEA[xa]; slice_a[j] = !lc->okA[xa]; lc->okA[xa] = true; }
    if (xb >= 0) { sb = w.lkB[xb]; eb = w.lkEB[xb]; slice_b[j] = !lc->okB[xb]; lc->okB[xb] = true; }
    if (a_ready) slice_a[j] = 0;  // the caller's left operand is already sliced into sa / ea
    SplitGemmArgs a;
    a.slicesA = sa; a.slicesB = sb; a.expA = ea; a.expB = eb; a.C = J.c;
    a.N = N; a.Kp = kpad(N); a.Q = nb * M; a.S = S; a.num_sms = g_num_sms; a.err = w.err; a.bn = 0;
    a.alpha = J.alpha; a.use_alpha = J.use_alpha; a.accumulate = J.accumulate;
    args.push_back(a);
    sig.push_back({N, nb * M});
  }
  // the jobs' slicings write disjoint slots: independent chains on the side streams, joined
  // before the one GEMM launch
  TRYS(fork_join(count, st, [&](int j, cudaStream_t s) -> int {
    const Job& J = jobs[j];
    const SplitGemmArgs& a = args[j];
    // left operand: rows of A (dagger: conjugated columns of the reversed spectrum)
    if (slice_a[j])
      TRYS(nspt_split_slice_df(S, J.a.p, J.a.bs, M, J.a.dag, J.a.dag ^ J.a.tr, J.a.dag, N, nb * M, 2,
                               (void*)a.slicesA, (int*)a.expA, s));
    // right operand: rows of B^T (dagger: conjugated rows of the reversed spectrum)
    if (slice_b[j])
      TRYS(nspt_split_slice_df(S, J.b.p, J.b.bs, M, J.b.dag, (!J.b.dag) ^ J.b.tr, J.b.dag, N, nb * M, 3,
                               (void*)a.slicesB, (int*)a.expB, s));
    return NSPT_OK;
  }));
  return nspt_split_gemm_batch(args.data(), count, S, choose_bn(signature(S, sig), N), g_num_sms, st);
}

}  // namespace

size_t nspt_split_ws_langevin(int N, int T, int nb, int M, int S) {
  return carve_langevin(nullptr, N, T, nb, M, S).total;
}

int nspt_split_langevin(int N, int T, int nb, int M, int S, double2* U, const double2* eta, double2* F, int flux,
                        double eps, void* ws, cudaStream_t st, int mode, const double2* Yin, int log2r) {
  const int E = N * N;
  const long long T1 = T + 1;
  const long long specE = (long long)M * E;  // one spectrum
  const int L = (int)llround(sqrt((double)N));
  double2 z[4][4];
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      const double ang = 2.0 * M_PI * flux * (mu < nu ? 1.0 : -1.0) / L;
      z[mu][nu] = (mu == nu) ? make_double2(0, 0) : make_double2(cos(ang), sin(ang));
    }
  LangevinWs w = carve_langevin(ws, N, T, nb, M, S);
  TRYC(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  // 1. spectra of the four links, [nb][4][M], and their transposes (right
  //    operands that are not daggered are sliced by rows of those)
  if (mode != NSPT_LMODE_UPDATE) TRYC(nspt_fft_fwd_df(U, T1, w.specU, E, T, nb * 4, M, 0, log2r, st));
  TRYC(nspt_fft_fwd_df(U, T1, w.specUT, E, T, nb * 4, M, 0, log2r, st, N));
  auto link = [&](int mu, int dag) { return SpecRef{w.specU + mu * specE, 4LL * M, dag}; };
  auto linkT = [&](int mu) { return SpecRef{w.specUT + mu * specE, 4LL * M, 0, 1}; };
  auto slot = [&](float4* base, int s) { return base + (long long)s * nb * specE; };
  Job jobs[kMaxJobs];
  LinkCache lc{&w, specE, 4LL * M, {}, {}};
  if (mode != NSPT_LMODE_UPDATE) {
  // 2. P1(mu,nu) = U_nu U_mu^+ (mu < nu) and Q(mu,nu) = U_mu U_nu: one launch of 18 products
  for (int i = 0; i < 6; ++i) {
    const int mu = kPairsS[i][0], nu = kPairsS[i][1];
    jobs[i] = Job{link(nu, 0), link(mu, 1), slot(w.specAcc, i), make_double2(1, 0), 0, 0};
  }
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu)
      if (mu != nu)
        jobs[6 + ord_idx(mu, nu)] = Job{link(mu, 0), linkT(nu), slot(w.specAcc, 6 + ord_idx(mu, nu)),
                                        make_double2(1, 0), 0, 0};
  TRYS(run_jobs(w, jobs, 18, N, nb, M, S, st, nullptr, nullptr, nullptr, nullptr, &lc));
  // truncate (Step 5) and return to the frequency domain
  TRYC(nspt_fft_inv_df(w.specAcc, w.serTmp, T1, E, T, 18 * nb, M, 0, log2r, st));
  TRYC(nspt_fft_fwd_df(w.serTmp, T1, w.specPQ, E, T, 18 * nb, M, 0, log2r, st));
  auto pq = [&](int s, int dag) { return SpecRef{slot(w.specPQ, s), (long long)M, dag}; };
  // 3. inner_mu = sum_nu z P1(mu,nu) U_nu^+ + conj(z) Q(mu,nu)^+ U_nu, six accumulating terms
  for (int tt = 0; tt < 6; ++tt) {
    for (int mu = 0; mu < 4; ++mu) {
      const int k = tt / 2;
      const int nu = k < mu ? k : k + 1;  // k-th neighbour of mu
      Job& J = jobs[mu];
      if (tt % 2 == 0) {
        J.a = (mu < nu) ? pq(pair_idx(mu, nu), 0) : pq(pair_idx(nu, mu), 1);
        J.b = link(nu, 1);
        J.alpha = z[mu][nu];
      } else {
        J.a = pq(6 + ord_idx(mu, nu), 1);
        J.b = linkT(nu);
        J.alpha = make_double2(z[mu][nu].x, -z[mu][nu].y);
      }
      J.c = slot(w.specIn, mu);
      J.use_alpha = 1;
      J.accumulate = tt > 0;
    }
    TRYS(run_jobs(w, jobs, 4, N, nb, M, S, st, nullptr, nullptr, nullptr, nullptr, &lc));
  }
  TRYC(nspt_fft_inv_df(w.specIn, w.serTmp, T1, E, T, 4 * nb, M, 0, log2r, st));
  TRYC(nspt_fft_fwd_df(w.serTmp, T1, w.specIn, E, T, 4 * nb, M, 0, log2r, st, N));  // transposed
  // 4. S_mu = U_mu inner_mu
  for (int mu = 0; mu < 4; ++mu)
    jobs[mu] = Job{link(mu, 0), SpecRef{slot(w.specIn, mu), (long long)M, 0, 1}, slot(w.specAcc, mu),
                   make_double2(1, 0), 0, 0};
  TRYS(run_jobs(w, jobs, 4, N, nb, M, S, st, nullptr, nullptr, nullptr, nullptr, &lc));
  for (int mu = 0; mu < 4; ++mu)
    TRYC(nspt_fft_inv_df(slot(w.specAcc, mu), w.serS + mu * T1 * E, 4 * T1, E, T, nb, M, 0, log2r, st));
  // 5. drift and Y = i X
  TRYC(nspt_tek_drift(w.serS, w.imtr, eta, F, w.serY, N, T, (long long)nb * 4, eps, st));
  }
  if (mode == NSPT_LMODE_DRIFT) return NSPT_OK;
  const double2* Ysrc = (mode == NSPT_LMODE_UPDATE) ? Yin : w.serY;
  // 6. exp_star(Y) by Paterson-Stockmeyer in the truncated ring (Y^(0) = 0, so Y^k
  //    starts at order k and every product runs at its own truncation on
  //    order-shifted series): Y^2 .. Y^s, then Q_j = B_j + Y^s Q_{j+1} for
  //    j = r-1 .. 0 with B_j = sum_{i<s} Y^i / (js+i)!, Q_j needed to order T - s j
  const long long ns = (long long)nb * 4, ser4 = ns * T1 * E;
  // C^(0..t) = (a * b)^(0..t) for series a (read to order ta >= t) and b (read to order t).
  // Consecutive products with the same left operand and transform length transform and slice
  // it once, read to the largest truncation ta of the run: with ta + t < Mt the circular
  // product of length Mt still equals the linear one through order t.
  const double2* a_done = nullptr;
  int a_Mt = 0, a_t = -1;
  auto star_t = [&](const double2* a, int ta, const double2* b, double2* c, int t) -> int {
    const int Mt = nspt_pow2_at_least(2 * (t + 1));
    if (ta < t || 2 * (ta + 1) > Mt) ta = t;
    const bool reuse = a == a_done && Mt == a_Mt && t <= a_t && a_t + t < Mt;
    if (!reuse) {
      TRYC(nspt_fft_fwd_df(a, T1, w.spY, E, ta, nb * 4, Mt, 0, log2r, st));
      a_done = a; a_Mt = Mt; a_t = ta;
    }
    TRYC(nspt_fft_fwd_df(b, T1, w.spR, E, t, nb * 4, Mt, 0, log2r, st, N));  // transposed: sliced by rows
    Job J{SpecRef{w.spY, (long long)Mt, 0}, SpecRef{w.spR, (long long)Mt, 0, 1}, w.spC, make_double2(1, 0), 0, 0};
    TRYS(run_jobs(w, &J, 1, N, nb * 4, Mt, S, st, w.slA[0], w.slB[0], w.expA[0], w.expB[0], nullptr, reuse));
    TRYC(nspt_fft_inv_df(w.spC, c, T1, E, t, nb * 4, Mt, 0, log2r, st));
    return NSPT_OK;
  };
  const int sb = nspt_ps_block(T), r = T / sb;
  const double2* Yp[NSPT_PS_MAX_BLOCK + 1] = {nullptr, Ysrc};
  for (int k = 2; k <= sb; ++k) {
    double2* Pk = w.serTmp + (k - 2) * ser4;
    TRYC(cudaMemsetAsync(Pk, 0, (size_t)ser4 * sizeof(double2), st));  // orders below k stay 0
    TRYS(star_t(Ysrc + E, nspt_ps_power_ta(T, sb, k), Yp[k - 1] + (k - 1) * E, Pk + k * E, T - k));
    Yp[k] = Pk;
  }
  double2* prod = w.serTmp + (sb - 1) * ser4;  // the slot after the powers Y^2..Y^s
  double2* Qs[2] = {w.serR[0], w.serR[1]};
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
  TRYC(nspt_ps_combine(Qs[0], block(r), sb - 1, nullptr, sb, T - sb * r, T, N, ns, st));
  for (int j = r - 1; j >= 0; --j) {
    const int t = T - sb * (j + 1);
    TRYS(star_t(Yp[sb] + sb * E, nspt_ps_horner_ta(T, sb, j), Qs[cur], prod, t));  // (Y^s Q_{j+1}) from order s
    TRYC(nspt_ps_combine(Qs[cur ^ 1], block(j), sb - 1, prod, sb, T - sb * j, T, N, ns, st));
    cur ^= 1;
  }
  double2* const expY = Qs[cur];
  // 7. U <- exp_star(i X) U, order 0 untouched
  TRYC(nspt_fft_fwd_df(expY, T1, w.spR, E, T, nb * 4, M, 0, log2r, st));
  Job J{SpecRef{w.spR, (long long)M, 0}, SpecRef{w.specUT, (long long)M, 0, 1}, w.spC, make_double2(1, 0), 0, 0};
  TRYS(run_jobs(w, &J, 1, N, nb * 4, M, S, st, w.slA[0], w.slB[0], w.expA[0], w.expB[0]));
  TRYC(nspt_fft_inv_df(w.spC, U, T1, E, T, nb * 4, M, 0, log2r, st, 1.0, 0, N, 1));
  return NSPT_OK;
}
