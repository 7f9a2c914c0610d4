// FP64 complex GEMM families on the CUDA cores (the plain FP64 form).
//
// One kernel serves every contraction of the product path, each output
// matrix q of batch element b being a sum of terms op(A_i) op(B_j):
//   MODE    C~_p = op(A~_p') op(B~_p'')      FFT-CONV Step 3 (Sec. 2); p' = p or
//                                             (M - p) mod M (spectrum of a dagger)
//   CONV    C_k = sum_{l=0}^{k} A_l B_{k-l}   naive star product, Eq. 5
//   CORR_A  C_j = sum_{t=0}^{T-j} A_{j+t} op(B_t)   backward dL/dA (correlation)
//   CORR_B  C_j = sum_{t=0}^{T-j} op(A_t) B_{j+t}   backward dL/dB
// op is identity or the conjugate transpose.  Tiles of 64x64 outputs,
// 256 threads, 4x4 complex outputs per thread, K staged 8 at a time through
// shared memory.  On B300 the FP64 pipe (about 1.1 TFLOP/s) bounds this kernel.
#include "common.cuh"
#include "zgemm64.cuh"
#include "prof.cuh"

namespace {
constexpr int BM = 64, BN = 64, BK = 8;

__device__ __forceinline__ void term_indices(const ZgemmParams& P, int q, int t, int& ia, int& ib) {
  switch (P.kind) {
    case ZG_MODE:
      ia = P.revA ? (P.nmat - q) % P.nmat : q;
      ib = P.revB ? (P.nmat - q) % P.nmat : q;
      break;
    case ZG_CONV: ia = t; ib = q - t; break;
    case ZG_CORR_A: ia = q + t; ib = t; break;
    default: ia = t; ib = q + t; break;  // ZG_CORR_B
  }
}

__device__ __forceinline__ int term_count(const ZgemmParams& P, int q) {
  switch (P.kind) {
    case ZG_MODE: return 1;
    case ZG_CONV: return q + 1;
    default: return P.T - q + 1;
  }
}

template <int OPA, int OPB>
__global__ void __launch_bounds__(256)
zgemm64_kernel(const ZgemmParams P) {
  __shared__ double2 sA[BK][BM];
  __shared__ double2 sB[BK][BN];
  const int N = P.N;
  const int tilesN = (N + BN - 1) / BN;
  const int m0 = (blockIdx.x / tilesN) * BM;
  const int n0 = (blockIdx.x % tilesN) * BN;
  const int q = (P.kind == ZG_CONV) ? (P.nmat - 1 - (int)blockIdx.y) : (int)blockIdx.y;
  const int b = blockIdx.z;
  const long long mat = (long long)N * N;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);

  const int cnt = term_count(P, q);
  for (int t = 0; t < cnt; ++t) {
    int ia, ib;
    term_indices(P, q, t, ia, ib);
    const double2* Am = P.A + ((long long)b * P.sA + ia) * mat;
    const double2* Bm = P.B + ((long long)b * P.sB + ib) * mat;
    for (int k0 = 0; k0 < N; k0 += BK) {
      // stage op(A)[m0..m0+63][k0..k0+7] into sA[k][m]
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * 256;
        int mm, kk;
        if (OPA == 0) { kk = idx & 7; mm = idx >> 3; } else { mm = idx & 63; kk = idx >> 6; }
        const int gm = m0 + mm, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gm < N && gk < N) {
          if (OPA == 0) v = Am[(long long)gm * N + gk];
          else v = cconj(Am[(long long)gk * N + gm]);
        }
        sA[kk][mm] = v;
      }
      // stage op(B)[k0..k0+7][n0..n0+63] into sB[k][n]
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int idx = tid + r * 256;
        int nn, kk;
        if (OPB == 0) { nn = idx & 63; kk = idx >> 6; } else { kk = idx & 7; nn = idx >> 3; }
        const int gn = n0 + nn, gk = k0 + kk;
        double2 v = make_double2(0.0, 0.0);
        if (gn < N && gk < N) {
          if (OPB == 0) v = Bm[(long long)gk * N + gn];
          else v = cconj(Bm[(long long)gn * N + gk]);
        }
        sB[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double2 a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = sB[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
            acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
            acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
            acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
          }
      }
      __syncthreads();
    }
  }
  double2* Cm = P.C + ((long long)b * P.sC + q) * mat;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= N) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double2 v = cmul(P.alpha, acc[i][j]);
      double2* dst = Cm + (long long)gm * N + gn;
      if (P.accumulate) v = cadd(*dst, v);
      *dst = v;
    }
  }
}
}  // namespace

cudaError_t nspt_zgemm64(const ZgemmParams& P, int batch, cudaStream_t st) {
  if (P.N <= 0 || P.nmat <= 0 || batch <= 0) return cudaSuccess;
  const int tiles = ((P.N + BM - 1) / BM) * ((P.N + BN - 1) / BN);
  dim3 grid(tiles, P.nmat, batch);
  ProfScope ps(P.kind == ZG_MODE ? NSPT_STAGE_GEMM_MODE : NSPT_STAGE_GEMM_CONV, st);
  if (P.opA == 0 && P.opB == 0) zgemm64_kernel<0, 0><<<grid, 256, 0, st>>>(P);
  else if (P.opA == 0) zgemm64_kernel<0, 1><<<grid, 256, 0, st>>>(P);
  else if (P.opB == 0) zgemm64_kernel<1, 0><<<grid, 256, 0, st>>>(P);
  else zgemm64_kernel<1, 1><<<grid, 256, 0, st>>>(P);
  return cudaGetLastError();
}
