// Pieces shared by the tensor-core mode-GEMM kernels (split_gemm.cu,
// split_gemm_ta.cu): tile constants, the per-problem parameter block of a
// (possibly grouped) launch, bounded mbarrier waits and the double-float
// recombination of the digit-group accumulators.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "split_gemm.cuh"
#include "tc_ptx.cuh"

namespace sg {

constexpr int BM = 128, KB = 32;
constexpr int NA_STAGES = 4;
constexpr uint32_t A_TILE = BM * KB * 2;  // 8 KB per part
constexpr int NGROUPS = 5;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// One problem of a (possibly grouped) launch; all of them travel in the kernel
// parameters, so a launch needs no device-side table and can be captured.
struct GemmProblem {  // aligned like its CUtensorMap members
  CUtensorMap mA, mB;    // slice planes of the left / right operand
  const int* expA;
  const int* expB;
  float4* C;
  long long ldcq;        // float4 entries from C_q to C_{q+1}
  int N, Q, tilesM, tilesN;
  long long tile_begin;  // first global tile index of this problem
  float4 alpha;          // C = alpha * A B (+ C): (re_hi, re_lo, im_hi, im_lo)
  int use_alpha, accumulate;
};

template <int MAXP>
struct GemmBatch {
  GemmProblem p[MAXP];
  int count;
  long long total_tiles;
  long long wait_ns;  // budget of the abortable device-side waits
};

// limit_ns: budget of this wait; the waits that may abandon the tile loop take the launch's
// budget (GemmBatch::wait_ns; < 0, a test hook: give up as soon as the barrier is not ready at the
// first try), the final drains of copies and MMAs already in flight always take WAIT_LIMIT_NS
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                         int code, long long limit_ns = (long long)WAIT_LIMIT_NS) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  if (limit_ns < 0) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
    return false;
  }
  const uint64_t t0 = tc::globaltimer();
  uint32_t n = 0;
  while (!tc::mbar_try_wait(bar, parity)) {
    if ((++n & 255) == 0) {
      if (*abort_flag) return false;
      if (tc::globaltimer() - t0 > (uint64_t)limit_ns) {
        *abort_flag = 1;
        atomicCAS(err, 0, code);
        return false;
      }
    }
  }
  return true;
}

// error-free sum of two floats (Knuth's TwoSum); the _rn intrinsics keep the
// compiler from contracting any step into an FMA with a neighbouring product
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float pow2f(int k) {
  k = max(-126, min(127, k));
  return __int_as_float((k + 127) << 23);
}

// double-float sum of the digit-group accumulators, largest first
__device__ __forceinline__ void df_sum(const float (&a)[NGROUPS], float& hi, float& lo) {
  float h, s2, s3, e1, e2, e3;
  two_sum(a[0], a[1], h, e1);
  two_sum(h, a[2], s2, e2);
  two_sum(s2, a[3], s3, e3);
  const float l = ((e1 + e2) + e3) + a[4];
  hi = __fadd_rn(s3, l);
  lo = __fsub_rn(l, __fsub_rn(hi, s3));
}


}  // namespace sg

// 4-D TMA map over digit slices: (k < N, row < N, plane < P, slice < nslices), row pitch Kp bf16,
// box (32, box_rows, P, box_slices): one copy brings every plane of box_slices consecutive slices;
// 64-byte swizzle (split_gemm.cu)
int nspt_make_slice_map(CUtensorMap* map, const void* base, int N, int Kp, int P, long long nslices, int box_rows,
                        int box_slices);

namespace sg {

// fills the parameter block of a launch over `count` problems with output tiles BM x bn
template <int MAXP>
int build_batch(GemmBatch<MAXP>* gb, const SplitGemmArgs* a, int count, int S, int bn) {
  long long tiles = 0;
  for (int i = 0; i < count; ++i) {
    GemmProblem& P = gb->p[i];
    // left operand: planes (re, im) per digit; right operand: (re, im, -re)
    // A: one slice (re, im) per copy; B: all S slices (re, im, -re) of a K block in one copy
    if (nspt_make_slice_map(&P.mA, a[i].slicesA, a[i].N, a[i].Kp, 2, (long long)a[i].Q * S, BM, 1)) return -5;
    if (nspt_make_slice_map(&P.mB, a[i].slicesB, a[i].N, a[i].Kp, 3, (long long)a[i].Q * S, bn, S)) return -5;
    P.expA = a[i].expA; P.expB = a[i].expB; P.C = a[i].C;
    P.ldcq = a[i].ldc_q ? a[i].ldc_q : (long long)a[i].N * a[i].N;
    P.N = a[i].N; P.Q = a[i].Q;
    P.tilesM = (a[i].N + BM - 1) / BM;
    P.tilesN = (a[i].N + bn - 1) / bn;
    P.tile_begin = tiles;
    P.use_alpha = a[i].use_alpha;
    P.accumulate = a[i].accumulate;
    const float rh = (float)a[i].alpha.x, ih = (float)a[i].alpha.y;
    P.alpha = make_float4(rh, (float)(a[i].alpha.x - (double)rh), ih, (float)(a[i].alpha.y - (double)ih));
    tiles += (long long)a[i].Q * P.tilesM * P.tilesN;
  }
  gb->count = count;
  gb->total_tiles = tiles;
  gb->wait_ns = nspt_split_wait_budget();
  return 0;
}

}  // namespace sg
