// Split-precision complex mode GEMM with three real products per complex
// product (the 3M method; Higham, "Stability of a method for multiplying
// complex matrices with three real matrix multiplications", SIMAX 1992):
//     P1 = A_re B_re,   P2 = A_im B_im,   P3 = (A_re + A_im)(B_re + B_im),
//     C_re = P1 - P2,   C_im = P3 - P1 - P2.
// FFT-CONV Step 3 on the tensor cores, as split_gemm.cu, for the plain product
// C~_q = A~_q B~_q only (no alpha, no accumulation).
//
// Operands: BF16 digit slices with three planes per digit, (re, im, re + im);
// the sum plane of a row is sliced at the row exponent e + 1 (|re + im| <
// 2^(e+1)), so P3 comes out in units four times those of P1 and P2 (an exact
// power of two).  Digit groups g = i + j as in split_gemm.cu: groups 0..3 own
// their accumulators, groups >= 4 share one.  Per group the accumulator holds
// [P1 | P2 | P3] for a tile of 128 rows x 32 complex columns (96 FP32 columns;
// five groups use 480 of the 512 TMEM columns), each product one MMA of
// N = 32 per slice pair and K step.  The epilogue forms, per group, the
// exact FP32 sums' combinations P1 - P2 and 4 P3 - P1 - P2 in double-float,
// sums the groups in double-float and applies 2^(e_A + e_B - 14).
//
// The structure follows split_gemm.cu: one CTA per SM, persistent over tiles;
// warp 0 lanes 0 and 1 issue the TMA loads (A: one copy per slice with its
// three planes; B: one copy per K block with every slice and plane), warp 1
// lane 0 issues tcgen05.mma, warps 2..9 drain TMEM (warp w reads lane quarter
// w % 4 and half of the tile's 32 columns).  S <= 6 only: the six-stage A
// ring holds a K block's slices, and the first K block of a tile issues its
// pairs digit group by digit group as the previous tile's epilogue frees the
// accumulators.  Every wait is bounded; on time-out the kernel records an
// error, drains its own copies and MMAs and frees TMEM.
#include "common.cuh"
#include "prof.cuh"
#include "split_gemm.cuh"
#include "tc_ptx.cuh"
#include "dfloat.cuh"
#include "split_gemm_common.cuh"

#include <cstring>
#include <memory>

namespace {

using namespace sg;

constexpr int BN3 = 32;       // complex output columns per tile
constexpr int NA3 = 6;        // A ring stages (one slice, three planes, each)
constexpr int NACC3 = 3 * BN3;  // accumulator columns per digit group: P1 | P2 | P3

template <int S>
struct Smem3 {
  static constexpr uint32_t A_PLANE = BM * KB * 2;   // 8 KB
  static constexpr uint32_t B_PLANE = BN3 * KB * 2;  // 2 KB
  uint8_t a[NA3][3][A_PLANE];      // [stage][re, im, sum]
  uint8_t b[2][S][3][B_PLANE];     // [buffer][slice][re, im, sum]
  uint64_t full_a[NA3], empty_a[NA3];
  uint64_t full_b[2], empty_b[2];
  uint64_t acc_full, acc_empty[NGROUPS], drain;
  uint32_t tmem_base;
  volatile int abort_flag;
};

template <int S, int MAXP>
__global__ void __launch_bounds__(320, 1)
split_gemm3m_kernel(const __grid_constant__ GemmBatch<MAXP> gb, int* err) {
  static_assert(S >= 2 && S <= NA3, "3M split GEMM: 2 <= S <= 6");
  static_assert(NGROUPS * NACC3 <= (int)TMEM_COLS, "accumulators exceed TMEM");
  constexpr uint32_t A_PLANE = Smem3<S>::A_PLANE, B_PLANE = Smem3<S>::B_PLANE;
  constexpr int G = S < NGROUPS ? S : NGROUPS;  // digit groups with pairs
  extern __shared__ uint8_t smem_raw[];
  Smem3<S>& sm = *reinterpret_cast<Smem3<S>*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = gb.total_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NA3; ++s) { tc::mbar_init(&sm.full_a[s], 1); tc::mbar_init(&sm.empty_a[s], 1); }
    for (int s = 0; s < 2; ++s) { tc::mbar_init(&sm.full_b[s], 1); tc::mbar_init(&sm.empty_b[s], 1); }
    tc::mbar_init(&sm.acc_full, 1);
    for (int g = 0; g < NGROUPS; ++g) tc::mbar_init(&sm.acc_empty[g], 256);
    tc::mbar_init(&sm.drain, 1);
    sm.abort_flag = 0;
    tc::fence_mbar_init();
    tc::fence_proxy_async();
    for (int p = 0; p < gb.count; ++p) {
      tc::prefetch_tmap(&gb.p[p].mA);
      tc::prefetch_tmap(&gb.p[p].mB);
    }
  }
  if (warp == 1) {
    tc::tmem_alloc(&sm.tmem_base, TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sm.tmem_base;

  if (warp == 0 && lane < 2) {
    // ---------------- TMA producers: lane 0 streams A slices, lane 1 B K blocks ----------------
    const bool isA = (lane == 0);
    int ia = 0, ib = 0;
    uint32_t pa = 0, pb = 0;
    uint32_t last_a_parity[NA3] = {}, last_b_parity[2] = {0, 0};
    bool issued_a[NA3] = {}, issued_b[2] = {false, false};
    int pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const long long lt = t - P.tile_begin;
      const int q = (int)(lt / (P.tilesM * P.tilesN));
      const int r = (int)(lt % (P.tilesM * P.tilesN));
      const int m0 = (r / P.tilesN) * BM, n0 = (r % P.tilesN) * BN3;
      const int nK = (P.N + KB - 1) / KB;
      bool ok = true;
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!isA) {
          if (!wait_bar(&sm.empty_b[ib], pb ^ 1, &sm.abort_flag, err, 1, gb.wait_ns)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&sm.full_b[ib], S * 3 * B_PLANE);
          tc::tma_load_4d(sm.b[ib][0][0], &P.mB, &sm.full_b[ib], kb * KB, n0, 0, q * S);  // [S][3][32][32]
          issued_b[ib] = true;
          last_b_parity[ib] = pb;
          if (++ib == 2) { ib = 0; pb ^= 1; }
        } else {
          for (int i = 0; i < S; ++i) {
            if (!wait_bar(&sm.empty_a[ia], pa ^ 1, &sm.abort_flag, err, 2, gb.wait_ns)) { ok = false; break; }
            tc::mbar_arrive_expect_tx(&sm.full_a[ia], 3 * A_PLANE);
            tc::tma_load_4d(sm.a[ia][0], &P.mA, &sm.full_a[ia], kb * KB, m0, 0, q * S + i);  // [3][128][32]
            issued_a[ia] = true;
            last_a_parity[ia] = pa;
            if (++ia == NA3) { ia = 0; pa ^= 1; }
          }
        }
      }
      if (!ok) break;
    }
    // make sure no TMA write into this CTA's shared memory is still in flight
    volatile int no_abort = 0;
    for (int s = 0; s < NA3; ++s)
      if (issued_a[s]) wait_bar(&sm.full_a[s], last_a_parity[s], &no_abort, err, 7);
    for (int s = 0; s < 2; ++s)
      if (issued_b[s]) wait_bar(&sm.full_b[s], last_b_parity[s], &no_abort, err, 7);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------ MMA issuer ------------------------------
    constexpr uint32_t ID = tc::idesc_bf16(BM, BN3, false);
    int ia = 0, ib = 0;
    uint32_t pa = 0, pb = 0, pacc = 0;
    bool any = false;
    int local = 0, pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x, ++local) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const int Nk = gb.p[pi].N;
      const int nK = (Nk + KB - 1) / KB;
      bool ok = true;
      tc::fence_after_sync();
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!wait_bar(&sm.full_b[ib], pb, &sm.abort_flag, err, 4, gb.wait_ns)) { ok = false; break; }
        tc::fence_after_sync();
        // the last K block may hold no more than 16 valid columns: one K = 16 step then
        const bool two_k = (Nk - kb * KB) > 16;
        const uint64_t b_0 = tc::desc_sw64(tc::smem_u32(sm.b[ib][0][0]));
        // B slice j, plane p: (j * 3 + p) planes of B_PLANE bytes further (descriptor units of 16 B)
        auto bdesc = [&](int j, int p) -> uint64_t { return b_0 + (uint64_t)((j * 3 + p) * (B_PLANE >> 4)); };
        // A operand (slice i's plane p, K step ks) against B slices j0 .. j0 + nj - 1 of the same
        // plane into group accumulators, in a row (collector reuse); ow_j0: the MMA of j0
        // overwrites its accumulator (first pair of that group and product in the tile)
        auto run = [&](uint64_t a, int i, int p, int ks, int j0, int nj, bool ow_j0, bool overwrite_first_pairs) {
#pragma unroll
          for (int jj = 0; jj < nj; ++jj) {
            const int j = j0 + jj;
            const int g = min(i + j, NGROUPS - 1);
            const uint32_t d = tmem + (uint32_t)(g * NACC3 + p * BN3);
            const bool ow = ks == 0 && ((jj == 0 && ow_j0) || (overwrite_first_pairs && j < NGROUPS));
            const int coll = nj == 1 ? tc::COLL_DISCARD
                             : jj == 0 ? tc::COLL_FILL : (jj == nj - 1 ? tc::COLL_LASTUSE : tc::COLL_USE);
            tc::mma_f16_coll(coll, d, a + 2 * ks, bdesc(j, p) + 2 * ks, ID, ow ? 0u : 1u);
          }
        };
        if (kb == 0) {
          // first K block: all S slices of A, then the pairs group by group; group g waits
          // until the previous tile's epilogue has read its accumulator
          uint64_t da[S][3];
          int stage[S];
          for (int i = 0; i < S && ok; ++i) {
            if (!wait_bar(&sm.full_a[ia], pa, &sm.abort_flag, err, 5, gb.wait_ns)) { ok = false; break; }
            stage[i] = ia;
#pragma unroll
            for (int p = 0; p < 3; ++p) da[i][p] = tc::desc_sw64(tc::smem_u32(sm.a[ia][p]));
            if (++ia == NA3) { ia = 0; pa ^= 1; }
          }
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (local > 0 && !wait_bar(&sm.acc_empty[g], pacc ^ 1, &sm.abort_flag, err, 3, gb.wait_ns)) { ok = false; break; }
            tc::fence_after_sync();
            if (g < NGROUPS - 1) {
              // pairs (i, g - i): one MMA each per product and K step; (0, g) overwrites
#pragma unroll
              for (int i = 0; i <= g; ++i)
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  run(da[i][p], i, p, 0, g - i, 1, i == 0, false);
                  if (two_k) run(da[i][p], i, p, 1, g - i, 1, false, false);
                }
            } else {
              // merged group: every pair with i + j >= NGROUPS - 1, slice by slice; (0, 4) overwrites
#pragma unroll
              for (int i = 0; i < S; ++i) {
                const int j0 = NGROUPS - 1 - i > 0 ? NGROUPS - 1 - i : 0, nj = S - i - j0;
                if (nj <= 0) continue;
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                  run(da[i][p], i, p, 0, j0, nj, i == 0, false);
                  if (two_k) run(da[i][p], i, p, 1, j0, nj, false, false);
                }
              }
            }
          }
          if (!ok) break;
          any = true;
          // every slice of this K block has had its last pair
          for (int i = 0; i < S; ++i) tc::mma_commit(&sm.empty_a[stage[i]]);
        } else {
#pragma unroll
          for (int i = 0; i < S; ++i) {
            if (!wait_bar(&sm.full_a[ia], pa, &sm.abort_flag, err, 5, gb.wait_ns)) { ok = false; break; }
            tc::fence_after_sync();
            // slice i meets B slices j < S - i; each A operand (plane, K step) against all of them
            // in a row, so that the tensor core reads it from shared memory once
#pragma unroll
            for (int p = 0; p < 3; ++p) {
              const uint64_t a = tc::desc_sw64(tc::smem_u32(sm.a[ia][p]));
              run(a, i, p, 0, 0, S - i, false, false);
              if (two_k) run(a, i, p, 1, 0, S - i, false, false);
            }
            any = true;
            tc::mma_commit(&sm.empty_a[ia]);
            if (++ia == NA3) { ia = 0; pa ^= 1; }
          }
        }
        if (!ok) break;
        tc::mma_commit(&sm.empty_b[ib]);
        if (++ib == 2) { ib = 0; pb ^= 1; }
      }
      if (!ok) break;
      tc::mma_commit(&sm.acc_full);
      pacc ^= 1;
    }
    if (any) {
      // all issued MMAs retire before TMEM can be released
      tc::mma_commit(&sm.drain);
      volatile int no_abort = 0;
      wait_bar(&sm.drain, 0, &no_abort, err, 8);
    }
  } else if (warp >= 2) {
    // ------------------------------ epilogue ------------------------------
    // warp w drains TMEM lanes 32*(w % 4) .. +31 and columns [16 half, 16 half + 16) of the tile
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row = quarter * 32 + lane;
    constexpr int HC = BN3 / 2;
    uint32_t pacc = 0;
    int pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const int N = P.N;
      const long long lt = t - P.tile_begin;
      const int tm = P.tilesM, tn = P.tilesN;
      const int q = (int)(lt / (tm * tn));
      const int r = (int)(lt % (tm * tn));
      const int m0 = (r / tn) * BM, n0 = (r % tn) * BN3 + half * HC;
      const int* __restrict__ expB = P.expB + (long long)q * N;
      const int m = m0 + row;
      const bool mvalid = m < N;
      const int ea = mvalid ? __ldg(P.expA + (long long)q * N + m) : 0;
      const float fa = pow2f(ea - 7);
      const bool fa_ok = (unsigned)(ea - 7 + 126) <= 253u;
      auto out_scale = [&](int eb) -> float {
        if (fa_ok && (unsigned)(eb - 7 + 126) <= 253u) return fa * pow2f(eb - 7);
        const int k = ea + eb - 14, k1 = k / 2;
        return pow2f(k1) * pow2f(k - k1);
      };
      float4* crow = P.C + (long long)q * P.ldcq + (long long)(mvalid ? m : 0) * N;
      if (!wait_bar(&sm.acc_full, pacc, &sm.abort_flag, err, 6, gb.wait_ns)) break;
      pacc ^= 1;
      tc::fence_after_sync();
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + half * HC;
      // per group: re_g = P1 - P2 and im_g = 4 P3 - (P1 + P2) as exact double-float pairs of the
      // exact FP32 group sums; groups 0..3 summed with TwoSum on the high parts, the merged
      // group's into the low parts
      float sr[HC], er[HC], si[HC], ei[HC];
#pragma unroll
      for (int g = 0; g < NGROUPS; ++g) {
        float p1[HC], p2[HC], p3[HC];
        if (g < G) {
          tc::tmem_ld16(lane_base + (uint32_t)(g * NACC3), p1);
          tc::tmem_ld16(lane_base + (uint32_t)(g * NACC3 + BN3), p2);
          tc::tmem_ld16(lane_base + (uint32_t)(g * NACC3 + 2 * BN3), p3);
          tc::tmem_wait_ld();
          tc::fence_before_sync();
          tc::mbar_arrive(&sm.acc_empty[g]);  // the next tile may overwrite this group now
        } else {
#pragma unroll
          for (int c = 0; c < HC; ++c) { p1[c] = 0.f; p2[c] = 0.f; p3[c] = 0.f; }
        }
#pragma unroll
        for (int c = 0; c < HC; ++c) {
          float rh, rl, uh, ul, ih, il;
          two_sum(p1[c], -p2[c], rh, rl);                // P1 - P2
          two_sum(p1[c], p2[c], uh, ul);                 // P1 + P2
          two_sum(__fmul_rn(4.f, p3[c]), -uh, ih, il);   // 4 P3 - (P1 + P2), high parts
          il = __fsub_rn(il, ul);
          if (g == 0) {
            sr[c] = rh; er[c] = rl; si[c] = ih; ei[c] = il;
          } else if (g < NGROUPS - 1) {
            float e1, e2;
            two_sum(sr[c], rh, sr[c], e1);
            two_sum(si[c], ih, si[c], e2);
            er[c] = er[c] + (e1 + rl);
            ei[c] = ei[c] + (e2 + il);
          } else {
            er[c] = er[c] + (rh + rl);
            ei[c] = ei[c] + (ih + il);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < HC; ++c) {
        const int n = n0 + c;
        if (!mvalid || n >= N) continue;
        const float rh = __fadd_rn(sr[c], er[c]), rl = __fsub_rn(er[c], __fsub_rn(rh, sr[c]));
        const float ih = __fadd_rn(si[c], ei[c]), il = __fsub_rn(ei[c], __fsub_rn(ih, si[c]));
        const float f = out_scale(__ldg(expB + n));
        crow[n] = make_float4(rh * f, rl * f, ih * f, il * f);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <int S>
size_t smem_bytes3() { return sizeof(Smem3<S>) + 1024; }

template <int S, int MAXP>
int launch3(const SplitGemmArgs* a, int count, cudaStream_t st, int num_sms) {
  std::unique_ptr<GemmBatch<MAXP>> gb(new GemmBatch<MAXP>());
  memset(gb.get(), 0, sizeof(GemmBatch<MAXP>));
  long long tiles = 0;
  for (int i = 0; i < count; ++i) {
    if (a[i].use_alpha || a[i].accumulate) return NSPT_ERR_UNSUPPORTED;
    GemmProblem& P = gb->p[i];
    // both operands: planes (re, im, re + im) per digit; A: one slice per copy, B: all S slices
    // of a K block in one copy
    if (nspt_make_slice_map(&P.mA, a[i].slicesA, a[i].N, a[i].Kp, 3, (long long)a[i].Q * S, BM, 1))
      return NSPT_ERR_CUDA;
    if (nspt_make_slice_map(&P.mB, a[i].slicesB, a[i].N, a[i].Kp, 3, (long long)a[i].Q * S, BN3, S))
      return NSPT_ERR_CUDA;
    P.expA = a[i].expA; P.expB = a[i].expB; P.C = a[i].C;
    P.ldcq = a[i].ldc_q ? a[i].ldc_q : (long long)a[i].N * a[i].N;
    P.N = a[i].N; P.Q = a[i].Q;
    P.tilesM = (a[i].N + BM - 1) / BM;
    P.tilesN = (a[i].N + BN3 - 1) / BN3;
    P.tile_begin = tiles;
    tiles += (long long)a[i].Q * P.tilesM * P.tilesN;
  }
  gb->count = count;
  gb->total_tiles = tiles;
  gb->wait_ns = nspt_split_wait_budget();
  int grid = num_sms;
  if (tiles < grid) grid = (int)tiles;
  if (grid < 1) return NSPT_OK;
  ProfScope ps(NSPT_STAGE_GEMM_TC, st);
  split_gemm3m_kernel<S, MAXP><<<grid, 320, smem_bytes3<S>(), st>>>(*gb, a[0].err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

template <int S>
int set_attr3() {
  cudaError_t e = cudaFuncSetAttribute(split_gemm3m_kernel<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes3<S>());
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

}  // namespace

int nspt_split_gemm3m_init() {
  int rc = set_attr3<2>();
  if (!rc) rc = set_attr3<3>();
  if (!rc) rc = set_attr3<4>();
  if (!rc) rc = set_attr3<5>();
  if (!rc) rc = set_attr3<6>();
  return rc;
}

int nspt_split_gemm3m(const SplitGemmArgs& a, cudaStream_t st) {
  switch (a.S) {
#define NSPT_CASE(s) case s: return launch3<s, 1>(&a, 1, st, a.num_sms);
    NSPT_CASE(2) NSPT_CASE(3) NSPT_CASE(4) NSPT_CASE(5) NSPT_CASE(6)
#undef NSPT_CASE
    default: return NSPT_ERR_UNSUPPORTED;
  }
}
