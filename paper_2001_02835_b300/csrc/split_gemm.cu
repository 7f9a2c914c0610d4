// Split-precision complex mode GEMM on the 5th-generation tensor cores
// (FFT-CONV Step 3, C~_q = A~_q B~_q for every mode q of every batch element).
//
// Operands arrive as BF16 slice planes written by the slicing kernel: row r
// of operand X (X = A, or B^T for the right operand, both K-major) is
//   X[r][k] = 2^(e_r - 7) * sum_{i<S} s_i[r][k],   s_i = d_i * 2^(-8 i),
// with balanced digits |d_i| <= 128 and one exponent e_r per row.  A product
// s_i t_j is an integer multiple of 2^(-8(i+j)) below 2^(14-8(i+j)), so the
// dot product of one digit group g = i + j stays on that grid and is exact in
// FP32 while it has fewer than 24 significant bits.  Groups g = 0..3 keep
// their own TMEM accumulators; groups g >= 4 share a fifth one, whose
// rounding (the tensor core truncates at each accumulation step) stays near
// 2^-56 of the result per step.  The complex product is embedded in two real
// MMAs of N = 96 per slice pair: the right operand's tile holds the rows
// [B_re; B_im; -B_re] (48 each), and
//     D_g[:, 0:96] += A_re [B_re; B_im]^T      -> (A_re B_re | A_re B_im)
//     D_g[:, 0:96] += (-A_im) [B_im; -B_re]^T  -> (-A_im B_im | A_im B_re)
// (A-negate bit of the instruction descriptor), so one accumulator of 96 FP32
// columns per group holds (re | im); 5 groups use 480 of the 512 TMEM columns
// for a 128 x 48 output tile.  The epilogue sums
// the groups in double-float (hi + lo float pair), applies
// 2^(e_A[m] + e_B[n] - 14) and writes float4 (re_hi, re_lo, im_hi, im_lo).
//
// Roles (one CTA per SM, persistent over tiles): warp 0 lanes 0 and 1 issue the
// TMA loads of A and B (4-D maps: one copy per A slice (re, im), one per B K
// block with all its slices and planes), warp 1 lane 0 issues tcgen05.mma,
// warps 2-9 drain TMEM (two per lane quarter: for a plain product one sums the
// real parts of the tile's columns and the other the imaginary parts, each
// group read in two wide loads; with alpha or accumulation each takes half of
// the columns, real and imaginary).  Per K block of 32, all S slices of the B
// tile (re, im, -re) are loaded once and the A slices stream through a ring
// (6 stages for S <= 6, else 4); the triangle of slice pairs i + j < S is
// issued against the resident B slices, each A operand (slice, plane, K step)
// against all its B slices in a row, so that the tensor core reads it from
// shared memory once (collector fill / use / last use); the issuing loop is
// unrolled over the slices, since every instruction between two MMAs of the
// single issuing thread lengthens the MMA interval.
// With S <= 6 the epilogue frees the digit groups one at a time and the first
// K block of the next tile issues its pairs group by group, so the TMEM drain
// overlaps the MMAs (all 480 accumulator columns are in use, so the
// accumulators cannot be double-buffered).  Every wait is bounded
// (globaltimer; the budget of the abortable waits is a launch parameter); on
// time-out the kernel records an error, drains its own TMA and MMA work and
// frees TMEM.
#include "common.cuh"
#include "prof.cuh"
#include "split_gemm.cuh"
#include "tc_ptx.cuh"
#include "dfloat.cuh"
#include "split_gemm_common.cuh"

#include <atomic>
#include <cstring>
#include <memory>

namespace {

using namespace sg;

// the real (part 0) or imaginary (part 1) columns of one digit group's accumulator,
// in loads of 32 and 16 columns that start at multiples of their width
template <int BN>
__device__ __forceinline__ void ld_part(uint32_t group_base, int part, float* v) {
  static_assert(BN == 32 || BN == 48, "tile width");
  if (BN == 48) {
    if (part == 0) { tc::tmem_ld32(group_base, v); tc::tmem_ld16(group_base + 32, v + 32); }
    else { tc::tmem_ld16(group_base + 48, v); tc::tmem_ld32(group_base + 64, v + 16); }
  } else {
    tc::tmem_ld32(group_base + (uint32_t)(part * 32), v);
  }
}

// With S <= 6 slices the A ring holds every slice of a K block (6 stages, still
// within shared memory next to the B tiles), so that the first K block of a
// tile can issue its pairs digit group by digit group while the epilogue of
// the previous tile frees the groups' accumulators one at a time.
template <int S>
__host__ __device__ constexpr bool group_overlap() { return S <= 6; }
template <int S>
__host__ __device__ constexpr int a_stages() { return group_overlap<S>() ? 6 : NA_STAGES; }

template <int S, int BN>
struct Smem {
  static constexpr uint32_t B_TILE = BN * KB * 2;  // per part
  static constexpr int NA = a_stages<S>();
  uint8_t a[NA][2][A_TILE];         // [stage][re/im]
  uint8_t b[2][S][3][B_TILE];       // [buffer][slice][re, im, -re]
  uint64_t full_a[NA], empty_a[NA];
  uint64_t full_b[2], empty_b[2];
  uint64_t acc_full, acc_empty[NGROUPS], drain;  // acc_empty[g]: group g's accumulator read
  uint32_t tmem_base;
  volatile int abort_flag;
};

template <int S, int BN, int MAXP>
__global__ void __launch_bounds__(320, 1)
split_gemm_kernel(const __grid_constant__ GemmBatch<MAXP> gb, int* err) {
  constexpr int NACC = 2 * BN;  // accumulator columns per group: (re | im)
  static_assert(NGROUPS * NACC <= (int)TMEM_COLS, "accumulators exceed TMEM");
  static_assert(BN % 16 == 0 && (BN / 8) * 8 == BN, "tile width");
  constexpr uint32_t B_TILE = Smem<S, BN>::B_TILE;
  constexpr int NA = Smem<S, BN>::NA;
  constexpr bool OVL = group_overlap<S>();
  constexpr int G = S < NGROUPS ? S : NGROUPS;  // digit groups with pairs
  extern __shared__ uint8_t smem_raw[];
  Smem<S, BN>& sm = *reinterpret_cast<Smem<S, BN>*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = gb.total_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NA; ++s) { tc::mbar_init(&sm.full_a[s], 1); tc::mbar_init(&sm.empty_a[s], 1); }
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
    // ---------------- TMA producers: lane 0 streams A slices, lane 1 B slices ----------------
    // (two threads, so that the next K block's B tile is requested as soon as its buffer frees,
    // not behind the waits of the A ring)
    const bool isA = (lane == 0);
    int ia = 0, ib = 0;
    uint32_t pa = 0, pb = 0;
    uint32_t last_a_parity[NA] = {}, last_b_parity[2] = {0, 0};
    bool issued_a[NA] = {}, issued_b[2] = {false, false};
    int pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const long long lt = t - P.tile_begin;
      const int q = (int)(lt / (P.tilesM * P.tilesN));
      const int r = (int)(lt % (P.tilesM * P.tilesN));
      const int m0 = (r / P.tilesN) * BM, n0 = (r % P.tilesN) * BN;
      const int nK = (P.N + KB - 1) / KB;
      bool ok = true;
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!isA) {
          if (!wait_bar(&sm.empty_b[ib], pb ^ 1, &sm.abort_flag, err, 1, gb.wait_ns)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&sm.full_b[ib], S * 3 * B_TILE);
          tc::tma_load_4d(sm.b[ib][0][0], &P.mB, &sm.full_b[ib], kb * KB, n0, 0, q * S);  // [S][3][BN][32]
          issued_b[ib] = true;
          last_b_parity[ib] = pb;
          if (++ib == 2) { ib = 0; pb ^= 1; }
        } else {
          for (int i = 0; i < S; ++i) {
            if (!wait_bar(&sm.empty_a[ia], pa ^ 1, &sm.abort_flag, err, 2, gb.wait_ns)) { ok = false; break; }
            tc::mbar_arrive_expect_tx(&sm.full_a[ia], 2 * A_TILE);
            tc::tma_load_4d(sm.a[ia][0], &P.mA, &sm.full_a[ia], kb * KB, m0, 0, q * S + i);  // [2][BM][32]
            issued_a[ia] = true;
            last_a_parity[ia] = pa;
            if (++ia == NA) { ia = 0; pa ^= 1; }
          }
        }
      }
      if (!ok) break;
    }
    // make sure no TMA write into this CTA's shared memory is still in flight
    volatile int no_abort = 0;
    for (int s = 0; s < NA; ++s)
      if (issued_a[s]) wait_bar(&sm.full_a[s], last_a_parity[s], &no_abort, err, 7);
    for (int s = 0; s < 2; ++s)
      if (issued_b[s]) wait_bar(&sm.full_b[s], last_b_parity[s], &no_abort, err, 7);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------ MMA issuer ------------------------------
    constexpr uint32_t ID = tc::idesc_bf16(BM, NACC, false);
    constexpr uint32_t IDN = tc::idesc_bf16(BM, NACC, true);
    int ia = 0, ib = 0;
    uint32_t pa = 0, pb = 0, pacc = 0;
    bool any = false;
    int local = 0, pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x, ++local) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const int Nk = gb.p[pi].N;
      const int nK = (Nk + KB - 1) / KB;
      bool ok = true;
      if (!OVL && local > 0) {
        for (int g = 0; g < G && ok; ++g) ok = wait_bar(&sm.acc_empty[g], pacc ^ 1, &sm.abort_flag, err, 3, gb.wait_ns);
        if (!ok) break;
      }
      tc::fence_after_sync();
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!wait_bar(&sm.full_b[ib], pb, &sm.abort_flag, err, 4, gb.wait_ns)) { ok = false; break; }
        tc::fence_after_sync();
        // the last K block may hold no more than 16 valid columns: one K = 16 step then
        const bool two_k = (Nk - kb * KB) > 16;
        const uint64_t b_0 = tc::desc_sw64(tc::smem_u32(sm.b[ib][0][0]));
        // one slice pair (i, j) into accumulator d: A_re [B_re; B_im] and (-A_im) [B_im; -B_re];
        // ow: the first MMA overwrites the accumulator (first pair of its group in a tile)
        auto pair = [&](uint64_t a_re, uint64_t a_im, int j, uint32_t d, bool ow) {
          const uint64_t b_re = b_0 + (uint64_t)(j * 3 * (B_TILE >> 4));  // rows [re; im]
          const uint64_t b_im = b_re + (B_TILE >> 4);                      // rows [im; -re]
          tc::mma_f16(d, a_re, b_re, ID, ow ? 0u : 1u);
          tc::mma_f16(d, a_im, b_im, IDN, 1u);
          if (two_k) {  // second K = 16 step: 32 bytes further inside the 64-byte swizzle row
            tc::mma_f16(d, a_re + 2, b_re + 2, ID, 1u);
            tc::mma_f16(d, a_im + 2, b_im + 2, IDN, 1u);
          }
        };
        if (OVL && kb == 0) {
          // first K block: all S slices of A, then the pairs group by group; group g waits
          // until the previous tile's epilogue has read its accumulator
          uint64_t dre[OVL ? S : 1], dim[OVL ? S : 1];
          int stage[OVL ? S : 1];
          for (int i = 0; i < S && ok; ++i) {
            if (!wait_bar(&sm.full_a[ia], pa, &sm.abort_flag, err, 5, gb.wait_ns)) { ok = false; break; }
            stage[i] = ia;
            dre[i] = tc::desc_sw64(tc::smem_u32(sm.a[ia][0]));
            dim[i] = tc::desc_sw64(tc::smem_u32(sm.a[ia][1]));
            if (++ia == NA) { ia = 0; pa ^= 1; }
          }
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (local > 0 && !wait_bar(&sm.acc_empty[g], pacc ^ 1, &sm.abort_flag, err, 3, gb.wait_ns)) { ok = false; break; }
            tc::fence_after_sync();
            const uint32_t d = tmem + (uint32_t)(g * NACC);
            if (g < NGROUPS - 1) {
#pragma unroll
              for (int i = 0; i <= g; ++i) pair(dre[i], dim[i], g - i, d, i == 0);
            } else {
              // merged group: every pair with i + j >= NGROUPS - 1, slice by slice, each A
              // operand against its B slices in a row (collector reuse, as below)
#pragma unroll
              for (int i = 0; i < S; ++i) {
                const int j0 = NGROUPS - 1 - i > 0 ? NGROUPS - 1 - i : 0, nj = S - i - j0;
                auto run = [&](uint64_t a, bool im, int ks) {
#pragma unroll
                  for (int jj = 0; jj < nj; ++jj) {
                    const int j = j0 + jj;
                    const uint64_t b = b_0 + (uint64_t)(j * 3 * (B_TILE >> 4)) + (im ? (B_TILE >> 4) : 0) + 2 * ks;
                    const bool ow = i == 0 && j == NGROUPS - 1 && !im && ks == 0;
                    const int coll = nj == 1 ? tc::COLL_DISCARD
                                     : jj == 0 ? tc::COLL_FILL : (jj == nj - 1 ? tc::COLL_LASTUSE : tc::COLL_USE);
                    tc::mma_f16_coll(coll, d, a, b, im ? IDN : ID, ow ? 0u : 1u);
                  }
                };
                run(dre[i], false, 0);
                run(dim[i], true, 0);
                if (two_k) {
                  run(dre[i] + 2, false, 1);
                  run(dim[i] + 2, true, 1);
                }
              }
            }
          }
          if (!ok) break;
          any = true;
          // every slice of this K block has had its last pair
          for (int i = 0; i < S; ++i) tc::mma_commit(&sm.empty_a[stage[i]]);
        } else {
          // unrolled over the slices: every loop bound, accumulator offset and collector use
          // below is a compile-time constant, so the issuing thread spends no instructions
          // on them between MMAs
#pragma unroll
          for (int i = 0; i < S; ++i) {
            if (!wait_bar(&sm.full_a[ia], pa, &sm.abort_flag, err, 5, gb.wait_ns)) { ok = false; break; }
            tc::fence_after_sync();
            // descriptors: start addresses differ only in bits 0-13, so they are formed once and
            // advanced by adding (byte offset >> 4)
            const uint64_t a_re = tc::desc_sw64(tc::smem_u32(sm.a[ia][0]));
            const uint64_t a_im = tc::desc_sw64(tc::smem_u32(sm.a[ia][1]));
            // (without the group overlap) in the first K block of a tile, the first pair of each
            // group (i = 0, j = g for g < 4, and j = 4 for the merged group) overwrites it
            const bool first = (kb == 0) && (i == 0);
            // slice i meets B slices j < S - i: the four A operands (re, -im) x (K step 0, 1)
            // are each issued against all of them in a row, so that the tensor core reads
            // each A operand from shared memory once (collector fill, use ..., last use)
            const int nj = S - i;
            auto run = [&](uint64_t a, bool im, int ks) {
#pragma unroll
              for (int j = 0; j < nj; ++j) {
                const int g = min(i + j, NGROUPS - 1);
                const uint64_t b = b_0 + (uint64_t)(j * 3 * (B_TILE >> 4)) + (im ? (B_TILE >> 4) : 0) + 2 * ks;
                const bool ow = first && !im && ks == 0 && j < NGROUPS;
                const int coll = nj == 1 ? tc::COLL_DISCARD
                                 : j == 0 ? tc::COLL_FILL : (j == nj - 1 ? tc::COLL_LASTUSE : tc::COLL_USE);
                tc::mma_f16_coll(coll, tmem + (uint32_t)(g * NACC), a, b, im ? IDN : ID, ow ? 0u : 1u);
              }
            };
            run(a_re, false, 0);
            run(a_im, true, 0);
            if (two_k) {
              run(a_re + 2, false, 1);
              run(a_im + 2, true, 1);
            }
            any = true;
            tc::mma_commit(&sm.empty_a[ia]);
            if (++ia == NA) { ia = 0; pa ^= 1; }
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
    // warps 2..9: warp w drains TMEM lanes 32*(w % 4) .. +31 (the quarter its
    // rank within the warpgroup may access) and half of the tile's columns
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;  // 0: columns [0, BN/2), 1: [BN/2, BN)
    const int row = quarter * 32 + lane;
    uint32_t pacc = 0;
    constexpr int HALF = BN / 2;
    int pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const int N = P.N;
      const long long lt = t - P.tile_begin;
      const int tm = P.tilesM, tn = P.tilesN;
      const int q = (int)(lt / (tm * tn));
      const int r = (int)(lt % (tm * tn));
      const int m0 = (r / tn) * BM, n0 = (r % tn) * BN + half * HALF;
      const int* __restrict__ expB = P.expB + (long long)q * N;
      const bool plain = !P.use_alpha && !P.accumulate;
      const bool use_alpha = P.use_alpha, accumulate = P.accumulate;
      const float4 alpha = P.alpha;
      const int m = m0 + row;
      const bool mvalid = m < N;
      const int ea = mvalid ? __ldg(P.expA + (long long)q * N + m) : 0;
      // the scale 2^(e_A + e_B - 14) of an output: fa * 2^(e_B - 7) when both factors are normal
      // floats (then the product is exact), else as two halves of the exponent (tiny or huge rows)
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
      if (plain) {
        // warps of half 0 sum the real parts of all BN columns, half 1 the imaginary parts:
        // each group is read in two loads per warp
        const uint32_t qbase = tmem + ((uint32_t)(quarter * 32) << 16);
        const int nb = (r % tn) * BN;
        float s_[BN], e_[BN];
#pragma unroll
        for (int g = 0; g < NGROUPS; ++g) {
          float v[BN];
          if (g < G) {
            ld_part<BN>(qbase + (uint32_t)(g * NACC), half, v);
            tc::tmem_wait_ld();
            tc::fence_before_sync();
            tc::mbar_arrive(&sm.acc_empty[g]);
          } else {
#pragma unroll
            for (int c = 0; c < BN; ++c) v[c] = 0.f;
          }
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            if (g == 0) {
              s_[c] = v[c]; e_[c] = 0.f;
            } else if (g < NGROUPS - 1) {
              float e1;
              two_sum(s_[c], v[c], s_[c], e1);
              e_[c] = (g == 1) ? e1 : e_[c] + e1;
            } else {
              e_[c] = e_[c] + v[c];
            }
          }
        }
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          const int n = nb + c;
          if (!mvalid || n >= N) continue;
          const float h = __fadd_rn(s_[c], e_[c]), l = __fsub_rn(e_[c], __fsub_rn(h, s_[c]));  // FastTwoSum
          const float f = out_scale(__ldg(expB + n));
          reinterpret_cast<float2*>(crow + n)[half] = make_float2(h * f, l * f);
        }
        continue;
      }
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16) + half * HALF;
      // digit groups one at a time, each released as soon as it is read, summed in
      // double-float in the order of df_sum: TwoSum chain over groups 0-3 into (s, e),
      // then e += group 4 (the merged group); hi = s + e, lo = e - (hi - s)
      float sr[HALF], er[HALF], si[HALF], ei[HALF];
#pragma unroll
      for (int g = 0; g < NGROUPS; ++g) {
        float re[HALF], im[HALF];
        if (g < G) {
#pragma unroll
          for (int ch = 0; ch < HALF / 8; ++ch) {
            tc::tmem_ld8(lane_base + (uint32_t)(g * NACC) + ch * 8, re + ch * 8);
            tc::tmem_ld8(lane_base + (uint32_t)(g * NACC + BN) + ch * 8, im + ch * 8);
          }
          tc::tmem_wait_ld();
          tc::fence_before_sync();
          tc::mbar_arrive(&sm.acc_empty[g]);  // the next tile may overwrite this group now
        } else {
#pragma unroll
          for (int c = 0; c < HALF; ++c) { re[c] = 0.f; im[c] = 0.f; }
        }
#pragma unroll
        for (int c = 0; c < HALF; ++c) {
          if (g == 0) {
            sr[c] = re[c]; er[c] = 0.f; si[c] = im[c]; ei[c] = 0.f;
          } else if (g < NGROUPS - 1) {
            float e1, e2;
            two_sum(sr[c], re[c], sr[c], e1);
            two_sum(si[c], im[c], si[c], e2);
            if (g == 1) { er[c] = e1; ei[c] = e2; } else { er[c] = er[c] + e1; ei[c] = ei[c] + e2; }
          } else {
            er[c] = er[c] + re[c];
            ei[c] = ei[c] + im[c];
          }
        }
      }
#pragma unroll
      for (int c = 0; c < HALF; ++c) {
        const int n = n0 + c;
        if (!mvalid || n >= N) continue;
        const float rh = __fadd_rn(sr[c], er[c]), rl = __fsub_rn(er[c], __fsub_rn(rh, sr[c]));
        const float ih = __fadd_rn(si[c], ei[c]), il = __fsub_rn(ei[c], __fsub_rn(ih, si[c]));
        const float f = out_scale(__ldg(expB + n));
        if (plain) {
          crow[n] = make_float4(rh * f, rl * f, ih * f, il * f);
        } else {
          cdf v{dfl{rh * f, rl * f}, dfl{ih * f, il * f}};
          if (use_alpha) v = cdf_mul(v, dfl{alpha.x, alpha.y}, dfl{alpha.z, alpha.w});
          if (accumulate) {
            const float4 o = crow[n];
            v = cdf_add(v, cdf{dfl{o.x, o.y}, dfl{o.z, o.w}});
          }
          crow[n] = make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------- host: tensor maps ----------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

template <int S, int BN>
size_t smem_bytes() { return sizeof(Smem<S, BN>) + 1024; }

template <int S, int BN, int MAXP>
int launch(const SplitGemmArgs* a, int count, cudaStream_t st, int num_sms) {
  std::unique_ptr<GemmBatch<MAXP>> gb(new GemmBatch<MAXP>());
  memset(gb.get(), 0, sizeof(GemmBatch<MAXP>));
  if (build_batch<MAXP>(gb.get(), a, count, S, BN)) return NSPT_ERR_CUDA;
  const long long tiles = gb->total_tiles;
  int grid = num_sms;
  if (tiles < grid) grid = (int)tiles;
  if (grid < 1) return NSPT_OK;
  ProfScope ps(NSPT_STAGE_GEMM_TC, st);
  split_gemm_kernel<S, BN, MAXP><<<grid, 320, smem_bytes<S, BN>(), st>>>(*gb, a[0].err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

template <int S, int BN>
int launch_any(const SplitGemmArgs* a, int count, cudaStream_t st, int num_sms) {
  if (count == 1) return launch<S, BN, 1>(a, count, st, num_sms);
  if (count <= NSPT_SPLIT_MAX_PROBLEMS) return launch<S, BN, NSPT_SPLIT_MAX_PROBLEMS>(a, count, st, num_sms);
  return NSPT_ERR_ARG;
}

template <int S>
int launch_bn(const SplitGemmArgs* a, int count, int bn, cudaStream_t st, int num_sms) {
  if (bn == 32) return launch_any<S, 32>(a, count, st, num_sms);
  return launch_any<S, 48>(a, count, st, num_sms);
}

template <int S, int BN, int MAXP>
int set_attr() {
  cudaError_t e = cudaFuncSetAttribute(split_gemm_kernel<S, BN, MAXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<S, BN>());
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

template <int S>
int set_attrs() {
  int rc = set_attr<S, 32, 1>();
  if (!rc) rc = set_attr<S, 48, 1>();
  if (!rc) rc = set_attr<S, 32, NSPT_SPLIT_MAX_PROBLEMS>();
  if (!rc) rc = set_attr<S, 48, NSPT_SPLIT_MAX_PROBLEMS>();
  return rc;
}

}  // namespace

// 3-D map over slice planes: (k < N, row < N, plane), row pitch Kp bf16.  A box row is 64 bytes
// (32 K values); 128-byte L2 promotion (256-byte promotion made the GEMM 2.5% slower at SU(225))
int nspt_make_slice_map(CUtensorMap* map, const void* base, int N, int Kp, int P, long long nslices, int box_rows,
                        int box_slices) {
  cuuint64_t dims[4] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)P, (cuuint64_t)nslices};
  cuuint64_t strides[3] = {(cuuint64_t)Kp * 2, (cuuint64_t)N * Kp * 2, (cuuint64_t)P * N * Kp * 2};
  cuuint32_t box[4] = {(cuuint32_t)KB, (cuuint32_t)box_rows, (cuuint32_t)P, (cuuint32_t)box_slices};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? NSPT_OK : NSPT_ERR_CUDA;
}

namespace {
std::atomic<long long> g_wait_budget{(long long)WAIT_LIMIT_NS};
}  // namespace

long long nspt_split_wait_budget() { return g_wait_budget.load(); }
void nspt_split_set_wait_budget(long long ns) { g_wait_budget.store(ns); }

int nspt_split_gemm_init() {
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) {
      nspt_set_last_cuda_error(e == cudaSuccess ? cudaErrorNotSupported : e);
      return NSPT_ERR_CUDA;
    }
    g_encode = (EncodeTiledFn)fn;
  }
  int rc = set_attrs<2>();
  if (!rc) rc = set_attrs<3>();
  if (!rc) rc = set_attrs<4>();
  if (!rc) rc = set_attrs<5>();
  if (!rc) rc = set_attrs<6>();
  if (!rc) rc = set_attrs<7>();
  if (!rc) rc = set_attrs<8>();
  if (!rc) rc = nspt_split_gemm_ta_init();
  if (!rc) rc = nspt_split_gemm3m_init();
  if (rc) return rc;
  return NSPT_OK;
}

int nspt_split_gemm_batch(const SplitGemmArgs* a, int count, int S, int bn, int num_sms, cudaStream_t st) {
  if (count < 1) return NSPT_OK;
  for (int i = 0; i < count; ++i)
    if (a[i].N > 1024 || a[i].N < 1 || a[i].S != S) return NSPT_ERR_UNSUPPORTED;
  if (bn == 40) return nspt_split_gemm_ta_batch(a, count, S, num_sms, st);
  switch (S) {
    case 2: return launch_bn<2>(a, count, bn, st, num_sms);
    case 3: return launch_bn<3>(a, count, bn, st, num_sms);
    case 4: return launch_bn<4>(a, count, bn, st, num_sms);
    case 5: return launch_bn<5>(a, count, bn, st, num_sms);
    case 6: return launch_bn<6>(a, count, bn, st, num_sms);
    case 7: return launch_bn<7>(a, count, bn, st, num_sms);
    case 8: return launch_bn<8>(a, count, bn, st, num_sms);
    default: return NSPT_ERR_ARG;
  }
}

int nspt_split_gemm(const SplitGemmArgs& a, cudaStream_t st) {
  return nspt_split_gemm_batch(&a, 1, a.S, a.bn ? a.bn : 48, a.num_sms, st);
}
