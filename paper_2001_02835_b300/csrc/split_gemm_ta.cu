// Split-precision complex mode GEMM with the left operand in tensor memory.
//
// Same product and digit-group accounting as split_gemm.cu (see there), but
// the A slices do not feed the MMAs from shared memory: after TMA lands an A
// slice (re, im) in shared memory, the eight epilogue warps -- idle while the
// MMAs of a tile run -- read one row each (undoing the 64-byte swizzle) and
// write it into one of two TMEM A slots with tcgen05.st (lane = row, two K
// elements per 32-bit column).  The MMAs then take A from TMEM
// (tcgen05.mma ... [d], [a_tmem], b_desc) and read only the right operand
// [B_re; B_im; -B_re] from shared memory: 2.5 KB per 128 x 80 x 16 MMA instead
// of 7 KB per 128 x 96 x 16 in the shared-memory form.  Tile 128 x 40; TMEM:
// 5 digit groups x 80 accumulator columns = 400, plus 2 slots x 2 parts x 16
// columns for A = 464 of 512.
#include <cstring>
#include <memory>

#include "common.cuh"
#include "dfloat.cuh"
#include "prof.cuh"
#include "split_gemm.cuh"
#include "split_gemm_common.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace sg;

constexpr int BNT = 40;                                  // output tile width
constexpr int NACCT = 2 * BNT;                           // accumulator columns per group (re | im)
constexpr uint32_t ACC_COLS = NGROUPS * NACCT;           // 400
constexpr uint32_t ASLOT0 = ACC_COLS;                    // A slot s, part c at ASLOT0 + (2 s + c) * 16
constexpr int A_SLOTS = 2;
constexpr uint32_t B_TILE_T = BNT * KB * 2;              // 2560 bytes per part
static_assert(ASLOT0 + A_SLOTS * 2 * 16 <= TMEM_COLS, "TMEM budget");
constexpr int NLOADER = 8;                               // loader / epilogue warps

template <int S>
struct SmemT {
  uint8_t a[NA_STAGES][2][A_TILE];   // TMA landing zone of A slices (re, im)
  uint8_t b[2][S][3][B_TILE_T];      // [buffer][slice][re, im, -re]
  uint64_t full_a[NA_STAGES], empty_a[NA_STAGES];
  uint64_t full_b[2], empty_b[2];
  uint64_t ta_full[A_SLOTS], ta_empty[A_SLOTS];
  uint64_t acc_full, acc_empty, drain;
  uint32_t tmem_base;
  volatile int abort_flag;
};

template <int S, int MAXP>
__global__ void __launch_bounds__(320, 1)
split_gemm_ta_kernel(const __grid_constant__ GemmBatch<MAXP> gb, int* err) {
  extern __shared__ uint8_t smem_raw[];
  SmemT<S>& sm = *reinterpret_cast<SmemT<S>*>((((uintptr_t)smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ntiles = gb.total_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NA_STAGES; ++s) { tc::mbar_init(&sm.full_a[s], 1); tc::mbar_init(&sm.empty_a[s], NLOADER); }
    for (int s = 0; s < 2; ++s) { tc::mbar_init(&sm.full_b[s], 1); tc::mbar_init(&sm.empty_b[s], 1); }
    for (int s = 0; s < A_SLOTS; ++s) { tc::mbar_init(&sm.ta_full[s], NLOADER); tc::mbar_init(&sm.ta_empty[s], 1); }
    tc::mbar_init(&sm.acc_full, 1);
    tc::mbar_init(&sm.acc_empty, NLOADER);
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

  if (warp == 0 && lane == 0) {
    // ------------------------------ TMA producer ------------------------------
    int ia = 0, ib = 0;
    uint32_t pa = 0, pb = 0;
    uint32_t last_a_parity[NA_STAGES] = {}, last_b_parity[2] = {0, 0};
    bool issued_a[NA_STAGES] = {}, issued_b[2] = {false, false};
    int pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const long long lt = t - P.tile_begin;
      const int q = (int)(lt / (P.tilesM * P.tilesN));
      const int r = (int)(lt % (P.tilesM * P.tilesN));
      const int m0 = (r / P.tilesN) * BM, n0 = (r % P.tilesN) * BNT;
      const int nK = (P.N + KB - 1) / KB;
      bool ok = true;
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!wait_bar(&sm.empty_b[ib], pb ^ 1, &sm.abort_flag, err, 1, gb.wait_ns)) { ok = false; break; }
        tc::mbar_arrive_expect_tx(&sm.full_b[ib], S * 3 * B_TILE_T);
        tc::tma_load_4d(sm.b[ib][0][0], &P.mB, &sm.full_b[ib], kb * KB, n0, 0, q * S);  // [S][3][BN][32]
        issued_b[ib] = true;
        last_b_parity[ib] = pb;
        if (++ib == 2) { ib = 0; pb ^= 1; }
        for (int i = 0; i < S; ++i) {
          if (!wait_bar(&sm.empty_a[ia], pa ^ 1, &sm.abort_flag, err, 2, gb.wait_ns)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&sm.full_a[ia], 2 * A_TILE);
          tc::tma_load_4d(sm.a[ia][0], &P.mA, &sm.full_a[ia], kb * KB, m0, 0, q * S + i);  // [2][BM][32]
          issued_a[ia] = true;
          last_a_parity[ia] = pa;
          if (++ia == NA_STAGES) { ia = 0; pa ^= 1; }
        }
      }
      if (!ok) break;
    }
    volatile int no_abort = 0;
    for (int s = 0; s < NA_STAGES; ++s)
      if (issued_a[s]) wait_bar(&sm.full_a[s], last_a_parity[s], &no_abort, err, 7);
    for (int s = 0; s < 2; ++s)
      if (issued_b[s]) wait_bar(&sm.full_b[s], last_b_parity[s], &no_abort, err, 7);
  } else if (warp == 1 && lane == 0) {
    // ------------------------------ MMA issuer ------------------------------
    constexpr uint32_t ID = tc::idesc_bf16(BM, NACCT, false);
    constexpr uint32_t IDN = tc::idesc_bf16(BM, NACCT, true);
    int ib = 0, is = 0;
    uint32_t pb = 0, ps = 0, pacc = 0;
    bool any = false;
    int local = 0, pi = 0;
    for (long long t = blockIdx.x; t < ntiles && !sm.abort_flag; t += gridDim.x, ++local) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const int Nk = gb.p[pi].N;
      const int nK = (Nk + KB - 1) / KB;
      if (local > 0) {
        if (!wait_bar(&sm.acc_empty, pacc ^ 1, &sm.abort_flag, err, 3, gb.wait_ns)) break;
      }
      tc::fence_after_sync();
      bool ok = true;
      for (int kb = 0; kb < nK && ok; ++kb) {
        if (!wait_bar(&sm.full_b[ib], pb, &sm.abort_flag, err, 4, gb.wait_ns)) { ok = false; break; }
        tc::fence_after_sync();
        const bool two_k = (Nk - kb * KB) > 16;
        const uint64_t b_0 = tc::desc_sw64(tc::smem_u32(sm.b[ib][0][0]));
        for (int i = 0; i < S; ++i) {
          if (!wait_bar(&sm.ta_full[is], ps, &sm.abort_flag, err, 5, gb.wait_ns)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t a_re = tmem + ASLOT0 + (uint32_t)(2 * is) * 16;
          const uint32_t a_im = a_re + 16;
          const bool first = (kb == 0) && (i == 0);
#pragma unroll
          for (int j = 0; j < S; ++j) {
            if (j + i >= S) break;
            const int g = min(i + j, NGROUPS - 1);
            const uint32_t d = tmem + (uint32_t)(g * NACCT);
            const uint64_t b_re = b_0 + (uint64_t)(j * 3 * (B_TILE_T >> 4));  // rows [re; im]
            const uint64_t b_im = b_re + (B_TILE_T >> 4);                      // rows [im; -re]
            tc::mma_f16_ts(d, a_re, b_re, ID, (first && j < NGROUPS) ? 0u : 1u);
            tc::mma_f16_ts(d, a_im, b_im, IDN, 1u);
            if (two_k) {  // second K = 16 step: 8 TMEM columns / 32 bytes further
              tc::mma_f16_ts(d, a_re + 8, b_re + 2, ID, 1u);
              tc::mma_f16_ts(d, a_im + 8, b_im + 2, IDN, 1u);
            }
          }
          any = true;
          tc::mma_commit(&sm.ta_empty[is]);
          if (++is == A_SLOTS) { is = 0; ps ^= 1; }
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
      tc::mma_commit(&sm.drain);
      volatile int no_abort = 0;
      wait_bar(&sm.drain, 0, &no_abort, err, 8);
    }
  } else if (warp >= 2) {
    // ------------------ A loaders, then epilogue of each tile ------------------
    const int quarter = warp & 3;           // TMEM lanes / tile rows 32*quarter .. +31
    const int part = (warp - 2) >> 2;       // loader: 0 = A_re, 1 = A_im; epilogue: column half
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    int ia = 0, is = 0;
    uint32_t pa = 0, ps = 0, pacc = 0;
    constexpr int G = S < NGROUPS ? S : NGROUPS;
    int pi = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok && !sm.abort_flag; t += gridDim.x) {
      while (pi + 1 < gb.count && t >= gb.p[pi + 1].tile_begin) ++pi;
      const GemmProblem& P = gb.p[pi];
      const int N = P.N;
      const int nK = (N + KB - 1) / KB;
      // ---- A slices of this tile into TMEM ----
      for (int kb = 0; kb < nK && ok; ++kb) {
        for (int i = 0; i < S; ++i) {
          if (!wait_bar(&sm.full_a[ia], pa, &sm.abort_flag, err, 9, gb.wait_ns)) { ok = false; break; }
          // row `row` of the 64-byte-swizzled tile: 16-byte chunk c sits at chunk c ^ ((row >> 1) & 3)
          const uint8_t* src = sm.a[ia][part] + row * 64;
          uint32_t v[16];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 x = *reinterpret_cast<const uint4*>(src + 16 * (c ^ ((row >> 1) & 3)));
            v[4 * c] = x.x; v[4 * c + 1] = x.y; v[4 * c + 2] = x.z; v[4 * c + 3] = x.w;
          }
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&sm.empty_a[ia]);  // shared-memory stage read
          if (++ia == NA_STAGES) { ia = 0; pa ^= 1; }
          if (!wait_bar(&sm.ta_empty[is], ps ^ 1, &sm.abort_flag, err, 10, gb.wait_ns)) { ok = false; break; }
          tc::fence_after_sync();
          tc::tmem_st16(lane_base + ASLOT0 + (uint32_t)(2 * is + part) * 16, v);
          tc::tmem_wait_st();
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&sm.ta_full[is]);
          if (++is == A_SLOTS) { is = 0; ps ^= 1; }
        }
      }
      if (!ok) break;
      // ---- epilogue: columns [0, 24) by part 0, [24, 40) by part 1 ----
      const long long lt = t - P.tile_begin;
      const int tm = P.tilesM, tn = P.tilesN;
      const int q = (int)(lt / (tm * tn));
      const int r = (int)(lt % (tm * tn));
      const int m0 = (r / tn) * BM;
      const int c0 = part == 0 ? 0 : 24, nch = part == 0 ? 3 : 2;
      const int n0 = (r % tn) * BNT + c0;
      const int* __restrict__ expB = P.expB + (long long)q * N;
      const bool plain = !P.use_alpha && !P.accumulate;
      const bool use_alpha = P.use_alpha, accumulate = P.accumulate;
      const float4 alpha = P.alpha;
      const int m = m0 + row;
      const bool mvalid = m < N;
      const int ea = mvalid ? __ldg(P.expA + (long long)q * N + m) : 0;
      float4* crow = P.C + (long long)q * P.ldcq + (long long)(mvalid ? m : 0) * N;
      if (!wait_bar(&sm.acc_full, pacc, &sm.abort_flag, err, 6, gb.wait_ns)) break;
      pacc ^= 1;
      tc::fence_after_sync();
#pragma unroll 1
      for (int ch = 0; ch < nch; ++ch) {
        float re[NGROUPS][8], im[NGROUPS][8];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          tc::tmem_ld8(lane_base + (uint32_t)(g * NACCT) + c0 + ch * 8, re[g]);
          tc::tmem_ld8(lane_base + (uint32_t)(g * NACCT + BNT) + c0 + ch * 8, im[g]);
        }
        tc::tmem_wait_ld();
#pragma unroll
        for (int g = G; g < NGROUPS; ++g)
#pragma unroll
          for (int c = 0; c < 8; ++c) { re[g][c] = 0.f; im[g][c] = 0.f; }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int n = n0 + ch * 8 + c;
          if (!mvalid || n >= N) continue;
          float ar[NGROUPS], ai[NGROUPS];
#pragma unroll
          for (int g = 0; g < NGROUPS; ++g) { ar[g] = re[g][c]; ai[g] = im[g][c]; }
          float rh, rl, ih, il;
          df_sum(ar, rh, rl);
          df_sum(ai, ih, il);
          const int k = ea + __ldg(expB + n) - 14;
          const int k1 = k / 2, k2 = k - k1;
          const float f = pow2f(k1) * pow2f(k2);
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
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sm.acc_empty);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <int S>
size_t smem_bytes_t() { return sizeof(SmemT<S>) + 1024; }

template <int S, int MAXP>
int launch_t(const SplitGemmArgs* a, int count, cudaStream_t st, int num_sms) {
  std::unique_ptr<GemmBatch<MAXP>> gb(new GemmBatch<MAXP>());
  memset(gb.get(), 0, sizeof(GemmBatch<MAXP>));
  if (build_batch<MAXP>(gb.get(), a, count, S, BNT)) return NSPT_ERR_CUDA;
  const long long tiles = gb->total_tiles;
  int grid = num_sms;
  if (tiles < grid) grid = (int)tiles;
  if (grid < 1) return NSPT_OK;
  ProfScope ps(NSPT_STAGE_GEMM_TC, st);
  split_gemm_ta_kernel<S, MAXP><<<grid, 320, smem_bytes_t<S>(), st>>>(*gb, a[0].err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

template <int S>
int launch_any_t(const SplitGemmArgs* a, int count, cudaStream_t st, int num_sms) {
  if (count == 1) return launch_t<S, 1>(a, count, st, num_sms);
  if (count <= NSPT_SPLIT_MAX_PROBLEMS) return launch_t<S, NSPT_SPLIT_MAX_PROBLEMS>(a, count, st, num_sms);
  return NSPT_ERR_ARG;
}

template <int S, int MAXP>
int set_attr_t() {
  cudaError_t e = cudaFuncSetAttribute(split_gemm_ta_kernel<S, MAXP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes_t<S>());
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}

}  // namespace

int nspt_split_gemm_ta_init() {
  int rc = NSPT_OK;
#define NSPT_T(s) if (!rc) rc = set_attr_t<s, 1>(); if (!rc) rc = set_attr_t<s, NSPT_SPLIT_MAX_PROBLEMS>();
  NSPT_T(2) NSPT_T(3) NSPT_T(4) NSPT_T(5) NSPT_T(6) NSPT_T(7) NSPT_T(8)
#undef NSPT_T
  return rc;
}

int nspt_split_gemm_ta_batch(const SplitGemmArgs* a, int count, int S, int num_sms, cudaStream_t st) {
  switch (S) {
    case 2: return launch_any_t<2>(a, count, st, num_sms);
    case 3: return launch_any_t<3>(a, count, st, num_sms);
    case 4: return launch_any_t<4>(a, count, st, num_sms);
    case 5: return launch_any_t<5>(a, count, st, num_sms);
    case 6: return launch_any_t<6>(a, count, st, num_sms);
    case 7: return launch_any_t<7>(a, count, st, num_sms);
    case 8: return launch_any_t<8>(a, count, st, num_sms);
    default: return NSPT_ERR_ARG;
  }
}
