// Launch counting, per-stage CUDA-event timing and NVTX ranges of the library's
// kernels.
//
// Every kernel launch of the library goes through a ProfScope, which counts
// it and, while profiling is on, records a CUDA event pair around it on the
// stream it is launched on.  nspt_profile_end() sums the event durations per
// stage.  Events are created in nspt_profile_begin(), outside any timed
// region; recording them inside a call is an ordinary stream operation.
#include <atomic>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "prof.cuh"

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
int g_cap = 0;
int g_n = 0;
std::vector<cudaEvent_t> g_ev;  // 2 per record
std::vector<int> g_stage;
const char* kNames[NSPT_STAGE_COUNT] = {"fft_fwd", "slice",   "gemm_mode", "fft_inv",  "gemm_conv",
                                        "tek_elementwise", "gemm_tc", "other", "md_force", "md_link"};
}  // namespace

ProfScope::ProfScope(int stage, cudaStream_t st, int nlaunch) : idx_(-1), st_(st) {
  g_launches.fetch_add(nlaunch, std::memory_order_relaxed);
  // a named range for timeline tools (no cost beyond a check when none is attached)
  nvtxRangePushA((stage >= 0 && stage < NSPT_STAGE_COUNT) ? kNames[stage] : "nspt");
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_n >= g_cap) return;
  idx_ = g_n++;
  g_stage[idx_] = stage;
  cudaEventRecord(g_ev[2 * idx_], st_);
}

ProfScope::~ProfScope() {
  if (idx_ >= 0) cudaEventRecord(g_ev[2 * idx_ + 1], st_);
  nvtxRangePop();
}

extern "C" {

NSPT_API long long nspt_launch_count(void) { return g_launches.load(); }

NSPT_API const char* nspt_stage_name(int stage) {
  return (stage >= 0 && stage < NSPT_STAGE_COUNT) ? kNames[stage] : "?";
}

NSPT_API int nspt_profile_begin(int max_records) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (max_records < 1) return NSPT_ERR_ARG;
  for (auto e : g_ev) cudaEventDestroy(e);
  g_ev.assign(2 * (size_t)max_records, nullptr);
  g_stage.assign(max_records, -1);
  for (auto& e : g_ev) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) { nspt_set_last_cuda_error(err); return NSPT_ERR_CUDA; }
  }
  g_cap = max_records;
  g_n = 0;
  g_on = true;
  return NSPT_OK;
}

NSPT_API int nspt_profile_end(int nstages, double* total_ms, long long* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  for (int s = 0; s < nstages; ++s) { total_ms[s] = 0.0; launches[s] = 0; }
  for (int i = 0; i < g_n; ++i) {
    cudaError_t err = cudaEventSynchronize(g_ev[2 * i + 1]);
    if (err != cudaSuccess) { nspt_set_last_cuda_error(err); return NSPT_ERR_CUDA; }
    float ms = 0.f;
    err = cudaEventElapsedTime(&ms, g_ev[2 * i], g_ev[2 * i + 1]);
    if (err != cudaSuccess) { nspt_set_last_cuda_error(err); return NSPT_ERR_CUDA; }
    const int s = g_stage[i];
    if (s >= 0 && s < nstages) { total_ms[s] += ms; launches[s] += 1; }
  }
  const int n = g_n;
  g_n = 0;
  return n;
}

}  // extern "C"
