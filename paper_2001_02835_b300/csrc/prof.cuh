#pragma once
#include <cuda_runtime.h>

enum { NSPT_STAGE_FFT_FWD = 0, NSPT_STAGE_SLICE = 1, NSPT_STAGE_GEMM_MODE = 2, NSPT_STAGE_FFT_INV = 3,
       NSPT_STAGE_GEMM_CONV = 4, NSPT_STAGE_TEK = 5, NSPT_STAGE_GEMM_TC = 6, NSPT_STAGE_OTHER = 7,
       // phases of a molecular-dynamics step (scopes around many launches, counting none)
       NSPT_STAGE_MD_FORCE = 8, NSPT_STAGE_MD_LINK = 9,
       NSPT_STAGE_COUNT = 10 };

// Counts `nlaunch` kernel launches and, while profiling, brackets them with events.
class ProfScope {
 public:
  ProfScope(int stage, cudaStream_t st, int nlaunch = 1);
  ~ProfScope();
 private:
  int idx_;
  cudaStream_t st_;
};
