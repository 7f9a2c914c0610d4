// Split-precision product path (placeholder until the tensor-core GEMM lands).
#include "common.cuh"
#include "split.cuh"

int nspt_split_init() { return NSPT_OK; }
size_t nspt_split_ws_mul(int, int, int, int, int) { return 0; }
size_t nspt_split_ws_bwd(int, int, int, int, int) { return 0; }
int nspt_split_mul(int, int, int, int, int, int, bool, const double2*, const double2*, double2*, void*, cudaStream_t) {
  return NSPT_ERR_UNSUPPORTED;
}
int nspt_split_bwd(int, int, int, int, int, int, const double2*, const double2*, const double2*, double2*, double2*,
                   void*, cudaStream_t) {
  return NSPT_ERR_UNSUPPORTED;
}
int nspt_split_langevin(int, int, int, int, int, double2*, const double2*, double2*, int, double, void*, cudaStream_t) {
  return NSPT_ERR_UNSUPPORTED;
}
