// Shared device/host helpers of the NSPT polynomial-matrix library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/nspt.h"

#define NSPT_CUDA_TRY(expr)                                        \
  do {                                                             \
    cudaError_t _e = (expr);                                       \
    if (_e != cudaSuccess) { nspt_set_last_cuda_error(_e); return NSPT_ERR_CUDA; } \
  } while (0)

void nspt_set_last_cuda_error(cudaError_t e);

// Per-order rescale fitted on the device: while an NsptDevLog2r scope is alive on this host
// thread, every order transform launched multiplies its log2r argument by *p, read when the
// kernel runs (the fit kernel writes *p earlier on the same stream), so the fitted mode needs
// no read-back and can be captured in a CUDA graph.  A null p means a fixed rescale.
const int* nspt_dev_log2r();
class NsptDevLog2r {
 public:
  explicit NsptDevLog2r(const int* p);
  ~NsptDevLog2r();
  NsptDevLog2r(const NsptDevLog2r&) = delete;
  NsptDevLog2r& operator=(const NsptDevLog2r&) = delete;

 private:
  const int* prev_;
};

// Pointer kinds of an entry point's buffers, checked on the host before any
// launch, so that a host pointer where device memory is expected (or the
// reverse) returns NSPT_ERR_ARG instead of faulting a kernel.  Skipped while
// `st` is being captured into a graph.  NULL entries are skipped.
inline int nspt_check_ptrs(cudaStream_t st, bool device, const void* const* ptrs, int n) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return NSPT_ERR_ARG;
  }
  if (cs != cudaStreamCaptureStatusNone) return NSPT_OK;
  for (int i = 0; i < n; ++i) {
    if (!ptrs[i]) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptrs[i]) != cudaSuccess) {
      cudaGetLastError();
      return NSPT_ERR_ARG;
    }
    const bool dev_ok = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    const bool host_ok = a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered ||
                         a.type == cudaMemoryTypeManaged;
    if (device ? !dev_ok : !host_ok) return NSPT_ERR_ARG;
  }
  return NSPT_OK;
}

// ---------------------------------------------------------------------------
// complex double helpers (interleaved re, im = double2)
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Workspace carving: 256-byte aligned bump allocator over a caller-owned buffer.
struct WsCarver {
  char* base;
  size_t off;
  size_t cap;
  __host__ WsCarver(void* b, size_t c) : base((char*)b), off(0), cap(c) {}
  template <typename T>
  __host__ T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += bytes;
    return p;
  }
  __host__ bool fits() const { return off <= cap; }
};

static inline int ilog2_exact(int M) {
  int s = 0;
  while ((1 << s) < M) ++s;
  return ((1 << s) == M) ? s : -1;
}
