// Allocation-free FFT-CONV product for callers that cannot allocate device
// memory themselves: code running where cudaMalloc is unavailable or
// forbidden (inside a host callback or a custom allocator hook, in processes
// whose device memory is owned and pooled by another framework, or in plug-in
// hosts that hand over only input and output buffers).  The three spectra the
// FP64 FFT-CONV product needs live in one fixed file-scope device array; the
// caller still passes the inputs and the output.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "zgemm64.cuh"

namespace {

// Fixed scratch: 32 MiB on every GPU that loads this library, held until exit.
constexpr size_t kScratchBytes = (size_t)32 << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_dev[64] = {nullptr};  // device address of g_noalloc_scratch, per device

int next_pow2(int x) {
  int m = 1;
  while (m < x) m <<= 1;
  return m;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Host code must not pass g_noalloc_scratch itself to a kernel: on the host
// that name is only a stand-in.  The device address is looked up once per
// device, with that device current.
int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  if (dev < 0 || dev >= 64) return NSPT_ERR_DEVICE;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      nspt_set_last_cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
      return NSPT_ERR_CUDA;
    }
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return NSPT_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = (const char*)a;
  const char* y = (const char*)b;
  return x < y + nb && y < x + na;
}

}  // namespace

extern "C" NSPT_API int nspt_polymat_mul_fft_noalloc(const void* A, const void* B, void* C, int N, int T, int batch,
                                                     void* stream) {
  if (!A || !B || !C || N < 1 || T < 0 || batch < 1 || N > 4096 || T > 255) return NSPT_ERR_ARG;
  const int M = next_pow2(2 * (T + 1));
  const long long E = (long long)N * N;
  const size_t spec = round256((size_t)batch * M * E * sizeof(double2));
  if (3 * spec > kScratchBytes) return NSPT_ERR_WORKSPACE;  // larger than the fixed scratch
  const size_t bytes = (size_t)batch * (T + 1) * E * sizeof(double2);
  if (overlaps(C, bytes, A, bytes) || overlaps(C, bytes, B, bytes)) return NSPT_ERR_ALIAS;
  int rc = nspt_init();
  if (rc) return rc;
  {
    const void* ptrs[3] = {A, B, C};
    if ((rc = nspt_check_ptrs((cudaStream_t)stream, true, ptrs, 3))) return rc;
  }
  void* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  double2* At = (double2*)base;
  double2* Bt = (double2*)((char*)base + spec);
  double2* Ct = (double2*)((char*)base + 2 * spec);
  cudaStream_t st = (cudaStream_t)stream;
  // every spectrum entry is written before it is read, so nothing needs clearing
  cudaError_t e = nspt_fft_fwd64((const double2*)A, T + 1, At, (int)E, T, batch, M, 0, 0, st);
  if (e == cudaSuccess) e = nspt_fft_fwd64((const double2*)B, T + 1, Bt, (int)E, T, batch, M, 0, 0, st);
  if (e == cudaSuccess) {
    ZgemmParams P;
    memset(&P, 0, sizeof(P));
    P.A = At; P.B = Bt; P.C = Ct; P.sA = M; P.sB = M; P.sC = M;
    P.N = N; P.kind = ZG_MODE; P.nmat = M; P.T = T;
    P.alpha = make_double2(1.0, 0.0);
    e = nspt_zgemm64(P, batch, st);
  }
  if (e == cudaSuccess) e = nspt_fft_inv64(Ct, (double2*)C, T + 1, (int)E, N, T, batch, M, 0, 0, 1.0, 0, st);
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}
