// Seeded noise of the Langevin step (Eq. 3; eta = sum_a xi_a T^a over
// orthonormal generators, xi_a ~ N(0, 1): traceless Hermitian with
// E|eta_ij|^2 = 1 off the diagonal), drawn on the device from the
// counter-based generator Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011), written from its
// definition.  Every value has one address, independent of the launch shape:
//   key      = (seed mod 2^32, seed div 2^32)
//   counter  = (block b, matrix c, t mod 2^32, t div 2^32), t the call's counter
//   block b  -> Gaussians 2b, 2b + 1 of matrix c (row-major position g = i N + j)
//   uniforms u1 = ((w0 >> 5) 2^26 + (w1 >> 6) + 1) 2^-53 in (0, 1],
//            u2 = ((w2 >> 5) 2^26 + (w3 >> 6)) 2^-53 in [0, 1),
//   Box-Muller: z_2b = r cos(2 pi u2), z_2b+1 = r sin(2 pi u2), r = sqrt(-2 ln u1)
//   eta_ij = (z_{iN+j} + i z_{jN+i}) / sqrt(2) (i < j), eta_ji = conj(eta_ij),
//   eta_ii = z_{iN+i} - (1/N) sum_k z_{kN+k}.
#include <cuda_runtime.h>

#include "../../include/nspt.h"
#include "common.cuh"
#include "prof.cuh"

namespace {

constexpr unsigned kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr unsigned kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

// ten rounds; the key is bumped by the Weyl constants after each round
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const unsigned hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += kPhiloxW0;
    k.y += kPhiloxW1;
  }
  return c;
}

// the Gaussians of every (matrix, block), into the real parts of eta (the imaginary parts are
// written by the assembly kernel)
__global__ void __launch_bounds__(256) noise_gauss_kernel(double2* __restrict__ eta, int N, long long nb,
                                                          long long total, unsigned long long seed,
                                                          unsigned long long counter,
                                                          const unsigned long long* __restrict__ dctr) {
  const unsigned long long t = counter + (dctr ? *dctr : 0ull);
  const long long E = (long long)N * N;
  const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long c = i / nb, b = i % nb;
    const uint4 w = philox4x32_10(make_uint4((unsigned)b, (unsigned)c, (unsigned)t, (unsigned)(t >> 32)), key);
    const unsigned long long k1 = ((unsigned long long)(w.x >> 5) << 26) + (w.y >> 6);
    const unsigned long long k2 = ((unsigned long long)(w.z >> 5) << 26) + (w.w >> 6);
    const double u1 = ((double)k1 + 1.0) * 0x1p-53, u2 = (double)k2 * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    double2* X = eta + c * E;
    const long long g = 2 * b;
    X[g].x = r * co;
    if (g + 1 < E) X[g + 1].x = r * s;
  }
}

// one CTA per matrix: the diagonal's mean (fixed-order reduction), then the Hermitian assembly;
// each pair (i, j), (j, i) is read and written by one thread only.  CTA 0 then advances the
// device counter (the Gaussians of this call were all drawn by the previous launch).
__global__ void __launch_bounds__(256) noise_assemble_kernel(double2* __restrict__ eta, int N,
                                                             unsigned long long* __restrict__ dctr) {
  double2* X = eta + (long long)blockIdx.x * N * N;
  __shared__ double part[8];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += X[(long long)i * N + i].x;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < 8; ++w) tot += part[w];
  const double mean = tot / N;
  const double h = 1.0 / sqrt(2.0);
  const long long E = (long long)N * N;
  for (long long e = threadIdx.x; e < E; e += blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    if (i < j) {
      const double zr = X[e].x, zi = X[(long long)j * N + i].x;
      X[e] = make_double2(zr * h, zi * h);
      X[(long long)j * N + i] = make_double2(zr * h, -(zi * h));
    } else if (i == j) {
      X[e] = make_double2(X[e].x - mean, 0.0);
    }
  }
  if (dctr && blockIdx.x == 0 && threadIdx.x == 0) *dctr += 1ull;
}

}  // namespace

int nspt_tek_noise(void* eta, int N, int count, unsigned long long seed, unsigned long long counter,
                   unsigned long long* d_counter, void* stream) {
  if (!eta || N < 1 || N > 4096 || count < 1) return NSPT_ERR_ARG;
  int rc = nspt_init();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  {
    const void* ptrs[2] = {eta, d_counter};
    if ((rc = nspt_check_ptrs(st, true, ptrs, 2))) return rc;
  }
  const long long nb = ((long long)N * N + 1) / 2, total = nb * count;
  // grid-stride over the blocks: eight CTAs of 256 threads per SM at most
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  const long long want = (total + 255) / 256, cap = 8LL * sms;
  const int grid = (int)(want < cap ? want : cap);
  {
    ProfScope ps(NSPT_STAGE_TEK, st);
    noise_gauss_kernel<<<grid, 256, 0, st>>>((double2*)eta, N, nb, total, seed, counter, d_counter);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  {
    ProfScope ps(NSPT_STAGE_TEK, st);
    noise_assemble_kernel<<<count, 256, 0, st>>>((double2*)eta, N, d_counter);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { nspt_set_last_cuda_error(e); return NSPT_ERR_CUDA; }
  return NSPT_OK;
}
