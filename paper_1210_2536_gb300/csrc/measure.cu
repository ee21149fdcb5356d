// A measured ceiling for gather-bound products.  SpMV with random column
// indices (the uniform and power-law structures) is bound by the rate at
// which the GPU serves independent random loads of x from L2, not by HBM
// bandwidth.  This kernel streams an index array (int32, 16-byte loads) and
// gathers x at those indices, 8 per thread, with nothing else to do: its rate
// is the ceiling a product's gathers can reach on this GPU.  The paper has no
// counterpart (it measures on CPUs); this is measurement support only.
// Beside it, the FP64 arithmetic ceiling: GB300 runs FP64 fused multiply-adds
// at a small fraction of its FP32 rate, low enough to bind FP64 products
// whose bytes stream at close to HBM speed.
#include <algorithm>
#include <chrono>
#include <vector>

#include "smat_internal.h"

namespace smat {

double host_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

namespace {

// A device-side hold of about ns nanoseconds: lane 0 polls %globaltimer with
// short sleeps between polls; the poll count is bounded (2^22), so the kernel
// ends even if the timer were to stall.
__global__ void hold_kernel(unsigned long long ns) {
  if (threadIdx.x != 0) return;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int i = 0; i < (1 << 22); ++i) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 >= ns) break;
    __nanosleep(256);
  }
}

}  // namespace

cudaError_t launch_hold(cudaStream_t s, double us) {
  us = us < 0.0 ? 0.0 : (us > HOLD_MAX_US ? HOLD_MAX_US : us);
  hold_kernel<<<1, 32, 0, s>>>((unsigned long long)(us * 1e3));
  return cudaGetLastError();
}

namespace {

// Indices uniform in [0, n): a 64-bit multiplicative hash of (seed, i).
__global__ void gather_index_kernel(int32_t *__restrict__ idx, long long nidx, long long n, unsigned long long seed) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nidx; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i + seed * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[i] = (int32_t)(z % (unsigned long long)n);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) gather_rate_kernel(const int32_t *__restrict__ idx, const T *__restrict__ x,
                                                          T *__restrict__ out, long long nthreads) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  const int4 a = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * t);
  const int4 b = __ldcs(reinterpret_cast<const int4 *>(idx) + 2 * t + 1);
  out[t] = __ldg(x + a.x) + __ldg(x + a.y) + __ldg(x + a.z) + __ldg(x + a.w) + __ldg(x + b.x) + __ldg(x + b.y) +
           __ldg(x + b.z) + __ldg(x + b.w);
}

template <typename T>
cudaError_t run_gather(long long n, long long nidx, int reps, double *rate) {
  void *pi = nullptr, *px = nullptr, *po = nullptr;
  const long long nt = nidx / 8;
  cudaError_t e = dev_alloc(&pi, (size_t)nidx * 4);
  if (e == cudaSuccess) e = dev_alloc(&px, (size_t)n * sizeof(T));
  if (e == cudaSuccess) e = dev_alloc(&po, (size_t)nt * sizeof(T));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<float> ms;
  if (e == cudaSuccess) {
    gather_index_kernel<<<1216, 256>>>((int32_t *)pi, nidx, n, 12345ull);
    e = cudaMemset(px, 0, (size_t)n * sizeof(T));
  }
  const unsigned grid = (unsigned)((nt + 255) / 256);
  double enq_us = 10.0;
  for (int r = -3; r < reps && e == cudaSuccess; ++r) {  // three untimed passes first
    e = queue_ahead(0, &enq_us, 1, [&]() -> cudaError_t {
      cudaError_t q = cudaEventRecord(e0);
      gather_rate_kernel<T><<<grid, 256>>>((const int32_t *)pi, (const T *)px, (T *)po, nt);
      if (q == cudaSuccess) q = cudaGetLastError();
      if (q == cudaSuccess) q = cudaEventRecord(e1);
      return q;
    });
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && r >= 0) ms.push_back(t);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(pi); dev_free(px); dev_free(po);
  if (e != cudaSuccess) return e;
  std::sort(ms.begin(), ms.end());
  *rate = (double)(nt * 8) / (ms[ms.size() / 2] * 1e-3);
  return cudaSuccess;
}

// FP64 fused multiply-adds: eight independent chains per thread, operands
// loaded at run time so nothing folds, one store per thread at the end.
__global__ void __launch_bounds__(256) fp64_fma_kernel(const double *__restrict__ bc, double *__restrict__ out,
                                                       int iters) {
  const double b = bc[0], c = bc[1];
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 1e-3 * (double)(threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t run_fp64(int reps, double *rate) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)sms * 8u;
  const int iters = 4096;
  void *pbc = nullptr, *po = nullptr;
  e = dev_alloc(&pbc, 2 * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc(&po, (size_t)grid * 256 * sizeof(double));
  const double bc[2] = {0.999, 1e-3};
  if (e == cudaSuccess) e = cudaMemcpy(pbc, bc, sizeof(bc), cudaMemcpyHostToDevice);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<float> ms;
  double enq_us = 10.0;
  for (int r = -3; r < reps && e == cudaSuccess; ++r) {  // three untimed passes first
    e = queue_ahead(0, &enq_us, 1, [&]() -> cudaError_t {
      cudaError_t q = cudaEventRecord(e0);
      fp64_fma_kernel<<<grid, 256>>>((const double *)pbc, (double *)po, iters);
      if (q == cudaSuccess) q = cudaGetLastError();
      if (q == cudaSuccess) q = cudaEventRecord(e1);
      return q;
    });
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess && r >= 0) ms.push_back(t);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dev_free(pbc); dev_free(po);
  if (e != cudaSuccess) return e;
  std::sort(ms.begin(), ms.end());
  *rate = (double)grid * 256.0 * iters * 8.0 / (ms[ms.size() / 2] * 1e-3);
  return cudaSuccess;
}

}  // namespace
}  // namespace smat

extern "C" smat_status_t smat_measure_fp64_rate(int32_t reps, double *fma_per_s) {
  if (!fma_per_s || reps < 1) return SMAT_ERR_INVALID_ARG;
  const cudaError_t e = smat::run_fp64(reps, fma_per_s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SMAT_ERR_ALLOC;
  }
  return e == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}

extern "C" smat_status_t smat_measure_gather_rate(int64_t n, int64_t nidx, smat_dtype_t dtype, int32_t reps,
                                                  double *gathers_per_s) {
  if (!gathers_per_s || n < 1 || n > INT32_MAX || nidx < 8 || reps < 1) return SMAT_ERR_INVALID_ARG;
  if (dtype != SMAT_F64 && dtype != SMAT_F32 && dtype != SMAT_BF16) return SMAT_ERR_INVALID_ARG;
  nidx = nidx / 8 * 8;
  const cudaError_t e = dtype == SMAT_F64 ? smat::run_gather<double>(n, nidx, reps, gathers_per_s)
                                          : smat::run_gather<float>(n, nidx, reps, gathers_per_s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SMAT_ERR_ALLOC;
  }
  return e == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}
