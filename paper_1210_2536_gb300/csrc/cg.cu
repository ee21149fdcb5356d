// Mixed-precision conjugate gradients around the adaptive SpMV.
//
// The paper reports SpMV in single and double precision (Sec. 7.2) and
// motivates the library by iterative solvers that call SpMV hundreds of times
// (Sec. 1, Sec. 7.3).  This solver keeps FP64 only where accuracy is decided:
// the outer loop forms r = b - A x with an FP64 handle and updates x in FP64
// (iterative refinement); the inner loop runs CG in FP32 on A d = r / ||r||
// through an FP32 (or BF16-valued) handle, whose products move half (or a
// third) of the bytes.
//
// Inner iterations keep every scalar on the device: each dot product is a
// deterministic two-stage reduction whose last block also forms alpha or beta,
// so an iteration is four launches with no host round trip, and chunks of
// iterations are replayed from a CUDA graph.  The host reads the residual only
// between chunks.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "smat_internal.h"

namespace smat {
namespace {

constexpr int CG_NT = 256;
constexpr int CG_BLOCKS = 152 * 4;

// Device-side scalars of one solve.
struct CgScalars {
  float rho, rho0, pq, alpha, beta;
  float pad;
  double dot64;
  unsigned int counter[4];
};

template <typename T>
__device__ __forceinline__ T block_sum(T v) {
  __shared__ T sh[CG_NT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  T r = 0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < CG_NT / 32 ? sh[threadIdx.x] : (T)0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// Last block to finish sums the per-block partials in block order (fixed,
// hence deterministic) and returns true in its thread 0 with *total set.
template <typename T>
__device__ __forceinline__ bool finish_reduce(T part, T *partials, unsigned int *counter, T *total) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  T s = 0;
  if (threadIdx.x < 32) {
    // lane l sums partials l, l+32, ... in order; then a fixed shuffle tree
    for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) s += ((volatile T *)partials)[b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  if (threadIdx.x == 0) {
    *total = s;
    *counter = 0;  // ready for the next launch
  }
  return threadIdx.x == 0;
}

// FP64 dot product a.b -> sc->dot64.
__global__ void __launch_bounds__(CG_NT) dot64_kernel(const double *__restrict__ a, const double *__restrict__ b,
                                                      long long n, double *partials, CgScalars *sc) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT)
    acc = fma(a[i], b[i], acc);
  double part = block_sum(acc);
  double tot;
  if (finish_reduce(part, partials, &sc->counter[0], &tot)) sc->dot64 = tot;
}

// r32 = (float)(r * inv_scale); d = 0; p = r32; rho = r32.r32, rho0 = rho.
__global__ void __launch_bounds__(CG_NT) inner_init_kernel(const double *__restrict__ r, double inv_scale, long long n,
                                                           float *__restrict__ res, float *__restrict__ p,
                                                           float *__restrict__ d, float *partials, CgScalars *sc) {
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT) {
    float v = (float)(r[i] * inv_scale);
    res[i] = v;
    p[i] = v;
    d[i] = 0.0f;
    acc = fmaf(v, v, acc);
  }
  float part = block_sum(acc);
  float tot;
  if (finish_reduce(part, partials, &sc->counter[1], &tot)) {
    sc->rho = tot;
    sc->rho0 = tot;
  }
}

// pq = p.q ; alpha = rho / pq (0 on breakdown).
__global__ void __launch_bounds__(CG_NT) pq_kernel(const float *__restrict__ p, const float *__restrict__ q,
                                                   long long n, float *partials, CgScalars *sc) {
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT)
    acc = fmaf(p[i], q[i], acc);
  float part = block_sum(acc);
  float tot;
  if (finish_reduce(part, partials, &sc->counter[2], &tot)) {
    sc->pq = tot;
    sc->alpha = (tot > 0.0f && sc->rho > 0.0f) ? sc->rho / tot : 0.0f;
  }
}

// d += alpha p ; res -= alpha q ; rho' = res.res ; beta = rho'/rho ; rho = rho'.
__global__ void __launch_bounds__(CG_NT) update_kernel(const float *__restrict__ p, const float *__restrict__ q,
                                                       float *__restrict__ d, float *__restrict__ res, long long n,
                                                       float *partials, CgScalars *sc) {
  const float alpha = sc->alpha;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT) {
    d[i] = fmaf(alpha, p[i], d[i]);
    float r = fmaf(-alpha, q[i], res[i]);
    res[i] = r;
    acc = fmaf(r, r, acc);
  }
  float part = block_sum(acc);
  float tot;
  if (finish_reduce(part, partials, &sc->counter[3], &tot)) {
    sc->beta = sc->rho > 0.0f ? tot / sc->rho : 0.0f;
    sc->rho = tot;
  }
}

// p = res + beta p.
__global__ void __launch_bounds__(CG_NT) direction_kernel(const float *__restrict__ res, float *__restrict__ p,
                                                          long long n, const CgScalars *sc) {
  const float beta = sc->beta;
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT)
    p[i] = fmaf(beta, p[i], res[i]);
}

// x += scale * (double) d.
__global__ void __launch_bounds__(CG_NT) refine_kernel(double *__restrict__ x, const float *__restrict__ d,
                                                       double scale, long long n) {
  for (long long i = (long long)blockIdx.x * CG_NT + threadIdx.x; i < n; i += (long long)gridDim.x * CG_NT)
    x[i] = fma(scale, (double)d[i], x[i]);
}

int blocks_for(long long n) {
  long long b = (n + CG_NT - 1) / CG_NT;
  return (int)(b < CG_BLOCKS ? (b < 1 ? 1 : b) : CG_BLOCKS);
}

struct Workspace {
  void *mem = nullptr;
  ~Workspace() { dev_free(mem); }
};

}  // namespace
}  // namespace smat

using namespace smat;

extern "C" void smat_cg_opts_default(smat_cg_opts_t *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-10;
  o->max_outer = 50;
  o->max_inner = 500;
  o->inner_rtol = 1e-4f;
  o->max_total_inner = 0;
  o->check_every = 10;
  o->use_graph = 1;
}

extern "C" smat_status_t smat_cg_mixed(smat_handle_t a64, smat_handle_t a32, const double *b, double *x,
                                       const smat_cg_opts_t *opts_in, smat_cg_info_t *info, void *stream) {
  if (!a64 || !a32 || !b || !x) return SMAT_ERR_INVALID_ARG;
  if (a64->dtype != SMAT_F64 || a32->dtype == SMAT_F64) return SMAT_ERR_INVALID_ARG;
  if (a64->m != a64->n || a32->m != a64->m || a32->n != a64->n) return SMAT_ERR_INVALID_ARG;
  smat_cg_opts_t o;
  if (opts_in) o = *opts_in; else smat_cg_opts_default(&o);
  if (o.check_every < 1) o.check_every = 1;
  const long long n = a64->n;
  smat_cg_info_t inf{};
  if (n == 0) {
    inf.converged = 1;
    if (info) *info = inf;
    return SMAT_OK;
  }
  cudaStream_t user = (cudaStream_t)stream;
  // workspace: r (f64), partials (f64, CG_BLOCKS), res/p/q/d (f32), scalars
  const size_t off_r = 0, off_part = off_r + (size_t)n * 8, off_res = off_part + (size_t)CG_BLOCKS * 8;
  const size_t off_p = off_res + (size_t)n * 4, off_q = off_p + (size_t)n * 4, off_d = off_q + (size_t)n * 4;
  const size_t off_sc = (off_d + (size_t)n * 4 + 255) / 256 * 256, total = off_sc + sizeof(CgScalars);
  Workspace ws;
  cudaError_t e = dev_alloc(&ws.mem, total);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SMAT_ERR_ALLOC : SMAT_ERR_CUDA;
  char *base = (char *)ws.mem;
  double *r = (double *)(base + off_r), *part64 = (double *)(base + off_part);
  float *part32 = (float *)(base + off_part);
  float *res = (float *)(base + off_res), *p = (float *)(base + off_p), *q = (float *)(base + off_q),
        *d = (float *)(base + off_d);
  CgScalars *sc = (CgScalars *)(base + off_sc);
  // a private stream (capturable), ordered after the caller's stream
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  smat_status_t status = SMAT_OK;
  const int gb = blocks_for(n);
  const double one = 1.0, mone = -1.0;
  const float onef = 1.0f, zerof = 0.0f;
  double nb = 0.0, nr = 0.0;
  auto chk = [&](cudaError_t ce) {
    if (ce != cudaSuccess && status == SMAT_OK) status = ce == cudaErrorMemoryAllocation ? SMAT_ERR_ALLOC : SMAT_ERR_CUDA;
    return ce == cudaSuccess;
  };
  auto spmv32 = [&]() -> bool {
    smat_status_t st = smat_spmv(a32, &onef, p, &zerof, q, s);
    if (st != SMAT_OK && status == SMAT_OK) status = st;
    return st == SMAT_OK;
  };
  auto inner_iteration = [&]() -> bool {
    if (!spmv32()) return false;
    pq_kernel<<<gb, CG_NT, 0, s>>>(p, q, n, part32, sc);
    update_kernel<<<gb, CG_NT, 0, s>>>(p, q, d, res, n, part32, sc);
    direction_kernel<<<gb, CG_NT, 0, s>>>(res, p, n, sc);
    return chk(cudaGetLastError());
  };
  auto residual_norm = [&](double *out) -> bool {
    // r = b - A64 x in FP64, then ||r||
    if (!chk(cudaMemcpyAsync(r, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s))) return false;
    smat_status_t st = smat_spmv(a64, &mone, x, &one, r, s);
    if (st != SMAT_OK) { if (status == SMAT_OK) status = st; return false; }
    dot64_kernel<<<gb, CG_NT, 0, s>>>(r, r, n, part64, sc);
    double v = 0.0;
    if (!chk(cudaMemcpyAsync(&v, &sc->dot64, 8, cudaMemcpyDeviceToHost, s))) return false;
    if (!chk(cudaStreamSynchronize(s))) return false;
    *out = std::sqrt(v);
    return true;
  };
  const auto t0 = std::chrono::steady_clock::now();
  do {
    if (!chk(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking))) break;
    if (!chk(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) break;
    if (!chk(cudaEventRecord(ev, user)) || !chk(cudaStreamWaitEvent(s, ev, 0))) break;
    if (!chk(cudaMemsetAsync(sc, 0, sizeof(CgScalars), s))) break;
    dot64_kernel<<<gb, CG_NT, 0, s>>>(b, b, n, part64, sc);
    double bb = 0.0;
    if (!chk(cudaMemcpyAsync(&bb, &sc->dot64, 8, cudaMemcpyDeviceToHost, s)) || !chk(cudaStreamSynchronize(s))) break;
    nb = std::sqrt(bb);
    if (nb == 0.0) {  // b = 0: x = 0 is the solution
      chk(cudaMemsetAsync(x, 0, (size_t)n * 8, s));
      nr = 0.0;
      inf.converged = 1;
      break;
    }
    if (!residual_norm(&nr)) break;
    const int chunk = o.check_every;
    while (nr / nb > o.rtol && inf.outer < o.max_outer &&
           (o.max_total_inner <= 0 || inf.inner_total < o.max_total_inner)) {
      inner_init_kernel<<<gb, CG_NT, 0, s>>>(r, 1.0 / nr, n, res, p, d, part32, sc);
      if (!chk(cudaGetLastError())) break;
      int it = 0;
      const float stop2 = o.inner_rtol * o.inner_rtol;
      bool ok = true;
      while (it < o.max_inner && (o.max_total_inner <= 0 || inf.inner_total + it < o.max_total_inner)) {
        int k = std::min(chunk, o.max_inner - it);
        if (o.max_total_inner > 0) k = std::min(k, o.max_total_inner - inf.inner_total - it);
        if (o.use_graph && k == chunk) {
          if (!gexec) {  // capture one chunk of iterations once, replay it afterwards
            if (!chk(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal))) { ok = false; break; }
            bool cap_ok = true;
            for (int j = 0; j < chunk && cap_ok; ++j) cap_ok = inner_iteration();
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (!cap_ok || !chk(ce)) { ok = false; break; }
            if (!chk(cudaGraphInstantiate(&gexec, graph, 0))) { ok = false; break; }
          }
          if (!chk(cudaGraphLaunch(gexec, s))) { ok = false; break; }
        } else {
          for (int j = 0; j < k && ok; ++j) ok = inner_iteration();
          if (!ok) break;
        }
        it += k;
        float rho = 0.0f, rho0 = 1.0f;
        float pair[2];
        if (!chk(cudaMemcpyAsync(pair, &sc->rho, sizeof(pair), cudaMemcpyDeviceToHost, s)) ||
            !chk(cudaStreamSynchronize(s))) { ok = false; break; }
        rho = pair[0];
        rho0 = pair[1];
        if (!(rho <= stop2 * rho0) && std::isfinite(rho) && rho > 0.0f) continue;
        break;
      }
      if (!ok) break;
      inf.inner_total += it;
      refine_kernel<<<gb, CG_NT, 0, s>>>(x, d, nr, n);
      if (!chk(cudaGetLastError())) break;
      ++inf.outer;
      if (!residual_norm(&nr)) break;
    }
  } while (false);
  if (s) cudaStreamSynchronize(s);
  // the caller's stream continues after the solve
  if (ev && s && status == SMAT_OK) {
    chk(cudaEventRecord(ev, s));
    chk(cudaStreamWaitEvent(user, ev, 0));
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (ev) cudaEventDestroy(ev);
  if (s) cudaStreamDestroy(s);
  inf.relres = nb > 0.0 ? nr / nb : 0.0;
  if (nb > 0.0 && inf.relres <= o.rtol) inf.converged = 1;
  inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) *info = inf;
  if (status != SMAT_OK) return status;
  return inf.converged ? SMAT_OK : SMAT_ERR_NOT_CONVERGED;
}
