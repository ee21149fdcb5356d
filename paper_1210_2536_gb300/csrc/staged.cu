// DIA product with the diagonal stripes staged in shared memory by bulk
// asynchronous copies (Sec. 2.1: DIA stores each occupied diagonal as one
// stripe of the pitch P, zero-filled; the product walks the rows and
// multiplies each stripe's value with x at the row plus the stripe's offset).
//
// DIA is a pure stream: Ndiags * P values, read once.  The plain DIA kernel
// keeps a few 16-byte loads per thread in flight, not enough to cover HBM
// latency on a 152-SM part.  Here one CTA per SM runs a pipeline: a producer
// warp issues, for each tile of T rows, one bulk copy per diagonal stripe
// (T * value-size bytes) into a ring of S stages, several tiles ahead of the
// eight consumer warps, which read values from shared memory, gather x
// through L1/L2, and write y once.  Tiles are dealt round-robin to the CTAs,
// and the tile height is chosen so that every CTA gets the same number of
// tiles within one.
#include <atomic>

#include "pipe.cuh"
#include "smat_internal.h"
#include "spmv_device.cuh"

namespace smat {
namespace {

// Launch shapes the tuner times (smat_set_kernel ids 1..2): consumer warps
// per CTA (plus one producer warp), CTAs per SM, stages, and the target
// bytes of one stage (every stripe's slice of one tile).  Of the shapes
// measured on GB300 ((16, 1, 4, 48), (16, 2, 3, 32), (24, 1, 4, 48) and
// (8, 2, 3, 32)), these two were the fastest for FP64 and for FP32 / BF16.
struct StagedCfg {
  int warps, ctas, stages, stage_kb;
};
constexpr StagedCfg ST_CFG[] = {{16, 1, 4, 48}, {16, 2, 3, 32}};
constexpr int ST_NCFG = 2;
// About one second at the GB300's 2.07 GHz SM clock.
constexpr long long ST_WAIT_CYCLES = 2000000000LL;

// Bounded waits in these kernels that ran out (each such product's y is
// invalid).  Read by smat_get_wait_timeouts.
__device__ unsigned long long g_wait_timeouts;

// Test hook (smat_test_stall_pipelines): consumers wait on a barrier that
// nothing arrives on, for `cycles`, so that the timeout path runs.
std::atomic<int> g_stall_on{0};
std::atomic<long long> g_stall_cycles{0};

__device__ __forceinline__ double to_compute(double v) { return v; }
__device__ __forceinline__ float to_compute(float v) { return v; }
__device__ __forceinline__ float to_compute(__nv_bfloat16 v) { return __bfloat162float(v); }

// full[S], empty[S], the test hook's stall barrier, then the offsets.
__host__ __device__ inline size_t staged_head_bytes(int S, long long nd) {
  return ((size_t)16 * S + 8 + (size_t)4 * nd + 127) / 128 * 128;
}

template <typename V, int MODE, int CFG, int NW = ST_CFG[CFG].warps>
__global__ void __launch_bounds__(32 * (ST_CFG[CFG].warps + 1), ST_CFG[CFG].ctas)
    dia_staged_kernel(const int32_t *__restrict__ off, int nd, const V *__restrict__ dval, long long P, int T_rows,
                      int S, long long ntiles, const typename Compute<V>::T *__restrict__ x,
                      Epi<typename Compute<V>::T, MODE> ep, typename Compute<V>::T *__restrict__ y, long long m,
                      long long n, long long wait_limit, int stall) {
  griddep_wait();
  typedef typename Compute<V>::T T;
  constexpr int U = 8;  // diagonals whose loads are issued together
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_err;
  __shared__ long long s_issued;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty = full + S;
  uint64_t *stall_bar = empty + S;  // never arrived on: the test hook's wait
  int32_t *s_off = reinterpret_cast<int32_t *>(stall_bar + 1);
  V *stages = reinterpret_cast<V *>(smem + staged_head_bytes(S, nd));
  const size_t stage_elems = (size_t)nd * T_rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NW);
    }
    mbar_init(stall_bar, 1);
    mbar_fence_init();
    s_err = 0;
    s_issued = 0;
  }
  for (int t = threadIdx.x; t < nd; t += blockDim.x) s_off[t] = off[t];
  __syncthreads();

  if (warp == NW) {  // producer: one bulk copy per stripe per tile
    const uint64_t pol = l2_evict_first_policy();
    long long j = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int s = (int)(j % S);
      if (j >= S && !__all_sync(0xffffffffu, mbar_wait(&empty[s], (unsigned)((j / S - 1) & 1), wait_limit))) {
        if (lane == 0) s_err = 1;
        break;
      }
      const long long r0 = tile * T_rows;
      const unsigned bytes = (unsigned)(min((long long)T_rows, P - r0) * (long long)sizeof(V));
      if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes * (unsigned)nd);
      __syncwarp();
      V *dst = stages + (size_t)s * stage_elems;
      for (int d = lane; d < nd; d += 32)
        bulk_g2s(dst + (size_t)d * T_rows, dval + (long long)d * P + r0, bytes, &full[s], pol);
    }
    if (lane == 0) s_issued = j;
  } else {  // consumers: one row per thread per pass, x gathered in coalesced warp runs
    const int c = threadIdx.x;
    long long j = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
      const int s = (int)(j % S);
      uint64_t *bar = stall ? stall_bar : &full[s];
      if (!__all_sync(0xffffffffu, mbar_wait(bar, stall ? 0u : (unsigned)((j / S) & 1), wait_limit))) {
        if (lane == 0) s_err = 1;
        break;
      }
      const V *sv = stages + (size_t)s * stage_elems;
      const long long r0 = tile * T_rows;
      const int rows = (int)min((long long)T_rows, m - r0);
      for (int g = c; g < rows; g += NW * 32) {
        const long long i = r0 + g;
        T acc = 0;
        for (int d = 0; d < nd; d += U) {
          T v[U], xv[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (d + u < nd) {  // uniform over the warp
              v[u] = to_compute(sv[(size_t)(d + u) * T_rows + g]);
              const long long col = i + s_off[d + u];
              xv[u] = (col >= 0 && col < n) ? __ldg(x + col) : (T)0;
            }
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (d + u < nd) acc = fused(acc, v[u], xv[u]);
        }
        y[i] = ep(acc, y, i);
      }
      fence_proxy_async_smem();  // reads of the stage before the copy that refills it
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  // No copy may still be landing when the CTA exits: wait (bounded, with
  // the full budget even when the test hook shortened the others) for the
  // last phase armed on every stage.  After a normal run all of them have
  // completed already.
  if (threadIdx.x == 0) {
    const long long J = s_issued;
    for (int s = 0; s < S && s < J; ++s) {
      const long long jl = s + (J - 1 - s) / S * S;
      if (!mbar_wait(&full[s], (unsigned)((jl / S) & 1), ST_WAIT_CYCLES)) s_err = 1;
    }
    if (s_err) atomicAdd(&g_wait_timeouts, 1ull);
  }
}

struct StagedGeom {
  int T;             // rows per tile (a multiple of 32)
  int S;             // stages
  long long ntiles;
  int grid;
  size_t smem;
};

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) {
    int c = 0;
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 152;
    cached[dev] = c;
  }
  return cached[dev];
}

// Tile height from the stage budget of configuration `cfg` (0-based), then
// lowered so that the tile count is (nearly) a multiple of the resident CTA
// count; false when even 32 rows of every stripe do not fit a stage.
bool staged_geom(int cfg, long long m, long long nd, int esz, StagedGeom *g) {
  if (cfg < 0 || cfg >= ST_NCFG || m <= 0 || nd <= 0) return false;
  const StagedCfg &c = ST_CFG[cfg];
  const long long tmax = (long long)((size_t)c.stage_kb * 1024 / ((size_t)nd * esz)) / 32 * 32;
  if (tmax < 32) return false;
  const long long ctas = (long long)sm_count() * c.ctas;
  long long nt = (m + tmax - 1) / tmax;
  const long long want = (nt + ctas - 1) / ctas * ctas;
  long long T = ((m + want - 1) / want + 31) / 32 * 32;
  if (T > tmax) T = tmax;
  nt = (m + T - 1) / T;
  g->T = (int)T;
  g->S = c.stages;
  g->ntiles = nt;
  g->grid = (int)std::min<long long>(nt, ctas);
  g->smem = staged_head_bytes(g->S, nd) + (size_t)g->S * nd * T * esz;
  return true;
}

template <typename V, int MODE, int CFG>
cudaError_t dia_staged_cfg(const smat_s *h, const StagedGeom &g, typename Compute<V>::T alpha, const void *x,
                           typename Compute<V>::T beta, void *y, cudaStream_t s, long long wait_limit) {
  typedef typename Compute<V>::T T;
  static size_t dyn_max = 0;  // per process; the attribute is per function
  if (dyn_max == 0) {
    // dynamic plus static shared memory may not exceed the opt-in limit
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, dia_staged_kernel<V, MODE, CFG>);
    if (e != cudaSuccess) return e;
    const size_t lim = (size_t)optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(dia_staged_kernel<V, MODE, CFG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    if (e != cudaSuccess) return e;
    dyn_max = lim;
  }
  if (g.smem > dyn_max) return cudaErrorNotSupported;
  (void)launch_pdl(dia_staged_kernel<V, MODE, CFG>, dim3(g.grid), dim3(32 * (ST_CFG[CFG].warps + 1)), g.smem, s,
      h->dia_off, (int)h->dia_nd, (const V *)h->dia_val, h->P, g.T, g.S, g.ntiles, (const T *)x,
      Epi<T, MODE>{alpha, beta}, (T *)y, h->m, h->n, wait_limit, g_stall_on.load() ? 1 : 0);
  return cudaGetLastError();
}

template <typename V, int MODE>
cudaError_t dia_staged_mode(int cfg, const smat_s *h, const StagedGeom &g, typename Compute<V>::T alpha,
                            const void *x, typename Compute<V>::T beta, void *y, cudaStream_t s,
                            long long wait_limit) {
  if (cfg == 0) return dia_staged_cfg<V, MODE, 0>(h, g, alpha, x, beta, y, s, wait_limit);
  return dia_staged_cfg<V, MODE, 1>(h, g, alpha, x, beta, y, s, wait_limit);
}

template <typename V>
cudaError_t dia_staged_typed(int cfg, const smat_s *h, const StagedGeom &g, const void *alpha_p, const void *x,
                             const void *beta_p, void *y, cudaStream_t s, long long wait_limit) {
  typedef typename Compute<V>::T T;
  const T alpha = *(const T *)alpha_p, beta = *(const T *)beta_p;
  switch (epi_mode((double)alpha, (double)beta)) {
    case EPI_COPY: return dia_staged_mode<V, EPI_COPY>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
    case EPI_SCALE: return dia_staged_mode<V, EPI_SCALE>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
    default: return dia_staged_mode<V, EPI_AXPBY>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
  }
}

}  // namespace

int dia_staged_kernels() { return ST_NCFG; }

bool dia_staged_ok(const smat_s *h, int kernel) {
  StagedGeom g;
  return h->dia_val && staged_geom(kernel - 1, h->m, h->dia_nd, h->esz, &g);
}

cudaError_t launch_dia_staged(const smat_s *h, int kernel, const void *alpha, const void *x, const void *beta,
                              void *y, cudaStream_t s, long long wait_limit) {
  StagedGeom g;
  const int cfg = kernel - 1;
  if (!h->dia_val || !staged_geom(cfg, h->m, h->dia_nd, h->esz, &g)) return cudaErrorNotSupported;
  if (wait_limit <= 0) wait_limit = ST_WAIT_CYCLES;
  if (g_stall_on.load() && g_stall_cycles.load() > 0) wait_limit = g_stall_cycles.load();
  switch (h->dtype) {
    case SMAT_F64: return dia_staged_typed<double>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
    case SMAT_F32: return dia_staged_typed<float>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
    default: return dia_staged_typed<__nv_bfloat16>(cfg, h, g, alpha, x, beta, y, s, wait_limit);
  }
}

cudaError_t wait_timeouts(unsigned long long *out) {
  return cudaMemcpyFromSymbol(out, g_wait_timeouts, sizeof(*out));
}

}  // namespace smat

extern "C" void smat_test_stall_pipelines(int32_t on, int64_t wait_cycles) {
  smat::g_stall_cycles = wait_cycles;
  smat::g_stall_on = on ? 1 : 0;
}

extern "C" smat_status_t smat_get_wait_timeouts(uint64_t *count) {
  if (!count) return SMAT_ERR_INVALID_ARG;
  unsigned long long c = 0;
  if (smat::wait_timeouts(&c) != cudaSuccess) return SMAT_ERR_CUDA;
  *count = (uint64_t)c;
  return SMAT_OK;
}
