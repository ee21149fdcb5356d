// Batched SpMV: many matrices of uneven size in one persistent launch.
//
// The paper motivates input adaptivity with algebraic multigrid, whose levels
// are different sparse matrices used one after another (Sec. 1): no single
// format fits all levels, and the coarse levels are far too small to fill a
// GPU on their own.  Here every matrix keeps the format its own tuning chose
// (CSR with 1/4/8/32 lanes per row, ELL, DIA or SELL; HYB and BCSR members
// run through their fastest measured CSR kernel); the products are cut into
// row (SELL: slice) tiles, sorted largest first into one work table per
// format kind, and persistent grids take tiles from atomic counters until
// the tables are empty.  The counter
// reset and the kernel are captured once in a CUDA graph, so one product of
// the whole batch is one graph launch.  An autotuner picks the tile size and
// the number of resident CTAs per SM by timing the captured graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "smat_internal.h"
#include "spmv_device.cuh"

namespace smat {
namespace {

enum : int { KIND_CSR = 0, KIND_ELL = 1, KIND_DIA = 2, KIND_SELL = 3, NKIND = 4 };

struct BatchMat {
  int kind, W, nd, epi, lane;
  long long m, n, K, P;
  const int32_t *rowptr, *colidx;
  const void *val;
  const int32_t *ecol;
  const void *eval;
  const int32_t *doff;
  const void *dval;
  const long long *sptr;
  const int32_t *swidth, *sperm, *scol;
  const void *sval;
  const void *x;
  void *y;
  double alpha, beta;
};

struct BatchTile {
  int mat, row0, row1, pad;
};

constexpr int BNT = 256;

// Rows [row0, row1) of a CSR product with W lanes per row (W = 1: one thread
// per row).  The loop bound is uniform over the block, so shuffles see every
// lane.
template <typename V, typename T, int W, int MODE>
__device__ __forceinline__ void csr_rows(const BatchMat &M, const Epi<T, MODE> &ep, long long row0, long long row1) {
  const int32_t *__restrict__ rowptr = M.rowptr;
  const int32_t *__restrict__ col = M.colidx;
  const V *__restrict__ val = (const V *)M.val;
  const T *__restrict__ x = (const T *)M.x;
  T *__restrict__ y = (T *)M.y;
  constexpr int RPB = BNT / W;
  constexpr int B = W == 1 ? 8 : 4;
  const int sub = threadIdx.x % W;
  for (long long base = row0; base < row1; base += RPB) {
    const long long row = base + threadIdx.x / W;
    T acc = 0;
    if (row < row1) {
      const int s = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
      for (int k = s + sub; k < e; k += B * W) {
        int c[B];
        T v[B], xv[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
          c[u] = k + u * W < e ? ld_idx(col + k + u * W) : 0;
          v[u] = k + u * W < e ? (T)ld_val(val + k + u * W) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < B; ++u) xv[u] = k + u * W < e ? __ldg(x + c[u]) : (T)0;
#pragma unroll
        for (int u = 0; u < B; ++u)
          if (k + u * W < e) acc = fused(acc, v[u], xv[u]);
      }
    }
    if (W > 1) {
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, W);
    }
    if (sub == 0 && row < row1) y[row] = ep(acc, y, row);
  }
}

// One tile of one member, in the member's format (KIND is the member's kind).
template <typename V, int KIND, int MODE>
__device__ __forceinline__ void batch_tile(const BatchMat &M, const BatchTile &tl) {
  typedef typename Compute<V>::T T;
  constexpr int R = 16 / (int)sizeof(V);
  const Epi<T, MODE> ep{(T)M.alpha, (T)M.beta};
  // tiles of ELL members start at multiples of BNT*R rows, so the
  // lane-striped mapping (32*R rows per warp) stays inside its tile
  if (KIND == KIND_ELL) {
    if (M.lane) {
      for (long long b = tl.row0 + (long long)(threadIdx.x >> 5) * 32 * R; b < tl.row1; b += (long long)BNT * R)
        ell_lane_group<V, R, MODE, 16 / R>(M.ecol, (const V *)M.eval, M.P, M.K, (const T *)M.x, ep, (T *)M.y, M.m, b,
                                           threadIdx.x & 31);
    } else {
      for (long long i0 = tl.row0 + (long long)threadIdx.x * R; i0 < tl.row1; i0 += (long long)BNT * R)
        ell_group<V, R, MODE>(M.ecol, (const V *)M.eval, M.P, M.K, (const T *)M.x, ep, (T *)M.y, M.m, i0);
    }
  } else if (KIND == KIND_DIA) {
    // The single-matrix kernel's bodies: FP64 lane-striped rows with 4
    // diagonals per batch (tiles start at multiples of BNT*R rows, so a
    // warp's 32*R rows stay inside its tile); FP32 and BF16 consecutive rows
    // with the unchecked interior path.  They need this kind's bound of 3 CTAs
    // per SM (80 registers; ptxas: an 8-byte spill for FP64, none otherwise).
    // The checked consecutive-row body that fits 64 registers took 0.431 ms
    // on the Galerkin hierarchy of the 27-point operator on 128^3 (DIA on its
    // two finest levels) against 0.244.
    if (sizeof(V) == 8) {
      for (long long b = tl.row0 + (long long)(threadIdx.x >> 5) * 32 * R; b < tl.row1; b += (long long)BNT * R)
        dia_lane_group<V, R, MODE, 4>(M.doff, M.nd, (const V *)M.dval, M.P, (const T *)M.x, ep, (T *)M.y, M.m, M.n, b,
                                      threadIdx.x & 31);
    } else {
      for (long long i0 = tl.row0 + (long long)threadIdx.x * R; i0 < tl.row1; i0 += (long long)BNT * R)
        dia_group<V, R, MODE, 16 / R, true>(M.doff, M.nd, (const V *)M.dval, M.P, (const T *)M.x, ep, (T *)M.y, M.m,
                                            M.n, i0);
    }
  } else if (KIND == KIND_SELL) {  // row0 / row1 are slice indices; a warp per slice
    for (long long sl = tl.row0 + threadIdx.x / 32; sl < tl.row1; sl += BNT / 32)
      sell_slice<V, MODE, 8>(M.sptr, M.swidth, M.sperm, M.scol, (const V *)M.sval, (const T *)M.x, ep, (T *)M.y, sl,
                             threadIdx.x & 31);
  } else {
    switch (M.W) {
      case 1: csr_rows<V, T, 1, MODE>(M, ep, tl.row0, tl.row1); break;
      case 4: csr_rows<V, T, 4, MODE>(M, ep, tl.row0, tl.row1); break;
      case 8: csr_rows<V, T, 8, MODE>(M, ep, tl.row0, tl.row1); break;
      default: csr_rows<V, T, 32, MODE>(M, ep, tl.row0, tl.row1); break;
    }
  }
}

// Persistent CTAs of one format kind take tiles of that kind from an atomic
// counter, largest first, until none are left.  One kernel per kind keeps
// each kernel's register budget to its own format's needs.
template <typename V, int KIND>
__global__ void __launch_bounds__(BNT, KIND == KIND_ELL ? 2 : (KIND == KIND_DIA ? 3 : 4)) batch_kernel(const BatchMat *__restrict__ mats,
                                                    const BatchTile *__restrict__ tiles, int ntiles,
                                                    unsigned int *counter) {
  __shared__ int s_t;
  for (;;) {
    if (threadIdx.x == 0) s_t = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int t = s_t;
    __syncthreads();  // every thread has read s_t before it is overwritten
    if (t >= ntiles) return;
    const BatchTile tl = tiles[t];
    const BatchMat &M = mats[tl.mat];
    switch (M.epi) {
      case EPI_COPY: batch_tile<V, KIND, EPI_COPY>(M, tl); break;
      case EPI_SCALE: batch_tile<V, KIND, EPI_SCALE>(M, tl); break;
      default: batch_tile<V, KIND, EPI_AXPBY>(M, tl); break;
    }
  }
}

template <int KIND>
cudaError_t launch_kind(smat_dtype_t dt, int grid, const BatchMat *mats, const BatchTile *tiles, int ntiles,
                        unsigned int *counter, cudaStream_t s) {
  switch (dt) {
    case SMAT_F64: batch_kernel<double, KIND><<<grid, BNT, 0, s>>>(mats, tiles, ntiles, counter); break;
    case SMAT_F32: batch_kernel<float, KIND><<<grid, BNT, 0, s>>>(mats, tiles, ntiles, counter); break;
    default: batch_kernel<__nv_bfloat16, KIND><<<grid, BNT, 0, s>>>(mats, tiles, ntiles, counter); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_kernel(int kind, smat_dtype_t dt, int grid, const BatchMat *mats, const BatchTile *tiles,
                                int ntiles, unsigned int *counter, cudaStream_t s) {
  if (kind == KIND_ELL) return launch_kind<KIND_ELL>(dt, grid, mats, tiles, ntiles, counter, s);
  if (kind == KIND_DIA) return launch_kind<KIND_DIA>(dt, grid, mats, tiles, ntiles, counter, s);
  if (kind == KIND_SELL) return launch_kind<KIND_SELL>(dt, grid, mats, tiles, ntiles, counter, s);
  return launch_kind<KIND_CSR>(dt, grid, mats, tiles, ntiles, counter, s);
}

}  // namespace
}  // namespace smat

struct smat_batch_s {
  std::vector<smat_handle_t> hs;
  smat_dtype_t dtype = SMAT_F64;
  std::vector<smat::BatchMat> mats;        // host copy of the descriptors
  std::vector<std::vector<int32_t>> rowptrs;  // CSR members: row pointers for nnz-balanced tiles
  std::vector<std::vector<long long>> sptrs;  // SELL members: slice pointers for slot-balanced tiles
  smat::BatchMat *d_mats = nullptr;
  smat::BatchTile *d_tiles = nullptr;
  unsigned int *d_counter = nullptr;  // one tile counter per format kind
  int ntiles = 0, grid = 0, tile_scale = 0, ctas_per_sm = 0;
  int kind_tiles[smat::NKIND] = {}, kind_first[smat::NKIND] = {}, kind_grid[smat::NKIND] = {};
  double tuned_ms = -1.0, graph_ms = -1.0, loop_ms = -1.0;
  bool loop = false;  // the members' own launches in turn won the tuning
  // Which members run their own plan's kernels inside the graph, on the
  // side branches own_st (0: none; 1: those whose plan has no batch kind;
  // 2: all), and the pointers and scalars baked into those launches.
  int own_mode = 0;
  std::vector<char> own;
  std::vector<const void *> own_x;
  std::vector<void *> own_y;
  std::vector<double> own_a, own_b;
  static constexpr int OWN_N = 4;
  cudaStream_t cap = nullptr, fork[smat::NKIND - 1] = {}, own_st[OWN_N] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[smat::NKIND - 1] = {}, ev_own[OWN_N] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ready = false;
};

namespace smat {
namespace {

smat_status_t st_of(cudaError_t e) {
  if (e == cudaSuccess) return SMAT_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SMAT_ERR_ALLOC;
  }
  return SMAT_ERR_CUDA;
}

#define BTRY(call)                    \
  do {                                \
    smat_status_t _s = st_of(call);   \
    if (_s != SMAT_OK) return _s;     \
  } while (0)

int csr_width(const smat_s *h) {
  switch (h->variant) {
    case SMAT_V_CSR_SCALAR: return 1;
    case SMAT_V_CSR_VEC4: return 4;
    case SMAT_V_CSR_VEC8: return 8;
    case SMAT_V_CSR_VEC32: return 32;
  }
  // merge-path / COO plans: the fastest measured CSR row kernel, else by mean row length
  int best = -1;
  float bt = 1e30f;
  const int ws[4] = {1, 4, 8, 32};
  for (int v = SMAT_V_CSR_SCALAR; v <= SMAT_V_CSR_VEC32; ++v)
    if (h->timings[v] > 0 && h->timings[v] < bt) { bt = h->timings[v]; best = ws[v]; }
  if (best > 0) return best;
  const double a = h->have_features ? h->f.aver_rd : 8.0;
  return a < 8.0 ? 4 : (a < 24.0 ? 8 : 32);
}

void free_graph(smat_batch_s *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Work table for a tile scale: CSR tiles hold about 2048*scale stored entries
// (whole rows, so one long row is a tile of its own); ELL/DIA tiles hold
// 256*R*scale rows.  Sorted by estimated work, largest first.
std::vector<BatchTile> make_tiles(const smat_batch_s *b, int scale) {
  struct Est { BatchTile t; long long w; };
  std::vector<Est> v;
  const int R = 16 / elem_size(b->dtype);
  for (size_t i = 0; i < b->mats.size(); ++i) {
    const BatchMat &M = b->mats[i];
    if (M.m == 0 || (!b->own.empty() && b->own[i])) continue;
    if (M.kind == KIND_CSR) {
      const std::vector<int32_t> &rp = b->rowptrs[i];
      const long long target = 2048LL * scale;
      long long r0 = 0;
      while (r0 < M.m) {
        long long r1 = r0;
        const long long cap_rows = 8192LL * scale;
        while (r1 < M.m && (long long)rp[r1] - rp[r0] < target && r1 - r0 < cap_rows) ++r1;
        if (r1 == r0) ++r1;
        v.push_back({{(int)i, (int)r0, (int)r1, 0}, (long long)rp[r1] - rp[r0] + (r1 - r0)});
        r0 = r1;
      }
    } else if (M.kind == KIND_SELL) {
      const std::vector<long long> &sp = b->sptrs[i];
      const long long ns = (long long)sp.size() - 1, target = 2048LL * scale, cap_sl = 8LL * 8 * scale;
      long long s0 = 0;
      while (s0 < ns) {
        long long s1 = s0;
        while (s1 < ns && sp[s1] - sp[s0] < target && s1 - s0 < cap_sl) ++s1;
        if (s1 == s0) ++s1;
        v.push_back({{(int)i, (int)s0, (int)s1, 0}, sp[s1] - sp[s0] + 32 * (s1 - s0)});
        s0 = s1;
      }
    } else {
      const long long rows = (long long)BNT * R * scale;
      const long long per_row = M.kind == KIND_ELL ? M.K : M.nd;
      for (long long r0 = 0; r0 < M.m; r0 += rows) {
        long long r1 = std::min(M.m, r0 + rows);
        v.push_back({{(int)i, (int)r0, (int)r1, 0}, (r1 - r0) * (per_row + 1)});
      }
    }
  }
  // grouped by format kind (CSR, ELL, DIA, SELL), each group largest first
  std::stable_sort(v.begin(), v.end(), [&](const Est &a, const Est &c) {
    const int ka = b->mats[(size_t)a.t.mat].kind, kc = b->mats[(size_t)c.t.mat].kind;
    return ka != kc ? ka < kc : a.w > c.w;
  });
  std::vector<BatchTile> out;
  out.reserve(v.size());
  for (auto &e : v) out.push_back(e.t);
  return out;
}

// A member the persistent kernel runs natively: CSR-scalar / vector, ELL,
// DIA, SELL (the others run there through a CSR row kernel).
bool batch_native(const smat_s *h) {
  switch (h->variant) {
    case SMAT_V_CSR_SCALAR: case SMAT_V_CSR_VEC4: case SMAT_V_CSR_VEC8: case SMAT_V_CSR_VEC32:
    case SMAT_V_ELL: case SMAT_V_DIA: case SMAT_V_SELL:
      return true;
  }
  return false;
}

// A member's own product (its plan's kernels) on stream st.
cudaError_t own_launch(const smat_batch_s *b, size_t i, cudaStream_t st) {
  const smat_s *h = b->hs[i];
  const double a = b->own_a[i], c = b->own_b[i];
  const float af = (float)a, cf = (float)c;
  const bool f64 = b->dtype == SMAT_F64;
  return launch_spmv(h, h->variant, f64 ? (const void *)&a : (const void *)&af, b->own_x[i],
                     f64 ? (const void *)&c : (const void *)&cf, b->own_y[i], st);
}

smat_status_t build_plan(smat_batch_s *b, int scale, int ctas_per_sm, int own_mode) {
  free_graph(b);
  const size_t n = b->hs.size();
  b->own_mode = own_mode;
  b->own.assign(n, 0);
  for (size_t i = 0; i < n; ++i)
    b->own[i] = b->mats[i].m > 0 && (own_mode == 2 || (own_mode == 1 && !batch_native(b->hs[i])));
  // the own launches' pointers and scalars, as the descriptors hold them now
  b->own_x.assign(n, nullptr);
  b->own_y.assign(n, nullptr);
  b->own_a.assign(n, 1.0);
  b->own_b.assign(n, 0.0);
  int k_own = 0;
  for (size_t i = 0; i < n; ++i)
    if (b->own[i]) {
      b->own_x[i] = b->mats[i].x; b->own_y[i] = b->mats[i].y;
      b->own_a[i] = b->mats[i].alpha; b->own_b[i] = b->mats[i].beta;
      // carries of merge / COO / SPLIT plans: the branch stream's own scratch,
      // allocated now, outside the capture
      Scratch sc{};
      BTRY(stream_scratch(b->hs[i], b->own_st[k_own % smat_batch_s::OWN_N], &sc, true));
      ++k_own;
    }
  dev_free(b->d_tiles);
  b->d_tiles = nullptr;
  std::vector<BatchTile> tiles = make_tiles(b, scale);
  b->ntiles = (int)tiles.size();
  for (int k = 0; k < NKIND; ++k) b->kind_tiles[k] = 0;
  for (const BatchTile &t : tiles) ++b->kind_tiles[b->mats[(size_t)t.mat].kind];
  b->kind_first[0] = 0;
  for (int k = 1; k < NKIND; ++k) b->kind_first[k] = b->kind_first[k - 1] + b->kind_tiles[k - 1];
  if (b->ntiles > 0) {
    void *p = nullptr;
    BTRY(dev_alloc(&p, tiles.size() * sizeof(BatchTile)));
    b->d_tiles = (BatchTile *)p;
    BTRY(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(BatchTile), cudaMemcpyHostToDevice));
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->grid = 0;
  for (int k = 0; k < NKIND; ++k) {
    b->kind_grid[k] = b->kind_tiles[k] > 0 ? std::min(sms * ctas_per_sm, b->kind_tiles[k]) : 0;
    b->grid += b->kind_grid[k];
  }
  b->tile_scale = scale;
  b->ctas_per_sm = ctas_per_sm;
  // capture: reset the tile counters, then one persistent kernel per format
  // kind on parallel branches of the graph
  BTRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaMemsetAsync(b->d_counter, 0, NKIND * sizeof(unsigned int), b->cap);
  if (err == cudaSuccess) err = cudaEventRecord(b->ev_fork, b->cap);
  cudaStream_t st[NKIND] = {b->cap, b->fork[0], b->fork[1], b->fork[2]};
  for (int k = 1; k < NKIND && err == cudaSuccess; ++k) err = cudaStreamWaitEvent(st[k], b->ev_fork, 0);
  for (int k = 0; k < NKIND && err == cudaSuccess; ++k)
    if (b->kind_tiles[k] > 0)
      err = launch_batch_kernel(k, b->dtype, b->kind_grid[k], b->d_mats, b->d_tiles + b->kind_first[k],
                                b->kind_tiles[k], b->d_counter + k, st[k]);
  for (int k = 1; k < NKIND && err == cudaSuccess; ++k) {
    err = cudaEventRecord(b->ev_join[k - 1], st[k]);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(b->cap, b->ev_join[k - 1], 0);
  }
  // the members that run their own plans, round robin on the side branches
  if (k_own > 0) {
    const int used = std::min(k_own, smat_batch_s::OWN_N);
    for (int k = 0; k < used && err == cudaSuccess; ++k) err = cudaStreamWaitEvent(b->own_st[k], b->ev_fork, 0);
    int j = 0;
    for (size_t i = 0; i < n && err == cudaSuccess; ++i)
      if (b->own[i]) err = own_launch(b, i, b->own_st[j++ % smat_batch_s::OWN_N]);
    for (int k = 0; k < used && err == cudaSuccess; ++k) {
      err = cudaEventRecord(b->ev_own[k], b->own_st[k]);
      if (err == cudaSuccess) err = cudaStreamWaitEvent(b->cap, b->ev_own[k], 0);
    }
  }
  cudaError_t e3 = cudaStreamEndCapture(b->cap, &b->graph);
  BTRY(err);
  BTRY(e3);
  BTRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  b->ready = true;
  return SMAT_OK;
}

}  // namespace
}  // namespace smat

using namespace smat;

extern "C" {

smat_status_t smat_batch_create(smat_batch_t *out, const smat_handle_t *hs, int32_t count) {
  if (!out || !hs || count <= 0) return SMAT_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return SMAT_ERR_INVALID_ARG;
    if (hs[i]->dtype != hs[0]->dtype) return SMAT_ERR_INVALID_ARG;
  }
  smat_batch_s *b = new (std::nothrow) smat_batch_s();
  if (!b) return SMAT_ERR_ALLOC;
  b->hs.assign(hs, hs + count);
  b->dtype = hs[0]->dtype;
  auto fail = [&](smat_status_t s) { smat_batch_destroy(b); return s; };
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int k = 0; k < NKIND - 1 && e == cudaSuccess; ++k)
    e = cudaStreamCreateWithFlags(&b->fork[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int k = 0; k < NKIND - 1 && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming);
  for (int k = 0; k < smat_batch_s::OWN_N && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&b->own_st[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_own[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return fail(SMAT_ERR_CUDA);
  void *p = nullptr;
  if ((e = dev_alloc(&p, NKIND * sizeof(unsigned int))) != cudaSuccess) return fail(st_of(e));
  b->d_counter = (unsigned int *)p;
  if ((e = dev_alloc(&p, sizeof(BatchMat) * (size_t)count)) != cudaSuccess) return fail(st_of(e));
  b->d_mats = (BatchMat *)p;
  *out = b;
  return SMAT_OK;
}

smat_status_t smat_batch_destroy(smat_batch_t b) {
  if (!b) return SMAT_OK;
  if (b->cap) cudaStreamSynchronize(b->cap);
  free_graph(b);
  dev_free(b->d_tiles);
  dev_free(b->d_mats);
  dev_free(b->d_counter);
  for (int k = 0; k < NKIND - 1; ++k) {
    if (b->fork[k]) cudaStreamDestroy(b->fork[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
  }
  for (int k = 0; k < smat_batch_s::OWN_N; ++k) {
    if (b->own_st[k]) cudaStreamDestroy(b->own_st[k]);
    if (b->ev_own[k]) cudaEventDestroy(b->ev_own[k]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
  return SMAT_OK;
}

smat_status_t smat_batch_tune(smat_batch_t b, const smat_batch_opts_t *opts, void *stream) {
  if (!b) return SMAT_ERR_INVALID_ARG;
  smat_batch_opts_t o;
  if (opts) o = *opts; else smat_batch_opts_default(&o);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)b->hs.size();
  b->mats.assign((size_t)n, BatchMat{});
  b->rowptrs.assign((size_t)n, {});
  b->sptrs.assign((size_t)n, {});
  const int tsz = b->dtype == SMAT_F64 ? 8 : 4;
  // per-matrix descriptors from each handle's plan, with scratch x / y for timing
  std::vector<void *> tmp;
  struct Free { std::vector<void *> &v; ~Free() { for (void *p : v) dev_free(p); } } guard{tmp};
  for (int i = 0; i < n; ++i) {
    smat_s *h = b->hs[(size_t)i];
    BatchMat &M = b->mats[(size_t)i];
    M.m = h->m; M.n = h->n; M.P = h->P;
    if (h->variant == SMAT_V_ELL && h->ell_val) {
      M.kind = KIND_ELL; M.ecol = h->ell_col; M.eval = h->ell_val; M.K = h->ell_K; M.lane = h->ell_lane;
    } else if (h->variant == SMAT_V_DIA && h->dia_val) {
      M.kind = KIND_DIA; M.doff = h->dia_off; M.dval = h->dia_val; M.nd = (int)h->dia_nd;
    } else if (h->variant == SMAT_V_SELL && h->sell_val) {
      M.kind = KIND_SELL; M.sptr = h->sell_ptr; M.swidth = h->sell_width; M.sperm = h->sell_perm;
      M.scol = h->sell_col; M.sval = h->sell_val;
      b->sptrs[(size_t)i].resize((size_t)h->sell_ns + 1);
      BTRY(cudaMemcpy(b->sptrs[(size_t)i].data(), h->sell_ptr, (size_t)(h->sell_ns + 1) * 8, cudaMemcpyDeviceToHost));
    } else {
      M.kind = KIND_CSR; M.W = csr_width(h); M.rowptr = h->rowptr; M.colidx = h->colidx; M.val = h->val;
      b->rowptrs[(size_t)i].resize((size_t)h->m + 1);
      BTRY(cudaMemcpy(b->rowptrs[(size_t)i].data(), h->rowptr, (size_t)(h->m + 1) * 4, cudaMemcpyDeviceToHost));
    }
    void *x = nullptr, *y = nullptr;
    BTRY(dev_alloc(&x, (size_t)std::max<int64_t>(h->n, 1) * tsz));
    tmp.push_back(x);
    BTRY(dev_alloc(&y, (size_t)std::max<int64_t>(h->m, 1) * tsz));
    tmp.push_back(y);
    BTRY(cudaMemsetAsync(x, 0, (size_t)std::max<int64_t>(h->n, 1) * tsz, s));
    M.x = x; M.y = y; M.alpha = 1.0; M.beta = 0.0; M.epi = EPI_COPY;
  }
  BTRY(cudaMemcpyAsync(b->d_mats, b->mats.data(), sizeof(BatchMat) * (size_t)n, cudaMemcpyHostToDevice, s));
  BTRY(cudaStreamSynchronize(s));
  if (o.mode < SMAT_BATCH_AUTO || o.mode > SMAT_BATCH_PER_MATRIX) return SMAT_ERR_INVALID_ARG;
  // autotune: tile scale x resident CTAs per SM, timed as the captured graph
  std::vector<int> scales, ctas;
  if (o.tile_scale > 0) scales.push_back(o.tile_scale); else scales = {1, 2, 4, 8};
  if (o.ctas_per_sm > 0) ctas.push_back(o.ctas_per_sm); else ctas = {2, 4, 8};
  cudaEvent_t e0, e1;
  BTRY(cudaEventCreate(&e0));
  BTRY(cudaEventCreate(&e1));
  struct EvFree { cudaEvent_t a, c; ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(c); } } evf{e0, e1};
  double best = 1e30;
  int best_s = scales[0], best_c = ctas[0], best_own = 0;
  const int reps = std::max(1, o.trial_reps);
  if (o.mode == SMAT_BATCH_PER_MATRIX) scales.clear();
  // own-launch modes worth timing: the non-native members on side branches
  // (when there are both kinds), and every member on them (AUTO only)
  bool any_own = false, any_native = false;
  for (int i = 0; i < n; ++i) {
    if (b->mats[(size_t)i].m == 0) continue;
    if (batch_native(b->hs[(size_t)i])) any_native = true; else any_own = true;
  }
  std::vector<int> owns;
  if (o.own_launches >= 0 && o.own_launches <= 2) {
    owns.push_back(o.own_launches);
  } else if (o.own_launches != -1) {
    return SMAT_ERR_INVALID_ARG;
  } else {
    owns.push_back(0);
    if (any_own && any_native) owns.push_back(1);
    if (o.mode == SMAT_BATCH_AUTO) owns.push_back(2);
  }
  struct Cand { int sc, cp, own; };
  std::vector<Cand> cands;
  for (int ow : owns) {
    if (ow == 2) {  // no persistent kernels: one shape only
      if (!scales.empty()) cands.push_back({scales[0], ctas[0], 2});
      continue;
    }
    for (int sc : scales)
      for (int cp : ctas) cands.push_back({sc, cp, ow});
  }
  double enq_us = 10.0;  // host time to queue one launch
  for (const Cand &cd : cands) {
    {
      const int sc = cd.sc, cp = cd.cp;
      {
        smat_status_t st = build_plan(b, sc, cp, cd.own);
        if (st != SMAT_OK) return st;
      }
      for (int w = 0; w < 2; ++w) BTRY(cudaGraphLaunch(b->exec, s));
      std::vector<float> ms((size_t)reps);
      for (int r = 0; r < reps; ++r) {
        // queued behind a device hold, so that the events bracket the graph alone
        BTRY(queue_ahead(s, &enq_us, 1, [&]() -> cudaError_t {
          cudaError_t q = cudaEventRecord(e0, s);
          if (q == cudaSuccess) q = cudaGraphLaunch(b->exec, s);
          if (q == cudaSuccess) q = cudaEventRecord(e1, s);
          return q;
        }));
        BTRY(cudaEventSynchronize(e1));
        BTRY(cudaEventElapsedTime(&ms[(size_t)r], e0, e1));
      }
      std::nth_element(ms.begin(), ms.begin() + reps / 2, ms.end());
      const double med = ms[(size_t)reps / 2];
      if (med < best) { best = med; best_s = sc; best_c = cp; best_own = cd.own; }
    }
  }
  b->graph_ms = scales.empty() ? -1.0 : best;
  // the members' own plans launched in turn, timed the same way
  b->loop = false;
  b->loop_ms = -1.0;
  if (o.mode != SMAT_BATCH_GRAPH) {
    const double one = 1.0, zero = 0.0;
    const float onef = 1.0f, zerof = 0.0f;
    const void *al = b->dtype == SMAT_F64 ? (const void *)&one : (const void *)&onef;
    const void *be = b->dtype == SMAT_F64 ? (const void *)&zero : (const void *)&zerof;
    auto run_loop = [&]() -> cudaError_t {
      for (int i = 0; i < n; ++i) {
        const BatchMat &M = b->mats[(size_t)i];
        if (M.m == 0) continue;
        const smat_s *h = b->hs[(size_t)i];
        cudaError_t e = launch_spmv(h, h->variant, al, M.x, be, M.y, s);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    };
    for (int w = 0; w < 2; ++w) BTRY(run_loop());
    std::vector<float> ms((size_t)reps);
    for (int r = 0; r < reps; ++r) {
      BTRY(queue_ahead(s, &enq_us, n, [&]() -> cudaError_t {
        cudaError_t q = cudaEventRecord(e0, s);
        if (q == cudaSuccess) q = run_loop();
        if (q == cudaSuccess) q = cudaEventRecord(e1, s);
        return q;
      }));
      BTRY(cudaEventSynchronize(e1));
      BTRY(cudaEventElapsedTime(&ms[(size_t)r], e0, e1));
    }
    std::nth_element(ms.begin(), ms.begin() + reps / 2, ms.end());
    b->loop_ms = ms[(size_t)reps / 2];
    b->loop = o.mode == SMAT_BATCH_PER_MATRIX || b->loop_ms < best;
  }
  if (b->loop) {
    free_graph(b);
    b->tuned_ms = b->loop_ms;
    b->ready = true;
  } else {
    smat_status_t st = build_plan(b, best_s, best_c, best_own);
    if (st != SMAT_OK) return st;
    b->tuned_ms = best;
  }
  // forget the timing buffers: the next smat_batch_spmv installs the caller's vectors
  for (auto &M : b->mats) { M.x = nullptr; M.y = nullptr; }
  BTRY(cudaStreamSynchronize(s));
  return SMAT_OK;
}

smat_status_t smat_batch_spmv(smat_batch_t b, const void *alphas, const void *const *xs, const void *betas,
                              void *const *ys, void *stream) {
  if (!b || !alphas || !betas || !xs || !ys) return SMAT_ERR_INVALID_ARG;
  if (!b->ready) return SMAT_ERR_UNSUPPORTED;
  const int n = (int)b->hs.size();
  bool changed = false;
  for (int i = 0; i < n; ++i) {
    BatchMat &M = b->mats[(size_t)i];
    const double a = b->dtype == SMAT_F64 ? ((const double *)alphas)[i] : (double)((const float *)alphas)[i];
    const double c = b->dtype == SMAT_F64 ? ((const double *)betas)[i] : (double)((const float *)betas)[i];
    if ((M.m > 0 && !ys[i]) || (M.n > 0 && M.m > 0 && !xs[i])) return SMAT_ERR_INVALID_ARG;
    // ELL and DIA members read x and write y with 16-byte vector accesses
    if ((M.kind == KIND_ELL || M.kind == KIND_DIA) && (((uintptr_t)xs[i] | (uintptr_t)ys[i]) & 15u) != 0)
      return SMAT_ERR_INVALID_ARG;
    if (M.x != xs[i] || M.y != ys[i] || M.alpha != a || M.beta != c) {
      M.x = xs[i]; M.y = ys[i]; M.alpha = a; M.beta = c;
      M.epi = epi_mode(a, c);
      changed = true;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (b->loop) {  // the members' own plans, in turn
    const size_t ts = b->dtype == SMAT_F64 ? sizeof(double) : sizeof(float);
    for (int i = 0; i < n; ++i) {
      const smat_s *h = b->hs[(size_t)i];
      if (h->m == 0) continue;
      BTRY(launch_spmv(h, h->variant, (const char *)alphas + ts * (size_t)i, xs[i], (const char *)betas + ts * (size_t)i,
                       ys[i], s));
    }
    return SMAT_OK;
  }
  // members with their own launches in the graph carry their pointers and
  // scalars in it: a change there means capturing the graph again (the
  // previous graph launch on `s` is finished with them once `s` reaches here)
  bool recapture = false;
  for (int i = 0; i < n && !recapture; ++i) {
    if (b->own.empty() || !b->own[(size_t)i]) continue;
    const BatchMat &M = b->mats[(size_t)i];
    recapture = M.x != b->own_x[(size_t)i] || M.y != b->own_y[(size_t)i] || M.alpha != b->own_a[(size_t)i] ||
                M.beta != b->own_b[(size_t)i];
  }
  if (recapture) {
    BTRY(cudaStreamSynchronize(s));
    smat_status_t st = build_plan(b, b->tile_scale, b->ctas_per_sm, b->own_mode);
    if (st != SMAT_OK) return st;
  }
  if (changed)
    BTRY(cudaMemcpyAsync(b->d_mats, b->mats.data(), sizeof(BatchMat) * (size_t)n, cudaMemcpyHostToDevice, s));
  BTRY(cudaGraphLaunch(b->exec, s));
  return SMAT_OK;
}

smat_status_t smat_batch_get_info(smat_batch_t b, smat_batch_info_t *info) {
  if (!b || !info) return SMAT_ERR_INVALID_ARG;
  info->count = (int32_t)b->hs.size();
  info->tiles = b->ntiles;
  info->grid = b->grid;
  info->tile_scale = b->tile_scale;
  info->ctas_per_sm = b->ctas_per_sm;
  info->tuned_ms = b->tuned_ms;
  info->per_matrix = b->loop ? 1 : 0;
  info->graph_ms = b->graph_ms;
  info->per_matrix_ms = b->loop_ms;
  info->own_launches = b->loop ? 0 : b->own_mode;
  return SMAT_OK;
}

void smat_batch_opts_default(smat_batch_opts_t *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tile_scale = 0;
  o->ctas_per_sm = 0;
  o->trial_reps = 10;
  o->mode = SMAT_BATCH_AUTO;
  o->own_launches = -1;
}

}  // extern "C"
