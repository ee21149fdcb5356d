// SpMV kernels y = alpha*A*x + beta*y for the four basic formats
// (arXiv 1210.2536, Sec. 2.1; the paper's kernel library maps each format to
// its best implementation, Sec. 3), and the launches of the further formats
// that reuse them (HYB: ELL + COO tail; SPLIT: long rows in CTA chunks and
// COO tiles of the short rows in one grid, then one closing pass).
// GPU implementations of CSR follow Bell & Garland (2008, cited by the paper:
// scalar and vector kernels) and Merrill & Garland (2016: merge-path); COO uses
// a tiled segmented reduction.
//
// The kernels stream the format's index and value arrays once with coalesced
// (ELL, DIA: 16-byte vector or lane-striped) loads, gather x through L1/L2 and
// write y once.  They are bound by HBM, by the random x gathers (more exactly
// by the rate of 32-byte L2 sector requests that the gathers and the streamed
// arrays make together), or (FP64) by the FP64 pipe, which GB300 runs at
// about 2 operations per clock per SM: every
// kernel spends one fused multiply-add per stored product, and only
// SMAT_V_CSR_SCALAR_EXACT rounds products and sums separately, in ascending
// column order, as the CSR definition does.  The alpha/beta epilogue is fused:
//   y_i = alpha*acc            if beta == 0 (y is not read)
//   y_i = alpha*acc + beta*y_i otherwise
// and alpha == 0 skips A and x altogether.  Storage V in {double, float,
// bf16}; compute T = double for V = double, float otherwise.
#include <cuda_bf16.h>

#include <algorithm>

#include "smat_internal.h"
#include "spmv_device.cuh"

namespace smat {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// K7: CSR-scalar, one thread per row.
// ---------------------------------------------------------------------------
template <typename V, typename T, bool EXACT, int MODE>
__global__ void __launch_bounds__(256) csr_scalar_kernel(const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ col,
                                                         const V *__restrict__ val, const T *__restrict__ x,
                                                         Epi<T, MODE, EXACT> ep, T *__restrict__ y, long long m) {
  griddep_wait();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = __ldg(rowptr + i), e = __ldg(rowptr + i + 1);
    T acc = 0;
    // eight entries per step, predicated: every index and value load, then
    // the gathers, then the in-order accumulation
    for (int k = s; k < e; k += 8) {
      int c[8];
      T v[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[u] = k + u < e ? ld_idx(col + k + u) : 0;
        v[u] = k + u < e ? (T)ld_val(val + k + u) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = k + u < e ? __ldg(x + c[u]) : (T)0;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k + u < e) acc = madd<EXACT>(acc, v[u], xv[u]);
    }
    y[i] = ep(acc, y, i);
  }
}

// ---------------------------------------------------------------------------
// K8: CSR-vector, W lanes per row, lane-strided loads, shuffle reduction.
// ---------------------------------------------------------------------------
template <typename V, typename T, int W, int MODE>
__global__ void __launch_bounds__(256) csr_vector_kernel(const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ col,
                                                         const V *__restrict__ val, const T *__restrict__ x,
                                                         Epi<T, MODE> ep, T *__restrict__ y, long long m) {
  griddep_wait();
  constexpr int RPW = 32 / W;  // rows per warp per step
  const int lane = threadIdx.x & 31, sub = lane % W;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r0 = warp * RPW; r0 < m; r0 += nwarps * RPW) {
    long long row = r0 + lane / W;
    T acc = 0;
    if (row < m) {
      const int s = __ldg(rowptr + row), e = __ldg(rowptr + row + 1);
      for (int k = s + sub; k < e; k += 4 * W) {
        int c[4];
        T v[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = k + u * W < e ? ld_idx(col + k + u * W) : 0;
          v[u] = k + u * W < e ? (T)ld_val(val + k + u * W) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = k + u * W < e ? __ldg(x + c[u]) : (T)0;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (k + u * W < e) acc = fused(acc, v[u], xv[u]);
      }
    }
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) acc += __shfl_down_sync(FULL, acc, o, W);
    if (sub == 0 && row < m) y[row] = ep(acc, y, row);
  }
}

// ---------------------------------------------------------------------------
// Tiled segmented reduction shared by merge-path CSR (K9) and COO (K12).
// A CTA consumes a tile of NT*IPT items; each thread walks IPT consecutive
// items, finishing the rows whose last nonzero it sees.  A thread's partial
// sum of the row still open at its end flows into the first row finished by a
// later thread.  Which thread that is follows from an integer max-scan of
// "last thread that finished a row", so the floating-point work is one add
// per partial (in thread order, hence deterministic) instead of a
// floating-point scan -- FP64 adds are scarce on GB300.  The partial of the
// row still open at the end of the tile becomes the tile's carry, added by a
// fix-up kernel.
// ---------------------------------------------------------------------------
// Fallback for tiles where a row spans many threads: a block-wide segmented
// scan of (finished-a-row, partial) pairs in thread order (deterministic).
template <typename T>
struct SegPair {
  int h;
  T v;
};

template <typename T>
__device__ __forceinline__ SegPair<T> seg_combine(SegPair<T> a, SegPair<T> b) {
  return SegPair<T>{a.h | b.h, b.h ? b.v : a.v + b.v};
}

template <typename T, int NT>
__device__ __forceinline__ SegPair<T> block_seg_scan(SegPair<T> x, SegPair<T> *total) {
  __shared__ int sh_h[NT / 32];
  __shared__ T sh_v[NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  SegPair<T> inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ph = __shfl_up_sync(FULL, inc.h, o);
    const T pv = __shfl_up_sync(FULL, inc.v, o);
    if (lane >= o) inc = seg_combine(SegPair<T>{ph, pv}, inc);
  }
  SegPair<T> exc{__shfl_up_sync(FULL, inc.h, 1), __shfl_up_sync(FULL, inc.v, 1)};
  if (lane == 0) exc = SegPair<T>{0, (T)0};
  if (lane == 31) { sh_h[w] = inc.h; sh_v[w] = inc.v; }
  __syncthreads();
  if (w == 0) {
    SegPair<T> wi{lane < NT / 32 ? sh_h[lane] : 0, lane < NT / 32 ? sh_v[lane] : (T)0};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ph = __shfl_up_sync(FULL, wi.h, o);
      const T pv = __shfl_up_sync(FULL, wi.v, o);
      if (lane >= o) wi = seg_combine(SegPair<T>{ph, pv}, wi);
    }
    int eh = __shfl_up_sync(FULL, wi.h, 1);
    T ev = __shfl_up_sync(FULL, wi.v, 1);
    if (lane == 0) { eh = 0; ev = (T)0; }
    if (lane < NT / 32) { sh_h[lane] = eh; sh_v[lane] = ev; }
    if (lane == NT / 32 - 1) *total = wi;
  }
  __syncthreads();
  return seg_combine(SegPair<T>{sh_h[w], sh_v[w]}, exc);
}

// h: this thread finished at least one row; c: its partial of the row open at
// its end.  Returns the sum of the earlier partials that belong to this
// thread's first finished row (meaningful when h); the last thread also
// returns the tile's open partial in *open.  Runs of up to 16 partials are
// summed serially (one add each); a tile with a longer run -- a row spanning
// many threads -- uses the block-wide segmented scan instead.
template <typename T, int NT>
__device__ __forceinline__ T tile_carries(bool h, T c, T *open) {
  __shared__ T s_c[NT];
  __shared__ int s_wmax[NT / 32];
  __shared__ SegPair<T> s_total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  s_c[threadIdx.x] = c;
  int v = h ? (int)threadIdx.x : -1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int p = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v = max(v, p);
  }
  if (lane == 31) s_wmax[w] = v;
  __syncthreads();
  int before = -1;
  for (int k = 0; k < w; ++k) before = max(before, s_wmax[k]);
  const int incl = max(v, before);        // last thread <= me that finished a row
  int excl = __shfl_up_sync(FULL, incl, 1);
  if (lane == 0) excl = before;          // last thread < me that finished a row
  const int run = h ? (int)threadIdx.x - max(excl, 0) : 0;
  const int open_run = threadIdx.x == NT - 1 ? NT - max(incl, 0) : 0;
  if (__syncthreads_or(run > 16 || open_run > 16)) {
    const SegPair<T> in = block_seg_scan<T, NT>(SegPair<T>{h ? 1 : 0, c}, &s_total);
    if (threadIdx.x == NT - 1) *open = s_total.v;
    return in.v;
  }
  T in = 0;
  if (h)
    for (int j = max(excl, 0); j < (int)threadIdx.x; ++j) in += s_c[j];
  if (threadIdx.x == NT - 1) {
    T o = 0;
    for (int j = max(incl, 0); j < NT; ++j) o += s_c[j];
    *open = o;
  }
  return in;
}

// Merge-path coordinate: number of row ends a among the first d merge items
// of (rowptr[1..m]) and (0..nnz-1), row ends first on ties.
__device__ __forceinline__ void merge_search(const int32_t *__restrict__ rowptr, long long m, long long nnz,
                                             long long d, long long *a, long long *b) {
  long long lo = d - nnz > 0 ? d - nnz : 0, hi = d < m ? d : m;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if ((long long)__ldg(rowptr + mid + 1) <= d - mid - 1) lo = mid + 1; else hi = mid;
  }
  *a = lo;
  *b = d - lo;
}

// s_v[j] = val[b0 + j], s_x[j] = x[col[b0 + j]] for j < cnt: IPT coalesced
// items per thread, every index and value load issued before the gathers.
// Merge-path coordinates (a, b) of every tile boundary d = t*tile, t = 0..ntiles
// (the last one clamped to m + nnz): one thread per boundary.
__global__ void merge_partition_kernel(const int32_t *__restrict__ rowptr, long long m, long long nnz, long long tile,
                                       long long ntiles, int2 *__restrict__ coords) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles;
       t += (long long)gridDim.x * blockDim.x) {
    const long long d = t * tile < m + nnz ? t * tile : m + nnz;
    long long a, b;
    merge_search(rowptr, m, nnz, d, &a, &b);
    coords[t] = make_int2((int)a, (int)b);
  }
}

template <typename V, typename T, int NT, int IPT>
__device__ __forceinline__ void stage_pairs(const int32_t *__restrict__ col, const V *__restrict__ val,
                                            const T *__restrict__ x, long long b0, int cnt, T *s_v, T *s_x) {
  int c[IPT];
  T v[IPT], xv[IPT];
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int j = threadIdx.x + q * NT;
    c[q] = j < cnt ? ld_idx(col + b0 + j) : 0;
    v[q] = j < cnt ? (T)ld_val(val + b0 + j) : (T)0;
  }
#pragma unroll
  for (int q = 0; q < IPT; ++q) xv[q] = (threadIdx.x + q * NT) < cnt ? __ldg(x + c[q]) : (T)0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    const int j = threadIdx.x + q * NT;
    if (j < cnt) {
      s_v[j] = v[q];
      s_x[j] = xv[q];
    }
  }
}

template <typename V, typename T, int NT, int IPT, int MODE>
__global__ void __launch_bounds__(NT) csr_merge_kernel(const int32_t *__restrict__ rowptr,
                                                       const int32_t *__restrict__ col,
                                                       const V *__restrict__ val, const T *__restrict__ x,
                                                       Epi<T, MODE> ep, T *__restrict__ y, long long m,
                                                       long long nnz, const int2 *__restrict__ coords,
                                                       int32_t *carry_row, T *carry_val) {
  griddep_wait();
  constexpr int TILE = NT * IPT;
  __shared__ int32_t s_rowend[TILE + 1];
  __shared__ T s_v[TILE], s_x[TILE];
  const long long total = m + nnz;
  const long long d0 = (long long)blockIdx.x * TILE;
  const long long d1 = d0 + TILE < total ? d0 + TILE : total;
  // the tile's merge-path coordinates, computed once per matrix
  const int2 c0 = __ldg(coords + blockIdx.x), c1 = __ldg(coords + blockIdx.x + 1);
  const long long a0 = c0.x, b0 = c0.y, a1 = c1.x, b1 = c1.y;
  const int nrows = (int)(a1 - a0), nnzs = (int)(b1 - b0);
  for (int i = threadIdx.x; i < nrows; i += NT) s_rowend[i] = __ldg(rowptr + a0 + 1 + i);
  stage_pairs<V, T, NT, IPT>(col, val, x, b0, nnzs, s_v, s_x);
  __syncthreads();
  // this thread's start on the tile's merge path
  const int items = (int)(d1 - d0);
  const int dt = min((int)threadIdx.x * IPT, items);
  int lo = dt - nnzs > 0 ? dt - nnzs : 0, hi = dt < nrows ? dt : nrows;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((long long)s_rowend[mid] <= b0 + (dt - mid - 1)) lo = mid + 1; else hi = mid;
  }
  int a = lo;
  long long b = b0 + (dt - lo);
  const int dend = min(dt + IPT, items);
  T acc = 0, first_acc = 0;
  int first_row = -1;
  for (int it = dt; it < dend; ++it) {
    if (a < nrows && (long long)s_rowend[a] <= b) {
      if (first_row < 0) {
        first_row = a;
        first_acc = acc;
      } else {
        long long r = a0 + a;
        y[r] = ep(acc, y, r);
      }
      acc = 0;
      ++a;
    } else {
      acc = fused(acc, s_v[b - b0], s_x[b - b0]);
      ++b;
    }
  }
  T tile_open = 0;
  const T incoming = tile_carries<T, NT>(first_row >= 0, acc, &tile_open);
  if (first_row >= 0) {
    long long r = a0 + first_row;
    y[r] = ep(incoming + first_acc, y, r);
  }
  if (threadIdx.x == NT - 1) {
    bool open = a1 < m && b1 > b0;
    carry_row[blockIdx.x] = open ? (int32_t)a1 : -1;
    carry_val[blockIdx.x] = open ? tile_open : (T)0;
  }
}

// 32-byte streaming loads (sm_100 and later): one L1 request per 32-byte
// sector.  Two 16-byte loads of one sector by the same thread are two
// requests, and on a kernel bound by the rate of sector requests the second
// one costs as much as the first (and comes back from L2 when the streamed
// line was evicted in between).  p must be 32-byte aligned.
__device__ __forceinline__ void ld32_i32(const int32_t *p, int *o) {
  asm("ld.global.cs.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
      : "l"(p));
}
__device__ __forceinline__ void ld32_f32(const float *p, float *o) {
  asm("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
      : "l"(p));
}
__device__ __forceinline__ void ld32_f64(const double *p, double *o) {
  asm("ld.global.cs.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(o[0]), "=d"(o[1]), "=d"(o[2]), "=d"(o[3]) : "l"(p));
}
__device__ __forceinline__ bool aligned32(const void *p) { return ((uintptr_t)p & 31u) == 0; }

// IPT consecutive int32 from p (16-byte aligned when `full`; 32-byte loads
// when 32-byte aligned, uniform over a tile since runs start at multiples of 8).
template <int IPT>
__device__ __forceinline__ void load_i32_run(const int32_t *__restrict__ p, bool full, int valid, int (&o)[IPT],
                                             int fill) {
  if (full && IPT % 8 == 0 && aligned32(p)) {
#pragma unroll
    for (int q = 0; q < IPT / 8; ++q) ld32_i32(p + 8 * q, o + 8 * q);
  } else if (full) {
#pragma unroll
    for (int q = 0; q < IPT / 4; ++q) {
      int4 v = __ldcs(reinterpret_cast<const int4 *>(p) + q);
      o[4 * q] = v.x; o[4 * q + 1] = v.y; o[4 * q + 2] = v.z; o[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < IPT; ++q) o[q] = q < valid ? ld_idx(p + q) : fill;
  }
}

template <typename V, int IPT>
__device__ __forceinline__ void load_val_run(const V *__restrict__ p, bool full, int valid,
                                             typename Compute<V>::T (&o)[IPT]) {
  constexpr int R = 16 / (int)sizeof(V);
  if constexpr (sizeof(V) == 8 && IPT % 4 == 0) {
    if (full && aligned32(p)) {
#pragma unroll
      for (int q = 0; q < IPT / 4; ++q) ld32_f64(reinterpret_cast<const double *>(p) + 4 * q, o + 4 * q);
      return;
    }
  } else if constexpr (sizeof(V) == 4 && IPT % 8 == 0) {
    if (full && aligned32(p)) {
#pragma unroll
      for (int q = 0; q < IPT / 8; ++q) ld32_f32(reinterpret_cast<const float *>(p) + 8 * q, o + 8 * q);
      return;
    }
  }
  if (full) {
#pragma unroll
    for (int q = 0; q < IPT / R; ++q) {
      typename Compute<V>::T t[R];
      load_vals<V, R>(p + q * R, t);
#pragma unroll
      for (int r = 0; r < R; ++r) o[q * R + r] = t[r];
    }
  } else {
#pragma unroll
    for (int q = 0; q < IPT; ++q) o[q] = q < valid ? (typename Compute<V>::T)ld_val(p + q) : 0;
  }
}

// One chunk of up to IPT consecutive stored entries of a COO tile: each
// product is one fused multiply-add into acc; where a row ends inside the
// chunk (row[k+1] differs) its sum is written, except the thread's first row
// end, which is held back in first_row / first_acc for the tile's carries.
template <typename T, int IPT, int MODE>
__device__ __forceinline__ void coo_chunk(const int (&r)[IPT], const int (&c)[IPT], const T (&v)[IPT], int r_next,
                                          int valid, const T *__restrict__ x, const Epi<T, MODE> &ep, T *__restrict__ y,
                                          T &acc, int &first_row, T &first_acc) {
  T xv[IPT];
#pragma unroll
  for (int q = 0; q < IPT; ++q) xv[q] = q < valid ? __ldg(x + c[q]) : (T)0;
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    if (q < valid) {
      acc = fused(acc, v[q], xv[q]);
      const int rn = q + 1 < IPT ? r[q + 1] : r_next;
      if (rn != r[q]) {  // last stored entry of row r[q]
        if (first_row < 0) {
          first_row = r[q];
          first_acc = acc;
        } else {
          y[r[q]] = ep(acc, y, (long long)r[q]);
        }
        acc = 0;
      }
    }
  }
}

// End of a COO tile [b0, tile_end): partial sums carried between the tile's
// threads, the held-back first row ends, and the row left open at the tile's
// end handed to the fix-up as (carry_row, carry_val)[tile].
template <typename T, int NT, int MODE>
__device__ __forceinline__ void coo_finish(long long tile_end, T acc, int first_row, T first_acc,
                                           const Epi<T, MODE> &ep, T *__restrict__ y, long long nnz,
                                           const int32_t *__restrict__ row, int32_t *carry_row, T *carry_val,
                                           long long tile) {
  T tile_open = 0;
  const T incoming = tile_carries<T, NT>(first_row >= 0, acc, &tile_open);
  if (first_row >= 0) y[first_row] = ep(incoming + first_acc, y, (long long)first_row);
  if (threadIdx.x == NT - 1) {
    // the row open at the end of the tile continues into the next tile
    const long long kl = tile_end - 1;
    const bool open = kl + 1 < nnz && __ldg(row + kl + 1) == __ldg(row + kl);
    carry_row[tile] = open ? __ldg(row + kl) : -1;
    carry_val[tile] = open ? tile_open : (T)0;
  }
}

// K12: COO.  A CTA owns NT*CH*8 consecutive stored entries; thread t owns
// CH*8 consecutive ones, read 8 at a time with 16-byte vector loads, and
// accumulates them with one fused multiply-add each.  A row ends at entry k
// when row[k+1] differs.  CH chunks per thread amortise the tile's fixed work
// (carry resolution, barriers) over more entries.
#ifndef SMAT_COO_MINB
#define SMAT_COO_MINB 1
#endif
template <typename V, typename T, int NT, int CH, int MODE>
__device__ __forceinline__ void coo_tile(const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                                         const V *__restrict__ val, const T *__restrict__ x, const Epi<T, MODE> &ep,
                                         T *__restrict__ y, long long nnz, int32_t *carry_row, T *carry_val,
                                         long long tile) {
  constexpr int IPT = 8, TILE = NT * CH * IPT;
  const long long b0 = tile * TILE;
  const long long kt = b0 + (long long)threadIdx.x * (CH * IPT);
  T acc = 0, first_acc = 0;
  int first_row = -1;
#ifdef SMAT_COO_UNROLL
#pragma unroll
#else
#pragma unroll 1
#endif
  for (int ch = 0; ch < CH; ++ch) {
    const long long k0 = kt + ch * IPT;
    const int valid = k0 >= nnz ? 0 : (int)min((long long)IPT, nnz - k0);
    if (CH == 1 && sizeof(V) == 8) {
      // FP64: the row after this thread's entries is the next lane's first
      // row (a lane past the end holds -1), so only lane 31 loads it: one L2
      // sector request fewer per thread on a kernel bound by their rate
      // (power-law SPLIT 176 -> 166.5 us).  The column and value loads go
      // first so the gathers do not wait for the shuffle.  In FP32 the
      // shuffle costs 8 registers (48 -> 56) and was 2-7 % slower.  Every
      // lane reaches the shuffle before any leaves.
      const bool full = valid == IPT;
      int r[IPT], c[IPT];
      T v[IPT];
      load_i32_run<IPT>(col + k0, full, valid, c, 0);
      load_val_run<V, IPT>(val + k0, full, valid, v);
      load_i32_run<IPT>(row + k0, full, valid, r, -1);
      int r_next = __shfl_down_sync(FULL, r[0], 1);
      if ((threadIdx.x & 31) == 31) r_next = (k0 + IPT < nnz) ? __ldg(row + k0 + IPT) : -1;
      if (valid == 0) break;
      coo_chunk<T, IPT, MODE>(r, c, v, r_next, valid, x, ep, y, acc, first_row, first_acc);
      continue;
    }
    if (valid == 0) break;
    const bool full = valid == IPT;
    int r[IPT], c[IPT];
    T v[IPT];
    load_i32_run<IPT>(row + k0, full, valid, r, -1);
    load_i32_run<IPT>(col + k0, full, valid, c, 0);
    load_val_run<V, IPT>(val + k0, full, valid, v);
    const int r_next = (k0 + IPT < nnz) ? __ldg(row + k0 + IPT) : -1;
    coo_chunk<T, IPT, MODE>(r, c, v, r_next, valid, x, ep, y, acc, first_row, first_acc);
  }
  coo_finish<T, NT, MODE>(min(b0 + TILE, nnz), acc, first_row, first_acc, ep, y, nnz, row, carry_row, carry_val,
                          tile);
}

template <typename V, typename T, int NT, int CH, int MODE>
__global__ void __launch_bounds__(NT, SMAT_COO_MINB) coo_kernel(const int32_t *__restrict__ row,
                                                                const int32_t *__restrict__ col,
                                                                const V *__restrict__ val, const T *__restrict__ x,
                                                                Epi<T, MODE> ep, T *__restrict__ y, long long nnz,
                                                                int32_t *carry_row, T *carry_val) {
  griddep_wait();
  coo_tile<V, T, NT, CH, MODE>(row, col, val, x, ep, y, nnz, carry_row, carry_val, blockIdx.x);
}

// COO launch shape (sweep knobs; these defaults measured fastest)
#ifndef SMAT_COO_NT
#define SMAT_COO_NT 256
#endif
#ifndef SMAT_COO_CH
#define SMAT_COO_CH 1
#endif
constexpr int COO_NT = SMAT_COO_NT, COO_CH = SMAT_COO_CH, COO_IPT = 8 * SMAT_COO_CH;
// SPLIT's short rows in tiles of one warp (32 threads x 8 entries) whose
// carries are resolved with shuffles alone, or (0) in the COO kernel's
// 256-thread tiles with a block-wide carry scan.
#ifndef SMAT_SPLIT_WARP_TILES
#define SMAT_SPLIT_WARP_TILES 1
#endif
constexpr bool SPLIT_WARP_TILES = SMAT_SPLIT_WARP_TILES != 0;
constexpr long long SPLIT_TILE = SPLIT_WARP_TILES ? 32LL * 8 : (long long)COO_NT * COO_IPT;
// The same choice for COO products (and HYB's COO tail).
#ifndef SMAT_COO_WARP_TILES
#define SMAT_COO_WARP_TILES 1
#endif
constexpr bool COO_WARP_TILES = SMAT_COO_WARP_TILES != 0;
constexpr long long COO_TILE = COO_WARP_TILES ? 32LL * 8 : (long long)COO_NT * COO_IPT;

// ---------------------------------------------------------------------------
// SPLIT, long rows (at least SPLIT_L = 1024 entries; measured on power-law
// matrices against 128 and 256, where rows of a few hundred entries paid a
// whole CTA's reduction for little work): one CTA of 256 threads per chunk of
// at most 4096 entries of one row.  Thread t takes entries first + t + 256 j (j < 16), so every
// column and value load is a contiguous warp access; one fused multiply-add
// per entry; the 256 partial sums are added in a fixed order (warp butterfly,
// then the 8 warp sums in turn) into part[chunk].  No row ends inside a
// chunk, so there is no segmented scan: a tile of a long row costs one plain
// block sum instead of the COO tile's carry resolution.
// ---------------------------------------------------------------------------
template <typename V, typename T>
__device__ __forceinline__ void split_chunk(long long c, const int32_t *__restrict__ cstart,
                                            const int32_t *__restrict__ cend, const int32_t *__restrict__ col,
                                            const V *__restrict__ val, const T *__restrict__ x,
                                            T *__restrict__ part) {
  __shared__ T s_w[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k0 = __ldg(cstart + c), k1 = __ldg(cend + c);
  T acc = 0;
  // steps j of 256 entries past the chunk's end are skipped by the whole
  // CTA (a uniform test), so short chunks issue only the work they hold
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    if (k0 + 256 * 8 * b >= k1) break;
    int cc[8];
    T v[8], xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + (int)threadIdx.x + 256 * (8 * b + q);
      const bool on = k < k1;
      cc[q] = on ? ld_idx(col + k) : -1;
      v[q] = on ? (T)ld_val(val + k) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) xv[q] = cc[q] >= 0 ? __ldg(x + cc[q]) : (T)0;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (k0 + 256 * (8 * b + q) < k1) acc = fused(acc, v[q], xv[q]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc = add_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if (lane == 0) s_w[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = s_w[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) t = add_rn(t, s_w[k]);
    part[c] = t;
  }
}

// SPLIT in one grid: blocks [0, nc) reduce the chunks of the long rows,
// blocks [nc, nc + tiles) are COO tiles of the short rows (the two sets
// write disjoint rows).  One launch instead of two keeps the GPU full across
// what was the boundary between them.
// Within one warp whose 32 lanes' chunks form a tile: the inclusive
// segmented sum of the lanes' open partial sums c, segments starting at the
// lanes where a row ended (their c opens the next row).  A lane with a row
// end gets the sum at the lane before it: the partials of the row its first
// row end closes.  *open is the sum at lane 31, the row left open at the
// tile's end.  Shuffles only; fixed order.
template <typename T>
__device__ __forceinline__ T warp_carries(bool h, T c, T *open) {
  const int lane = threadIdx.x & 31;
  int f = h ? 1 : 0;
  T v = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T vu = __shfl_up_sync(FULL, v, o);
    const int fu = __shfl_up_sync(FULL, f, o);
    if (lane >= o) {
      if (!f) v = vu + v;
      f |= fu;
    }
  }
  *open = __shfl_sync(FULL, v, 31);
  const T prev = __shfl_up_sync(FULL, v, 1);
  return lane == 0 ? (T)0 : prev;
}

// A COO tile of one warp: lane l owns the 8 stored entries at b0 + 8 l; rows
// ending inside a lane's entries are written as in the block tiles, the
// first one after the warp's carries, and the row open at the tile's end is
// handed to the fix-up as (carry_row, carry_val)[tile].
template <typename V, typename T, int MODE>
__device__ __forceinline__ void coo_warp_tile(const int32_t *__restrict__ row, const int32_t *__restrict__ col,
                                              const V *__restrict__ val, const T *__restrict__ x,
                                              const Epi<T, MODE> &ep, T *__restrict__ y, long long nnz,
                                              int32_t *carry_row, T *carry_val, long long tile) {
  constexpr int IPT = 8;
  const int lane = threadIdx.x & 31;
  const long long b0 = tile * (32LL * IPT);
  if (b0 >= nnz) return;  // the whole warp
  const long long k0 = b0 + (long long)lane * IPT;
  const int valid = k0 >= nnz ? 0 : (int)min((long long)IPT, nnz - k0);
  const bool full = valid == IPT;
  int r[IPT], c[IPT];
  T v[IPT];
  load_i32_run<IPT>(col + k0, full, valid, c, 0);
  load_val_run<V, IPT>(val + k0, full, valid, v);
  load_i32_run<IPT>(row + k0, full, valid, r, -1);
  // the row after a lane's entries is the next lane's first row (a lane past
  // the end holds -1); lane 31 loads it
  int r_next = __shfl_down_sync(FULL, r[0], 1);
  if (lane == 31) r_next = (k0 + IPT < nnz) ? __ldg(row + k0 + IPT) : -1;
  T acc = 0, first_acc = 0;
  int first_row = -1;
  if (valid > 0) coo_chunk<T, IPT, MODE>(r, c, v, r_next, valid, x, ep, y, acc, first_row, first_acc);
  T open;
  const T incoming = warp_carries<T>(first_row >= 0, acc, &open);
  if (first_row >= 0) y[first_row] = ep(incoming + first_acc, y, (long long)first_row);
  if (lane == 31) {
    const long long kl = min(b0 + 32LL * IPT, nnz) - 1;
    const bool opn = kl + 1 < nnz && __ldg(row + kl + 1) == __ldg(row + kl);
    carry_row[tile] = opn ? __ldg(row + kl) : -1;
    carry_val[tile] = opn ? open : (T)0;
  }
}

// COO products in warp tiles (coo_warp_tile), 8 tiles per 256-thread CTA.
template <typename V, typename T, int MODE>
__global__ void __launch_bounds__(COO_NT, SMAT_COO_MINB) coo_warp_kernel(const int32_t *__restrict__ row,
                                                                     const int32_t *__restrict__ col,
                                                                     const V *__restrict__ val,
                                                                     const T *__restrict__ x, Epi<T, MODE> ep,
                                                                     T *__restrict__ y, long long nnz,
                                                                     int32_t *carry_row, T *carry_val) {
  griddep_wait();
  coo_warp_tile<V, T, MODE>(row, col, val, x, ep, y, nnz, carry_row, carry_val,
                            (long long)blockIdx.x * (COO_NT / 32) + (threadIdx.x >> 5));
}

template <typename V, typename T, int MODE>
__global__ void __launch_bounds__(COO_NT, SMAT_COO_MINB) split_main_kernel(
    const int32_t *__restrict__ cstart, const int32_t *__restrict__ cend, const int32_t *__restrict__ col,
    const V *__restrict__ val, T *__restrict__ part, long long nc, const int32_t *__restrict__ srow,
    const int32_t *__restrict__ scol, const V *__restrict__ sval, long long ns, const T *__restrict__ x,
    Epi<T, MODE> ep, T *__restrict__ y, int32_t *carry_row, T *carry_val) {
  griddep_wait();
  static_assert(COO_NT == 256, "the chunk path assumes 256 threads");
  if ((long long)blockIdx.x < nc)
    split_chunk<V, T>(blockIdx.x, cstart, cend, col, val, x, part);
  else if (SPLIT_WARP_TILES)
    coo_warp_tile<V, T, MODE>(srow, scol, sval, x, ep, y, ns, carry_row, carry_val,
                              ((long long)blockIdx.x - nc) * (COO_NT / 32) + (threadIdx.x >> 5));
  else
    coo_tile<V, T, COO_NT, COO_CH, MODE>(srow, scol, sval, x, ep, y, ns, carry_row, carry_val,
                                         (long long)blockIdx.x - nc);
}

// A long row: its chunk sums added in chunk order, then the epilogue.
template <typename T, int MODE>
__device__ __forceinline__ void split_row(long long l, const int32_t *__restrict__ lrows,
                                          const int32_t *__restrict__ lchunk, const T *__restrict__ part,
                                          const Epi<T, MODE> &ep, T *__restrict__ y) {
  const int c0 = lchunk[l], c1 = lchunk[l + 1];
  T t = part[c0];
  for (int c = c0 + 1; c < c1; ++c) t = add_rn(t, part[c]);
  const long long r = lrows[l];
  y[r] = ep(t, y, r);
}

// Fix-up: y[r] += alpha * (sum of the carries of row r), runs of equal rows
// summed in tile order by the run's first entry.
template <typename T, int MODE>
__device__ __forceinline__ void carry_fixup(long long c, const int32_t *__restrict__ carry_row,
                                            const T *__restrict__ carry_val, long long ntiles,
                                            const Epi<T, MODE> &ep, T *__restrict__ y) {
  const int r = carry_row[c];
  if (r < 0 || (c > 0 && carry_row[c - 1] == r)) return;
  T s = carry_val[c];
  for (long long q = c + 1; q < ntiles && carry_row[q] == r; ++q) s = add_rn(s, carry_val[q]);
  y[r] = add_rn(y[r], MODE == EPI_COPY ? s : mul_rn(ep.alpha, s));
}

template <typename T, int MODE>
__global__ void carry_fixup_kernel(const int32_t *__restrict__ carry_row, const T *__restrict__ carry_val,
                                   long long ntiles, Epi<T, MODE> ep, T *__restrict__ y) {
  griddep_wait();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ntiles;
       c += (long long)gridDim.x * blockDim.x)
    carry_fixup<T, MODE>(c, carry_row, carry_val, ntiles, ep, y);
}

// SPLIT's closing pass over three disjoint sets of rows: the long rows
// (chunk sums, epilogue), the carries of the short rows' COO tiles, and the
// empty rows (y = beta y, or 0).
template <typename T, int MODE>
__global__ void split_finish_kernel(const int32_t *__restrict__ lrows, const int32_t *__restrict__ lchunk,
                                    const T *__restrict__ part, long long nl, const int32_t *__restrict__ carry_row,
                                    const T *__restrict__ carry_val, long long ntiles,
                                    const int32_t *__restrict__ empty, long long ne, Epi<T, MODE> ep,
                                    T *__restrict__ y) {
  griddep_wait();
  const long long total = nl + ntiles + ne;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    if (i < nl) {
      split_row<T, MODE>(i, lrows, lchunk, part, ep, y);
    } else if (i < nl + ntiles) {
      carry_fixup<T, MODE>(i - nl, carry_row, carry_val, ntiles, ep, y);
    } else {
      const int r = empty[i - nl - ntiles];
      y[r] = MODE == EPI_AXPBY ? mul_rn(ep.beta, y[r]) : (T)0;
    }
  }
}

template <typename T, int MODE>
__global__ void scale_rows_kernel(const int32_t *__restrict__ rows, long long count, Epi<T, MODE> ep,
                                  T *__restrict__ y) {
  griddep_wait();
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < count;
       c += (long long)gridDim.x * blockDim.x) {
    int r = rows[c];
    y[r] = MODE == EPI_AXPBY ? mul_rn(ep.beta, y[r]) : (T)0;
  }
}

// ---------------------------------------------------------------------------
// K10: ELL, column-major, R consecutive rows per thread so that every slot is
// one 16-byte load of values (and 4R bytes of columns).  U slots are loaded
// before their gathers are issued (U*R = 8 gathers in flight per thread);
// padding (column -1) gathers x[0] and is dropped by a select, so no load
// sits behind a branch.
// ---------------------------------------------------------------------------
template <typename V, int R, int MODE, int U, bool LANE>
__global__ void __launch_bounds__(256) ell_kernel(const int32_t *__restrict__ ecol, const V *__restrict__ eval,
                                                  long long P, long long K,
                                                  const typename Compute<V>::T *__restrict__ x,
                                                  Epi<typename Compute<V>::T, MODE> ep,
                                                  typename Compute<V>::T *__restrict__ y, long long m) {
  griddep_wait();
  if (LANE) {  // lane-striped rows (a per-handle measured choice)
    const long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32LL * R);
    if (base < m) ell_lane_group<V, R, MODE, U>(ecol, eval, P, K, x, ep, y, m, base, threadIdx.x & 31);
  } else {
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R;
    if (i0 < m) ell_group<V, R, MODE, U>(ecol, eval, P, K, x, ep, y, m, i0);
  }
}

// ---------------------------------------------------------------------------
// K11: DIA, diagonal-major, R consecutive rows per thread, offsets staged in
// shared memory, U diagonals loaded per step.  Fill zeros are multiplied like
// stored values (Table "Performance features of the four formats": extra
// computation decided by zero filling); positions whose column falls outside
// the matrix gather x[0] and are dropped by a select.
// ---------------------------------------------------------------------------
template <typename V, int R, int MODE, int U>
__global__ void __launch_bounds__(256) dia_kernel(const int32_t *__restrict__ off, int nd,
                                                  const V *__restrict__ dval, long long P,
                                                  const typename Compute<V>::T *__restrict__ x,
                                                  Epi<typename Compute<V>::T, MODE> ep,
                                                  typename Compute<V>::T *__restrict__ y, long long m,
                                                  long long n) {
  griddep_wait();
  extern __shared__ int32_t s_off[];
  for (int t = threadIdx.x; t < nd; t += blockDim.x) s_off[t] = off[t];
  __syncthreads();
  if (sizeof(V) == 8) {  // FP64: lane-striped rows (measured faster on every matrix tried)
    const long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32LL * R);
    if (base < m) dia_lane_group<V, R, MODE, U>(s_off, nd, dval, P, x, ep, y, m, n, base, threadIdx.x & 31);
  } else {
    const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R;
    if (i0 < m) dia_group<V, R, MODE, U>(s_off, nd, dval, P, x, ep, y, m, n, i0);
  }
}

int grid_for(long long work, int block, int max_blocks) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

constexpr int MERGE_NT = 256, MERGE_IPT = 8;
// A COO product over (row, col, val) of length nnz, then the carry fix-up.
template <typename V, typename T, int MODE>
cudaError_t launch_coo(const Scratch &sc, const int32_t *row, const int32_t *col, const V *val, const T *x,
                       const Epi<T, MODE> &ep, T *y, long long nnz, cudaStream_t s) {
  const long long tiles = (nnz + COO_TILE - 1) / COO_TILE;
  int32_t *crow = (int32_t *)sc.carry;
  T *cval = (T *)((char *)sc.carry + ((tiles * 4 + 15) / 16) * 16);
  if (COO_WARP_TILES)
    (void)launch_pdl(coo_warp_kernel<V, T, MODE>, dim3((unsigned)((tiles + COO_NT / 32 - 1) / (COO_NT / 32))), dim3(COO_NT), 0,
        s, row, col, val, x, ep, y, nnz, crow, cval);
  else
    (void)launch_pdl(coo_kernel<V, T, COO_NT, COO_CH, MODE>, dim3((unsigned)tiles), dim3(COO_NT), 0, s, row, col, val, x, ep, y, nnz, crow, cval);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (tiles > 1) (void)launch_pdl(carry_fixup_kernel<T, MODE>, dim3(grid_for(tiles, 256, 152 * 8)), dim3(256), 0, s, crow, cval, tiles, ep, y);
  return cudaGetLastError();
}

// ELL / DIA launches with a batch width U chosen at run time from 1..16/R.
// The ELL arrays are passed in: the handle's ELL format, or HYB's ELL part.
struct EllPart {
  const int32_t *col;
  const void *val;
  long long K;
};

template <typename V, int MODE, int U>
void launch_ell_u(const smat_s *h, const EllPart &e, bool lane, const typename Compute<V>::T *x,
                  const Epi<typename Compute<V>::T, MODE> &ep, typename Compute<V>::T *y, cudaStream_t s) {
  constexpr int R = 16 / (int)sizeof(V);
  const long long m = h->m;
  const int g = grid_for((m + R - 1) / R, 256, 1 << 30);
  if (lane)
    (void)launch_pdl(ell_kernel<V, R, MODE, U, true>, dim3(g), dim3(256), 0, s, e.col, (const V *)e.val, h->P, e.K, x, ep, y, m);
  else
    (void)launch_pdl(ell_kernel<V, R, MODE, U, false>, dim3(g), dim3(256), 0, s, e.col, (const V *)e.val, h->P, e.K, x, ep, y, m);
}

template <typename V, int MODE, int U>
void launch_dia_u(const smat_s *h, const typename Compute<V>::T *x, const Epi<typename Compute<V>::T, MODE> &ep,
                  typename Compute<V>::T *y, cudaStream_t s) {
  constexpr int R = 16 / (int)sizeof(V);
  const long long m = h->m;
  (void)launch_pdl(dia_kernel<V, R, MODE, U>, dim3(grid_for((m + R - 1) / R, 256, 1 << 30)), dim3(256), (size_t)h->dia_nd * 4, s,
      h->dia_off, (int)h->dia_nd, (const V *)h->dia_val, h->P, x, ep, y, m, h->n);
}

template <typename V, int MODE, bool DIA>
void launch_ell_dia(const smat_s *h, const typename Compute<V>::T *x, const Epi<typename Compute<V>::T, MODE> &ep,
                    typename Compute<V>::T *y, cudaStream_t s, int u_req, int lane_req,
                    const EllPart *part = nullptr) {
  constexpr int UMAX = 16 / (16 / (int)sizeof(V));  // 16 / R
  const EllPart e = part ? *part : EllPart{h->ell_col, h->ell_val, h->ell_K};
  const bool lane = lane_req >= 0 ? lane_req != 0 : (part ? false : h->ell_lane != 0);
  const int u_tuned = part ? 0 : (DIA ? h->dia_u : h->ell_u);
  const int u = u_req > 0 ? u_req : (u_tuned > 0 ? u_tuned : batch_width(DIA ? h->dia_nd : e.K, UMAX));
#define SMAT_UCASE(k)                                                      \
  case k:                                                                  \
    if constexpr (k <= UMAX) {                                             \
      if (DIA) launch_dia_u<V, MODE, k>(h, x, ep, y, s);                   \
      else launch_ell_u<V, MODE, k>(h, e, lane, x, ep, y, s);              \
    }                                                                      \
    break;
  switch (u) {
    SMAT_UCASE(1) SMAT_UCASE(2) SMAT_UCASE(3) SMAT_UCASE(4) SMAT_UCASE(5) SMAT_UCASE(6) SMAT_UCASE(7)
    default:
      if constexpr (UMAX >= 8) {
        if (DIA) launch_dia_u<V, MODE, 8>(h, x, ep, y, s);
        else launch_ell_u<V, MODE, 8>(h, e, lane, x, ep, y, s);
      }
      break;
  }
#undef SMAT_UCASE
}

template <typename V, int MODE>
cudaError_t spmv_mode(const smat_s *h, const Scratch &sc, int variant, typename Compute<V>::T alpha, const void *x_p,
                      typename Compute<V>::T beta, void *y_p, cudaStream_t s, int u_req, int lane_req) {
  typedef typename Compute<V>::T T;
  const Epi<T, MODE> ep{alpha, beta};
  const T *x = (const T *)x_p;
  T *y = (T *)y_p;
  const V *val = (const V *)h->val;
  const long long m = h->m;
  switch (variant) {
    case SMAT_V_CSR_SCALAR:
      (void)launch_pdl(csr_scalar_kernel<V, T, false, MODE>, dim3(grid_for(m, 256, 1 << 20)), dim3(256), 0, s, h->rowptr, h->colidx, val, x,
                                                                                     Epi<T, MODE, false>{alpha, beta}, y, m);
      break;
    case SMAT_V_CSR_SCALAR_EXACT:
      (void)launch_pdl(csr_scalar_kernel<V, T, true, MODE>, dim3(grid_for(m, 256, 1 << 20)), dim3(256), 0, s, h->rowptr, h->colidx, val, x,
                                                                                    Epi<T, MODE, true>{alpha, beta}, y, m);
      break;
    case SMAT_V_CSR_VEC4:
      (void)launch_pdl(csr_vector_kernel<V, T, 4, MODE>, dim3(grid_for(m * 4, 256, 1 << 20)), dim3(256), 0, s, h->rowptr, h->colidx, val, x, ep, y, m);
      break;
    case SMAT_V_CSR_VEC8:
      (void)launch_pdl(csr_vector_kernel<V, T, 8, MODE>, dim3(grid_for(m * 8, 256, 1 << 20)), dim3(256), 0, s, h->rowptr, h->colidx, val, x, ep, y, m);
      break;
    case SMAT_V_CSR_VEC32:
      (void)launch_pdl(csr_vector_kernel<V, T, 32, MODE>, dim3(grid_for(m * 32, 256, 1 << 20)), dim3(256), 0, s, h->rowptr, h->colidx, val, x, ep, y, m);
      break;
    case SMAT_V_CSR_MERGE: {
      long long tiles = (m + h->nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT);
      int32_t *crow = (int32_t *)sc.carry;
      T *cval = (T *)((char *)sc.carry + ((tiles * 4 + 15) / 16) * 16);
      (void)launch_pdl(csr_merge_kernel<V, T, MERGE_NT, MERGE_IPT, MODE>, dim3((unsigned)tiles), dim3(MERGE_NT), 0, s,
          h->rowptr, h->colidx, val, x, ep, y, m, h->nnz, (const int2 *)h->merge_coords, crow, cval);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      if (tiles > 1)
        (void)launch_pdl(carry_fixup_kernel<T, MODE>, dim3(grid_for(tiles, 256, 152 * 8)), dim3(256), 0, s, crow, cval, tiles, ep, y);
    } break;
    case SMAT_V_ELL:
      launch_ell_dia<V, MODE, false>(h, x, ep, y, s, u_req, lane_req);
      break;
    case SMAT_V_DIA:
      if (lane_req >= 2 || (lane_req < 0 && h->dia_staged))
        return launch_dia_staged(h, lane_req >= 2 ? lane_req - 1 : h->dia_staged, &alpha, x, &beta, y, s);
      launch_ell_dia<V, MODE, true>(h, x, ep, y, s, u_req, lane_req);
      break;
    case SMAT_V_COO: {
      if (h->coo_nempty > 0) {
        (void)launch_pdl(scale_rows_kernel<T, MODE>, dim3(grid_for(h->coo_nempty, 256, 152 * 8)), dim3(256), 0, s, h->coo_empty, h->coo_nempty,
                                                                                          ep, y);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      if (h->nnz == 0) break;
      return launch_coo<V, T, MODE>(sc, h->coo_row, h->colidx, val, x, ep, y, h->nnz, s);
    }
    case SMAT_V_HYB: {
      // the ELL part writes every row (y = alpha*part + beta*y), then the COO
      // tail adds alpha*(its sums): y = alpha*acc + 1*y
      const EllPart part{h->hyb_ecol, h->hyb_eval, h->hyb_K};
      launch_ell_dia<V, MODE, false>(h, x, ep, y, s, 0, 0, &part);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess || h->hyb_ncoo == 0) return e;
      const Epi<T, EPI_AXPBY> add{alpha, (T)1};
      return launch_coo<V, T, EPI_AXPBY>(sc, h->hyb_crow, h->hyb_ccol, (const V *)h->hyb_cval, x, add, y,
                                         h->hyb_ncoo, s);
    }
    case SMAT_V_SPLIT: {
      // two launches: the chunks of the long rows and the COO tiles of the
      // short ones in one grid, then one pass for the long rows' sums, the
      // tiles' carries and the empty rows
      const long long nc = h->split_nc, ns = h->split_ns;
      const long long tiles = (ns + SPLIT_TILE - 1) / SPLIT_TILE;
      const long long tile_ctas = SPLIT_WARP_TILES ? (tiles + COO_NT / 32 - 1) / (COO_NT / 32) : tiles;
      int32_t *crow = (int32_t *)sc.carry;
      T *cval = (T *)((char *)sc.carry + ((tiles * 4 + 15) / 16) * 16);
      if (nc + tile_ctas > 0) {
        (void)launch_pdl(split_main_kernel<V, T, MODE>, dim3((unsigned)(nc + tile_ctas)), dim3(COO_NT), 0, s,
            h->split_cstart, h->split_cend, h->colidx, val, (T *)sc.part, nc, h->split_srow, h->split_scol,
            (const V *)h->split_sval, ns, x, ep, y, crow, cval);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
      }
      const long long nl = nc > 0 ? h->split_nl : 0, nt = tiles > 1 ? tiles : 0;
      if (nl + nt + h->split_ne > 0)
        (void)launch_pdl(split_finish_kernel<T, MODE>, dim3(grid_for(nl + nt + h->split_ne, 256, 152 * 8)), dim3(256), 0, s,
            h->split_lrows, h->split_lchunk, (const T *)sc.part, nl, crow, cval, nt, h->split_empty, h->split_ne, ep,
            y);
    } break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename V>
cudaError_t spmv_typed(const smat_s *h, const Scratch &sc, int variant, const void *alpha_p, const void *x_p,
                       const void *beta_p, void *y_p, cudaStream_t s, int u_req, int lane_req) {
  typedef typename Compute<V>::T T;
  const T alpha = *(const T *)alpha_p, beta = *(const T *)beta_p;
  if (h->m == 0) return cudaSuccess;
  switch (epi_mode((double)alpha, (double)beta)) {
    case EPI_COPY: return spmv_mode<V, EPI_COPY>(h, sc, variant, alpha, x_p, beta, y_p, s, u_req, lane_req);
    case EPI_SCALE: return spmv_mode<V, EPI_SCALE>(h, sc, variant, alpha, x_p, beta, y_p, s, u_req, lane_req);
    default: return spmv_mode<V, EPI_AXPBY>(h, sc, variant, alpha, x_p, beta, y_p, s, u_req, lane_req);
  }
}

}  // namespace

long long merge_tiles(long long m, long long nnz) { return (m + nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT); }

cudaError_t launch_merge_partition(const int32_t *rowptr, long long m, long long nnz, void *coords, cudaStream_t s) {
  const long long tiles = merge_tiles(m, nnz);
  merge_partition_kernel<<<grid_for(tiles + 1, 256, 152 * 8), 256, 0, s>>>(rowptr, m, nnz, MERGE_NT * MERGE_IPT,
                                                                          tiles, (int2 *)coords);
  return cudaGetLastError();
}

size_t carry_bytes_needed(const smat_s *h, int variant) {
  long long tiles = 0;
  if (variant == SMAT_V_CSR_MERGE) tiles = (h->m + h->nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT);
  else if (variant == SMAT_V_COO) tiles = (h->nnz + COO_TILE - 1) / COO_TILE;
  else if (variant == SMAT_V_HYB) tiles = (h->hyb_ncoo + COO_TILE - 1) / COO_TILE;
  else if (variant == SMAT_V_SPLIT) tiles = (h->split_ns + SPLIT_TILE - 1) / SPLIT_TILE;
  else return 0;
  size_t tsz = h->dtype == SMAT_F64 ? 8 : 4;
  return (size_t)((tiles * 4 + 15) / 16) * 16 + (size_t)tiles * tsz;
}

int spmv_launch_count(const smat_s *h, int variant) {
  if (h->m == 0) return 0;
  if (variant == SMAT_V_CSR_MERGE) {
    long long tiles = (h->m + h->nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT);
    return 1 + (tiles > 1);
  }
  if (variant == SMAT_V_COO) {
    long long tiles = (h->nnz + COO_TILE - 1) / COO_TILE;
    return (h->coo_nempty > 0) + (h->nnz > 0) + (tiles > 1);
  }
  if (variant == SMAT_V_HYB) {
    long long tiles = (h->hyb_ncoo + COO_TILE - 1) / COO_TILE;
    return 1 + (h->hyb_ncoo > 0) + (tiles > 1);
  }
  if (variant == SMAT_V_SPLIT) {  // the main grid, then the closing pass when it has rows to do
    const long long tiles = (h->split_ns + SPLIT_TILE - 1) / SPLIT_TILE;
    const long long nl = h->split_nc > 0 ? h->split_nl : 0, nt = tiles > 1 ? tiles : 0;
    return (h->split_nc + tiles > 0) + (nl + nt + h->split_ne > 0);
  }
  if (variant == SMAT_V_SELL) return h->sell_ns > 0;
  if (variant == SMAT_V_BCSR) return h->bcsr_mb > 0;
  return 1;
}

// alpha == 0: y = beta*y (0 when beta == 0) without reading A or x, so that
// non-finite values in x cannot reach y (the BLAS convention).
template <typename T>
__global__ void beta_only_kernel(T *__restrict__ y, long long m, T beta) {
  griddep_wait();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    y[i] = mul_rn(beta, y[i]);
}

template <typename T>
cudaError_t beta_only(const smat_s *h, const void *beta_p, void *y, cudaStream_t s) {
  const T beta = *(const T *)beta_p;
  if (h->m == 0) return cudaSuccess;
  if (beta == (T)0) return cudaMemsetAsync(y, 0, (size_t)h->m * sizeof(T), s);
  (void)launch_pdl(beta_only_kernel<T>, dim3(grid_for(h->m, 256, 152 * 8)), dim3(256), 0, s, (T *)y, h->m, beta);
  return cudaGetLastError();
}

cudaError_t launch_spmv(const smat_s *h, int variant, const void *alpha, const void *x, const void *beta,
                        void *y, cudaStream_t s, bool claim) {
  if (h->dtype == SMAT_F64 ? *(const double *)alpha == 0.0 : *(const float *)alpha == 0.0f)
    return h->dtype == SMAT_F64 ? beta_only<double>(h, beta, y, s) : beta_only<float>(h, beta, y, s);
  // ELL, DIA and HYB read x and write y, and BCSR reads x, with vector
  // accesses of up to 16 bytes; vectors that are not 16-byte aligned take the
  // CSR-scalar kernel instead.
  if ((variant == SMAT_V_ELL || variant == SMAT_V_DIA || variant == SMAT_V_HYB || variant == SMAT_V_BCSR) &&
      (((uintptr_t)x | (uintptr_t)y) & 15u) != 0)
    variant = SMAT_V_CSR_SCALAR;
  if (variant == SMAT_V_SELL || variant == SMAT_V_BCSR) return launch_spmv_ext(h, variant, alpha, x, beta, y, s);
  Scratch sc{nullptr, nullptr};
  if (carry_bytes_needed(h, variant) > 0 || variant == SMAT_V_SPLIT) {
    cudaError_t e = stream_scratch(h, s, &sc, claim);
    if (e != cudaSuccess) return e;
  }
  switch (h->dtype) {
    case SMAT_F64: return spmv_typed<double>(h, sc, variant, alpha, x, beta, y, s, 0, -1);
    case SMAT_F32: return spmv_typed<float>(h, sc, variant, alpha, x, beta, y, s, 0, -1);
    default: return spmv_typed<__nv_bfloat16>(h, sc, variant, alpha, x, beta, y, s, 0, -1);
  }
}

int batch_width_candidates(const smat_s *h, int variant, int out[2]) {
  const int umax = 16 / (16 / elem_size(h->dtype));
  const long long count = variant == SMAT_V_DIA ? h->dia_nd : h->ell_K;
  out[0] = umax;                      // full width (dead slots when count < umax)
  out[1] = batch_width(count, umax);  // fewest dead slots
  return out[1] != out[0] ? 2 : 1;
}

cudaError_t launch_spmv_width(const smat_s *h, int variant, int u, int lane, const void *alpha, const void *x,
                              const void *beta, void *y, cudaStream_t s) {
  const Scratch none{nullptr, nullptr};  // ELL / DIA use no scratch
  switch (h->dtype) {
    case SMAT_F64: return spmv_typed<double>(h, none, variant, alpha, x, beta, y, s, u, lane);
    case SMAT_F32: return spmv_typed<float>(h, none, variant, alpha, x, beta, y, s, u, lane);
    default: return spmv_typed<__nv_bfloat16>(h, none, variant, alpha, x, beta, y, s, u, lane);
  }
}

}  // namespace smat

// ---------------------------------------------------------------------------
// Merge-path CSR SpMV that allocates nothing.
//
// Some callers cannot call cudaMalloc: a solver that runs under a memory
// manager owning every device byte, code that must not synchronise the device
// (cudaMalloc/cudaFree may), or a host whose allocation calls are forbidden
// once its time-critical loop has started.  For them this entry point keeps
// the only scratch the kernel needs -- one carry (row, partial sum) per tile
// -- in a fixed array in the library's own device memory.  Every GPU that
// loads the library holds that array (1.25 MiB) until the process exits.
// The array's address is looked up once per device, on the first call made
// with that device current; make that first call before any stream capture.
// All calls share the array, so calls whose kernels overlap on the GPU race:
// order them on one stream, or synchronise between them.  Nothing in the
// array has to start at zero: each call writes every carry and tile
// coordinate it later reads.
// ---------------------------------------------------------------------------
#include <mutex>

namespace smat {
namespace {

// The array holds three regions, for at most 65,536 tiles of 2048 merge items:
constexpr long long NOALLOC_MAX_TILES = 65536;
// [0, 256 KiB): each tile's carry row, int32
constexpr size_t NOALLOC_ROW_BYTES = NOALLOC_MAX_TILES * 4;
// [256 KiB, 768 KiB): each tile's carry value, 8 bytes (FP64) or 4 (FP32)
constexpr size_t NOALLOC_VAL_BYTES = NOALLOC_MAX_TILES * 8;
// [768 KiB, 1.25 MiB + 8 B): the merge-path coordinate (row, entry) of each
// of the tiles + 1 tile boundaries, int2
constexpr size_t NOALLOC_COORD_OFFSET = NOALLOC_ROW_BYTES + NOALLOC_VAL_BYTES;
constexpr size_t NOALLOC_BYTES = NOALLOC_COORD_OFFSET + (NOALLOC_MAX_TILES + 1) * 8;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array for the current device, looked up on
// the first call with that device current and kept for the process's life:
// after cudaDeviceReset the kept address is stale, so this entry point must
// not be called again in a process that has reset a device it used.
cudaError_t noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

template <typename V, int MODE>
cudaError_t merge_noalloc_mode(long long m, long long nnz, const int32_t *rowptr, const int32_t *colidx,
                               const void *vals, typename Compute<V>::T alpha, const void *x_p,
                               typename Compute<V>::T beta, void *y_p, unsigned char *scratch, cudaStream_t s) {
  typedef typename Compute<V>::T T;
  const Epi<T, MODE> ep{alpha, beta};
  const long long tiles = (m + nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT);
  int32_t *crow = (int32_t *)scratch;
  T *cval = (T *)(scratch + NOALLOC_ROW_BYTES);
  int2 *coords = (int2 *)(scratch + NOALLOC_COORD_OFFSET);
  cudaError_t e = launch_merge_partition(rowptr, m, nnz, coords, s);
  if (e != cudaSuccess) return e;
  csr_merge_kernel<V, T, MERGE_NT, MERGE_IPT, MODE><<<(unsigned)tiles, MERGE_NT, 0, s>>>(
      rowptr, colidx, (const V *)vals, (const T *)x_p, ep, (T *)y_p, m, nnz, coords, crow, cval);
  e = cudaGetLastError();
  if (e != cudaSuccess || tiles <= 1) return e;
  carry_fixup_kernel<T, MODE><<<grid_for(tiles, 256, 152 * 8), 256, 0, s>>>(crow, cval, tiles, ep, (T *)y_p);
  return cudaGetLastError();
}

template <typename V>
cudaError_t merge_noalloc_typed(long long m, long long nnz, const int32_t *rowptr, const int32_t *colidx,
                                const void *vals, const void *alpha_p, const void *x_p, const void *beta_p,
                                void *y_p, unsigned char *scratch, cudaStream_t s) {
  typedef typename Compute<V>::T T;
  const T alpha = *(const T *)alpha_p, beta = *(const T *)beta_p;
  // alpha == 0: y = beta*y (0 when beta == 0), reading neither A nor x, as in
  // smat_spmv, so that non-finite values in x cannot reach y
  if (alpha == (T)0) {
    if (beta == (T)0) return cudaMemsetAsync(y_p, 0, (size_t)m * sizeof(T), s);
    beta_only_kernel<T><<<grid_for(m, 256, 152 * 8), 256, 0, s>>>((T *)y_p, m, beta);
    return cudaGetLastError();
  }
  switch (epi_mode((double)alpha, (double)beta)) {
    case EPI_COPY: return merge_noalloc_mode<V, EPI_COPY>(m, nnz, rowptr, colidx, vals, alpha, x_p, beta, y_p, scratch, s);
    case EPI_SCALE: return merge_noalloc_mode<V, EPI_SCALE>(m, nnz, rowptr, colidx, vals, alpha, x_p, beta, y_p, scratch, s);
    default: return merge_noalloc_mode<V, EPI_AXPBY>(m, nnz, rowptr, colidx, vals, alpha, x_p, beta, y_p, scratch, s);
  }
}

}  // namespace
}  // namespace smat

extern "C" smat_status_t smat_spmv_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                                                     const int32_t *colidx, const void *vals, smat_dtype_t dtype,
                                                     const void *alpha, const void *x, const void *beta, void *y,
                                                     void *stream) {
  using namespace smat;
  if (m < 0 || n < 0 || nnz < 0 || !alpha || !beta) return SMAT_ERR_INVALID_ARG;
  if (dtype != SMAT_F64 && dtype != SMAT_F32 && dtype != SMAT_BF16) return SMAT_ERR_INVALID_ARG;
  if (m == 0) return SMAT_OK;
  if (!rowptr || !y || (nnz > 0 && (!colidx || !vals || !x))) return SMAT_ERR_INVALID_ARG;
  if (m > INT32_MAX - 1 || n > INT32_MAX || nnz > INT32_MAX) return SMAT_ERR_UNSUPPORTED;
  const long long tiles = (m + nnz + MERGE_NT * MERGE_IPT - 1) / (MERGE_NT * MERGE_IPT);
  if (tiles > NOALLOC_MAX_TILES) return SMAT_ERR_UNSUPPORTED;  // beyond the fixed scratch
  void *scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return SMAT_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *sc = (unsigned char *)scratch;
  switch (dtype) {
    case SMAT_F64: e = merge_noalloc_typed<double>(m, nnz, rowptr, colidx, vals, alpha, x, beta, y, sc, s); break;
    case SMAT_F32: e = merge_noalloc_typed<float>(m, nnz, rowptr, colidx, vals, alpha, x, beta, y, sc, s); break;
    default: e = merge_noalloc_typed<__nv_bfloat16>(m, nnz, rowptr, colidx, vals, alpha, x, beta, y, sc, s); break;
  }
  return e == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}
