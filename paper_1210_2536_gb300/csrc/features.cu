// CSR validation and feature extraction on the GPU (arXiv 1210.2536, Sec. 4,
// Table "Feature parameters of a sparse matrix").
//
// Everything here is integer work over rowptr and colidx, so the results are
// exact and independent of scheduling:
//   row_stats   : max_RD, min_RD, sum rd^2, empty rows      (one read of rowptr)
//   hist_diag   : row-degree histogram h[k] and the count of stored entries on
//                 every diagonal d = j - i                  (one read of colidx)
//   diag_reduce : Ndiags, number of "true" diagonals and the occupied offsets
// The floating-point features are finished on the host from these integers.
#include <algorithm>
#include <climits>

#include "smat_internal.h"

namespace smat {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int warp_max(int v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
__device__ __forceinline__ int warp_min(int v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Row containing flattened nonzero k, given each lane's row start (lanes past
// the group hold INT_MAX): the largest lane L with start_L <= k.
__device__ __forceinline__ int row_lane_of(int start_of_my_row, long long k) {
  int L = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    int cand = L + step;
    int sc = __shfl_sync(FULL, start_of_my_row, cand & 31);
    if (cand < 32 && (long long)sc <= k) L = cand;
  }
  return L;
}

// ---------------------------------------------------------------------------
// K1: validation, in two balanced passes.  Per row: the row pointer must not
// fall, and the row's first entry is marked in a bitmap over the stored
// entries.  Per entry (4 per thread, one 16-byte load): the column must lie
// in [0, n), and must be below the next entry's unless a row starts there.
// Work is spread by rows and by entries, so a few very long rows do not hold
// one warp while the others idle.  Every index read is clamped into the
// arrays, so malformed input cannot send either pass out of bounds.
// ---------------------------------------------------------------------------
__global__ void validate_rows_kernel(const int32_t *__restrict__ rowptr, long long m, long long nnz,
                                     unsigned *__restrict__ starts, int *flag) {
  int err = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (rowptr[0] != 0 || (long long)rowptr[m] != nnz)) err |= ERRF_ROWPTR;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (long long)gridDim.x * blockDim.x) {
    const long long s = rowptr[r], e = rowptr[r + 1];
    if (e < s) err |= ERRF_ROWPTR;
    if (s >= 0 && s < nnz) atomicOr(&starts[s >> 5], 1u << (s & 31));
  }
  err = __reduce_or_sync(FULL, err);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(flag, err);
}

__global__ void validate_cols_kernel(const int32_t *__restrict__ col, long long nnz, long long n,
                                     const unsigned *__restrict__ starts, int *flag) {
  int err = 0;
  const long long chunks = (nnz + 3) / 4;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < chunks;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k0 = 4 * t;
    int c[5];
    if (k0 + 4 <= nnz) {
      const int4 v = __ldcs(reinterpret_cast<const int4 *>(col) + t);
      c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) c[i] = k0 + i < nnz ? col[k0 + i] : 0;
    }
    c[4] = k0 + 4 < nnz ? __ldg(col + k0 + 4) : 0;
    // entries k0 + 1 .. k0 + 4 sit in word k0 >> 5, or k0 + 4 in the next one
    const unsigned w0 = starts[k0 >> 5];
    const unsigned w1 = ((k0 + 4) & 31) == 0 ? starts[(k0 + 4) >> 5] : w0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const long long k = k0 + i;
      if (k >= nnz) break;
      if (c[i] < 0 || (long long)c[i] >= n) err |= ERRF_COL_RANGE;
      const long long k1 = k + 1;
      if (k1 < nnz) {
        const unsigned w = (k1 >> 5) == (k0 >> 5) ? w0 : w1;
        if (!((w >> (k1 & 31)) & 1u) && c[i + 1] <= c[i]) err |= ERRF_COL_ORDER;
      }
    }
  }
  err = __reduce_or_sync(FULL, err);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(flag, err);
}

// ---------------------------------------------------------------------------
// K2a: integer statistics of the row degrees.
// ---------------------------------------------------------------------------
__global__ void row_stats_kernel(const int32_t *__restrict__ rowptr, long long m, RowStats *out) {
  unsigned long long s2 = 0;
  int mx = 0, mn = INT_MAX, emp = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    int rd = rowptr[i + 1] - rowptr[i];
    s2 += (unsigned long long)rd * (unsigned long long)rd;
    mx = max(mx, rd);
    mn = min(mn, rd);
    emp += (rd == 0);
  }
  s2 = warp_sum(s2);
  mx = warp_max(mx);
  mn = warp_min(mn);
  emp = warp_sum(emp);
  __shared__ unsigned long long sh_s2[32];
  __shared__ int sh_mx[32], sh_mn[32], sh_emp[32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh_s2[w] = s2; sh_mx[w] = mx; sh_mn[w] = mn; sh_emp[w] = emp; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    s2 = lane < nw ? sh_s2[lane] : 0;
    mx = lane < nw ? sh_mx[lane] : 0;
    mn = lane < nw ? sh_mn[lane] : INT_MAX;
    emp = lane < nw ? sh_emp[lane] : 0;
    s2 = warp_sum(s2);
    mx = warp_max(mx);
    mn = warp_min(mn);
    emp = warp_sum(emp);
    if (lane == 0) {
      if (s2) atomicAdd(&out->s2, s2);
      atomicMax(&out->max_rd, mx);
      atomicMin(&out->min_rd, mn);
      if (emp) atomicAdd(&out->empty_rows, emp);
    }
  }
}

// ---------------------------------------------------------------------------
// K2b + K3: row-degree histogram and per-diagonal counts in one pass.
// A warp owns 32 consecutive rows and walks their nonzeros as one contiguous,
// coalesced range.  Counts are aggregated first across the warp
// (__match_any_sync), then in a per-CTA shared hash table; only the table's
// final entries (or overflow) reach global memory.  Banded matrices thus
// issue a handful of global atomics per CTA instead of one per nonzero.
// ---------------------------------------------------------------------------
constexpr int HT = 2048;           // hash slots per CTA
constexpr int HT_PROBES = 8;
constexpr int HIST_SH = 1024;      // privatised histogram bins
constexpr int EMPTY_KEY = INT_MIN;

// Adds c to diagonal d's count in the CTA's table; when its probes find no
// slot, to the global count, and marks the table full so that the CTA's
// later entries go to the global counts directly (random-column matrices).
__device__ __forceinline__ void ht_add(int *keys, int *cnts, int *g_cnt, long long m, int d, int c, int *full) {
  unsigned h = ((unsigned)d * 2654435761u) >> (32 - 11);
#pragma unroll 1
  for (int p = 0; p < HT_PROBES; ++p) {
    int prev = atomicCAS(&keys[h], EMPTY_KEY, d);
    if (prev == EMPTY_KEY || prev == d) {
      atomicAdd(&cnts[h], c);
      return;
    }
    h = (h + 1) & (HT - 1);
  }
  *full = 1;
  atomicAdd(&g_cnt[(long long)d + m - 1], c);
}

__global__ void __launch_bounds__(256) hist_diag_kernel(const int32_t *__restrict__ rowptr,
                                                        const int32_t *__restrict__ col, long long m,
                                                        int *hist, long long hist_len, int *g_cnt) {
  __shared__ int keys[HT], cnts[HT], sh_hist[HIST_SH];
  __shared__ int ht_full;
  if (threadIdx.x == 0) ht_full = 0;
  for (int t = threadIdx.x; t < HT; t += blockDim.x) { keys[t] = EMPTY_KEY; cnts[t] = 0; }
  for (int t = threadIdx.x; t < HIST_SH; t += blockDim.x) sh_hist[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r0 = warp * 32; r0 < m; r0 += nwarps * 32) {
    long long r = r0 + lane;
    int s = INT_MAX, e = 0;
    if (r < m) { s = rowptr[r]; e = rowptr[r + 1]; }
    // histogram of row degrees
    {
      int rd = e - s;
      bool small = (r < m) && rd < HIST_SH;
      unsigned act = __ballot_sync(FULL, small);
      if (small) {
        unsigned peers = __match_any_sync(act, rd);
        if (lane == __ffs(peers) - 1) atomicAdd(&sh_hist[rd], __popc(peers));
      } else if (r < m) {
        atomicAdd(&hist[rd], 1);
      }
    }
    int rows = (int)min(32LL, m - r0);
    long long gs = __shfl_sync(FULL, s, 0);
    long long ge = __shfl_sync(FULL, e, rows - 1);
    for (long long base = gs; base < ge; base += 32) {
      long long k = base + lane;
      bool active = k < ge;
      int L = row_lane_of(s, k);
      // one decision for the whole warp (lane 0's view of the flag)
      const int full = __shfl_sync(FULL, *(volatile int *)&ht_full, 0);
      if (full) {
        if (active) atomicAdd(&g_cnt[(long long)(col[k] - (int)(r0 + L)) + m - 1], 1);
        continue;
      }
      unsigned act = __ballot_sync(FULL, active);
      if (active) {
        int d = col[k] - (int)(r0 + L);
        unsigned peers = __match_any_sync(act, d);
        if (lane == __ffs(peers) - 1) ht_add(keys, cnts, g_cnt, m, d, __popc(peers), &ht_full);
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < HT; t += blockDim.x)
    if (keys[t] != EMPTY_KEY) atomicAdd(&g_cnt[(long long)keys[t] + m - 1], cnts[t]);
  for (int t = threadIdx.x; t < HIST_SH && t < hist_len; t += blockDim.x)
    if (sh_hist[t]) atomicAdd(&hist[t], sh_hist[t]);
}

// ---------------------------------------------------------------------------
// K3b: occupied / "true" diagonals, plus the occupied offsets (unordered; the
// host sorts them) up to `cap` of them.  counts = {Ndiags, Ntrue, appended};
// "appended" is exact while it stays at most cap, and otherwise only ends
// above cap.
// ---------------------------------------------------------------------------
__global__ void diag_reduce_kernel(const int *__restrict__ cnt, long long m, long long n, int tau_num,
                                   int tau_den, unsigned long long *counts, int32_t *offsets,
                                   long long cap) {
  long long nd = m + n - 1;
  unsigned long long occ = 0, tru = 0;
  const int lane = threadIdx.x & 31;
  // the trip count is the same for the whole warp, so the ballot below sees
  // every lane: one append per warp and pass instead of one per diagonal
  for (long long base = (long long)blockIdx.x * blockDim.x; base < nd; base += (long long)gridDim.x * blockDim.x) {
    const long long t = base + threadIdx.x;
    const int c = t < nd ? cnt[t] : 0;
    const long long d = t - (m - 1);
    if (c > 0) {
      long long len = d >= 0 ? min(m, n - d) : min(m + d, n);
      ++occ;
      if ((long long)tau_den * c > (long long)tau_num * len) ++tru;
    }
    const unsigned b = __ballot_sync(FULL, c > 0);
    if (b) {
      // once the count seen is above cap the host drops the offsets anyway
      // (it keeps them only when the final count is at most cap), so later
      // warps stop appending; the count still ends above cap
      const int leader = __ffs(b) - 1;
      unsigned long long idx0 = 0;
      int skip = 0;
      if (lane == leader) {
        if (*(volatile unsigned long long *)&counts[2] > (unsigned long long)cap) skip = 1;
        else idx0 = atomicAdd(&counts[2], (unsigned long long)__popc(b));
      }
      skip = __shfl_sync(FULL, skip, leader);
      idx0 = __shfl_sync(FULL, idx0, leader);
      if (!skip && c > 0) {
        const unsigned long long idx = idx0 + __popc(b & ((1u << lane) - 1u));
        if ((long long)idx < cap) offsets[idx] = (int32_t)d;
      }
    }
  }
  occ = warp_sum(occ);
  tru = warp_sum(tru);
  if ((threadIdx.x & 31) == 0) {
    if (occ) atomicAdd(&counts[0], occ);
    if (tru) atomicAdd(&counts[1], tru);
  }
}

int grid_for(long long work, int block, int max_blocks) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

}  // namespace

size_t validate_starts_words(int64_t nnz) { return (size_t)(nnz / 32 + 2); }

cudaError_t launch_validate(const smat_s *h, int *d_flag, unsigned *d_starts, cudaStream_t s) {
  validate_rows_kernel<<<grid_for(std::max<int64_t>(h->m, 1), 256, 152 * 16), 256, 0, s>>>(h->rowptr, h->m, h->nnz,
                                                                                          d_starts, d_flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || h->nnz == 0) return e;
  validate_cols_kernel<<<grid_for((h->nnz + 3) / 4, 256, 152 * 16), 256, 0, s>>>(h->colidx, h->nnz, h->n, d_starts,
                                                                               d_flag);
  return cudaGetLastError();
}

cudaError_t launch_row_stats(const int32_t *rowptr, int64_t m, RowStats *d_stats, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int g = grid_for(m, 256, 152 * 8);
  row_stats_kernel<<<g, 256, 0, s>>>(rowptr, m, d_stats);
  return cudaGetLastError();
}

cudaError_t launch_hist_diag(const int32_t *rowptr, const int32_t *colidx, int64_t m, int *d_hist,
                             int64_t hist_len, int *d_diag_cnt, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  int g = grid_for((m + 31) / 32 * 32, 256, 152 * 8);
  hist_diag_kernel<<<g, 256, 0, s>>>(rowptr, colidx, m, d_hist, hist_len, d_diag_cnt);
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const int *d_diag_cnt, int64_t m, int64_t n, int tau_num, int tau_den,
                               unsigned long long *d_counts, int32_t *d_offsets, int64_t cap,
                               cudaStream_t s) {
  if (m + n - 1 <= 0) return cudaSuccess;
  int g = grid_for(m + n - 1, 256, 152 * 8);
  diag_reduce_kernel<<<g, 256, 0, s>>>(d_diag_cnt, m, n, tau_num, tau_den, d_counts, d_offsets, cap);
  return cudaGetLastError();
}

}  // namespace smat
