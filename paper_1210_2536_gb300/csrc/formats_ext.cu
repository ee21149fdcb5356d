// Further GPU storage formats: HYB (Bell & Garland, 2009), SELL-C-sigma
// (Kreutzer, Hager, Wellein, Fehske & Bishop, 2014), BCSR with b x b blocks
// (register blocking, Im & Yelick) and SPLIT (long rows in chunks, the rest as
// COO).  arXiv 1210.2536 works with DIA, ELL, CSR and COO (Sec. 2.1) and leaves
// more formats to future work (Sec. 8); these join the same execute-and-measure
// search (Sec. 6).  This file holds their conversions and the SELL and BCSR
// kernels; HYB and SPLIT run through kernels of spmv.cu.
//
// Layouts (the oracle builds the same arrays element for element):
//   HYB   ELL part ecol/eval[s*P + i] for s < K (slots past a row's length:
//         column -1, value +0; rows M..P-1 likewise), then a COO part
//         (row, col, val) of every row's entries past its first K, in CSR
//         order.  K = the largest k with 3 * #{rows with >= k entries} >= M.
//   SELL  C = 32 rows per slice.  perm[p] = the row at sorted position p:
//         rows sorted by decreasing length inside windows of sigma rows
//         (equal lengths keep row order), -1 for positions M..Mp-1 (Mp = M
//         rounded up to 32).  width[s] = longest length in slice s;
//         sptr[s] = sum of 32 * width over earlier slices; entry j of the row
//         at position 32s + l is slot sptr[s] + 32j + l (col -1 / +0 past
//         the row's length).
//   BCSR  browptr[ceil(M/b) + 1]; bcol[k] ascending within a block row;
//         bval[k*b*b + r*b + c] = a(I*b + r, bcol[k]*b + c), +0 where nothing
//         is stored (also past the matrix edge).
//   SPLIT rows of >= SPLIT_L (1024) entries ("long", listed ascending) cut into
//         chunks of <= SPLIT_CK entries (row, first, end entry per chunk, a
//         long row's chunks consecutive); the other non-empty rows' entries
//         as a COO in CSR order; empty rows listed.
#include <algorithm>
#include <climits>

#include "smat_internal.h"
#include "spmv_device.cuh"

namespace smat {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SELL_C = 32;
#ifndef SMAT_SELL_U
#define SMAT_SELL_U 8
#endif
constexpr int SELL_U = SMAT_SELL_U;  // slots loaded before their gathers

template <int B> struct Raw;
template <> struct Raw<8> { typedef unsigned long long T; };
template <> struct Raw<4> { typedef unsigned int T; };
template <> struct Raw<2> { typedef unsigned short T; };

int grid_for(long long work, int block, int max_blocks) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Exclusive scan of n int64 counts into out[0..n] (out[n] = total), in three
// passes: tile sums, a scan of the tile sums in one block, tile scans.
// ---------------------------------------------------------------------------
constexpr int SCAN_NT = 256, SCAN_IPT = 8, SCAN_TILE = SCAN_NT * SCAN_IPT;

// Exclusive scan of one value per thread over the block; *total gets the sum.
__device__ long long block_exclusive(long long v, long long *total) {
  __shared__ long long s_w[SCAN_NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long p = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += p;
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  long long before = 0, all = 0;
  for (int k = 0; k < SCAN_NT / 32; ++k) {
    if (k < w) before += s_w[k];
    all += s_w[k];
  }
  __syncthreads();
  *total = all;
  return before + inc - v;
}

__global__ void scan_tile_sums(const long long *__restrict__ in, long long n, long long *__restrict__ sums) {
  const long long b0 = (long long)blockIdx.x * SCAN_TILE;
  long long v = 0;
  for (int q = 0; q < SCAN_IPT; ++q) {
    const long long i = b0 + threadIdx.x + (long long)q * SCAN_NT;
    if (i < n) v += in[i];
  }
  long long total;
  block_exclusive(v, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_tile_offsets(long long *sums, long long ntiles) {
  long long carry = 0;
  for (long long c0 = 0; c0 < ntiles; c0 += SCAN_NT) {
    const long long i = c0 + threadIdx.x;
    const long long v = i < ntiles ? sums[i] : 0;
    long long total;
    const long long ex = block_exclusive(v, &total);
    if (i < ntiles) sums[i] = carry + ex;
    carry += total;
  }
}

__global__ void scan_tiles(const long long *__restrict__ in, long long n, const long long *__restrict__ offs,
                           long long *__restrict__ out) {
  const long long t0 = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_IPT;
  long long v[SCAN_IPT], sum = 0;
  for (int q = 0; q < SCAN_IPT; ++q) {
    v[q] = t0 + q < n ? in[t0 + q] : 0;
    sum += v[q];
  }
  long long total;
  long long run = offs[blockIdx.x] + block_exclusive(sum, &total);
  for (int q = 0; q < SCAN_IPT; ++q) {
    if (t0 + q < n) out[t0 + q] = run;
    if (t0 + q == n - 1) out[n] = run + v[q];
    run += v[q];
  }
}

// ---------------------------------------------------------------------------
// HYB
// ---------------------------------------------------------------------------
__global__ void hyb_tail_counts(const int32_t *__restrict__ rowptr, long long m, long long K,
                                long long *__restrict__ cnt) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const long long rd = rowptr[i + 1] - rowptr[i];
    cnt[i] = rd > K ? rd - K : 0;
  }
}

template <typename B>
__global__ void to_hyb_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const B *__restrict__ val, long long m, long long P, long long K,
                              const long long *__restrict__ off, int32_t *__restrict__ ecol, B *__restrict__ eval,
                              int32_t *__restrict__ crow, int32_t *__restrict__ ccol, B *__restrict__ cval) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (long long)gridDim.x * blockDim.x) {
    long long s = 0, rd = 0;
    if (i < m) { s = rowptr[i]; rd = rowptr[i + 1] - s; }
    for (long long q = 0; q < K; ++q) {
      const long long pos = q * P + i;
      const bool on = q < rd;
      ecol[pos] = on ? col[s + q] : -1;
      eval[pos] = on ? val[s + q] : (B)0;
    }
    if (i < m)
      for (long long q = K; q < rd; ++q) {
        const long long o = off[i] + q - K;
        crow[o] = (int32_t)i;
        ccol[o] = col[s + q];
        cval[o] = val[s + q];
      }
  }
}

// ---------------------------------------------------------------------------
// SELL-C-sigma
// ---------------------------------------------------------------------------
// One block per window: each row's sorted position is the number of rows in
// its window that are longer, or as long and earlier.
__global__ void sell_sort_kernel(const int32_t *__restrict__ rowptr, long long m, int sigma, int32_t *__restrict__ perm) {
  extern __shared__ int s_len[];
  const long long w0 = (long long)blockIdx.x * sigma;
  const int cnt = (int)(m - w0 < sigma ? m - w0 : sigma);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) s_len[q] = rowptr[w0 + q + 1] - rowptr[w0 + q];
  __syncthreads();
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    const int lq = s_len[q];
    int rank = 0;
    for (int t = 0; t < cnt; ++t) {
      const int lt = s_len[t];
      rank += (lt > lq) || (lt == lq && t < q);
    }
    perm[w0 + rank] = (int32_t)(w0 + q);
  }
}

// A warp per slice: its width (the longest row) and 32 * width slots; marks
// the pad positions past M.
__global__ void sell_width_kernel(const int32_t *__restrict__ rowptr, long long m, long long mp, int32_t *perm,
                                  int32_t *__restrict__ width, long long *__restrict__ cnt) {
  const long long stride = (long long)gridDim.x * blockDim.x;  // a multiple of 32
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < mp; p += stride) {
    int len = 0;
    if (p < m) {
      const int r = perm[p];
      len = rowptr[r + 1] - rowptr[r];
    } else {
      perm[p] = -1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) len = max(len, __shfl_xor_sync(FULL, len, o));
    if ((threadIdx.x & 31) == 0) {
      width[p / SELL_C] = len;
      cnt[p / SELL_C] = (long long)SELL_C * len;
    }
  }
}

template <typename B>
__global__ void to_sell_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const B *__restrict__ val, long long mp, const int32_t *__restrict__ perm,
                               const int32_t *__restrict__ width, const long long *__restrict__ sptr,
                               int32_t *__restrict__ scol, B *__restrict__ sval) {
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < mp; p += (long long)gridDim.x * blockDim.x) {
    const long long sl = p / SELL_C;
    const int r = perm[p];
    long long k0 = 0, len = 0;
    if (r >= 0) { k0 = rowptr[r]; len = rowptr[r + 1] - k0; }
    const long long base = sptr[sl] + (p % SELL_C);
    const int w = width[sl];
    for (int j = 0; j < w; ++j) {
      const long long slot = base + (long long)j * SELL_C;
      const bool on = j < len;
      scol[slot] = on ? col[k0 + j] : -1;
      sval[slot] = on ? val[k0 + j] : (B)0;
    }
  }
}

// ---------------------------------------------------------------------------
// BCSR
// ---------------------------------------------------------------------------
// Thread per block row: a merge of its (up to) b sorted rows, counting the
// distinct block columns.
template <int BS>
__global__ void bcsr_count_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col, long long m,
                                  long long mb, long long *__restrict__ cnt) {
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < mb; I += (long long)gridDim.x * blockDim.x) {
    int p[BS], e[BS];
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      const long long i = I * BS + r;
      p[r] = i < m ? rowptr[i] : 0;
      e[r] = i < m ? rowptr[i + 1] : 0;
    }
    long long c = 0;
    while (true) {
      unsigned jmin = UINT_MAX;
#pragma unroll
      for (int r = 0; r < BS; ++r)
        if (p[r] < e[r]) jmin = min(jmin, (unsigned)col[p[r]] / BS);
      if (jmin == UINT_MAX) break;
      ++c;
#pragma unroll
      for (int r = 0; r < BS; ++r)
        while (p[r] < e[r] && (unsigned)col[p[r]] / BS == jmin) ++p[r];
    }
    cnt[I] = c;
  }
}

template <int BS, typename B>
__global__ void to_bcsr_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const B *__restrict__ val, long long m, long long mb, const long long *__restrict__ brp,
                               int32_t *__restrict__ browptr, int32_t *__restrict__ bcol, B *__restrict__ bval) {
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < mb; I += (long long)gridDim.x * blockDim.x) {
    const long long k0 = brp[I];
    browptr[I] = (int32_t)k0;
    if (I == mb - 1) browptr[mb] = (int32_t)brp[mb];
    int p[BS], e[BS];
#pragma unroll
    for (int r = 0; r < BS; ++r) {
      const long long i = I * BS + r;
      p[r] = i < m ? rowptr[i] : 0;
      e[r] = i < m ? rowptr[i + 1] : 0;
    }
    long long k = k0;
    while (true) {  // the block columns, ascending; their blocks zeroed
      unsigned jmin = UINT_MAX;
#pragma unroll
      for (int r = 0; r < BS; ++r)
        if (p[r] < e[r]) jmin = min(jmin, (unsigned)col[p[r]] / BS);
      if (jmin == UINT_MAX) break;
      bcol[k] = (int32_t)jmin;
      for (int q = 0; q < BS * BS; ++q) bval[k * BS * BS + q] = (B)0;
      ++k;
#pragma unroll
      for (int r = 0; r < BS; ++r)
        while (p[r] < e[r] && (unsigned)col[p[r]] / BS == jmin) ++p[r];
    }
    for (int r = 0; r < BS; ++r) {  // scatter each row's entries into its blocks
      const long long i = I * BS + r;
      if (i >= m) break;
      long long kb = k0;
      for (long long q = rowptr[i]; q < rowptr[i + 1]; ++q) {
        const int J = col[q] / BS;
        while (bcol[kb] < J) ++kb;
        bval[kb * BS * BS + r * BS + (col[q] - J * BS)] = val[q];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// SPLIT: per-row counts, then each row's entries to their place
// ---------------------------------------------------------------------------
__global__ void split_counts_kernel(const int32_t *__restrict__ rowptr, long long m, long long *__restrict__ cl,
                                    long long *__restrict__ cc, long long *__restrict__ cs,
                                    long long *__restrict__ ce) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const long long rd = rowptr[i + 1] - rowptr[i];
    const bool lng = rd >= SPLIT_L;
    cl[i] = lng;
    cc[i] = lng ? (rd + SPLIT_CK - 1) / SPLIT_CK : 0;
    cs[i] = (!lng && rd > 0) ? rd : 0;
    ce[i] = rd == 0;
  }
}

template <typename B>
__global__ void split_fill_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                  const B *__restrict__ val, long long m, const long long *__restrict__ pl,
                                  const long long *__restrict__ pc, const long long *__restrict__ ps,
                                  const long long *__restrict__ pe, int32_t *__restrict__ lrows,
                                  int32_t *__restrict__ lchunk, int32_t *__restrict__ crow, int32_t *__restrict__ cstart,
                                  int32_t *__restrict__ cend, int32_t *__restrict__ srow, int32_t *__restrict__ scol,
                                  B *__restrict__ sval, int32_t *__restrict__ empty) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const long long s0 = rowptr[i], e0 = rowptr[i + 1], rd = e0 - s0;
    if (rd == 0) {
      empty[pe[i]] = (int32_t)i;
    } else if (rd >= SPLIT_L) {
      const long long l = pl[i];
      lrows[l] = (int32_t)i;
      lchunk[l] = (int32_t)pc[i];
      long long c = pc[i];
      for (long long k = s0; k < e0; k += SPLIT_CK, ++c) {
        crow[c] = (int32_t)i;
        cstart[c] = (int32_t)k;
        cend[c] = (int32_t)(k + SPLIT_CK < e0 ? k + SPLIT_CK : e0);
      }
    } else {
      long long o = ps[i];
      for (long long k = s0; k < e0; ++k, ++o) {
        srow[o] = (int32_t)i;
        scol[o] = col[k];
        sval[o] = val[k];
      }
    }
    if (i == 0) lchunk[pl[m]] = (int32_t)pc[m];  // one past the last long row
  }
}

// ---------------------------------------------------------------------------
// SELL SpMV: a warp per slice (sell_slice), a lane per row.
// ---------------------------------------------------------------------------
template <typename V, int MODE, int U>
__global__ void __launch_bounds__(256) sell_kernel(const long long *__restrict__ sptr, const int32_t *__restrict__ width,
                                                   const int32_t *__restrict__ perm, const int32_t *__restrict__ scol,
                                                   const V *__restrict__ sval, const typename Compute<V>::T *__restrict__ x,
                                                   Epi<typename Compute<V>::T, MODE> ep,
                                                   typename Compute<V>::T *__restrict__ y, long long ns) {
  griddep_wait();
  const long long sl = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / SELL_C;
  if (sl >= ns) return;
  sell_slice<V, MODE, U>(sptr, width, perm, scol, sval, x, ep, y, sl, threadIdx.x & 31);
}

// ---------------------------------------------------------------------------
// BCSR SpMV: BS consecutive lanes per block row, lane r computing row r of
// it; each block contributes one vector load of the lane's BS values and one
// of x[J*BS .. J*BS + BS) (shared by the BS lanes).
// ---------------------------------------------------------------------------
template <typename V, int BS>
__device__ __forceinline__ void load_block_row(const V *p, typename Compute<V>::T (&o)[BS]) {
  constexpr int BYTES = BS * (int)sizeof(V);
  if constexpr (sizeof(V) == 8) {
#pragma unroll
    for (int q = 0; q < BS / 2; ++q) {
      const double2 d = __ldcs(reinterpret_cast<const double2 *>(p) + q);
      o[2 * q] = d.x;
      o[2 * q + 1] = d.y;
    }
  } else if constexpr (sizeof(V) == 4) {
    if constexpr (BYTES == 8) {
      const float2 f = __ldcs(reinterpret_cast<const float2 *>(p));
      o[0] = f.x;
      o[1] = f.y;
    } else {
#pragma unroll
      for (int q = 0; q < BS / 4; ++q) {
        const float4 f = __ldcs(reinterpret_cast<const float4 *>(p) + q);
        o[4 * q] = f.x; o[4 * q + 1] = f.y; o[4 * q + 2] = f.z; o[4 * q + 3] = f.w;
      }
    }
  } else {  // bfloat16: widen by placing the 16 bits on top of an FP32 word
    unsigned w[BS / 2];
    if constexpr (BYTES == 4) {
      w[0] = __ldcs(reinterpret_cast<const unsigned *>(p));
    } else if constexpr (BYTES == 8) {
      const uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
      w[0] = u.x; w[1] = u.y;
    } else {
      const uint4 u = __ldcs(reinterpret_cast<const uint4 *>(p));
      w[0] = u.x; w[1] = u.y; w[2] = u.z; w[3] = u.w;
    }
#pragma unroll
    for (int q = 0; q < BS / 2; ++q) {
      o[2 * q] = __uint_as_float(w[q] << 16);
      o[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
  }
}

template <typename T, int BS>
__device__ __forceinline__ void load_x_block(const T *__restrict__ x, long long j0, long long n, T (&o)[BS]) {
  if (j0 + BS <= n) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int q = 0; q < BS / 2; ++q) {
        const double2 d = __ldg(reinterpret_cast<const double2 *>(x + j0) + q);
        o[2 * q] = d.x;
        o[2 * q + 1] = d.y;
      }
    } else if constexpr (BS == 2) {
      const float2 f = __ldg(reinterpret_cast<const float2 *>(x + j0));
      o[0] = f.x;
      o[1] = f.y;
    } else {
#pragma unroll
      for (int q = 0; q < BS / 4; ++q) {
        const float4 f = __ldg(reinterpret_cast<const float4 *>(x + j0) + q);
        o[4 * q] = f.x; o[4 * q + 1] = f.y; o[4 * q + 2] = f.z; o[4 * q + 3] = f.w;
      }
    }
  } else {  // the last block column may reach past column n - 1 (zero fill there)
#pragma unroll
    for (int c = 0; c < BS; ++c) o[c] = j0 + c < n ? __ldg(x + j0 + c) : (T)0;
  }
}

#ifndef SMAT_BCSR_R2
#define SMAT_BCSR_R2 1
#endif
constexpr int BCSR_R2 = SMAT_BCSR_R2;  // block rows per lane group

// R2 consecutive block rows per group of BS lanes, stepped together so that
// the loads of all R2 blocks of a step are in flight at once.  Measured on
// GB300 (block-diagonal 8x8, 7-point, uniform; FP64 and FP32): R2 = 1 is
// fastest, the extra registers of R2 = 2 or 4 cost more occupancy than the
// loads in flight gain.  When every block row holds the same number cb of
// blocks, block row I's blocks are I*cb ... I*cb + cb - 1 and the block-row
// pointers are not read: the value loads start at once and x waits for one
// load (the block column) instead of two.
template <typename V, int BS, int R2, int MODE>
__global__ void __launch_bounds__(256) bcsr_kernel(const int32_t *__restrict__ browptr, const int32_t *__restrict__ bcol,
                                                   const V *__restrict__ bval, const typename Compute<V>::T *__restrict__ x,
                                                   Epi<typename Compute<V>::T, MODE> ep,
                                                   typename Compute<V>::T *__restrict__ y, long long m, long long n,
                                                   long long mb, int cb) {
  griddep_wait();
  typedef typename Compute<V>::T T;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long I0 = gid / BS * R2;
  const int r = (int)(gid % BS);
  if (I0 >= mb) return;
  int k[R2], kend[R2], steps = 0;
#pragma unroll
  for (int q = 0; q < R2; ++q) {
    const bool in = I0 + q < mb;
    if (cb > 0) {
      k[q] = in ? (int)((I0 + q) * cb) : 0;
      kend[q] = in ? k[q] + cb : 0;
    } else {
      k[q] = in ? __ldg(browptr + I0 + q) : 0;
      kend[q] = in ? __ldg(browptr + I0 + q + 1) : 0;
    }
    steps = max(steps, kend[q] - k[q]);
  }
  T acc[R2];
#pragma unroll
  for (int q = 0; q < R2; ++q) acc[q] = 0;
  for (int t = 0; t < steps; ++t) {
    T a[R2][BS], xv[R2][BS];
#pragma unroll
    for (int q = 0; q < R2; ++q) {
      if (k[q] + t < kend[q]) {
        const long long kk = k[q] + t;
        const long long J = ld_idx(bcol + kk);
        load_block_row<V, BS>(bval + (kk * BS + r) * BS, a[q]);
        load_x_block<T, BS>(x, J * BS, n, xv[q]);
      } else {
#pragma unroll
        for (int c = 0; c < BS; ++c) a[q][c] = xv[q][c] = (T)0;
      }
    }
#pragma unroll
    for (int q = 0; q < R2; ++q)
#pragma unroll
      for (int c = 0; c < BS; ++c) acc[q] = fused(acc[q], a[q][c], xv[q][c]);
  }
#pragma unroll
  for (int q = 0; q < R2; ++q) {
    const long long row = (I0 + q) * BS + r;
    if (row < m) y[row] = ep(acc[q], y, row);
  }
}

template <typename V, int MODE>
cudaError_t ext_mode(const smat_s *h, int variant, typename Compute<V>::T alpha, const void *x_p,
                     typename Compute<V>::T beta, void *y_p, cudaStream_t s) {
  typedef typename Compute<V>::T T;
  const Epi<T, MODE> ep{alpha, beta};
  const T *x = (const T *)x_p;
  T *y = (T *)y_p;
  if (variant == SMAT_V_SELL) {
    const long long ns = h->sell_ns;
    if (ns == 0) return cudaSuccess;
    (void)launch_pdl(sell_kernel<V, MODE, SELL_U>, dim3(grid_for(ns * SELL_C, 256, INT_MAX)), dim3(256), 0, s,
        h->sell_ptr, h->sell_width, h->sell_perm, h->sell_col, (const V *)h->sell_val, x, ep, y, ns);
    return cudaGetLastError();
  }
  const long long mb = h->bcsr_mb;
  const int g = grid_for((mb + BCSR_R2 - 1) / BCSR_R2 * h->bcsr_b, 256, INT_MAX);
  switch (h->bcsr_b) {
    case 2: (void)launch_pdl(bcsr_kernel<V, 2, BCSR_R2, MODE>, dim3(g), dim3(256), 0, s, h->bcsr_rowptr, h->bcsr_col, (const V *)h->bcsr_val, x,
                                                                 ep, y, h->m, h->n, mb, h->bcsr_cb); break;
    case 4: (void)launch_pdl(bcsr_kernel<V, 4, BCSR_R2, MODE>, dim3(g), dim3(256), 0, s, h->bcsr_rowptr, h->bcsr_col, (const V *)h->bcsr_val, x,
                                                                 ep, y, h->m, h->n, mb, h->bcsr_cb); break;
    default: (void)launch_pdl(bcsr_kernel<V, 8, BCSR_R2, MODE>, dim3(g), dim3(256), 0, s, h->bcsr_rowptr, h->bcsr_col, (const V *)h->bcsr_val, x,
                                                                  ep, y, h->m, h->n, mb, h->bcsr_cb); break;
  }
  return cudaGetLastError();
}

template <typename V>
cudaError_t ext_typed(const smat_s *h, int variant, const void *alpha_p, const void *x, const void *beta_p, void *y,
                      cudaStream_t s) {
  typedef typename Compute<V>::T T;
  const T alpha = *(const T *)alpha_p, beta = *(const T *)beta_p;
  if (h->m == 0) return cudaSuccess;
  switch (epi_mode((double)alpha, (double)beta)) {
    case EPI_COPY: return ext_mode<V, EPI_COPY>(h, variant, alpha, x, beta, y, s);
    case EPI_SCALE: return ext_mode<V, EPI_SCALE>(h, variant, alpha, x, beta, y, s);
    default: return ext_mode<V, EPI_AXPBY>(h, variant, alpha, x, beta, y, s);
  }
}

}  // namespace

cudaError_t exclusive_scan(const long long *in, long long n, long long *out, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(out, 0, sizeof(long long), s);
  const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  void *sums = nullptr;
  cudaError_t e = dev_alloc(&sums, (size_t)tiles * sizeof(long long));
  if (e != cudaSuccess) return e;
  scan_tile_sums<<<(unsigned)tiles, SCAN_NT, 0, s>>>(in, n, (long long *)sums);
  scan_tile_offsets<<<1, SCAN_NT, 0, s>>>((long long *)sums, tiles);
  scan_tiles<<<(unsigned)tiles, SCAN_NT, 0, s>>>(in, n, (const long long *)sums, out);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(sums);
  return e;
}

cudaError_t launch_hyb_tail_counts(const smat_s *h, int64_t K, long long *cnt, cudaStream_t s) {
  if (h->m <= 0) return cudaSuccess;
  hyb_tail_counts<<<grid_for(h->m, 256, 152 * 16), 256, 0, s>>>(h->rowptr, h->m, K, cnt);
  return cudaGetLastError();
}

cudaError_t launch_to_hyb(const smat_s *h, int64_t K, const long long *off, int32_t *ecol, void *eval, int32_t *crow,
                          int32_t *ccol, void *cval, cudaStream_t s) {
  if (h->P <= 0) return cudaSuccess;
  const int g = grid_for(h->P, 256, 152 * 16);
  switch (h->esz) {
    case 8: to_hyb_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<8>::T *)h->val, h->m, h->P, K, off, ecol,
                                              (Raw<8>::T *)eval, crow, ccol, (Raw<8>::T *)cval); break;
    case 4: to_hyb_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<4>::T *)h->val, h->m, h->P, K, off, ecol,
                                              (Raw<4>::T *)eval, crow, ccol, (Raw<4>::T *)cval); break;
    default: to_hyb_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<2>::T *)h->val, h->m, h->P, K, off, ecol,
                                               (Raw<2>::T *)eval, crow, ccol, (Raw<2>::T *)cval); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sell_layout(const smat_s *h, int sigma, int32_t *perm, int32_t *width, long long *cnt,
                               cudaStream_t s) {
  if (h->m <= 0) return cudaSuccess;
  const long long windows = (h->m + sigma - 1) / sigma;
  sell_sort_kernel<<<(unsigned)windows, 1024, (size_t)sigma * sizeof(int), s>>>(h->rowptr, h->m, sigma, perm);
  const long long mp = (h->m + SELL_C - 1) / SELL_C * SELL_C;
  sell_width_kernel<<<grid_for(mp, 256, 152 * 16), 256, 0, s>>>(h->rowptr, h->m, mp, perm, width, cnt);
  return cudaGetLastError();
}

cudaError_t launch_to_sell(const smat_s *h, cudaStream_t s) {
  const long long mp = h->sell_ns * SELL_C;
  if (mp <= 0) return cudaSuccess;
  const int g = grid_for(mp, 256, 152 * 16);
  switch (h->esz) {
    case 8: to_sell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<8>::T *)h->val, mp, h->sell_perm,
                                               h->sell_width, h->sell_ptr, h->sell_col, (Raw<8>::T *)h->sell_val); break;
    case 4: to_sell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<4>::T *)h->val, mp, h->sell_perm,
                                               h->sell_width, h->sell_ptr, h->sell_col, (Raw<4>::T *)h->sell_val); break;
    default: to_sell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<2>::T *)h->val, mp, h->sell_perm,
                                                h->sell_width, h->sell_ptr, h->sell_col, (Raw<2>::T *)h->sell_val); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_bcsr_count(const smat_s *h, int b, long long *cnt, cudaStream_t s) {
  const long long mb = (h->m + b - 1) / b;
  if (mb <= 0) return cudaSuccess;
  const int g = grid_for(mb, 128, 152 * 32);
  switch (b) {
    case 2: bcsr_count_kernel<2><<<g, 128, 0, s>>>(h->rowptr, h->colidx, h->m, mb, cnt); break;
    case 4: bcsr_count_kernel<4><<<g, 128, 0, s>>>(h->rowptr, h->colidx, h->m, mb, cnt); break;
    default: bcsr_count_kernel<8><<<g, 128, 0, s>>>(h->rowptr, h->colidx, h->m, mb, cnt); break;
  }
  return cudaGetLastError();
}

template <int BS>
static cudaError_t to_bcsr_b(const smat_s *h, const long long *brp, cudaStream_t s) {
  const long long mb = h->bcsr_mb;
  const int g = grid_for(mb, 128, 152 * 32);
  switch (h->esz) {
    case 8: to_bcsr_kernel<BS><<<g, 128, 0, s>>>(h->rowptr, h->colidx, (const Raw<8>::T *)h->val, h->m, mb, brp,
                                                   h->bcsr_rowptr, h->bcsr_col, (Raw<8>::T *)h->bcsr_val); break;
    case 4: to_bcsr_kernel<BS><<<g, 128, 0, s>>>(h->rowptr, h->colidx, (const Raw<4>::T *)h->val, h->m, mb, brp,
                                                   h->bcsr_rowptr, h->bcsr_col, (Raw<4>::T *)h->bcsr_val); break;
    default: to_bcsr_kernel<BS><<<g, 128, 0, s>>>(h->rowptr, h->colidx, (const Raw<2>::T *)h->val, h->m, mb, brp,
                                                    h->bcsr_rowptr, h->bcsr_col, (Raw<2>::T *)h->bcsr_val); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_bcsr(const smat_s *h, const long long *brp, cudaStream_t s) {
  if (h->bcsr_mb <= 0) return cudaSuccess;
  switch (h->bcsr_b) {
    case 2: return to_bcsr_b<2>(h, brp, s);
    case 4: return to_bcsr_b<4>(h, brp, s);
    default: return to_bcsr_b<8>(h, brp, s);
  }
}

__global__ void bcsr_uniform_kernel(const long long *__restrict__ brp, long long mb, long long c, int *__restrict__ flag) {
  for (long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x; I < mb; I += (long long)gridDim.x * blockDim.x)
    if (brp[I + 1] - brp[I] != c) *flag = 1;
}

cudaError_t launch_bcsr_uniform(const smat_s *h, long long c, int *flag, cudaStream_t s) {
  if (h->bcsr_mb <= 0) return cudaSuccess;
  bcsr_uniform_kernel<<<grid_for(h->bcsr_mb, 256, 152 * 8), 256, 0, s>>>(h->bcsr_brp64, h->bcsr_mb, c, flag);
  return cudaGetLastError();
}

cudaError_t launch_split_counts(const smat_s *h, long long *cl, long long *cc, long long *cs, long long *ce,
                                cudaStream_t s) {
  if (h->m <= 0) return cudaSuccess;
  split_counts_kernel<<<grid_for(h->m, 256, 152 * 16), 256, 0, s>>>(h->rowptr, h->m, cl, cc, cs, ce);
  return cudaGetLastError();
}

cudaError_t launch_split_fill(const smat_s *h, const long long *pl, const long long *pc, const long long *ps,
                              const long long *pe, cudaStream_t s) {
  if (h->m <= 0) return cudaSuccess;
  const int g = grid_for(h->m, 256, 152 * 16);
  switch (h->esz) {
    case 8: split_fill_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<8>::T *)h->val, h->m, pl, pc, ps, pe,
                                                  h->split_lrows, h->split_lchunk, h->split_crow, h->split_cstart,
                                                  h->split_cend, h->split_srow, h->split_scol,
                                                  (Raw<8>::T *)h->split_sval, h->split_empty); break;
    case 4: split_fill_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<4>::T *)h->val, h->m, pl, pc, ps, pe,
                                                  h->split_lrows, h->split_lchunk, h->split_crow, h->split_cstart,
                                                  h->split_cend, h->split_srow, h->split_scol,
                                                  (Raw<4>::T *)h->split_sval, h->split_empty); break;
    default: split_fill_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Raw<2>::T *)h->val, h->m, pl, pc, ps, pe,
                                                   h->split_lrows, h->split_lchunk, h->split_crow, h->split_cstart,
                                                   h->split_cend, h->split_srow, h->split_scol,
                                                   (Raw<2>::T *)h->split_sval, h->split_empty); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_spmv_ext(const smat_s *h, int variant, const void *alpha, const void *x, const void *beta, void *y,
                            cudaStream_t s) {
  switch (h->dtype) {
    case SMAT_F64: return ext_typed<double>(h, variant, alpha, x, beta, y, s);
    case SMAT_F32: return ext_typed<float>(h, variant, alpha, x, beta, y, s);
    default: return ext_typed<__nv_bfloat16>(h, variant, alpha, x, beta, y, s);
  }
}

}  // namespace smat
