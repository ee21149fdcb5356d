// CSR -> COO / ELL / DIA conversions (arXiv 1210.2536, Sec. 2.1: the four
// basic storage formats; Table "Performance features of the four formats")
// and the value casts used for reduced-precision storage.
//
// Layouts (the paper's figure of the data structures is not available; these
// are the standard definitions):
//   ELL  col/val[s * P + i] = s-th stored entry of row i, s < K = max_RD;
//        padding (and rows M..P-1) hold column -1 and value +0.
//   DIA  val[t * P + i] = a(i, i + off[t]) or +0 where not stored; offsets
//        ascending.
//   COO  row[k] for every stored entry, in CSR order (col and val are CSR's).
// Every output element is written exactly once, with coalesced stores, and
// values are moved as raw bits.
#include "smat_internal.h"

namespace smat {
namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int B> struct Bits;
template <> struct Bits<8> { typedef unsigned long long T; };
template <> struct Bits<4> { typedef unsigned int T; };
template <> struct Bits<2> { typedef unsigned short T; };

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

// COO row indices: a warp expands 32 rows over their contiguous nonzero range.
__global__ void to_coo_kernel(const int32_t *__restrict__ rowptr, long long m, int32_t *__restrict__ row) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r0 = warp * 32; r0 < m; r0 += nwarps * 32) {
    long long r = r0 + lane;
    int s = 0x7fffffff, e = 0;
    if (r < m) { s = rowptr[r]; e = rowptr[r + 1]; }
    int rows = (int)min(32LL, m - r0);
    long long gs = __shfl_sync(FULL, s, 0), ge = __shfl_sync(FULL, e, rows - 1);
    for (long long base = gs; base < ge; base += 32) {
      long long k = base + lane;
      int L = row_lane_of(s, k);
      if (k < ge) row[k] = (int32_t)(r0 + L);
    }
  }
}

__global__ void empty_rows_kernel(const int32_t *__restrict__ rowptr, long long m, int32_t *list, int *count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x)
    if (rowptr[i + 1] == rowptr[i]) list[atomicAdd(count, 1)] = (int32_t)i;
}

// ELL: thread per row (and per pad row up to P).
template <typename B>
__global__ void to_ell_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const B *__restrict__ val, long long m, long long P, long long K,
                              int32_t *__restrict__ ecol, B *__restrict__ eval) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    long long s = 0, rd = 0;
    if (i < m) { s = rowptr[i]; rd = rowptr[i + 1] - s; }
    for (long long q = 0; q < K; ++q) {
      long long pos = q * P + i;
      if (q < rd) {
        ecol[pos] = col[s + q];
        eval[pos] = val[s + q];
      } else {
        ecol[pos] = -1;
        eval[pos] = (B)0;
      }
    }
  }
}

// DIA: thread per row; the row's sorted columns are merged against the
// ascending offsets, so each output element is produced in one pass.
template <typename B>
__global__ void to_dia_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const B *__restrict__ val, long long m, long long P,
                              const int32_t *__restrict__ off, long long nd, B *__restrict__ dval) {
  extern __shared__ int32_t s_off[];
  const bool in_smem = nd <= 4096;
  if (in_smem) {
    for (long long t = threadIdx.x; t < nd; t += blockDim.x) s_off[t] = off[t];
    __syncthreads();
  }
  const int32_t *o = in_smem ? s_off : off;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x) {
    long long k = 0, e = 0;
    if (i < m) { k = rowptr[i]; e = rowptr[i + 1]; }
    for (long long t = 0; t < nd; ++t) {
      long long j = i + o[t];
      while (k < e && col[k] < j) ++k;
      B v = (B)0;
      if (k < e && col[k] == j) { v = val[k]; ++k; }
      dval[t * P + i] = v;
    }
  }
}

__global__ void cast_f32_kernel(const double *__restrict__ in, float *__restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __double2float_rn(in[i]);
}

__global__ void cast_bf16_kernel(const double *__restrict__ in, uint16_t *__restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __bfloat16_as_ushort(__double2bfloat16(in[i]));
}

int grid_for(long long work, int block, int max_blocks) {
  long long g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

}  // namespace

cudaError_t launch_to_coo(const smat_s *h, int32_t *row, cudaStream_t s) {
  if (h->m <= 0 || h->nnz <= 0) return cudaSuccess;
  to_coo_kernel<<<grid_for((h->m + 31) / 32 * 32, 256, 152 * 16), 256, 0, s>>>(h->rowptr, h->m, row);
  return cudaGetLastError();
}

cudaError_t launch_empty_rows(const smat_s *h, int32_t *list, int *d_count, cudaStream_t s) {
  if (h->m <= 0) return cudaSuccess;
  empty_rows_kernel<<<grid_for(h->m, 256, 152 * 8), 256, 0, s>>>(h->rowptr, h->m, list, d_count);
  return cudaGetLastError();
}

cudaError_t launch_to_ell(const smat_s *h, int64_t K, int32_t *col, void *val, cudaStream_t s) {
  if (h->P <= 0 || K <= 0) return cudaSuccess;
  int g = grid_for(h->P, 256, 152 * 16);
  switch (h->esz) {
    case 8: to_ell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Bits<8>::T *)h->val, h->m, h->P, K,
                                              col, (Bits<8>::T *)val); break;
    case 4: to_ell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Bits<4>::T *)h->val, h->m, h->P, K,
                                              col, (Bits<4>::T *)val); break;
    default: to_ell_kernel<<<g, 256, 0, s>>>(h->rowptr, h->colidx, (const Bits<2>::T *)h->val, h->m, h->P, K,
                                               col, (Bits<2>::T *)val); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_to_dia(const smat_s *h, const int32_t *d_off, int64_t nd, void *val, cudaStream_t s) {
  if (h->P <= 0 || nd <= 0) return cudaSuccess;
  int g = grid_for(h->P, 256, 152 * 16);
  size_t sm = nd <= 4096 ? (size_t)nd * sizeof(int32_t) : 0;
  switch (h->esz) {
    case 8: to_dia_kernel<<<g, 256, sm, s>>>(h->rowptr, h->colidx, (const Bits<8>::T *)h->val, h->m, h->P,
                                               d_off, nd, (Bits<8>::T *)val); break;
    case 4: to_dia_kernel<<<g, 256, sm, s>>>(h->rowptr, h->colidx, (const Bits<4>::T *)h->val, h->m, h->P,
                                               d_off, nd, (Bits<4>::T *)val); break;
    default: to_dia_kernel<<<g, 256, sm, s>>>(h->rowptr, h->colidx, (const Bits<2>::T *)h->val, h->m, h->P,
                                                d_off, nd, (Bits<2>::T *)val); break;
  }
  return cudaGetLastError();
}

}  // namespace smat

extern "C" smat_status_t smat_cast_f64_to_f32(const double *in, float *out, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return SMAT_ERR_INVALID_ARG;
  if (n == 0) return SMAT_OK;
  smat::cast_f32_kernel<<<smat::grid_for(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}

extern "C" smat_status_t smat_cast_f64_to_bf16(const double *in, uint16_t *out, int64_t n, void *stream) {
  if (n < 0 || (n > 0 && (!in || !out))) return SMAT_ERR_INVALID_ARG;
  if (n == 0) return SMAT_OK;
  smat::cast_bf16_kernel<<<smat::grid_for(n, 256, 152 * 16), 256, 0, (cudaStream_t)stream>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}
