/*
 * CPU ORACLE for the SMAT hot path (arXiv 1210.2536).  TEST INFRASTRUCTURE.
 *
 * Plain, slow, obviously correct C, in FP64, compiled with -ffp-contract=off so
 * that every multiply and add below is one IEEE round-to-nearest operation in
 * the order written.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg and reference arm may load this library; the product path
 * never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Each function cites the passage of the paper it follows.  Where the paper is
 * silent the reading taken is stated next to the code:
 *   - NNZ counts stored entries (structural nonzeros, explicit zeros included).
 *   - var_RD is the population variance (denominator M), Sec. 4.
 *   - a "true" diagonal holds more than tau = num/den of its positions
 *     (default 3/5); the paper gives no value, Sec. 4.
 *   - R is the negated slope of an unweighted least-squares line through
 *     (ln k, ln h[k]) for the row-degree histogram h, k >= 1 with h[k] > 0;
 *     with fewer than two points R = 0 and R_valid = 0, Sec. 4.
 *   - Ratios with a zero denominator are 0.
 *   - DIA/ELL/COO layouts (the paper's figure of the four formats is not
 *     available): DIA diagonal-major with pitch P, ELL column-major with pitch
 *     P, COO in CSR order; padding is column -1 / value +0.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* SpMV  y = alpha*A*x + beta*y  on CSR (Sec. 2.1: CSR is the unified input  */
/* and default format; Sec. 3).                                              */
/* Row i: acc = 0; acc = acc + a_ik * x_k in ascending storage order; then   */
/* y_i = alpha*acc            if beta == 0  (y is not read, BLAS convention) */
/* y_i = alpha*acc + beta*y_i otherwise.                                     */
/* ------------------------------------------------------------------------ */
static void spmv_rows(int64_t r0, int64_t r1, const int32_t *rowptr, const int32_t *colidx,
                      const double *val, const double *x, double alpha, double beta, double *y) {
  for (int64_t i = r0; i < r1; ++i) {
    double acc = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      double prod = val[k] * x[colidx[k]];
      acc = acc + prod;
    }
    double ax = alpha * acc;
    if (beta == 0.0) {
      y[i] = ax;
    } else {
      double by = beta * y[i];
      y[i] = ax + by;
    }
  }
}

void oracle_spmv_csr(int64_t m, const int32_t *rowptr, const int32_t *colidx, const double *val,
                     const double *x, double alpha, double beta, double *y) {
  spmv_rows(0, m, rowptr, colidx, val, x, alpha, beta, y);
}

/* Same product on several threads with the paper's nonzero-balanced row split
 * (Sec. 6): each thread gets about NNZ/T nonzeros, rounded to whole rows.  A
 * row is owned by one thread, so the result is bitwise the serial one. */
typedef struct {
  int64_t r0, r1;
  const int32_t *rowptr, *colidx;
  const double *val, *x;
  double alpha, beta;
  double *y;
} spmv_job_t;

static void *spmv_worker(void *arg) {
  spmv_job_t *J = (spmv_job_t *)arg;
  spmv_rows(J->r0, J->r1, J->rowptr, J->colidx, J->val, J->x, J->alpha, J->beta, J->y);
  return NULL;
}

static int64_t first_row_at_or_after(const int32_t *rowptr, int64_t m, int64_t target) {
  int64_t lo = 0, hi = m; /* first row i with rowptr[i] >= target */
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if ((int64_t)rowptr[mid] >= target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

void oracle_partition_rows(int64_t m, const int32_t *rowptr, int nthreads, int64_t *bounds) {
  int64_t base = rowptr[0], nnz = (int64_t)rowptr[m] - base;
  bounds[0] = 0;
  for (int t = 1; t < nthreads; ++t) {
    int64_t target = base + nnz * t / nthreads;
    int64_t r = first_row_at_or_after(rowptr, m, target);
    if (r < bounds[t - 1]) r = bounds[t - 1];
    bounds[t] = r;
  }
  bounds[nthreads] = m;
}

int oracle_spmv_csr_threads(int64_t m, const int32_t *rowptr, const int32_t *colidx,
                            const double *val, const double *x, double alpha, double beta,
                            double *y, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  int64_t *b = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nthreads + 1));
  spmv_job_t *jobs = (spmv_job_t *)malloc(sizeof(spmv_job_t) * (size_t)nthreads);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  if (!b || !jobs || !th) { free(b); free(jobs); free(th); return -1; }
  oracle_partition_rows(m, rowptr, nthreads, b);
  for (int t = 0; t < nthreads; ++t) {
    spmv_job_t J = {b[t], b[t + 1], rowptr, colidx, val, x, alpha, beta, y};
    jobs[t] = J;
  }
  int *started = (int *)calloc((size_t)nthreads, sizeof(int));
  for (int t = 1; t < nthreads; ++t)
    started[t] = pthread_create(&th[t], NULL, spmv_worker, &jobs[t]) == 0;
  spmv_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) {
    if (started[t]) pthread_join(th[t], NULL); else spmv_worker(&jobs[t]);
  }
  free(started); free(b); free(jobs); free(th);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Feature parameters (Sec. 4, Table "Feature parameters of a sparse        */
/* matrix"): M, N, NNZ, aver_RD, Ndiags, NTdiags_ratio, ER_DIA, max_RD,      */
/* min_RD, var_RD, ER_ELL, R.                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t m, n, nnz;
  int64_t max_rd, min_rd;
  int64_t ndiags, ntdiags;     /* occupied diagonals, "true" diagonals      */
  int64_t empty_rows;
  int64_t s2_lo, s2_hi;        /* sum of rd^2 as a 128-bit integer          */
  double aver_rd;              /* NNZ / M                                   */
  double var_rd;               /* (M*S2 - NNZ^2) / M^2                      */
  double er_dia;               /* NNZ / (Ndiags * M)                        */
  double er_ell;               /* NNZ / (max_RD * M)                        */
  double ntdiags_ratio;        /* true diagonals / Ndiags                   */
  double r;                    /* power-law exponent estimate               */
  int64_t r_valid;
} oracle_features_t;

/* Length of diagonal d = j - i of an M x N matrix. */
static int64_t diag_len(int64_t m, int64_t n, int64_t d) {
  int64_t len = (d >= 0) ? ((m < n - d) ? m : n - d) : ((m + d < n) ? m + d : n);
  return len < 0 ? 0 : len;
}

/* R: least squares through (ln k, ln h[k]) (Sec. 4: P(k) ~ k^-R). */
static void power_law_fit(const int64_t *hist, int64_t max_rd, double *r, int64_t *valid) {
  double np = 0.0, sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
  for (int64_t k = 1; k <= max_rd; ++k) {
    if (hist[k] <= 0) continue;
    double lx = log((double)k);
    double ly = log((double)hist[k]);
    np = np + 1.0;
    sx = sx + lx;
    sy = sy + ly;
    sxx = sxx + lx * lx;
    sxy = sxy + lx * ly;
  }
  if (np < 2.0) { *r = 0.0; *valid = 0; return; }
  double num = np * sxy - sx * sy;
  double den = np * sxx - sx * sx;
  *r = -(num / den);
  *valid = 1;
}

/* hist must hold max_RD+1 entries (call oracle_max_rd first); diag_cnt must
 * hold M+N-1 entries, indexed by d + M - 1. */
int64_t oracle_max_rd(int64_t m, const int32_t *rowptr) {
  int64_t mx = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t rd = (int64_t)rowptr[i + 1] - rowptr[i];
    if (rd > mx) mx = rd;
  }
  return mx;
}

void oracle_features(int64_t m, int64_t n, const int32_t *rowptr, const int32_t *colidx,
                     int64_t tau_num, int64_t tau_den, int64_t *hist, int64_t *diag_cnt,
                     oracle_features_t *f) {
  memset(f, 0, sizeof(*f));
  f->m = m;
  f->n = n;
  f->nnz = (m > 0) ? rowptr[m] : 0;
  /* row degrees */
  int64_t mx = 0, mn = (m > 0) ? INT64_MAX : 0, empty = 0;
  unsigned __int128 s2 = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t rd = (int64_t)rowptr[i + 1] - rowptr[i];
    if (rd > mx) mx = rd;
    if (rd < mn) mn = rd;
    if (rd == 0) ++empty;
    s2 += (unsigned __int128)((uint64_t)rd * (uint64_t)rd);
  }
  f->max_rd = mx;
  f->min_rd = mn;
  f->empty_rows = empty;
  f->s2_lo = (int64_t)(uint64_t)s2;
  f->s2_hi = (int64_t)(uint64_t)(s2 >> 64);
  for (int64_t k = 0; k <= mx; ++k) hist[k] = 0;
  for (int64_t i = 0; i < m; ++i) hist[rowptr[i + 1] - rowptr[i]] += 1;
  /* diagonals d = j - i, d in [-(M-1), N-1] */
  int64_t nd = (m + n > 0) ? m + n - 1 : 0;
  for (int64_t d = 0; d < nd; ++d) diag_cnt[d] = 0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
      diag_cnt[(int64_t)colidx[k] - i + m - 1] += 1;
  int64_t occ = 0, tru = 0;
  for (int64_t t = 0; t < nd; ++t) {
    if (diag_cnt[t] == 0) continue;
    ++occ;
    int64_t len = diag_len(m, n, t - (m - 1));
    if (tau_den * diag_cnt[t] > tau_num * len) ++tru;
  }
  f->ndiags = occ;
  f->ntdiags = tru;
  /* ratios: exact integers, each converted to double once, one division */
  f->aver_rd = (m > 0) ? (double)f->nnz / (double)m : 0.0;
  if (m > 0) {
    __int128 num = (__int128)m * (__int128)s2 - (__int128)f->nnz * (__int128)f->nnz;
    __int128 den = (__int128)m * (__int128)m;
    f->var_rd = (double)num / (double)den;
  }
  f->er_dia = (occ > 0 && m > 0) ? (double)f->nnz / (double)(occ * m) : 0.0;
  f->er_ell = (mx > 0 && m > 0) ? (double)f->nnz / (double)(mx * m) : 0.0;
  f->ntdiags_ratio = (occ > 0) ? (double)tru / (double)occ : 0.0;
  power_law_fit(hist, mx, &f->r, &f->r_valid);
}

/* ------------------------------------------------------------------------ */
/* Format conversions from CSR (Sec. 2.1; Table "Performance features of the */
/* four formats").  Values are copied as raw bytes of width elem_size, so    */
/* the same functions serve FP64, FP32 and BF16 storage.                      */
/* ------------------------------------------------------------------------ */

/* ELL: K slots per row, column-major with pitch P >= M: slot s of row i lives
 * at s*P + i.  Slot s < rd_i holds the s-th CSR entry of row i; the rest, and
 * rows M..P-1, hold column -1 and value +0. */
void oracle_to_ell(int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *val,
                   int64_t elem_size, int64_t K, int64_t P, int32_t *ell_col, void *ell_val) {
  unsigned char *ov = (unsigned char *)ell_val;
  const unsigned char *iv = (const unsigned char *)val;
  for (int64_t s = 0; s < K; ++s) {
    for (int64_t i = 0; i < P; ++i) {
      int64_t pos = s * P + i;
      int64_t rd = (i < m) ? (int64_t)rowptr[i + 1] - rowptr[i] : 0;
      if (s < rd) {
        int64_t k = rowptr[i] + s;
        ell_col[pos] = colidx[k];
        memcpy(ov + pos * elem_size, iv + k * elem_size, (size_t)elem_size);
      } else {
        ell_col[pos] = -1;
        memset(ov + pos * elem_size, 0, (size_t)elem_size);
      }
    }
  }
}

/* DIA offsets: the occupied diagonals d = j - i in ascending order.  Returns
 * their number; offsets may be NULL to count only. */
int64_t oracle_dia_offsets(int64_t m, int64_t n, const int32_t *rowptr, const int32_t *colidx,
                           int32_t *offsets) {
  int64_t nd = (m + n > 0) ? m + n - 1 : 0;
  unsigned char *seen = (unsigned char *)calloc((size_t)(nd > 0 ? nd : 1), 1);
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) seen[(int64_t)colidx[k] - i + m - 1] = 1;
  int64_t c = 0;
  for (int64_t t = 0; t < nd; ++t)
    if (seen[t]) {
      if (offsets) offsets[c] = (int32_t)(t - (m - 1));
      ++c;
    }
  free(seen);
  return c;
}

/* DIA values: element (i, i + off_t) at t*P + i; +0 where not stored
 * (including positions whose column falls outside the matrix). */
void oracle_to_dia(int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *val,
                   int64_t elem_size, const int32_t *offsets, int64_t ndiags, int64_t P,
                   void *dia_val) {
  unsigned char *ov = (unsigned char *)dia_val;
  const unsigned char *iv = (const unsigned char *)val;
  memset(ov, 0, (size_t)(ndiags * P * elem_size));
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int64_t d = (int64_t)colidx[k] - i;
      int64_t lo = 0, hi = ndiags; /* find t with offsets[t] == d */
      while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (offsets[mid] < d) lo = mid + 1; else hi = mid;
      }
      memcpy(ov + (lo * P + i) * elem_size, iv + k * elem_size, (size_t)elem_size);
    }
  }
}

/* COO in CSR order: row[k] = i for rowptr[i] <= k < rowptr[i+1]. */
void oracle_to_coo(int64_t m, const int32_t *rowptr, int32_t *row) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) row[k] = (int32_t)i;
}

/* ------------------------------------------------------------------------ */
/* Further GPU formats.  Sec. 2.1 covers DIA, ELL, CSR and COO; Sec. 1 and    */
/* Sec. 8 leave more formats to future work.  The three below follow the      */
/* published methods named beside each; the layouts are this library's.       */
/* ------------------------------------------------------------------------ */

/* HYB (Bell & Garland, 2009): an ELL part of width K plus a COO part holding
 * each row's entries past its first K.  K is the largest k >= 0 for which at
 * least a third of the rows hold k or more entries (3 * #{i : rd_i >= k} >= M);
 * K = 0 when M = 0. */
int64_t oracle_hyb_width(int64_t m, const int32_t *rowptr) {
  if (m <= 0) return 0;
  int64_t maxrd = oracle_max_rd(m, rowptr);
  int64_t *hist = (int64_t *)calloc((size_t)maxrd + 1, sizeof(int64_t));
  for (int64_t i = 0; i < m; ++i) hist[rowptr[i + 1] - rowptr[i]] += 1;
  int64_t rows_ge = 0, K = 0;
  for (int64_t k = maxrd; k >= 1; --k) {
    rows_ge += hist[k];               /* rows with k or more entries */
    if (3 * rows_ge >= m) { K = k; break; }
  }
  free(hist);
  return K;
}

/* ELL part: slot s < min(rd_i, K) of row i, at s*P + i, holds the row's s-th
 * entry; every other slot (and rows M..P-1) holds column -1 / value +0.
 * COO part: the entries of each row past its first K, rows ascending and
 * columns ascending within a row.  Returns the COO part's length; the COO
 * arrays may be NULL to count only, the ELL arrays NULL to skip them. */
int64_t oracle_to_hyb(int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *val,
                      int64_t elem_size, int64_t K, int64_t P, int32_t *ell_col, void *ell_val,
                      int32_t *coo_row, int32_t *coo_col, void *coo_val) {
  const unsigned char *iv = (const unsigned char *)val;
  if (ell_col && ell_val) {
    unsigned char *ev = (unsigned char *)ell_val;
    for (int64_t s = 0; s < K; ++s)
      for (int64_t i = 0; i < P; ++i) {
        int64_t pos = s * P + i;
        int64_t rd = (i < m) ? (int64_t)rowptr[i + 1] - rowptr[i] : 0;
        if (s < rd) {
          ell_col[pos] = colidx[rowptr[i] + s];
          memcpy(ev + pos * elem_size, iv + (rowptr[i] + s) * elem_size, (size_t)elem_size);
        } else {
          ell_col[pos] = -1;
          memset(ev + pos * elem_size, 0, (size_t)elem_size);
        }
      }
  }
  int64_t c = 0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = (int64_t)rowptr[i] + K; k < rowptr[i + 1]; ++k) {
      if (coo_row) {
        coo_row[c] = (int32_t)i;
        coo_col[c] = colidx[k];
        memcpy((unsigned char *)coo_val + c * elem_size, iv + k * elem_size, (size_t)elem_size);
      }
      ++c;
    }
  return c;
}

/* SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske & Bishop, 2014).  Rows are
 * sorted by decreasing length inside windows of sigma consecutive rows (equal
 * lengths keep their row order); the sorted sequence, padded with empty
 * positions to Mp = M rounded up to C, is cut into slices of C positions, and
 * each slice is a C-row column-major ELL block as wide as its longest row.
 *   perm[p]       row at sorted position p (-1 for positions M..Mp-1)
 *   width[s]      longest row length in slice s
 *   slice_ptr[s]  sum over slices t < s of C * width[t]  (nslices + 1 values)
 * Entry j of the row at position s*C + l is slot slice_ptr[s] + j*C + l;
 * slots past the row's length hold column -1 / value +0.  sigma must be a
 * positive multiple of C.  Returns the number of slots; perm, width and
 * slice_ptr must hold Mp, Mp/C and Mp/C + 1 values. */
typedef struct { int64_t len, row; } sell_key;
static int sell_key_cmp(const void *a, const void *b) {
  const sell_key *x = (const sell_key *)a, *y = (const sell_key *)b;
  if (x->len != y->len) return x->len > y->len ? -1 : 1;   /* longer first */
  return x->row < y->row ? -1 : (x->row > y->row ? 1 : 0);  /* then row order */
}
int64_t oracle_sell_layout(int64_t m, const int32_t *rowptr, int64_t C, int64_t sigma, int32_t *perm,
                           int32_t *width, int64_t *slice_ptr) {
  const int64_t Mp = (m + C - 1) / C * C, ns = Mp / C;
  sell_key *keys = (sell_key *)malloc((size_t)(sigma > 0 ? sigma : 1) * sizeof(sell_key));
  for (int64_t w0 = 0; w0 < m; w0 += sigma) {
    int64_t cnt = (m - w0 < sigma) ? m - w0 : sigma;
    for (int64_t q = 0; q < cnt; ++q) {
      keys[q].row = w0 + q;
      keys[q].len = (int64_t)rowptr[w0 + q + 1] - rowptr[w0 + q];
    }
    qsort(keys, (size_t)cnt, sizeof(sell_key), sell_key_cmp);
    for (int64_t q = 0; q < cnt; ++q) perm[w0 + q] = (int32_t)keys[q].row;
  }
  free(keys);
  for (int64_t p = m; p < Mp; ++p) perm[p] = -1;
  slice_ptr[0] = 0;
  for (int64_t s = 0; s < ns; ++s) {
    int64_t wmax = 0;
    for (int64_t l = 0; l < C; ++l) {
      int32_t r = perm[s * C + l];
      int64_t len = r >= 0 ? (int64_t)rowptr[r + 1] - rowptr[r] : 0;
      if (len > wmax) wmax = len;
    }
    width[s] = (int32_t)wmax;
    slice_ptr[s + 1] = slice_ptr[s] + C * wmax;
  }
  return slice_ptr[ns];
}

void oracle_to_sell(int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *val, int64_t elem_size,
                    int64_t C, const int32_t *perm, const int32_t *width, const int64_t *slice_ptr,
                    int32_t *sell_col, void *sell_val) {
  const int64_t ns = (m + C - 1) / C;
  const unsigned char *iv = (const unsigned char *)val;
  unsigned char *ov = (unsigned char *)sell_val;
  for (int64_t s = 0; s < ns; ++s)
    for (int64_t j = 0; j < width[s]; ++j)
      for (int64_t l = 0; l < C; ++l) {
        int64_t slot = slice_ptr[s] + j * C + l;
        int32_t r = perm[s * C + l];
        int64_t len = r >= 0 ? (int64_t)rowptr[r + 1] - rowptr[r] : 0;
        if (j < len) {
          sell_col[slot] = colidx[rowptr[r] + j];
          memcpy(ov + slot * elem_size, iv + (rowptr[r] + j) * elem_size, (size_t)elem_size);
        } else {
          sell_col[slot] = -1;
          memset(ov + slot * elem_size, 0, (size_t)elem_size);
        }
      }
}

/* BCSR with b x b blocks (block compressed sparse row, the register-blocked
 * format of Im & Yelick).  Block row I covers rows I*b .. I*b+b-1; its blocks
 * are the distinct block columns J = col / b of those rows' entries, in
 * ascending order.  Block k stores a(I*b + r, J*b + c) at k*b*b + r*b + c and
 * +0 where nothing is stored (also past the last row or column).  browptr
 * holds ceil(M/b) + 1 values.  Returns the number of blocks; bcol and bval may
 * be NULL to count only (browptr is still filled). */
static int int_cmp(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}
int64_t oracle_to_bcsr(int64_t m, int64_t n, const int32_t *rowptr, const int32_t *colidx, const void *val,
                       int64_t elem_size, int64_t b, int32_t *browptr, int32_t *bcol, void *bval) {
  const int64_t mb = (m + b - 1) / b, nbc = (n + b - 1) / b;
  int64_t *stamp = (int64_t *)malloc((size_t)(nbc > 0 ? nbc : 1) * sizeof(int64_t));
  int32_t *list = (int32_t *)malloc((size_t)(nbc > 0 ? nbc : 1) * sizeof(int32_t));
  for (int64_t J = 0; J < nbc; ++J) stamp[J] = -1;
  const unsigned char *iv = (const unsigned char *)val;
  unsigned char *ov = (unsigned char *)bval;
  int64_t nb = 0;
  browptr[0] = 0;
  for (int64_t I = 0; I < mb; ++I) {
    int64_t cnt = 0;
    for (int64_t i = I * b; i < I * b + b && i < m; ++i)
      for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        int32_t J = colidx[k] / (int32_t)b;
        if (stamp[J] != I) { stamp[J] = I; list[cnt++] = J; }
      }
    qsort(list, (size_t)cnt, sizeof(int32_t), int_cmp);
    if (bcol && bval) {
      for (int64_t q = 0; q < cnt; ++q) bcol[nb + q] = list[q];
      memset(ov + nb * b * b * elem_size, 0, (size_t)(cnt * b * b * elem_size));
      for (int64_t i = I * b; i < I * b + b && i < m; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
          int32_t J = colidx[k] / (int32_t)b;
          int64_t lo = 0, hi = cnt;  /* block q with list[q] == J */
          while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (list[mid] < J) lo = mid + 1; else hi = mid;
          }
          int64_t pos = (nb + lo) * b * b + (i - I * b) * b + (colidx[k] - (int64_t)J * b);
          memcpy(ov + pos * elem_size, iv + k * elem_size, (size_t)elem_size);
        }
    }
    nb += cnt;
    browptr[I + 1] = (int32_t)nb;
  }
  free(stamp);
  free(list);
  return nb;
}

/* Block size: the b in {2, 4, 8} whose BCSR moves the fewest bytes,
 * nblocks(b) * (b*b*elem_size + 4) + 4 * (ceil(M/b) + 1); ties go to the
 * smaller b.  Returns b and writes the block count. */
int64_t oracle_bcsr_choose(int64_t m, int64_t n, const int32_t *rowptr, const int32_t *colidx, int64_t elem_size,
                           int64_t *nblocks) {
  int64_t best_b = 0, best_nb = 0;
  double best_bytes = 0.0;
  int32_t *brp = (int32_t *)malloc((size_t)(m / 2 + 2) * sizeof(int32_t));
  for (int64_t b = 2; b <= 8; b *= 2) {
    int64_t nb = oracle_to_bcsr(m, n, rowptr, colidx, NULL, elem_size, b, brp, NULL, NULL);
    double bytes = (double)nb * (double)(b * b * elem_size + 4) + 4.0 * (double)((m + b - 1) / b + 1);
    if (best_b == 0 || bytes < best_bytes) { best_b = b; best_nb = nb; best_bytes = bytes; }
  }
  free(brp);
  *nblocks = best_nb;
  return best_b;
}

/* SPLIT: rows split by length.  Rows with at least L stored entries ("long")
 * are listed in ascending order and cut into chunks of at most CK consecutive
 * entries (a long row's chunks in order; chunk c covers entries
 * [cstart[c], cend[c]) of row crow[c]); every other non-empty row ("short")
 * goes, in CSR order, to a COO of its entries; empty rows are listed.  Each
 * output array may be NULL to count only.  Writes the counts to cnt[4] =
 * {long rows, chunks, short entries, empty rows}. */
void oracle_split(int64_t m, const int32_t *rowptr, const int32_t *colidx, const void *val, int64_t elem_size,
                  int64_t L, int64_t CK, int32_t *lrows, int32_t *crow, int32_t *cstart, int32_t *cend,
                  int32_t *srow, int32_t *scol, void *sval, int32_t *empty, int64_t *cnt) {
  const unsigned char *iv = (const unsigned char *)val;
  int64_t nl = 0, nc = 0, ns = 0, ne = 0;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t s0 = rowptr[i], e0 = rowptr[i + 1], rd = e0 - s0;
    if (rd == 0) {
      if (empty) empty[ne] = (int32_t)i;
      ++ne;
    } else if (rd >= L) {
      if (lrows) lrows[nl] = (int32_t)i;
      ++nl;
      for (int64_t k = s0; k < e0; k += CK) {
        if (crow) {
          crow[nc] = (int32_t)i;
          cstart[nc] = (int32_t)k;
          cend[nc] = (int32_t)(k + CK < e0 ? k + CK : e0);
        }
        ++nc;
      }
    } else {
      for (int64_t k = s0; k < e0; ++k) {
        if (srow) {
          srow[ns] = (int32_t)i;
          scol[ns] = colidx[k];
          memcpy((unsigned char *)sval + ns * elem_size, iv + k * elem_size, (size_t)elem_size);
        }
        ++ns;
      }
    }
  }
  cnt[0] = nl; cnt[1] = nc; cnt[2] = ns; cnt[3] = ne;
}

/* ------------------------------------------------------------------------ */
/* BF16 storage: round-to-nearest-even of an FP64 value to the bfloat16 grid */
/* (1 sign, 8 exponent, 7 fraction bits; IEEE 754 rounding), written from    */
/* the definition on the FP64 bit pattern.  Returns the 16-bit pattern.      */
/* ------------------------------------------------------------------------ */
static uint16_t bf16_from_double(double v) {
  uint64_t b;
  memcpy(&b, &v, 8);
  uint16_t sign = (uint16_t)((b >> 63) << 15);
  int64_t e = (int64_t)((b >> 52) & 0x7FF);
  uint64_t f = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7FF) return f ? (uint16_t)(sign | 0x7FC0) : (uint16_t)(sign | 0x7F80);
  if (e == 0 && f == 0) return sign;
  /* |v| = sig * 2^(ex), sig an integer */
  uint64_t sig;
  int64_t ex;
  if (e == 0) { sig = f; ex = -1074; } else { sig = f | (1ull << 52); ex = e - 1075; }
  /* target spacing: normals with unbiased exponent E >= -126 have spacing
   * 2^(E-7); below 2^-126 the spacing is 2^-133 (subnormals). */
  int64_t top = 63 - __builtin_clzll(sig) + ex; /* floor(log2 |v|) */
  int64_t E = top < -126 ? -126 : top;
  int64_t q = E - 7;                            /* spacing exponent */
  /* rounded integer multiple of 2^q */
  uint64_t mult;
  int64_t shift = q - ex;
  if (shift <= 0) {
    mult = sig << (-shift); /* exact (cannot happen for doubles beyond range) */
  } else if (shift >= 64) {
    mult = 0;
    /* value < 2^(q-1)... only exact halfway counts; sig < 2^53 so < half */
  } else {
    uint64_t qt = sig >> shift;
    uint64_t rem = sig & ((1ull << shift) - 1);
    uint64_t half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (qt & 1))) ++qt;
    mult = qt;
  }
  if (mult == 0) return sign;
  /* value = mult * 2^q; renormalise (rounding may carry to 2^8) */
  int64_t mt = 63 - __builtin_clzll(mult);
  int64_t vexp = mt + q; /* floor(log2) of the result */
  if (vexp > 127) return (uint16_t)(sign | 0x7F80);
  if (vexp < -126) { /* subnormal: fraction field = mult (spacing 2^-133) */
    return (uint16_t)(sign | (uint16_t)mult);
  }
  /* here mt is 7, or 8 when rounding carried into the next binade */
  uint64_t frac = (mult >> (mt - 7)) & 0x7F;
  uint16_t biased = (uint16_t)(vexp + 127);
  return (uint16_t)(sign | (biased << 7) | (uint16_t)frac);
}

void oracle_round_bf16(int64_t n, const double *in, uint16_t *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = bf16_from_double(in[i]);
}

/* bfloat16 pattern -> FP64 (exact). */
void oracle_bf16_to_double(int64_t n, const uint16_t *in, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u = (uint32_t)in[i] << 16;
    float f;
    memcpy(&f, &u, 4);
    out[i] = (double)f;
  }
}

/* ------------------------------------------------------------------------ */
/* Learned selector: MLP 12 -> 64 -> ReLU -> 64 -> ReLU -> 8 with softmax    */
/* cross-entropy against a target distribution over the 8 kernel variants.   */
/* It replaces the paper's C5.0 ruleset classifier f(x, TH) -> C (Sec. 5,    */
/* Eq. "mapping") with a network trained on measured timings.                 */
/* Parameter layout (row-major, out x in):                                    */
/*   W1[64][12] b1[64] W2[64][64] b2[64] W3[8][64] b3[8]   (5512 values)     */
/* ------------------------------------------------------------------------ */
#define MLP_IN 12
#define MLP_H 64
#define MLP_OUT 8

static void mlp_offsets(int64_t *o) {
  o[0] = 0;                       /* W1 */
  o[1] = o[0] + MLP_H * MLP_IN;   /* b1 */
  o[2] = o[1] + MLP_H;            /* W2 */
  o[3] = o[2] + MLP_H * MLP_H;    /* b2 */
  o[4] = o[3] + MLP_H;            /* W3 */
  o[5] = o[4] + MLP_OUT * MLP_H;  /* b3 */
  o[6] = o[5] + MLP_OUT;          /* total */
}

int64_t oracle_mlp_param_count(void) {
  int64_t o[7];
  mlp_offsets(o);
  return o[6];
}

static void mlp_forward_one(const double *p, const double *x, double *h1, double *h2, double *z) {
  int64_t o[7];
  mlp_offsets(o);
  const double *W1 = p + o[0], *b1 = p + o[1], *W2 = p + o[2], *b2 = p + o[3], *W3 = p + o[4],
               *b3 = p + o[5];
  for (int j = 0; j < MLP_H; ++j) {
    double a = b1[j];
    for (int i = 0; i < MLP_IN; ++i) a = a + W1[j * MLP_IN + i] * x[i];
    h1[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < MLP_H; ++j) {
    double a = b2[j];
    for (int i = 0; i < MLP_H; ++i) a = a + W2[j * MLP_H + i] * h1[i];
    h2[j] = a > 0.0 ? a : 0.0;
  }
  for (int c = 0; c < MLP_OUT; ++c) {
    double a = b3[c];
    for (int i = 0; i < MLP_H; ++i) a = a + W3[c * MLP_H + i] * h2[i];
    z[c] = a;
  }
}

/* logits[B][8] */
void oracle_mlp_forward(const double *params, int64_t B, const double *X, double *logits) {
  double h1[MLP_H], h2[MLP_H];
  for (int64_t b = 0; b < B; ++b) mlp_forward_one(params, X + b * MLP_IN, h1, h2, logits + b * MLP_OUT);
}

/* Mean cross-entropy  L = -(1/B) sum_b sum_c T[b][c] * log softmax(z_b)_c
 * and its gradient with respect to every parameter (backpropagation). */
double oracle_mlp_loss_grad(const double *params, int64_t B, const double *X, const double *T,
                            double *grad) {
  int64_t o[7];
  mlp_offsets(o);
  const double *W2 = params + o[2], *W3 = params + o[4];
  double *gW1 = grad + o[0], *gb1 = grad + o[1], *gW2 = grad + o[2], *gb2 = grad + o[3],
         *gW3 = grad + o[4], *gb3 = grad + o[5];
  for (int64_t i = 0; i < o[6]; ++i) grad[i] = 0.0;
  double loss = 0.0;
  double h1[MLP_H], h2[MLP_H], z[MLP_OUT], dz[MLP_OUT], dh2[MLP_H], dh1[MLP_H];
  for (int64_t b = 0; b < B; ++b) {
    const double *x = X + b * MLP_IN, *t = T + b * MLP_OUT;
    mlp_forward_one(params, x, h1, h2, z);
    double zmax = z[0];
    for (int c = 1; c < MLP_OUT; ++c) if (z[c] > zmax) zmax = z[c];
    double se = 0.0;
    for (int c = 0; c < MLP_OUT; ++c) se = se + exp(z[c] - zmax);
    double lse = zmax + log(se);
    double tsum = 0.0;
    for (int c = 0; c < MLP_OUT; ++c) {
      loss = loss - t[c] * (z[c] - lse);
      tsum = tsum + t[c];
    }
    /* dL/dz_c = (tsum * softmax_c - t_c) / B */
    for (int c = 0; c < MLP_OUT; ++c) dz[c] = (tsum * exp(z[c] - lse) - t[c]) / (double)B;
    for (int c = 0; c < MLP_OUT; ++c) {
      gb3[c] = gb3[c] + dz[c];
      for (int i = 0; i < MLP_H; ++i) gW3[c * MLP_H + i] = gW3[c * MLP_H + i] + dz[c] * h2[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double a = 0.0;
      for (int c = 0; c < MLP_OUT; ++c) a = a + W3[c * MLP_H + i] * dz[c];
      dh2[i] = h2[i] > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_H; ++j) {
      gb2[j] = gb2[j] + dh2[j];
      for (int i = 0; i < MLP_H; ++i) gW2[j * MLP_H + i] = gW2[j * MLP_H + i] + dh2[j] * h1[i];
    }
    for (int i = 0; i < MLP_H; ++i) {
      double a = 0.0;
      for (int j = 0; j < MLP_H; ++j) a = a + W2[j * MLP_H + i] * dh2[j];
      dh1[i] = h1[i] > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < MLP_H; ++j) {
      gb1[j] = gb1[j] + dh1[j];
      for (int i = 0; i < MLP_IN; ++i) gW1[j * MLP_IN + i] = gW1[j * MLP_IN + i] + dh1[j] * x[i];
    }
  }
  return loss / (double)B;
}

/* One Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) with step count t >= 1:
 *   m = b1*m + (1-b1)*g ; v = b2*v + (1-b2)*g^2
 *   p = p - lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)               */
void oracle_adam(int64_t n, double *p, const double *g, double *m, double *v, int64_t t,
                 double lr, double b1, double b2, double eps) {
  double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    double mh = m[i] / c1, vh = v[i] / c2;
    p[i] = p[i] - lr * mh / (sqrt(vh) + eps);
  }
}
