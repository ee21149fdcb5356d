/*
 * Seeded synthetic sparse matrices and vectors.
 *
 * This file produces INPUTS only.  It holds none of the SpMV auto-tuning
 * method's arithmetic (no SpMV, no feature, no format conversion), so both the
 * CPU oracle and the CUDA library can be fed from it.
 *
 * Structure classes stand in for the application classes of the sparse-matrix
 * collection the paper studies (Table "Application distribution of UF
 * collection", Sec. 2.2): 2-D / 3-D PDE stencils, uniform random graphs,
 * power-law (small-world) networks and dense block structure.
 *
 * Randomness: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  Every
 * draw is a pure function of (seed, row, purpose, index), so the output does
 * not depend on the number of threads that build it.
 *
 * Output rows hold sorted, unique column indices (canonical CSR).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11, Sec. 4): two 32x32->64 multiplies per round, a     */
/* Weyl-sequence key schedule, 10 rounds.                                    */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
  uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void synth_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k[0] += PHILOX_W0;
      k[1] += PHILOX_W1;
    }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof(c));
}

/* Purposes (third counter word) keep independent draws apart. */
enum { P_ROWLEN = 1, P_COLS = 2, P_VALS = 3, P_VEC = 4, P_META = 5 };

static void draw(uint64_t seed, uint64_t row, uint32_t purpose, uint32_t idx, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)row, (uint32_t)(row >> 32), purpose, idx};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  synth_philox4x32_10(ctr, key, out);
}

/* 53-bit uniform in the open interval (0, 1) from two 32-bit words. */
static double u01(uint32_t a, uint32_t b) {
  uint64_t m = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return ((double)m + 0.5) * (1.0 / 9007199254740992.0);
}

/* Uniform integer in [0, n) from two words (multiply-high, bias < n / 2^64). */
static int64_t uint_below(uint32_t a, uint32_t b, int64_t n) {
  uint64_t r = ((uint64_t)a << 32) | b;
  return (int64_t)(((unsigned __int128)r * (uint64_t)n) >> 64);
}

/* ------------------------------------------------------------------------ */
/* Generator kinds and their parameters p[]                                  */
/*   SYN_STENCIL2D5   p0 = mx, p1 = my        values 4 / -1                  */
/*   SYN_STENCIL3D7   p0 = m  (m^3 grid)      values 6 / -1                  */
/*   SYN_STENCIL3D27  p0 = m  (m^3 grid)      values 26 / -1                 */
/*   SYN_UNIFORM      p0 = n, p1 = lambda     Poisson(lambda) row lengths    */
/*   SYN_POWERLAW     p0 = n, p1 = alpha, p2 = kmax   Zipf(alpha) on [1,kmax] */
/*   SYN_BLOCKDIAG    p0 = n, p1 = b          dense b x b diagonal blocks    */
/*   SYN_BOX3D        p0 = m, p1 = r          (2r+1)^3-point box stencil on  */
/*                    an m^3 grid, values (2r+1)^3-1 / -1 (r = 1 is the      */
/*                    27-point stencil); the wide operators of coarse        */
/*                    multigrid levels                                       */
/* Random kinds draw columns uniformly without replacement and N(0,1) values. */
/* Stencils use natural (x fastest) ordering and Dirichlet boundaries.       */
/* ------------------------------------------------------------------------ */
enum { SYN_STENCIL2D5 = 0, SYN_STENCIL3D7 = 1, SYN_STENCIL3D27 = 2,
       SYN_UNIFORM = 3, SYN_POWERLAW = 4, SYN_BLOCKDIAG = 5, SYN_BOX3D = 6 };

typedef struct {
  int kind;
  double p[4];
  uint64_t seed;
  int64_t n_rows, n_cols;
  int32_t *rowlen;        /* phase 1 output */
  const int64_t *rowptr;  /* phase 2 input  */
  int32_t *colidx;        /* phase 2 output */
  double *val;            /* phase 2 output */
  const double *zipf_cdf; /* power-law only */
  int64_t zipf_k;
  int64_t r0, r1;
  int err;
} job_t;

int64_t synth_dims(int kind, const double *p, int64_t *n_rows, int64_t *n_cols) {
  int64_t r = 0;
  switch (kind) {
    case SYN_STENCIL2D5: r = (int64_t)p[0] * (int64_t)p[1]; break;
    case SYN_STENCIL3D7:
    case SYN_STENCIL3D27:
    case SYN_BOX3D: { int64_t m = (int64_t)p[0]; r = m * m * m; } break;
    case SYN_UNIFORM:
    case SYN_POWERLAW:
    case SYN_BLOCKDIAG: r = (int64_t)p[0]; break;
    default: return -1;
  }
  *n_rows = r;
  *n_cols = r;
  return r;
}

static int32_t poisson_draw(double lambda, double u, double z) {
  if (lambda <= 0.0) return 0;
  if (lambda <= 64.0) { /* inversion of the CDF */
    double p = exp(-lambda), F = p;
    int32_t k = 0;
    while (u > F && k < 100000) {
      ++k;
      p *= lambda / (double)k;
      F += p;
      if (p == 0.0) break;
    }
    return k;
  }
  /* large mean: normal approximation N(lambda, lambda), rounded */
  double v = floor(lambda + sqrt(lambda) * z + 0.5);
  if (v < 0.0) v = 0.0;
  if (v > 2147483647.0) v = 2147483647.0;
  return (int32_t)v;
}

static void gauss_pair(uint32_t w[4], double *z0, double *z1) {
  double u1 = u01(w[0], w[1]), u2 = u01(w[2], w[3]);
  double r = sqrt(-2.0 * log(u1));
  double t = 6.283185307179586476925286766559 * u2;
  *z0 = r * cos(t);
  *z1 = r * sin(t);
}

/* Grid points within r of coordinate c on a line of m points. */
static int64_t box_span(int64_t c, int64_t m, int64_t r) {
  int64_t lo = c - r < 0 ? 0 : c - r, hi = c + r > m - 1 ? m - 1 : c + r;
  return hi - lo + 1;
}

static int64_t stencil_len(int kind, const double *p, int64_t i) {
  if (kind == SYN_STENCIL2D5) {
    int64_t mx = (int64_t)p[0], my = (int64_t)p[1];
    int64_t ix = i % mx, iy = i / mx;
    return 1 + (ix > 0) + (ix < mx - 1) + (iy > 0) + (iy < my - 1);
  }
  int64_t m = (int64_t)p[0];
  int64_t ix = i % m, iy = (i / m) % m, iz = i / (m * m);
  if (kind == SYN_BOX3D) {
    int64_t r = (int64_t)p[1];
    int64_t nx = box_span(ix, m, r), ny = box_span(iy, m, r), nz = box_span(iz, m, r);
    return nx * ny * nz;
  }
  if (kind == SYN_STENCIL3D7)
    return 1 + (ix > 0) + (ix < m - 1) + (iy > 0) + (iy < m - 1) + (iz > 0) + (iz < m - 1);
  int64_t nx = 1 + (ix > 0) + (ix < m - 1), ny = 1 + (iy > 0) + (iy < m - 1),
          nz = 1 + (iz > 0) + (iz < m - 1);
  return nx * ny * nz;
}

static void stencil_fill(int kind, const double *p, int64_t i, int32_t *col, double *val) {
  int64_t k = 0;
  if (kind == SYN_STENCIL2D5) {
    int64_t mx = (int64_t)p[0], my = (int64_t)p[1];
    int64_t ix = i % mx, iy = i / mx;
    if (iy > 0) { col[k] = (int32_t)(i - mx); val[k++] = -1.0; }
    if (ix > 0) { col[k] = (int32_t)(i - 1); val[k++] = -1.0; }
    col[k] = (int32_t)i; val[k++] = 4.0;
    if (ix < mx - 1) { col[k] = (int32_t)(i + 1); val[k++] = -1.0; }
    if (iy < my - 1) { col[k] = (int32_t)(i + mx); val[k++] = -1.0; }
    return;
  }
  int64_t m = (int64_t)p[0], m2 = m * m;
  int64_t ix = i % m, iy = (i / m) % m, iz = i / m2;
  if (kind == SYN_STENCIL3D7) {
    if (iz > 0) { col[k] = (int32_t)(i - m2); val[k++] = -1.0; }
    if (iy > 0) { col[k] = (int32_t)(i - m); val[k++] = -1.0; }
    if (ix > 0) { col[k] = (int32_t)(i - 1); val[k++] = -1.0; }
    col[k] = (int32_t)i; val[k++] = 6.0;
    if (ix < m - 1) { col[k] = (int32_t)(i + 1); val[k++] = -1.0; }
    if (iy < m - 1) { col[k] = (int32_t)(i + m); val[k++] = -1.0; }
    if (iz < m - 1) { col[k] = (int32_t)(i + m2); val[k++] = -1.0; }
    return;
  }
  /* 27-point (r = 1) and box stencils: every grid point within r in each
     coordinate, in ascending column order */
  const int64_t r = kind == SYN_BOX3D ? (int64_t)p[1] : 1;
  const double centre = (double)((2 * r + 1) * (2 * r + 1) * (2 * r + 1) - 1);
  for (int64_t dz = -r; dz <= r; ++dz) {
    if (iz + dz < 0 || iz + dz >= m) continue;
    for (int64_t dy = -r; dy <= r; ++dy) {
      if (iy + dy < 0 || iy + dy >= m) continue;
      for (int64_t dx = -r; dx <= r; ++dx) {
        if (ix + dx < 0 || ix + dx >= m) continue;
        col[k] = (int32_t)(i + dz * m2 + dy * m + dx);
        val[k++] = (dx == 0 && dy == 0 && dz == 0) ? centre : -1.0;
      }
    }
  }
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

static void sort_i32(int32_t *a, int64_t n) {
  if (n < 32) {
    for (int64_t i = 1; i < n; ++i) {
      int32_t v = a[i];
      int64_t j = i - 1;
      while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
      a[j + 1] = v;
    }
  } else {
    qsort(a, (size_t)n, sizeof(int32_t), cmp_i32);
  }
}

/* rd distinct columns of [0, n), sorted, as a pure function of (seed, row). */
static void uniform_columns(uint64_t seed, int64_t row, int64_t n, int64_t rd, int32_t *col) {
  if (rd <= 0) return;
  if (2 * rd > n) { /* selection sampling (Knuth, TAOCP Vol. 2, Algorithm S) */
    int64_t need = rd, k = 0;
    uint32_t w[4];
    for (int64_t j = 0; j < n && need > 0; ++j) {
      if ((j & 1) == 0) draw(seed, (uint64_t)row, P_COLS | (0xFFu << 8), (uint32_t)(j >> 1), w);
      double u = (j & 1) ? u01(w[2], w[3]) : u01(w[0], w[1]);
      if ((double)(n - j) * u < (double)need) { col[k++] = (int32_t)j; --need; }
    }
    return;
  }
  int64_t have = 0;
  uint32_t round = 0;
  while (have < rd) {
    uint32_t w[4];
    for (int64_t j = have; j < rd; ++j) {
      int64_t t = j - have;
      if ((t & 1) == 0) draw(seed, (uint64_t)row, P_COLS | (round << 8), (uint32_t)(t >> 1), w);
      col[j] = (int32_t)((t & 1) ? uint_below(w[2], w[3], n) : uint_below(w[0], w[1], n));
    }
    sort_i32(col, rd);
    int64_t u = 0;
    for (int64_t j = 0; j < rd; ++j)
      if (u == 0 || col[j] != col[u - 1]) col[u++] = col[j];
    have = u;
    ++round;
  }
}

static void *rowlen_worker(void *arg) {
  job_t *J = (job_t *)arg;
  for (int64_t i = J->r0; i < J->r1; ++i) {
    int64_t len = 0;
    switch (J->kind) {
      case SYN_STENCIL2D5:
      case SYN_STENCIL3D7:
      case SYN_STENCIL3D27:
      case SYN_BOX3D: len = stencil_len(J->kind, J->p, i); break;
      case SYN_UNIFORM: {
        uint32_t w[4];
        draw(J->seed, (uint64_t)i, P_ROWLEN, 0, w);
        double z0, z1;
        uint32_t w2[4] = {w[0], w[1], w[2], w[3]};
        gauss_pair(w2, &z0, &z1);
        len = poisson_draw(J->p[1], u01(w[0], w[1]), z0);
        if (len > J->n_cols) len = J->n_cols;
      } break;
      case SYN_POWERLAW: {
        uint32_t w[4];
        draw(J->seed, (uint64_t)i, P_ROWLEN, 0, w);
        double u = u01(w[0], w[1]) * J->zipf_cdf[J->zipf_k - 1];
        int64_t lo = 0, hi = J->zipf_k - 1; /* first k with cdf[k] >= u */
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (J->zipf_cdf[mid] >= u) hi = mid; else lo = mid + 1;
        }
        len = lo + 1;
      } break;
      case SYN_BLOCKDIAG: {
        int64_t b = (int64_t)J->p[1], s = (i / b) * b;
        len = (J->n_cols - s < b) ? J->n_cols - s : b;
      } break;
    }
    J->rowlen[i] = (int32_t)len;
  }
  return NULL;
}

static void *fill_worker(void *arg) {
  job_t *J = (job_t *)arg;
  for (int64_t i = J->r0; i < J->r1; ++i) {
    int64_t s = J->rowptr[i], len = J->rowptr[i + 1] - s;
    int32_t *col = J->colidx + s;
    double *val = J->val + s;
    switch (J->kind) {
      case SYN_STENCIL2D5:
      case SYN_STENCIL3D7:
      case SYN_STENCIL3D27:
      case SYN_BOX3D: stencil_fill(J->kind, J->p, i, col, val); continue;
      case SYN_UNIFORM:
      case SYN_POWERLAW: uniform_columns(J->seed, i, J->n_cols, len, col); break;
      case SYN_BLOCKDIAG: {
        int64_t b = (int64_t)J->p[1], s0 = (i / b) * b;
        for (int64_t k = 0; k < len; ++k) col[k] = (int32_t)(s0 + k);
      } break;
    }
    uint32_t w[4];
    for (int64_t k = 0; k < len; k += 2) {
      draw(J->seed, (uint64_t)i, P_VALS, (uint32_t)(k >> 1), w);
      double z0, z1;
      gauss_pair(w, &z0, &z1);
      val[k] = z0;
      if (k + 1 < len) val[k + 1] = z1;
    }
  }
  return NULL;
}

static int nthreads_auto(int nt) {
  if (nt > 0) return nt;
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  if (c < 1) c = 1;
  if (c > 64) c = 64;
  return (int)c;
}

static int run_jobs(job_t *proto, int64_t n_rows, int nthreads, void *(*fn)(void *)) {
  int nt = nthreads_auto(nthreads);
  if (n_rows < 4096) nt = 1;
  job_t *jobs = (job_t *)calloc((size_t)nt, sizeof(job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -2; }
  for (int t = 0; t < nt; ++t) {
    jobs[t] = *proto;
    jobs[t].r0 = n_rows * t / nt;
    jobs[t].r1 = n_rows * (t + 1) / nt;
  }
  for (int t = 1; t < nt; ++t)
    if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) { jobs[t].err = 1; fn(&jobs[t]); }
  fn(&jobs[0]);
  for (int t = 1; t < nt; ++t)
    if (!jobs[t].err) pthread_join(th[t], NULL);
  free(jobs);
  free(th);
  return 0;
}

static double *zipf_table(double alpha, int64_t kmax) {
  double *cdf = (double *)malloc((size_t)kmax * sizeof(double));
  if (!cdf) return NULL;
  double acc = 0.0;
  for (int64_t k = 1; k <= kmax; ++k) {
    acc += pow((double)k, -alpha);
    cdf[k - 1] = acc;
  }
  return cdf;
}

/* Mean of Zipf(alpha) truncated to [1, kmax]. */
double synth_zipf_mean(double alpha, int64_t kmax) {
  double s0 = 0.0, s1 = 0.0;
  for (int64_t k = 1; k <= kmax; ++k) {
    double w = pow((double)k, -alpha);
    s0 += w;
    s1 += w * (double)k;
  }
  return s1 / s0;
}

/* Phase 1: row lengths.  Returns 0 on success. */
int synth_rowlen(int kind, const double *p, uint64_t seed, int32_t *rowlen, int nthreads) {
  job_t J;
  memset(&J, 0, sizeof(J));
  J.kind = kind;
  memcpy(J.p, p, sizeof(J.p));
  J.seed = seed;
  if (synth_dims(kind, p, &J.n_rows, &J.n_cols) < 0) return -1;
  J.rowlen = rowlen;
  double *cdf = NULL;
  if (kind == SYN_POWERLAW) {
    int64_t kmax = (int64_t)p[2];
    if (kmax > J.n_cols) kmax = J.n_cols;
    if (kmax < 1) kmax = 1;
    cdf = zipf_table(p[1], kmax);
    if (!cdf) return -2;
    J.zipf_cdf = cdf;
    J.zipf_k = kmax;
  }
  int rc = run_jobs(&J, J.n_rows, nthreads, rowlen_worker);
  free(cdf);
  return rc;
}

/* Phase 2: columns and values, given rowptr = exclusive scan of the lengths. */
int synth_fill(int kind, const double *p, uint64_t seed, const int64_t *rowptr,
               int32_t *colidx, double *val, int nthreads) {
  job_t J;
  memset(&J, 0, sizeof(J));
  J.kind = kind;
  memcpy(J.p, p, sizeof(J.p));
  J.seed = seed;
  if (synth_dims(kind, p, &J.n_rows, &J.n_cols) < 0) return -1;
  J.rowptr = rowptr;
  J.colidx = colidx;
  J.val = val;
  return run_jobs(&J, J.n_rows, nthreads, fill_worker);
}

/* n values uniform on [lo, hi), keyed by (seed, stream). */
void synth_uniform(uint64_t seed, uint32_t stream, int64_t n, double lo, double hi, double *out) {
  uint32_t w[4];
  for (int64_t i = 0; i < n; i += 2) {
    draw(seed, (uint64_t)(i >> 1), P_VEC, stream, w);
    out[i] = lo + (hi - lo) * u01(w[0], w[1]);
    if (i + 1 < n) out[i + 1] = lo + (hi - lo) * u01(w[2], w[3]);
  }
}

/* n standard normal values keyed by (seed, stream). */
void synth_normal(uint64_t seed, uint32_t stream, int64_t n, double *out) {
  uint32_t w[4];
  for (int64_t i = 0; i < n; i += 2) {
    draw(seed, (uint64_t)(i >> 1), P_META, stream, w);
    double z0, z1;
    gauss_pair(w, &z0, &z1);
    out[i] = z0;
    if (i + 1 < n) out[i + 1] = z1;
  }
}
