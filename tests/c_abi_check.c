/* A plain C program against include/smat.h.
 * Part 1: builds a 2-D 5-point Laplacian in host memory, creates a handle,
 * tunes it exhaustively and multiplies y = 2*A*x - y with host buffers;
 * prints the plan and y[0..3] so the test can compare them with the oracle.
 * Part 2: a random matrix with non-integer values (3000 x 2500, 0..20
 * entries per row, some rows empty) placed in DEVICE memory with the CUDA
 * runtime, handed to smat_create as device pointers, tuned, and multiplied by
 * smat_spmv on device vectors (y = -0.75*A*x + 0.5*y); the matrix, x, y0 and
 * the product go to the file named by argv[1] for a row-by-row check.
 * Part 3: device CSR with a row whose columns are not increasing must be
 * refused with SMAT_ERR_INVALID_CSR.
 * Part 4: on the part-1 handle, three smat_spmv_host_pipelined calls with
 * different pinned x (the handle's two staging sets in turn, y = A*x and
 * y = 0.5*A*x - y), then one synchronisation of the default stream; each y
 * must equal the synchronous smat_spmv_host result bit for bit.
 * Exit code = first failing status (0 = ok). */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "smat.h"

#define CHECK(call)                                                            \
  do {                                                                         \
    smat_status_t s_ = (call);                                                 \
    if (s_ != SMAT_OK) {                                                       \
      fprintf(stderr, "%s: %s\n", #call, smat_status_string(s_));               \
      return (int)s_;                                                          \
    }                                                                          \
  } while (0)

#define CUDA_CHECK(call)                                                       \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));               \
      return 100;                                                              \
    }                                                                          \
  } while (0)

/* 64-bit linear congruential generator (Knuth's MMIX constants), top bits */
static uint64_t lcg_state = 0x9E3779B97F4A7C15ull;
static uint32_t lcg_next(void) {
  lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
  return (uint32_t)(lcg_state >> 33);
}

static void *to_device(const void *host, size_t bytes) {
  void *d = NULL;
  if (cudaMalloc(&d, bytes ? bytes : 16) != cudaSuccess) return NULL;
  if (bytes && cudaMemcpy(d, host, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return NULL;
  return d;
}

static int part2(const char *path) {
  const int m = 3000, n = 2500;
  int32_t *rowptr = malloc(sizeof(int32_t) * (m + 1));
  int32_t *col = malloc(sizeof(int32_t) * 21 * (size_t)m);
  double *val = malloc(sizeof(double) * 21 * (size_t)m);
  double *x = malloc(sizeof(double) * n), *y0 = malloc(sizeof(double) * m), *y = malloc(sizeof(double) * m);
  int32_t k = 0;
  for (int i = 0; i < m; ++i) {
    rowptr[i] = k;
    const int len = (int)(lcg_next() % 21);          /* 0..20 entries */
    int c = (int)(lcg_next() % 97);
    for (int t = 0; t < len && c < n; ++t) {          /* strictly increasing columns */
      col[k] = c;
      val[k++] = ((double)lcg_next() / 2147483648.0 - 0.5) * 3.7;
      c += 1 + (int)(lcg_next() % 211);
    }
  }
  rowptr[m] = k;
  for (int j = 0; j < n; ++j) x[j] = (double)lcg_next() / 2147483648.0 - 0.5;
  for (int i = 0; i < m; ++i) y0[i] = (double)lcg_next() / 2147483648.0 - 0.5;
  int32_t *d_rp = to_device(rowptr, sizeof(int32_t) * (m + 1));
  int32_t *d_col = to_device(col, sizeof(int32_t) * (size_t)k);
  double *d_val = to_device(val, sizeof(double) * (size_t)k);
  double *d_x = to_device(x, sizeof(double) * n), *d_y = to_device(y0, sizeof(double) * m);
  if (!d_rp || !d_col || !d_val || !d_x || !d_y) return 101;
  smat_handle_t h = NULL;
  CHECK(smat_create(&h, m, n, k, d_rp, d_col, d_val, SMAT_F64));
  smat_tune_opts_t o;
  smat_tune_opts_default(&o);
  o.mode = SMAT_TUNE_EXHAUSTIVE;
  o.trial_reps = 3;
  CHECK(smat_tune(h, &o, NULL));
  int32_t variant = -1, trialled = 0;
  double tune_ms = 0.0;
  float conf = 0.0f;
  CHECK(smat_get_plan(h, &variant, &tune_ms, &conf, &trialled));
  const double alpha = -0.75, beta = 0.5;
  CHECK(smat_spmv(h, &alpha, d_x, &beta, d_y, NULL));
  CUDA_CHECK(cudaDeviceSynchronize());
  CUDA_CHECK(cudaMemcpy(y, d_y, sizeof(double) * m, cudaMemcpyDeviceToHost));
  CHECK(smat_destroy(h));
  FILE *fo = fopen(path, "wb");
  if (!fo) return 102;
  const int64_t dims[3] = {m, n, k};
  fwrite(dims, sizeof(int64_t), 3, fo);
  fwrite(rowptr, sizeof(int32_t), (size_t)m + 1, fo);
  fwrite(col, sizeof(int32_t), (size_t)k, fo);
  fwrite(val, sizeof(double), (size_t)k, fo);
  fwrite(x, sizeof(double), (size_t)n, fo);
  fwrite(y0, sizeof(double), (size_t)m, fo);
  fwrite(y, sizeof(double), (size_t)m, fo);
  fclose(fo);
  printf("part2 nnz %d variant %d\n", (int)k, variant);
  cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val); cudaFree(d_x); cudaFree(d_y);
  free(rowptr); free(col); free(val); free(x); free(y0); free(y);
  return 0;
}

static int part3(void) {
  /* row 1 holds columns 3, 1: not increasing */
  const int32_t rowptr[4] = {0, 1, 3, 4}, col[4] = {0, 3, 1, 2};
  const double val[4] = {1.0, 2.0, 3.0, 4.0};
  int32_t *d_rp = to_device(rowptr, sizeof rowptr), *d_col = to_device(col, sizeof col);
  double *d_val = to_device(val, sizeof val);
  if (!d_rp || !d_col || !d_val) return 103;
  smat_handle_t h = NULL;
  const smat_status_t st = smat_create(&h, 3, 4, 4, d_rp, d_col, d_val, SMAT_F64);
  printf("part3 status %d handle %s\n", (int)st, h ? "set" : "null");
  cudaFree(d_rp); cudaFree(d_col); cudaFree(d_val);
  return st == SMAT_ERR_INVALID_CSR && !h ? 0 : 104;
}

static int part4(smat_handle_t h, int m) {
  double *xs = NULL, *ys = NULL;
  if (cudaMallocHost((void **)&xs, sizeof(double) * 3 * (size_t)m) != cudaSuccess) return 105;
  if (cudaMallocHost((void **)&ys, sizeof(double) * 3 * (size_t)m) != cudaSuccess) return 105;
  double *ref = malloc(sizeof(double) * (size_t)m);
  const double alphas[3] = {1.0, 0.5, -2.0}, betas[3] = {0.0, -1.0, 0.0};
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < m; ++i) {
      xs[(size_t)c * m + i] = (double)((i * (c + 3)) % 11) - 5.0 + 0.25 * c;
      ys[(size_t)c * m + i] = (double)(i % 3);
    }
  for (int c = 0; c < 3; ++c)
    CHECK(smat_spmv_host_pipelined(h, &alphas[c], xs + (size_t)c * m, &betas[c], ys + (size_t)c * m, NULL));
  CUDA_CHECK(cudaStreamSynchronize(NULL));
  int bad = 0;
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < m; ++i) ref[i] = (double)(i % 3);
    CHECK(smat_spmv_host(h, &alphas[c], xs + (size_t)c * m, &betas[c], ref, NULL));
    for (int i = 0; i < m; ++i) bad += ref[i] != ys[(size_t)c * m + i];
  }
  printf("part4 mismatches %d\n", bad);
  cudaFreeHost(xs); cudaFreeHost(ys); free(ref);
  return bad ? 106 : 0;
}

int main(int argc, char **argv) {
  const int g = 32, m = g * g;
  int32_t *rowptr = malloc(sizeof(int32_t) * (m + 1));
  int32_t *col = malloc(sizeof(int32_t) * 5 * m);
  double *val = malloc(sizeof(double) * 5 * m), *x = malloc(sizeof(double) * m), *y = malloc(sizeof(double) * m);
  int k = 0;
  for (int i = 0; i < m; ++i) {
    int ix = i % g, iy = i / g;
    rowptr[i] = k;
    if (iy > 0) { col[k] = i - g; val[k++] = -1.0; }
    if (ix > 0) { col[k] = i - 1; val[k++] = -1.0; }
    col[k] = i; val[k++] = 4.0;
    if (ix < g - 1) { col[k] = i + 1; val[k++] = -1.0; }
    if (iy < g - 1) { col[k] = i + g; val[k++] = -1.0; }
    x[i] = (double)(i % 7) - 3.0;
    y[i] = 1.0;
  }
  rowptr[m] = k;
  smat_handle_t h = NULL;
  CHECK(smat_create(&h, m, m, k, rowptr, col, val, SMAT_F64));
  smat_tune_opts_t o;
  smat_tune_opts_default(&o);
  o.mode = SMAT_TUNE_EXHAUSTIVE;
  o.trial_reps = 3;
  CHECK(smat_tune(h, &o, NULL));
  smat_features_t f;
  CHECK(smat_get_features(h, &f));
  int32_t variant = -1, trialled = 0;
  double tune_ms = 0.0;
  float conf = 0.0f;
  CHECK(smat_get_plan(h, &variant, &tune_ms, &conf, &trialled));
  const double alpha = 2.0, beta = -1.0;
  CHECK(smat_spmv_host(h, &alpha, x, &beta, y, NULL));
  printf("nnz %lld ndiags %lld variant %d\n", (long long)f.nnz, (long long)f.ndiags, variant);
  printf("y %.17g %.17g %.17g %.17g\n", y[0], y[1], y[g], y[m - 1]);
  const int r4 = argc > 1 ? part4(h, m) : 0;
  if (r4) return r4;
  CHECK(smat_destroy(h));
  free(rowptr); free(col); free(val); free(x); free(y);
  if (argc > 1) {
    const int r2 = part2(argv[1]);
    if (r2) return r2;
    return part3();
  }
  return 0;
}
