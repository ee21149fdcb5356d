/* A plain C program against include/smat.h: builds a 2-D 5-point Laplacian
 * in host memory, creates a handle, tunes it exhaustively and multiplies
 * y = 2*A*x - y with host buffers.  Prints the plan and y[0..3] so the test can
 * compare them with the oracle.  Exit code = first failing status (0 = ok). */
#include <stdio.h>
#include <stdlib.h>

#include "smat.h"

#define CHECK(call)                                                            \
  do {                                                                         \
    smat_status_t s_ = (call);                                                 \
    if (s_ != SMAT_OK) {                                                       \
      fprintf(stderr, "%s: %s\n", #call, smat_status_string(s_));               \
      return (int)s_;                                                          \
    }                                                                          \
  } while (0)

int main(void) {
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
  CHECK(smat_destroy(h));
  free(rowptr); free(col); free(val); free(x); free(y);
  return 0;
}
