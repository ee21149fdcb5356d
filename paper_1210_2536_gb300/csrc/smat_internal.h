// Internal declarations shared by the libsmat translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "smat.h"

namespace smat {

// Storage element size per dtype.
inline int elem_size(smat_dtype_t t) { return t == SMAT_F64 ? 8 : (t == SMAT_F32 ? 4 : 2); }
inline int64_t pitch_of(int64_t m) { return (m + 31) / 32 * 32; }

// Device allocation with a host-side failure hook (smat_test_fail_alloc_after)
// that makes a chosen allocation fail, for error-path tests.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);

// Plan cache (plan_cache.cu): the structural key, computed once per handle,
// and the process-wide table of plans.
smat_status_t ensure_plan_key(smat_s *h, cudaStream_t s);
bool plan_cache_lookup(const smat_s *h, int *variant, int *sell_sigma);
void plan_cache_store(const smat_s *h, int variant, int sell_sigma);

// Device-side error flags set by validation kernels (never trap).
enum : int {
  ERRF_ROWPTR = 1,     // rowptr[0] != 0, rowptr[m] != nnz or decreasing
  ERRF_COL_RANGE = 2,  // column outside [0, n)
  ERRF_COL_ORDER = 4,  // columns not strictly increasing in a row
};

// Integer statistics of the row degrees (one pass over rowptr).
struct RowStats {
  unsigned long long s2;  // sum of rd^2
  int max_rd;
  int min_rd;
  int empty_rows;
  int pad;
};

// Selector model (process-wide).
struct Model {
  bool loaded = false;
  float mean[12], stdv[12];
  float params[SMAT_MLP_PARAMS];
};
Model &model();

}  // namespace smat

// The handle.
struct smat_s {
  int64_t m = 0, n = 0, nnz = 0;
  smat_dtype_t dtype = SMAT_F64;
  int esz = 8;
  int64_t P = 0;  // pitch of ELL / DIA arrays

  // CSR (always present)
  int32_t *rowptr = nullptr, *colidx = nullptr;
  void *val = nullptr;

  // structural key of the plan cache (the structure never changes)
  uint64_t plan_key = 0;
  bool have_plan_key = false;
  bool plan_cached = false;  // the last smat_tune took its plan from the cache

  // features
  bool have_features = false;
  smat_features_t f{};
  std::vector<int64_t> hist;         // row-degree histogram
  std::vector<int32_t> dia_offsets;  // occupied diagonals, ascending (when counted)
  bool dia_offsets_complete = false;
  int32_t tau_num = 3, tau_den = 5;
  int32_t fill_ratio_max = 20;
  double bytes_cap = 4.0;

  // ELL
  int64_t ell_K = 0;
  int ell_u = 0, dia_u = 0;  // measured batch widths (0: not measured yet)
  int ell_lane = 0;          // measured ELL row mapping: 0 consecutive rows per thread, 1 lane-striped
  int dia_staged = 0;        // measured DIA kernel: 0 direct loads, 1.. stripes staged by bulk copies (shape id)
  int32_t *ell_col = nullptr;
  void *ell_val = nullptr;
  // DIA
  int64_t dia_nd = 0;
  int32_t *dia_off = nullptr;
  void *dia_val = nullptr;
  // COO
  int32_t *coo_row = nullptr;
  int32_t *coo_empty = nullptr;  // list of empty rows (y = beta*y there)
  int64_t coo_nempty = 0;

  // HYB: ELL part (K x P) + COO part
  int64_t hyb_K = 0, hyb_ncoo = 0;
  int32_t *hyb_ecol = nullptr, *hyb_crow = nullptr, *hyb_ccol = nullptr;
  void *hyb_eval = nullptr, *hyb_cval = nullptr;
  bool hyb_built = false;
  // SELL-32-sigma: layout (perm, width, slice pointers) then col / val
  int32_t sell_sigma = 256;
  int64_t sell_ns = 0, sell_slots = 0;
  int32_t *sell_perm = nullptr, *sell_width = nullptr, *sell_col = nullptr;
  long long *sell_ptr = nullptr;
  void *sell_val = nullptr;
  // BCSR: block size, block rows, blocks; 64-bit block row starts until filled
  int32_t bcsr_b = 0;
  int64_t bcsr_mb = 0, bcsr_nb = 0;
  long long *bcsr_brp64 = nullptr;
  int32_t bcsr_cb = 0;  // blocks in every block row when all block rows hold the same count, else 0
  int32_t *bcsr_rowptr = nullptr, *bcsr_col = nullptr;
  void *bcsr_val = nullptr;
  // SPLIT: rows of >= SPLIT_L entries in chunks of <= SPLIT_CK, short rows as COO
  int64_t split_nl = 0, split_nc = 0, split_ns = 0, split_ne = 0;
  int32_t *split_lchunk = nullptr;  // first chunk of each long row, nl + 1 values
  int32_t *split_lrows = nullptr, *split_crow = nullptr, *split_cstart = nullptr, *split_cend = nullptr;
  int32_t *split_srow = nullptr, *split_scol = nullptr, *split_empty = nullptr;
  void *split_sval = nullptr, *split_part = nullptr;
  bool split_built = false;
  // measured layouts of HYB / SELL / BCSR / SPLIT (index v - SMAT_V_HYB):
  // stored slots (fill included) and bytes, for their admissibility bits
  bool ext_known[4] = {false, false, false, false};
  double ext_slots[4] = {0, 0, 0, 0}, ext_bytes[4] = {0, 0, 0, 0};

  // merge-path tile coordinates (int2 per tile boundary), computed once
  void *merge_coords = nullptr;
  // scratch for merge-path and COO carries
  void *carry = nullptr;
  size_t carry_bytes = 0;
  // The buffers above serve the first stream that runs products on the
  // handle; every further stream gets scratch of its own on its first product
  // there, so products on different streams never share carries.
  struct StreamScratch {
    cudaStream_t stream;
    void *p;
    size_t bytes;
  };
  mutable std::mutex scratch_mu;
  mutable bool scratch_owned = false;
  mutable cudaStream_t scratch_owner = nullptr;
  mutable std::vector<StreamScratch> more_scratch;

  // host-buffer staging for smat_spmv_host
  void *stage_x = nullptr, *stage_y = nullptr;
  // smat_spmv_host_pipelined: two staging sets used in turn, the handle's own
  // copy-in, compute and copy-out streams, and per set the events that order
  // a set's next use after its previous one
  void *pstage_x[2] = {}, *pstage_y[2] = {};
  cudaStream_t pst[3] = {};
  cudaEvent_t pev_x[2] = {}, pev_run[2] = {}, pev_out[2] = {};
  bool pused[2] = {};
  long long pcalls = 0;

  // plan
  int32_t variant = SMAT_V_CSR_SCALAR;
  double tune_ms = 0.0;
  float confidence = -1.0f;
  int32_t trialled = 0;
  float timings[SMAT_NUM_ALL_VARIANTS];
};

namespace smat {

// ---- launchers (return cudaError_t of the launch) ----
// Validation writes its error flags to d_flag and uses d_starts, zeroed
// words of one bit per stored entry (validate_starts_words of them).
size_t validate_starts_words(int64_t nnz);
cudaError_t launch_validate(const smat_s *h, int *d_flag, unsigned *d_starts, cudaStream_t s);
cudaError_t launch_row_stats(const int32_t *rowptr, int64_t m, RowStats *d_stats, cudaStream_t s);
cudaError_t launch_hist_diag(const int32_t *rowptr, const int32_t *colidx, int64_t m,
                             int *d_hist, int64_t hist_len, int *d_diag_cnt, cudaStream_t s);
cudaError_t launch_diag_reduce(const int *d_diag_cnt, int64_t m, int64_t n, int tau_num,
                               int tau_den, unsigned long long *d_counts, int32_t *d_offsets,
                               int64_t offsets_cap, cudaStream_t s);

cudaError_t launch_to_coo(const smat_s *h, int32_t *row, cudaStream_t s);
cudaError_t launch_empty_rows(const smat_s *h, int32_t *list, int *d_count, cudaStream_t s);
cudaError_t launch_to_ell(const smat_s *h, int64_t K, int32_t *col, void *val, cudaStream_t s);
cudaError_t launch_to_dia(const smat_s *h, const int32_t *d_off, int64_t nd, void *val,
                          cudaStream_t s);

// Further formats (formats_ext.cu).  exclusive_scan writes out[0..n] and
// synchronises `s`.
cudaError_t exclusive_scan(const long long *in, long long n, long long *out, cudaStream_t s);
cudaError_t launch_hyb_tail_counts(const smat_s *h, int64_t K, long long *cnt, cudaStream_t s);
cudaError_t launch_to_hyb(const smat_s *h, int64_t K, const long long *off, int32_t *ecol, void *eval,
                          int32_t *crow, int32_t *ccol, void *cval, cudaStream_t s);
cudaError_t launch_sell_layout(const smat_s *h, int sigma, int32_t *perm, int32_t *width, long long *cnt,
                               cudaStream_t s);
cudaError_t launch_to_sell(const smat_s *h, cudaStream_t s);
cudaError_t launch_bcsr_count(const smat_s *h, int b, long long *cnt, cudaStream_t s);
#ifndef SMAT_SPLIT_L
#define SMAT_SPLIT_L 1024
#endif
constexpr int64_t SPLIT_L = SMAT_SPLIT_L, SPLIT_CK = 4096;
// SPLIT conversion: per-row counts (long flag, chunks, short entries, empty
// flag) for the scans, then the fill from their exclusive scans.
cudaError_t launch_split_counts(const smat_s *h, long long *cl, long long *cc, long long *cs, long long *ce,
                                cudaStream_t s);
cudaError_t launch_split_fill(const smat_s *h, const long long *pl, const long long *pc, const long long *ps,
                              const long long *pe, cudaStream_t s);
cudaError_t launch_to_bcsr(const smat_s *h, const long long *brp, cudaStream_t s);
// Sets *flag (zeroed by the caller) when a block row of the built layout holds
// a block count other than c.
cudaError_t launch_bcsr_uniform(const smat_s *h, long long c, int *flag, cudaStream_t s);
// SELL / BCSR products (HYB runs through the ELL and COO kernels of spmv.cu).
cudaError_t launch_spmv_ext(const smat_s *h, int variant, const void *alpha, const void *x,
                            const void *beta, void *y, cudaStream_t s);

// Merge-path tiles of an m x ? matrix with nnz entries, and the kernel that
// writes their (ntiles + 1) boundary coordinates (int2) to `coords`.
long long merge_tiles(long long m, long long nnz);
cudaError_t launch_merge_partition(const int32_t *rowptr, long long m, long long nnz, void *coords,
                                   cudaStream_t s);
// Per-product scratch: carries (merge-path, COO, HYB and SPLIT tails) and
// SPLIT's chunk sums.
struct Scratch {
  void *carry;
  void *part;
};
// The scratch a product on stream s uses (see smat_s::more_scratch); a stream
// that is capturing a graph and has none yet gets cudaErrorStreamCaptureUnsupported.
// claim = false (the tuner's own products, which never overlap other calls)
// uses the handle's buffers without making s their owner.
cudaError_t stream_scratch(const smat_s *h, cudaStream_t s, Scratch *out, bool claim = true);
void free_stream_scratch(smat_s *h);
// Size in bytes of the carry scratch a variant needs (0 if none).
size_t carry_bytes_needed(const smat_s *h, int variant);
// Kernel launches one product through `variant` issues.
int spmv_launch_count(const smat_s *h, int variant);
// Candidate batch widths of an ELL / DIA product (returns how many: 1 or 2).
int batch_width_candidates(const smat_s *h, int variant, int out[2]);
// ELL / DIA product with an explicit batch width and (ELL) row mapping
// (lane: -1 the handle's, 0 consecutive rows per thread, 1 lane-striped; for
// DIA 2 + k is staged shape k), for measuring them.
cudaError_t launch_spmv_width(const smat_s *h, int variant, int u, int lane, const void *alpha, const void *x,
                              const void *beta, void *y, cudaStream_t s);
// DIA with its stripes staged in shared memory by bulk copies (staged.cu),
// in launch shapes 1..dia_staged_kernels(): whether the handle's DIA arrays
// fit shape `kernel`'s tiles, and the product (alpha/beta host scalars of the
// compute type; wait_limit in SM cycles, 0 for the default of about one second).
int dia_staged_kernels();
bool dia_staged_ok(const smat_s *h, int kernel);
cudaError_t launch_dia_staged(const smat_s *h, int kernel, const void *alpha, const void *x, const void *beta,
                              void *y, cudaStream_t s, long long wait_limit = 0);
// SpMV through one variant; alpha/beta are host scalars of the compute type.
// claim: as in stream_scratch (false for the tuner's timing products).
cudaError_t launch_spmv(const smat_s *h, int variant, const void *alpha, const void *x,
                        const void *beta, void *y, cudaStream_t s, bool claim = true);

// MLP forward over standardised inputs (device), used by the selector.
cudaError_t launch_mlp_forward(const float *params, const float *X, int B, float *logits,
                               cudaStream_t s);

// ---- timing support (measure.cu) ----
// Host wall clock in milliseconds (steady).
double host_ms();
// Holds stream s on the device for about `us` microseconds (clamped to
// [0, 4000]): one thread polls the global nanosecond timer, with short sleeps
// and a bounded number of polls, so it ends whatever the timer does.
cudaError_t launch_hold(cudaStream_t s, double us);
constexpr double HOLD_MAX_US = 4000.0;

// Queues timed work behind a device hold that outlasts the host's time to
// enqueue it, so that the GPU reaches the work only once all of it is queued
// and no host launch latency falls between a pair of timing events (a short
// kernel enqueued behind an idle GPU is otherwise timed together with the
// host's latency to submit it).  enqueue() issues `units` launches with their
// events and does not synchronise; *enq_us carries the host's enqueue time
// per unit from one call to the next.  When the enqueue outlasted the hold,
// the stream is drained and the same work queued again behind a hold sized
// from the enqueue just measured (three attempts at most).
template <typename F>
cudaError_t queue_ahead(cudaStream_t s, double *enq_us, int units, F &&enqueue) {
  const double n = units > 1 ? (double)units : 1.0;
  for (int attempt = 0;; ++attempt) {
    double hold = 20.0 + 1.5 * *enq_us * n;
    hold = hold < HOLD_MAX_US ? hold : HOLD_MAX_US;
    cudaError_t e = launch_hold(s, hold);
    if (e != cudaSuccess) return e;
    const double t0 = host_ms();
    e = enqueue();
    const double dt = (host_ms() - t0) * 1e3;
    if (e != cudaSuccess) return e;
    *enq_us = dt / n;
    if (dt < hold || attempt == 2) return cudaSuccess;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
  }
}

}  // namespace smat
