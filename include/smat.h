/*
 * smat.h -- C ABI of libsmat, an input-adaptive sparse matrix-vector multiply
 * library for NVIDIA GB300 (sm_103a), after SMAT (Li, Zhang, Tan, Chen,
 * "SMAT: An Input Adaptive Sparse Matrix-Vector Multiplication Auto-Tuner",
 * arXiv 1210.2536).
 *
 * The caller hands in a matrix in CSR only (Sec. 3: the unified CSR interface)
 * and asks for y = alpha*A*x + beta*y.  The library extracts the matrix's
 * feature parameters on the GPU (Sec. 4), chooses a storage format and kernel
 * (Sec. 5-6: a learned classifier with an execute-and-measure fallback),
 * converts CSR to that format (Sec. 2.1) and runs the product.
 *
 * Conventions for every entry point:
 *   - Plain C types only.  Streams are cudaStream_t passed as void*; NULL is
 *     the legacy default stream.
 *   - Every call returns an smat_status_t; no C++ exception crosses the ABI
 *     and no kernel traps.  Errors detected on the device (invalid CSR) are
 *     reported through a flag the host reads.
 *   - Indices are int32 (M, N, NNZ <= 2^31 - 1).  Rows must hold strictly
 *     increasing column indices (canonical CSR); anything else is
 *     SMAT_ERR_INVALID_CSR.
 *   - Value storage: SMAT_F64 computes in FP64 with FP64 x and y.  SMAT_F32 and
 *     SMAT_BF16 store values in FP32 / bfloat16 and compute with FP32
 *     accumulation, FP32 x and y, FP32 alpha and beta.
 *   - alpha and beta are HOST pointers to one scalar of the compute type.
 *     beta == 0 means y is only written (NaN in y is ignored, as in BLAS);
 *     alpha == 0 gives y = beta*y (0 when beta == 0) without reading A or x.
 *
 * Thread safety: calls on different handles are independent.  Products
 * (smat_spmv, smat_spmv_variant) on one handle may run concurrently from
 * different streams and host threads: the kernels that carry partial sums
 * between CTAs (merge-path, COO, HYB, SPLIT) use the handle's own scratch on
 * the first stream that runs products on it and scratch of their own on every
 * further stream, allocated on that stream's first product (so a stream that
 * is capturing a CUDA graph must have run a product on the handle before, or
 * be its first stream; otherwise the product reports SMAT_ERR_CUDA).
 * smat_tune, smat_convert, smat_destroy and the host-buffer products
 * (smat_spmv_host*, which share the handle's staging buffers) must not overlap
 * with other calls on the handle.  The selector model and the plan cache are
 * process-wide and guarded: smat_load_model / smat_set_model may run while
 * other threads tune (a tuning predicts from a copy of the model).
 */
#ifndef SMAT_H
#define SMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smat_s *smat_handle_t;
typedef struct smat_batch_s *smat_batch_t;
typedef struct smat_segments_s *smat_segments_t;

typedef enum {
  SMAT_OK = 0,
  SMAT_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, bad enum          */
  SMAT_ERR_INVALID_CSR = 2, /* rowptr not monotone / wrong ends, column out of
                               range, or columns not strictly increasing      */
  SMAT_ERR_ALLOC = 3,       /* device or host allocation failed               */
  SMAT_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed           */
  SMAT_ERR_UNSUPPORTED = 5, /* sizes beyond int32 indexing, format not
                               admissible for this matrix                      */
  SMAT_ERR_MODEL = 6,       /* selector model missing or malformed            */
  SMAT_ERR_NOT_CONVERGED = 7 /* iterative solve stopped before its tolerance  */
} smat_status_t;

typedef enum { SMAT_F64 = 0, SMAT_F32 = 1, SMAT_BF16 = 2 } smat_dtype_t;

/* Storage formats: the four basic formats of Sec. 2.1, then GPU formats of
 * the kind Sec. 8 leaves to future work (HYB: Bell & Garland's ELL + COO
 * split; SELL: Kreutzer et al.'s SELL-C-sigma with C = 32; BCSR: b x b blocks,
 * b in {2, 4, 8}; SPLIT: rows of at least 1024 entries in chunks of at most
 * 4096, each chunk summed by one CTA, the other rows as a COO). */
typedef enum {
  SMAT_FMT_CSR = 0, SMAT_FMT_ELL = 1, SMAT_FMT_DIA = 2, SMAT_FMT_COO = 3,
  SMAT_FMT_HYB = 4, SMAT_FMT_SELL = 5, SMAT_FMT_BCSR = 6, SMAT_FMT_SPLIT = 7
} smat_format_t;

/* Kernel variants the selector chooses among (the paper's kernel library maps
 * each format to its best implementation, Sec. 3).  On the GPU the CSR format
 * has five implementations. */
typedef enum {
  SMAT_V_CSR_SCALAR = 0, /* one thread per row                              */
  SMAT_V_CSR_VEC4 = 1,   /* 4 lanes per row, shuffle reduction              */
  SMAT_V_CSR_VEC8 = 2,   /* 8 lanes per row                                  */
  SMAT_V_CSR_VEC32 = 3,  /* one warp per row                                 */
  SMAT_V_CSR_MERGE = 4,  /* merge-path split of rows + nonzeros              */
  SMAT_V_ELL = 5,        /* column-major ELL, 16-byte vector loads           */
  SMAT_V_DIA = 6,        /* diagonal-major DIA                               */
  SMAT_V_COO = 7,        /* COO with segmented reduction                     */
  SMAT_NUM_VARIANTS = 8,
  /* Not a selector class: CSR-scalar that rounds every product and every
   * sum separately, in ascending column order -- the operations of the CSR
   * definition.  In FP64 its result is bitwise reproducible against a plain
   * sequential implementation; it costs two FP64 operations per nonzero
   * instead of one.  Only smat_spmv_variant runs it. */
  SMAT_V_CSR_SCALAR_EXACT = 8,
  /* Further formats (not classes of the learned selector, whose 8 classes
   * are fixed; the search times them beside its pick, see smat_tune). */
  SMAT_V_HYB = 9,        /* ELL part + COO tail                               */
  SMAT_V_SELL = 10,      /* SELL-32-sigma, a warp per slice                   */
  SMAT_V_BCSR = 11,      /* b x b blocks, b lanes per block row               */
  SMAT_V_SPLIT = 12,     /* long rows in CTA chunks + COO of the short rows   */
  SMAT_NUM_ALL_VARIANTS = 13
} smat_variant_t;

/* Feature parameters (Sec. 4, Table "Feature parameters of a sparse matrix").
 * Integer members are exact.  Each double is computed from exact integers:
 *   aver_rd = NNZ / M
 *   var_rd  = (M * S2 - NNZ^2) / M^2, S2 = sum of squared row degrees
 *             (population variance of the row degree)
 *   er_dia  = NNZ / (Ndiags * M),  er_ell = NNZ / (max_RD * M)
 *   ntdiags_ratio = (# diagonals filled above tau) / Ndiags
 * with each integer operand converted to double once and one division.
 *   r = -slope of the least-squares line through (ln k, ln h[k]) over row
 *       degrees k >= 1 with h[k] > 0 (P(k) ~ k^-R); r_valid = 0 and r = 0 when
 *       fewer than two degrees occur.
 * Ratios whose denominator is 0 are 0.
 * `admissible` bits 9-12 (HYB, SELL, BCSR, SPLIT) are set once the format's
 * layout has been measured (by smat_tune, smat_convert or a product through
 * it): each needs its stored slots (fill included) <= fill_ratio_max * NNZ
 * and its bytes <= bytes_cap * CSR bytes; HYB also an ELL width K >= 1, SPLIT
 * at least one row of 1024 or more entries. */
typedef struct {
  int64_t m, n, nnz;
  int64_t max_rd, min_rd, empty_rows;
  int64_t ndiags, ntdiags;
  uint64_t s2;
  double aver_rd, var_rd, er_dia, er_ell, ntdiags_ratio, r;
  int32_t r_valid;
  uint32_t admissible; /* bit v set: variant v may be used for this matrix */
} smat_features_t;

/* Selection modes for smat_tune. */
typedef enum {
  SMAT_TUNE_LEARNED = 0,    /* MLP over the features; execute-and-measure when its
                               confidence is below the threshold (Sec. 6)      */
  SMAT_TUNE_EXHAUSTIVE = 1, /* time every admissible variant, keep the fastest
                               (the brute-force search of Sec. 7.3)          */
  SMAT_TUNE_RULES = 2,      /* the paper's published thresholds (Sec. 4)       */
  SMAT_TUNE_FIXED = 3       /* use opts.fixed_variant                          */
} smat_tune_mode_t;

typedef struct {
  int32_t mode;            /* smat_tune_mode_t                                  */
  int32_t fixed_variant;   /* for SMAT_TUNE_FIXED                                */
  float conf_threshold;    /* learned mode: trial when max probability < this  */
  int32_t fallback_topk;   /* learned mode: variants trialled on fallback (0=all) */
  int32_t tau_num, tau_den;/* "true" diagonal: > tau_num/tau_den filled (3/5)  */
  int32_t fill_ratio_max;  /* DIA/ELL admissible while Ndiags, max_RD <= this *
                              aver_RD (Sec. 2.3: 20, i.e. >= 5% fill)          */
  double bytes_cap;        /* DIA/ELL admissible while their bytes <= this *
                              CSR bytes (default 4)                            */
  int32_t trial_reps;      /* timed products per variant: the median of that
                              many repetitions of one product, or, for
                              products under about 40 us, of
                              max(min(trial_reps, 3), ceil(trial_reps / g))
                              repetitions of g back-to-back products spanning
                              about 40 us (the event-timed duration of one
                              short kernel moves in steps of about 2 us);
                              each block of repetitions is queued behind a
                              short device hold so that no host launch
                              latency falls between its events              */
  int32_t trial_warmup;    /* untimed repetitions per variant                  */
  double trial_budget_ms;  /* stop trialling further variants past this       */
  uint32_t allowed;        /* bit mask over smat_variant_t (0 = all)           */
  int32_t keep_formats;    /* 1: keep every converted format after tuning      */
  int32_t sell_sigma;      /* SELL sort window in rows: a multiple of 32 in
                              [32, 8192] (default 256)                         */
  int32_t trial_extended;  /* learned mode: also time HYB / SELL / BCSR / SPLIT when
                              they move at most 1.25x the matrix bytes of the
                              selector's pick (BCSR only for max_RD <= 64);
                              default 1                                       */
  int32_t plan_cache;      /* 1 (modes other than FIXED): take the plan recorded
                              in the process-wide plan cache for this structure
                              when it is admissible and allowed, else tune and
                              record the result; default 0                    */
  float trial_race;        /* trials: a candidate whose median over its first 3
                              timed products exceeds this many times the best
                              so far is not timed further (its timing is that
                              median); 0 times every candidate fully;
                              default 1.3                                     */
  float trial_tie;         /* trials: candidates whose median is within this
                              fraction of the fastest count as equally fast
                              (Sec. 7.3 counts near-equal performance as a
                              hit); among them the pick is the one whose
                              format moves the fewest matrix bytes
                              (smat_variant_bytes), then the lowest variant
                              id, so that plans of matrices whose variants all
                              run alike are reproducible; 0 breaks only exact
                              ties that way, < 0 keeps the fastest median;
                              default 0.02                                    */
} smat_tune_opts_t;

/* Fill *opts with the defaults above. */
void smat_tune_opts_default(smat_tune_opts_t *opts);

/* Short English text for a status code (static storage). */
const char *smat_status_string(smat_status_t s);

/* ------------------------------------------------------------------------ */
/* Matrix handle (Sec. 3: the unified CSR interface)                         */
/* ------------------------------------------------------------------------ */

/* Create a handle from a CSR matrix with m rows, n columns and nnz stored
 * entries: rowptr[m+1], colidx[nnz] (int32), vals[nnz] of the storage type.
 * The three pointers may be host or device memory (detected); they are copied
 * into library-owned device memory before the call returns, so the caller may
 * free them afterwards.  The copy is validated on the GPU (rowptr[0] = 0,
 * rowptr[m] = nnz, monotone rowptr, 0 <= col < n, strictly increasing columns
 * in each row); a violation returns SMAT_ERR_INVALID_CSR and no handle.  Until
 * smat_tune runs, the plan is CSR-scalar (Sec. 4: CSR is the default format).
 * m = 0 or nnz = 0 is allowed.  Errors: INVALID_ARG, INVALID_CSR, ALLOC, CUDA,
 * UNSUPPORTED (m, n or nnz > 2^31 - 1). */
smat_status_t smat_create(smat_handle_t *out, int64_t m, int64_t n, int64_t nnz,
                          const int32_t *rowptr, const int32_t *colidx, const void *vals,
                          smat_dtype_t dtype);

/* Free the handle and everything it owns.  NULL is a no-op.  The handle must
 * not be in use on any stream. */
smat_status_t smat_destroy(smat_handle_t h);

/* Run-time stage of Sec. 6: extract features (Sec. 4) if not done yet, choose
 * a variant by opts->mode (NULL: learned when a model is loaded, otherwise
 * exhaustive), convert CSR to its format (Sec. 2.1) and store the plan.  Work
 * is issued on `stream`; the call returns after synchronising it.
 * Exhaustive mode times every admissible variant, HYB / SELL / BCSR included;
 * learned mode times the further formats beside the selector's pick when
 * opts->trial_extended is set (see smat_tune_opts_t); rules mode never picks
 * them; fixed mode accepts them. */
smat_status_t smat_tune(smat_handle_t h, const smat_tune_opts_t *opts, void *stream);

/* y = alpha*A*x + beta*y through the handle's plan.  x[n] and y[m] are DEVICE
 * pointers of the compute type; alpha and beta HOST pointers.  Asynchronous on
 * `stream`; only launch errors are reported.  x and y must not overlap.  ELL
 * and DIA plans use 16-byte vector accesses to x and y; when either is not
 * 16-byte aligned the product runs through the CSR-scalar kernel instead. */
smat_status_t smat_spmv(smat_handle_t h, const void *alpha, const void *x, const void *beta,
                        void *y, void *stream);

/* Same product through a chosen variant (its format is built on first use;
 * SMAT_ERR_UNSUPPORTED if the variant is not admissible and cannot be built).
 * The first product through a variant builds its format and, like smat_tune,
 * must not overlap other calls on the handle. */
smat_status_t smat_spmv_variant(smat_handle_t h, smat_variant_t v, const void *alpha,
                                const void *x, const void *beta, void *y, void *stream);

/* count independent products y_i = alpha_i*A_i*x_i + beta_i*y_i, each through
 * its handle's plan, run side by side on library-owned streams (16 per
 * device, created on the first call with that device current): they start
 * after the work queued on `stream` so far, and work queued on `stream` after
 * the call starts after all of them.  Products that stress different limits
 * (random gathers, HBM streaming) then overlap; on GB300 the structures
 * suite's eight products ran 6 % faster this way than one after another.
 * hs[count]: handles (their plans must be built, e.g. by smat_tune); alphas /
 * betas[count]: HOST pointers to one scalar of each handle's compute type;
 * xs / ys[count]: DEVICE vectors as for smat_spmv.  A handle may appear more
 * than once only if those products write different y.  Each internal stream
 * gets its own scratch on a handle's first product there, so make a first
 * call before any stream capture.  Errors as for smat_spmv; INVALID_ARG for
 * count < 0 or NULL arrays; nothing is launched when a handle fails its
 * check. */
smat_status_t smat_spmv_many(const smat_handle_t *hs, int32_t count, const void *const *alphas,
                             const void *const *xs, const void *const *betas, void *const *ys, void *stream);

/* The kernel behind a variant whose format has more than one implementation
 * (the per-format choice of implementation, Sec. 3).  The library times the
 * candidates when it builds the format and keeps the faster; smat_get_kernel
 * reads that choice and smat_set_kernel pins one for later products:
 *   SMAT_V_DIA  0: direct 16-byte loads; 1..2: the stripes of each tile of
 *               rows staged in shared memory by bulk asynchronous copies, a
 *               producer warp feeding a ring of stages, in two launch
 *               shapes (consumer warps, CTAs per SM, stages, stage size):
 *               1 (16, 1, 4, 48 KB), 2 (16, 2, 3, 32 KB); a shape needs 32
 *               rows of every stripe within its stage;
 *   SMAT_V_ELL  0: consecutive rows per thread; 1: lane-striped rows.
 * Returns SMAT_ERR_UNSUPPORTED when the variant's format is not built yet (a
 * tune picked it, or a product through smat_spmv_variant built it) or the
 * kernel cannot run this matrix; SMAT_ERR_INVALID_ARG for other variants or
 * kernel ids.  Must not overlap products on the handle. */
smat_status_t smat_set_kernel(smat_handle_t h, smat_variant_t v, int32_t kernel);
smat_status_t smat_get_kernel(smat_handle_t h, smat_variant_t v, int32_t *kernel);

/* Same product with x and y in HOST memory (pinned or pageable): x is copied to
 * a device staging buffer, the product runs through the plan, y is copied
 * back (and, when beta != 0, copied in first).  Returns after `stream` has
 * finished, so y is ready on return. */
smat_status_t smat_spmv_host(smat_handle_t h, const void *alpha, const void *x_host,
                             const void *beta, void *y_host, void *stream);

/* Matrix bytes one product through variant v reads (the format's arrays; x
 * and y, common to every variant, excluded): the quantity the execute-and-
 * measure search breaks near-ties on.  Computes the features first if
 * needed; SMAT_ERR_UNSUPPORTED for HYB / SELL / BCSR / SPLIT before their
 * layout has been measured (by smat_tune or smat_convert). */
smat_status_t smat_variant_bytes(smat_handle_t h, smat_variant_t v, double *bytes);

/* Number of kernel launches one product through variant v issues on this
 * handle (merge-path and COO add a carry fix-up launch when they span more
 * than one tile; COO adds one for empty rows).  Writes 0 for v not built. */
smat_status_t smat_spmv_launches(smat_handle_t h, smat_variant_t v, int32_t *launches);

/* The same host-buffer product without the final synchronisation: the copy
 * in, the product and the copy out are only enqueued on `stream`, so products
 * of different handles on different streams overlap their transfers with each
 * other's kernels.  x_host and y_host should be page-locked (pinned) for the
 * copies to be asynchronous; y_host is valid once `stream` has finished.
 * Calls on one handle share its staging buffers and must be ordered. */
smat_status_t smat_spmv_host_async(smat_handle_t h, const void *alpha, const void *x_host, const void *beta,
                                   void *y_host, void *stream);

/* Host-buffer products in a pipeline.  The same product as
 * smat_spmv_host_async, but the handle keeps two staging sets, used by
 * consecutive calls in turn, and copies and computes on three streams of its
 * own: a call's copy in waits only until the product two calls back has read
 * its staging set, so one call's transfers overlap the previous call's
 * product (and, across handles, other handles' products).  Ordering:
 *  - x_host (and y_host when beta != 0) is read by a copy that is NOT ordered
 *    after earlier work on `stream`: it must hold its values when the call is
 *    made, and stay unchanged until `stream` has finished;
 *  - y_host is written by a copy that `stream` waits for: it is valid once
 *    `stream` has finished (e.g. cudaStreamSynchronize);
 *  - calls on one handle must not overlap on the host.
 * x_host and y_host should be pinned.  Returns SMAT_ERR_UNSUPPORTED when
 * `stream` is capturing a graph (the copies do not run on it), or when the
 * plan is not built.  The staging sets and streams are freed by smat_destroy,
 * which waits for them first. */
smat_status_t smat_spmv_host_pipelined(smat_handle_t h, const void *alpha, const void *x_host, const void *beta,
                                       void *y_host, void *stream);

/* Feature parameters (computes them on `stream` = NULL if not yet done). */
smat_status_t smat_get_features(smat_handle_t h, smat_features_t *out);

/* The 12 selector inputs before standardisation: log1p of M, N, NNZ, aver_RD,
 * max_RD, min_RD, var_RD, Ndiags, then NTdiags_ratio, ER_DIA, ER_ELL and R. */
smat_status_t smat_get_feature_vector(smat_handle_t h, float out[12]);

/* Current plan: variant, wall time of the last smat_tune in ms, selector
 * confidence (max softmax probability; -1 when no model was used) and whether
 * the execute-and-measure fallback ran. */
smat_status_t smat_get_plan(smat_handle_t h, int32_t *variant, double *tune_ms, float *confidence,
                            int32_t *trialled);

/* 1 when the last smat_tune took its plan from the plan cache, else 0. */
smat_status_t smat_get_plan_source(smat_handle_t h, int32_t *from_cache);

/* ------------------------------------------------------------------------ */
/* Tuned-plan cache: smat_tune's decisions kept per matrix structure, so a  */
/* later handle or run reuses them (the paper's offline stage runs once per */
/* platform, Sec. 5; this keeps the online stage's result too).  Host-side  */
/* and thread-safe.                                                         */
/* ------------------------------------------------------------------------ */

/* 64-bit key of h's structure: M, N, NNZ, the storage dtype, rowptr and
 * colidx (not the values).  Each stored index adds
 * mix(mix(tag << 56 ^ position) + (uint32_t)value) modulo 2^64, tag 1 for
 * rowptr[0..M], 2 for colidx[0..NNZ); mix is the SplitMix64 finaliser; the
 * key is mix(sum + mix(4M) + mix(4N + 1) + mix(4 NNZ + 2) + mix(4 dtype + 3)).
 * One pass over rowptr and colidx on `stream`, computed once per handle;
 * returns after `stream` has finished. */
smat_status_t smat_plan_key(smat_handle_t h, uint64_t *key, void *stream);

/* Write every cached plan to `path` as text: "smat-plan-cache 1", then one
 * line "<key hex> <dtype> <M> <N> <NNZ> <variant> <sell sigma>" per plan.
 * SMAT_ERR_INVALID_ARG if the file cannot be written. */
smat_status_t smat_plan_cache_save(const char *path);

/* Merge the plans of a file written by smat_plan_cache_save (a loaded entry
 * replaces one with the same key).  A missing or malformed file changes
 * nothing and returns SMAT_ERR_INVALID_ARG. */
smat_status_t smat_plan_cache_load(const char *path);

/* Drop every recorded plan (handles keep the plans they already chose). */
void smat_plan_cache_clear(void);

/* Number of recorded plans (structures) in the process-wide table. */
int64_t smat_plan_cache_size(void);

/* Median trial time per variant in ms from the last smat_tune (-1 = not run),
 * for all SMAT_NUM_ALL_VARIANTS variants; a candidate stopped by racing
 * (opts.trial_race) reports the median of its first 3 timed products. */
smat_status_t smat_get_timings(smat_handle_t h, float ms[SMAT_NUM_ALL_VARIANTS]);

/* Build format `fmt` on the device now (CSR is always there).  UNSUPPORTED if
 * the format is not admissible (fill or byte cap).  SELL uses the sort window
 * of the last smat_tune (256 before any). */
smat_status_t smat_convert(smat_handle_t h, smat_format_t fmt, void *stream);

/* Layout of a built format:
 *   ELL: dims = {K = max_RD, P = pitch}, arrays col int32[K*P], val[K*P]
 *   DIA: dims = {Ndiags, P},             arrays offsets int32[Ndiags], val[Ndiags*P]
 *   COO: dims = {NNZ, 0},                arrays row int32[NNZ] (col and val are CSR's)
 *   HYB: dims = {K, Ncoo}: ELL part col/val[K*P] (as ELL, width K = the
 *        largest k with 3 * #{rows with >= k entries} >= M), then the COO part
 *        row[Ncoo], col[Ncoo], val[Ncoo] of each row's entries past its first K
 *   SELL: dims = {Nslices, Nslots}: perm int32[32*Nslices] (row at each sorted
 *        position, -1 past M), width int32[Nslices], col/val[Nslots]; entry j
 *        of position 32s + l at sum_{t<s} 32*width[t] + 32j + l
 *   BCSR: dims = {b, Nblocks}: browptr int32[ceil(M/b)+1], bcol int32[Nblocks],
 *        val[Nblocks*b*b] row-major per block
 *   SPLIT: dims = {Nchunks, Nshort}: per chunk (row, first entry, end entry)
 *        int32[Nchunks] each, chunks of one row consecutive and in order; the
 *        short rows' COO row[Nshort], col[Nshort], val[Nshort] in CSR order
 * P is M rounded up to a multiple of 32; padding holds column -1 / value +0. */
smat_status_t smat_format_dims(smat_handle_t h, smat_format_t fmt, int64_t dims[2]);

/* Copy a built format to caller memory (host or device, detected):
 *   ELL: idx <- col, val <- val;  DIA: idx <- offsets, val <- val;
 *   COO: idx <- row (val unused);
 *   HYB: idx <- ELL col, COO row, COO col; val <- ELL val, COO val;
 *   SELL: idx <- perm, width, col; val <- val;
 *   BCSR: idx <- browptr, bcol; val <- val;
 *   SPLIT: idx <- chunk rows, chunk starts, chunk ends, COO row, COO col;
 *          val <- COO val.
 * Arrays are concatenated in the order listed.  Sizes as in smat_format_dims. */
smat_status_t smat_export_format(smat_handle_t h, smat_format_t fmt, int32_t *idx, void *val);

/* Measured ceiling for gather-bound products (no counterpart in the paper,
 * which measures on CPUs): a kernel streams nidx int32 indices, uniform in
 * [0, n), and gathers x[index] from an x of n elements of dtype's compute type
 * (FP64, or FP32 for FP32 / BF16 storage), 8 per thread and nothing else.
 * Runs 3 untimed and `reps` timed passes on the legacy default stream and
 * writes the median rate in gathers per second.  SpMV on random columns
 * (x resident in L2) cannot gather faster; the benchmark reports products'
 * fraction of this rate beside their HBM fraction.  Allocates and frees its
 * own device buffers (nidx*4 + n*8 + nidx bytes at most).  Errors:
 * INVALID_ARG (n < 1, n > 2^31 - 1, nidx < 8, reps < 1), ALLOC, CUDA. */
smat_status_t smat_measure_gather_rate(int64_t n, int64_t nidx, smat_dtype_t dtype, int32_t reps,
                                       double *gathers_per_s);

/* Measured ceiling for FP64-arithmetic-bound products (no counterpart in the
 * paper): a kernel of 8 CTAs of 256 threads per SM runs eight independent
 * chains of 4096 FP64 fused multiply-adds per thread and nothing else.  Runs
 * 3 untimed and `reps` timed passes on the legacy default stream and writes
 * the median rate in fused multiply-adds per second (2 flops each).  An FP64
 * product spends one such operation per stored slot, so it cannot run faster
 * than slots / rate; the benchmark uses this as the FP64 roof.  Allocates and
 * frees its own small device buffers.  Errors: INVALID_ARG (reps < 1), ALLOC,
 * CUDA. */
smat_status_t smat_measure_fp64_rate(int32_t reps, double *fma_per_s);

/* Bounded waits in the library's pipelined kernels (the staged DIA product)
 * that ran out since the library was loaded, on the current device: each such
 * wait means a product whose y is not valid (its kernel gave up after about
 * one second instead of hanging).  Stays 0 in correct operation.  Copies the
 * device counter to *count (synchronous).  Errors: INVALID_ARG (NULL), CUDA. */
smat_status_t smat_get_wait_timeouts(uint64_t *count);

/* ------------------------------------------------------------------------ */
/* Learned selector (replaces the ruleset classifier of Sec. 5)             */
/* MLP 12 -> 64 -> ReLU -> 64 -> ReLU -> 8 over standardised features.       */
/* Parameters, FP32, row-major out x in:                                     */
/*   W1[64][12] b1[64] W2[64][64] b2[64] W3[8][64] b3[8]  (5512 floats)      */
/* ------------------------------------------------------------------------ */
#define SMAT_MLP_PARAMS 5512

/* Install the process-wide selector: parameters plus the standardisation
 * mean[12] and std[12] (host pointers, copied).  NULL params uninstalls. */
smat_status_t smat_set_model(const float *params, const float *mean, const float *std);

/* Load a model file written by the training driver (magic "SMATMLP1",
 * int32 version 1, mean[12], std[12], params[5512], all little-endian FP32). */
smat_status_t smat_load_model(const char *path);

/* Forward pass for B samples: X[B][12] (already standardised) -> logits[B][8].
 * All pointers are DEVICE memory; asynchronous on `stream`. */
smat_status_t smat_mlp_forward(const float *params, const float *X, int32_t B, float *logits,
                               void *stream);

/* Mean soft-target cross-entropy L = -(1/B) sum_b sum_c T[b][c] log softmax(z_b)_c
 * and dL/dparams (backpropagation), for B samples.  Device pointers:
 * params[5512], X[B][12], T[B][8], grad[5512], loss[1].  `work` is caller
 * scratch of smat_mlp_work_floats(B) floats.  Deterministic. */
int64_t smat_mlp_work_floats(int32_t B);
smat_status_t smat_mlp_loss_grad(const float *params, const float *X, const float *T, int32_t B,
                                 float *grad, float *loss, float *work, void *stream);

/* One Adam step (Kingma & Ba 2015) on n parameters; t >= 1 is the step count.
 * Device pointers p, g, m, v. */
smat_status_t smat_mlp_adam(float *p, const float *g, float *m, float *v, int64_t n, int32_t t,
                            float lr, float beta1, float beta2, float eps, void *stream);

/* ------------------------------------------------------------------------ */
/* Batched products: many matrices in one persistent launch                  */
/* The paper motivates adaptivity with algebraic multigrid, whose levels are */
/* different matrices used in turn, so one format does not fit them all     */
/* (Sec. 1).                                                                 */
/* ------------------------------------------------------------------------ */
typedef enum {
  SMAT_BATCH_AUTO = 0,        /* time the graph plans and the per-matrix launches */
  SMAT_BATCH_GRAPH = 1,       /* the persistent launch, captured in a graph       */
  SMAT_BATCH_PER_MATRIX = 2   /* each member's own plan, launched in turn         */
} smat_batch_mode_t;

typedef struct {
  int32_t tile_scale;   /* tile size multiplier; 0 = autotune over {1,2,4,8}     */
  int32_t ctas_per_sm;  /* resident CTAs per SM; 0 = autotune over {2,4,8}       */
  int32_t trial_reps;   /* timed launches per autotuning candidate             */
  int32_t mode;         /* smat_batch_mode_t; default SMAT_BATCH_AUTO          */
  int32_t own_launches; /* graph plans: members running their own plans'
                           kernels on side branches of the graph, beside the
                           persistent kernels: 0 none, 1 the members whose
                           plan has no batch kind (SPLIT, COO, HYB, BCSR,
                           merge-path), 2 all; -1 (default) times 0, 1 (when
                           there are members of both sorts) and, in AUTO
                           mode, 2, and keeps the fastest                     */
} smat_batch_opts_t;

typedef struct {
  int32_t count, tiles, grid, tile_scale, ctas_per_sm;
  double tuned_ms;      /* median time of one product of the chosen plan       */
  int32_t per_matrix;   /* 1: the members' own launches won the tuning         */
  double graph_ms;      /* median time of the best graph plan (-1: not timed)  */
  double per_matrix_ms; /* median time of the per-matrix launches (-1: not timed) */
  int32_t own_launches; /* members running their own plans' kernels on side
                           branches of the graph: 0 none, 1 those whose plan
                           has no batch kind, 2 all                         */
} smat_batch_info_t;

/* Defaults: tile_scale 0 and ctas_per_sm 0 (both autotuned), trial_reps 10,
 * mode SMAT_BATCH_AUTO.  NULL is a no-op. */
void smat_batch_opts_default(smat_batch_opts_t *opts);

/* Group `count` handles of one storage dtype.  The handles stay owned by the
 * caller and must outlive the batch; tune each first (each keeps its plan's
 * format: CSR kernels map to 1/4/8/32 lanes per row, merge-path and COO plans
 * to the fastest measured CSR row kernel, ELL and DIA stay ELL and DIA). */
smat_status_t smat_batch_create(smat_batch_t *out, const smat_handle_t *hs, int32_t count);

/* Build the work table (row tiles of every product, largest first), capture
 * the persistent launch in a CUDA graph and autotune tile size and CTAs per
 * SM by timing the graph.  Members whose plan the persistent kernel has no
 * body for can instead run their own plan's kernels on side branches of the
 * same graph (opts.own_launches); their pointers and scalars are then part of
 * the graph, which smat_batch_spmv captures again when they change.  In SMAT_BATCH_AUTO mode the members' own launches,
 * one after another, are timed too and kept when faster, so a batch is never
 * slower than the loop it replaces (a few large members in formats whose
 * single-matrix kernels outrun the persistent kernel's bodies).  Returns
 * after `stream` has finished.  Must run again if a member handle is
 * re-tuned. */
smat_status_t smat_batch_tune(smat_batch_t b, const smat_batch_opts_t *opts, void *stream);

/* y_i = alpha_i A_i x_i + beta_i y_i for every member i in one graph launch
 * (or, when the tuning chose them, the members' own launches in turn) on
 * `stream`.  alphas / betas: HOST arrays of `count` scalars of the compute
 * type; xs / ys: HOST arrays of `count` DEVICE pointers, 16-byte aligned for
 * ELL and DIA members (SMAT_ERR_INVALID_ARG otherwise).  Descriptors are
 * re-uploaded only when a pointer or scalar changed.  Asynchronous; calls on
 * one batch must be ordered (same stream or synchronised). */
smat_status_t smat_batch_spmv(smat_batch_t b, const void *alphas, const void *const *xs, const void *betas,
                              void *const *ys, void *stream);

/* The batch's shape and its tuning outcome (fields of smat_batch_info_t).
 * INVALID_ARG for a NULL batch or info. */
smat_status_t smat_batch_get_info(smat_batch_t b, smat_batch_info_t *info);

/* Free the batch (not its handles).  NULL is a no-op. */
smat_status_t smat_batch_destroy(smat_batch_t b);

/* ------------------------------------------------------------------------ */
/* Per-segment plans (Sec. 6: the multi-threaded SMAT splits the nonzeros    */
/* evenly over threads at whole rows and may choose a format per segment)    */
/* ------------------------------------------------------------------------ */

/* Split h's rows into `nseg` segments holding about NNZ/nseg stored entries
 * each (boundaries at whole rows, rounded down to multiples of 8 rows; fewer
 * segments when rows are too long to split), give every segment its own
 * handle tuned with `opts` (NULL: as in smat_tune), and batch them when every
 * segment's plan is one the batched kernel runs natively (CSR-scalar /
 * vector, ELL, DIA, SELL); otherwise give each segment a stream of its own.
 * h must stay alive while the segments exist.  Returns after `stream` is
 * idle. */
smat_status_t smat_segments_create(smat_segments_t *out, smat_handle_t h, int32_t nseg,
                                   const smat_tune_opts_t *opts, void *stream);

/* y = alpha*A*x + beta*y with every segment in its own format: one batched
 * launch, or each segment's own kernels on its own stream (forked from
 * `stream` by an event and joined back to it, so the call stays ordered on
 * `stream`); x[n], y[m] DEVICE pointers of the compute type, alpha/beta HOST
 * scalars.  Vectors that are not 16-byte aligned take h's own plan. */
smat_status_t smat_segments_spmv(smat_segments_t s, const void *alpha, const void *x, const void *beta, void *y,
                                 void *stream);

/* Number of segments, each segment's variant (variants[nseg]) and row starts
 * (row_starts[nseg + 1]); the arrays may be NULL. */
smat_status_t smat_segments_info(smat_segments_t s, int32_t *nseg, int32_t *variants, int64_t *row_starts);

/* Free the segments' handles, streams and batch (not the parent handle).
 * NULL is a no-op. */
smat_status_t smat_segments_destroy(smat_segments_t s);

/* ------------------------------------------------------------------------ */
/* Mixed-precision conjugate gradients (iterative refinement)               */
/* The paper measures SpMV in single and double precision (Sec. 7.2) and     */
/* motivates the library by solvers that call it hundreds of times (Sec. 1,  */
/* Sec. 7.3, Eq. "num_iter").                                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double rtol;             /* stop when ||b - A x||_2 <= rtol ||b||_2 (FP64 residual) */
  int32_t max_outer;       /* refinement steps                                  */
  int32_t max_inner;       /* inner CG iterations per refinement step          */
  float inner_rtol;        /* inner CG stops when ||res|| <= inner_rtol ||res_0|| */
  int32_t max_total_inner; /* cap on all inner iterations together (0 = none)  */
  int32_t check_every;     /* inner iterations between host convergence checks */
  int32_t use_graph;       /* replay chunks of inner iterations from a CUDA graph */
} smat_cg_opts_t;

typedef struct {
  int32_t outer;        /* refinement steps taken                                */
  int32_t inner_total;  /* inner CG iterations taken                             */
  double relres;        /* final ||b - A x||_2 / ||b||_2, computed in FP64       */
  double seconds;       /* wall time of the call                                 */
  int32_t converged;    /* relres <= rtol                                        */
} smat_cg_info_t;

/* rtol 1e-10, max_outer 50, max_inner 500, inner_rtol 1e-4, no total cap,
 * check_every 10, use_graph 1. */
void smat_cg_opts_default(smat_cg_opts_t *opts);

/* Solve A x = b for symmetric positive definite A.  a64 is an SMAT_F64 handle
 * of A (its plan forms the residual r = b - A x in FP64); a32 is an SMAT_F32
 * or SMAT_BF16 handle of the same matrix (its plan runs the inner FP32 CG on
 * A d = r / ||r||); both should be tuned.  Each refinement step updates
 * x += ||r|| d in FP64.  b[n] and x[n] are DEVICE FP64 arrays; x holds the
 * initial guess on entry and the solution on return.  opts may be NULL.
 * Work runs on a private stream ordered after `stream`; the call returns
 * when the solve has finished.  Returns SMAT_ERR_NOT_CONVERGED (with *info
 * filled) when a limit stops it first; INVALID_ARG for a non-square matrix or
 * wrong handle dtypes.  Workspace: 8n + 16n bytes, allocated per call. */
smat_status_t smat_cg_mixed(smat_handle_t a64, smat_handle_t a32, const double *b, double *x,
                            const smat_cg_opts_t *opts, smat_cg_info_t *info, void *stream);

/* ------------------------------------------------------------------------ */
/* Value casts for reduced-precision storage (device arrays, n elements)    */
/* ------------------------------------------------------------------------ */
/* FP64 -> FP32, round to nearest even. */
smat_status_t smat_cast_f64_to_f32(const double *in, float *out, int64_t n, void *stream);
/* FP64 -> bfloat16 (uint16 bit patterns), round to nearest even, one rounding. */
smat_status_t smat_cast_f64_to_bf16(const double *in, uint16_t *out, int64_t n, void *stream);

/* ------------------------------------------------------------------------ */
/* Allocation-free product (the paper has no counterpart to this entry point) */
/* ------------------------------------------------------------------------ */
/* y = alpha*A*x + beta*y by merge-path CSR for callers that cannot allocate
 * device memory: a solver whose memory manager owns every device byte, code
 * that must not synchronise the device the way cudaMalloc/cudaFree may, or a
 * host that forbids allocation once its time-critical loop runs.  No handle
 * and no allocation: the caller passes the CSR arrays (rowptr[m+1],
 * colidx[nnz], vals[nnz] of the storage type), x[n] and y[m], all DEVICE
 * pointers, and alpha/beta as HOST pointers to one scalar of the compute type
 * (FP64 for SMAT_F64, FP32 otherwise).  The input must be canonical CSR; it is
 * not validated.  alpha == 0 gives y = beta*y (0 when beta == 0) without
 * reading A or x, and beta == 0 makes y write-only, as in smat_spmv.
 * The kernels' only scratch, one carry and one merge-path coordinate per
 * tile of 2048 merge items, lives in a fixed 1.25 MiB array in the library's
 * device memory, held by every GPU that loads the library until the process
 * exits.  Limit: ceil((m + nnz) /
 * 2048) <= 65536, i.e. m + nnz <= 134,217,728; larger inputs return
 * SMAT_ERR_UNSUPPORTED without launching anything.  The first call on each
 * device looks up the array's address (cudaGetSymbolAddress) and keeps it for
 * the rest of the process; make that first call before any stream capture,
 * and do not call this entry point again after a cudaDeviceReset of a device
 * it has used (the kept address would be stale).  Every call shares the array, so calls
 * whose kernels overlap on the GPU race: order them on one stream or
 * synchronise between them.  Asynchronous on `stream`; only launch errors are
 * reported. */
smat_status_t smat_spmv_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                                          const int32_t *colidx, const void *vals, smat_dtype_t dtype,
                                          const void *alpha, const void *x, const void *beta, void *y,
                                          void *stream);

/* ------------------------------------------------------------------------ */
/* Testing hook                                                              */
/* ------------------------------------------------------------------------ */
/* Make the k-th device allocation from now on fail (k >= 1), as if the GPU
 * were out of memory; k = 0 disables.  Host-side only: lets tests check that
 * every entry point returns SMAT_ERR_ALLOC and frees what it had allocated. */
void smat_test_fail_alloc_after(int32_t k);

/* Make the pipelined kernels' bounded waits run out (on != 0), as if a copy
 * never landed: their consumer warps wait on a barrier that nothing arrives
 * on, for wait_cycles SM cycles (0 keeps the default of about one second),
 * then give up; the kernel still waits for its own copies before it leaves,
 * counts the timeout (smat_get_wait_timeouts) and returns, leaving the
 * context usable.  The products run meanwhile are invalid.  on = 0 restores
 * normal operation.  For tests of the failure path. */
void smat_test_stall_pipelines(int32_t on, int64_t wait_cycles);

/* ------------------------------------------------------------------------ */
/* Device memory                                                             */
/* ------------------------------------------------------------------------ */
/* The library takes device memory from a stream-ordered pool of its own that
 * keeps up to 1 GiB of freed blocks for later allocations (a cudaMalloc and
 * cudaFree pair costs 60-120 us on GB300; tuning makes dozens).  This call
 * waits for the device and returns every cached block to the system. */
smat_status_t smat_release_cached_memory(void);

#ifdef __cplusplus
}
#endif
#endif /* SMAT_H */
