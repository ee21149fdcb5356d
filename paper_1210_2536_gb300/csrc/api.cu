// C ABI of libsmat: the unified CSR interface (arXiv 1210.2536, Sec. 3) and
// the run-time stage (Sec. 6): feature extraction -> format search ->
// confidence check -> execute & measure -> convert -> SpMV.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "smat_internal.h"

namespace smat {

// ---------------------------------------------------------------------------
// Allocation with a test hook (error-path tests inject a failure on the host):
// smat_test_fail_alloc_after(k), or SMAT_TEST_FAIL_ALLOC_AFTER=k in the
// environment when the library loads, makes the k-th allocation fail.
// ---------------------------------------------------------------------------
static std::atomic<long> g_alloc_fail_at{0};
static std::atomic<long> g_alloc_count{0};
static const bool g_alloc_env = [] {
  const char *e = std::getenv("SMAT_TEST_FAIL_ALLOC_AFTER");
  if (e && *e) g_alloc_fail_at = std::atol(e);
  return true;
}();

// An NVTX range for the length of a scope (the tuning phases show up by name
// in profilers; without one attached the calls do nothing).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

static bool inject_alloc_failure() {
  const long k = ++g_alloc_count;
  const long f = g_alloc_fail_at.load();
  return f > 0 && k == f;
}

// Device memory comes from a library-owned stream-ordered pool of the current
// device, which keeps up to 1 GiB of freed blocks for the next allocation: a
// cudaMalloc + cudaFree pair costs 60-120 us on GB300, a pooled one about
// 2 us, and one tuning makes dozens (features, layouts, conversions, trials).
// Without a pool (creation failed) allocation falls back to cudaMalloc.
struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t s = nullptr;  // orders the pool's long-lived allocations and frees
  bool tried = false;
};

std::mutex &pool_mu() {
  static std::mutex mu;
  return mu;
}

DevPool *pools() {
  static DevPool p[64];
  return p;
}

DevPool &dev_pool() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(pool_mu());
  DevPool &d = pools()[dev & 63];
  if (!d.tried) {
    d.tried = true;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    uint64_t keep = 1ull << 30;
    if (cudaMemPoolCreate(&d.pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess ||
        cudaStreamCreateWithFlags(&d.s, cudaStreamNonBlocking) != cudaSuccess) {
      if (d.pool) cudaMemPoolDestroy(d.pool);
      d.pool = nullptr;
      cudaGetLastError();
    }
  }
  return d;
}

// Long-lived buffers (formats, handle copies): ready for every stream when
// this returns.
cudaError_t dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  DevPool &d = dev_pool();
  if (!d.pool) return cudaMalloc(p, bytes);
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, d.pool, d.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d.s);
  if (e != cudaSuccess && *p) {
    cudaFreeAsync(*p, d.s);
    *p = nullptr;
  }
  return e;
}

// As cudaFree: the device is synchronised first, so no kernel in any stream
// still uses the block when the pool may hand it out again.
void dev_free(void *p) {
  if (!p) return;
  DevPool &d = dev_pool();
  if (!d.pool) {
    cudaFree(p);
    return;
  }
  cudaDeviceSynchronize();
  cudaFreeAsync(p, d.s);
}

// Temporaries used on one stream only: allocated and freed in that stream's
// order, with no synchronisation at all.
cudaError_t tmp_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  DevPool &d = dev_pool();
  if (!d.pool) return cudaMalloc(p, bytes);
  return cudaMallocFromPoolAsync(p, bytes, d.pool, s);
}

void tmp_free(void *p, cudaStream_t s) {
  if (!p) return;
  DevPool &d = dev_pool();
  if (!d.pool) {
    cudaFree(p);
    return;
  }
  cudaFreeAsync(p, s);
}

Model &model() {
  static Model m;
  return m;
}

// The selector model is process-wide: it is replaced under this lock, and a
// tuning reads a copy taken under it, so loading a model while other threads
// tune is safe.
std::mutex &model_mu() {
  static std::mutex mu;
  return mu;
}

bool model_loaded() {
  std::lock_guard<std::mutex> lk(model_mu());
  return model().loaded;
}

bool model_copy(Model *out) {
  std::lock_guard<std::mutex> lk(model_mu());
  if (!model().loaded) return false;
  *out = model();
  return true;
}

namespace {

// A temporary device buffer used on one stream, freed in that stream's order.
struct DevBuf {
  void *p = nullptr;
  cudaStream_t s;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { tmp_free(p, s); }
  cudaError_t alloc(size_t bytes) { return tmp_alloc(&p, bytes, s); }
  template <typename T> T *as() const { return (T *)p; }
};

smat_status_t st_of(cudaError_t e) {
  if (e == cudaSuccess) return SMAT_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return SMAT_ERR_ALLOC;
  }
  return SMAT_ERR_CUDA;
}

#define TRY(call)                               \
  do {                                          \
    smat_status_t _s = st_of(call);             \
    if (_s != SMAT_OK) return _s;               \
  } while (0)
#define TRYS(call)                              \
  do {                                          \
    smat_status_t _s = (call);                  \
    if (_s != SMAT_OK) return _s;               \
  } while (0)

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int tsize(const smat_s *h) { return h->dtype == SMAT_F64 ? 8 : 4; }

int variant_format(int v) {
  if (v == SMAT_V_ELL) return SMAT_FMT_ELL;
  if (v == SMAT_V_DIA) return SMAT_FMT_DIA;
  if (v == SMAT_V_COO) return SMAT_FMT_COO;
  if (v == SMAT_V_HYB) return SMAT_FMT_HYB;
  if (v == SMAT_V_SELL) return SMAT_FMT_SELL;
  if (v == SMAT_V_BCSR) return SMAT_FMT_BCSR;
  if (v == SMAT_V_SPLIT) return SMAT_FMT_SPLIT;
  return SMAT_FMT_CSR;
}

constexpr uint32_t ALL_VARIANTS = ((1u << SMAT_NUM_ALL_VARIANTS) - 1) & ~(1u << SMAT_V_CSR_SCALAR_EXACT);

double csr_bytes(const smat_s *h) { return (double)(h->esz + 4) * h->nnz + 4.0 * (h->m + 1); }
double ell_bytes(const smat_s *h) { return (double)(h->esz + 4) * h->f.max_rd * h->P; }
double dia_bytes(const smat_s *h) { return (double)h->esz * h->f.ndiags * h->P + 4.0 * h->f.ndiags; }

// Matrix bytes one product through `v` reads (x and y are common to all).
double variant_bytes(const smat_s *h, int v) {
  switch (v) {
    case SMAT_V_ELL: return ell_bytes(h);
    case SMAT_V_DIA: return dia_bytes(h);
    case SMAT_V_COO: return (double)(h->esz + 8) * h->nnz;
    case SMAT_V_HYB: case SMAT_V_SELL: case SMAT_V_BCSR: case SMAT_V_SPLIT: return h->ext_bytes[v - SMAT_V_HYB];
    default: return csr_bytes(h);
  }
}

// HYB / SELL / BCSR / SPLIT: admissible once their layout is measured, under
// the same two limits as ELL and DIA (stored slots <= fill_ratio_max x NNZ,
// bytes <= bytes_cap x CSR bytes); HYB also needs an ELL part, SPLIT a long
// row (without one it is the COO plan).
uint32_t ext_bits(const smat_s *h) {
  uint32_t mask = 0;
  const double cap = h->bytes_cap * std::max(csr_bytes(h), 1.0);
  const double lim = (double)h->fill_ratio_max * (double)h->nnz;
  for (int e = 0; e < 4; ++e) {
    if (!h->ext_known[e] || h->nnz == 0 || h->m == 0) continue;
    if (e == 0 && h->hyb_K < 1) continue;
    if (e == SMAT_V_SPLIT - SMAT_V_HYB && h->split_nl < 1) continue;
    if (h->ext_slots[e] <= lim && h->ext_bytes[e] <= cap) mask |= 1u << (SMAT_V_HYB + e);
  }
  return mask;
}

// ---------------------------------------------------------------------------
// Feature extraction (Sec. 4): integer passes on the GPU, then the doubles
// from exact integers, each operand converted once and one division.
// ---------------------------------------------------------------------------
void power_law_fit(const std::vector<int64_t> &hist, double *R, int32_t *valid) {
  double cnt = 0.0, sum_x = 0.0, sum_y = 0.0, sum_xx = 0.0, sum_xy = 0.0;
  for (size_t k = 1; k < hist.size(); ++k) {
    if (hist[k] <= 0) continue;
    const double lk = std::log((double)k), lh = std::log((double)hist[k]);
    cnt = cnt + 1.0;
    sum_x = sum_x + lk;
    sum_y = sum_y + lh;
    sum_xx = sum_xx + lk * lk;
    sum_xy = sum_xy + lk * lh;
  }
  if (cnt < 2.0) {
    *R = 0.0;
    *valid = 0;
    return;
  }
  const double slope_num = cnt * sum_xy - sum_x * sum_y;
  const double slope_den = cnt * sum_xx - sum_x * sum_x;
  *R = -(slope_num / slope_den);
  *valid = 1;
}

void update_admissible(smat_s *h) {
  smat_features_t &f = h->f;
  uint32_t mask = (1u << SMAT_V_CSR_SCALAR) | (1u << SMAT_V_CSR_VEC4) | (1u << SMAT_V_CSR_VEC8) |
                  (1u << SMAT_V_CSR_VEC32) | (1u << SMAT_V_CSR_MERGE) | (1u << SMAT_V_COO);
  const double cap = h->bytes_cap * std::max(csr_bytes(h), 1.0);
  // Sec. 2.3: DIA / ELL only while Ndiags (max_RD) <= 20 x aver_RD, i.e.
  // at least 5% of the stored slots are nonzeros; plus a hard byte cap.
  const __int128 lim = (__int128)h->fill_ratio_max * f.nnz;
  if (f.m > 0 && f.max_rd > 0 && (__int128)f.max_rd * f.m <= lim && ell_bytes(h) <= cap) mask |= 1u << SMAT_V_ELL;
  // the DIA kernel stages its offsets in shared memory: at most 8192 of them
  if (f.m > 0 && f.ndiags > 0 && f.ndiags <= 8192 && h->dia_offsets_complete && (__int128)f.ndiags * f.m <= lim &&
      dia_bytes(h) <= cap)
    mask |= 1u << SMAT_V_DIA;
  f.admissible = mask | ext_bits(h);
}

smat_status_t compute_features(smat_s *h, cudaStream_t s) {
  smat_features_t f{};
  f.m = h->m;
  f.n = h->n;
  f.nnz = h->nnz;
  RowStats st{0ull, 0, h->m > 0 ? INT_MAX : 0, 0, 0};
  if (h->m > 0) {
    DevBuf d_st(s);
    TRY(d_st.alloc(sizeof(RowStats)));
    TRY(cudaMemcpyAsync(d_st.p, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    TRY(launch_row_stats(h->rowptr, h->m, d_st.as<RowStats>(), s));
    TRY(cudaMemcpyAsync(&st, d_st.p, sizeof(st), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
  }
  f.max_rd = st.max_rd;
  f.min_rd = st.min_rd;
  f.empty_rows = st.empty_rows;
  f.s2 = st.s2;
  const int64_t hist_len = f.max_rd + 1;
  h->hist.assign((size_t)hist_len, 0);
  h->dia_offsets.clear();
  h->dia_offsets_complete = false;
  const int64_t nd_all = h->m + h->n - 1;
  if (h->m > 0 && h->n > 0) {
    DevBuf d_hist(s), d_cnt(s), d_counts(s), d_off(s);
    TRY(d_hist.alloc((size_t)hist_len * sizeof(int)));
    TRY(d_cnt.alloc((size_t)nd_all * sizeof(int)));
    TRY(cudaMemsetAsync(d_hist.p, 0, (size_t)hist_len * sizeof(int), s));
    TRY(cudaMemsetAsync(d_cnt.p, 0, (size_t)nd_all * sizeof(int), s));
    TRY(launch_hist_diag(h->rowptr, h->colidx, h->m, d_hist.as<int>(), hist_len, d_cnt.as<int>(), s));
    // offsets are kept while DIA can still be admissible (Ndiags <= 20 aver_RD)
    int64_t cap = (int64_t)((__int128)h->fill_ratio_max * h->nnz / h->m) + 1;
    cap = std::max<int64_t>(cap, 64);
    cap = std::min<int64_t>(cap, nd_all);
    TRY(d_counts.alloc(3 * sizeof(unsigned long long)));
    TRY(d_off.alloc((size_t)cap * sizeof(int32_t)));
    TRY(cudaMemsetAsync(d_counts.p, 0, 3 * sizeof(unsigned long long), s));
    TRY(launch_diag_reduce(d_cnt.as<int>(), h->m, h->n, h->tau_num, h->tau_den,
                           d_counts.as<unsigned long long>(), d_off.as<int32_t>(), cap, s));
    unsigned long long counts[3];
    std::vector<int> hist32((size_t)hist_len);
    TRY(cudaMemcpyAsync(counts, d_counts.p, sizeof(counts), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(hist32.data(), d_hist.p, (size_t)hist_len * sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    for (int64_t k = 0; k < hist_len; ++k) h->hist[(size_t)k] = hist32[(size_t)k];
    f.ndiags = (int64_t)counts[0];
    f.ntdiags = (int64_t)counts[1];
    if ((int64_t)counts[2] <= cap) {
      h->dia_offsets.resize((size_t)counts[2]);
      TRY(cudaMemcpy(h->dia_offsets.data(), d_off.p, (size_t)counts[2] * sizeof(int32_t), cudaMemcpyDeviceToHost));
      std::sort(h->dia_offsets.begin(), h->dia_offsets.end());
      h->dia_offsets_complete = true;
    }
  } else if (h->m > 0) {
    h->hist[0] = h->m;  // no columns: every row is empty
  }
  if (h->m > 0) {
    const double M = (double)h->m;
    f.aver_rd = (double)h->nnz / M;
    const __int128 var_num = (__int128)h->m * (__int128)f.s2 - (__int128)h->nnz * (__int128)h->nnz;
    const __int128 var_den = (__int128)h->m * (__int128)h->m;
    f.var_rd = (double)var_num / (double)var_den;
    f.er_dia = f.ndiags > 0 ? (double)h->nnz / (double)(f.ndiags * h->m) : 0.0;
    f.er_ell = f.max_rd > 0 ? (double)h->nnz / (double)(f.max_rd * h->m) : 0.0;
  }
  f.ntdiags_ratio = f.ndiags > 0 ? (double)f.ntdiags / (double)f.ndiags : 0.0;
  power_law_fit(h->hist, &f.r, &f.r_valid);
  h->f = f;
  h->have_features = true;
  update_admissible(h);
  return SMAT_OK;
}

void feature_vector(const smat_features_t &f, float out[12]) {
  out[0] = (float)std::log1p((double)f.m);
  out[1] = (float)std::log1p((double)f.n);
  out[2] = (float)std::log1p((double)f.nnz);
  out[3] = (float)std::log1p(f.aver_rd);
  out[4] = (float)std::log1p((double)f.max_rd);
  out[5] = (float)std::log1p((double)f.min_rd);
  out[6] = (float)std::log1p(f.var_rd);
  out[7] = (float)std::log1p((double)f.ndiags);
  out[8] = (float)f.ntdiags_ratio;
  out[9] = (float)f.er_dia;
  out[10] = (float)f.er_ell;
  out[11] = (float)(f.r_valid ? std::max(-100.0, std::min(100.0, f.r)) : 0.0);
}

// ---------------------------------------------------------------------------
// Format construction (Sec. 2.1).
// ---------------------------------------------------------------------------
void free_format(smat_s *h, int fmt) {
  if (fmt == SMAT_FMT_ELL) {
    dev_free(h->ell_col); dev_free(h->ell_val);
    h->ell_col = nullptr; h->ell_val = nullptr; h->ell_K = 0;
  } else if (fmt == SMAT_FMT_DIA) {
    dev_free(h->dia_off); dev_free(h->dia_val);
    h->dia_off = nullptr; h->dia_val = nullptr; h->dia_nd = 0;
  } else if (fmt == SMAT_FMT_COO) {
    dev_free(h->coo_row); dev_free(h->coo_empty);
    h->coo_row = nullptr; h->coo_empty = nullptr; h->coo_nempty = 0;
  } else if (fmt == SMAT_FMT_HYB) {
    dev_free(h->hyb_ecol); dev_free(h->hyb_eval); dev_free(h->hyb_crow); dev_free(h->hyb_ccol); dev_free(h->hyb_cval);
    h->hyb_ecol = h->hyb_crow = h->hyb_ccol = nullptr; h->hyb_eval = h->hyb_cval = nullptr; h->hyb_built = false;
  } else if (fmt == SMAT_FMT_SELL) {  // the layout (perm, width, slice pointers) stays
    dev_free(h->sell_col); dev_free(h->sell_val);
    h->sell_col = nullptr; h->sell_val = nullptr;
  } else if (fmt == SMAT_FMT_BCSR) {  // the 64-bit block row starts stay
    dev_free(h->bcsr_rowptr); dev_free(h->bcsr_col); dev_free(h->bcsr_val);
    h->bcsr_rowptr = h->bcsr_col = nullptr; h->bcsr_val = nullptr;
    h->bcsr_cb = 0;
  } else if (fmt == SMAT_FMT_SPLIT) {
    for (int32_t **p : {&h->split_lchunk, &h->split_lrows, &h->split_crow, &h->split_cstart, &h->split_cend,
                        &h->split_srow, &h->split_scol, &h->split_empty}) {
      dev_free(*p);
      *p = nullptr;
    }
    dev_free(h->split_sval); dev_free(h->split_part);
    h->split_sval = h->split_part = nullptr;
    h->split_built = false;
  }
}

void free_sell_layout(smat_s *h) {
  free_format(h, SMAT_FMT_SELL);
  dev_free(h->sell_perm); dev_free(h->sell_width); dev_free(h->sell_ptr);
  h->sell_perm = h->sell_width = nullptr; h->sell_ptr = nullptr; h->sell_ns = h->sell_slots = 0;
  h->ext_known[SMAT_V_SELL - SMAT_V_HYB] = false;
}

void free_ext_layouts(smat_s *h) {
  free_format(h, SMAT_FMT_HYB);
  free_sell_layout(h);
  free_format(h, SMAT_FMT_BCSR);
  dev_free(h->bcsr_brp64);
  h->bcsr_brp64 = nullptr;
  free_format(h, SMAT_FMT_SPLIT);
}

// Layout of a further format -- sizes without the values: HYB's width K and
// tail length from the row-degree histogram; SELL's sorted order, slice widths
// and slice pointers; BCSR's block size (the b in {2, 4, 8} with the fewest
// bytes; ties to the smaller) and block row starts.  Sets the admissibility bit.
smat_status_t ext_layout(smat_s *h, int v, int sigma, cudaStream_t s) {
  const int e = v - SMAT_V_HYB;
  if (!h->have_features) TRYS(compute_features(h, s));
  if (v == SMAT_V_SELL && h->ext_known[e] && sigma != h->sell_sigma) free_sell_layout(h);
  if (h->ext_known[e]) return SMAT_OK;
  if (v == SMAT_V_SELL) h->sell_sigma = sigma;
  const int esz = h->esz;
  if (h->m > 0 && h->nnz > 0) {
    if (v == SMAT_V_HYB) {
      int64_t rows_ge = 0, K = 0;
      for (int64_t k = (int64_t)h->hist.size() - 1; k >= 1; --k) {
        rows_ge += h->hist[(size_t)k];
        if (3 * rows_ge >= h->m) { K = k; break; }
      }
      int64_t ncoo = 0;
      for (int64_t k = K + 1; k < (int64_t)h->hist.size(); ++k) ncoo += h->hist[(size_t)k] * (k - K);
      h->hyb_K = K;
      h->hyb_ncoo = ncoo;
      h->ext_slots[e] = (double)K * h->m + (double)ncoo;
      h->ext_bytes[e] = (double)(esz + 4) * K * h->P + (double)(esz + 8) * ncoo;
    } else if (v == SMAT_V_SPLIT) {
      int64_t nl = 0, nc = 0, ns = 0;
      for (int64_t k = 1; k < (int64_t)h->hist.size(); ++k) {
        const int64_t c = h->hist[(size_t)k];
        if (k >= SPLIT_L) {
          nl += c;
          nc += c * ((k + SPLIT_CK - 1) / SPLIT_CK);
        } else {
          ns += c * k;
        }
      }
      h->split_nl = nl; h->split_nc = nc; h->split_ns = ns; h->split_ne = h->hist.empty() ? 0 : h->hist[0];
      h->ext_slots[e] = (double)h->nnz;
      h->ext_bytes[e] = (double)(esz + 4) * (h->nnz - ns) + 12.0 * nc + 4.0 * (2 * nl + 1) + (double)(esz + 8) * ns +
                        4.0 * h->split_ne;
    } else if (v == SMAT_V_SELL) {
      free_sell_layout(h);  // drop what an earlier, failed attempt left
      const int64_t mp = (h->m + 31) / 32 * 32, ns = mp / 32;
      void *perm = nullptr, *width = nullptr, *ptr = nullptr;
      DevBuf cnt(s);
      TRY(dev_alloc(&perm, (size_t)mp * 4));
      h->sell_perm = (int32_t *)perm;
      TRY(dev_alloc(&width, (size_t)ns * 4));
      h->sell_width = (int32_t *)width;
      TRY(dev_alloc(&ptr, (size_t)(ns + 1) * 8));
      h->sell_ptr = (long long *)ptr;
      TRY(cnt.alloc((size_t)ns * 8));
      TRY(launch_sell_layout(h, sigma, h->sell_perm, h->sell_width, cnt.as<long long>(), s));
      TRY(exclusive_scan(cnt.as<long long>(), ns, h->sell_ptr, s));
      long long slots = 0;
      TRY(cudaMemcpy(&slots, h->sell_ptr + ns, 8, cudaMemcpyDeviceToHost));
      h->sell_ns = ns;
      h->sell_slots = slots;
      h->ext_slots[e] = (double)slots;
      h->ext_bytes[e] = (double)(esz + 4) * slots + 4.0 * mp + 12.0 * ns + 8.0;
    } else {
      free_format(h, SMAT_FMT_BCSR);
      dev_free(h->bcsr_brp64);
      h->bcsr_brp64 = nullptr;
      h->bcsr_b = 0;
      double best_bytes = 0.0;
      for (int b = 2; b <= 8; b *= 2) {
        const int64_t mb = (h->m + b - 1) / b;
        DevBuf cnt(s);
        void *brp = nullptr;
        TRY(cnt.alloc((size_t)mb * 8));
        TRY(dev_alloc(&brp, (size_t)(mb + 1) * 8));
        cudaError_t err = launch_bcsr_count(h, b, cnt.as<long long>(), s);
        if (err == cudaSuccess) err = exclusive_scan(cnt.as<long long>(), mb, (long long *)brp, s);
        long long nb = 0;
        if (err == cudaSuccess) err = cudaMemcpy(&nb, (long long *)brp + mb, 8, cudaMemcpyDeviceToHost);
        if (err != cudaSuccess) { dev_free(brp); return st_of(err); }
        const double bytes = (double)nb * (double)(b * b * esz + 4) + 4.0 * (double)(mb + 1);
        if (h->bcsr_b == 0 || bytes < best_bytes) {
          dev_free(h->bcsr_brp64);
          h->bcsr_brp64 = (long long *)brp;
          h->bcsr_b = b; h->bcsr_mb = mb; h->bcsr_nb = nb;
          best_bytes = bytes;
        } else {
          dev_free(brp);
        }
      }
      h->ext_slots[e] = (double)h->bcsr_nb * h->bcsr_b * h->bcsr_b;
      h->ext_bytes[e] = best_bytes;
    }
  }
  h->ext_known[e] = true;
  update_admissible(h);
  return SMAT_OK;
}

// Products per timed repetition: enough back to back that a repetition spans
// about 40 us, since on this GPU the event-timed duration of a single short
// kernel moves in steps of about 2 us (measured: an empty kernel 3.5-3.8 us,
// 256 KB and 4 MB reads both 5.6-5.8 us), too coarse to rank products of
// 5-20 us one launch at a time.
int products_per_rep(float ms_per_product) {
  const float target_ms = 0.040f;
  if (!(ms_per_product > 0.0f)) return 1;
  const int g = (int)std::ceil(target_ms / ms_per_product);
  return g < 1 ? 1 : (g > 32 ? 32 : g);
}

// Kernel search for ELL / DIA (the paper's per-format implementation choice,
// Sec. 3): time the candidate batch widths once on zero vectors, keep the
// faster; for ELL then time the lane-striped row mapping at that width, for
// DIA the kernel whose stripes are staged by bulk copies.  Run when the
// format is built.
smat_status_t measure_batch_width(smat_s *h, int variant, cudaStream_t s) {
  int cand[2];
  const int nc = batch_width_candidates(h, variant, cand);
  int &slot = variant == SMAT_V_DIA ? h->dia_u : h->ell_u;
  const bool try_lane = variant == SMAT_V_ELL;
  const bool try_staged = variant == SMAT_V_DIA && dia_staged_ok(h, 1);
  if (nc == 1 && !try_lane && !try_staged) {
    slot = cand[0];
    return SMAT_OK;
  }
  DevBuf x(s), y(s);
  const size_t xs = (size_t)std::max<int64_t>(h->n, 1) * tsize(h), ys = (size_t)std::max<int64_t>(h->m, 1) * tsize(h);
  TRY(x.alloc(xs));
  TRY(y.alloc(ys));
  TRY(cudaMemsetAsync(x.p, 0, xs, s));
  const double one = 1.0, zero = 0.0;
  const float onef = 1.0f, zerof = 0.0f;
  const void *a = h->dtype == SMAT_F64 ? (const void *)&one : (const void *)&onef;
  const void *b = h->dtype == SMAT_F64 ? (const void *)&zero : (const void *)&zerof;
  cudaEvent_t ev[10] = {};  // two per repetition (at most 5)
  struct EvFree {
    cudaEvent_t *v;
    ~EvFree() { for (int k = 0; k < 10; ++k) if (v[k]) cudaEventDestroy(v[k]); }
  } evf{ev};
  for (int k = 0; k < 10; ++k) TRY(cudaEventCreate(&ev[k]));
  double enq_us = 10.0;  // host time to queue one timed product
  // nrep repetitions of `group` products each, queued together behind a
  // device hold so that each pair of events brackets its products alone;
  // per-product milliseconds in ms[0..nrep)
  auto blocks = [&](int u, int lane, int group, int nrep, float *ms) -> smat_status_t {
    TRY(queue_ahead(s, &enq_us, group * nrep, [&]() -> cudaError_t {
      cudaError_t q = cudaSuccess;
      for (int r = 0; r < nrep && q == cudaSuccess; ++r) {
        q = cudaEventRecord(ev[2 * r], s);
        for (int g = 0; g < group && q == cudaSuccess; ++g)
          q = launch_spmv_width(h, variant, u, lane, a, x.p, b, y.p, s);
        if (q == cudaSuccess) q = cudaEventRecord(ev[2 * r + 1], s);
      }
      return q;
    }));
    TRY(cudaEventSynchronize(ev[2 * nrep - 1]));
    for (int r = 0; r < nrep; ++r) {
      TRY(cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]));
      ms[r] /= (float)group;
    }
    return SMAT_OK;
  };
  auto time_it = [&](int u, int lane, float *med) -> smat_status_t {
    for (int w = 0; w < 2; ++w) TRY(launch_spmv_width(h, variant, u, lane, a, x.p, b, y.p, s));
    float wms;
    TRYS(blocks(u, lane, 1, 1, &wms));  // one product alone sizes the repetitions
    const int group = products_per_rep(wms);
    const int nrep = group > 1 ? 3 : 5;   // about as many products as five single ones
    float ms[5];
    TRYS(blocks(u, lane, group, nrep, ms));
    std::sort(ms, ms + nrep);
    *med = ms[nrep / 2];
    return SMAT_OK;
  };
  float best = 1e30f;
  int best_u = cand[0];
  for (int c = 0; c < nc; ++c) {
    float med;
    TRYS(time_it(cand[c], 0, &med));
    if (med < best) { best = med; best_u = cand[c]; }
  }
  slot = best_u;
  if (try_lane) {
    float med;
    TRYS(time_it(best_u, 1, &med));
    h->ell_lane = med < best ? 1 : 0;
  }
  if (try_staged) {
    h->dia_staged = 0;
    for (int k = 1; k <= dia_staged_kernels(); ++k) {
      if (!dia_staged_ok(h, k)) continue;
      float med;
      TRYS(time_it(best_u, 1 + k, &med));
      if (med < best) { best = med; h->dia_staged = k; }
    }
  }
  return SMAT_OK;
}

smat_status_t build_format(smat_s *h, int fmt, cudaStream_t s) {
  if (fmt == SMAT_FMT_CSR) return SMAT_OK;
  if (!h->have_features) TRYS(compute_features(h, s));
  if (fmt == SMAT_FMT_ELL) {
    if (h->ell_val) return SMAT_OK;
    if (!(h->f.admissible & (1u << SMAT_V_ELL))) return SMAT_ERR_UNSUPPORTED;
    const int64_t K = h->f.max_rd;
    if (K == 0) return SMAT_ERR_UNSUPPORTED;
    void *c = nullptr, *v = nullptr;
    TRY(dev_alloc(&c, (size_t)(K * h->P) * 4));
    cudaError_t e = dev_alloc(&v, (size_t)(K * h->P) * h->esz);
    if (e != cudaSuccess) { dev_free(c); return st_of(e); }
    h->ell_col = (int32_t *)c; h->ell_val = v; h->ell_K = K; h->ell_u = 0; h->ell_lane = 0;
    TRY(launch_to_ell(h, K, h->ell_col, h->ell_val, s));
    return measure_batch_width(h, SMAT_V_ELL, s);
  }
  if (fmt == SMAT_FMT_DIA) {
    if (h->dia_val) return SMAT_OK;
    if (!(h->f.admissible & (1u << SMAT_V_DIA))) return SMAT_ERR_UNSUPPORTED;
    const int64_t nd = (int64_t)h->dia_offsets.size();
    void *o = nullptr, *v = nullptr;
    TRY(dev_alloc(&o, (size_t)nd * 4));
    cudaError_t e = dev_alloc(&v, (size_t)(nd * h->P) * h->esz);
    if (e != cudaSuccess) { dev_free(o); return st_of(e); }
    h->dia_off = (int32_t *)o; h->dia_val = v; h->dia_nd = nd;
    TRY(cudaMemcpyAsync(h->dia_off, h->dia_offsets.data(), (size_t)nd * 4, cudaMemcpyHostToDevice, s));
    TRY(launch_to_dia(h, h->dia_off, nd, h->dia_val, s));
    TRY(cudaStreamSynchronize(s));  // the host offsets buffer must outlive the copy
    h->dia_u = 0;
    h->dia_staged = 0;
    return measure_batch_width(h, SMAT_V_DIA, s);
  }
  if (fmt == SMAT_FMT_COO) {
    if (h->coo_row || h->coo_empty) return SMAT_OK;
    void *r = nullptr;
    if (h->nnz > 0) {
      TRY(dev_alloc(&r, (size_t)h->nnz * 4));
      h->coo_row = (int32_t *)r;
      TRY(launch_to_coo(h, h->coo_row, s));
    }
    if (h->f.empty_rows > 0) {
      void *l = nullptr;
      DevBuf cnt(s);
      TRY(dev_alloc(&l, (size_t)h->f.empty_rows * 4));
      h->coo_empty = (int32_t *)l;
      h->coo_nempty = h->f.empty_rows;
      TRY(cnt.alloc(sizeof(int)));
      TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int), s));
      TRY(launch_empty_rows(h, h->coo_empty, cnt.as<int>(), s));
      TRY(cudaStreamSynchronize(s));
    }
    return SMAT_OK;
  }
  if (fmt == SMAT_FMT_HYB || fmt == SMAT_FMT_SELL || fmt == SMAT_FMT_BCSR || fmt == SMAT_FMT_SPLIT) {
    const int v = fmt == SMAT_FMT_HYB ? SMAT_V_HYB
                  : fmt == SMAT_FMT_SELL ? SMAT_V_SELL
                  : fmt == SMAT_FMT_BCSR ? SMAT_V_BCSR : SMAT_V_SPLIT;
    TRYS(ext_layout(h, v, h->sell_sigma, s));
    if (!(h->f.admissible & (1u << v))) return SMAT_ERR_UNSUPPORTED;
    struct Undo {  // a failed build leaves no half-built format behind
      smat_s *h; int fmt; bool armed = true;
      ~Undo() { if (armed) free_format(h, fmt); }
    } undo{h, fmt};
    void *p = nullptr;
    if (fmt == SMAT_FMT_HYB) {
      if (h->hyb_built) { undo.armed = false; return SMAT_OK; }
      const int64_t K = h->hyb_K, nc = h->hyb_ncoo;
      TRY(dev_alloc(&p, (size_t)(K * h->P) * 4)); h->hyb_ecol = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)(K * h->P) * h->esz)); h->hyb_eval = p;
      TRY(dev_alloc(&p, (size_t)nc * 4)); h->hyb_crow = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)nc * 4)); h->hyb_ccol = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)nc * h->esz)); h->hyb_cval = p;
      DevBuf cnt(s), off(s);
      TRY(cnt.alloc((size_t)h->m * 8));
      TRY(off.alloc((size_t)(h->m + 1) * 8));
      TRY(launch_hyb_tail_counts(h, K, cnt.as<long long>(), s));
      TRY(exclusive_scan(cnt.as<long long>(), h->m, off.as<long long>(), s));
      TRY(launch_to_hyb(h, K, off.as<long long>(), h->hyb_ecol, h->hyb_eval, h->hyb_crow, h->hyb_ccol, h->hyb_cval, s));
      TRY(cudaStreamSynchronize(s));
      h->hyb_built = true;
    } else if (fmt == SMAT_FMT_SELL) {
      if (h->sell_val) { undo.armed = false; return SMAT_OK; }
      TRY(dev_alloc(&p, (size_t)h->sell_slots * 4)); h->sell_col = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)h->sell_slots * h->esz)); h->sell_val = p;
      TRY(launch_to_sell(h, s));
    } else if (fmt == SMAT_FMT_SPLIT) {
      if (h->split_built) { undo.armed = false; return SMAT_OK; }
      const size_t nl = (size_t)h->split_nl, nc = (size_t)h->split_nc, ns = (size_t)h->split_ns,
                   ne = (size_t)h->split_ne;
      TRY(dev_alloc(&p, (nl + 1) * 4)); h->split_lchunk = (int32_t *)p;
      TRY(dev_alloc(&p, nl * 4)); h->split_lrows = (int32_t *)p;
      TRY(dev_alloc(&p, nc * 4)); h->split_crow = (int32_t *)p;
      TRY(dev_alloc(&p, nc * 4)); h->split_cstart = (int32_t *)p;
      TRY(dev_alloc(&p, nc * 4)); h->split_cend = (int32_t *)p;
      TRY(dev_alloc(&p, ns * 4)); h->split_srow = (int32_t *)p;
      TRY(dev_alloc(&p, ns * 4)); h->split_scol = (int32_t *)p;
      TRY(dev_alloc(&p, ns * h->esz)); h->split_sval = p;
      TRY(dev_alloc(&p, ne * 4)); h->split_empty = (int32_t *)p;
      TRY(dev_alloc(&p, nc * tsize(h))); h->split_part = p;
      DevBuf cnt(s), pre(s);
      const size_t M = (size_t)h->m;
      TRY(cnt.alloc(4 * M * 8));
      TRY(pre.alloc(4 * (M + 1) * 8));
      long long *c = cnt.as<long long>(), *q = pre.as<long long>();
      TRY(launch_split_counts(h, c, c + M, c + 2 * M, c + 3 * M, s));
      for (int k = 0; k < 4; ++k) TRY(exclusive_scan(c + k * M, (long long)M, q + k * (M + 1), s));
      TRY(launch_split_fill(h, q, q + (M + 1), q + 2 * (M + 1), q + 3 * (M + 1), s));
      TRY(cudaStreamSynchronize(s));
      h->split_built = true;
    } else {
      if (h->bcsr_val) { undo.armed = false; return SMAT_OK; }
      const int64_t bb = (int64_t)h->bcsr_b * h->bcsr_b;
      TRY(dev_alloc(&p, (size_t)(h->bcsr_mb + 1) * 4)); h->bcsr_rowptr = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)h->bcsr_nb * 4)); h->bcsr_col = (int32_t *)p;
      TRY(dev_alloc(&p, (size_t)(h->bcsr_nb * bb) * h->esz)); h->bcsr_val = p;
      TRY(launch_to_bcsr(h, h->bcsr_brp64, s));
      h->bcsr_cb = 0;
      if (h->bcsr_mb > 0 && h->bcsr_nb > 0 && h->bcsr_nb % h->bcsr_mb == 0) {
        DevBuf flag(s);
        TRY(flag.alloc(4));
        TRY(cudaMemsetAsync(flag.p, 0, 4, s));
        TRY(launch_bcsr_uniform(h, h->bcsr_nb / h->bcsr_mb, flag.as<int>(), s));
        int f = 1;
        TRY(cudaMemcpyAsync(&f, flag.p, 4, cudaMemcpyDeviceToHost, s));
        TRY(cudaStreamSynchronize(s));
        if (f == 0) h->bcsr_cb = (int32_t)(h->bcsr_nb / h->bcsr_mb);
      }
    }
    undo.armed = false;
    return SMAT_OK;
  }
  return SMAT_ERR_INVALID_ARG;
}

}  // namespace

cudaError_t stream_scratch(const smat_s *h, cudaStream_t s, Scratch *out, bool claim) {
  std::lock_guard<std::mutex> lock(h->scratch_mu);
  if (!claim) {
    *out = Scratch{h->carry, h->split_part};
    return cudaSuccess;
  }
  if (!h->scratch_owned || h->scratch_owner == s) {
    h->scratch_owned = true;
    h->scratch_owner = s;
    *out = Scratch{h->carry, h->split_part};
    return cudaSuccess;
  }
  const size_t carry = (h->carry_bytes + 255) / 256 * 256;
  const size_t need = carry + (size_t)h->split_nc * (h->dtype == SMAT_F64 ? 8 : 4);
  smat_s::StreamScratch *hit = nullptr;
  for (auto &e : h->more_scratch)
    if (e.stream == s) hit = &e;
  if (!hit || hit->bytes < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return cudaErrorStreamCaptureUnsupported;
    void *p = nullptr;
    cudaError_t e = dev_alloc(&p, need > 0 ? need : 256);
    if (e != cudaSuccess) return e;
    if (hit) {
      cudaStreamSynchronize(s);  // the old buffer's products on s are done
      dev_free(hit->p);
      hit->p = p;
      hit->bytes = need;
    } else {
      h->more_scratch.push_back({s, p, need});
      hit = &h->more_scratch.back();
    }
  }
  *out = Scratch{hit->p, (char *)hit->p + carry};
  return cudaSuccess;
}

void free_stream_scratch(smat_s *h) {
  for (auto &e : h->more_scratch) dev_free(e.p);
  h->more_scratch.clear();
}

namespace {

smat_status_t ensure_scratch(smat_s *h, int variant) {
  size_t need = carry_bytes_needed(h, variant);
  if (need <= h->carry_bytes) return SMAT_OK;
  void *p = nullptr;
  TRY(dev_alloc(&p, need));
  dev_free(h->carry);
  h->carry = p;
  h->carry_bytes = need;
  return SMAT_OK;
}

bool variant_ready(const smat_s *h, int v) {
  int fmt = variant_format(v);
  if (v == SMAT_V_CSR_MERGE && h->m > 0 && !h->merge_coords) return false;
  if (fmt == SMAT_FMT_ELL && !h->ell_val) return false;
  if (fmt == SMAT_FMT_DIA && !h->dia_val) return false;
  if (fmt == SMAT_FMT_COO && !h->coo_row && !(h->nnz == 0)) return false;
  if (fmt == SMAT_FMT_COO && h->f.empty_rows > 0 && !h->coo_empty) return false;
  if (fmt == SMAT_FMT_HYB && !h->hyb_built) return false;
  if (fmt == SMAT_FMT_SELL && !h->sell_val) return false;
  if (fmt == SMAT_FMT_BCSR && !h->bcsr_val) return false;
  if (fmt == SMAT_FMT_SPLIT && !h->split_built) return false;
  if (carry_bytes_needed(h, v) > h->carry_bytes) return false;
  return true;
}

smat_status_t prepare_variant(smat_s *h, int v, cudaStream_t s) {
  if (v < 0 || v >= SMAT_NUM_ALL_VARIANTS) return SMAT_ERR_INVALID_ARG;
  int fmt = variant_format(v);
  if (fmt != SMAT_FMT_CSR && !h->have_features) TRYS(compute_features(h, s));
  TRYS(build_format(h, fmt, s));
  TRYS(ensure_scratch(h, v));
  if (v == SMAT_V_CSR_MERGE && !h->merge_coords && h->m > 0) {
    void *p = nullptr;
    TRY(dev_alloc(&p, (size_t)(merge_tiles(h->m, h->nnz) + 1) * 8));
    h->merge_coords = p;
    TRY(launch_merge_partition(h->rowptr, h->m, h->nnz, h->merge_coords, s));
  }
  return SMAT_OK;
}

// ---------------------------------------------------------------------------
// Execute & measure (Sec. 6) / brute-force search (Sec. 7.3): median of timed
// repetitions per candidate, on zero vectors.
// ---------------------------------------------------------------------------
smat_status_t trial(smat_s *h, const std::vector<int> &cands, const smat_tune_opts_t &o, cudaStream_t s,
                    int *best) {
  Range r("trial");
  DevBuf x(s), y(s);
  TRY(x.alloc((size_t)std::max<int64_t>(h->n, 1) * tsize(h)));
  TRY(y.alloc((size_t)std::max<int64_t>(h->m, 1) * tsize(h)));
  TRY(cudaMemsetAsync(x.p, 0, (size_t)std::max<int64_t>(h->n, 1) * tsize(h), s));
  TRY(cudaMemsetAsync(y.p, 0, (size_t)std::max<int64_t>(h->m, 1) * tsize(h), s));
  const double one = 1.0, zero = 0.0;
  const float onef = 1.0f, zerof = 0.0f;
  const void *a = h->dtype == SMAT_F64 ? (const void *)&one : (const void *)&onef;
  const void *b = h->dtype == SMAT_F64 ? (const void *)&zero : (const void *)&zerof;
  const int reps_max = std::max(1, o.trial_reps);
  std::vector<cudaEvent_t> ev((size_t)reps_max * 2 + 2);  // two per repetition, two for the sizing product
  for (auto &e : ev) TRY(cudaEventCreate(&e));
  struct EvGuard {
    std::vector<cudaEvent_t> &v;
    ~EvGuard() { for (auto e : v) if (e) cudaEventDestroy(e); }
  } guard{ev};
  const double t_start = now_ms();
  float best_ms = 1e30f;
  double enq_us = 10.0;  // host time to queue one timed product
  *best = -1;
  std::vector<std::pair<int, float>> timed_here;
  for (int v : cands) {
    if (*best >= 0 && now_ms() - t_start > o.trial_budget_ms) break;
    smat_status_t ps = prepare_variant(h, v, s);
    if (ps == SMAT_ERR_UNSUPPORTED || ps == SMAT_ERR_ALLOC) continue;  // skip, keep searching
    TRYS(ps);
    for (int w = 0; w < o.trial_warmup; ++w) TRY(launch_spmv(h, v, a, x.p, b, y.p, s, false));
    // one product timed alone sizes the repetitions: `group` products each,
    // and fewer repetitions when grouped, so that a candidate costs about
    // trial_reps products as before (at least 3 repetitions)
    int group = 1;
    {
      const size_t w0 = (size_t)reps_max * 2;
      TRY(queue_ahead(s, &enq_us, 1, [&]() -> cudaError_t {
        cudaError_t q = cudaEventRecord(ev[w0], s);
        if (q == cudaSuccess) q = launch_spmv(h, v, a, x.p, b, y.p, s, false);
        if (q == cudaSuccess) q = cudaEventRecord(ev[w0 + 1], s);
        return q;
      }));
      TRY(cudaEventSynchronize(ev[w0 + 1]));
      float wms = 0.0f;
      TRY(cudaEventElapsedTime(&wms, ev[w0], ev[w0 + 1]));
      group = products_per_rep(wms);
    }
    const int reps = std::max(std::min(reps_max, 3), (reps_max + group - 1) / group);
    // racing: a candidate whose first few products already take trial_race
    // times the best so far stops there (its median of those is kept)
    const int first = (o.trial_race > 0.0f && best_ms < 1e30f) ? std::min(reps, 3) : reps;
    int done = 0;
    // each repetition times `group` products back to back, queued behind a
    // device hold so that its pair of events brackets the products alone
    auto timed = [&](int upto) -> cudaError_t {
      cudaError_t e = queue_ahead(s, &enq_us, (upto - done) * group, [&]() -> cudaError_t {
        for (int r = done; r < upto; ++r) {
          cudaError_t q = cudaEventRecord(ev[2 * r], s);
          for (int g = 0; g < group && q == cudaSuccess; ++g) q = launch_spmv(h, v, a, x.p, b, y.p, s, false);
          if (q == cudaSuccess) q = cudaEventRecord(ev[2 * r + 1], s);
          if (q != cudaSuccess) return q;
        }
        return cudaSuccess;
      });
      if (e != cudaSuccess) return e;
      done = upto;
      return cudaStreamSynchronize(s);
    };
    auto median = [&](std::vector<float> &ms) -> cudaError_t {
      ms.resize((size_t)done);
      for (int r = 0; r < done; ++r) {
        cudaError_t e = cudaEventElapsedTime(&ms[(size_t)r], ev[2 * r], ev[2 * r + 1]);
        if (e != cudaSuccess) return e;
        ms[(size_t)r] /= (float)group;
      }
      std::nth_element(ms.begin(), ms.begin() + done / 2, ms.end());
      return cudaSuccess;
    };
    std::vector<float> ms;
    TRY(timed(first));
    TRY(median(ms));
    float med = ms[(size_t)done / 2];
    if (done < reps && !(med > o.trial_race * best_ms)) {
      TRY(timed(reps));
      TRY(median(ms));
      med = ms[(size_t)done / 2];
    }
    h->timings[v] = med;
    timed_here.emplace_back(v, med);
    if (med < best_ms) {
      best_ms = med;
      *best = v;
    }
    if (!o.keep_formats) {
      // drop a trialled format right away unless it is the best so far
      for (int fmt = SMAT_FMT_ELL; fmt <= SMAT_FMT_SPLIT; ++fmt)
        if (fmt != variant_format(*best)) free_format(h, fmt);
    }
  }
  if (*best < 0) {
    *best = SMAT_V_CSR_SCALAR;
    return SMAT_OK;
  }
  // near-ties: among the candidates within trial_tie of the fastest (0: among
  // exactly equal medians), the one whose format moves the fewest matrix
  // bytes (it contends least when other products run beside it), then the
  // lowest variant id
  if (o.trial_tie >= 0.0f) {
    const float lim = best_ms * (1.0f + o.trial_tie);
    int pick = *best;
    double pick_bytes = variant_bytes(h, pick);
    for (const auto &t : timed_here)
      if (t.second <= lim) {
        const double b = variant_bytes(h, t.first);
        if (b < pick_bytes || (b == pick_bytes && t.first < pick)) {
          pick = t.first;
          pick_bytes = b;
        }
      }
    if (pick != *best) {
      const int fastest = *best;
      smat_status_t ps = variant_ready(h, pick) ? SMAT_OK : prepare_variant(h, pick, s);
      if (ps == SMAT_OK && variant_ready(h, pick)) {
        *best = pick;
        if (!o.keep_formats && variant_format(fastest) != variant_format(pick)) free_format(h, variant_format(fastest));
      } else if (ps != SMAT_ERR_UNSUPPORTED && ps != SMAT_ERR_ALLOC) {
        return ps;
      }
    }
  }
  return SMAT_OK;
}

// The paper's observations (Sec. 4) as an ordered rule set: DIA, ELL, CSR, COO
// (Sec. 6 gives this order).  CSR maps to the CSR-vector width that fits the
// mean row length.
int rules_select(const smat_features_t &f, uint32_t ok) {
  if ((ok >> SMAT_V_DIA) & 1u) {
    if (f.ndiags <= 500 && (f.ndiags < 25 || f.er_dia > 0.6 || f.ntdiags_ratio > 0.4)) return SMAT_V_DIA;
  }
  if ((ok >> SMAT_V_ELL) & 1u) {
    if ((f.max_rd < 5 || f.er_ell > 0.9) && f.var_rd < 0.5) return SMAT_V_ELL;
  }
  int csr = f.aver_rd < 8.0 ? SMAT_V_CSR_VEC4 : (f.aver_rd < 24.0 ? SMAT_V_CSR_VEC8 : SMAT_V_CSR_VEC32);
  bool small_world = f.r_valid && f.r >= 1.0 && f.r < 4.0;
  if (small_world && ((ok >> SMAT_V_COO) & 1u)) return SMAT_V_COO;
  if ((ok >> csr) & 1u) return csr;
  for (int v = 0; v < SMAT_NUM_VARIANTS; ++v)
    if ((ok >> v) & 1u) return v;
  return SMAT_V_CSR_SCALAR;
}

smat_status_t mlp_probs(const smat_s *h, float probs[SMAT_NUM_VARIANTS], cudaStream_t s) {
  Range r("mlp");
  Model M;
  if (!model_copy(&M)) return SMAT_ERR_MODEL;
  float v[12];
  feature_vector(h->f, v);
  for (int i = 0; i < 12; ++i) v[i] = (v[i] - M.mean[i]) / (M.stdv[i] > 0 ? M.stdv[i] : 1.0f);
  DevBuf d(s);
  const size_t np = SMAT_MLP_PARAMS;
  TRY(d.alloc((np + 12 + 8) * sizeof(float)));
  float *dp = d.as<float>(), *dx = dp + np, *dz = dx + 12;
  TRY(cudaMemcpyAsync(dp, M.params, np * sizeof(float), cudaMemcpyHostToDevice, s));
  TRY(cudaMemcpyAsync(dx, v, 12 * sizeof(float), cudaMemcpyHostToDevice, s));
  TRY(launch_mlp_forward(dp, dx, 1, dz, s));
  float z[8];
  TRY(cudaMemcpyAsync(z, dz, sizeof(z), cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  float zmax = -INFINITY;
  for (int c = 0; c < 8; ++c)
    if ((h->f.admissible >> c) & 1u) zmax = std::max(zmax, z[c]);
  double se = 0.0;
  for (int c = 0; c < 8; ++c) se += ((h->f.admissible >> c) & 1u) ? std::exp((double)(z[c] - zmax)) : 0.0;
  for (int c = 0; c < 8; ++c)
    probs[c] = ((h->f.admissible >> c) & 1u) ? (float)(std::exp((double)(z[c] - zmax)) / se) : 0.0f;
  return SMAT_OK;
}

smat_status_t check_handle(const smat_s *h) { return h ? SMAT_OK : SMAT_ERR_INVALID_ARG; }

// Streams on which smat_spmv_many runs independent products side by side,
// one set per device, created on first use and kept for the process.
struct ForkPool {
  static constexpr int N = 16;
  cudaStream_t s[N] = {};
  cudaEvent_t join[N] = {};
  cudaEvent_t fork = nullptr;
  std::mutex mu;
};

cudaError_t fork_pool(ForkPool **out) {
  static ForkPool pools[64];
  static std::mutex init_mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  ForkPool &p = pools[dev];
  std::lock_guard<std::mutex> lock(init_mu);
  if (!p.fork) {
    for (int k = 0; k < ForkPool::N; ++k) {
      if (!p.s[k]) e = cudaStreamCreateWithFlags(&p.s[k], cudaStreamNonBlocking);
      if (e == cudaSuccess && !p.join[k]) e = cudaEventCreateWithFlags(&p.join[k], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
    e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = &p;
  return cudaSuccess;
}

}  // namespace
}  // namespace smat

using namespace smat;

extern "C" {

void smat_tune_opts_default(smat_tune_opts_t *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = SMAT_TUNE_LEARNED;
  o->fixed_variant = SMAT_V_CSR_SCALAR;
  o->conf_threshold = 0.6f;
  o->fallback_topk = 3;
  o->tau_num = 3;
  o->tau_den = 5;
  o->fill_ratio_max = 20;
  o->bytes_cap = 4.0;
  o->trial_reps = 10;
  o->trial_warmup = 2;
  o->trial_budget_ms = 2000.0;
  o->allowed = 0;
  o->keep_formats = 0;
  o->sell_sigma = 256;
  o->trial_extended = 1;
  o->plan_cache = 0;
  o->trial_race = 1.3f;
  o->trial_tie = 0.02f;
}

const char *smat_status_string(smat_status_t s) {
  switch (s) {
    case SMAT_OK: return "ok";
    case SMAT_ERR_INVALID_ARG: return "invalid argument";
    case SMAT_ERR_INVALID_CSR: return "invalid CSR structure";
    case SMAT_ERR_ALLOC: return "allocation failed";
    case SMAT_ERR_CUDA: return "CUDA error";
    case SMAT_ERR_UNSUPPORTED: return "unsupported (size or format not admissible)";
    case SMAT_ERR_MODEL: return "selector model missing or malformed";
    case SMAT_ERR_NOT_CONVERGED: return "not converged";
  }
  return "unknown status";
}

smat_status_t smat_release_cached_memory(void) {
  std::lock_guard<std::mutex> lk(pool_mu());
  bool ok = true;
  int cur = 0;
  cudaGetDevice(&cur);
  for (int dev = 0; dev < 64; ++dev) {
    DevPool &d = pools()[dev];
    if (!d.pool) continue;
    ok = cudaSetDevice(dev) == cudaSuccess && ok;
    ok = cudaDeviceSynchronize() == cudaSuccess && ok;
    ok = cudaMemPoolTrimTo(d.pool, 0) == cudaSuccess && ok;
  }
  cudaSetDevice(cur);
  return ok ? SMAT_OK : SMAT_ERR_CUDA;
}

void smat_test_fail_alloc_after(int32_t k) {
  g_alloc_count = 0;
  g_alloc_fail_at = k;
}

smat_status_t smat_create(smat_handle_t *out, int64_t m, int64_t n, int64_t nnz, const int32_t *rowptr,
                          const int32_t *colidx, const void *vals, smat_dtype_t dtype) {
  if (!out) return SMAT_ERR_INVALID_ARG;
  *out = nullptr;
  if (m < 0 || n < 0 || nnz < 0 || !rowptr) return SMAT_ERR_INVALID_ARG;
  if (dtype != SMAT_F64 && dtype != SMAT_F32 && dtype != SMAT_BF16) return SMAT_ERR_INVALID_ARG;
  if (nnz > 0 && (!colidx || !vals)) return SMAT_ERR_INVALID_ARG;
  if (m > INT32_MAX - 1 || n > INT32_MAX || nnz > INT32_MAX || m + n > (int64_t)INT32_MAX * 2)
    return SMAT_ERR_UNSUPPORTED;
  smat_s *h = new (std::nothrow) smat_s();
  if (!h) return SMAT_ERR_ALLOC;
  h->m = m; h->n = n; h->nnz = nnz; h->dtype = dtype; h->esz = elem_size(dtype); h->P = pitch_of(m);
  for (auto &t : h->timings) t = -1.0f;
  auto fail = [&](smat_status_t s) { smat_destroy(h); return s; };
  void *p = nullptr;
  cudaError_t e = dev_alloc(&p, (size_t)(m + 1) * 4);
  if (e != cudaSuccess) return fail(st_of(e));
  h->rowptr = (int32_t *)p;
  if (nnz > 0) {
    if ((e = dev_alloc(&p, (size_t)nnz * 4)) != cudaSuccess) return fail(st_of(e));
    h->colidx = (int32_t *)p;
    if ((e = dev_alloc(&p, (size_t)nnz * h->esz)) != cudaSuccess) return fail(st_of(e));
    h->val = p;
  }
  if ((e = cudaMemcpy(h->rowptr, rowptr, (size_t)(m + 1) * 4, cudaMemcpyDefault)) != cudaSuccess) return fail(st_of(e));
  if (nnz > 0) {
    if ((e = cudaMemcpy(h->colidx, colidx, (size_t)nnz * 4, cudaMemcpyDefault)) != cudaSuccess) return fail(st_of(e));
    if ((e = cudaMemcpy(h->val, vals, (size_t)nnz * h->esz, cudaMemcpyDefault)) != cudaSuccess) return fail(st_of(e));
  }
  // K1: structural validation on the device, reported through a flag.
  // One block: the flag, then one bit per stored entry for the row starts.
  void *flag = nullptr;
  const size_t vbytes = 16 + validate_starts_words(nnz) * 4;
  if ((e = dev_alloc(&flag, vbytes)) != cudaSuccess) return fail(st_of(e));
  int hf = 0;
  e = cudaMemset(flag, 0, vbytes);
  if (e == cudaSuccess) e = launch_validate(h, (int *)flag, (unsigned *)((char *)flag + 16), 0);
  if (e == cudaSuccess) e = cudaMemcpy(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost);
  dev_free(flag);
  if (e != cudaSuccess) return fail(st_of(e));
  if (hf) return fail(SMAT_ERR_INVALID_CSR);
  *out = h;
  return SMAT_OK;
}

smat_status_t smat_destroy(smat_handle_t h) {
  if (!h) return SMAT_OK;
  dev_free(h->rowptr); dev_free(h->colidx); dev_free(h->val);
  free_format(h, SMAT_FMT_ELL); free_format(h, SMAT_FMT_DIA); free_format(h, SMAT_FMT_COO);
  free_ext_layouts(h);
  dev_free(h->carry); dev_free(h->stage_x); dev_free(h->stage_y); dev_free(h->merge_coords);
  if (h->pst[0]) {
    for (cudaStream_t st : h->pst) cudaStreamSynchronize(st);
    for (int q = 0; q < 2; ++q) {
      cudaEventDestroy(h->pev_x[q]); cudaEventDestroy(h->pev_run[q]); cudaEventDestroy(h->pev_out[q]);
      dev_free(h->pstage_x[q]); dev_free(h->pstage_y[q]);
    }
  }
  free_stream_scratch(h);
  if (h->pst[0])
    for (cudaStream_t st : h->pst) cudaStreamDestroy(st);
  delete h;
  return SMAT_OK;
}

smat_status_t smat_tune(smat_handle_t h, const smat_tune_opts_t *opts_in, void *stream) {
  TRYS(check_handle(h));
  cudaStream_t s = (cudaStream_t)stream;
  smat_tune_opts_t o;
  if (opts_in) o = *opts_in; else { smat_tune_opts_default(&o); if (!model_loaded()) o.mode = SMAT_TUNE_EXHAUSTIVE; }
  if (o.mode < SMAT_TUNE_LEARNED || o.mode > SMAT_TUNE_FIXED) return SMAT_ERR_INVALID_ARG;
  if (o.tau_den <= 0 || o.tau_num < 0 || o.fill_ratio_max <= 0) return SMAT_ERR_INVALID_ARG;
  if (o.sell_sigma == 0) o.sell_sigma = 256;
  if (o.sell_sigma < 32 || o.sell_sigma > 8192 || o.sell_sigma % 32 != 0) return SMAT_ERR_INVALID_ARG;
  const double t0 = now_ms();
  Range r_tune("smat_tune");
  if (!h->have_features || o.tau_num != h->tau_num || o.tau_den != h->tau_den ||
      o.fill_ratio_max != h->fill_ratio_max) {
    Range r("features");
    h->tau_num = o.tau_num; h->tau_den = o.tau_den; h->fill_ratio_max = o.fill_ratio_max;
    h->bytes_cap = o.bytes_cap > 0 ? o.bytes_cap : 4.0;
    TRYS(compute_features(h, s));
  } else if (o.bytes_cap > 0 && o.bytes_cap != h->bytes_cap) {
    h->bytes_cap = o.bytes_cap;
    update_admissible(h);
  }
  for (auto &t : h->timings) t = -1.0f;
  const uint32_t allowed = (o.allowed ? o.allowed : ALL_VARIANTS) & ALL_VARIANTS;
  h->plan_cached = false;
  h->confidence = -1.0f;
  h->trialled = 0;
  int v = SMAT_V_CSR_SCALAR;
  const bool use_cache = o.plan_cache && o.mode != SMAT_TUNE_FIXED;
  if (use_cache) {  // a plan recorded for this structure, if still admissible and allowed
    Range r("plan_cache");
    TRYS(ensure_plan_key(h, s));
    int cv = -1, csig = 0;
    if (plan_cache_lookup(h, &cv, &csig) && cv != SMAT_V_CSR_SCALAR_EXACT && ((allowed >> cv) & 1u)) {
      if (cv >= SMAT_V_HYB) {
        smat_status_t es = ext_layout(h, cv, cv == SMAT_V_SELL ? csig : o.sell_sigma, s);
        if (es != SMAT_OK && es != SMAT_ERR_ALLOC) return es;
      }
      if ((h->f.admissible >> cv) & 1u) {
        v = cv;
        h->plan_cached = true;
      }
    }
  }
  if (!h->plan_cached) {
    Range r_select("select");
    // layouts of the further formats the chosen mode may use
    for (int e = SMAT_V_HYB; e <= SMAT_V_SPLIT; ++e) {
      if (!((allowed >> e) & 1u)) continue;
      const bool want = o.mode == SMAT_TUNE_EXHAUSTIVE || (o.mode == SMAT_TUNE_FIXED && o.fixed_variant == e) ||
                        (o.mode == SMAT_TUNE_LEARNED && o.trial_extended &&
                         (e != SMAT_V_BCSR || h->f.max_rd <= 64));
      if (want) {
        smat_status_t es = ext_layout(h, e, o.sell_sigma, s);
        if (es == SMAT_ERR_ALLOC) continue;  // an unaffordable layout is not a candidate
        TRYS(es);
      }
    }
    const uint32_t ok = h->f.admissible & allowed;
    if (!ok) return SMAT_ERR_UNSUPPORTED;
    std::vector<int> cands;
    for (int c : {SMAT_V_DIA, SMAT_V_ELL, SMAT_V_CSR_SCALAR, SMAT_V_CSR_VEC4, SMAT_V_CSR_VEC8, SMAT_V_CSR_VEC32,
                  SMAT_V_CSR_MERGE, SMAT_V_COO})
      if ((ok >> c) & 1u) cands.push_back(c);
    std::vector<int> ext;
    for (int c = SMAT_V_HYB; c <= SMAT_V_SPLIT; ++c)
      if ((ok >> c) & 1u) ext.push_back(c);
    switch (o.mode) {
      case SMAT_TUNE_FIXED:
        if (o.fixed_variant < 0 || o.fixed_variant >= SMAT_NUM_ALL_VARIANTS ||
            o.fixed_variant == SMAT_V_CSR_SCALAR_EXACT)
          return SMAT_ERR_INVALID_ARG;
        if (!((ok >> o.fixed_variant) & 1u)) return SMAT_ERR_UNSUPPORTED;
        v = o.fixed_variant;
        break;
      case SMAT_TUNE_RULES:
        v = rules_select(h->f, ok);
        break;
      case SMAT_TUNE_EXHAUSTIVE:
        cands.insert(cands.end(), ext.begin(), ext.end());
        if (cands.empty()) return SMAT_ERR_UNSUPPORTED;
        TRYS(trial(h, cands, o, s, &v));
        h->trialled = 1;
        break;
      case SMAT_TUNE_LEARNED: {
        if (!model_loaded()) return SMAT_ERR_MODEL;
        float p[SMAT_NUM_VARIANTS];
        TRYS(mlp_probs(h, p, s));
        int arg = -1;
        for (int c = 0; c < SMAT_NUM_VARIANTS; ++c)
          if (((ok >> c) & 1u) && (arg < 0 || p[c] > p[arg])) arg = c;
        if (arg < 0) {  // only further formats are allowed: time them
          TRYS(trial(h, ext, o, s, &v));
          h->trialled = 1;
          break;
        }
        v = arg;
        h->confidence = p[arg];
        std::vector<int> top{arg};
        if (p[arg] < o.conf_threshold) {
          top = cands;
          std::sort(top.begin(), top.end(), [&](int a, int b) { return p[a] > p[b]; });
          if (o.fallback_topk > 0 && (int)top.size() > o.fallback_topk) top.resize((size_t)o.fallback_topk);
        }
        // the selector's classes do not include the further formats: time those
        // that move at most 1.25x the matrix bytes of its pick beside it (their
        // access patterns can beat a format that moves a little less)
        bool more = false;
        if (o.trial_extended)
          for (int c : ext)
            if (variant_bytes(h, c) <= 1.25 * variant_bytes(h, arg)) { top.push_back(c); more = true; }
        if (top.size() > 1 || more) {
          TRYS(trial(h, top, o, s, &v));
          h->trialled = 1;
        }
      } break;
    }
  }
  {
    Range r("prepare");
    TRYS(prepare_variant(h, v, s));
  }
  if (!o.keep_formats)
    for (int fmt = SMAT_FMT_ELL; fmt <= SMAT_FMT_SPLIT; ++fmt)
      if (fmt != variant_format(v)) free_format(h, fmt);
  TRY(cudaStreamSynchronize(s));
  h->variant = v;
  if (use_cache && !h->plan_cached) plan_cache_store(h, v, h->sell_sigma);
  h->tune_ms = now_ms() - t0;
  return SMAT_OK;
}

smat_status_t smat_get_plan_source(smat_handle_t h, int32_t *from_cache) {
  TRYS(check_handle(h));
  if (!from_cache) return SMAT_ERR_INVALID_ARG;
  *from_cache = h->plan_cached ? 1 : 0;
  return SMAT_OK;
}

smat_status_t smat_set_kernel(smat_handle_t h, smat_variant_t v, int32_t kernel) {
  TRYS(check_handle(h));
  if (v == SMAT_V_DIA) {
    if (kernel < 0 || kernel > dia_staged_kernels()) return SMAT_ERR_INVALID_ARG;
    if (!h->dia_val || (kernel > 0 && !dia_staged_ok(h, kernel))) return SMAT_ERR_UNSUPPORTED;
    h->dia_staged = kernel;
    return SMAT_OK;
  }
  if (v == SMAT_V_ELL) {
    if (kernel != 0 && kernel != 1) return SMAT_ERR_INVALID_ARG;
    if (!h->ell_val) return SMAT_ERR_UNSUPPORTED;
    h->ell_lane = kernel;
    return SMAT_OK;
  }
  return SMAT_ERR_INVALID_ARG;
}

smat_status_t smat_get_kernel(smat_handle_t h, smat_variant_t v, int32_t *kernel) {
  TRYS(check_handle(h));
  if (!kernel) return SMAT_ERR_INVALID_ARG;
  if (v == SMAT_V_DIA) {
    if (!h->dia_val) return SMAT_ERR_UNSUPPORTED;
    *kernel = h->dia_staged;
    return SMAT_OK;
  }
  if (v == SMAT_V_ELL) {
    if (!h->ell_val) return SMAT_ERR_UNSUPPORTED;
    *kernel = h->ell_lane;
    return SMAT_OK;
  }
  return SMAT_ERR_INVALID_ARG;
}

smat_status_t smat_spmv_many(const smat_handle_t *hs, int32_t count, const void *const *alphas,
                             const void *const *xs, const void *const *betas, void *const *ys, void *stream) {
  if (count < 0 || (count > 0 && (!hs || !alphas || !xs || !betas || !ys))) return SMAT_ERR_INVALID_ARG;
  for (int32_t i = 0; i < count; ++i) {
    const smat_s *h = hs[i];
    TRYS(check_handle(h));
    if (!alphas[i] || !betas[i] || (h->m > 0 && !ys[i]) || (h->n > 0 && !xs[i])) return SMAT_ERR_INVALID_ARG;
    if (!variant_ready(h, h->variant)) return SMAT_ERR_UNSUPPORTED;
  }
  cudaStream_t user = (cudaStream_t)stream;
  if (count == 1) {
    TRY(launch_spmv(hs[0], hs[0]->variant, alphas[0], xs[0], betas[0], ys[0], user));
    return SMAT_OK;
  }
  if (count == 0) return SMAT_OK;
  ForkPool *pool = nullptr;
  TRY(fork_pool(&pool));
  std::lock_guard<std::mutex> lock(pool->mu);
  TRY(cudaEventRecord(pool->fork, user));
  const int used = std::min<int>(count, ForkPool::N);
  for (int k = 0; k < used; ++k) TRY(cudaStreamWaitEvent(pool->s[k], pool->fork, 0));
  for (int32_t i = 0; i < count; ++i)
    TRY(launch_spmv(hs[i], hs[i]->variant, alphas[i], xs[i], betas[i], ys[i], pool->s[i % ForkPool::N]));
  for (int k = 0; k < used; ++k) {
    TRY(cudaEventRecord(pool->join[k], pool->s[k]));
    TRY(cudaStreamWaitEvent(user, pool->join[k], 0));
  }
  return SMAT_OK;
}

smat_status_t smat_spmv(smat_handle_t h, const void *alpha, const void *x, const void *beta, void *y,
                        void *stream) {
  TRYS(check_handle(h));
  if (!alpha || !beta || (h->m > 0 && !y) || (h->n > 0 && !x)) return SMAT_ERR_INVALID_ARG;
  if (!variant_ready(h, h->variant)) return SMAT_ERR_UNSUPPORTED;
  TRY(launch_spmv(h, h->variant, alpha, x, beta, y, (cudaStream_t)stream));
  return SMAT_OK;
}

smat_status_t smat_spmv_variant(smat_handle_t h, smat_variant_t v, const void *alpha, const void *x,
                                const void *beta, void *y, void *stream) {
  TRYS(check_handle(h));
  if (!alpha || !beta || (h->m > 0 && !y) || (h->n > 0 && !x)) return SMAT_ERR_INVALID_ARG;
  if ((int)v < 0 || (int)v >= SMAT_NUM_ALL_VARIANTS) return SMAT_ERR_INVALID_ARG;
  if (!variant_ready(h, v)) {
    TRYS(prepare_variant(h, v, (cudaStream_t)stream));
    if (!variant_ready(h, v)) return SMAT_ERR_UNSUPPORTED;
  }
  TRY(launch_spmv(h, v, alpha, x, beta, y, (cudaStream_t)stream));
  return SMAT_OK;
}

smat_status_t smat_spmv_host_async(smat_handle_t h, const void *alpha, const void *x_host, const void *beta,
                                   void *y_host, void *stream) {
  TRYS(check_handle(h));
  if (!alpha || !beta || (h->m > 0 && !y_host) || (h->n > 0 && !x_host)) return SMAT_ERR_INVALID_ARG;
  if (!variant_ready(h, h->variant)) return SMAT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ts = (size_t)tsize(h);
  if (!h->stage_x && h->n > 0) TRY(dev_alloc(&h->stage_x, (size_t)h->n * ts));
  if (!h->stage_y && h->m > 0) TRY(dev_alloc(&h->stage_y, (size_t)h->m * ts));
  const bool beta_zero = h->dtype == SMAT_F64 ? *(const double *)beta == 0.0 : *(const float *)beta == 0.0f;
  if (h->n > 0) TRY(cudaMemcpyAsync(h->stage_x, x_host, (size_t)h->n * ts, cudaMemcpyHostToDevice, s));
  if (!beta_zero && h->m > 0)
    TRY(cudaMemcpyAsync(h->stage_y, y_host, (size_t)h->m * ts, cudaMemcpyHostToDevice, s));
  TRY(launch_spmv(h, h->variant, alpha, h->stage_x, beta, h->stage_y, s));
  if (h->m > 0) TRY(cudaMemcpyAsync(y_host, h->stage_y, (size_t)h->m * ts, cudaMemcpyDeviceToHost, s));
  return SMAT_OK;
}

smat_status_t smat_spmv_host(smat_handle_t h, const void *alpha, const void *x_host, const void *beta,
                             void *y_host, void *stream) {
  TRYS(check_handle(h));
  if (!alpha || !beta || (h->m > 0 && !y_host) || (h->n > 0 && !x_host)) return SMAT_ERR_INVALID_ARG;
  if (!variant_ready(h, h->variant)) return SMAT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ts = (size_t)tsize(h);
  if (!h->stage_x && h->n > 0) TRY(dev_alloc(&h->stage_x, (size_t)h->n * ts));
  if (!h->stage_y && h->m > 0) TRY(dev_alloc(&h->stage_y, (size_t)h->m * ts));
  const bool beta_zero = h->dtype == SMAT_F64 ? *(const double *)beta == 0.0 : *(const float *)beta == 0.0f;
  if (h->n > 0) TRY(cudaMemcpyAsync(h->stage_x, x_host, (size_t)h->n * ts, cudaMemcpyHostToDevice, s));
  if (!beta_zero && h->m > 0)
    TRY(cudaMemcpyAsync(h->stage_y, y_host, (size_t)h->m * ts, cudaMemcpyHostToDevice, s));
  TRY(launch_spmv(h, h->variant, alpha, h->stage_x, beta, h->stage_y, s));
  if (h->m > 0) TRY(cudaMemcpyAsync(y_host, h->stage_y, (size_t)h->m * ts, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  return SMAT_OK;
}

// Host-buffer products in a pipeline: the handle keeps two staging sets and
// three streams of its own.  Call k uses set k % 2: its copy in waits only
// for the product of call k - 2 (which read that set's x), its product for
// its copy in and for the copy out of call k - 2 (which read that set's y),
// its copy out for its product; the caller's stream waits for the copy out.
// So consecutive calls overlap one call's transfers with another's product,
// and products of different handles overlap each other.
smat_status_t smat_spmv_host_pipelined(smat_handle_t h, const void *alpha, const void *x_host, const void *beta,
                                       void *y_host, void *stream) {
  TRYS(check_handle(h));
  if (!alpha || !beta || (h->m > 0 && !y_host) || (h->n > 0 && !x_host)) return SMAT_ERR_INVALID_ARG;
  if (!variant_ready(h, h->variant)) return SMAT_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return SMAT_ERR_UNSUPPORTED;  // its streams are not the caller's
  if (!h->pst[0]) {
    cudaStream_t st[3] = {};
    cudaEvent_t ev[6] = {};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&st[k], cudaStreamNonBlocking);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (cudaStream_t x : st) if (x) cudaStreamDestroy(x);
      for (cudaEvent_t x : ev) if (x) cudaEventDestroy(x);
      return st_of(e);
    }
    for (int k = 0; k < 3; ++k) h->pst[k] = st[k];
    for (int q = 0; q < 2; ++q) { h->pev_x[q] = ev[q]; h->pev_run[q] = ev[2 + q]; h->pev_out[q] = ev[4 + q]; }
  }
  const int q = (int)(h->pcalls & 1);
  const size_t ts = (size_t)tsize(h);
  if (!h->pstage_x[q] && h->n > 0) TRY(dev_alloc(&h->pstage_x[q], (size_t)h->n * ts));
  if (!h->pstage_y[q] && h->m > 0) TRY(dev_alloc(&h->pstage_y[q], (size_t)h->m * ts));
  const bool beta_zero = h->dtype == SMAT_F64 ? *(const double *)beta == 0.0 : *(const float *)beta == 0.0f;
  cudaStream_t in = h->pst[0], run = h->pst[1], out = h->pst[2];
  if (h->pused[q]) {
    TRY(cudaStreamWaitEvent(in, h->pev_run[q], 0));
    if (!beta_zero) TRY(cudaStreamWaitEvent(in, h->pev_out[q], 0));
  }
  if (h->n > 0) TRY(cudaMemcpyAsync(h->pstage_x[q], x_host, (size_t)h->n * ts, cudaMemcpyHostToDevice, in));
  if (!beta_zero && h->m > 0)
    TRY(cudaMemcpyAsync(h->pstage_y[q], y_host, (size_t)h->m * ts, cudaMemcpyHostToDevice, in));
  TRY(cudaEventRecord(h->pev_x[q], in));
  TRY(cudaStreamWaitEvent(run, h->pev_x[q], 0));
  if (h->pused[q]) TRY(cudaStreamWaitEvent(run, h->pev_out[q], 0));
  TRY(launch_spmv(h, h->variant, alpha, h->pstage_x[q], beta, h->pstage_y[q], run));
  TRY(cudaEventRecord(h->pev_run[q], run));
  TRY(cudaStreamWaitEvent(out, h->pev_run[q], 0));
  if (h->m > 0) TRY(cudaMemcpyAsync(y_host, h->pstage_y[q], (size_t)h->m * ts, cudaMemcpyDeviceToHost, out));
  TRY(cudaEventRecord(h->pev_out[q], out));
  TRY(cudaStreamWaitEvent(s, h->pev_out[q], 0));
  h->pused[q] = true;
  ++h->pcalls;
  return SMAT_OK;
}

smat_status_t smat_variant_bytes(smat_handle_t h, smat_variant_t v, double *bytes) {
  TRYS(check_handle(h));
  if (!bytes || (int)v < 0 || (int)v >= SMAT_NUM_ALL_VARIANTS) return SMAT_ERR_INVALID_ARG;
  if (!h->have_features) TRYS(compute_features(h, 0));
  if (v >= SMAT_V_HYB && v <= SMAT_V_SPLIT && !h->ext_known[v - SMAT_V_HYB]) return SMAT_ERR_UNSUPPORTED;
  *bytes = variant_bytes(h, (int)v);
  return SMAT_OK;
}

smat_status_t smat_spmv_launches(smat_handle_t h, smat_variant_t v, int32_t *launches) {
  TRYS(check_handle(h));
  if (!launches || (int)v < 0 || (int)v >= SMAT_NUM_ALL_VARIANTS) return SMAT_ERR_INVALID_ARG;
  *launches = variant_ready(h, v) ? spmv_launch_count(h, v) : 0;
  return SMAT_OK;
}

smat_status_t smat_get_features(smat_handle_t h, smat_features_t *out) {
  TRYS(check_handle(h));
  if (!out) return SMAT_ERR_INVALID_ARG;
  if (!h->have_features) TRYS(compute_features(h, 0));
  *out = h->f;
  return SMAT_OK;
}

smat_status_t smat_get_feature_vector(smat_handle_t h, float out[12]) {
  TRYS(check_handle(h));
  if (!out) return SMAT_ERR_INVALID_ARG;
  if (!h->have_features) TRYS(compute_features(h, 0));
  feature_vector(h->f, out);
  return SMAT_OK;
}

smat_status_t smat_get_plan(smat_handle_t h, int32_t *variant, double *tune_ms, float *confidence,
                            int32_t *trialled) {
  TRYS(check_handle(h));
  if (variant) *variant = h->variant;
  if (tune_ms) *tune_ms = h->tune_ms;
  if (confidence) *confidence = h->confidence;
  if (trialled) *trialled = h->trialled;
  return SMAT_OK;
}

smat_status_t smat_get_timings(smat_handle_t h, float ms[SMAT_NUM_ALL_VARIANTS]) {
  TRYS(check_handle(h));
  if (!ms) return SMAT_ERR_INVALID_ARG;
  for (int v = 0; v < SMAT_NUM_ALL_VARIANTS; ++v) ms[v] = h->timings[v];
  return SMAT_OK;
}

smat_status_t smat_convert(smat_handle_t h, smat_format_t fmt, void *stream) {
  TRYS(check_handle(h));
  if (fmt < SMAT_FMT_CSR || fmt > SMAT_FMT_SPLIT) return SMAT_ERR_INVALID_ARG;
  TRYS(build_format(h, fmt, (cudaStream_t)stream));
  TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return SMAT_OK;
}

smat_status_t smat_format_dims(smat_handle_t h, smat_format_t fmt, int64_t dims[2]) {
  TRYS(check_handle(h));
  if (!dims) return SMAT_ERR_INVALID_ARG;
  switch (fmt) {
    case SMAT_FMT_ELL: if (!h->ell_val) return SMAT_ERR_UNSUPPORTED; dims[0] = h->ell_K; dims[1] = h->P; break;
    case SMAT_FMT_DIA: if (!h->dia_val) return SMAT_ERR_UNSUPPORTED; dims[0] = h->dia_nd; dims[1] = h->P; break;
    case SMAT_FMT_COO: if (!h->coo_row && h->nnz > 0) return SMAT_ERR_UNSUPPORTED; dims[0] = h->nnz; dims[1] = 0; break;
    case SMAT_FMT_CSR: dims[0] = h->m; dims[1] = h->nnz; break;
    case SMAT_FMT_HYB: if (!h->hyb_built) return SMAT_ERR_UNSUPPORTED; dims[0] = h->hyb_K; dims[1] = h->hyb_ncoo; break;
    case SMAT_FMT_SELL: if (!h->sell_val) return SMAT_ERR_UNSUPPORTED; dims[0] = h->sell_ns; dims[1] = h->sell_slots; break;
    case SMAT_FMT_BCSR: if (!h->bcsr_val) return SMAT_ERR_UNSUPPORTED; dims[0] = h->bcsr_b; dims[1] = h->bcsr_nb; break;
    case SMAT_FMT_SPLIT: if (!h->split_built) return SMAT_ERR_UNSUPPORTED; dims[0] = h->split_nc; dims[1] = h->split_ns; break;
    default: return SMAT_ERR_INVALID_ARG;
  }
  return SMAT_OK;
}

smat_status_t smat_export_format(smat_handle_t h, smat_format_t fmt, int32_t *idx, void *val) {
  TRYS(check_handle(h));
  int64_t d[2];
  TRYS(smat_format_dims(h, fmt, d));
  switch (fmt) {
    case SMAT_FMT_ELL:
      if (!idx || !val) return SMAT_ERR_INVALID_ARG;
      TRY(cudaMemcpy(idx, h->ell_col, (size_t)(d[0] * d[1]) * 4, cudaMemcpyDefault));
      TRY(cudaMemcpy(val, h->ell_val, (size_t)(d[0] * d[1]) * h->esz, cudaMemcpyDefault));
      break;
    case SMAT_FMT_DIA:
      if (!idx || !val) return SMAT_ERR_INVALID_ARG;
      TRY(cudaMemcpy(idx, h->dia_off, (size_t)d[0] * 4, cudaMemcpyDefault));
      TRY(cudaMemcpy(val, h->dia_val, (size_t)(d[0] * d[1]) * h->esz, cudaMemcpyDefault));
      break;
    case SMAT_FMT_COO:
      if (!idx) return SMAT_ERR_INVALID_ARG;
      if (h->nnz > 0) TRY(cudaMemcpy(idx, h->coo_row, (size_t)h->nnz * 4, cudaMemcpyDefault));
      break;
    case SMAT_FMT_HYB: {
      if (!idx || !val) return SMAT_ERR_INVALID_ARG;
      const size_t ne = (size_t)(h->hyb_K * h->P), nc = (size_t)h->hyb_ncoo;
      if (ne) TRY(cudaMemcpy(idx, h->hyb_ecol, ne * 4, cudaMemcpyDefault));
      if (nc) TRY(cudaMemcpy(idx + ne, h->hyb_crow, nc * 4, cudaMemcpyDefault));
      if (nc) TRY(cudaMemcpy(idx + ne + nc, h->hyb_ccol, nc * 4, cudaMemcpyDefault));
      if (ne) TRY(cudaMemcpy(val, h->hyb_eval, ne * h->esz, cudaMemcpyDefault));
      if (nc) TRY(cudaMemcpy((char *)val + ne * h->esz, h->hyb_cval, nc * h->esz, cudaMemcpyDefault));
    } break;
    case SMAT_FMT_SELL: {
      if (!idx || !val) return SMAT_ERR_INVALID_ARG;
      const size_t ns = (size_t)h->sell_ns, sl = (size_t)h->sell_slots;
      if (ns) TRY(cudaMemcpy(idx, h->sell_perm, ns * 32 * 4, cudaMemcpyDefault));
      if (ns) TRY(cudaMemcpy(idx + ns * 32, h->sell_width, ns * 4, cudaMemcpyDefault));
      if (sl) TRY(cudaMemcpy(idx + ns * 33, h->sell_col, sl * 4, cudaMemcpyDefault));
      if (sl) TRY(cudaMemcpy(val, h->sell_val, sl * h->esz, cudaMemcpyDefault));
    } break;
    case SMAT_FMT_BCSR: {
      if (!idx || !val) return SMAT_ERR_INVALID_ARG;
      const size_t mb = (size_t)h->bcsr_mb, nb = (size_t)h->bcsr_nb, bb = (size_t)h->bcsr_b * h->bcsr_b;
      TRY(cudaMemcpy(idx, h->bcsr_rowptr, (mb + 1) * 4, cudaMemcpyDefault));
      if (nb) TRY(cudaMemcpy(idx + mb + 1, h->bcsr_col, nb * 4, cudaMemcpyDefault));
      if (nb) TRY(cudaMemcpy(val, h->bcsr_val, nb * bb * h->esz, cudaMemcpyDefault));
    } break;
    case SMAT_FMT_SPLIT: {
      if (!idx || (!val && h->split_ns > 0)) return SMAT_ERR_INVALID_ARG;
      const size_t nc = (size_t)h->split_nc, ns = (size_t)h->split_ns;
      if (nc) TRY(cudaMemcpy(idx, h->split_crow, nc * 4, cudaMemcpyDefault));
      if (nc) TRY(cudaMemcpy(idx + nc, h->split_cstart, nc * 4, cudaMemcpyDefault));
      if (nc) TRY(cudaMemcpy(idx + 2 * nc, h->split_cend, nc * 4, cudaMemcpyDefault));
      if (ns) TRY(cudaMemcpy(idx + 3 * nc, h->split_srow, ns * 4, cudaMemcpyDefault));
      if (ns) TRY(cudaMemcpy(idx + 3 * nc + ns, h->split_scol, ns * 4, cudaMemcpyDefault));
      if (ns) TRY(cudaMemcpy(val, h->split_sval, ns * h->esz, cudaMemcpyDefault));
    } break;
    default:
      return SMAT_ERR_INVALID_ARG;
  }
  return SMAT_OK;
}

smat_status_t smat_set_model(const float *params, const float *mean, const float *stdv) {
  std::lock_guard<std::mutex> lk(model_mu());
  Model &M = model();
  if (!params) {
    M.loaded = false;
    return SMAT_OK;
  }
  if (!mean || !stdv) return SMAT_ERR_INVALID_ARG;
  std::memcpy(M.params, params, sizeof(M.params));
  std::memcpy(M.mean, mean, sizeof(M.mean));
  std::memcpy(M.stdv, stdv, sizeof(M.stdv));
  M.loaded = true;
  return SMAT_OK;
}

smat_status_t smat_load_model(const char *path) {
  if (!path || !*path) path = std::getenv("SMAT_MODEL_PATH");  // NULL: the file SMAT_MODEL_PATH names
  if (!path || !*path) return SMAT_ERR_INVALID_ARG;
  FILE *fp = std::fopen(path, "rb");
  if (!fp) return SMAT_ERR_MODEL;
  char magic[8];
  int32_t ver = 0;
  std::vector<float> buf(12 + 12 + SMAT_MLP_PARAMS);
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "SMATMLP1", 8) == 0 &&
            std::fread(&ver, 4, 1, fp) == 1 && ver == 1 &&
            std::fread(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
  std::fclose(fp);
  if (!ok) return SMAT_ERR_MODEL;
  for (float v : buf)
    if (!std::isfinite(v)) return SMAT_ERR_MODEL;
  return smat_set_model(buf.data() + 24, buf.data(), buf.data() + 12);
}

}  // extern "C"
