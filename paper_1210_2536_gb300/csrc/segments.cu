// Per-segment plans: the matrix's rows are split into segments holding about
// equal numbers of stored entries, and every segment gets its own format
// (arXiv 1210.2536, Sec. 6: the multi-threaded SMAT divides the nonzeros
// evenly over threads, rounds to whole rows, and may choose a different
// format per thread's segment, which pays for matrices whose structure
// changes from one part to another).
//
// Each segment becomes a handle of its own (a copy of its rows, row pointers
// rebased to 0, all N columns), tuned by its own features.  When every
// segment's plan is a kind the batched kernel runs natively (CSR with 1/4/8/32
// lanes, ELL, DIA, SELL) the segments run together as one batched launch
// (batch.cu); otherwise (COO, merge-path, HYB, BCSR) each segment runs its own
// plan on a stream of its own, forked from and joined back to the caller's
// stream, so the segments' kernels overlap.  Both read the shared x and write
// each segment's slice of y.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "smat_internal.h"

struct smat_segments_s {
  smat_handle_t parent = nullptr;
  std::vector<smat_handle_t> subs;
  std::vector<int64_t> starts;  // row starts, size nseg + 1
  smat_batch_t batch = nullptr;  // when every plan is batch-native
  std::vector<cudaStream_t> streams;  // otherwise: a stream per segment
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
};

namespace {

bool batch_native(int v) {
  return v == SMAT_V_CSR_SCALAR || v == SMAT_V_CSR_VEC4 || v == SMAT_V_CSR_VEC8 || v == SMAT_V_CSR_VEC32 ||
         v == SMAT_V_ELL || v == SMAT_V_DIA || v == SMAT_V_SELL;
}

}  // namespace

extern "C" {

smat_status_t smat_segments_destroy(smat_segments_t s) {
  if (!s) return SMAT_OK;
  smat_batch_destroy(s->batch);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t e : s->joins) cudaEventDestroy(e);
  if (s->fork) cudaEventDestroy(s->fork);
  for (smat_handle_t h : s->subs) smat_destroy(h);
  delete s;
  return SMAT_OK;
}

smat_status_t smat_segments_create(smat_segments_t *out, smat_handle_t h, int32_t nseg, const smat_tune_opts_t *opts,
                                   void *stream) {
  if (!out || !h || nseg < 1) return SMAT_ERR_INVALID_ARG;
  *out = nullptr;
  if (h->m == 0) return SMAT_ERR_UNSUPPORTED;
  std::vector<int32_t> rp((size_t)h->m + 1);
  if (cudaMemcpy(rp.data(), h->rowptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SMAT_ERR_CUDA;
  // nonzero-balanced split at whole rows, boundaries rounded to 8 rows so that
  // every segment's slice of y starts 16-byte aligned
  std::vector<int64_t> starts{0};
  for (int t = 1; t < nseg; ++t) {
    const int64_t target = (int64_t)h->nnz * t / nseg;
    int64_t r = std::lower_bound(rp.begin(), rp.end(), (int32_t)target) - rp.begin();
    r = r / 8 * 8;
    if (r > starts.back() && r < h->m) starts.push_back(r);
  }
  starts.push_back(h->m);
  smat_segments_s *s = new (std::nothrow) smat_segments_s();
  if (!s) return SMAT_ERR_ALLOC;
  s->parent = h;
  s->starts = starts;
  auto fail = [&](smat_status_t st) {
    smat_segments_destroy(s);
    return st;
  };
  for (size_t k = 0; k + 1 < starts.size(); ++k) {
    const int64_t r0 = starts[k], r1 = starts[k + 1];
    const int64_t base = rp[(size_t)r0], nnz = (int64_t)rp[(size_t)r1] - base;
    std::vector<int32_t> sub_rp((size_t)(r1 - r0 + 1));
    for (int64_t i = r0; i <= r1; ++i) sub_rp[(size_t)(i - r0)] = rp[(size_t)i] - (int32_t)base;
    smat_handle_t sub = nullptr;
    smat_status_t st = smat_create(&sub, r1 - r0, h->n, nnz, sub_rp.data(), nnz ? h->colidx + base : nullptr,
                                   nnz ? (const char *)h->val + base * h->esz : nullptr, h->dtype);
    if (st != SMAT_OK) return fail(st);
    s->subs.push_back(sub);
    if ((st = smat_tune(sub, opts, stream)) != SMAT_OK) return fail(st);
  }
  bool native = true;
  for (smat_handle_t sub : s->subs) native = native && batch_native(sub->variant);
  if (native) {
    smat_status_t st = smat_batch_create(&s->batch, s->subs.data(), (int32_t)s->subs.size());
    if (st == SMAT_OK) st = smat_batch_tune(s->batch, nullptr, stream);
    if (st != SMAT_OK) return fail(st);
  } else {
    s->streams.assign(s->subs.size(), nullptr);
    s->joins.assign(s->subs.size(), nullptr);
    if (cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming) != cudaSuccess) return fail(SMAT_ERR_CUDA);
    for (size_t k = 0; k < s->subs.size(); ++k)
      if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s->joins[k], cudaEventDisableTiming) != cudaSuccess)
        return fail(SMAT_ERR_CUDA);
  }
  *out = s;
  return SMAT_OK;
}

smat_status_t smat_segments_spmv(smat_segments_t s, const void *alpha, const void *x, const void *beta, void *y,
                                 void *stream) {
  if (!s || !alpha || !beta || !x || !y) return SMAT_ERR_INVALID_ARG;
  const size_t n = s->subs.size();
  const int tsz = s->parent->dtype == SMAT_F64 ? 8 : 4;
  if ((((uintptr_t)x | (uintptr_t)y) & 15u) != 0)  // segments with vector accesses need aligned vectors
    return smat_spmv(s->parent, alpha, x, beta, y, stream);
  if (!s->batch) {  // each segment through its own plan, on its own stream
    cudaStream_t cs = (cudaStream_t)stream;
    if (cudaEventRecord(s->fork, cs) != cudaSuccess) return SMAT_ERR_CUDA;
    for (size_t k = 0; k < n; ++k) {
      if (cudaStreamWaitEvent(s->streams[k], s->fork, 0) != cudaSuccess) return SMAT_ERR_CUDA;
      smat_status_t st = smat_spmv(s->subs[k], alpha, x, beta, (char *)y + s->starts[k] * tsz, s->streams[k]);
      if (st != SMAT_OK) return st;
      if (cudaEventRecord(s->joins[k], s->streams[k]) != cudaSuccess ||
          cudaStreamWaitEvent(cs, s->joins[k], 0) != cudaSuccess)
        return SMAT_ERR_CUDA;
    }
    return SMAT_OK;
  }
  std::vector<const void *> xs(n, x);
  std::vector<void *> ys(n);
  std::vector<unsigned char> al(n * (size_t)tsz), be(n * (size_t)tsz);
  for (size_t k = 0; k < n; ++k) {
    ys[k] = (char *)y + s->starts[k] * tsz;
    std::memcpy(&al[k * (size_t)tsz], alpha, (size_t)tsz);
    std::memcpy(&be[k * (size_t)tsz], beta, (size_t)tsz);
  }
  return smat_batch_spmv(s->batch, al.data(), xs.data(), be.data(), ys.data(), stream);
}

smat_status_t smat_segments_info(smat_segments_t s, int32_t *nseg, int32_t *variants, int64_t *row_starts) {
  if (!s || !nseg) return SMAT_ERR_INVALID_ARG;
  *nseg = (int32_t)s->subs.size();
  for (size_t k = 0; k < s->subs.size(); ++k) {
    if (variants) variants[k] = s->subs[k]->variant;
    if (row_starts) row_starts[k] = s->starts[k];
  }
  if (row_starts) row_starts[s->subs.size()] = s->starts.back();
  return SMAT_OK;
}

}  // extern "C"
