// Device-side building blocks of the SpMV kernels, shared by the single-
// matrix kernels (spmv.cu) and the batched persistent kernel (batch.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace smat {
namespace {

// Programmatic dependent launch.  The product kernels are launched so that
// the GPU may begin scheduling one while the previous kernel of the stream
// drains (on GB300 this removed about 2 us of idle time per launch in a
// sequence of streaming kernels).  The first thing each such kernel does is
// griddep_wait(): it returns once the previous kernel has completed and its
// writes are visible, so stream order holds exactly as for a plain launch
// (and it is a no-op when the kernel was launched the plain way).
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename V> struct Compute { typedef float T; };
template <> struct Compute<double> { typedef double T; };

// Matrix arrays are read once per product: load them with the streaming
// (evict-first) policy so that x, which every product gathers from, stays in L2.
__device__ __forceinline__ double ld_val(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const float *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_val(const __nv_bfloat16 *p) {
  return __uint_as_float((unsigned)__ldcs(reinterpret_cast<const unsigned short *>(p)) << 16);
}
__device__ __forceinline__ int ld_idx(const int32_t *p) { return __ldcs(p); }

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// acc + v*x.  GB300 executes FP64 arithmetic at about 2 operations per clock
// per SM, so FP64 SpMV is bound by the FP64 pipe about as much as by HBM:
// every kernel spends exactly one fused multiply-add per stored product.
// The EXACT flavour (CSR-scalar only) instead rounds the product and the sum
// separately, in ascending column order -- the CSR definition operation for
// operation -- at twice the FP64 cost.
__device__ __forceinline__ double fused(double acc, double v, double x) { return fma(v, x, acc); }
__device__ __forceinline__ float fused(float acc, float v, float x) { return fmaf(v, x, acc); }
template <bool EXACT>
__device__ __forceinline__ double madd(double acc, double v, double x) {
  return EXACT ? __dadd_rn(acc, __dmul_rn(v, x)) : fma(v, x, acc);
}
template <bool EXACT>
__device__ __forceinline__ float madd(float acc, float v, float x) { return fmaf(v, x, acc); }

// The epilogue y_i = alpha*acc (+ beta*y_i) in one of three forms chosen on
// the host, so no kernel compares alpha or beta (FP64 compares occupy the
// same scarce FP64 pipe as the products):
//   EPI_COPY   beta == 0, alpha == 1:  y_i = acc
//   EPI_SCALE  beta == 0:              y_i = alpha*acc        (y not read)
//   EPI_AXPBY  otherwise:              y_i = alpha*acc + beta*y_i
// EXACT rounds beta*y_i and the sum separately; otherwise they are fused.
enum : int { EPI_COPY = 0, EPI_SCALE = 1, EPI_AXPBY = 2 };

// Batch width for `count` slots (ELL) or diagonals (DIA) with at most umax per
// batch: all of them when they fit, else the width in [umax/2, umax] that
// leaves the fewest unused slots in the last batch (the wider on ties).
inline int batch_width(long long count, int umax) {
  if (count <= umax) return count < 1 ? 1 : (int)count;
  int best = umax;
  long long waste = (count + umax - 1) / umax * umax - count;
  for (int u = umax - 1; u >= umax / 2 && u >= 1; --u) {
    const long long w = (count + u - 1) / u * u - count;
    if (w < waste) { waste = w; best = u; }
  }
  return best;
}

inline int epi_mode(double alpha, double beta) {
  return beta != 0.0 ? EPI_AXPBY : (alpha != 1.0 ? EPI_SCALE : EPI_COPY);
}

template <typename T, int MODE, bool EXACT = false>
struct Epi {
  T alpha, beta;
  __device__ __forceinline__ T operator()(T acc, const T *y, long long i) const {
    if (MODE == EPI_COPY) return acc;
    const T ax = mul_rn(alpha, acc);
    if (MODE == EPI_SCALE) return ax;
    return EXACT ? add_rn(ax, mul_rn(beta, y[i])) : fused(ax, beta, y[i]);
  }
};

// 16-byte vector loads of R consecutive values (R * sizeof(V) == 16) and of
// R consecutive column indices.
template <typename V, int R> struct VecOf;
template <> struct VecOf<double, 2> { typedef double2 T; };
template <> struct VecOf<float, 4> { typedef float4 T; };
template <> struct VecOf<__nv_bfloat16, 8> { typedef uint4 T; };

template <typename V, int R>
__device__ __forceinline__ void load_vals(const V *p, typename Compute<V>::T (&out)[R]);
template <>
__device__ __forceinline__ void load_vals<double, 2>(const double *p, double (&out)[2]) {
  double2 v = __ldcs(reinterpret_cast<const double2 *>(p));
  out[0] = v.x; out[1] = v.y;
}
template <>
__device__ __forceinline__ void load_vals<float, 4>(const float *p, float (&out)[4]) {
  float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void load_vals<__nv_bfloat16, 8>(const __nv_bfloat16 *p, float (&out)[8]) {
  uint4 v = __ldcs(reinterpret_cast<const uint4 *>(p));
  unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    out[2 * q] = __uint_as_float(w[q] << 16);
    out[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
  }
}

template <int R>
__device__ __forceinline__ void load_cols(const int32_t *p, int (&c)[R]) {
  if constexpr (R == 2) {
    int2 v = __ldcs(reinterpret_cast<const int2 *>(p));
    c[0] = v.x; c[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      int4 v = __ldcs(reinterpret_cast<const int4 *>(p) + q);
      c[4 * q] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
    }
  }
}

// y[i0 .. i0+R) from R accumulators: one vector store (and load when beta != 0)
// for full groups, scalar at the tail.
template <typename T, int R> struct YVec;
template <> struct YVec<double, 2> {
  static __device__ __forceinline__ void ld(const double *p, double (&o)[2]) { double2 v = *reinterpret_cast<const double2 *>(p); o[0] = v.x; o[1] = v.y; }
  static __device__ __forceinline__ void st(double *p, const double (&o)[2]) { *reinterpret_cast<double2 *>(p) = make_double2(o[0], o[1]); }
};
template <> struct YVec<float, 4> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[4]) { float4 v = *reinterpret_cast<const float4 *>(p); o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
  static __device__ __forceinline__ void st(float *p, const float (&o)[4]) { *reinterpret_cast<float4 *>(p) = make_float4(o[0], o[1], o[2], o[3]); }
};
template <> struct YVec<float, 8> {
  static __device__ __forceinline__ void ld(const float *p, float (&o)[8]) {
    float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
  static __device__ __forceinline__ void st(float *p, const float (&o)[8]) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(o[0], o[1], o[2], o[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(o[4], o[5], o[6], o[7]);
  }
};

template <typename T, int R, int MODE>
__device__ __forceinline__ void write_rows(T *__restrict__ y, long long i0, long long m, const T (&acc)[R],
                                           const Epi<T, MODE> &ep) {
  if (i0 + R <= m) {
    T out[R];
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = MODE == EPI_COPY ? acc[r] : mul_rn(ep.alpha, acc[r]);
    if (MODE == EPI_AXPBY) {
      T yo[R];
      YVec<T, R>::ld(y + i0, yo);
#pragma unroll
      for (int r = 0; r < R; ++r) out[r] = fused(out[r], ep.beta, yo[r]);
    }
    YVec<T, R>::st(y + i0, out);
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (i0 + r < m) y[i0 + r] = ep(acc[r], y, i0 + r);
  }
}

// One thread's R consecutive rows [i0, i0 + R) of an ELL product
// (column-major, pitch P, K slots).  U slots are loaded before their gathers
// are issued (U <= 16/R; the host picks U so that few batch slots go unused,
// since an unused slot still issues its multiply-adds); padding (column -1)
// is dropped.
template <typename V, int R, int MODE, int U = 16 / R>
__device__ __forceinline__ void ell_group(const int32_t *__restrict__ ecol, const V *__restrict__ eval, long long P,
                                          long long K, const typename Compute<V>::T *__restrict__ x,
                                          const Epi<typename Compute<V>::T, MODE> &ep,
                                          typename Compute<V>::T *__restrict__ y, long long m, long long i0) {
  typedef typename Compute<V>::T T;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0;
  for (long long q = 0; q < K; q += U) {
    T v[U][R], xv[U][R];
    int c[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (q + u < K) {
        load_vals<V, R>(eval + (q + u) * P + i0, v[u]);
        load_cols<R>(ecol + (q + u) * P + i0, c[u]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) { v[u][r] = 0; c[u][r] = -1; }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) xv[u][r] = c[u][r] >= 0 ? __ldg(x + c[u][r]) : (T)0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q + u < K) {  // uniform across the warp: dead slots issue no FP work
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (c[u][r] >= 0) acc[r] = fused(acc[r], v[u][r], xv[u][r]);
      }
  }
  write_rows<T, R, MODE>(y, i0, m, acc, ep);
}

// ELL with lane-striped rows: lane l of a warp takes rows base + l + 32 r
// (r < R), so each slot's column and value loads are contiguous 32-element
// warp accesses.
template <typename V, int R, int MODE, int U>
__device__ __forceinline__ void ell_lane_group(const int32_t *__restrict__ ecol, const V *__restrict__ eval,
                                               long long P, long long K, const typename Compute<V>::T *__restrict__ x,
                                               const Epi<typename Compute<V>::T, MODE> &ep,
                                               typename Compute<V>::T *__restrict__ y, long long m, long long base,
                                               int lane) {
  typedef typename Compute<V>::T T;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0;
  for (long long q = 0; q < K; q += U) {
    T v[U][R], xv[U][R];
    int c[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long i = base + lane + 32 * r;
        const bool on = q + u < K && i < P;
        c[u][r] = on ? ld_idx(ecol + (q + u) * P + i) : -1;
        v[u][r] = on ? (T)ld_val(eval + (q + u) * P + i) : (T)0;
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int r = 0; r < R; ++r) xv[u][r] = c[u][r] >= 0 ? __ldg(x + c[u][r]) : (T)0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (q + u < K) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (c[u][r] >= 0) acc[r] = fused(acc[r], v[u][r], xv[u][r]);
      }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = base + lane + 32 * r;
    if (i < m) y[i] = ep(acc[r], y, i);
  }
}

// One thread's R consecutive rows of a DIA product; `off` holds the nd
// ascending diagonal offsets (shared or global memory), U diagonals per batch
// (chosen on the host as for ELL).  Fill zeros are
// multiplied like stored values; positions whose column falls outside the
// matrix are dropped.
template <typename V, int R, int MODE, int U = 16 / R, bool FAST = true>
__device__ __forceinline__ void dia_group(const int32_t *off, int nd, const V *__restrict__ dval, long long P,
                                          const typename Compute<V>::T *__restrict__ x,
                                          const Epi<typename Compute<V>::T, MODE> &ep,
                                          typename Compute<V>::T *__restrict__ y, long long m, long long n,
                                          long long i0) {
  typedef typename Compute<V>::T T;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0;
  for (int t = 0; t < nd; t += U) {
    T v[U][R], xv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool live = t + u < nd;
      const long long j0 = i0 + (live ? off[t + u] : 0);
      if (live) {
        load_vals<V, R>(dval + (long long)(t + u) * P + i0, v[u]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) v[u][r] = 0;
      }
      if (FAST && live && j0 >= 0 && j0 + R <= n) {  // the whole window inside x: no per-row checks
        const T *xp = x + j0;
        if constexpr (sizeof(T) == 4 && R % 4 == 0) {
          // i0 is a multiple of R, so the window is 16-byte aligned exactly when
          // the diagonal's offset is a multiple of 4 (uniform over the warp)
          if ((j0 & 3) == 0) {
#pragma unroll
            for (int q = 0; q < R / 4; ++q) {
              const float4 f = __ldg(reinterpret_cast<const float4 *>(xp) + q);
              xv[u][4 * q] = f.x; xv[u][4 * q + 1] = f.y; xv[u][4 * q + 2] = f.z; xv[u][4 * q + 3] = f.w;
            }
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) xv[u][r] = __ldg(xp + r);
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) xv[u][r] = __ldg(xp + r);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) xv[u][r] = (live && j0 + r >= 0 && j0 + r < n) ? __ldg(x + j0 + r) : (T)0;
      }
    }
    // out-of-range positions hold a stored +0 and read x as 0: no predicate
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (t + u < nd) {  // uniform across the warp: dead slots issue no FP work
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fused(acc[r], v[u][r], xv[u][r]);
      }
  }
  write_rows<T, R, MODE>(y, i0, m, acc, ep);
}

// DIA with lane-striped rows: lane l of a warp takes rows base + l + 32 r
// (r < R), so every value load and every x load of a diagonal is one
// contiguous 32-element warp access.
template <typename V, int R, int MODE, int U>
__device__ __forceinline__ void dia_lane_group(const int32_t *off, int nd, const V *__restrict__ dval, long long P,
                                               const typename Compute<V>::T *__restrict__ x,
                                               const Epi<typename Compute<V>::T, MODE> &ep,
                                               typename Compute<V>::T *__restrict__ y, long long m, long long n,
                                               long long base, int lane) {
  typedef typename Compute<V>::T T;
  T acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0;
  for (int t = 0; t < nd; t += U) {
    T v[U][R], xv[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool live = t + u < nd;
      const long long o = live ? off[t + u] : 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const long long i = base + lane + 32 * r;
        const long long j = i + o;
        const bool in = live && i < m && j >= 0 && j < n;
        v[u][r] = (live && i < P) ? (T)ld_val(dval + (long long)(t + u) * P + i) : (T)0;
        xv[u][r] = in ? __ldg(x + j) : (T)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (t + u < nd) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fused(acc[r], v[u][r], xv[u][r]);
      }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long i = base + lane + 32 * r;
    if (i < m) y[i] = ep(acc[r], y, i);
  }
}

// One SELL-32 slice: lane l computes the row at sorted position 32*sl + l over
// the slice's `w` slots, U slots loaded before their gathers.  w is uniform
// over the warp, so no lane diverges; padding (column -1) gathers x[0] and is
// dropped by a select.
template <typename V, int MODE, int U>
__device__ __forceinline__ void sell_slice(const long long *__restrict__ sptr, const int32_t *__restrict__ width,
                                           const int32_t *__restrict__ perm, const int32_t *__restrict__ scol,
                                           const V *__restrict__ sval, const typename Compute<V>::T *__restrict__ x,
                                           const Epi<typename Compute<V>::T, MODE> &ep,
                                           typename Compute<V>::T *__restrict__ y, long long sl, int lane) {
  typedef typename Compute<V>::T T;
  const long long base = __ldg(sptr + sl) + lane;
  const int w = __ldg(width + sl);
  T acc = 0;
  for (int j = 0; j < w; j += U) {
    int c[U];
    T v[U], xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool on = j + u < w;
      c[u] = on ? ld_idx(scol + base + (long long)(j + u) * 32) : -1;
      v[u] = on ? (T)ld_val(sval + base + (long long)(j + u) * 32) : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = __ldg(x + (c[u] > 0 ? c[u] : 0));
#pragma unroll
    for (int u = 0; u < U; ++u) acc = fused(acc, v[u], c[u] >= 0 ? xv[u] : (T)0);
  }
  const int r = __ldg(perm + sl * 32 + lane);
  if (r >= 0) y[r] = ep(acc, y, (long long)r);
}

}  // namespace
}  // namespace smat
