// Learned format selector: a 12 -> 64 -> 64 -> 8 MLP over the feature
// parameters.  It takes the place of the paper's C5.0 ruleset classifier
// f(x, TH) -> {DIA, ELL, CSR, COO} (arXiv 1210.2536, Sec. 5, Eq. "mapping"),
// predicting one of the eight GPU kernel variants, and its softmax maximum
// plays the role of the rule confidence checked against a threshold (Sec. 6).
//
// Inference and training run in these kernels: a CTA holds the whole network
// (5512 FP32 parameters) in shared memory and processes 32 samples.
// Gradients are reduced per CTA and then across CTAs in a fixed order, so a
// training step is deterministic.
#include <cmath>

#include "smat_internal.h"

namespace smat {
namespace {

constexpr int IN = 12, H = 64, OUT = 8, S = 32, NT = 256;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + OUT * H, NP = OB3 + OUT;
static_assert(NP == SMAT_MLP_PARAMS, "parameter layout");

// shared layout (floats)
constexpr int SW = 0, SX = SW + NP, SH1 = SX + S * IN, SH2 = SH1 + S * H, SZ = SH2 + S * H, SDZ = SZ + S * OUT,
              SDH2 = SDZ + S * OUT, SDH1 = SDH2 + S * H, SFWD = SDZ, STOT = SDH1 + S * H;

__device__ void block_forward(float *sm, const float *__restrict__ params, const float *__restrict__ X, int s0,
                              int ns) {
  for (int p = threadIdx.x; p < NP; p += NT) sm[SW + p] = params[p];
  for (int q = threadIdx.x; q < S * IN; q += NT) {
    int s = q / IN;
    sm[SX + q] = s < ns ? X[(long long)(s0 + s) * IN + q % IN] : 0.0f;
  }
  __syncthreads();
  const float *W1 = sm + SW + OW1, *b1 = sm + SW + OB1, *W2 = sm + SW + OW2, *b2 = sm + SW + OB2,
              *W3 = sm + SW + OW3, *b3 = sm + SW + OB3;
  for (int q = threadIdx.x; q < S * H; q += NT) {
    int s = q / H, j = q % H;
    float a = b1[j];
#pragma unroll
    for (int i = 0; i < IN; ++i) a = fmaf(W1[j * IN + i], sm[SX + s * IN + i], a);
    sm[SH1 + q] = a > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < S * H; q += NT) {
    int s = q / H, j = q % H;
    float a = b2[j];
#pragma unroll 8
    for (int i = 0; i < H; ++i) a = fmaf(W2[j * H + i], sm[SH1 + s * H + i], a);
    sm[SH2 + q] = a > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < S * OUT; q += NT) {
    int s = q / OUT, c = q % OUT;
    float a = b3[c];
#pragma unroll 8
    for (int i = 0; i < H; ++i) a = fmaf(W3[c * H + i], sm[SH2 + s * H + i], a);
    sm[SZ + q] = a;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) mlp_forward_kernel(const float *__restrict__ params,
                                                         const float *__restrict__ X, int B,
                                                         float *__restrict__ logits) {
  extern __shared__ float sm[];
  const int s0 = blockIdx.x * S, ns = min(S, B - s0);
  block_forward(sm, params, X, s0, ns);
  for (int q = threadIdx.x; q < ns * OUT; q += NT) logits[(long long)s0 * OUT + q] = sm[SZ + q];
}

// Soft-target cross-entropy and backpropagation for one CTA's samples; the
// CTA's gradient sums go to work[blockIdx.x][0..NP) and its loss sum to
// work[blockIdx.x][NP].
__global__ void __launch_bounds__(NT) mlp_loss_grad_kernel(const float *__restrict__ params,
                                                           const float *__restrict__ X,
                                                           const float *__restrict__ T, int B,
                                                           float *__restrict__ work) {
  extern __shared__ float sm[];
  const int s0 = blockIdx.x * S, ns = min(S, B - s0);
  block_forward(sm, params, X, s0, ns);
  __shared__ float s_loss[S];
  const float invB = 1.0f / (float)B;
  if (threadIdx.x < S) {
    int s = threadIdx.x;
    float lossv = 0.0f;
    if (s < ns) {
      const float *z = sm + SZ + s * OUT;
      const float *t = T + (long long)(s0 + s) * OUT;
      float zmax = z[0];
      for (int c = 1; c < OUT; ++c) zmax = fmaxf(zmax, z[c]);
      float se = 0.0f;
      for (int c = 0; c < OUT; ++c) se += expf(z[c] - zmax);
      float lse = zmax + logf(se), tsum = 0.0f;
      for (int c = 0; c < OUT; ++c) {
        lossv -= t[c] * (z[c] - lse);
        tsum += t[c];
      }
      for (int c = 0; c < OUT; ++c) sm[SDZ + s * OUT + c] = (tsum * expf(z[c] - lse) - t[c]) * invB;
    } else {
      for (int c = 0; c < OUT; ++c) sm[SDZ + s * OUT + c] = 0.0f;
    }
    s_loss[s] = lossv;
  }
  __syncthreads();
  const float *W2 = sm + SW + OW2, *W3 = sm + SW + OW3;
  float *out = work + (long long)blockIdx.x * (NP + 1);
  // layer 3
  for (int q = threadIdx.x; q < OUT * H; q += NT) {
    int c = q / H, i = q % H;
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g = fmaf(sm[SDZ + s * OUT + c], sm[SH2 + s * H + i], g);
    out[OW3 + q] = g;
  }
  if (threadIdx.x < OUT) {
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g += sm[SDZ + s * OUT + threadIdx.x];
    out[OB3 + threadIdx.x] = g;
  }
  for (int q = threadIdx.x; q < S * H; q += NT) {
    int s = q / H, i = q % H;
    float a = 0.0f;
#pragma unroll
    for (int c = 0; c < OUT; ++c) a = fmaf(W3[c * H + i], sm[SDZ + s * OUT + c], a);
    sm[SDH2 + q] = sm[SH2 + q] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // layer 2
  for (int q = threadIdx.x; q < H * H; q += NT) {
    int j = q / H, i = q % H;
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g = fmaf(sm[SDH2 + s * H + j], sm[SH1 + s * H + i], g);
    out[OW2 + q] = g;
  }
  if (threadIdx.x < H) {
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g += sm[SDH2 + s * H + threadIdx.x];
    out[OB2 + threadIdx.x] = g;
  }
  for (int q = threadIdx.x; q < S * H; q += NT) {
    int s = q / H, i = q % H;
    float a = 0.0f;
#pragma unroll 8
    for (int j = 0; j < H; ++j) a = fmaf(W2[j * H + i], sm[SDH2 + s * H + j], a);
    sm[SDH1 + q] = sm[SH1 + q] > 0.0f ? a : 0.0f;
  }
  __syncthreads();
  // layer 1
  for (int q = threadIdx.x; q < H * IN; q += NT) {
    int j = q / IN, i = q % IN;
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g = fmaf(sm[SDH1 + s * H + j], sm[SX + s * IN + i], g);
    out[OW1 + q] = g;
  }
  if (threadIdx.x < H) {
    float g = 0.0f;
    for (int s = 0; s < ns; ++s) g += sm[SDH1 + s * H + threadIdx.x];
    out[OB1 + threadIdx.x] = g;
  }
  if (threadIdx.x == 0) {
    float l = 0.0f;
    for (int s = 0; s < ns; ++s) l += s_loss[s];
    out[NP] = l;
  }
}

// grad[p] = sum over CTAs in index order; loss = (sum of CTA losses) / B.
__global__ void mlp_reduce_kernel(const float *__restrict__ work, int nblk, int B, float *__restrict__ grad,
                                  float *__restrict__ loss) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= NP; p += gridDim.x * blockDim.x) {
    float a = 0.0f;
    for (int c = 0; c < nblk; ++c) a += work[(long long)c * (NP + 1) + p];
    if (p < NP) grad[p] = a;
    else *loss = a / (float)B;
  }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

cudaError_t set_smem(const void *fn) {
  static bool done[2] = {false, false};
  int k = fn == (const void *)mlp_forward_kernel ? 0 : 1;
  if (done[k]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(STOT * sizeof(float)));
  if (e == cudaSuccess) done[k] = true;
  return e;
}

}  // namespace

cudaError_t launch_mlp_forward(const float *params, const float *X, int B, float *logits, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  cudaError_t e = set_smem((const void *)mlp_forward_kernel);
  if (e != cudaSuccess) return e;
  mlp_forward_kernel<<<(B + S - 1) / S, NT, SFWD * sizeof(float) + 0, s>>>(params, X, B, logits);
  return cudaGetLastError();
}

}  // namespace smat

using namespace smat;

extern "C" {

smat_status_t smat_mlp_forward(const float *params, const float *X, int32_t B, float *logits, void *stream) {
  if (B < 0 || (B > 0 && (!params || !X || !logits))) return SMAT_ERR_INVALID_ARG;
  return launch_mlp_forward(params, X, B, logits, (cudaStream_t)stream) == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}

int64_t smat_mlp_work_floats(int32_t B) { return (int64_t)((B + S - 1) / S) * (NP + 1); }

smat_status_t smat_mlp_loss_grad(const float *params, const float *X, const float *T, int32_t B, float *grad,
                                 float *loss, float *work, void *stream) {
  if (B <= 0 || !params || !X || !T || !grad || !loss || !work) return SMAT_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (set_smem((const void *)mlp_loss_grad_kernel) != cudaSuccess) return SMAT_ERR_CUDA;
  int nblk = (B + S - 1) / S;
  mlp_loss_grad_kernel<<<nblk, NT, STOT * sizeof(float), s>>>(params, X, T, B, work);
  if (cudaGetLastError() != cudaSuccess) return SMAT_ERR_CUDA;
  mlp_reduce_kernel<<<(NP + 1 + 255) / 256, 256, 0, s>>>(work, nblk, B, grad, loss);
  return cudaGetLastError() == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}

smat_status_t smat_mlp_adam(float *p, const float *g, float *m, float *v, int64_t n, int32_t t, float lr,
                            float beta1, float beta2, float eps, void *stream) {
  if (n < 0 || t < 1 || (n > 0 && (!p || !g || !m || !v))) return SMAT_ERR_INVALID_ARG;
  if (n == 0) return SMAT_OK;
  float c1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  float c2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  int g_ = (int)std::min<long long>((n + 255) / 256, 4096);
  adam_kernel<<<g_, 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? SMAT_OK : SMAT_ERR_CUDA;
}

}  // extern "C"
