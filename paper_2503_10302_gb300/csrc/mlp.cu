// Learned beta-ladder predictor: an fp32 MLP 259 -> 256 -> 256 -> 256 -> 32
// with a monotone head, trained with Adam on the squared ladder error plus an
// optional relative-gap term.  The paper has no learned
// component; the predictor replaces the adaptive-ladder preprocessing of
// Algorithm S2 by a network reading cheap instance features and short pilot
// histograms, on the grounds that ladders of one size are nearly identical
// across instances (Fig. S12).  These are tiny dense layers, so they run as
// plain SIMT kernels: a 64x64-tiled GEMM with bias / ReLU / ReLU-mask
// epilogues, a warp-per-sample head (scan and reverse scan over the 32
// outputs), column sums for bias gradients, and an elementwise Adam step.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "internal.h"

namespace {

constexpr int kIn = 259, kHid = 256, kOut = 32, kLayers = 4;
constexpr int kDims[kLayers + 1] = {kIn, kHid, kHid, kHid, kOut};

// C[m][n] (ldc) = epi( sum_k A(m,k) B(k,n) ) with A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  Epilogues: + bias[n]; ReLU; multiply by
// (mask[m*ldmask + n] > 0).
template <bool BIAS, bool RELU, bool MASK>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A,
                                                   int sam, int sak, const float *__restrict__ B,
                                                   int sbk, int sbn, float *__restrict__ C, int ldc,
                                                   const float *__restrict__ bias,
                                                   const float *__restrict__ mask, int ldmask) {
  __shared__ float As[16][64 + 1];
  __shared__ float Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e >> 6, mm = e & 63;
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[(size_t)m * sam + (size_t)k * sak] : 0.f;
      const int n = n0 + mm;
      Bs[kk][mm] = (n < N && k < K) ? B[(size_t)k * sbk + (size_t)n * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (BIAS) v += bias[n];
      if (RELU) v = fmaxf(v, 0.f);
      if (MASK) v = (mask[(size_t)m * ldmask + n] > 0.f) ? v : 0.f;
      C[(size_t)m * ldc + n] = v;
    }
  }
}

__device__ __forceinline__ float softplus_f(float x) {
  return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x)));
}

// One warp per sample: beta_k = beta_min + sum_{m<=k} softplus(o_m);
// loss_s = sum_k (beta_k - y_k)^2 + gw (32/31) sum_{k>=1} r_k^2 with the
// relative gap error r_k = (softplus(o_k) - d_k) / d_k, d_k = y_k - y_{k-1},
// so that sum_s loss_s / (B * 32) is the mean squared ladder error plus gw
// times the mean squared relative gap error; dO_m = sigmoid(o_m) (sum_{k>=m}
// dL/dbeta_k + [m >= 1] 2 gw r_m / (d_m B * 31)) with dL/dbeta_k =
// 2 (beta_k - y_k) / (B * 32).
__global__ void head_kernel(int B, const float *O, const float *Y, float beta_min, float gw, float *beta_out,
                            float *dO, float *loss_s) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  const float o = O[(size_t)warp * kOut + lane];
  const float sp = softplus_f(o);
  float c = sp;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float v = __shfl_up_sync(0xFFFFFFFFu, c, d);
    if (lane >= d) c += v;
  }
  const float beta = beta_min + c;
  if (beta_out) beta_out[(size_t)warp * kOut + lane] = beta;
  if (!Y) return;
  const float y = Y[(size_t)warp * kOut + lane];
  const float yprev = __shfl_up_sync(0xFFFFFFFFu, y, 1);
  const float diff = beta - y;
  float l = diff * diff;
  float r = 0.f, dgap = 1.f;
  if (gw != 0.f && lane >= 1) {
    dgap = y - yprev;
    r = (sp - dgap) / dgap;
    l += gw * (32.f / 31.f) * r * r;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, d);
  if (lane == 0) loss_s[warp] = l;
  float g = 2.f * diff / (float)(B * kOut);
  // suffix sum over k >= m
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float v = __shfl_down_sync(0xFFFFFFFFu, g, d);
    if (lane + d < 32) g += v;
  }
  const float sig = 1.f / (1.f + expf(-o));
  float dov = sig * g;
  if (gw != 0.f && lane >= 1) dov += sig * (2.f * gw * r / dgap / (float)(B * (kOut - 1)));
  dO[(size_t)warp * kOut + lane] = dov;
}

// out[n] = sum_m X[m][n] (bias gradients), one thread per column.
__global__ void colsum_kernel(int M, int N, const float *X, float *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += X[(size_t)m * N + n];
  out[n] = s;
}

// loss = sum_s loss_s / (B * 32), one block, fixed reduction order.
__global__ void loss_kernel(int B, const float *loss_s, float *loss) {
  __shared__ float part[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < B; i += 256) s += loss_s[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = part[0] / (float)(B * kOut);
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / c1) / (sqrt(v / c2) + eps) with c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void adam_kernel(int n, float *p, const float *g, float *m, float *v, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

namespace pc {

size_t mlp_param_count() {
  size_t n = 0;
  for (int l = 0; l < kLayers; ++l) n += (size_t)kDims[l + 1] * kDims[l] + kDims[l + 1];
  return n;
}

}  // namespace pc

struct pc_mlp {
  pc_ctx *ctx = nullptr;
  int device = 0;    // the context's device, kept for pc_mlp_destroy
  float beta_min = 0.f;
  float gap_weight = 0.f;   // weight of the relative-gap term of the loss
  int64_t t = 0;
  size_t n_params = 0;
  size_t w_off[kLayers], b_off[kLayers];
  pc::DevBuf<float> params, grads, m, v;
  int cap = 0;   // batch capacity of the activation buffers
  pc::DevBuf<float> X, H[3], O, dO, dH[3], Y, beta, loss_s, loss;
  pc::PinnedBuf<float> host_loss;
};

using namespace pc;

namespace {

template <bool BIAS, bool RELU, bool MASK>
int gemm(cudaStream_t st, int M, int N, int K, const float *A, int sam, int sak, const float *B, int sbk,
         int sbn, float *C, int ldc, const float *bias, const float *mask, int ldmask) {
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
  gemm_kernel<BIAS, RELU, MASK><<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, mask,
                                                       ldmask);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

int ensure_batch(pc_mlp *mm, int batch) {
  if (batch <= mm->cap) return PC_OK;
  int rc;
  const size_t b = (size_t)batch;
  if ((rc = mm->X.alloc(b * kIn)) || (rc = mm->O.alloc(b * kOut)) || (rc = mm->dO.alloc(b * kOut)) ||
      (rc = mm->Y.alloc(b * kOut)) || (rc = mm->beta.alloc(b * kOut)) || (rc = mm->loss_s.alloc(b)) ||
      (rc = mm->loss.alloc(1)))
    return rc;
  for (int l = 0; l < 3; ++l)
    if ((rc = mm->H[l].alloc(b * kHid)) || (rc = mm->dH[l].alloc(b * kHid))) return rc;
  if ((rc = mm->host_loss.reserve(1))) return rc;
  mm->cap = batch;
  return PC_OK;
}

// Forward pass from X (device, [batch][259]) to O; beta if requested.
int forward(pc_mlp *mm, int batch, const float *X, float *beta_dev) {
  cudaStream_t st = mm->ctx->stream;
  const float *p = mm->params.p;
  const float *in = X;
  int rc;
  for (int l = 0; l < 3; ++l) {
    if ((rc = gemm<true, true, false>(st, batch, kDims[l + 1], kDims[l], in, kDims[l], 1, p + mm->w_off[l], 1,
                                      kDims[l], mm->H[l].p, kDims[l + 1], p + mm->b_off[l], nullptr, 0)))
      return rc;
    in = mm->H[l].p;
  }
  if ((rc = gemm<true, false, false>(st, batch, kOut, kHid, in, kHid, 1, p + mm->w_off[3], 1, kHid, mm->O.p,
                                     kOut, p + mm->b_off[3], nullptr, 0)))
    return rc;
  if (beta_dev) {
    head_kernel<<<(batch * 32 + 255) / 256, 256, 0, st>>>(batch, mm->O.p, nullptr, mm->beta_min, 0.f, beta_dev,
                                                          nullptr, nullptr);
    PC_CUDA_TRY(cudaGetLastError());
  }
  return PC_OK;
}

// Loss and gradients into mm->grads for X, Y on the device.
int backward(pc_mlp *mm, int batch, const float *X, const float *Y) {
  cudaStream_t st = mm->ctx->stream;
  int rc = forward(mm, batch, X, nullptr);
  if (rc) return rc;
  head_kernel<<<(batch * 32 + 255) / 256, 256, 0, st>>>(batch, mm->O.p, Y, mm->beta_min, mm->gap_weight,
                                                        mm->beta.p, mm->dO.p, mm->loss_s.p);
  PC_CUDA_TRY(cudaGetLastError());
  loss_kernel<<<1, 256, 0, st>>>(batch, mm->loss_s.p, mm->loss.p);
  PC_CUDA_TRY(cudaGetLastError());
  const float *p = mm->params.p;
  float *g = mm->grads.p;
  const float *dZ = mm->dO.p;
  for (int l = kLayers - 1; l >= 0; --l) {
    const int out = kDims[l + 1], in = kDims[l];
    const float *Hin = (l == 0) ? X : mm->H[l - 1].p;
    // dW[out][in] = sum_b dZ[b][out] Hin[b][in]
    if ((rc = gemm<false, false, false>(st, out, in, batch, dZ, 1, out, Hin, in, 1, g + mm->w_off[l], in,
                                        nullptr, nullptr, 0)))
      return rc;
    colsum_kernel<<<(out + 127) / 128, 128, 0, st>>>(batch, out, dZ, g + mm->b_off[l]);
    PC_CUDA_TRY(cudaGetLastError());
    if (l > 0) {
      // dZ_{l-1}[b][in] = (sum_o dZ[b][o] W[o][in]) * (H_{l-1} > 0)
      if ((rc = gemm<false, false, true>(st, batch, in, out, dZ, out, 1, p + mm->w_off[l], in, 1,
                                         mm->dH[l - 1].p, in, nullptr, mm->H[l - 1].p, in)))
        return rc;
      dZ = mm->dH[l - 1].p;
    }
  }
  return PC_OK;
}

int adam(pc_mlp *mm, float lr) {
  mm->t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = (float)(1.0 - std::pow(0.9, (double)mm->t));
  const float c2 = (float)(1.0 - std::pow(0.999, (double)mm->t));
  const int n = (int)mm->n_params;
  adam_kernel<<<(n + 255) / 256, 256, 0, mm->ctx->stream>>>(n, mm->params.p, mm->grads.p, mm->m.p, mm->v.p, lr,
                                                             b1, b2, c1, c2, eps);
  PC_CUDA_TRY(cudaGetLastError());
  return PC_OK;
}

}  // namespace

namespace pc {

pc_ctx *mlp_context(pc_mlp *mm) { return mm->ctx; }

int mlp_input(pc_mlp *mm, int batch, float **X_dev) {
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  *X_dev = mm->X.p;
  return PC_OK;
}

int mlp_forward_input(pc_mlp *mm, int batch, const float **beta_dev) {
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  if ((rc = forward(mm, batch, mm->X.p, mm->beta.p))) return rc;
  *beta_dev = mm->beta.p;
  return PC_OK;
}

}  // namespace pc

namespace {

// Weights file: magic, the five layer widths, beta_min, then W[l] ([out][in]
// row-major) and b[l] of every layer as little-endian fp32.
constexpr char kMlpMagic[8] = {'P', 'C', 'M', 'L', 'P', '0', '0', '1'};

}  // namespace

extern "C" {

int pc_mlp_create(pc_ctx *c, pc_mlp **out, const float *const *W, const float *const *b, float beta_min) try {
  if (!c || !out || !W || !b) return fail(PC_EINVAL, "NULL argument");
  *out = nullptr;
  PC_CUDA_TRY(cudaSetDevice(c->device));
  pc_mlp *mm = new pc_mlp();
  mm->ctx = c;
  mm->device = c->device;
  mm->beta_min = beta_min;
  size_t off = 0;
  for (int l = 0; l < kLayers; ++l) {
    mm->w_off[l] = off;
    off += (size_t)kDims[l + 1] * kDims[l];
    mm->b_off[l] = off;
    off += (size_t)kDims[l + 1];
  }
  mm->n_params = off;
  std::vector<float> h(off);
  for (int l = 0; l < kLayers; ++l) {
    if (!W[l] || !b[l]) {
      delete mm;
      return fail(PC_EINVAL, "NULL weight");
    }
    std::memcpy(h.data() + mm->w_off[l], W[l], sizeof(float) * kDims[l + 1] * kDims[l]);
    std::memcpy(h.data() + mm->b_off[l], b[l], sizeof(float) * kDims[l + 1]);
  }
  int rc;
  if ((rc = mm->params.alloc(off)) || (rc = mm->grads.alloc(off)) || (rc = mm->m.alloc(off)) ||
      (rc = mm->v.alloc(off)) || (rc = mm->m.zero(c->stream)) || (rc = mm->v.zero(c->stream))) {
    delete mm;
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(mm->params.p, h.data(), off * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete mm;
    return fail(PC_ECUDA, cudaGetErrorString(e));
  }
  *out = mm;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

void pc_mlp_destroy(pc_mlp *mm) try {
  if (!mm) return;
  // the context may already be gone: use only the device recorded at
  // creation (cudaFree waits for the device's work on these buffers)
  cudaSetDevice(mm->device);
  delete mm;
} catch (...) {
}

int pc_mlp_forward(pc_mlp *mm, int batch, const float *X, float *beta) try {
  if (!mm || !X || !beta || batch < 1) return fail(PC_EINVAL, "bad arguments");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  cudaStream_t st = mm->ctx->stream;
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(mm->X.p, X, (size_t)batch * kIn * 4, cudaMemcpyHostToDevice, st));
  if ((rc = forward(mm, batch, mm->X.p, mm->beta.p))) return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(beta, mm->beta.p, (size_t)batch * kOut * 4, cudaMemcpyDeviceToHost, st));
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_grads(pc_mlp *mm, int batch, const float *X, const float *Y, float *loss, float *const *gW,
                 float *const *gb) try {
  if (!mm || !X || !Y || batch < 1) return fail(PC_EINVAL, "bad arguments");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  cudaStream_t st = mm->ctx->stream;
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(mm->X.p, X, (size_t)batch * kIn * 4, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(mm->Y.p, Y, (size_t)batch * kOut * 4, cudaMemcpyHostToDevice, st));
  if ((rc = backward(mm, batch, mm->X.p, mm->Y.p))) return rc;
  std::vector<float> h(mm->n_params);
  PC_CUDA_TRY(cudaMemcpyAsync(h.data(), mm->grads.p, h.size() * 4, cudaMemcpyDeviceToHost, st));
  float l = 0.f;
  PC_CUDA_TRY(cudaMemcpyAsync(&l, mm->loss.p, 4, cudaMemcpyDeviceToHost, st));
  PC_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = l;
  for (int k = 0; k < kLayers; ++k) {
    if (gW && gW[k]) std::memcpy(gW[k], h.data() + mm->w_off[k], sizeof(float) * kDims[k + 1] * kDims[k]);
    if (gb && gb[k]) std::memcpy(gb[k], h.data() + mm->b_off[k], sizeof(float) * kDims[k + 1]);
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_train_step_dev(pc_mlp *mm, int batch, const float *X_dev, const float *Y_dev, float lr,
                          float *loss_dev) try {
  if (!mm || !X_dev || !Y_dev || batch < 1) return fail(PC_EINVAL, "bad arguments");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  if ((rc = backward(mm, batch, X_dev, Y_dev))) return rc;
  if (loss_dev)
    PC_CUDA_TRY(cudaMemcpyAsync(loss_dev, mm->loss.p, 4, cudaMemcpyDeviceToDevice, mm->ctx->stream));
  return adam(mm, lr);
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_train_step(pc_mlp *mm, int batch, const float *X, const float *Y, float lr, float *loss) try {
  if (!mm || !X || !Y || batch < 1) return fail(PC_EINVAL, "bad arguments");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  cudaStream_t st = mm->ctx->stream;
  int rc = ensure_batch(mm, batch);
  if (rc) return rc;
  PC_CUDA_TRY(cudaMemcpyAsync(mm->X.p, X, (size_t)batch * kIn * 4, cudaMemcpyHostToDevice, st));
  PC_CUDA_TRY(cudaMemcpyAsync(mm->Y.p, Y, (size_t)batch * kOut * 4, cudaMemcpyHostToDevice, st));
  if ((rc = backward(mm, batch, mm->X.p, mm->Y.p))) return rc;
  if ((rc = adam(mm, lr))) return rc;
  if (loss) {
    PC_CUDA_TRY(cudaMemcpyAsync(mm->host_loss.p, mm->loss.p, 4, cudaMemcpyDeviceToHost, st));
    PC_CUDA_TRY(cudaStreamSynchronize(st));
    *loss = mm->host_loss.p[0];
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_get_params(pc_mlp *mm, float *const *W, float *const *b) try {
  if (!mm) return fail(PC_EINVAL, "NULL argument");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  std::vector<float> h(mm->n_params);
  PC_CUDA_TRY(cudaMemcpyAsync(h.data(), mm->params.p, h.size() * 4, cudaMemcpyDeviceToHost, mm->ctx->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(mm->ctx->stream));
  for (int k = 0; k < kLayers; ++k) {
    if (W && W[k]) std::memcpy(W[k], h.data() + mm->w_off[k], sizeof(float) * kDims[k + 1] * kDims[k]);
    if (b && b[k]) std::memcpy(b[k], h.data() + mm->b_off[k], sizeof(float) * kDims[k + 1]);
  }
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_set_gap_weight(pc_mlp *mm, float w) try {
  if (!mm || !std::isfinite(w) || w < 0.f) return fail(PC_EINVAL, "gap weight must be finite and >= 0");
  mm->gap_weight = w;
  return PC_OK;
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_save(pc_mlp *mm, const char *path) try {
  if (!mm || !path) return fail(PC_EINVAL, "NULL argument");
  PC_CUDA_TRY(cudaSetDevice(mm->ctx->device));
  std::vector<float> h(mm->n_params);
  PC_CUDA_TRY(cudaMemcpyAsync(h.data(), mm->params.p, h.size() * 4, cudaMemcpyDeviceToHost, mm->ctx->stream));
  PC_CUDA_TRY(cudaStreamSynchronize(mm->ctx->stream));
  FILE *f = fopen(path, "wb");
  if (!f) return fail(PC_EINVAL, std::string("cannot open ") + path);
  int32_t dims[kLayers + 1];
  for (int l = 0; l <= kLayers; ++l) dims[l] = kDims[l];
  bool ok = fwrite(kMlpMagic, 1, 8, f) == 8 && fwrite(dims, 4, kLayers + 1, f) == (size_t)kLayers + 1 &&
            fwrite(&mm->beta_min, 4, 1, f) == 1;
  for (int l = 0; ok && l < kLayers; ++l) {
    const size_t nw = (size_t)kDims[l + 1] * kDims[l], nb = (size_t)kDims[l + 1];
    ok = fwrite(h.data() + mm->w_off[l], 4, nw, f) == nw && fwrite(h.data() + mm->b_off[l], 4, nb, f) == nb;
  }
  if (fclose(f) != 0) ok = false;
  return ok ? PC_OK : fail(PC_EINVAL, std::string("write failed: ") + path);
} catch (...) {
  return pc::fail_exception();
}

int pc_mlp_load(pc_ctx *c, const char *path, pc_mlp **out) try {
  if (!c || !path || !out) return fail(PC_EINVAL, "NULL argument");
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return fail(PC_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t dims[kLayers + 1];
  float beta_min = 0.f;
  bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMlpMagic, 8) == 0 &&
            fread(dims, 4, kLayers + 1, f) == (size_t)kLayers + 1 && fread(&beta_min, 4, 1, f) == 1;
  for (int l = 0; ok && l <= kLayers; ++l) ok = dims[l] == kDims[l];
  std::vector<std::vector<float>> W(kLayers), b(kLayers);
  for (int l = 0; ok && l < kLayers; ++l) {
    W[l].resize((size_t)kDims[l + 1] * kDims[l]);
    b[l].resize((size_t)kDims[l + 1]);
    ok = fread(W[l].data(), 4, W[l].size(), f) == W[l].size() && fread(b[l].data(), 4, b[l].size(), f) == b[l].size();
  }
  fclose(f);
  if (!ok) return fail(PC_EINVAL, std::string("not a ladder-MLP weights file of this network: ") + path);
  const float *Wp[kLayers], *bp[kLayers];
  for (int l = 0; l < kLayers; ++l) {
    Wp[l] = W[l].data();
    bp[l] = b[l].data();
  }
  return pc_mlp_create(c, out, Wp, bp, beta_min);
} catch (...) {
  return pc::fail_exception();
}

}  // extern "C"
