// The learned mode switch: feature extraction from round traces, and the
// forward pass, gradient and Adam training of its 8-16-16-1 network on the
// GPU. Sums over samples run in a fixed order (per-sample terms first, then
// one tree per parameter), so training is reproducible bit for bit.
//
// Gradient of the weighted logistic loss (per sample i, W = sum of weights):
//   z = w3 . h2 + b3,  h2 = tanh(W2 h1 + b2),  h1 = tanh(W1 x + b1)
//   dL/dz   = wt_i (sigmoid(z) - y_i) / W
//   dL/dw3  = dz h2,   dL/db3 = dz
//   d2      = dz w3 * (1 - h2^2):  dL/dW2 = d2 h1^T, dL/db2 = d2
//   d1      = (W2^T d2) * (1 - h1^2): dL/dW1 = d1 x^T, dL/db1 = d1
#include <cmath>
#include <cstring>
#include <vector>

#include "ipgc_internal.h"

namespace ipgc {

__global__ void features_kernel(const ipgc_trace_rec* __restrict__ tr, int32_t rounds, int32_t n,
                                int64_t nnz, float* __restrict__ feats) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rounds) return;
  const ipgc_trace_rec r = tr[i];
  policy_features(n, nnz, r.round, r.wl_size, r.wl_small, r.deg_sum, r.max_color,
                  feats + (size_t)i * kMlpIn);
}

__device__ __forceinline__ float softplus(float z) {
  return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z)));
}

__device__ __forceinline__ float sigmoid(float z) { return 1.0f / (1.0f + expf(-z)); }

// Per-sample forward pass; h1, h2 receive the hidden activations.
__device__ __forceinline__ float mlp_forward_one(const float* __restrict__ w,
                                                 const float* __restrict__ x, float h1[kMlpH],
                                                 float h2[kMlpH]) {
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float a = w[kB1 + j];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) a += w[kW1 + j * kMlpIn + k] * x[k];
    h1[j] = tanhf(a);
  }
  float z = w[kB3];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    float a = w[kB2 + j];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) a += w[kW2 + j * kMlpH + k] * h1[k];
    h2[j] = tanhf(a);
    z += w[kW3 + j] * h2[j];
  }
  return z;
}

__global__ void mlp_forward_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                   int32_t n, float* __restrict__ prob) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float h1[kMlpH], h2[kMlpH];
  prob[i] = sigmoid(mlp_forward_one(w, x + (size_t)i * kMlpIn, h1, h2));
}

// Per-sample loss and gradient terms into G[param][n] (param kMlpParams is
// the loss term); parameter-major so the writes are coalesced.
__global__ void mlp_terms_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                 const float* __restrict__ y, const float* __restrict__ wt,
                                 int32_t n, float inv_wsum, float* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* xi = x + (size_t)i * kMlpIn;
  float h1[kMlpH], h2[kMlpH];
  const float z = mlp_forward_one(w, xi, h1, h2);
  const float yi = y[i], wi = wt[i] * inv_wsum;
  const size_t N = (size_t)n;
  G[(size_t)kMlpParams * N + i] = wi * (softplus(z) - yi * z);
  const float dz = wi * (sigmoid(z) - yi);
  G[(size_t)kB3 * N + i] = dz;
  float d2[kMlpH];
#pragma unroll
  for (int j = 0; j < kMlpH; ++j) {
    G[(size_t)(kW3 + j) * N + i] = dz * h2[j];
    d2[j] = dz * w[kW3 + j] * (1.0f - h2[j] * h2[j]);
    G[(size_t)(kB2 + j) * N + i] = d2[j];
#pragma unroll
    for (int k = 0; k < kMlpH; ++k) G[(size_t)(kW2 + j * kMlpH + k) * N + i] = d2[j] * h1[k];
  }
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < kMlpH; ++j) s += w[kW2 + j * kMlpH + k] * d2[j];
    const float d1 = s * (1.0f - h1[k] * h1[k]);
    G[(size_t)(kB1 + k) * N + i] = d1;
#pragma unroll
    for (int c = 0; c < kMlpIn; ++c) G[(size_t)(kW1 + k * kMlpIn + c) * N + i] = d1 * xi[c];
  }
}

// One block per row of G: out[row] = sum over the n samples, in a fixed
// order (strided per-thread sums, then a shared-memory tree).
__global__ void rows_sum_kernel(const float* __restrict__ G, int32_t n, float* __restrict__ out) {
  __shared__ float s[256];
  const float* row = G + (size_t)blockIdx.x * n;
  float a = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += row[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

}  // namespace ipgc

namespace {

int check(cudaError_t e) { return e == cudaSuccess ? IPGC_OK : IPGC_ERR_CUDA; }

// weighted sum of the sample weights on the host side is avoided: the sum is
// taken on the device in the same fixed order as the gradient
int weight_sum(const float* wt, int32_t n, float* scratch, cudaStream_t s, float* out) {
  ipgc::rows_sum_kernel<<<1, 256, 0, s>>>(wt, n, scratch);
  if (cudaGetLastError() != cudaSuccess) return IPGC_ERR_CUDA;
  if (cudaMemcpyAsync(out, scratch, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return IPGC_ERR_CUDA;
  return IPGC_OK;
}

int grad_with(const float* w, const float* x, const float* y, const float* wt, int32_t n,
              float inv_wsum, float* grad, float* loss, float* scratch, cudaStream_t s) {
  const int blocks = (n + 255) / 256;
  ipgc::mlp_terms_kernel<<<blocks, 256, 0, s>>>(w, x, y, wt, n, inv_wsum, scratch);
  if (cudaGetLastError() != cudaSuccess) return IPGC_ERR_CUDA;
  ipgc::rows_sum_kernel<<<ipgc::kMlpParams, 256, 0, s>>>(scratch, n, grad);
  if (cudaGetLastError() != cudaSuccess) return IPGC_ERR_CUDA;
  if (loss) {
    ipgc::rows_sum_kernel<<<1, 256, 0, s>>>(scratch + (size_t)ipgc::kMlpParams * n, n, loss);
    if (cudaGetLastError() != cudaSuccess) return IPGC_ERR_CUDA;
  }
  return IPGC_OK;
}

}  // namespace

extern "C" {

int ipgc_policy_features(const ipgc_trace_rec* trace, int32_t rounds, int32_t n, int64_t nnz,
                         float* feats, void* stream) {
  if (rounds < 0 || n < 0 || nnz < 0 || (rounds > 0 && (!trace || !feats))) return IPGC_ERR_INVALID;
  if (rounds == 0) return IPGC_OK;
  ipgc::features_kernel<<<(rounds + 127) / 128, 128, 0, (cudaStream_t)stream>>>(trace, rounds, n,
                                                                                nnz, feats);
  return check(cudaGetLastError());
}

int ipgc_mlp_forward(const float* w, const float* x, int32_t n, float* prob, void* stream) {
  if (n < 0 || (n > 0 && (!w || !x || !prob))) return IPGC_ERR_INVALID;
  if (n == 0) return IPGC_OK;
  ipgc::mlp_forward_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, x, n, prob);
  return check(cudaGetLastError());
}

int ipgc_mlp_grad(const float* w, const float* x, const float* y, const float* wt, int32_t n,
                  float* grad, float* loss, float* scratch, void* stream) {
  if (n <= 0 || !w || !x || !y || !wt || !grad || !scratch) return IPGC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  float wsum = 0;
  int rc = weight_sum(wt, n, scratch, s, &wsum);
  if (rc != IPGC_OK) return rc;
  if (!(wsum > 0)) return IPGC_ERR_INVALID;
  return grad_with(w, x, y, wt, n, 1.0f / wsum, grad, loss, scratch, s);
}

int ipgc_mlp_train(ipgc_ctx* ctx, const float* x, const float* y, const float* wt, int32_t n,
                   int32_t epochs, float lr, float* w_inout, float* loss_out, void* stream) {
  if (!ctx || n <= 0 || epochs < 0 || !x || !y || !wt || !w_inout || !(lr > 0))
    return IPGC_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t scratch_n = (size_t)(ipgc::kMlpParams + 1) * n;
  const size_t bytes = sizeof(float) * (scratch_n + 4 * (size_t)ipgc::kMlpParams + 16);
  float* buf = nullptr;
  if (cudaMalloc((void**)&buf, bytes) != cudaSuccess) {
    ipgc::ctx_note_cuda_error(ctx, (int)cudaErrorMemoryAllocation);
    return IPGC_ERR_OOM;
  }
  float* scratch = buf;
  float* grad = scratch + scratch_n;
  float* m = grad + ipgc::kMlpParams;
  float* v = m + ipgc::kMlpParams;
  float* loss = v + ipgc::kMlpParams;
  int rc = IPGC_OK;
  float wsum = 0;
  if (cudaMemsetAsync(m, 0, sizeof(float) * 2 * ipgc::kMlpParams, s) != cudaSuccess) rc = IPGC_ERR_CUDA;
  if (rc == IPGC_OK) rc = weight_sum(wt, n, scratch, s, &wsum);
  if (rc == IPGC_OK && !(wsum > 0)) rc = IPGC_ERR_INVALID;
  double b1t = 1.0, b2t = 1.0;
  for (int32_t e = 0; rc == IPGC_OK && e < epochs; ++e) {
    rc = grad_with(w_inout, x, y, wt, n, 1.0f / wsum, grad, e + 1 == epochs ? loss : nullptr,
                   scratch, s);
    if (rc != IPGC_OK) break;
    b1t *= 0.9;
    b2t *= 0.999;
    ipgc::adam_kernel<<<(ipgc::kMlpParams + 127) / 128, 128, 0, s>>>(
        w_inout, m, v, grad, lr, (float)(1.0 - b1t), (float)(1.0 - b2t));
    if (cudaGetLastError() != cudaSuccess) rc = IPGC_ERR_CUDA;
  }
  if (rc == IPGC_OK && loss_out && epochs > 0) {
    if (cudaMemcpyAsync(loss_out, loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = IPGC_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == IPGC_OK) rc = IPGC_ERR_CUDA;
  cudaFree(buf);
  return rc;
}

}  // extern "C"
