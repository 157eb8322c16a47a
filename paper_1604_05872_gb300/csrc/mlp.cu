// Learned cost model: a two-hidden-layer tanh MLP that predicts the log time
// per element of a (form, degree, variant, tile) candidate from loop-nest
// features.  Hand-written training and inference kernels: forward, loss and
// gradient (rows in parallel, then one reduction thread per parameter, no
// atomics, so gradients are deterministic) and an Adam update.
//
// Parameter layout (float): W1[H][D] b1[H] W2[H][H] b2[H] w3[H] b3.
// The paper leaves a better cost model than pure operation counts as an open
// question (Section 8, "Limitations and future work"); this model is trained
// on timings the pipeline measures and is checked against measured time.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/fea.h"

namespace fea {

int set_error(int code, const char* msg);

namespace {

struct Off {
  int W1, b1, W2, b2, w3, b3, total;
};
__host__ __device__ inline Off offsets(int D, int H) {
  Off o;
  o.W1 = 0;
  o.b1 = H * D;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.w3 = o.b2 + H;
  o.b3 = o.w3 + H;
  o.total = o.b3 + 1;
  return o;
}

constexpr int kMaxD = 32;

template <int H>
__device__ __forceinline__ float forward_row(const float* p, const Off& o, int D, const float* x, float* a1, float* a2) {
#pragma unroll 1
  for (int i = 0; i < H; ++i) {
    float z = p[o.b1 + i];
    for (int d = 0; d < D; ++d) z = fmaf(p[o.W1 + i * D + d], x[d], z);
    a1[i] = tanhf(z);
  }
#pragma unroll 1
  for (int i = 0; i < H; ++i) {
    float z = p[o.b2 + i];
#pragma unroll 8
    for (int j = 0; j < H; ++j) z = fmaf(p[o.W2 + i * H + j], a1[j], z);
    a2[i] = tanhf(z);
  }
  float y = p[o.b3];
#pragma unroll
  for (int i = 0; i < H; ++i) y = fmaf(p[o.w3 + i], a2[i], y);
  return y;
}

template <int H>
__global__ void mlp_forward_kernel(const float* __restrict__ params, int D, const float* __restrict__ X, int n,
                                   float* __restrict__ y) {
  extern __shared__ float sp[];
  const Off o = offsets(D, H);
  for (int k = threadIdx.x; k < o.total; k += blockDim.x) sp[k] = params[k];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  float x[kMaxD];
  for (int d = 0; d < D; ++d) x[d] = X[(size_t)row * D + d];
  float a1[H], a2[H];
  y[row] = forward_row<H>(sp, o, D, x, a1, a2);
}

// Per row: forward, residual g = 2 (yhat - y) / n, and the back-propagated
// pre-activation gradients; stored to scratch [n][4H + 2]: a1, a2, dz1, dz2, g, r^2.
template <int H>
__global__ void mlp_rows_kernel(const float* __restrict__ params, int D, const float* __restrict__ X,
                                const float* __restrict__ Y, int n, float* __restrict__ S) {
  extern __shared__ float sp[];
  const Off o = offsets(D, H);
  for (int k = threadIdx.x; k < o.total; k += blockDim.x) sp[k] = params[k];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  float x[kMaxD];
  for (int d = 0; d < D; ++d) x[d] = X[(size_t)row * D + d];
  float a1[H], a2[H];
  const float yh = forward_row<H>(sp, o, D, x, a1, a2);
  const float r = yh - Y[row];
  const float g = 2.0f * r / (float)n;
  float* s = S + (size_t)row * (4 * H + 2);
  float dz2[H];
#pragma unroll
  for (int i = 0; i < H; ++i) dz2[i] = g * sp[o.w3 + i] * (1.0f - a2[i] * a2[i]);
#pragma unroll 1
  for (int j = 0; j < H; ++j) {
    float da = 0.f;
#pragma unroll 8
    for (int i = 0; i < H; ++i) da = fmaf(sp[o.W2 + i * H + j], dz2[i], da);
    s[2 * H + j] = da * (1.0f - a1[j] * a1[j]);  // dz1
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    s[i] = a1[i];
    s[H + i] = a2[i];
    s[3 * H + i] = dz2[i];
  }
  s[4 * H] = g;
  s[4 * H + 1] = r * r;
}

// One thread per parameter: sum its gradient over the rows; thread `total`
// sums the loss.
template <int H>
__global__ void mlp_reduce_kernel(int D, const float* __restrict__ X, int n, const float* __restrict__ S,
                                  float* __restrict__ grad, float* __restrict__ loss) {
  const Off o = offsets(D, H);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > o.total) return;
  const int st = 4 * H + 2;
  float acc = 0.f;
  if (k == o.total) {
    for (int r = 0; r < n; ++r) acc += S[(size_t)r * st + 4 * H + 1];
    if (loss) *loss = acc / (float)n;
    return;
  }
  if (k < o.b1) {
    const int i = k / D, d = k % D;
    for (int r = 0; r < n; ++r) acc = fmaf(S[(size_t)r * st + 2 * H + i], X[(size_t)r * D + d], acc);
  } else if (k < o.W2) {
    const int i = k - o.b1;
    for (int r = 0; r < n; ++r) acc += S[(size_t)r * st + 2 * H + i];
  } else if (k < o.b2) {
    const int i = (k - o.W2) / H, j = (k - o.W2) % H;
    for (int r = 0; r < n; ++r) acc = fmaf(S[(size_t)r * st + 3 * H + i], S[(size_t)r * st + j], acc);
  } else if (k < o.w3) {
    const int i = k - o.b2;
    for (int r = 0; r < n; ++r) acc += S[(size_t)r * st + 3 * H + i];
  } else if (k < o.b3) {
    const int i = k - o.w3;
    for (int r = 0; r < n; ++r) acc = fmaf(S[(size_t)r * st + 4 * H], S[(size_t)r * st + H + i], acc);
  } else {
    for (int r = 0; r < n; ++r) acc += S[(size_t)r * st + 4 * H];
  }
  grad[k] = acc;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

bool valid_hidden(int H) { return H == 16 || H == 32 || H == 64; }

}  // namespace
}  // namespace fea

using namespace fea;

extern "C" {

int fea_mlp_num_params(int d_in, int hidden) {
  if (d_in < 1 || d_in > kMaxD || !valid_hidden(hidden)) return -1;
  return offsets(d_in, hidden).total;
}

int64_t fea_mlp_scratch_floats(int n, int hidden) {
  if (n < 0 || !valid_hidden(hidden)) return -1;
  return (int64_t)n * (4 * hidden + 2);
}

int fea_mlp_forward(const float* params, int d_in, int hidden, const float* X, int n, float* y, void* stream) {
  if (d_in < 1 || d_in > kMaxD || !valid_hidden(hidden) || n < 0 || (n && (!params || !X || !y)))
    return set_error(FEA_EINVAL, "bad MLP forward arguments");
  if (n == 0) return FEA_OK;
  const Off o = offsets(d_in, hidden);
  const int T = 128, B = (n + T - 1) / T;
  const size_t sm = (size_t)o.total * 4;
  cudaStream_t s = (cudaStream_t)stream;
  if (hidden == 16) mlp_forward_kernel<16><<<B, T, sm, s>>>(params, d_in, X, n, y);
  else if (hidden == 32) mlp_forward_kernel<32><<<B, T, sm, s>>>(params, d_in, X, n, y);
  else mlp_forward_kernel<64><<<B, T, sm, s>>>(params, d_in, X, n, y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEA_OK : set_error(FEA_ECUDA, cudaGetErrorString(e));
}

int fea_mlp_loss_grad(const float* params, int d_in, int hidden, const float* X, const float* y, int n, float* grad,
                      float* loss, float* scratch, void* stream) {
  if (d_in < 1 || d_in > kMaxD || !valid_hidden(hidden) || n < 1 || !params || !X || !y || !grad || !scratch)
    return set_error(FEA_EINVAL, "bad MLP gradient arguments");
  const Off o = offsets(d_in, hidden);
  const int T = 128;
  const size_t sm = (size_t)o.total * 4;
  cudaStream_t s = (cudaStream_t)stream;
  const int Br = (n + T - 1) / T, Bp = (o.total + 1 + T - 1) / T;
  if (hidden == 16) {
    mlp_rows_kernel<16><<<Br, T, sm, s>>>(params, d_in, X, y, n, scratch);
    mlp_reduce_kernel<16><<<Bp, T, 0, s>>>(d_in, X, n, scratch, grad, loss);
  } else if (hidden == 32) {
    mlp_rows_kernel<32><<<Br, T, sm, s>>>(params, d_in, X, y, n, scratch);
    mlp_reduce_kernel<32><<<Bp, T, 0, s>>>(d_in, X, n, scratch, grad, loss);
  } else {
    mlp_rows_kernel<64><<<Br, T, sm, s>>>(params, d_in, X, y, n, scratch);
    mlp_reduce_kernel<64><<<Bp, T, 0, s>>>(d_in, X, n, scratch, grad, loss);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEA_OK : set_error(FEA_ECUDA, cudaGetErrorString(e));
}

int fea_mlp_adam(float* params, const float* grad, float* m, float* v, int nparam, float lr, float beta1, float beta2,
                 float eps, int step, void* stream) {
  if (nparam < 1 || !params || !grad || !m || !v || step < 1) return set_error(FEA_EINVAL, "bad Adam arguments");
  const float c1 = 1.0f - std::pow(beta1, (float)step), c2 = 1.0f - std::pow(beta2, (float)step);
  const int T = 256;
  adam_kernel<<<(nparam + T - 1) / T, T, 0, (cudaStream_t)stream>>>(params, grad, m, v, nparam, lr, beta1, beta2, eps,
                                                                     c1, c2);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? FEA_OK : set_error(FEA_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
