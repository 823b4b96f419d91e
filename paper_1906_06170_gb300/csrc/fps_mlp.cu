// Threshold-predicting MLP: training and inference kernels (no paper
// counterpart -- the learned filter of the batched search).
//
//   x  = [166 query bits, popc(q) / 166]        167 features (padded to 168)
//   h1 = relu(W1 x + b1)                        W1: 256 x 167
//   h2 = relu(W2 h1 + b2)                       W2: 256 x 256
//   y  = w3 . h2 + b3                           predicted k-th distance
//
// Weights are kept as FP32 masters (for Adam) and BF16 copies used by every
// product; layer inputs are rounded to BF16; all sums accumulate in FP32.
// Loss: mean pinball (quantile) loss, so predictions err on the high side.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fps_internal.h"

namespace fps {
namespace {

constexpr int kIn = 167, kInPad = 168, kH = 256;
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
                 kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kNParams = kOffB3 + 1;

struct Mlp {
  int device = 0;
  float* master = nullptr;       // kNParams
  float* grad = nullptr;         // kNParams
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  __nv_bfloat16* w1b = nullptr;  // 256 x 168
  __nv_bfloat16* w2b = nullptr;  // 256 x 256
  __nv_bfloat16* w3b = nullptr;  // 256
  float* loss = nullptr;         // device scalar
  int64_t step = 0;
  // activation workspace for a batch of up to cap rows
  int cap = 0;
  __nv_bfloat16* X = nullptr;    // cap x 168
  float* z1 = nullptr;           // cap x 256
  __nv_bfloat16* h1b = nullptr;
  float* z2 = nullptr;
  __nv_bfloat16* h2b = nullptr;
  float* y = nullptr;            // cap
  float* dy = nullptr;
  float* dh2 = nullptr;          // cap x 256
  float* dh1 = nullptr;
  std::mutex mu;
};

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

__global__ void features_kernel(const uint64_t* q, int B, __nv_bfloat16* X) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const uint64_t w[3] = {q[3 * b], q[3 * b + 1], q[3 * b + 2]};
  const int pc = __popcll(w[0]) + __popcll(w[1]) + __popcll(w[2]);
  for (int j = threadIdx.x; j < kInPad; j += blockDim.x) {
    float f = 0.f;
    if (j < kBits)
      f = static_cast<float>((w[j >> 6] >> (j & 63)) & 1ull);
    else if (j == kBits)
      f = static_cast<float>(pc) / 166.0f;
    X[static_cast<size_t>(b) * kInPad + j] = __float2bfloat16_rn(f);
  }
}

// C(m, n) = sum_k A(m, k) B(k, n) with A(m, k) = A[m*ars + k*acs], B(k, n) = B[k*brs + n*bcs].
// Epilogue: + bias[n]; C written (FP32); optional BF16 copy of relu(C); optional
// multiply by [mask(m, n) > 0] (ReLU derivative) before writing.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const TA* __restrict__ A, int64_t ars,
                                                    int64_t acs, const TB* __restrict__ Bm, int64_t brs, int64_t bcs,
                                                    float* __restrict__ C, int64_t ldc, const float* __restrict__ bias,
                                                    __nv_bfloat16* __restrict__ Crelu, int64_t ldr,
                                                    const float* __restrict__ mask, int64_t ldm) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int i = threadIdx.x; i < BM * BK; i += 256) {
      int mm = i % BM, kk = i / BM;
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? to_f(A[gm * ars + gk * acs]) : 0.f;
    }
    for (int i = threadIdx.x; i < BN * BK; i += 256) {
      int nn = i % BN, kk = i / BN;
      int gn = n0 + nn, gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? to_f(Bm[gk * brs + gn * bcs]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j] + (bias ? bias[gn] : 0.f);
      if (mask && !(mask[gm * ldm + gn] > 0.f)) v = 0.f;
      C[gm * ldc + gn] = v;
      if (Crelu) Crelu[gm * ldr + gn] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
    }
  }
}

// y[b] = h2b[b] . w3b + b3 (one warp per row)
__global__ void output_kernel(const __nv_bfloat16* h2b, const __nv_bfloat16* w3b, const float* b3, int B, float* y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  float s = 0.f;
  for (int n = lane; n < kH; n += 32)
    s = fmaf(__bfloat162float(h2b[static_cast<size_t>(warp) * kH + n]), __bfloat162float(w3b[n]), s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (lane == 0) y[warp] = s + b3[0];
}

// dL/dy of the mean pinball loss, and the loss itself (summed into *loss)
__global__ void pinball_kernel(const float* y, const float* t, int B, float q, float* dy, float* loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (b < B) {
    const float r = t[b] - y[b];
    dy[b] = (r > 0.f ? -q : 1.f - q) / static_cast<float>(B);
    l = fmaxf(q * r, (q - 1.f) * r) / static_cast<float>(B);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dh2[b][n] = dy[b] * w3b[n] * [z2[b][n] > 0]
__global__ void dh2_kernel(const float* dy, const __nv_bfloat16* w3b, const float* z2, int B, float* dh2) {
  const size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  if (i >= static_cast<size_t>(B) * kH) return;
  const int b = static_cast<int>(i / kH), n = static_cast<int>(i % kH);
  dh2[i] = z2[i] > 0.f ? dy[b] * __bfloat162float(w3b[n]) : 0.f;
}

// out[n] = sum_b A[b][n] * (wt ? wt[b] : 1)   (A as float or bf16, row stride lda)
template <typename T>
__global__ void colsum_kernel(const T* A, int64_t lda, int B, int N, const float* wt, float* out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s = fmaf(to_f(A[b * lda + n]), wt ? wt[b] : 1.f, s);
  out[n] = s;
}

__global__ void sum_kernel(const float* a, int B, float* out) {
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += a[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  __shared__ float part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (static_cast<int>(blockDim.x) + 31) / 32; ++i) t += part[i];
    *out = t;
  }
}

// BF16 copies of the weight matrices from the FP32 masters
__global__ void refresh_bf16_kernel(const float* p, __nv_bfloat16* w1b, __nv_bfloat16* w2b, __nv_bfloat16* w3b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kH * kInPad) {
    int n = i / kInPad, k = i % kInPad;
    w1b[i] = __float2bfloat16_rn(k < kIn ? p[kOffW1 + n * kIn + k] : 0.f);
  }
  if (i < kH * kH) w2b[i] = __float2bfloat16_rn(p[kOffW2 + i]);
  if (i < kH) w3b[i] = __float2bfloat16_rn(p[kOffW3 + i]);
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int64_t n, float lr, float c1, float c2) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

template <typename TA, typename TB>
cudaError_t gemm(int M, int N, int K, const TA* A, int64_t ars, int64_t acs, const TB* Bm, int64_t brs, int64_t bcs,
                 float* C, int64_t ldc, const float* bias, __nv_bfloat16* Crelu, int64_t ldr, const float* mask,
                 int64_t ldm, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  gemm_kernel<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, ars, acs, Bm, brs, bcs, C, ldc, bias, Crelu, ldr, mask, ldm);
  return cudaGetLastError();
}

void free_ws(Mlp* M) {
  cudaFree(M->X);
  cudaFree(M->z1);
  cudaFree(M->h1b);
  cudaFree(M->z2);
  cudaFree(M->h2b);
  cudaFree(M->y);
  cudaFree(M->dy);
  cudaFree(M->dh2);
  cudaFree(M->dh1);
  M->X = nullptr;
  M->z1 = M->z2 = M->y = M->dy = M->dh2 = M->dh1 = nullptr;
  M->h1b = M->h2b = nullptr;
  M->cap = 0;
}

bool ensure_ws(Mlp* M, int B) {
  if (B <= M->cap) return true;
  free_ws(M);
  const size_t b = static_cast<size_t>(B);
  bool ok = cudaMalloc(&M->X, b * kInPad * 2) == cudaSuccess && cudaMalloc(&M->z1, b * kH * 4) == cudaSuccess &&
            cudaMalloc(&M->h1b, b * kH * 2) == cudaSuccess && cudaMalloc(&M->z2, b * kH * 4) == cudaSuccess &&
            cudaMalloc(&M->h2b, b * kH * 2) == cudaSuccess && cudaMalloc(&M->y, b * 4) == cudaSuccess &&
            cudaMalloc(&M->dy, b * 4) == cudaSuccess && cudaMalloc(&M->dh2, b * kH * 4) == cudaSuccess &&
            cudaMalloc(&M->dh1, b * kH * 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_ws(M);
    return false;
  }
  M->cap = B;
  return true;
}

cudaError_t forward(Mlp* M, const uint64_t* q, int B, cudaStream_t s) {
  features_kernel<<<B, 64, 0, s>>>(q, B, M->X);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)  // z1 = X W1^T + b1; h1b = bf16(relu(z1))
    e = gemm<__nv_bfloat16, __nv_bfloat16>(B, kH, kInPad, M->X, kInPad, 1, M->w1b, 1, kInPad, M->z1, kH,
                                           M->master + kOffB1, M->h1b, kH, nullptr, 0, s);
  if (e == cudaSuccess)
    e = gemm<__nv_bfloat16, __nv_bfloat16>(B, kH, kH, M->h1b, kH, 1, M->w2b, 1, kH, M->z2, kH, M->master + kOffB2,
                                           M->h2b, kH, nullptr, 0, s);
  if (e == cudaSuccess) {
    output_kernel<<<(B * 32 + 255) / 256, 256, 0, s>>>(M->h2b, M->w3b, M->master + kOffB3, B, M->y);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t backward(Mlp* M, const float* t, int B, float quantile, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(M->loss, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  pinball_kernel<<<(B + 255) / 256, 256, 0, s>>>(M->y, t, B, quantile, M->dy, M->loss);
  float* g = M->grad;
  // output layer
  colsum_kernel<__nv_bfloat16><<<1, kH, 0, s>>>(M->h2b, kH, B, kH, M->dy, g + kOffW3);
  sum_kernel<<<1, 256, 0, s>>>(M->dy, B, g + kOffB3);
  dh2_kernel<<<(B * kH + 255) / 256, 256, 0, s>>>(M->dy, M->w3b, M->z2, B, M->dh2);
  e = cudaGetLastError();
  // W2: dW2[n][k] = sum_b dh2[b][n] h1b[b][k]
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16>(kH, kH, B, M->dh2, 1, kH, M->h1b, kH, 1, g + kOffW2, kH, nullptr, nullptr, 0,
                                   nullptr, 0, s);
  if (e == cudaSuccess) {
    colsum_kernel<float><<<1, kH, 0, s>>>(M->dh2, kH, B, kH, nullptr, g + kOffB2);
    e = cudaGetLastError();
  }
  // dh1[b][k] = sum_n dh2[b][n] W2b[n][k], times [z1 > 0]
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16>(B, kH, kH, M->dh2, kH, 1, M->w2b, kH, 1, M->dh1, kH, nullptr, nullptr, 0, M->z1, kH,
                                   s);
  // W1: dW1[n][k] = sum_b dh1[b][n] X[b][k]  (k < 167)
  if (e == cudaSuccess)
    e = gemm<float, __nv_bfloat16>(kH, kIn, B, M->dh1, 1, kH, M->X, kInPad, 1, g + kOffW1, kIn, nullptr, nullptr, 0,
                                   nullptr, 0, s);
  if (e == cudaSuccess) {
    colsum_kernel<float><<<1, kH, 0, s>>>(M->dh1, kH, B, kH, nullptr, g + kOffB1);
    e = cudaGetLastError();
  }
  return e;
}

struct Guard {
  int prev = -1;
  bool ok = false;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace
}  // namespace fps

using fps::Mlp;

extern "C" {

size_t fps_mlp_param_count(void) { return fps::kNParams; }

fps_status fps_mlp_create(int device, fps_mlp* out) {
  if (!out) return FPS_ERR_INVALID_ARG;
  *out = nullptr;
  Mlp* M = new (std::nothrow) Mlp();
  if (!M) return FPS_ERR_NOMEM;
  M->device = device;
  fps::Guard g(device);
  const size_t pb = fps::kNParams * sizeof(float);
  bool ok = g.ok && cudaMalloc(&M->master, pb) == cudaSuccess && cudaMalloc(&M->grad, pb) == cudaSuccess &&
            cudaMalloc(&M->m, pb) == cudaSuccess && cudaMalloc(&M->v, pb) == cudaSuccess &&
            cudaMalloc(&M->w1b, fps::kH * fps::kInPad * 2) == cudaSuccess &&
            cudaMalloc(&M->w2b, fps::kH * fps::kH * 2) == cudaSuccess &&
            cudaMalloc(&M->w3b, fps::kH * 2) == cudaSuccess && cudaMalloc(&M->loss, sizeof(float)) == cudaSuccess &&
            cudaMemset(M->master, 0, pb) == cudaSuccess && cudaMemset(M->m, 0, pb) == cudaSuccess &&
            cudaMemset(M->v, 0, pb) == cudaSuccess;
  if (ok) {
    fps::refresh_bf16_kernel<<<(fps::kH * fps::kH + 255) / 256, 256>>>(M->master, M->w1b, M->w2b, M->w3b);
    ok = cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    fps_mlp_release(reinterpret_cast<fps_mlp>(M));
    return FPS_ERR_CUDA;
  }
  *out = reinterpret_cast<fps_mlp>(M);
  return FPS_OK;
}

fps_status fps_mlp_release(fps_mlp mlp) {
  if (!mlp) return FPS_OK;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  fps::Guard g(M->device);
  fps::free_ws(M);
  cudaFree(M->master);
  cudaFree(M->grad);
  cudaFree(M->m);
  cudaFree(M->v);
  cudaFree(M->w1b);
  cudaFree(M->w2b);
  cudaFree(M->w3b);
  cudaFree(M->loss);
  delete M;
  return FPS_OK;
}

fps_status fps_mlp_set_params(fps_mlp mlp, const float* host, size_t n) {
  if (!mlp || !host || n != fps::kNParams) return FPS_ERR_INVALID_ARG;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  std::lock_guard<std::mutex> lock(M->mu);
  fps::Guard g(M->device);
  const size_t pb = n * sizeof(float);
  if (cudaMemcpy(M->master, host, pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(M->m, 0, pb) != cudaSuccess || cudaMemset(M->v, 0, pb) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  M->step = 0;
  fps::refresh_bf16_kernel<<<(fps::kH * fps::kH + 255) / 256, 256>>>(M->master, M->w1b, M->w2b, M->w3b);
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return FPS_ERR_CUDA;
  return FPS_OK;
}

fps_status fps_mlp_get_params(fps_mlp mlp, float* host, size_t n) {
  if (!mlp || !host || n != fps::kNParams) return FPS_ERR_INVALID_ARG;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  std::lock_guard<std::mutex> lock(M->mu);
  fps::Guard g(M->device);
  if (cudaMemcpy(host, M->master, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  return FPS_OK;
}

fps_status fps_mlp_predict(fps_mlp mlp, const uint64_t* queries, int Q, float* out, void* cuda_stream) {
  if (!mlp || Q < 0 || (Q > 0 && (!queries || !out))) return FPS_ERR_INVALID_ARG;
  if (Q == 0) return FPS_OK;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  std::lock_guard<std::mutex> lock(M->mu);
  fps::Guard g(M->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (!fps::ensure_ws(M, Q)) return FPS_ERR_CUDA;
  if (fps::forward(M, queries, Q, s) != cudaSuccess ||
      cudaMemcpyAsync(out, M->y, sizeof(float) * Q, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  return FPS_OK;
}

fps_status fps_mlp_grad(fps_mlp mlp, const uint64_t* queries, const float* targets, int B, float quantile,
                        float* grad_host, float* loss_host, void* cuda_stream) {
  if (!mlp || B <= 0 || !queries || !targets || !(quantile > 0.f && quantile < 1.f)) return FPS_ERR_INVALID_ARG;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  std::lock_guard<std::mutex> lock(M->mu);
  fps::Guard g(M->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (!fps::ensure_ws(M, B)) return FPS_ERR_CUDA;
  if (fps::forward(M, queries, B, s) != cudaSuccess || fps::backward(M, targets, B, quantile, s) != cudaSuccess) {
    cudaGetLastError();
    return FPS_ERR_CUDA;
  }
  if (grad_host && cudaMemcpyAsync(grad_host, M->grad, fps::kNParams * sizeof(float), cudaMemcpyDeviceToHost, s) !=
                       cudaSuccess)
    return FPS_ERR_CUDA;
  if (loss_host && cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return FPS_ERR_CUDA;
  if ((grad_host || loss_host) && cudaStreamSynchronize(s) != cudaSuccess) return FPS_ERR_CUDA;
  return FPS_OK;
}

fps_status fps_mlp_train_step(fps_mlp mlp, const uint64_t* queries, const float* targets, int B, float quantile,
                              float lr, float* loss_host, void* cuda_stream) {
  fps_status st = fps_mlp_grad(mlp, queries, targets, B, quantile, nullptr, nullptr, cuda_stream);
  if (st != FPS_OK) return st;
  Mlp* M = reinterpret_cast<Mlp*>(mlp);
  std::lock_guard<std::mutex> lock(M->mu);
  fps::Guard g(M->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  M->step += 1;
  const float c1 = 1.f - std::pow(0.9f, static_cast<float>(M->step));
  const float c2 = 1.f - std::pow(0.999f, static_cast<float>(M->step));
  fps::adam_kernel<<<static_cast<int>((fps::kNParams + 255) / 256), 256, 0, s>>>(M->master, M->grad, M->m, M->v,
                                                                                 fps::kNParams, lr, c1, c2);
  fps::refresh_bf16_kernel<<<(fps::kH * fps::kH + 255) / 256, 256, 0, s>>>(M->master, M->w1b, M->w2b, M->w3b);
  if (cudaGetLastError() != cudaSuccess) return FPS_ERR_CUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FPS_ERR_CUDA;
  }
  return FPS_OK;
}

}  // extern "C"
