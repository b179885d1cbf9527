// Learned T0 predictor: a 6 -> 128 -> 128 -> 2 multilayer perceptron (tanh hidden layers,
// linear output) with BF16 weights and FP32 accumulation, trained on the GPU by these
// kernels (forward, mean-squared-error loss, backward, Adam). The inputs are features of
// the linear system and the clock budget (Sec. VI: kappa, the eigenvalue bounds, N, Q_PE),
// the outputs the optimal Hamiltonian-simulation time T0* and the clock count, replacing the
// power-law fit T0* ~ kappa of Sec. VI where the network is available.
//
// Parameter vector (FP32 master copy, flat): W1 [128][6], b1 [128], W2 [128][128], b2 [128],
// W3 [2][128], b3 [2]. Forward and backward read the BF16 rounding of W1, W2, W3 (refreshed
// after every update); gradients and Adam moments are FP32.
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "hhl_common.cuh"

namespace hhl {
namespace {

constexpr int kIn = HHL_MLP_IN, kH = HHL_MLP_HIDDEN, kOut = HHL_MLP_OUT;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kOut * kH, kParams = kOffB3 + kOut;
static_assert(kParams == HHL_MLP_PARAMS, "parameter layout");
constexpr int kRows = 32;  // rows per CTA
constexpr int kThr = 128;  // one thread per hidden unit
constexpr size_t kFwdSmem = ((size_t)(kH + 2 * kRows) * (kH + 1) + kRows * kIn) * sizeof(float);
constexpr size_t kBwdSmem = ((size_t)(kH + 4 * kRows) * (kH + 1) + kRows * kIn + kRows * kOut) * sizeof(float);

// forward for kRows rows; if act1/act2 given, the activations are stored (training)
__global__ void __launch_bounds__(kThr) k_mlp_forward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ p,
                                                      const float* __restrict__ x, int rows, float* __restrict__ y,
                                                      float* __restrict__ act1, float* __restrict__ act2) {
  extern __shared__ float smem_f[];
  float(*sW2)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f);
  float(*h1)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + kH * (kH + 1));
  float(*h2)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + (kH + kRows) * (kH + 1));
  float(*sx)[kIn] = reinterpret_cast<float(*)[kIn]>(smem_f + (kH + 2 * kRows) * (kH + 1));
  const int j = threadIdx.x;
  const int r0 = blockIdx.x * kRows;
  for (int e = j; e < kH * kH; e += kThr) sW2[e / kH][e % kH] = __bfloat162float(wb[kOffW2 + e]);
  for (int e = j; e < kRows * kIn; e += kThr) {
    const int r = e / kIn, i = e % kIn;
    sx[r][i] = (r0 + r < rows) ? x[(size_t)(r0 + r) * kIn + i] : 0.f;
  }
  __syncthreads();
  float w1[kIn];
#pragma unroll
  for (int i = 0; i < kIn; ++i) w1[i] = __bfloat162float(wb[kOffW1 + j * kIn + i]);
  const float bb1 = p[kOffB1 + j], bb2 = p[kOffB2 + j];
  for (int r = 0; r < kRows; ++r) {
    float a = bb1;
#pragma unroll
    for (int i = 0; i < kIn; ++i) a = fmaf(w1[i], sx[r][i], a);
    h1[r][j] = tanhf(a);
  }
  __syncthreads();
  for (int r = 0; r < kRows; ++r) {
    float a = bb2;
#pragma unroll 8
    for (int k = 0; k < kH; ++k) a = fmaf(sW2[j][k], h1[r][k], a);
    h2[r][j] = tanhf(a);
  }
  __syncthreads();
  if (j < kRows * kOut) {
    const int r = j / kOut, o = j % kOut;
    float a = p[kOffB3 + o];
    for (int k = 0; k < kH; ++k) a = fmaf(__bfloat162float(wb[kOffW3 + o * kH + k]), h2[r][k], a);
    if (r0 + r < rows) y[(size_t)(r0 + r) * kOut + o] = a;
  }
  if (act1 != nullptr) {
    for (int r = 0; r < kRows; ++r)
      if (r0 + r < rows) {
        act1[(size_t)(r0 + r) * kH + j] = h1[r][j];
        act2[(size_t)(r0 + r) * kH + j] = h2[r][j];
      }
  }
}

// loss = sum_{r,o} (y - t)^2 / (rows * kOut); gy = d loss / d y
__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ t, int rows, float* __restrict__ gy,
                           float* __restrict__ loss) {
  const float scale = 1.f / (float)(rows * kOut);
  float acc = 0.f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * kOut; e += gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    gy[e] = 2.f * d * scale;
    acc += d * d * scale;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// backward for kRows rows; gradients accumulated (atomically) into g (kParams floats)
__global__ void __launch_bounds__(kThr) k_mlp_backward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ x,
                                                       const float* __restrict__ act1, const float* __restrict__ act2,
                                                       const float* __restrict__ gy, int rows, float* __restrict__ g) {
  extern __shared__ float smem_f[];
  float(*sW2)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f);
  float(*h1)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + kH * (kH + 1));
  float(*h2)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + (kH + kRows) * (kH + 1));
  float(*ga2)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + (kH + 2 * kRows) * (kH + 1));
  float(*ga1)[kH + 1] = reinterpret_cast<float(*)[kH + 1]>(smem_f + (kH + 3 * kRows) * (kH + 1));
  float(*sx)[kIn] = reinterpret_cast<float(*)[kIn]>(smem_f + (kH + 4 * kRows) * (kH + 1));
  float(*sgy)[kOut] = reinterpret_cast<float(*)[kOut]>(smem_f + (kH + 4 * kRows) * (kH + 1) + kRows * kIn);
  const int j = threadIdx.x;
  const int r0 = blockIdx.x * kRows;
  for (int e = j; e < kH * kH; e += kThr) sW2[e / kH][e % kH] = __bfloat162float(wb[kOffW2 + e]);
  for (int e = j; e < kRows * kIn; e += kThr) {
    const int r = e / kIn, i = e % kIn;
    sx[r][i] = (r0 + r < rows) ? x[(size_t)(r0 + r) * kIn + i] : 0.f;
  }
  if (j < kRows * kOut) {
    const int r = j / kOut, o = j % kOut;
    sgy[r][o] = (r0 + r < rows) ? gy[(size_t)(r0 + r) * kOut + o] : 0.f;
  }
  for (int r = 0; r < kRows; ++r) {
    const bool ok = r0 + r < rows;
    h1[r][j] = ok ? act1[(size_t)(r0 + r) * kH + j] : 0.f;
    h2[r][j] = ok ? act2[(size_t)(r0 + r) * kH + j] : 0.f;
  }
  __syncthreads();
  // output layer
  const float w30 = __bfloat162float(wb[kOffW3 + j]), w31 = __bfloat162float(wb[kOffW3 + kH + j]);
  float gw30 = 0.f, gw31 = 0.f;
  for (int r = 0; r < kRows; ++r) {
    gw30 = fmaf(sgy[r][0], h2[r][j], gw30);
    gw31 = fmaf(sgy[r][1], h2[r][j], gw31);
    const float gh2 = w30 * sgy[r][0] + w31 * sgy[r][1];
    ga2[r][j] = gh2 * (1.f - h2[r][j] * h2[r][j]);
  }
  atomicAdd(&g[kOffW3 + j], gw30);
  atomicAdd(&g[kOffW3 + kH + j], gw31);
  if (j < kOut) {
    float gb = 0.f;
    for (int r = 0; r < kRows; ++r) gb += sgy[r][j];
    atomicAdd(&g[kOffB3 + j], gb);
  }
  __syncthreads();
  // hidden layer 2: gW2[j][k] = sum_r ga2[r][j] h1[r][k]; gb2[j]; gh1[r][k] = sum_j W2[j][k] ga2[r][j]
  {
    float gb = 0.f;
    for (int r = 0; r < kRows; ++r) gb += ga2[r][j];
    atomicAdd(&g[kOffB2 + j], gb);
    for (int k = 0; k < kH; ++k) {
      float a = 0.f;
      for (int r = 0; r < kRows; ++r) a = fmaf(ga2[r][j], h1[r][k], a);
      atomicAdd(&g[kOffW2 + j * kH + k], a);
    }
  }
  for (int r = 0; r < kRows; ++r) {
    float a = 0.f;
#pragma unroll 8
    for (int jj = 0; jj < kH; ++jj) a = fmaf(sW2[jj][j], ga2[r][jj], a);
    ga1[r][j] = a * (1.f - h1[r][j] * h1[r][j]);
  }
  __syncthreads();
  // hidden layer 1
  {
    float gb = 0.f, gw[kIn] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int r = 0; r < kRows; ++r) {
      gb += ga1[r][j];
#pragma unroll
      for (int i = 0; i < kIn; ++i) gw[i] = fmaf(ga1[r][j], sx[r][i], gw[i]);
    }
    atomicAdd(&g[kOffB1 + j], gb);
#pragma unroll
    for (int i = 0; i < kIn; ++i) atomicAdd(&g[kOffW1 + j * kIn + i], gw[i]);
  }
}

// Adam on the FP32 master parameters, then the BF16 copy.
__global__ void k_mlp_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, float lr, float b1c, float b2c) {
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kParams; e += gridDim.x * blockDim.x) {
    const float gr = g[e];
    const float mm = beta1 * m[e] + (1.f - beta1) * gr;
    const float vv = beta2 * v[e] + (1.f - beta2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    const float upd = lr * (mm / b1c) / (sqrtf(vv / b2c) + eps);
    const float w = p[e] - upd;
    p[e] = w;
    wb[e] = __float2bfloat16_rn(w);
  }
}

__global__ void k_mlp_round(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kParams; e += gridDim.x * blockDim.x)
    wb[e] = __float2bfloat16_rn(p[e]);
}

}  // namespace
}  // namespace hhl

struct hhl_mlp_s {
  float* p = nullptr;           // FP32 master parameters
  float* m = nullptr;           // Adam moments
  float* v = nullptr;
  float* g = nullptr;           // gradient accumulator
  __nv_bfloat16* wb = nullptr;  // BF16 copy used by forward / backward
  float* act = nullptr;         // activations (2 x cap x 128)
  float* y = nullptr;           // outputs (cap x 2)
  float* gy = nullptr;
  int cap = 0;
  int64_t step = 0;
};

namespace hhl {
namespace {

hhl_status mlp_reserve(hhl_mlp_s* n, int rows) {
  if (rows <= n->cap) return HHL_OK;
  if (n->act) cudaFree(n->act);
  if (n->y) cudaFree(n->y);
  if (n->gy) cudaFree(n->gy);
  n->act = nullptr;
  n->y = nullptr;
  n->gy = nullptr;
  if (cudaMalloc(&n->act, (size_t)2 * rows * kH * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->y, (size_t)rows * kOut * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->gy, (size_t)rows * kOut * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    n->cap = 0;
    return fail(HHL_ERR_OOM, "MLP activation buffers");
  }
  n->cap = rows;
  return HHL_OK;
}

hhl_status mlp_grad(hhl_mlp_s* n, const float* x, const float* t, int rows, float* loss, cudaStream_t st) {
  hhl_status s = mlp_reserve(n, rows);
  if (s != HHL_OK) return s;
  const int blocks = (rows + kRows - 1) / kRows;
  HHL_CUDA_TRY(cudaMemsetAsync(n->g, 0, kParams * sizeof(float), st));
  HHL_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), st));
  float* a1 = n->act;
  float* a2 = n->act + (size_t)n->cap * kH;
  HHL_PROF_BEGIN(st);
  k_mlp_forward<<<blocks, kThr, kFwdSmem, st>>>(n->wb, n->p, x, rows, n->y, a1, a2);
  HHL_LAUNCH_CHECK("k_mlp_forward");
  HHL_PROF_BEGIN(st);
  k_mlp_loss<<<std::min(64, (rows * kOut + 255) / 256), 256, 0, st>>>(n->y, t, rows, n->gy, loss);
  HHL_LAUNCH_CHECK("k_mlp_loss");
  HHL_PROF_BEGIN(st);
  k_mlp_backward<<<blocks, kThr, kBwdSmem, st>>>(n->wb, x, a1, a2, n->gy, rows, n->g);
  HHL_LAUNCH_CHECK("k_mlp_backward");
  return HHL_OK;
}

}  // namespace
}  // namespace hhl

extern "C" {

hhl_status hhl_mlp_create(hhl_mlp_t* out) {
  using namespace hhl;
  if (out == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  hhl_mlp_s* n = new hhl_mlp_s();
  if (cudaMalloc(&n->p, kParams * sizeof(float)) != cudaSuccess || cudaMalloc(&n->m, kParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->v, kParams * sizeof(float)) != cudaSuccess || cudaMalloc(&n->g, kParams * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&n->wb, kParams * sizeof(__nv_bfloat16)) != cudaSuccess) {
    cudaGetLastError();
    hhl_mlp_destroy(n);
    return fail(HHL_ERR_OOM, "MLP parameter buffers");
  }
  if (cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem) != cudaSuccess ||
      cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem) != cudaSuccess) {
    cudaGetLastError();
    hhl_mlp_destroy(n);
    return fail(HHL_ERR_CUDA, "MLP kernel attributes");
  }
  cudaMemset(n->p, 0, kParams * sizeof(float));
  cudaMemset(n->m, 0, kParams * sizeof(float));
  cudaMemset(n->v, 0, kParams * sizeof(float));
  cudaMemset(n->wb, 0, kParams * sizeof(__nv_bfloat16));
  *out = n;
  return HHL_OK;
}

void hhl_mlp_destroy(hhl_mlp_t n) {
  if (n == nullptr) return;
  void* ptrs[] = {n->p, n->m, n->v, n->g, n->wb, n->act, n->y, n->gy};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete n;
}

hhl_status hhl_mlp_set_params(hhl_mlp_t n, const float* host_params, void* stream) {
  using namespace hhl;
  if (n == nullptr || host_params == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  HHL_CUDA_TRY(cudaMemcpyAsync(n->p, host_params, kParams * sizeof(float), cudaMemcpyHostToDevice, st));
  HHL_CUDA_TRY(cudaMemsetAsync(n->m, 0, kParams * sizeof(float), st));
  HHL_CUDA_TRY(cudaMemsetAsync(n->v, 0, kParams * sizeof(float), st));
  n->step = 0;
  HHL_PROF_BEGIN(st);
  k_mlp_round<<<(kParams + 255) / 256, 256, 0, st>>>(n->p, n->wb);
  HHL_LAUNCH_CHECK("k_mlp_round");
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  return HHL_OK;
}

hhl_status hhl_mlp_get_params(hhl_mlp_t n, float* host_params, void* stream) {
  using namespace hhl;
  if (n == nullptr || host_params == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  HHL_CUDA_TRY(cudaMemcpyAsync(host_params, n->p, kParams * sizeof(float), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  return HHL_OK;
}

hhl_status hhl_mlp_forward(hhl_mlp_t n, const float* x_dev, int32_t rows, float* y_dev, void* stream) {
  using namespace hhl;
  if (n == nullptr || x_dev == nullptr || y_dev == nullptr || rows < 1) return fail(HHL_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  HHL_PROF_BEGIN(st);
  k_mlp_forward<<<(rows + kRows - 1) / kRows, kThr, kFwdSmem, st>>>(n->wb, n->p, x_dev, rows, y_dev, nullptr, nullptr);
  HHL_LAUNCH_CHECK("k_mlp_forward");
  return HHL_OK;
}

hhl_status hhl_t0_predict(hhl_mlp_t n, const float* features_dev, int32_t rows, float* out_dev, void* stream) {
  return hhl_mlp_forward(n, features_dev, rows, out_dev, stream);
}

hhl_status hhl_mlp_gradients(hhl_mlp_t n, const float* x_dev, const float* t_dev, int32_t rows, float* grad_dev,
                             float* loss_dev, void* stream) {
  using namespace hhl;
  if (n == nullptr || x_dev == nullptr || t_dev == nullptr || grad_dev == nullptr || loss_dev == nullptr || rows < 1)
    return fail(HHL_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  hhl_status s = mlp_grad(n, x_dev, t_dev, rows, loss_dev, st);
  if (s != HHL_OK) return s;
  HHL_CUDA_TRY(cudaMemcpyAsync(grad_dev, n->g, kParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return HHL_OK;
}

hhl_status hhl_mlp_train_step(hhl_mlp_t n, const float* x_dev, const float* t_dev, int32_t rows, float lr,
                              float* loss_dev, void* stream) {
  using namespace hhl;
  if (n == nullptr || x_dev == nullptr || t_dev == nullptr || loss_dev == nullptr || rows < 1 || !(lr > 0.f))
    return fail(HHL_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  hhl_status s = mlp_grad(n, x_dev, t_dev, rows, loss_dev, st);
  if (s != HHL_OK) return s;
  n->step += 1;
  const float b1c = 1.f - powf(0.9f, (float)n->step), b2c = 1.f - powf(0.999f, (float)n->step);
  HHL_PROF_BEGIN(st);
  k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(n->p, n->m, n->v, n->g, n->wb, lr, b1c, b2c);
  HHL_LAUNCH_CHECK("k_mlp_adam");
  return HHL_OK;
}

}  // extern "C"
