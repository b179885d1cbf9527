// hhl_controlled_u_noalloc: one clock-controlled U on complex64 rows, with no device
// allocation at call time.
//
// Who needs it: callers that must not allocate device memory once they are running. A host
// that hands all device memory to its own pool allocator cannot let a library call
// cudaMalloc behind the pool's back, and a latency-bound loop cannot afford the implicit
// device synchronisation that cudaMalloc and cudaFree may cause. Such callers still own
// their inputs and outputs; what this entry point takes off them is the library's own
// scratch buffer.
//
// How: the product rows are staged in a fixed, file-scope device array (kMaxScratchAmps
// complex64 values = 8 MiB, held on every GPU that loads the library until the process
// exits). Host code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it together with the unique id of the CUDA context it belongs to; that first
// call should therefore come before any stream capture. A device reset (cudaDeviceReset by
// the caller or by another library) ends that context: the next call sees a new context id
// and looks the address up again instead of writing through a stale one. Every
// call overwrites the part of the array it uses before reading it, so no state is carried
// from one call to the next, but all calls share the one array: calls whose kernels may
// overlap on the GPU (different streams without ordering between them) race on it.
#include <cuda.h>

#include <mutex>

#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int64_t kMaxScratchAmps = 1LL << 20;  // 8 MiB of complex64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kMaxScratchAmps];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kMaxDevices] = {0};  // context id each cached address belongs to

__device__ __forceinline__ int64_t row_with_bit_na(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}

// out[i][n] = sum_m U'[n][m] * S[row(i)][m], U' = U or U^dagger (read from U directly).
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_ctrl_gemm_noalloc(const float2* __restrict__ S, float2* __restrict__ out,
                                                           const float2* __restrict__ U, int n_s, int k,
                                                           int64_t m_sub, int adjoint) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ float2 As[BK][BM + 1];
  __shared__ float2 Bs[BK][BN];
  const int64_t N = 1LL << n_s;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  float accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TN; ++c) { accr[a][c] = 0.f; acci[a][c] = 0.f; }
  for (int64_t m0 = 0; m0 < N; m0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const int64_t i = i0 + r, m = m0 + kk;
      As[kk][r] = (i < m_sub && m < N) ? S[row_with_bit_na(i, k) * N + m] : make_float2(0.f, 0.f);
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int kk = e / BN, c = e % BN;
      const int64_t m = m0 + kk, n = n0 + c;
      float2 v = make_float2(0.f, 0.f);
      if (m < N && n < N) {
        if (adjoint) {
          const float2 u = U[m * N + n];  // (U^dagger)[n][m] = conj(U[m][n])
          v = make_float2(u.x, -u.y);
        } else {
          v = U[n * N + m];
        }
      }
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float2 a[TM], b[TN];
#pragma unroll
      for (int x = 0; x < TM; ++x) a[x] = As[kk][ty + 16 * x];
#pragma unroll
      for (int y = 0; y < TN; ++y) b[y] = Bs[kk][tx + 16 * y];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) {
          accr[x][y] = fmaf(a[x].x, b[y].x, accr[x][y]);
          accr[x][y] = fmaf(-a[x].y, b[y].y, accr[x][y]);
          acci[x][y] = fmaf(a[x].x, b[y].y, acci[x][y]);
          acci[x][y] = fmaf(a[x].y, b[y].x, acci[x][y]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int64_t i = i0 + ty + 16 * x;
    if (i >= m_sub) continue;
#pragma unroll
    for (int y = 0; y < TN; ++y) {
      const int64_t n = n0 + tx + 16 * y;
      if (n < N) out[i * N + n] = make_float2(accr[x][y], acci[x][y]);
    }
  }
}

__global__ void k_rows_scatter_noalloc(float2* __restrict__ S, const float2* __restrict__ out, int n_s, int k,
                                       int64_t m_sub) {
  const int64_t N = 1LL << n_s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m_sub * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e >> n_s, m = e & (N - 1);
    S[row_with_bit_na(i, k) * N + m] = out[e];
  }
}

// Unique id of the current CUDA context (cuCtxGetId: never reused within a process), 0 when
// the driver does not provide it (the cache is then per device only).
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (GetCurrent)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (GetId)p;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device, looked up once per device and
// context.
hhl_status scratch_address(void** out) {
  int dev = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(HHL_ERR_UNSUPPORTED, "device ordinal beyond the scratch table");
  // (before the runtime has made a context current on this thread the id reads 0, and the
  // next call looks the address up once more: harmless, the address is the same)
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_ptr[dev];
  return HHL_OK;
}

}  // namespace

}  // namespace hhl

extern "C" hhl_status hhl_controlled_u_noalloc(const void* u_dev, void* half_dev, int32_t n_sys_qubits,
                                               int32_t n_clock, int32_t k, int32_t adjoint, void* stream) {
  using namespace hhl;
  if (u_dev == nullptr || half_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL matrix or state");
  if (n_sys_qubits < 1 || n_sys_qubits > 12 || n_clock < 1 || n_clock > 16 || k < 0 || k >= n_clock)
    return fail(HHL_ERR_INVALID_ARG, "need 1 <= n_sys_qubits <= 12, 1 <= n_clock <= 16, 0 <= k < n_clock");
  const int64_t N = 1LL << n_sys_qubits;
  const int64_t m_sub = (1LL << n_clock) / 2;
  if (m_sub * N > kMaxScratchAmps)
    return fail(HHL_ERR_INVALID_ARG, "needs " + std::to_string(m_sub * N) + " complex64 scratch values (2^(n_clock-1) * 2^n_sys_qubits); the fixed limit is " +
                                         std::to_string(kMaxScratchAmps) + " (8 MiB)");
  void* scratch = nullptr;
  hhl_status s = scratch_address(&scratch);
  if (s != HHL_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((m_sub + 63) / 64));
  HHL_PROF_BEGIN(st);
  k_ctrl_gemm_noalloc<64, 64, 16><<<grid, 256, 0, st>>>((const float2*)half_dev, (float2*)scratch, (const float2*)u_dev,
                                                        n_sys_qubits, k, m_sub, adjoint ? 1 : 0);
  HHL_LAUNCH_CHECK("k_ctrl_gemm_noalloc");
  int64_t g = (m_sub * N + 255) / 256;
  if (g > 152 * 32) g = 152 * 32;
  HHL_PROF_BEGIN(st);
  k_rows_scatter_noalloc<<<(unsigned)g, 256, 0, st>>>((float2*)half_dev, (const float2*)scratch, n_sys_qubits, k, m_sub);
  HHL_LAUNCH_CHECK("k_rows_scatter_noalloc");
  return HHL_OK;
}
