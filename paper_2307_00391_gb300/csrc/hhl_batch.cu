// Batched HHL: many instances of uneven size (system register n_s, clock n_c, right-hand
// side, T0), complex64 amplitudes, run as one CUDA graph.
//
// Each instance runs the postselected solve of the single-plan path (hhl_solve_postselected:
// QPE by doubling from the prepared clock = 0 row, the clock block with the anc = 0 weights
// summed, the uncompute and final Hadamards folded by halving into one row). What changes is
// how the controlled products get their operands: a batch of a few hundred instances cannot
// hold every U_k (at N = 4096 the split-FP16 operands of one instance alone are ~6.4 GB), so
// every U_k comes from the eigen-decomposition of the Toeplitz tridiagonal A. With
// v_j(i) = sqrt(2/(N+1)) sin(i j pi/(N+1)), the product formula
// sin a sin b = (cos(a-b) - cos(a+b))/2 turns U_k = V diag(e^{i lambdahat_j t_k}) V^T into
//     U_k[n][m] = g_k(|n - m|) - g_k(n + m)   (1-based n, m),
//     g_k(d) = 1/(N+1) sum_{j=1..N} cos(d j pi/(N+1)) e^{i lambdahat_j t_k}.
// The g_k of every instance (2N+2 values per k, O(N^2) FP64 work each, kept as double-float
// pairs: n_c (2N+2) x 16 bytes per instance) depend on A, T0 and k only, so one FP64 kernel
// computes them when the batch is created, as a plan computes its U_k. The tree steps on
// fewer than 128 rows generate U_k on the fly from g_k (k_toeplitz_rows); the larger ones get
// their GEMM operand (the split-FP16 real embedding for the tensor-core GEMM, or the complex64
// matrix for the CUDA-core GEMM) from one expansion kernel into a per-stream workspace right
// before it is used.
//
// Instances are spread over worker streams by decreasing GEMM work (longest processing
// time first); every stream owns a workspace sized for its largest instance. The whole
// batch (every instance's solve, from the preparation of its right-hand side to its
// dissipation) is captured once into a graph, forked over the worker streams, and replayed
// with one launch per run. The GEMM implementation of each instance (CUDA cores, or tcgen05
// with 128- or 256-column tiles) is given by the caller (an autotuned table) or by a size rule.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include <cuda_fp16.h>

#include "hhl_common.cuh"

namespace hhl {
namespace {

constexpr double kPiB = 3.14159265358979323846;

// g_k(d) for d in [0, 2N+2) and every k: block (x = d chunk, y = k).
__global__ void __launch_bounds__(256) k_ugen_g(int N, const double2* __restrict__ ph /* n_c x N */,
                                               const double* __restrict__ cos_tab /* 2N+2 */,
                                               float4* __restrict__ g /* n_c x (2N+2) */) {
  extern __shared__ double2 sh_ph[];
  const int k = blockIdx.y;
  const int M = 2 * N + 2;
  for (int j = threadIdx.x; j < N; j += blockDim.x) sh_ph[j] = ph[(size_t)k * N + j];
  __syncthreads();
  const double inv = 1.0 / (double)(N + 1);
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < M; d += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    int q = 0;  // (d * j) mod M, j = 1..N
    for (int j = 1; j <= N; ++j) {
      q += d;
      if (q >= M) q -= M;
      const double c = cos_tab[q];
      const double2 p = sh_ph[j - 1];
      re = fma(c, p.x, re);
      im = fma(c, p.y, im);
    }
    // double-float (hi + lo) in FP32, so that the expansion below runs in FP32 arithmetic
    const double gr = re * inv, gi = im * inv;
    const float rh = (float)gr, ih = (float)gi;
    g[(size_t)k * M + d] = make_float4(rh, (float)(gr - (double)rh), ih, (float)(gi - (double)ih));
  }
}

// v (scaled by 2^15) -> FP16 hi = nearest(v), lo = nearest(v - hi), as the tcgen05 GEMM expects.
__device__ __forceinline__ void f16_split(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__device__ __forceinline__ float2 u_elem(const float4* __restrict__ g, int n, int m) { return toeplitz_u(g, n, m); }

// Split-FP16 real embedding of U_k (adjoint: U_k^dagger = conj(U_k), A real symmetric),
// scaled by 2^15: hi / lo (2N x 2N), rows = output real column, columns = input real index.
// One thread per (n, m) writes the 2 x 2 block [[Re, -Im], [Im, Re]] at rows 2n, 2n+1 and
// columns 2m, 2m+1.
__global__ void k_ugen_embed_tc(int n_s, const float4* __restrict__ g, int adjoint, __half* __restrict__ hi,
                                __half* __restrict__ lo) {
  const int N = 1 << n_s;
  const int64_t N2 = 2LL * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e >> n_s), m = (int)(e & (N - 1));
    float2 u = u_elem(g, n, m);
    if (adjoint) u.y = -u.y;
    __half hr, hi_, lr, li;
    f16_split(u.x * 32768.0f, hr, lr);
    f16_split(u.y * 32768.0f, hi_, li);
    const __half nhi = __hneg(hi_), nli = __hneg(li);
    const int64_t r0 = (2LL * n) * N2 + 2LL * m, r1 = r0 + N2;
    *reinterpret_cast<uint32_t*>(hi + r0) = pack_h2(hr, nhi);
    *reinterpret_cast<uint32_t*>(hi + r1) = pack_h2(hi_, hr);
    *reinterpret_cast<uint32_t*>(lo + r0) = pack_h2(lr, nli);
    *reinterpret_cast<uint32_t*>(lo + r1) = pack_h2(li, lr);
  }
}

// Complex64 operand of the CUDA-core GEMM: B[m][n] = U_k[n][m] (= U_k[m][n]) or conj.
__global__ void k_ugen_embed_simt(int n_s, const float4* __restrict__ g, int adjoint, float2* __restrict__ B) {
  const int N = 1 << n_s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)N * N;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(e >> n_s), n = (int)(e & (N - 1));
    float2 u = u_elem(g, n, m);
    if (adjoint) u.y = -u.y;
    B[e] = u;
  }
}

struct Work {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  int64_t capN = 0, cap_msub = 0;
  void* ubuf = nullptr;    // operand: tc hi|lo (2 x 4N^2 FP16) or simt (N^2 complex64)
  __half* a_hi = nullptr;  // tc split rows (M_sub x 2N FP16)
  __half* a_lo = nullptr;
  void* scratch = nullptr; // simt GEMM output rows (M_sub x N complex64)
  TcWork tcw;              // none: the batch's GEMMs run one CTA per tile (no split tiles)
};

int gemm_rule(int n_s, int n_c) {
  if (n_c < 8 || n_s < 6) return 0;
  return n_s == 6 ? 128 : 256;
}

}  // namespace
}  // namespace hhl

using hhl::Plan;
using hhl::fail;

struct hhl_batch_s {
  int count = 0;
  std::vector<Plan> plans;
  std::vector<int> gemm;       // 0 SIMT, 128 / 256 tcgen05 tile width
  std::vector<int> stream_of;
  std::vector<size_t> state_off, b_off, out_off, ph_off, cos_off, g_off, rot_off;
  std::vector<CUtensorMap> maps;  // 4 per instance (tc): A_hi, A_lo, B_hi, B_lo
  std::vector<hhl::Work> work;
  void* arena = nullptr;       // all states
  double* d_b = nullptr;       // packed complex128 right-hand sides
  double* d_out = nullptr;     // packed [4 + 2N] measurement blocks
  double* d_eps = nullptr;     // count
  double* d_scal = nullptr;    // 16 per instance
  void* d_bs = nullptr;        // packed N complex64 per instance
  void* d_rot = nullptr;       // packed R complex64 (cos, sin) per instance
  double2* d_ph = nullptr;     // packed n_c x N phases per instance
  double* d_cos = nullptr;     // packed 2N+2 cosines per instance
  float4* d_g = nullptr;       // packed n_c x (2N+2) per instance (double-float)
  int* d_err = nullptr;
  size_t state_bytes = 0, work_bytes = 0;
  double gemm_flops = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t graph_launches = 0;
  std::vector<double> host_b;  // staging for hhl_batch_run_host
};

namespace hhl {
namespace {

void free_batch(hhl_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto& w : b->work) {
    if (w.ubuf) cudaFree(w.ubuf);
    if (w.a_hi) cudaFree(w.a_hi);
    if (w.a_lo) cudaFree(w.a_lo);
    if (w.scratch) cudaFree(w.scratch);
    if (w.done) cudaEventDestroy(w.done);
    if (w.s) cudaStreamDestroy(w.s);
  }
  void* ptrs[] = {b->arena, b->d_b, b->d_out, b->d_eps, b->d_scal, b->d_bs, b->d_rot, b->d_ph, b->d_cos, b->d_g, b->d_err};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete b;
}

// Enqueue the whole circuit of instance i on its worker stream.
hhl_status enqueue_instance(hhl_batch_s* B, int i) {
  Plan& p = B->plans[i];
  Work& w = B->work[B->stream_of[i]];
  cudaStream_t st = w.s;
  void* state = (char*)B->arena + B->state_off[i];
  char* s0 = (char*)state;
  char* s1 = s0 + (size_t)(p.R * p.N) * 8;
  const double* b = B->d_b + B->b_off[i];
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal, 0, 16 * sizeof(double), st));
  hhl_status s = launch_bnorm(b, p.N, p.d_scal, st);
  // the postselected solve (the same circuit rearranged for its prepared input; see
  // hhl_solve_postselected): only the clock = 0 row of the anc = 0 half is prepared
  if (s == HHL_OK) s = launch_prep_row(p, b, state, st);
  if (s != HHL_OK) return s;
  const int M = (int)(2 * p.N + 2);
  // tree step k: expansion (rows [2^k, 2^(k+1)) = U_k rows [0, 2^k), anc = 0 half) or
  // reduction (rows [0, 2^k) += U_k^dagger rows [2^k, 2^(k+1)), anc = 1 half, the last step
  // scaled by 2^(-n_c/2)), on tcgen05 where the instance has tiles and 2^k >= 128 rows
  auto step = [&](int k, bool reduce) -> hhl_status {
    const float4* gk = B->d_g + B->g_off[i] + (size_t)k * M;
    const int64_t N2 = 2 * p.N;
    const int64_t m = 1LL << k;
    RowMap rows;
    rows.in_off = reduce ? m : 0;
    rows.out_off = reduce ? 0 : m;
    rows.accumulate = reduce ? 1 : 0;
    if (reduce && k == 0) rows.scale = 1.0 / sqrt((double)p.R);
    void* half = reduce ? (void*)s1 : (void*)s0;
    const int g = (int)std::min<int64_t>((p.N * p.N + 255) / 256, 152 * 16);
    if (m < toeplitz_rows_limit())  // few rows: U_k generated on the fly, no N x N operand
      return launch_toeplitz_rows((float2*)half, p.n_s, gk, reduce ? 1 : 0, rows, m, st);
    if (B->gemm[i] == 0 || rows.scale != 1.0) {
      HHL_PROF_BEGIN(st);
      k_ugen_embed_simt<<<g, 256, 0, st>>>(p.n_s, gk, reduce ? 1 : 0, (float2*)w.ubuf);
      HHL_LAUNCH_CHECK("k_ugen_embed_simt");
      return launch_ctrl_u_simt_map(p, half, rows, m, w.ubuf, st);
    }
    __half* hi = (__half*)w.ubuf;
    __half* lo = hi + N2 * N2;
    HHL_PROF_BEGIN(st);
    k_ugen_embed_tc<<<g, 256, 0, st>>>(p.n_s, gk, reduce ? 1 : 0, hi, lo);
    HHL_LAUNCH_CHECK("k_ugen_embed_tc");
    const CUtensorMap* mp = &B->maps[(size_t)i * 4];
    return launch_tc_gemm_map(p.n_s, m, rows, half, w.a_hi, w.a_lo, mp[0], mp[1], mp[2], mp[3], B->gemm[i], B->d_err, w.tcw, 0,
                              st);
  };
  for (int k = 0; k < p.n_c && s == HHL_OK; ++k) s = step(k, false);
  if (s == HHL_OK) s = launch_clock_block(p, state, st);
  if (s == HHL_OK) s = launch_measure_sums(p, state, st);  // |S0|^2, |S1|^2 before the reduction
  for (int k = p.n_c - 1; k >= 0 && s == HHL_OK; --k) s = step(k, true);
  if (s == HHL_OK) s = launch_measure_row(p, state, B->d_out + B->out_off[i], st);
  if (s == HHL_OK) s = launch_dissipation(p, state, B->d_eps + i, nullptr, st);
  return s;
}

hhl_status capture(hhl_batch_s* B, cudaStream_t origin) {
  if (B->exec) return HHL_OK;
  cudaStream_t cap = nullptr;
  HHL_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaEvent_t fork = nullptr;
  HHL_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  const uint64_t l0 = g_launches.load();
  hhl_status s = HHL_OK;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  // every replay starts with a clear GEMM error flag (a memset node ahead of the fork)
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_err, 0, sizeof(int), cap);
  if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
  for (auto& w : B->work)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.s, fork, 0);
  std::vector<int> order(B->count);
  std::iota(order.begin(), order.end(), 0);
  for (int i : order)
    if (e == cudaSuccess && s == HHL_OK) s = enqueue_instance(B, i);
  for (auto& w : B->work) {
    if (e == cudaSuccess) e = cudaEventRecord(w.done, w.s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, w.done, 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  cudaEventDestroy(fork);
  cudaStreamDestroy(cap);
  if (s != HHL_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "batch capture");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  B->graph = graph;
  HHL_CUDA_TRY(cudaGraphInstantiate(&B->exec, graph, 0));
  B->graph_launches = g_launches.load() - l0;
  (void)origin;
  return HHL_OK;
}

}  // namespace
}  // namespace hhl

extern "C" {

hhl_status hhl_batch_create(const hhl_problem* probs, const hhl_params* params, int32_t count,
                            const int32_t* gemm_choice, int32_t streams, hhl_batch_t* out) {
  using namespace hhl;
  if (out == nullptr || probs == nullptr || params == nullptr || count < 1) return fail(HHL_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  if (streams < 1) streams = 8;
  hhl_batch_s* B = new hhl_batch_s();
  B->count = count;
  B->plans.resize(count);
  B->gemm.resize(count);
  B->stream_of.resize(count);
  std::vector<std::vector<double>> lam(count);
  for (int i = 0; i < count; ++i) {
    const hhl_problem& pr = probs[i];
    const hhl_params& pa = params[i];
    if (pa.precision != HHL_PREC_C64 || pa.expm_mode != HHL_EXPM_DENSE || pa.full_uncompute) {
      free_batch(B);
      return fail(HHL_ERR_UNSUPPORTED, "batch instances are complex64, dense, postselect-early");
    }
    if (pr.kind != HHL_MATRIX_TRIDIAG || pr.n_sys_qubits < 1) {
      free_batch(B);
      return fail(HHL_ERR_UNSUPPORTED, "batch instances need a tridiagonal A");
    }
    const int64_t N = 1LL << pr.n_sys_qubits;
    for (int64_t j = 1; j < N; ++j)
      if (pr.diag[j] != pr.diag[0] || (j + 1 < N && pr.off[j] != pr.off[0])) {
        free_batch(B);
        return fail(HHL_ERR_UNSUPPORTED, "batch instances need a Toeplitz tridiagonal A (just-in-time U_k)");
      }
    hhl_status s = plan_scalars(&pr, &pa, B->plans[i], &lam[i]);
    if (s != HHL_OK) {
      free_batch(B);
      return s;
    }
    Plan& p = B->plans[i];
    const int rule = gemm_rule(p.n_s, p.n_c);
    int gsel = gemm_choice ? gemm_choice[i] : -1;
    if (gsel != 0 && gsel != 128 && gsel != 256) gsel = rule;
    if (gsel != 0 && (p.R / 2 < 128 || 2 * p.N < gsel)) gsel = 0;  // tile does not fit
    B->gemm[i] = gsel;
    p.gemm_impl = gsel ? HHL_GEMM_TCGEN05 : HHL_GEMM_SIMT;
    // the two trees: sum over k of 2^k rows each (expansion and reduction)
    B->gemm_flops += 2.0 * 8.0 * (double)(p.R - 1) * (double)p.N * (double)p.N;
  }
  // LPT assignment of instances to worker streams by GEMM work
  streams = std::min(streams, count);
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  // work of an instance: the GEMM rows of its two trees (2^n_c) and its 2 n_c operand
  // generations, each over N^2 entries
  auto cost = [&](int i) {
    const Plan& q = B->plans[i];
    return (double)(q.R + 2 * q.n_c) * (double)q.N * (double)q.N + 1.0;
  };
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<double> load(streams, 0.0);
  B->work.resize(streams);
  for (int i : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += cost(i);
    B->stream_of[i] = w;
    B->work[w].capN = std::max<int64_t>(B->work[w].capN, B->plans[i].N);
    B->work[w].cap_msub = std::max<int64_t>(B->work[w].cap_msub, B->plans[i].R / 2);
  }
  // offsets
  size_t so = 0, bo = 0, oo = 0, po = 0, co = 0, go = 0, ro = 0;
  B->state_off.resize(count); B->b_off.resize(count); B->out_off.resize(count); B->ph_off.resize(count);
  B->cos_off.resize(count); B->g_off.resize(count); B->rot_off.resize(count);
  for (int i = 0; i < count; ++i) {
    const Plan& p = B->plans[i];
    B->state_off[i] = so; so += (size_t)(2 * p.R * p.N) * 8;
    B->b_off[i] = bo;     bo += (size_t)2 * p.N;
    B->out_off[i] = oo;   oo += (size_t)(4 + 2 * p.N);
    B->ph_off[i] = po;    po += (size_t)p.n_c * p.N;
    B->cos_off[i] = co;   co += (size_t)(2 * p.N + 2);
    B->g_off[i] = go;     go += (size_t)p.n_c * (2 * p.N + 2);
    B->rot_off[i] = ro;   ro += (size_t)p.R;
  }
  B->state_bytes = so;
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return false;
    }
    return true;
  };
  bool ok = alloc(&B->arena, so) && alloc((void**)&B->d_b, bo * sizeof(double)) &&
            alloc((void**)&B->d_out, oo * sizeof(double)) && alloc((void**)&B->d_eps, count * sizeof(double)) &&
            alloc((void**)&B->d_scal, (size_t)count * 16 * sizeof(double)) &&
            alloc(&B->d_bs, (bo / 2) * sizeof(float2)) && alloc(&B->d_rot, ro * sizeof(float2)) &&
            alloc((void**)&B->d_ph, po * sizeof(double2)) && alloc((void**)&B->d_cos, co * sizeof(double)) &&
            alloc((void**)&B->d_g, go * sizeof(float4)) && alloc((void**)&B->d_err, sizeof(int));
  for (auto& w : B->work) {
    if (!ok) break;
    const int64_t N2 = 2 * w.capN;
    // ubuf holds the FP16 hi|lo embedding (2 x 4 N^2 x 2 bytes) or the complex64 SIMT operand
    // (N^2 x 8 bytes), whichever the instances of this stream need (16 N^2 bytes cover both)
    ok = alloc(&w.ubuf, (size_t)2 * N2 * N2 * sizeof(__half)) && alloc((void**)&w.a_hi, (size_t)w.cap_msub * N2 * 2) &&
         alloc((void**)&w.a_lo, (size_t)w.cap_msub * N2 * 2) && alloc(&w.scratch, (size_t)w.cap_msub * w.capN * 8);
    B->work_bytes += (size_t)2 * N2 * N2 * 2 + 2 * (size_t)w.cap_msub * N2 * 2 + (size_t)w.cap_msub * w.capN * 8;
    if (ok) ok = cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    free_batch(B);
    return fail(HHL_ERR_OOM, "batch device allocation failed");
  }
  // host tables: phases e^{i lambdahat_j t_k}, cosines cos(q pi/(N+1)), rotation (cos, sin)(theta_y/2)
  std::vector<double2> ph;
  std::vector<double> cs;
  std::vector<float2> rot;
  for (int i = 0; i < count; ++i) {
    Plan& p = B->plans[i];
    ph.resize((size_t)p.n_c * p.N);
    for (int k = 0; k < p.n_c; ++k) {
      const double t = p.t0 * (double)(1LL << k) / (double)p.R;
      for (int64_t j = 0; j < p.N; ++j) {
        const double a = lam[i][j] / p.lam_ub * t;
        ph[(size_t)k * p.N + j] = make_double2(cos(a), sin(a));
      }
    }
    cs.resize(2 * p.N + 2);
    for (int64_t q = 0; q < 2 * p.N + 2; ++q) cs[q] = cos((double)q * kPiB / (double)(p.N + 1));
    rot.resize(p.R);
    for (int64_t y = 0; y < p.R; ++y) rot[y] = make_float2((float)cos(p.theta[y] / 2), (float)sin(p.theta[y] / 2));
    cudaMemcpy(B->d_ph + B->ph_off[i], ph.data(), ph.size() * sizeof(double2), cudaMemcpyHostToDevice);
    cudaMemcpy(B->d_cos + B->cos_off[i], cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy((float2*)B->d_rot + B->rot_off[i], rot.data(), rot.size() * sizeof(float2), cudaMemcpyHostToDevice);
    // device pointers of the per-instance plan view
    Work& w = B->work[B->stream_of[i]];
    p.d_scal = B->d_scal + (size_t)16 * i;
    p.d_bs = (float2*)B->d_bs + B->b_off[i] / 2;
    p.d_rot = (float2*)B->d_rot + B->rot_off[i];
    p.d_scratch = w.scratch;
    if (B->gemm[i]) {
      CUtensorMap m4[4];
      const int64_t N2 = 2 * p.N;
      hhl_status s = tc_make_map(&m4[0], w.a_hi, N2, p.R / 2, 128);
      if (s == HHL_OK) s = tc_make_map(&m4[1], w.a_lo, N2, p.R / 2, 128);
      if (s == HHL_OK) s = tc_make_map(&m4[2], (__half*)w.ubuf, N2, N2, B->gemm[i]);
      if (s == HHL_OK) s = tc_make_map(&m4[3], (__half*)w.ubuf + N2 * N2, N2, N2, B->gemm[i]);
      if (s != HHL_OK) {
        free_batch(B);
        return s;
      }
      B->maps.insert(B->maps.end(), m4, m4 + 4);
    } else {
      B->maps.insert(B->maps.end(), 4, CUtensorMap{});
    }
  }
  hhl_status s = HHL_OK;
  if (cudaError_t me = cudaMemset(B->d_err, 0, sizeof(int)); me != cudaSuccess) s = cuda_fail(me, "cudaMemset(error flag)");
  if (s == HHL_OK) s = tc_init_kernels();
  if (s == HHL_OK) {
    int64_t maxN = 0;
    for (const Plan& p : B->plans) maxN = std::max<int64_t>(maxN, p.N);
    cudaError_t e = cudaFuncSetAttribute(k_ugen_g, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max<int64_t>(maxN * (int64_t)sizeof(double2), 1024));
    if (e != cudaSuccess) s = cuda_fail(e, "cudaFuncSetAttribute(k_ugen_g)");
  }
  // g_k for every k of every instance, once (they depend on A, T0 and k only)
  for (int i = 0; i < count && s == HHL_OK; ++i) {
    const Plan& p = B->plans[i];
    const int M = (int)(2 * p.N + 2);
    dim3 grid((unsigned)((M + 255) / 256), (unsigned)p.n_c);
    k_ugen_g<<<grid, 256, p.N * sizeof(double2), B->work[B->stream_of[i]].s>>>(
        (int)p.N, B->d_ph + B->ph_off[i], B->d_cos + B->cos_off[i], B->d_g + B->g_off[i]);
    if (cudaError_t le = cudaGetLastError(); le != cudaSuccess) s = cuda_fail(le, "k_ugen_g");
  }
  if (s == HHL_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) s = cuda_fail(e, "batch setup");
  }
  if (s != HHL_OK) {
    free_batch(B);
    return s;
  }
  *out = B;
  return HHL_OK;
}

hhl_status hhl_batch_plan(const hhl_problem* probs, const hhl_params* params, int32_t count, hhl_batch_t* out) {
  return hhl_batch_create(probs, params, count, nullptr, 8, out);
}

void hhl_batch_destroy(hhl_batch_t b) { hhl::free_batch(b); }

hhl_status hhl_batch_get_info(hhl_batch_t b, hhl_batch_info* info) {
  if (b == nullptr || info == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL batch or info");
  memset(info, 0, sizeof(*info));
  info->count = b->count;
  info->streams = (int32_t)b->work.size();
  info->state_bytes = b->state_bytes;
  info->workspace_bytes = b->work_bytes;
  info->gemm_flops = b->gemm_flops;
  info->graph_launches = b->graph_launches;
  info->b_doubles = 0;
  info->out_doubles = 0;
  for (int i = 0; i < b->count; ++i) {
    info->b_doubles += 2 * b->plans[i].N;
    info->out_doubles += 4 + 2 * b->plans[i].N;
  }
  return HHL_OK;
}

hhl_status hhl_batch_instance(hhl_batch_t b, int32_t i, int32_t* n_sys_qubits, int32_t* n_clock, int32_t* gemm,
                              int64_t* b_offset, int64_t* out_offset, double* t0) {
  if (b == nullptr || i < 0 || i >= b->count) return fail(HHL_ERR_INVALID_ARG, "bad batch or index");
  if (n_sys_qubits) *n_sys_qubits = b->plans[i].n_s;
  if (n_clock) *n_clock = b->plans[i].n_c;
  if (gemm) *gemm = b->gemm[i];
  if (b_offset) *b_offset = (int64_t)b->b_off[i];
  if (out_offset) *out_offset = (int64_t)b->out_off[i];
  if (t0) *t0 = b->plans[i].t0;
  return HHL_OK;
}

hhl_status hhl_batch_run(hhl_batch_t b, const double* b_dev, double* out_dev, double* eps_dev, void* stream) {
  using namespace hhl;
  if (b == nullptr || b_dev == nullptr || out_dev == nullptr || eps_dev == nullptr)
    return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t bo = 0, oo = 0;
  for (int i = 0; i < b->count; ++i) {
    bo += 2 * b->plans[i].N;
    oo += 4 + 2 * b->plans[i].N;
  }
  hhl_status s = capture(b, st);
  if (s != HHL_OK) return s;
  HHL_CUDA_TRY(cudaMemcpyAsync(b->d_b, b_dev, bo * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HHL_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  g_launches.fetch_add(b->graph_launches, std::memory_order_relaxed);
  HHL_CUDA_TRY(cudaMemcpyAsync(out_dev, b->d_out, oo * sizeof(double), cudaMemcpyDeviceToDevice, st));
  HHL_CUDA_TRY(cudaMemcpyAsync(eps_dev, b->d_eps, b->count * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return HHL_OK;
}

hhl_status hhl_batch_run_eager(hhl_batch_t b, void* stream) {
  using namespace hhl;
  if (b == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL batch");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t fork = nullptr;
  HHL_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  HHL_CUDA_TRY(cudaMemsetAsync(b->d_err, 0, sizeof(int), st));
  HHL_CUDA_TRY(cudaEventRecord(fork, st));
  for (auto& w : b->work) HHL_CUDA_TRY(cudaStreamWaitEvent(w.s, fork, 0));
  hhl_status s = HHL_OK;
  for (int i = 0; i < b->count && s == HHL_OK; ++i) s = enqueue_instance(b, i);
  for (auto& w : b->work) {
    HHL_CUDA_TRY(cudaEventRecord(w.done, w.s));
    HHL_CUDA_TRY(cudaStreamWaitEvent(st, w.done, 0));
  }
  cudaEventDestroy(fork);
  return s;
}

hhl_status hhl_batch_run_host(hhl_batch_t b, const double* b_host, double* out_host, double* eps_host, void* stream) {
  using namespace hhl;
  if (b == nullptr || b_host == nullptr || out_host == nullptr || eps_host == nullptr)
    return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  size_t bo = 0, oo = 0;
  for (int i = 0; i < b->count; ++i) {
    bo += 2 * b->plans[i].N;
    oo += 4 + 2 * b->plans[i].N;
  }
  hhl_status s = capture(b, st);
  if (s != HHL_OK) return s;
  HHL_CUDA_TRY(cudaMemcpyAsync(b->d_b, b_host, bo * sizeof(double), cudaMemcpyHostToDevice, st));
  HHL_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  g_launches.fetch_add(b->graph_launches, std::memory_order_relaxed);
  HHL_CUDA_TRY(cudaMemcpyAsync(out_host, b->d_out, oo * sizeof(double), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaMemcpyAsync(eps_host, b->d_eps, b->count * sizeof(double), cudaMemcpyDeviceToHost, st));
  return hhl_batch_status(b, stream);
}

hhl_status hhl_batch_status(hhl_batch_t b, void* stream) {
  using namespace hhl;
  if (b == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL batch");
  cudaStream_t st = (cudaStream_t)stream;
  int err = 0;
  HHL_CUDA_TRY(cudaMemcpyAsync(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  return tc_flag_status(err);
}

}  // extern "C"
