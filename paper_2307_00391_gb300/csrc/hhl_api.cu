// Host side of the C ABI: validation, the FP64 planner (a0), and the entry points that
// sequence the kernels on the caller's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "hhl_common.cuh"

namespace hhl {

std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_prof_on{false};
static thread_local std::string t_last_error;

// ------------------------------------------------------------------ per-kernel timing
namespace {
struct ProfPending {
  cudaEvent_t a, b;
  std::string name;
};
struct ProfAgg {
  uint64_t launches = 0;
  double ms = 0.0;
};
std::mutex g_prof_mu;
std::vector<ProfPending> g_prof_pending;
std::vector<cudaEvent_t> g_event_pool;
std::map<std::string, ProfAgg> g_prof_agg;
thread_local cudaEvent_t t_begin_ev = nullptr;
thread_local cudaStream_t t_begin_st = nullptr;

cudaEvent_t pooled_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_resolve() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      ProfAgg& g = g_prof_agg[r.name];
      g.launches += 1;
      g.ms += ms;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof_pending.clear();
}
}  // namespace

void prof_begin(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    t_begin_ev = nullptr;  // launches captured into a graph are timed as a whole by the caller
    return;
  }
  t_begin_ev = pooled_event();
  t_begin_st = st;
  if (t_begin_ev) cudaEventRecord(t_begin_ev, st);
}

void prof_end(const char* name) {
  if (t_begin_ev == nullptr) return;
  cudaEvent_t b = pooled_event();
  if (b == nullptr) return;
  cudaEventRecord(b, t_begin_st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back({t_begin_ev, b, name});
  t_begin_ev = nullptr;
}

// The largest dynamic shared memory set so far per (device, kernel): the attribute is only
// ever raised. Launches of one kernel with different sizes (the instances of a batch, captured
// into one graph) then all stay within the attribute, whichever size was set last.
cudaError_t raise_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set_to;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set_to[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

void set_error(const std::string& msg) { t_last_error = msg; }
hhl_status fail(hhl_status s, const std::string& msg) {
  t_last_error = msg;
  return s;
}
hhl_status cuda_fail(cudaError_t e, const char* what) {
  t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HHL_ERR_OOM : HHL_ERR_CUDA;
}

namespace {

constexpr double kPi = 3.14159265358979323846;

// Host fault injection for testing error paths: HHL_FAULT=alloc|plan|launch.
bool fault(const char* what) {
  const char* f = getenv("HHL_FAULT");
  return f != nullptr && strcmp(f, what) == 0;
}

// Tree steps of the postselected solve on fewer rows than one tcgen05 tile (2^k < 128) run on
// CUDA cores, so tcgen05 plans also keep CUDA-core operands for k < kTreeSimtBits.
constexpr int kTreeSimtBits = 7;

// The GEMM operands of U_k (d_u: N x N complex128 on the device).
hhl_status store_operands_k(Plan& p, const double2* d_u, int k, cudaStream_t st) {
  if (p.gemm_impl == HHL_GEMM_SIMT) return launch_store_operands(p, d_u, k, st);
  hhl_status s = tc_prepare_operands(p, d_u, k, st);
  if (s == HHL_OK && k < kTreeSimtBits && p.d_bfwd != nullptr) s = launch_store_operands(p, d_u, k, st);
  return s;
}

hhl_status dev_alloc(void** p, size_t bytes, uint64_t* counter) {
  if (fault("alloc")) return fail(HHL_ERR_OOM, "injected allocation failure (HHL_FAULT=alloc)");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(HHL_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  if (counter) *counter += bytes;
  return HHL_OK;
}

// Cyclic Jacobi eigen-decomposition of a real symmetric n x n matrix (row-major, destroyed).
// On return w holds the eigenvalues and v (row-major) the eigenvectors as columns.
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = c * vkp - s * vkq;
          v[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[(size_t)i * n + i];
}

// Eigen-data of A for building U_k: vectors (columns) vr/vi (N x J), eigenvalues lam (J),
// and a weight applied to every projector (1/2 for the real embedding of a complex A).
struct Eigen {
  int J = 0;
  std::vector<double> lam, vr, vi;
  double wgt = 1.0;
  bool have_vectors = false;
  bool toeplitz = false;  // analytic sine basis: U_k from the g_k formula, no vectors needed
};

bool is_toeplitz(const double* d, const double* o, int64_t n) {
  for (int64_t i = 1; i < n; ++i)
    if (d[i] != d[0]) return false;
  for (int64_t i = 1; i + 1 < n; ++i)
    if (o[i] != o[0]) return false;
  return true;
}

hhl_status validate(const hhl_problem* pr, const hhl_params* pa) {
  if (pr == nullptr || pa == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL problem or params");
  if (pr->kind != HHL_MATRIX_TRIDIAG && pr->kind != HHL_MATRIX_DENSE && pr->kind != HHL_MATRIX_UNITARY)
    return fail(HHL_ERR_INVALID_ARG, "bad matrix kind");
  if (pa->expm_mode != HHL_EXPM_DENSE && pa->expm_mode != HHL_EXPM_TROTTER) return fail(HHL_ERR_INVALID_ARG, "bad expm_mode");
  if (pa->precision != HHL_PREC_C64 && pa->precision != HHL_PREC_C128) return fail(HHL_ERR_INVALID_ARG, "bad precision");
  if (pa->n_clock < 1 || pa->n_clock > 13) return fail(HHL_ERR_INVALID_ARG, "n_clock must be in 1..13");
  const int max_ns = pa->expm_mode == HHL_EXPM_DENSE ? 12 : 24;
  if (pr->n_sys_qubits < 1 || pr->n_sys_qubits > max_ns)
    return fail(HHL_ERR_INVALID_ARG, "n_sys_qubits out of range (dense <= 12, Trotter <= 24)");
  if (pr->n_sys_qubits + pa->n_clock + 1 > 34) return fail(HHL_ERR_INVALID_ARG, "more than 34 qubits");
  if (pa->t0_rule < HHL_T0_USER || pa->t0_rule > HHL_T0_RANGE_FILL) return fail(HHL_ERR_INVALID_ARG, "bad t0_rule");
  if (pa->t0_rule == HHL_T0_USER && !(pa->t0 > 0.0 && std::isfinite(pa->t0)))
    return fail(HHL_ERR_INVALID_ARG, "HHL_T0_USER needs a finite t0 > 0");
  if (pa->t0_convention != HHL_T0_TOTAL && pa->t0_convention != HHL_T0_PER_UNIT)
    return fail(HHL_ERR_INVALID_ARG, "bad t0_convention");
  if (!(pa->C >= 0.0) || !std::isfinite(pa->C)) return fail(HHL_ERR_INVALID_ARG, "C must be finite and >= 0");
  if (pa->gemm_impl < HHL_GEMM_AUTO || pa->gemm_impl > HHL_GEMM_TCGEN05) return fail(HHL_ERR_INVALID_ARG, "bad gemm_impl");
  if (pa->gemm_impl == HHL_GEMM_TCGEN05 && pa->precision != HHL_PREC_C64)
    return fail(HHL_ERR_UNSUPPORTED, "the tcgen05 GEMM is complex64 only");
  if (pa->expm_mode == HHL_EXPM_TROTTER && !(pa->trotter_dt > 0.0)) return fail(HHL_ERR_INVALID_ARG, "trotter_dt must be > 0");
  if (pa->trotter_steps_max < 0) return fail(HHL_ERR_INVALID_ARG, "trotter_steps_max < 0");
  if (pa->signed_clock != 0 && pa->signed_clock != 1) return fail(HHL_ERR_INVALID_ARG, "signed_clock must be 0 or 1");
  if (pa->signed_clock && pa->n_clock < 2) return fail(HHL_ERR_INVALID_ARG, "a signed clock needs n_clock >= 2");
  if (!std::isfinite(pr->nu) || !std::isfinite(pr->wall_lo) || !std::isfinite(pr->wall_hi))
    return fail(HHL_ERR_INVALID_ARG, "non-finite nu or wall value");
  const int64_t N = 1LL << pr->n_sys_qubits;
  if (pr->kind == HHL_MATRIX_TRIDIAG) {
    if (pr->diag == nullptr || (N > 1 && pr->off == nullptr)) return fail(HHL_ERR_INVALID_ARG, "tridiagonal A needs diag and off");
    for (int64_t i = 0; i < N; ++i)
      if (!std::isfinite(pr->diag[i])) return fail(HHL_ERR_NUMERIC, "non-finite diag entry");
    for (int64_t i = 0; i + 1 < N; ++i)
      if (!std::isfinite(pr->off[i])) return fail(HHL_ERR_NUMERIC, "non-finite off entry");
  } else {
    if (N > 256) return fail(HHL_ERR_UNSUPPORTED, "dense A is limited to N <= 256");
    if (pa->expm_mode == HHL_EXPM_TROTTER) return fail(HHL_ERR_UNSUPPORTED, "Trotter mode needs a tridiagonal A");
    if (pr->dense_re == nullptr) return fail(HHL_ERR_INVALID_ARG, "dense A needs dense_re");
    double amax = 0.0;
    for (int64_t i = 0; i < N * N; ++i) {
      const double im = pr->dense_im ? pr->dense_im[i] : 0.0;
      if (!std::isfinite(pr->dense_re[i]) || !std::isfinite(im)) return fail(HHL_ERR_NUMERIC, "non-finite A entry");
      amax = std::max(amax, std::hypot(pr->dense_re[i], im));
    }
    if (pr->kind == HHL_MATRIX_UNITARY) {
      // Q Q^dagger = I to 1e-10, and a finite angle per clock value
      for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
          double sr = 0.0, si = 0.0;
          for (int64_t k = 0; k < N; ++k) {
            const double ar = pr->dense_re[i * N + k], ai = pr->dense_im ? pr->dense_im[i * N + k] : 0.0;
            const double br = pr->dense_re[j * N + k], bi = pr->dense_im ? -pr->dense_im[j * N + k] : 0.0;
            sr += ar * br - ai * bi;
            si += ar * bi + ai * br;
          }
          if (std::hypot(sr - (i == j ? 1.0 : 0.0), si) > 1e-10) return fail(HHL_ERR_INVALID_ARG, "Q is not unitary");
        }
      if (pa->theta_table == nullptr) return fail(HHL_ERR_INVALID_ARG, "a UNITARY plan needs theta_table");
      for (int64_t y = 0; y < (1LL << pa->n_clock); ++y)
        if (!std::isfinite(pa->theta_table[y])) return fail(HHL_ERR_NUMERIC, "non-finite theta_table entry");
    } else {
      for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
          const double re1 = pr->dense_re[i * N + j], re2 = pr->dense_re[j * N + i];
          const double im1 = pr->dense_im ? pr->dense_im[i * N + j] : 0.0;
          const double im2 = pr->dense_im ? pr->dense_im[j * N + i] : 0.0;
          if (std::hypot(re1 - re2, im1 + im2) > 1e-12 * amax) return fail(HHL_ERR_NOT_HERMITIAN, "A is not Hermitian");
        }
    }
  }
  return HHL_OK;
}

hhl_status eigen_of(const hhl_problem* pr, bool need_vectors, Plan& p, Eigen& eg) {
  const int64_t N = p.N;
  const int n = (int)N;
  if (pr->kind == HHL_MATRIX_TRIDIAG && (N == 1 || is_toeplitz(pr->diag, pr->off, N))) {
    // Toeplitz tridiagonal: lambda_j = d + 2 o cos(j pi/(N+1)), v_j(i) = sqrt(2/(N+1)) sin(i j pi/(N+1)).
    const double d = pr->diag[0], o = N > 1 ? pr->off[0] : 0.0;
    eg.J = n;
    eg.toeplitz = true;
    eg.lam.resize(n);
    for (int j = 1; j <= n; ++j) eg.lam[j - 1] = d + 2.0 * o * cos(j * kPi / (N + 1));
    if (need_vectors) {
      eg.vr.resize((size_t)n * n);
      const double s = sqrt(2.0 / (N + 1));
      for (int i = 1; i <= n; ++i)
        for (int j = 1; j <= n; ++j) eg.vr[(size_t)(i - 1) * n + (j - 1)] = s * sin((double)i * j * kPi / (N + 1));
      eg.have_vectors = true;
    }
    return HHL_OK;
  }
  if (N > 256) return fail(HHL_ERR_UNSUPPORTED, "non-Toeplitz A is limited to N <= 256");
  if (pr->kind == HHL_MATRIX_TRIDIAG || pr->dense_im == nullptr) {
    std::vector<double> a((size_t)n * n, 0.0);
    if (pr->kind == HHL_MATRIX_TRIDIAG) {
      for (int i = 0; i < n; ++i) a[(size_t)i * n + i] = pr->diag[i];
      for (int i = 0; i + 1 < n; ++i) a[(size_t)i * n + i + 1] = a[(size_t)(i + 1) * n + i] = pr->off[i];
    } else {
      for (size_t i = 0; i < (size_t)n * n; ++i) a[i] = pr->dense_re[i];
    }
    jacobi_eigen(n, a, eg.lam, eg.vr);
    eg.J = n;
    eg.have_vectors = true;
    return HHL_OK;
  }
  // Complex Hermitian: the real symmetric embedding [[Re, -Im], [Im, Re]] (2N x 2N) has every
  // eigenvalue of A twice; each real eigenvector [p; q] gives the complex eigenvector p + i q,
  // and the projectors of one pair add up to twice the complex projector (weight 1/2).
  const int m = 2 * n;
  std::vector<double> a((size_t)m * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double re = pr->dense_re[(size_t)i * n + j], im = pr->dense_im[(size_t)i * n + j];
      a[(size_t)i * m + j] = re;
      a[(size_t)i * m + (j + n)] = -im;
      a[(size_t)(i + n) * m + j] = im;
      a[(size_t)(i + n) * m + (j + n)] = re;
    }
  std::vector<double> v;
  jacobi_eigen(m, a, eg.lam, v);
  eg.J = m;
  eg.vr.resize((size_t)n * m);
  eg.vi.resize((size_t)n * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      eg.vr[(size_t)i * m + j] = v[(size_t)i * m + j];
      eg.vi[(size_t)i * m + j] = v[(size_t)(i + n) * m + j];
    }
  eg.wgt = 0.5;
  eg.have_vectors = true;
  return HHL_OK;
}

// Host part of the plan (a0): register sizes, lambda_ub, eigenvalues (and eigenvectors when
// asked), kappa, T0, C and the rotation angles.
hhl_status plan_host(const hhl_problem* prob, const hhl_params* params, Plan& p, Eigen& eg, bool need_vectors) {
  p.n_s = prob->n_sys_qubits;
  p.n_c = params->n_clock;
  p.n = p.n_s + p.n_c + 1;
  p.N = 1LL << p.n_s;
  p.R = 1LL << p.n_c;
  p.prec = params->precision;
  p.expm_mode = params->expm_mode;
  p.full = params->full_uncompute ? 1 : 0;
  p.nu = prob->nu;
  p.wall_lo = prob->wall_lo;
  p.wall_hi = prob->wall_hi;
  p.trotter_dt = params->trotter_dt;
  p.trotter_max = params->trotter_steps_max;
  cudaGetDevice(&p.device);

  // lambda_ub: Gershgorin bound max_i sum_j |A_ij|
  const int64_t N = p.N;
  double lub = 0.0;
  if (prob->kind == HHL_MATRIX_TRIDIAG) {
    for (int64_t i = 0; i < N; ++i) {
      double r = fabs(prob->diag[i]);
      if (i > 0) r += fabs(prob->off[i - 1]);
      if (i + 1 < N) r += fabs(prob->off[i]);
      lub = std::max(lub, r);
    }
  } else {
    for (int64_t i = 0; i < N; ++i) {
      double r = 0.0;
      for (int64_t j = 0; j < N; ++j) r += std::hypot(prob->dense_re[i * N + j], prob->dense_im ? prob->dense_im[i * N + j] : 0.0);
      lub = std::max(lub, r);
    }
  }
  if (!(lub > 0.0)) { return fail(HHL_ERR_SINGULAR, "A is zero"); }
  p.lam_ub = lub;
  if (prob->kind == HHL_MATRIX_UNITARY) {
    // phase estimation of Q itself: no spectrum to plan, the angles are the caller's
    p.lam_ub = 1.0;
    p.lam_min = p.lam_max = p.kappa = 1.0;
    p.t0 = 2.0 * kPi;
    p.C = 1.0;
    p.theta.assign(params->theta_table, params->theta_table + p.R);
    return HHL_OK;
  }

  const bool dense = p.expm_mode == HHL_EXPM_DENSE;
  if (!dense && !(prob->kind == HHL_MATRIX_TRIDIAG && is_toeplitz(prob->diag, prob->off, N)))
    return fail(HHL_ERR_UNSUPPORTED, "Trotter mode needs a Toeplitz tridiagonal A");
  const bool toeplitz_a = prob->kind == HHL_MATRIX_TRIDIAG && (N == 1 || is_toeplitz(prob->diag, prob->off, N));
  hhl_status s = eigen_of(prob, dense && need_vectors && !toeplitz_a, p, eg);
  if (s != HHL_OK) { return s; }
  double lmin = 1e300, lmax = -1e300, amin = 1e300, amax = 0.0;
  for (double l : eg.lam) {
    lmin = std::min(lmin, l);
    lmax = std::max(lmax, l);
    amin = std::min(amin, fabs(l));
    amax = std::max(amax, fabs(l));
  }
  if (amin <= 1e-14 * amax) { return fail(HHL_ERR_SINGULAR, "A is singular"); }
  if (lmin <= 0.0 && !params->signed_clock)
    return fail(HHL_ERR_UNSUPPORTED, "A must be positive definite (unsigned clock reading; signed_clock = 1 for an indefinite A)");
  p.lam_min = lmin;
  p.lam_max = lmax;
  p.kappa = amax / amin;

  // T0 (total convention) and C
  switch (params->t0_rule) {
    case HHL_T0_RANGE_FILL: p.t0 = 2.0 * kPi * (double)(params->signed_clock ? p.R / 2 - 1 : p.R - 1); break;
    case HHL_T0_POWER_LAW: p.t0 = exp(0.918) * pow(p.kappa, -0.363) * (double)p.R; break;
    default: p.t0 = params->t0_convention == HHL_T0_PER_UNIT ? params->t0 * (double)p.R : params->t0; break;
  }
  if (params->t0_scale > 0.0) p.t0 *= params->t0_scale;
  p.C = params->C > 0.0 ? params->C : 2.0 * kPi / p.t0;
  p.theta.assign(p.R, 0.0);
  for (int64_t y = 1; y < p.R; ++y) {
    // two's complement for a signed clock: the top half of the values are negative
    const int64_t ys = (params->signed_clock && y >= p.R / 2) ? y - p.R : y;
    const double lam = 2.0 * kPi * (double)ys / p.t0;
    p.theta[y] = 2.0 * asin(std::max(-1.0, std::min(1.0, p.C / lam)));
  }

  return HHL_OK;
}

}  // namespace

hhl_status plan_scalars(const hhl_problem* prob, const hhl_params* params, Plan& p,
                        std::vector<double>* eigenvalues) {
  hhl_status s = validate(prob, params);
  if (s != HHL_OK) return s;
  Eigen eg;
  s = plan_host(prob, params, p, eg, false);
  if (s == HHL_OK && eigenvalues) *eigenvalues = eg.lam;
  return s;
}

}  // namespace hhl

using hhl::Plan;
using hhl::fail;

struct hhl_plan_s {
  Plan p;
  void* d_meas = nullptr;  // 4 + 2N doubles
  double* d_u = nullptr;   // N doubles + 1 (eps)
  double* d_cdf = nullptr; // N doubles: running sum of the outcome probabilities (shots)
  double* d_bsplit = nullptr;  // 2N doubles: host re / im staging
  double2* d_qpp = nullptr;    // 6N complex128: the LCU register (two halves) and a spare half
};

extern "C" {

int hhl_api_version(void) { return HHL_API_VERSION; }

const char* hhl_status_string(hhl_status s) {
  switch (s) {
    case HHL_OK: return "ok";
    case HHL_ERR_INVALID_ARG: return "invalid argument";
    case HHL_ERR_NOT_HERMITIAN: return "matrix not Hermitian";
    case HHL_ERR_SINGULAR: return "singular system or zero right-hand side";
    case HHL_ERR_OOM: return "out of device memory";
    case HHL_ERR_CUDA: return "CUDA error";
    case HHL_ERR_TIMEOUT: return "device wait timed out";
    case HHL_ERR_NUMERIC: return "non-finite value";
    case HHL_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char* hhl_last_error(void) { return hhl::t_last_error.c_str(); }

uint64_t hhl_kernel_launch_count(void) { return hhl::g_launches.load(); }

void hhl_profile_enable(int32_t on) { hhl::g_prof_on.store(on != 0); }

void hhl_profile_reset(void) {
  hhl::prof_resolve();
  std::lock_guard<std::mutex> lk(hhl::g_prof_mu);
  hhl::g_prof_agg.clear();
}

int32_t hhl_profile_count(void) {
  hhl::prof_resolve();
  std::lock_guard<std::mutex> lk(hhl::g_prof_mu);
  return (int32_t)hhl::g_prof_agg.size();
}

hhl_status hhl_profile_get(int32_t index, char* name, int32_t name_len, uint64_t* launches, double* total_ms) {
  hhl::prof_resolve();
  std::lock_guard<std::mutex> lk(hhl::g_prof_mu);
  if (index < 0 || index >= (int32_t)hhl::g_prof_agg.size() || name == nullptr || name_len < 1)
    return fail(HHL_ERR_INVALID_ARG, "bad profile index or name buffer");
  auto it = hhl::g_prof_agg.begin();
  std::advance(it, index);
  snprintf(name, (size_t)name_len, "%s", it->first.c_str());
  if (launches) *launches = it->second.launches;
  if (total_ms) *total_ms = it->second.ms;
  return HHL_OK;
}

void hhl_params_default(hhl_params* p) {
  if (p == nullptr) return;
  memset(p, 0, sizeof(*p));
  p->n_clock = 6;
  p->t0_rule = HHL_T0_RANGE_FILL;
  p->t0_convention = HHL_T0_TOTAL;
  p->precision = HHL_PREC_C64;
  p->t0 = 0.0;
  p->C = 0.0;
  p->expm_mode = HHL_EXPM_DENSE;
  p->full_uncompute = 0;
  p->trotter_dt = 1.0;
  p->trotter_steps_max = 0;
  p->gemm_impl = HHL_GEMM_AUTO;
}

hhl_status hhl_plan_create(const hhl_problem* prob, const hhl_params* params, hhl_plan_t* out) {
  using namespace hhl;
  const auto t_start = std::chrono::steady_clock::now();
  if (out == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL out");
  *out = nullptr;
  hhl_status s = validate(prob, params);
  if (s != HHL_OK) return s;
  if (fault("plan")) return fail(HHL_ERR_INVALID_ARG, "injected planner failure (HHL_FAULT=plan)");

  hhl_plan_s* h = new hhl_plan_s();
  Plan& p = h->p;
  Eigen eg;
  s = plan_host(prob, params, p, eg, true);
  if (s != HHL_OK) { delete h; return s; }
  const int64_t N = p.N;
  const bool dense = p.expm_mode == HHL_EXPM_DENSE;

  // device buffers
  cudaStream_t st = nullptr;

  HHL_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  const size_t ab = p.amp_bytes();
  const size_t rsz = p.prec == HHL_PREC_C64 ? sizeof(float2) : sizeof(double2);
#define HHL_ALLOC(ptr, bytes, counter)                                          \
  do {                                                                          \
    hhl_status _s = dev_alloc((void**)&(ptr), (bytes), (counter));              \
    if (_s != HHL_OK) { cudaStreamDestroy(st); hhl_plan_destroy(h); return _s; } \
  } while (0)
#define HHL_PLAN_CUDA(expr)                                                          \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess) { cudaStreamDestroy(st); hhl_plan_destroy(h); return cuda_fail(_e, #expr); } \
  } while (0)
#define HHL_PLAN_TRY(expr)                                                  \
  do {                                                                      \
    hhl_status _s = (expr);                                                 \
    if (_s != HHL_OK) { cudaStreamSynchronize(st); cudaStreamDestroy(st); hhl_plan_destroy(h); return _s; } \
  } while (0)

  HHL_ALLOC(p.d_scal, 16 * sizeof(double), &p.workspace_bytes);
  HHL_PLAN_CUDA(cudaMemsetAsync(p.d_scal, 0, 16 * sizeof(double), st));
  HHL_ALLOC(p.d_b, (size_t)N * 2 * sizeof(double), &p.workspace_bytes);
  HHL_ALLOC(p.d_bs, (size_t)std::max<int64_t>(N, 2) * ab, &p.workspace_bytes);
  HHL_ALLOC(h->d_bsplit, (size_t)N * 2 * sizeof(double), &p.workspace_bytes);
  HHL_ALLOC(h->d_meas, (size_t)(4 + 2 * N) * sizeof(double), &p.workspace_bytes);
  HHL_ALLOC(h->d_u, (size_t)(N + 1) * sizeof(double), &p.workspace_bytes);
  HHL_ALLOC(h->d_cdf, (size_t)N * sizeof(double), &p.workspace_bytes);
  HHL_ALLOC(p.d_rot, (size_t)p.R * rsz, &p.table_bytes);
  {
    std::vector<double> rot(2 * p.R);
    for (int64_t y = 0; y < p.R; ++y) {
      rot[2 * y] = cos(p.theta[y] / 2.0);
      rot[2 * y + 1] = sin(p.theta[y] / 2.0);
    }
    if (p.prec == HHL_PREC_C64) {
      std::vector<float> rf(2 * p.R);
      for (size_t i = 0; i < rf.size(); ++i) rf[i] = (float)rot[i];
      HHL_PLAN_CUDA(cudaMemcpyAsync(p.d_rot, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice, st));
      HHL_PLAN_CUDA(cudaStreamSynchronize(st));
    } else {
      HHL_PLAN_CUDA(cudaMemcpyAsync(p.d_rot, rot.data(), rot.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      HHL_PLAN_CUDA(cudaStreamSynchronize(st));
    }
  }

  {
    // GEMM output rows (dense) or the Trotter pass's interior edges (32 per warp window)
    size_t scratch_amps = (size_t)(p.R / 2) * N;
    if (!dense) scratch_amps = (size_t)trotter_side_amps(N, p.R);
    HHL_ALLOC(p.d_scratch, scratch_amps * ab, &p.workspace_bytes);
  }
  if (dense) {
    p.gemm_impl = params->gemm_impl;
    if (p.gemm_impl == HHL_GEMM_AUTO) p.gemm_impl = tc_supported(p) ? HHL_GEMM_TCGEN05 : HHL_GEMM_SIMT;
    if (p.gemm_impl == HHL_GEMM_TCGEN05 && !tc_supported(p)) {
      cudaStreamDestroy(st);
      hhl_plan_destroy(h);
      return fail(HHL_ERR_UNSUPPORTED, "tcgen05 GEMM not available for this size/precision");
    }
    const size_t mat = (size_t)N * N;
    // CUDA-core operands: every k (SIMT plans), or the k whose tree steps of the postselected
    // solve have fewer rows than one tcgen05 tile (2^k < 128) (tcgen05 plans)
    // (complex64 plans of a Toeplitz A keep the g_k tables instead: their small steps generate
    // U_k on the fly)
    if (eg.toeplitz && p.prec == HHL_PREC_C64)
      HHL_ALLOC(p.d_gdf, (size_t)p.n_c * (2 * N + 2) * sizeof(float4), &p.table_bytes);
    const int n_simt = p.gemm_impl == HHL_GEMM_SIMT ? p.n_c : (p.d_gdf != nullptr ? 0 : std::min(p.n_c, kTreeSimtBits));
    if (n_simt > 0) {
      HHL_ALLOC(p.d_bfwd, (size_t)n_simt * mat * ab, &p.table_bytes);
      HHL_ALLOC(p.d_badj, (size_t)n_simt * mat * ab, &p.table_bytes);
    }
    // Toeplitz A (the channel-flow operators): U_k[n][m] = g_k(n-m) - g_k(n+m+2) from the
    // analytic sine basis, O(N^2) per k. Otherwise the eigenvectors go to the device once and
    // every U_k is one FP64 eigen-product (O(N^3)).
    double *d_vr = nullptr, *d_vi = nullptr, *d_c = nullptr, *d_s = nullptr, *d_ctab = nullptr;
    double2 *d_u = nullptr, *d_g = nullptr;
    const int J = eg.J;
    uint64_t tmp_bytes = 0;
    auto free_tmp = [&]() {
      if (d_vr) cudaFree(d_vr);
      if (d_vi) cudaFree(d_vi);
      if (d_c) cudaFree(d_c);
      if (d_s) cudaFree(d_s);
      if (d_u) cudaFree(d_u);
      if (d_ctab) cudaFree(d_ctab);
      if (d_g) cudaFree(d_g);
    };
    hhl_status ts = HHL_OK;
    if (prob->kind == HHL_MATRIX_UNITARY) {
      // U_k = Q^(2^k) by repeated squaring in FP64 on the host, then the same operands
      ts = dev_alloc((void**)&d_u, mat * sizeof(double2), &tmp_bytes);
      if (ts != HHL_OK) { cudaStreamDestroy(st); hhl_plan_destroy(h); return ts; }
      std::vector<double> qr(mat), qi(mat), tr(mat), ti(mat), up(2 * mat);
      for (size_t e = 0; e < mat; ++e) {
        qr[e] = prob->dense_re[e];
        qi[e] = prob->dense_im ? prob->dense_im[e] : 0.0;
      }
      cudaError_t ue = cudaSuccess;
      for (int k = 0; k < p.n_c && ue == cudaSuccess; ++k) {
        if (k > 0) {
          // row i of Q^2 accumulates row l of Q scaled by Q[i][l], l in increasing order
          // (unit-stride inner loop; the zero entries of a block-structured Q are skipped)
          std::fill(tr.begin(), tr.end(), 0.0);
          std::fill(ti.begin(), ti.end(), 0.0);
          for (int64_t i = 0; i < N; ++i)
            for (int64_t l = 0; l < N; ++l) {
              const double ar = qr[i * N + l], ai = qi[i * N + l];
              if (ar == 0.0 && ai == 0.0) continue;
              const double* br = &qr[l * N];
              const double* bi = &qi[l * N];
              double* cr = &tr[i * N];
              double* ci = &ti[i * N];
              for (int64_t j = 0; j < N; ++j) {
                cr[j] += ar * br[j] - ai * bi[j];
                ci[j] += ar * bi[j] + ai * br[j];
              }
            }
          qr.swap(tr);
          qi.swap(ti);
        }
        for (size_t e = 0; e < mat; ++e) {
          up[2 * e] = qr[e];
          up[2 * e + 1] = qi[e];
        }
        ue = cudaMemcpyAsync(d_u, up.data(), 2 * mat * sizeof(double), cudaMemcpyHostToDevice, st);
        hhl_status ks = ue == cudaSuccess ? store_operands_k(p, d_u, k, st) : HHL_OK;
        if (ks != HHL_OK) { cudaStreamSynchronize(st); cudaFree(d_u); cudaStreamDestroy(st); hhl_plan_destroy(h); return ks; }
        if (ue == cudaSuccess) ue = cudaStreamSynchronize(st);  // the host buffer is reused next k
      }
      cudaFree(d_u);
      if (ue != cudaSuccess) { cudaStreamDestroy(st); hhl_plan_destroy(h); return cuda_fail(ue, "plan powers of Q"); }
      p.gemm_flops = (double)(p.full ? 3 : 2) * p.n_c * 8.0 * (double)(p.R / 2) * (double)N * (double)N;
    } else {
    if (!eg.toeplitz) ts = dev_alloc((void**)&d_vr, (size_t)N * J * sizeof(double), &tmp_bytes);
    if (ts == HHL_OK && !eg.vi.empty()) ts = dev_alloc((void**)&d_vi, (size_t)N * J * sizeof(double), &tmp_bytes);
    if (ts == HHL_OK) ts = dev_alloc((void**)&d_c, (size_t)J * sizeof(double), &tmp_bytes);
    if (ts == HHL_OK) ts = dev_alloc((void**)&d_s, (size_t)J * sizeof(double), &tmp_bytes);
    if (ts == HHL_OK) ts = dev_alloc((void**)&d_u, mat * sizeof(double2), &tmp_bytes);
    if (ts == HHL_OK && eg.toeplitz) ts = dev_alloc((void**)&d_ctab, (size_t)(2 * N + 2) * sizeof(double), &tmp_bytes);
    if (ts == HHL_OK && eg.toeplitz) ts = dev_alloc((void**)&d_g, (size_t)(2 * N + 2) * sizeof(double2), &tmp_bytes);
    if (ts != HHL_OK) { free_tmp(); cudaStreamDestroy(st); hhl_plan_destroy(h); return ts; }
    cudaError_t ce = cudaSuccess;
    std::vector<double> ctab;
    if (eg.toeplitz) {
      ctab.resize(2 * N + 2);
      for (int64_t q = 0; q < 2 * N + 2; ++q) ctab[q] = cos((double)q * kPi / (double)(N + 1));
      ce = cudaMemcpyAsync(d_ctab, ctab.data(), ctab.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
      ce = cudaMemcpyAsync(d_vr, eg.vr.data(), (size_t)N * J * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    if (ce == cudaSuccess && d_vi)
      ce = cudaMemcpyAsync(d_vi, eg.vi.data(), (size_t)N * J * sizeof(double), cudaMemcpyHostToDevice, st);
    std::vector<double> ch(J), sh(J);
    for (int k = 0; k < p.n_c && ce == cudaSuccess; ++k) {
      const double t = p.t0 * (double)(1LL << k) / (double)p.R;
      for (int j = 0; j < J; ++j) {
        const double ph = (eg.lam[j] / p.lam_ub) * t;
        ch[j] = cos(ph);
        sh[j] = sin(ph);
      }
      ce = cudaMemcpyAsync(d_c, ch.data(), J * sizeof(double), cudaMemcpyHostToDevice, st);
      if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_s, sh.data(), J * sizeof(double), cudaMemcpyHostToDevice, st);
      if (ce != cudaSuccess) break;
      hhl_status ks = eg.toeplitz ? launch_toeplitz_expm((int)N, d_c, d_s, d_ctab, d_g, d_u, st)
                                  : launch_expm_eigen((int)N, J, d_vr, d_vi, d_c, d_s, eg.wgt, d_u, st);
      if (ks == HHL_OK && p.d_gdf != nullptr) ks = launch_g_to_df((int)N, d_g, p.d_gdf + (size_t)k * (2 * N + 2), st);
      if (ks == HHL_OK) ks = store_operands_k(p, d_u, k, st);
      if (ks != HHL_OK) { cudaStreamSynchronize(st); free_tmp(); cudaStreamDestroy(st); hhl_plan_destroy(h); return ks; }
      ce = cudaStreamSynchronize(st);  // host phase buffers are reused next iteration
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    free_tmp();
    if (ce != cudaSuccess) { cudaStreamDestroy(st); hhl_plan_destroy(h); return cuda_fail(ce, "plan exponentials"); }
    const int mult = p.full ? 3 : 2;
    p.gemm_flops = (double)mult * p.n_c * 8.0 * (double)(p.R / 2) * (double)N * (double)N;
    }
  } else {
    // Strang blocks of exp(i s M) for the Toeplitz Ahat: E blocks [[d, o], [o, d]] on
    // pairs (2i, 2i+1) and O blocks [[0, o], [o, 0]] on pairs (2i+1, 2i+2).
    p.gemm_impl = HHL_GEMM_SIMT;
    const double dh = prob->diag[0] / p.lam_ub, oh = N > 1 ? prob->off[0] / p.lam_ub : 0.0;
    p.trot_r.resize(p.n_c);
    p.trot_blocks.assign((size_t)p.n_c * 24, 0.0);
    // exp(i s [[d, o], [o, d]]) = e^{i s d} R(s o) and exp(i s [[0, o], [o, 0]]) = R(s o),
    // R(th) = [[cos th, i sin th], [i sin th, cos th]]. Per k: cos, sin of (tau/2) o and
    // tau o, then tau and d (the E phases are applied once per pass).
    for (int k = 0; k < p.n_c; ++k) {
      const double t = p.t0 * (double)(1LL << k) / (double)p.R;
      int r = (int)std::ceil(t / p.trotter_dt);
      if (r < 1) r = 1;
      if (p.trotter_max > 0 && r > p.trotter_max) r = p.trotter_max;
      p.trot_r[k] = r;
      const double tau = t / r;
      double* q = &p.trot_blocks[(size_t)k * 24];
      q[0] = cos(0.5 * tau * oh);
      q[1] = sin(0.5 * tau * oh);
      q[2] = cos(tau * oh);
      q[3] = sin(tau * oh);
      q[4] = tau;
      q[5] = dh;
    }
    p.trot_diag_hat = dh;
    p.trot_off_hat = oh;
    HHL_ALLOC(p.d_trot, p.trot_blocks.size() * sizeof(double), &p.table_bytes);
    HHL_PLAN_CUDA(cudaMemcpyAsync(p.d_trot, p.trot_blocks.data(), p.trot_blocks.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, st));
    std::vector<unsigned char> lists;
    hhl::trotter_build_passes(p, &lists);
    p.trotter_passes = (int64_t)p.trot_pass[0].size() + (int64_t)p.trot_pass[1].size() * (p.full ? 2 : 1);
    for (int dir = 0; dir < 2; ++dir)
      for (const TrotPassDesc& d : p.trot_pass[dir]) {
        const double rows = d.single_k >= 0 ? (double)(p.R / 2) : (double)p.R * (1.0 - 1.0 / (double)(1 << d.gbits));
        p.trotter_bytes += (dir == 1 && p.full ? 2.0 : 1.0) * 2.0 * rows * (double)N * (double)ab;
      }
    HHL_ALLOC(p.d_trot_lists, lists.size(), &p.table_bytes);
    HHL_PLAN_CUDA(cudaMemcpyAsync(p.d_trot_lists, lists.data(), lists.size(), cudaMemcpyHostToDevice, st));
    HHL_PLAN_CUDA(cudaStreamSynchronize(st));
  }
  cudaStreamDestroy(st);
  p.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  *out = h;
  return HHL_OK;
#undef HHL_ALLOC
#undef HHL_PLAN_CUDA
#undef HHL_PLAN_TRY
}

hhl_status hhl_plan(const hhl_problem* prob, const hhl_params* params, hhl_plan_t* out) {
  return hhl_plan_create(prob, params, out);
}

void hhl_plan_destroy(hhl_plan_t plan) {
  if (plan == nullptr) return;
  Plan& p = plan->p;
  void* ptrs[] = {p.d_bfwd, p.d_badj, p.d_gdf, p.d_rot, p.d_scal, p.d_b, p.d_bs, p.d_scratch, p.d_trot,
                  p.d_trot_lists, plan->d_meas, plan->d_u, plan->d_cdf, plan->d_bsplit, plan->d_qpp};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  hhl::tc_free(p);
  delete plan;
}

hhl_status hhl_plan_get_info(hhl_plan_t plan, hhl_plan_info* info) {
  if (plan == nullptr || info == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL plan or info");
  const Plan& p = plan->p;
  memset(info, 0, sizeof(*info));
  info->n_sys_qubits = p.n_s;
  info->n_clock = p.n_c;
  info->n_qubits = p.n;
  info->precision = p.prec;
  info->expm_mode = p.expm_mode;
  info->gemm_impl = p.gemm_impl;
  info->lambda_ub = p.lam_ub;
  info->lambda_min = p.lam_min;
  info->lambda_max = p.lam_max;
  info->kappa = p.kappa;
  info->t0 = p.t0;
  info->C = p.C;
  info->state_bytes = (uint64_t)(2 * p.R * p.N) * p.amp_bytes();
  info->table_bytes = p.table_bytes;
  info->workspace_bytes = p.workspace_bytes;
  info->gemm_flops = p.gemm_flops;
  info->trotter_passes = p.trotter_passes;
  info->trotter_bytes = p.trotter_bytes;
  info->plan_seconds = p.plan_seconds;
  return HHL_OK;
}

uint64_t hhl_state_bytes(hhl_plan_t plan) {
  if (plan == nullptr) return 0;
  return (uint64_t)(2 * plan->p.R * plan->p.N) * plan->p.amp_bytes();
}

hhl_status hhl_prepare_rhs(hhl_plan_t plan, const double* b_dev, void* state_dev, void* stream) {
  if (plan == nullptr || b_dev == nullptr || state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal, 0, sizeof(double), st));
  hhl_status s = hhl::launch_bnorm(b_dev, p.N, p.d_scal, st);
  if (s != HHL_OK) return s;
  return hhl::launch_prep_fill(p, b_dev, state_dev, st);
}

hhl_status hhl_prepare_rhs_host(hhl_plan_t plan, const double* b_re, const double* b_im, void* state_dev,
                                void* stream) {
  if (plan == nullptr || b_re == nullptr || state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  HHL_CUDA_TRY(cudaMemcpyAsync(plan->d_bsplit, b_re, p.N * sizeof(double), cudaMemcpyHostToDevice, st));
  if (b_im) HHL_CUDA_TRY(cudaMemcpyAsync(plan->d_bsplit + p.N, b_im, p.N * sizeof(double), cudaMemcpyHostToDevice, st));
  hhl_status s = hhl::launch_interleave(plan->d_bsplit, b_im ? plan->d_bsplit + p.N : nullptr, p.N, p.d_b, st);
  if (s != HHL_OK) return s;
  return hhl_prepare_rhs(plan, p.d_b, state_dev, stream);
}

hhl_status hhl_prepare_rhs_qsp1(hhl_plan_t plan, const double* b_dev, void* state_dev, void* stream) {
  if (plan == nullptr || b_dev == nullptr || state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  if (p.N < 2) return fail(HHL_ERR_UNSUPPORTED, "QSP-1 needs at least one system qubit");
  return hhl::launch_prep_qsp1(p, b_dev, plan->d_bsplit, (double2*)p.d_b, state_dev, (cudaStream_t)stream);
}

hhl_status hhl_qpp_dissipation(hhl_plan_t plan, const void* state_dev, double* eps, double* p0, void* stream) {
  if (plan == nullptr || state_dev == nullptr || eps == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->d_qpp == nullptr) {  // first call: the plan-owned LCU register
    HHL_CUDA_TRY(cudaStreamSynchronize(st));
    HHL_CUDA_TRY(cudaMalloc((void**)&plan->d_qpp, (size_t)6 * p.N * sizeof(double2)));
    p.workspace_bytes += (uint64_t)6 * p.N * sizeof(double2);
  }
  hhl_status s = hhl::launch_qpp_dissipation(p, state_dev, plan->d_qpp, p.d_scal + 5, st);
  if (s != HHL_OK) return s;
  double acc[2] = {0.0, 0.0};
  HHL_CUDA_TRY(cudaMemcpyAsync(acc, p.d_scal + 5, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  if (!(acc[0] > 0.0)) return fail(HHL_ERR_SINGULAR, "the velocity register is zero");
  const double h = 1.0 / (double)(p.N + 1);
  *eps = p.nu / h * (4.0 * acc[1] * acc[0] - p.wall_lo * p.wall_lo - p.wall_hi * p.wall_hi);
  if (p0 != nullptr) *p0 = acc[1];
  return HHL_OK;
}

hhl_status hhl_prepare_rhs_qsp2(hhl_plan_t plan, const int64_t* idx_dev, const double* val_dev, int64_t count,
                                void* state_dev, void* stream) {
  if (plan == nullptr || idx_dev == nullptr || val_dev == nullptr || state_dev == nullptr)
    return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  Plan& p = plan->p;
  if (p.N < 2) return fail(HHL_ERR_UNSUPPORTED, "QSP-2 needs at least one system qubit");
  if (count < 1 || count > p.N) return fail(HHL_ERR_INVALID_ARG, "count must be in 1..N");
  return hhl::launch_prep_qsp2(p, idx_dev, val_dev, count, (double2*)p.d_b, state_dev, (cudaStream_t)stream);
}

static hhl_status ctrl_u(const Plan& p, void* half, int k, bool adj, cudaStream_t st) {
  if (p.gemm_impl == HHL_GEMM_TCGEN05) return hhl::launch_ctrl_u_tc(p, half, k, adj, st);
  return hhl::launch_ctrl_u_dense(p, half, k, adj, st);
}

hhl_status hhl_apply_stage(hhl_plan_t plan, int32_t stage, void* state_dev, void* stream) {
  if (plan == nullptr || state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  if (hhl::fault("launch")) return fail(HHL_ERR_CUDA, "injected launch failure (HHL_FAULT=launch)");
  const Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  char* s0 = (char*)state_dev;
  char* s1 = s0 + (size_t)(p.R * p.N) * p.amp_bytes();
  hhl_status s = HHL_OK;
  switch (stage) {
    case HHL_STAGE_QPE_U:
      if (p.expm_mode == HHL_EXPM_TROTTER) return hhl::launch_trotter(p, s0, false, st);
      s = hhl::tc_reset_error(p, st);  // a new circuit: the GEMM status covers it alone
      for (int k = 0; k < p.n_c && s == HHL_OK; ++k) s = ctrl_u(p, s0, k, false, st);
      return s;
    case HHL_STAGE_CLOCK_BLOCK:
      return hhl::launch_clock_block(p, state_dev, st);
    case HHL_STAGE_UNCOMPUTE_U:
      if (p.expm_mode == HHL_EXPM_TROTTER) {
        s = hhl::launch_trotter(p, s1, true, st);
        if (s == HHL_OK && p.full) s = hhl::launch_trotter(p, s0, true, st);
        return s;
      }
      for (int k = p.n_c - 1; k >= 0 && s == HHL_OK; --k) {
        s = ctrl_u(p, s1, k, true, st);
        if (s == HHL_OK && p.full) s = ctrl_u(p, s0, k, true, st);
      }
      return s;
    case HHL_STAGE_FINAL_H:
      return hhl::launch_final_h(p, state_dev, st);
    default:
      return fail(HHL_ERR_INVALID_ARG, "bad stage");
  }
}

hhl_status hhl_apply_circuit(hhl_plan_t plan, void* state_dev, void* stream) {
  for (int stage = HHL_STAGE_QPE_U; stage <= HHL_STAGE_FINAL_H; ++stage) {
    hhl_status s = hhl_apply_stage(plan, stage, state_dev, stream);
    if (s != HHL_OK) return s;
  }
  return HHL_OK;
}

hhl_status hhl_solve_postselected(hhl_plan_t plan, const double* b_dev, void* state_dev, double* out_dev,
                                  double* eps_dev, void* stream) {
  if (plan == nullptr || b_dev == nullptr || state_dev == nullptr || out_dev == nullptr)
    return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = plan->p;
  const bool dense = p.expm_mode == HHL_EXPM_DENSE;
  std::string why;
  if (dense && p.full) return fail(HHL_ERR_UNSUPPORTED, "the postselected solve needs full_uncompute = 0");
  if (!dense && !hhl::trotter_tree_supported(p, &why)) return fail(HHL_ERR_UNSUPPORTED, why);
  cudaStream_t st = (cudaStream_t)stream;
  char* s0 = (char*)state_dev;
  char* s1 = s0 + (size_t)(p.R * p.N) * p.amp_bytes();
  // the trees as controlled-product GEMMs (dense plans) or Strang passes (Trotter plans)
  auto tree = [&](void* half, bool reduce) -> hhl_status {
    if (!dense) return hhl::launch_trotter_tree(p, half, reduce, st);
    for (int j = 0; j < p.n_c; ++j) {
      hhl_status ts = hhl::launch_ctrl_u_tree(p, half, reduce ? p.n_c - 1 - j : j, reduce, st);
      if (ts != HHL_OK) return ts;
    }
    return HHL_OK;
  };
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal, 0, sizeof(double), st));
  hhl_status s = hhl::tc_reset_error(p, st);
  if (s == HHL_OK) s = hhl::launch_bnorm(b_dev, p.N, p.d_scal, st);
  if (s == HHL_OK) s = hhl::launch_prep_row(p, b_dev, s0, st);
  if (s == HHL_OK) s = tree(s0, false);                                // QPE by doubling
  // the clock block writes the whole anc = 1 half; the weights |S0|^2, |S1|^2 (= P(anc = 1))
  // come from its pass B on the split path, else from a read of both halves
  bool summed = false;
  if (s == HHL_OK) s = [&]() -> hhl_status {
    HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal + 1, 0, 3 * sizeof(double), st));
    return HHL_OK;
  }();
  if (s == HHL_OK) s = hhl::launch_clock_block_sums(p, state_dev, p.d_scal + 1, &summed, st);
  if (s == HHL_OK && !summed) s = hhl::launch_clock_block(p, state_dev, st);
  if (s == HHL_OK && !summed) s = hhl::launch_measure_sums(p, state_dev, st);
  if (s == HHL_OK) s = tree(s1, true);                                 // uncompute + H + clock = 0
  if (s == HHL_OK) s = hhl::launch_measure_row(p, state_dev, out_dev, st);
  if (s == HHL_OK && eps_dev != nullptr) s = hhl::launch_dissipation(p, state_dev, eps_dev, nullptr, st);
  return s;
}

hhl_status hhl_measure_async(hhl_plan_t plan, const void* state_dev, double* out_dev, void* stream) {
  if (plan == nullptr || state_dev == nullptr || out_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  return hhl::launch_measure(plan->p, state_dev, out_dev, (cudaStream_t)stream);
}

hhl_status hhl_measure(hhl_plan_t plan, const void* state_dev, hhl_measurement* out, double* x_host, void* stream) {
  if (plan == nullptr || state_dev == nullptr || out == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  hhl_status s = hhl::launch_measure(p, state_dev, (double*)plan->d_meas, st);
  if (s != HHL_OK) return s;
  double sc[4];
  HHL_CUDA_TRY(cudaMemcpyAsync(sc, plan->d_meas, sizeof(sc), cudaMemcpyDeviceToHost, st));
  if (x_host) HHL_CUDA_TRY(cudaMemcpyAsync(x_host, (double*)plan->d_meas + 4, 2 * p.N * sizeof(double), cudaMemcpyDeviceToHost, st));
  int tc_err = 0;
  if (int* ef = hhl::tc_error_flag(p)) HHL_CUDA_TRY(cudaMemcpyAsync(&tc_err, ef, sizeof(int), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  if (tc_err != 0) return hhl::tc_flag_status(tc_err);
  out->p_success = sc[0];
  out->p_anc1 = sc[1];
  out->norm = sc[2];
  out->b_norm = sc[3];
  if (!(sc[3] > 0.0)) return fail(HHL_ERR_SINGULAR, "|b| = 0");
  if (!(sc[0] > 0.0)) return fail(HHL_ERR_SINGULAR, "postselection probability is 0");
  return HHL_OK;
}

hhl_status hhl_plan_status(hhl_plan_t plan, void* stream) {
  if (plan == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL plan");
  cudaStream_t st = (cudaStream_t)stream;
  int tc_err = 0;
  if (int* ef = hhl::tc_error_flag(plan->p))
    HHL_CUDA_TRY(cudaMemcpyAsync(&tc_err, ef, sizeof(int), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  return hhl::tc_flag_status(tc_err);
}

hhl_status hhl_sample(hhl_plan_t plan, const void* state_dev, const double* uniforms_dev, int64_t shots,
                      uint64_t* counts_dev, void* stream) {
  if (plan == nullptr || state_dev == nullptr || counts_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  if (shots < 0 || (shots > 0 && uniforms_dev == nullptr)) return fail(HHL_ERR_INVALID_ARG, "bad shots / uniforms");
  return hhl::launch_sample(plan->p, state_dev, uniforms_dev, shots, counts_dev, plan->d_cdf, (cudaStream_t)stream);
}

hhl_status hhl_dissipation_async(hhl_plan_t plan, const void* state_dev, double* eps_dev, void* stream) {
  if (plan == nullptr || state_dev == nullptr || eps_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  return hhl::launch_dissipation(plan->p, state_dev, eps_dev, nullptr, (cudaStream_t)stream);
}

hhl_status hhl_dissipation(hhl_plan_t plan, const void* state_dev, double* eps_out, double* u_host, void* stream) {
  if (plan == nullptr || state_dev == nullptr || eps_out == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = plan->p;
  cudaStream_t st = (cudaStream_t)stream;
  hhl_status s = hhl::launch_dissipation(p, state_dev, plan->d_u + p.N, u_host ? plan->d_u : nullptr, st);
  if (s != HHL_OK) return s;
  double bn2 = 0.0;
  HHL_CUDA_TRY(cudaMemcpyAsync(eps_out, plan->d_u + p.N, sizeof(double), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaMemcpyAsync(&bn2, p.d_scal, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (u_host) HHL_CUDA_TRY(cudaMemcpyAsync(u_host, plan->d_u, p.N * sizeof(double), cudaMemcpyDeviceToHost, st));
  HHL_CUDA_TRY(cudaStreamSynchronize(st));
  if (!(bn2 > 0.0)) return fail(HHL_ERR_SINGULAR, "|b| = 0");
  return HHL_OK;
}

hhl_status hhl_apply_qft(void* state_dev, int32_t n_qubits, int32_t lo, int32_t m, int32_t inverse, int32_t precision,
                         void* stream) {
  if (state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL state");
  if (n_qubits < 1 || n_qubits > 34 || m < 1 || m > 13 || lo < 0 || lo + m > n_qubits)
    return fail(HHL_ERR_INVALID_ARG, "register out of range (1 <= m <= 13, lo + m <= n <= 34)");
  if (precision != HHL_PREC_C64 && precision != HHL_PREC_C128) return fail(HHL_ERR_INVALID_ARG, "bad precision");
  return hhl::launch_qft_register(state_dev, n_qubits, lo, m, inverse != 0, precision, (cudaStream_t)stream);
}

hhl_status hhl_qft_whole(void* state_dev, int32_t n_qubits, int32_t n_states, int32_t direction, int32_t precision,
                         void* stream) {
  if (state_dev == nullptr) return fail(HHL_ERR_INVALID_ARG, "NULL state");
  if (n_qubits < 1 || n_qubits > 32 || n_states < 1 || (n_states & (n_states - 1)) != 0)
    return fail(HHL_ERR_INVALID_ARG, "register out of range (1 <= n <= 32, n_states a power of two)");
  int lo = 0;
  while ((1 << lo) < n_states) ++lo;
  if (n_qubits + lo > 34) return fail(HHL_ERR_INVALID_ARG, "n + log2(n_states) > 34");
  if (direction != 0 && direction != 1) return fail(HHL_ERR_INVALID_ARG, "direction must be 0 or 1");
  if (precision != HHL_PREC_C64 && precision != HHL_PREC_C128) return fail(HHL_ERR_INVALID_ARG, "bad precision");
  return hhl::launch_qft_whole(state_dev, n_qubits, n_states, direction, precision, (cudaStream_t)stream);
}

}  // extern "C"
