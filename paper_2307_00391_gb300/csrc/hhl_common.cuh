// Internal definitions shared by the translation units of libhhl (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hhl.h"

namespace hhl {

// ------------------------------------------------------------------ error reporting
void set_error(const std::string& msg);
// Raise (never lower) a kernel's dynamic shared-memory limit on the current device.
cudaError_t raise_dyn_smem(const void* func, size_t bytes);
hhl_status fail(hhl_status s, const std::string& msg);
hhl_status cuda_fail(cudaError_t e, const char* what);
extern std::atomic<uint64_t> g_launches;

#define HHL_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::hhl::cuda_fail(_e, #expr); \
  } while (0)

// Per-kernel timing (hhl_profile_*): when enabled, an event pair brackets every launch on
// its stream; the pairs are resolved into per-kernel totals when the profile is read.
extern std::atomic<bool> g_prof_on;
void prof_begin(cudaStream_t st);
void prof_end(const char* name);
#define HHL_PROF_BEGIN(st)                                            \
  do {                                                                \
    if (::hhl::g_prof_on.load(std::memory_order_relaxed)) ::hhl::prof_begin(st); \
  } while (0)

// Check the launch just issued, count it, and close its timing record.
#define HHL_LAUNCH_CHECK(name)                                 \
  do {                                                         \
    ::hhl::g_launches.fetch_add(1, std::memory_order_relaxed); \
    cudaError_t _e = cudaGetLastError();                       \
    if (::hhl::g_prof_on.load(std::memory_order_relaxed)) ::hhl::prof_end(name); \
    if (_e != cudaSuccess) return ::hhl::cuda_fail(_e, name);  \
  } while (0)

// ------------------------------------------------------------------ complex helpers
template <class R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };


template <class R> __host__ __device__ __forceinline__ typename Cx<R>::T mk(R re, R im) {
  typename Cx<R>::T z; z.x = re; z.y = im; return z;
}
template <class T> __host__ __device__ __forceinline__ T cadd(T a, T b) { T z; z.x = a.x + b.x; z.y = a.y + b.y; return z; }
template <class T> __host__ __device__ __forceinline__ T csub(T a, T b) { T z; z.x = a.x - b.x; z.y = a.y - b.y; return z; }
template <class T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
  T z; z.x = a.x * b.x - a.y * b.y; z.y = a.x * b.y + a.y * b.x; return z;
}
template <class T> __host__ __device__ __forceinline__ T cconjmul(T a, T b) {  // a * conj(b)
  T z; z.x = a.x * b.x + a.y * b.y; z.y = a.y * b.x - a.x * b.y; return z;
}
template <class T, class S> __host__ __device__ __forceinline__ T cscale(T a, S s) { T z; z.x = a.x * s; z.y = a.y * s; return z; }

// ------------------------------------------------------------------ double-float arithmetic
// The complex128 kernels keep FP64 amplitudes in memory but compute on GB300's FP32 pipe (the
// FP64 pipe is about 1/32 of its rate): a value is the unevaluated sum h + l of two floats
// (about 48 significant bits; Dekker's error-free transformations, Knuth's two-sum). Loads
// split a double into its truncated top 24 significant bits and the rest with integer
// operations only; stores rebuild the double exactly from the two floats and add them with
// one FP64 addition.
struct df {
  float h, l;
  df() = default;
  __host__ __device__ constexpr df(float h_, float l_) : h(h_), l(l_) {}
  __host__ __device__ explicit constexpr df(int v) : h((float)v), l(0.0f) {}
  __host__ __device__ explicit df(double v) : h((float)v), l((float)(v - (double)(float)v)) {}  // (set-up only)
};
struct dfc {
  df x, y;  // real, imaginary
};

// s + e = a + b exactly (any a, b)
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const df s = df_two_sum(a.h, b.h);
  return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ df df_neg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}
// a + w b and a - w b in one go (the two-FMA rotation forms)
__device__ __forceinline__ df df_fma(df w, df b, df a) {
  const float p = __fmul_rn(w.h, b.h);
  float pe = __fmaf_rn(w.h, b.h, -p);
  pe = __fmaf_rn(w.h, b.l, pe);
  pe = __fmaf_rn(w.l, b.h, pe);
  const df s = df_two_sum(a.h, p);
  return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, pe)));
}
__device__ __forceinline__ df df_fnma(df w, df b, df a) { return df_fma(df_neg(w), b, a); }
// The same without the final renormalisation (12 instead of 15 operations): the tail may grow
// to a few units in the last place of the head over a run of such steps, which the error-free
// head sum absorbs; a chain of them ends with df_renorm.
__device__ __forceinline__ df df_fma_lazy(df w, df b, df a) {
  const float p = __fmul_rn(w.h, b.h);
  float pe = __fmaf_rn(w.h, b.h, -p);
  pe = __fmaf_rn(w.h, b.l, pe);
  pe = __fmaf_rn(w.l, b.h, pe);
  const df s = df_two_sum(a.h, p);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, pe))};
}
__device__ __forceinline__ df df_fnma_lazy(df w, df b, df a) { return df_fma_lazy(df_neg(w), b, a); }
__device__ __forceinline__ df df_renorm(df a) { return df_two_sum(a.h, a.l); }
__device__ __forceinline__ df df_scale(df a, float s) {  // s a power of two or any float
  const float p = __fmul_rn(a.h, s);
  const float e = __fmaf_rn(a.h, s, -p);
  return df_fast_two_sum(p, __fmaf_rn(a.l, s, e));
}

// FP64 -> double-float without the FP64 pipe: h = the sign, exponent and top 23 stored
// significand bits of x (truncation), l = the 29 remaining bits scaled to their weight.
// Magnitudes below 2^-126 read as zero (their l below 2^-74), far below any amplitude bound.
__device__ __forceinline__ df df_from_double(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const unsigned sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7FFu);
  const unsigned m23 = ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23);
  const float tail = __fmul_rn(__uint2float_rn(lo32 & 0x1FFFFFFFu), __uint_as_float((unsigned)(e - 948) << 23));
  const float l = __uint_as_float(__float_as_uint(tail) | sign);
  return {e > 896 ? h : 0.0f, e > 948 ? l : 0.0f};
}
// float -> double exactly, integer operations only (normal floats; zero and subnormals -> 0)
__device__ __forceinline__ double df_f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b >> 3) & 0xFFFFFu);
  return e == 0 ? 0.0 : __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double df_to_double(df v) { return __dadd_rn(df_f2d(v.h), df_f2d(v.l)); }

template <> struct Cx<df> { using T = dfc; };
__device__ __forceinline__ dfc dfc_from(double2 z) { return {df_from_double(z.x), df_from_double(z.y)}; }
__device__ __forceinline__ double2 dfc_to(dfc z) { return make_double2(df_to_double(z.x), df_to_double(z.y)); }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.x, b.x), df_add(a.y, b.y)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return {df_sub(a.x, b.x), df_sub(a.y, b.y)}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return {df_sub(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ dfc dfc_scale(dfc a, df s) { return {df_mul(a.x, s), df_mul(a.y, s)}; }
// Lazy forms (no final renormalisation; the tail may grow to a few units in the last place of
// the head, which the next error-free head operation absorbs; the store's exact FP64
// reconstruction takes any head and tail).
__device__ __forceinline__ df df_add_lazy(df a, df b) {
  const df s = df_two_sum(a.h, b.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ df df_mul_lazy(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}
// Operators, so that the complex templates (cadd, csub, cmul, cscale, mk) serve dfc as they
// serve float2 and double2 (Cx<df>::T = dfc); they are the lazy forms.
__device__ __forceinline__ df operator+(df a, df b) { return df_add_lazy(a, b); }
__device__ __forceinline__ df operator-(df a) { return df_neg(a); }
__device__ __forceinline__ df operator-(df a, df b) { return df_add_lazy(a, df_neg(b)); }
__device__ __forceinline__ df operator*(df a, df b) { return df_mul_lazy(a, b); }
__device__ __forceinline__ df operator*(df a, float b) {
  const float p = __fmul_rn(a.h, b);
  return {p, __fmaf_rn(a.l, b, __fmaf_rn(a.h, b, -p))};
}
// the double-float pair of an FP64 value (FP64 operations: table set-up only)
__device__ __forceinline__ df df_of(double v) { return df(v); }
// host: the double-float pair of an FP64 constant
inline void df_split(double v, float* h, float* l) {
  *h = (float)v;
  *l = (float)(v - (double)*h);
}

// ------------------------------------------------------------------ row maps of the controlled products
// Which state rows a controlled-U GEMM reads and writes. The circuit's controlled U_k (k >= 0):
// the rows with clock bit k set, in place. The trees of the postselected solve (k = -1):
// contiguous input rows i + in_off, output rows i + out_off, overwritten (expansion) or added
// to (reduction), the stored value multiplied by `scale`.
struct RowMap {
  int k = -1;
  int accumulate = 0;
  int64_t in_off = 0, out_off = 0;
  double scale = 1.0;
};
__host__ __device__ __forceinline__ int64_t rowmap_bit(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}
__host__ __device__ __forceinline__ int64_t rowmap_in(const RowMap& m, int64_t i) {
  return m.k >= 0 ? rowmap_bit(i, m.k) : i + m.in_off;
}
__host__ __device__ __forceinline__ int64_t rowmap_out(const RowMap& m, int64_t i) {
  return m.k >= 0 ? rowmap_bit(i, m.k) : i + m.out_off;
}
inline RowMap circuit_rows(int k) {
  RowMap m;
  m.k = k;
  return m;
}

// U_k[n][m] = g(|n-m|) - g(n+m+2) (0-based n, m; a Toeplitz tridiagonal A's exp(i Ahat t_k)
// from its analytic sine basis) from the double-float table g (hi re, lo re, hi im, lo im), in
// FP32: the difference of the high parts is exact for close values and the low parts restore
// the rest.
__device__ __forceinline__ float2 toeplitz_u(const float4* __restrict__ g, int n, int m) {
  const float4 a = g[n > m ? n - m : m - n], b = g[n + m + 2];
  return make_float2((a.x - b.x) + (a.y - b.y), (a.z - b.z) + (a.w - b.w));
}

// ------------------------------------------------------------------ the plan
// One Trotter pass: clock bits [kb, kb + gbits) (single_k >= 0: the one bit single_k, rows
// with that bit set) and the offset of its per-row-pattern layer lists in the plan's table.
struct TrotPassDesc {
  int kb = 0, gbits = 0, single_k = -1, max_layers = 0;
  int64_t list_off = 0;
};

struct Plan {
  int n_s = 0, n_c = 0, n = 0;
  int prec = HHL_PREC_C64;
  int expm_mode = HHL_EXPM_DENSE;
  int full = 0;
  int gemm_impl = HHL_GEMM_SIMT;
  int64_t N = 0;   // 2^n_s
  int64_t R = 0;   // 2^n_c
  double lam_ub = 0, lam_min = 0, lam_max = 0, kappa = 0, t0 = 0, C = 0;
  double nu = 0, wall_lo = 0, wall_hi = 0;
  std::vector<double> theta;  // rotation angles, 2^n_c
  // device tables
  void* d_bfwd = nullptr;     // n_c matrices, B_fwd[k][m][n] = U_k[n][m]   (SIMT GEMM operand)
  void* d_badj = nullptr;     // n_c matrices, B_adj[k][m][n] = conj(U_k[m][n])
  void* d_tc = nullptr;       // tcgen05 operands (split-FP16 real embeddings), see hhl_gemm_tc.cu
  void* d_rot = nullptr;      // 2^n_c (cos(theta/2), sin(theta/2)) pairs, amplitude precision
  double* d_scal = nullptr;   // device scalars: [0] |b|^2, [1..3] measure sums, [4] eps sum, [5] p_anc1
  double* d_b = nullptr;      // N complex128: host-prepared b
  void* d_bs = nullptr;       // N amplitudes: b / (|b| 2^(n_c/2)), one anc = 0 row
  void* d_scratch = nullptr;  // GEMM output rows: 2^(n_c-1) * N amplitudes
  float4* d_gdf = nullptr;    // Toeplitz A, complex64: per k the 2N+2 double-float g_k values
  // Trotter (Toeplitz tridiagonal): per k the step count and the 2x2 blocks
  std::vector<int> trot_r;
  std::vector<double> trot_blocks;  // per k: E(tau/2), E(tau), O(tau): 3 x 8 doubles
  double* d_trot = nullptr;
  double trot_diag_hat = 0, trot_off_hat = 0;  // the Toeplitz Ahat's diagonal and off-diagonal
  std::vector<TrotPassDesc> trot_pass[2];     // QPE (forward) and uncompute (adjoint) passes
  void* d_trot_lists = nullptr;               // the passes' layer lists
  double trotter_dt = 1.0;
  int trotter_max = 0;
  uint64_t table_bytes = 0, workspace_bytes = 0;
  double gemm_flops = 0;
  int64_t trotter_passes = 0;
  double trotter_bytes = 0;
  double plan_seconds = 0;
  int device = 0;
  size_t amp_bytes() const { return prec == HHL_PREC_C64 ? 8 : 16; }
};

// Validation and the host part of planning (a0) without device work; the eigenvalues of A
// are returned when asked (analytic for a Toeplitz tridiagonal A).
hhl_status plan_scalars(const hhl_problem* prob, const hhl_params* params, Plan& p, std::vector<double>* eigenvalues);

// Launchers (host side of the kernels); all return HHL_OK or an error.
hhl_status launch_bnorm(const double* b, int64_t N, double* acc, cudaStream_t st);
hhl_status launch_prep_fill(const Plan& p, const double* b, void* state, cudaStream_t st);
hhl_status launch_ctrl_u_dense(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st);
// SIMT controlled product with an explicit operand B[m][n] (U^T forward, conj(U) adjoint).
hhl_status launch_ctrl_u_simt(const Plan& p, void* half, int k, const void* B, cudaStream_t st);
// The same on m_sub rows mapped by `rows` (the trees of the postselected solve).
hhl_status launch_ctrl_u_simt_map(const Plan& p, void* half, const RowMap& rows, int64_t m_sub, const void* B,
                                  cudaStream_t st);
// One tree step of the dense postselected solve: expansion (rows [2^k, 2^(k+1)) = U_k rows
// [0, 2^k)) or reduction (rows [0, 2^k) += U_k^dagger rows [2^k, 2^(k+1)), the last one, k = 0,
// scaled by 2^(-n_c/2)), on the plan's operands (tcgen05 where 2^k >= 128, else CUDA cores).
hhl_status launch_ctrl_u_tree(const Plan& p, void* half, int k, bool reduce, cudaStream_t st);
hhl_status launch_clock_block(const Plan& p, void* state, cudaStream_t st);
// The clock block for the postselected solve (postselect-early plans on the split-pass path):
// the anc = 0 half is not stored; the weights of the two halves after the block are added to
// sums[0] and sums[1]. *done = false when the plan takes another path (then nothing is launched).
hhl_status launch_clock_block_sums(const Plan& p, void* state, double* sums, bool* done, cudaStream_t st);
hhl_status launch_final_h(const Plan& p, void* state, cudaStream_t st);
hhl_status launch_measure(const Plan& p, const void* state, double* out, cudaStream_t st);
// The read-outs of the postselected solve: launch_measure_sums before the reduction tree
// (|S0|^2 and |S1|^2 into the plan scalars), launch_measure_row after it (|v|^2 of the
// clock = 0 row of the anc = 1 half, then the measurement block as hhl_measure_async writes it).
hhl_status launch_measure_sums(const Plan& p, const void* state, cudaStream_t st);
hhl_status launch_measure_row(const Plan& p, const void* state, double* out, cudaStream_t st);
// a1 for the postselected solve: b / (|b| 2^(n_c/2)) into the clock = 0 row of the anc = 0 half only.
hhl_status launch_prep_row(const Plan& p, const double* b, void* state, cudaStream_t st);
hhl_status launch_dissipation(const Plan& p, const void* state, double* eps, double* u_dev, cudaStream_t st);
hhl_status launch_sample(const Plan& p, const void* state, const double* uniforms, int64_t shots, uint64_t* counts,
                         double* cdf, cudaStream_t st);
hhl_status launch_prep_qsp1(const Plan& p, const double* b, double* tree, double2* psi, void* state,
                            cudaStream_t st);
hhl_status launch_prep_qsp2(const Plan& p, const int64_t* idx, const double* val, int64_t count, double2* psi,
                            void* state, cudaStream_t st);
hhl_status launch_qpp_dissipation(const Plan& p, const void* state, double2* reg, double* acc, cudaStream_t st);
hhl_status launch_qft_register(void* state, int n, int lo, int m, bool inverse, int prec, cudaStream_t st);
// Whole-register QFT (direction 0, output in bit-reversed order) or inverse QFT (direction 1,
// input in bit-reversed order) of `outer` consecutive n-qubit states.
hhl_status launch_qft_whole(void* state, int n, int outer, int direction, int prec, cudaStream_t st);
hhl_status launch_expm_eigen(int N, int J, const double* d_vr, const double* d_vi, const double* d_cos,
                             const double* d_sin, double wgt, double2* d_u, cudaStream_t st);
hhl_status launch_store_operands(const Plan& p, const double2* d_u, int k, cudaStream_t st);
// All controlled products of QPE (adjoint: of the uncompute) on one half, in grouped passes.
hhl_status launch_trotter(const Plan& p, void* half, bool adjoint, cudaStream_t st);
// The tree passes of the postselected solve: QPE by doubling from the clock = 0 row of the
// anc = 0 half (reduce = false), or the uncompute, final Hadamards and postselection folded
// into the clock = 0 row of the anc = 1 half (reduce = true).
bool trotter_tree_supported(const Plan& p, std::string* why);
hhl_status launch_trotter_tree(const Plan& p, void* half, bool reduce, cudaStream_t st);
// U = exp(i Ahat t) (N x N complex128) for a Toeplitz tridiagonal A from the analytic sine
// basis: d_c / d_s = cos / sin(lambdahat_j t), d_ctab[q] = cos(q pi/(N+1)), q < 2N+2.
hhl_status launch_toeplitz_expm(int N, const double* d_c, const double* d_s, const double* d_ctab, double2* d_g,
                                double2* d_u, cudaStream_t st);
// g (FP64, 2N+2) -> its double-float copy gdf.
hhl_status launch_g_to_df(int N, const double2* d_g, float4* gdf, cudaStream_t st);
// The controlled product on m rows mapped by `rows` with U_k (or U_k^dagger, adjoint) generated
// on the fly from its double-float g table (complex64; the small steps of the trees).
int64_t toeplitz_rows_limit();
hhl_status launch_toeplitz_rows(float2* half, int n_s, const float4* g, int adjoint, const RowMap& rows, int64_t m,
                                cudaStream_t st);
// Plan time: group the clock bits into passes, fill p.trot_pass and the layer-list table
// (bytes, to be uploaded to p.d_trot_lists); returns the number of lists.
size_t trotter_build_passes(Plan& p, std::vector<unsigned char>* table);
int64_t trotter_side_amps(int64_t N, int64_t R);  // side-buffer amplitudes of a Trotter plan
hhl_status launch_interleave(const double* re, const double* im, int64_t n, double* out, cudaStream_t st);

// tcgen05 GEMM (hhl_gemm_tc.cu)
bool tc_supported(const Plan& p);
hhl_status tc_prepare_operands(Plan& p, const double2* d_u, int k, cudaStream_t st);
hhl_status launch_ctrl_u_tc(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st);
void tc_free(Plan& p);
int* tc_error_flag(const Plan& p);  // device flag: 1-3, 5 a bounded GEMM wait ran out, 4 operand out of range
// Clear that flag on the stream (at the start of each circuit, so that a status reports only
// the GEMMs of the circuit since then).
hhl_status tc_reset_error(const Plan& p, cudaStream_t st);
// Map a read-back flag value to a status (HHL_OK for 0).
hhl_status tc_flag_status(int flag);
}  // namespace hhl
#include <cuda.h>
namespace hhl {
// Workspace of the stream-K tcgen05 GEMM: two partial 128 x 256 FP32 tiles per CTA of the
// largest grid (one CTA per SM). One per stream that runs GEMMs: a launch and its fixup use it.
struct TcWork {
  float* ws = nullptr;
  int grid_cap = 0;        // CTAs of the largest grid
};
int tc_num_sms();
hhl_status tc_work_alloc(TcWork& w, size_t* bytes);
void tc_work_free(TcWork& w);
// The split-FP16 tcgen05 GEMM with explicit operands (row gather + stream-K GEMM of one
// controlled product) on m_sub (a multiple of 128) rows mapped by `rows`: bn = 128 or 256
// output real columns per tile; the maps describe the FP16 a_hi / a_lo (M_sub x 2N) and the
// embedded operand hi / lo (2N x 2N, both scaled by 2^15) with boxes (32 x 128) and (32 x bn).
// streamk = 0: one CTA per output tile; 1: stream-K over the SMs when the tiles are few.
// slice4 (optional): the embedded operand's hi / lo maps with a (32 x bn / 4) box, which lets
// a one-CTA-per-tile launch share each B tile across a cluster of 4 CTAs (TMA multicast).
hhl_status launch_tc_gemm_map(int n_s, int64_t m_sub, const RowMap& rows, void* half, void* a_hi, void* a_lo,
                              const CUtensorMap& map_ahi, const CUtensorMap& map_alo, const CUtensorMap& map_bhi,
                              const CUtensorMap& map_blo, int bn, int* err, const TcWork& w, int streamk,
                              cudaStream_t st, const CUtensorMap* slice4 = nullptr);
// The plan's tcgen05 product on mapped rows (m_sub a multiple of 128).
hhl_status launch_ctrl_u_tc_map(const Plan& p, void* half, const RowMap& rows, int64_t m_sub, int k, bool adjoint,
                                cudaStream_t st);
hhl_status tc_make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows);
hhl_status tc_init_kernels();

}  // namespace hhl
