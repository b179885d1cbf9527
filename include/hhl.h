/*
 * hhl.h - C ABI of the GB300 (sm_103a) state-vector engine for the HHL quantum
 * linear-systems circuit (QLSA-1) applied to discretised Poiseuille and Couette flow
 * (Bharadwaj & Sreenivasan, "Hybrid quantum algorithms for flow problems").
 *
 * The problem the calls follow is the one stated in Sec. IV: a Hermitian, non-singular
 * A in C^{N x N} (N = 2^n), b in C^N, a number of phase-estimation (clock) qubits and a
 * Hamiltonian-simulation time T0 (Sec. VI); the output is the postselected state
 * proportional to A^{-1} b, its success probability, and the viscous dissipation rate
 * eps = nu <(du/dy)^2> of the resulting velocity field (Sec. VII, App. D).
 *
 * Register layout of a state buffer (the only layout this library reads or writes):
 *   amplitude index = sys | clk << n_s | anc << (n_s + n_c),   qubit q = index bit q.
 * So the buffer is the row-major array S[anc][clk][sys] of 2^(n_s+n_c+1) amplitudes,
 * complex64 (float re, float im) or complex128 (double re, double im) interleaved.
 *
 * Conventions (readings of the paper, which is silent on them):
 *   Ahat = A / lambda_ub, lambda_ub = max_i sum_j |A_ij| (Gershgorin bound);
 *   U_k  = exp(+i Ahat T0 2^k / 2^n_c) for clock bit k ("total" T0 convention);
 *   QFT|x> = 2^(-m/2) sum_y exp(+2 pi i x y / 2^m)|y>, inverse QFT its inverse;
 *   RY(theta) = exp(-i theta Y / 2); theta_y = 2 arcsin(min(1, C T0 / (2 pi y))), theta_0 = 0;
 *   C = 2 pi / T0 unless given.
 *
 * Ownership: the caller owns every state buffer and stream. A plan owns the device copies
 * of its tables (U_k matrices or Trotter blocks, rotation angles, twiddles), a small
 * workspace, and frees them in hhl_plan_destroy. Device pointers are plain
 * cudaMalloc'ed (or PyTorch-allocated) addresses on the current device; streams are
 * cudaStream_t passed as void* (NULL = legacy default stream).
 *
 * Errors: no call throws or aborts. Every call returns an hhl_status; the thread-local
 * text of the last failure is hhl_last_error(). Arguments are validated on the host
 * before any CUDA call. Device-side failures map to HHL_ERR_CUDA; a bounded device wait
 * that runs out maps to HHL_ERR_TIMEOUT.
 *
 * Threading: a plan may be used from one host thread at a time; calls are asynchronous
 * on the given stream except where a host result is returned (hhl_measure,
 * hhl_dissipation), which synchronise that stream.
 */
#ifndef HHL_H_
#define HHL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HHL_API_VERSION 1

typedef enum hhl_status {
  HHL_OK = 0,
  HHL_ERR_INVALID_ARG = 1,   /* a NULL pointer, a size out of range, a bad enum value */
  HHL_ERR_NOT_HERMITIAN = 2, /* |A_ij - conj(A_ji)| > 1e-12 max|A| */
  HHL_ERR_SINGULAR = 3,      /* |lambda|_min <= 1e-14 |lambda|_max, or |b| = 0 */
  HHL_ERR_OOM = 4,           /* device allocation failed */
  HHL_ERR_CUDA = 5,          /* a CUDA runtime call or kernel launch failed */
  HHL_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
  HHL_ERR_NUMERIC = 7,       /* a non-finite value where a finite one is required */
  HHL_ERR_UNSUPPORTED = 8    /* a valid request the library does not implement */
} hhl_status;

typedef enum hhl_matrix_kind {
  HHL_MATRIX_TRIDIAG = 0, /* real symmetric tridiagonal: diag[N], off[N-1] */
  HHL_MATRIX_DENSE = 1,   /* Hermitian, row-major dense_re/dense_im (N <= 256) */
  HHL_MATRIX_UNITARY = 2  /* a unitary Q, row-major dense_re/dense_im (N <= 256): the circuit is
                             run with U_k = Q^(2^k) (phase estimation of Q itself) and with the
                             rotation angles of params.theta_table; the QADC - controlled
                             rotation - QDAC step of the QPP protocol (App. D) is this circuit
                             with Q an amplitude-estimation iterate (on the data register, or
                             on the swap-test register of STEPS 1-3). Dense mode only. */
} hhl_matrix_kind;

typedef enum hhl_t0_rule {
  HHL_T0_USER = 0,       /* params.t0 as given (in params.t0_convention) */
  HHL_T0_POWER_LAW = 1,  /* T0_per_unit = exp(0.918) kappa^-0.363: the T0*-kappa fit of
                            Sec. VI read as a power law (a fallback; unpinned) */
  HHL_T0_RANGE_FILL = 2  /* T0 = 2 pi (2^n_c - 1): lambdahat = 1 maps to the top clock value */
} hhl_t0_rule;

typedef enum hhl_t0_convention {
  HHL_T0_TOTAL = 0,    /* U_k = exp(i Ahat T0 2^k / 2^n_c) */
  HHL_T0_PER_UNIT = 1  /* U_k = exp(i Ahat T0 2^k): converted by T0_total = 2^n_c T0 */
} hhl_t0_convention;

typedef enum hhl_expm_mode {
  HHL_EXPM_DENSE = 0,  /* U_k as dense N x N matrices; controlled U_k = complex GEMM */
  HHL_EXPM_TROTTER = 1 /* U_k as a second-order Strang product of two-level gates
                          (Toeplitz tridiagonal A only) */
} hhl_expm_mode;

typedef enum hhl_precision {
  HHL_PREC_C64 = 32, /* complex64 amplitudes; FP64 angles, norms, probabilities */
  HHL_PREC_C128 = 64 /* complex128 amplitudes throughout */
} hhl_precision;

typedef enum hhl_gemm_impl {
  HHL_GEMM_AUTO = 0,    /* tensor cores (tcgen05, split FP16) for complex64 where built */
  HHL_GEMM_SIMT = 1,    /* CUDA-core FMA tiles (FP32 or FP64) */
  HHL_GEMM_TCGEN05 = 2  /* force the tcgen05 path (complex64 only) */
} hhl_gemm_impl;

/* The linear system A x = b of the steady channel flow (Sec. II Eq. 3, App. A.1). All
 * pointers are HOST memory, read during hhl_plan_create only. */
typedef struct hhl_problem {
  int32_t kind;           /* hhl_matrix_kind */
  int32_t n_sys_qubits;   /* n_s >= 1; N = 2^n_s */
  const double* diag;     /* TRIDIAG: A_ii, length N */
  const double* off;      /* TRIDIAG: A_{i,i+1} = A_{i+1,i}, length N-1 */
  const double* dense_re; /* DENSE: Re A, row-major N x N */
  const double* dense_im; /* DENSE: Im A, row-major N x N, or NULL for real symmetric */
  double nu;              /* kinematic viscosity of the dissipation readout */
  double wall_lo;         /* u(y=0) */
  double wall_hi;         /* u(y=1) */
} hhl_problem;

typedef struct hhl_params {
  int32_t n_clock;           /* n_c, 1..16 phase-estimation qubits */
  int32_t t0_rule;           /* hhl_t0_rule */
  int32_t t0_convention;     /* hhl_t0_convention (HHL_T0_USER only) */
  int32_t precision;         /* hhl_precision */
  double t0;                 /* HHL_T0_USER: the simulation time */
  double C;                  /* inversion constant; 0 => 2 pi / T0 */
  int32_t expm_mode;         /* hhl_expm_mode */
  int32_t full_uncompute;    /* 1: uncompute both ancilla halves (the whole circuit);
                                0: after the inversion rotation only the anc = 1 half is
                                carried on (the anc = 0 half is left as rotated); the
                                postselected result is identical */
  double trotter_dt;         /* Strang step bound: r_k = clamp(ceil(t_k / dt), 1, max) */
  int32_t trotter_steps_max; /* 0 = no cap */
  int32_t gemm_impl;         /* hhl_gemm_impl */
  double t0_scale;           /* multiplies the T0 of the rule (0 or 1: unchanged) */
  const double* theta_table; /* UNITARY: theta_y for y = 0 .. 2^n_c - 1 (HOST, read by
                                hhl_plan_create); ignored otherwise */
  int32_t signed_clock;      /* 1: read the clock in two's complement, y_s = y - 2^n_c for
                                y >= 2^(n_c-1), so that an indefinite A (the Hermitian dilation
                                [[0, M], [M^T, 0]] of a one-shot time-stepping system, App. A
                                Eqs. FE_OBM / BE_OBM) is inverted with the sign of each
                                eigenvalue: sin(theta_y / 2) = clip(C / lambda~_ys, -1, 1),
                                lambda~_ys = 2 pi y_s / T0; RANGE_FILL then takes
                                T0 = 2 pi (2^(n_c-1) - 1). 0: unsigned, A positive definite. */
} hhl_params;

typedef struct hhl_plan_info {
  int32_t n_sys_qubits, n_clock, n_qubits, precision, expm_mode, gemm_impl;
  double lambda_ub;       /* Gershgorin bound used to normalise A */
  double lambda_min;      /* smallest eigenvalue of A (0 if not computed) */
  double lambda_max;      /* largest eigenvalue of A (0 if not computed) */
  double kappa;           /* condition number */
  double t0;              /* T0 in the total convention */
  double C;               /* inversion constant */
  uint64_t state_bytes;   /* bytes of one state buffer for this plan */
  uint64_t table_bytes;   /* device bytes of U_k / Trotter / angle tables */
  uint64_t workspace_bytes;
  double gemm_flops;      /* algorithmic flops of the controlled-U GEMMs of one circuit */
  int64_t trotter_passes; /* Trotter mode: HBM passes (k_trotter_pass launches) of one circuit */
  double plan_seconds;    /* wall time of hhl_plan_create */
  double trotter_bytes;   /* Trotter mode: algorithmic HBM bytes (read + write) of those passes:
                             every system row a pass changes, read and written once */
} hhl_plan_info;

typedef struct hhl_measurement {
  double p_success; /* |v|^2, v = amplitudes with anc = 1 and clock = 0 */
  double p_anc1;    /* total weight of the anc = 1 half */
  double norm;      /* total weight of the state */
  double b_norm;    /* |b| recorded by the last hhl_prepare_rhs on this plan */
} hhl_measurement;

typedef struct hhl_plan_s* hhl_plan_t;

/* Version / diagnostics */
int hhl_api_version(void);
const char* hhl_status_string(hhl_status s);
const char* hhl_last_error(void); /* thread-local detail of the last failure */

/* Fill p with the defaults: n_clock 6, RANGE_FILL, TOTAL, C64, DENSE, postselect-early
 * uncompute, trotter_dt 1, no step cap, GEMM AUTO. */
void hhl_params_default(hhl_params* p);

/* a0 - classical pre-computation (Sec. II.A: the parameters "beta" computed
 * classically; Sec. VI: exp(i A T0) through the spectral decomposition of A).
 * Validates A, normalises it by lambda_ub, computes kappa, T0, C, the rotation angles
 * theta_y in FP64, the U_k matrices (dense mode; on the device, FP64) or the Strang
 * blocks (Trotter mode), and uploads the tables. On success *out owns device memory.
 * Requires A positive definite (the clock value is read as an unsigned fraction) unless
 * params.signed_clock = 1. */
hhl_status hhl_plan_create(const hhl_problem* prob, const hhl_params* params, hhl_plan_t* out);
void hhl_plan_destroy(hhl_plan_t plan);
/* The same call under the name of the hot-path contract (hhl_plan_create). */
hhl_status hhl_plan(const hhl_problem* prob, const hhl_params* params, hhl_plan_t* out);
hhl_status hhl_plan_get_info(hhl_plan_t plan, hhl_plan_info* info);
uint64_t hhl_state_bytes(hhl_plan_t plan);

/* a1 - amplitude encoding of b (Sec. IV.A: the right-hand side loaded as a quantum state)
 * followed by a Hadamard on every clock qubit: S[0][c][:] = b / (|b| 2^(n_c/2)),
 * S[1][:][:] = 0. b_dev: DEVICE complex128 (re, im interleaved), length N. |b| is kept
 * on the device for the dissipation readout. Error if |b| = 0 is detected later by
 * hhl_measure / hhl_dissipation (HHL_ERR_SINGULAR). */
hhl_status hhl_prepare_rhs(hhl_plan_t plan, const double* b_dev, void* state_dev, void* stream);

/* As hhl_prepare_rhs with b in HOST memory (b_im may be NULL for real b): copies b to
 * a plan-owned device buffer on the stream, then encodes it. */
hhl_status hhl_prepare_rhs_host(hhl_plan_t plan, const double* b_re, const double* b_im,
                                void* state_dev, void* stream);

/* a1, gate-level form (App. C, QSP-1): the system register is prepared from |0> by the
 * binary tree of uniformly controlled RY rotations (level l rotates qubit n_s-1-l by the
 * paper's R_y(theta), theta = arccos sqrt(p(zero child) / p(node)), conditioned on the l more
 * significant qubits), and the Hadamard layer on the clock puts that state into every clock
 * row: the anc = 0 half holds |b|-amplitude encoding / 2^(n_c/2), the anc = 1 half is zero.
 * The tree encodes magnitudes: for b_i >= 0 (every flow right-hand side) the result equals
 * hhl_prepare_rhs. |b| is recorded for the read-outs. b_dev: DEVICE, N real doubles. Uses
 * plan-owned scratch; asynchronous. */
hhl_status hhl_prepare_rhs_qsp1(hhl_plan_t plan, const double* b_dev, void* state_dev, void* stream);

/* a1, sparse gate-level form (Sec. III and App. C, QSP-2): for a right-hand side with `count`
 * nonzero entries (the one-shot FE / BE systems of App. A, all registers but the data
 * ones in |0>), only the nodes of the binary decision tree that lie on a path to a nonzero
 * leaf get their rotation (the paper's R_y(theta), theta = arccos sqrt(p(zero child) /
 * p(node)), on qubit n_s-1-l conditioned on the node's l more significant bits): O(count n_s)
 * gates instead of O(N); a negative value gets its sign by a Z on its path. Then the clock
 * Hadamard layer as in hhl_prepare_rhs_qsp1; |val| is recorded for the read-outs.
 * idx_dev: DEVICE int64[count], strictly increasing positions in [0, N) (entries outside
 * that range are ignored; unsorted or repeated positions give an undefined state, not a
 * memory error); val_dev: DEVICE double[count], real. Uses plan-owned scratch; asynchronous.
 * Errors: NULL pointers, count outside 1..N (HHL_ERR_INVALID_ARG). */
hhl_status hhl_prepare_rhs_qsp2(hhl_plan_t plan, const int64_t* idx_dev, const double* val_dev, int64_t count,
                                void* state_dev, void* stream);

/* a7, quantum post-processing form (App. D, the LCU derivative of the QPP protocol): the
 * denormalised velocity u (as hhl_dissipation reads it from the postselected row) and the
 * walls are loaded into a register of 2N points, w = (u_1 .. u_N, u_{N+1}, 0 ..., u_0),
 * normalised; the LCU circuit for (I - P) / 2 (P the cyclic increment; one ancilla: H, Z,
 * controlled P, H) runs on it gate by gate, and the probability p0 of ancilla 0 gives every
 * forward difference at once: eps = nu / h (4 p0 |w|^2 - u_0^2 - u_{N+1}^2), h = 1/(N+1), the
 * same quantity as hhl_dissipation (Sec. VII) read from one probability. *eps and *p0 (may be
 * NULL) are HOST outputs; the call synchronises the stream. The first call on a plan
 * allocates its LCU register (6N complex128 of device memory, freed with the plan).
 * Errors: NULL arguments; HHL_ERR_SINGULAR for a zero register. */
hhl_status hhl_qpp_dissipation(hhl_plan_t plan, const void* state_dev, double* eps, double* p0, void* stream);

/* Host builders of the QPP nonlinear transform (App. D: the QADC by phase estimation of an
 * amplitude-estimation iterate, the squaring rotation, the QDAC), for a UNITARY plan on the
 * HHL kernels. zeta: HOST, 2^a_bits real amplitudes of a normalised state |zeta> = U_V |0>
 * (U_V the Householder reflection taking |0> to |zeta>). form 0: amplitude-estimation form,
 * system register data (low a bits) and address (high a bits), dimension n^2 (n = 2^a_bits,
 * a_bits <= 4); form 1: the swap-test form as App. D prints it (STEPS 1-5), per address s the
 * data register ua, the address clone a1 and the swap-test qubit a2, index
 * ua + n a1 + n^2 a2 + 2 n^2 s, dimension 2 n^3 (a_bits <= 2). All outputs are HOST FP64
 * arrays; the calls use no GPU. Errors: NULL pointers or sizes out of range
 * (HHL_ERR_INVALID_ARG). */
/* q_out (dim x dim, row-major, real): the iterate, block diagonal over the address. Form 0:
 * block k = -U_V S_0 U_V^T S_k (S_j flips the sign of |j>); form 1: block s = -A S_s A^T S_good
 * with A = (H on a2)(SWAP(ua, a1) controlled by a2)(H on a2)(U_V on ua), S_good = -Z on a2 and
 * S_s the flip of |0>_ua |s>_a1 |0>_a2. */
hhl_status hhl_qpp_iterate(const double* zeta, int32_t a_bits, int32_t form, double* q_out);
/* theta_out (2^n_clock): the squaring rotation per clock value y, theta_y = 2 arcsin(c z^2)
 * with z^2 = sin^2(pi y / 2^n_clock) (form 0) or 2 sin^2(pi y / 2^n_clock) - 1 (form 1); |c| <= 1. */
hhl_status hhl_qpp_rotation_table(int32_t n_clock, double c, int32_t form, double* theta_out);
/* b_out (dim, real): the start state, the uniform address times |zeta> (form 0) or the state
 * after STEPS 1-3 (form 1: amplitude (z_i [j = s] +- [i = s] z_j) / (2 sqrt n), + for a2 = 0). */
hhl_status hhl_qpp_start_state(const double* zeta, int32_t a_bits, int32_t form, double* b_out);
/* squares_out (n complex, re/im interleaved): the postselected vector v (dim complex, re/im
 * interleaved) projected, address block by address block, on that block's start state
 * (normalised): ~ c z_s^2 / sqrt(n). */
hhl_status hhl_qpp_project(const double* v, const double* b_start, int32_t a_bits, int32_t form, double* squares_out);

/* a2..a5 - the circuit after state preparation, in place (Sec. IV/VI, standard HHL):
 * clock-bit-controlled U_k for k = 0..n_c-1, inverse QFT on the clock, clock-controlled
 * RY on the ancilla, QFT on the clock, controlled U_k^dagger for k = n_c-1..0, Hadamard on
 * every clock qubit. With full_uncompute = 0 the last three stages act on the anc = 1
 * half only. */
hhl_status hhl_apply_circuit(hhl_plan_t plan, void* state_dev, void* stream);

/* The stages of hhl_apply_circuit one at a time, for checking each kernel on its own.
 * HHL_STAGE_QPE_U: controlled U_k, k = 0..n_c-1, on the anc = 0 half.
 * HHL_STAGE_CLOCK_BLOCK: inverse QFT + controlled RY + QFT, fused.
 * HHL_STAGE_UNCOMPUTE_U: controlled U_k^dagger on the anc = 1 half (and anc = 0 if full).
 * HHL_STAGE_FINAL_H: Hadamards on the clock of the same half or halves. */
typedef enum hhl_stage {
  HHL_STAGE_QPE_U = 0,
  HHL_STAGE_CLOCK_BLOCK = 1,
  HHL_STAGE_UNCOMPUTE_U = 2,
  HHL_STAGE_FINAL_H = 3
} hhl_stage;
hhl_status hhl_apply_stage(hhl_plan_t plan, int32_t stage, void* state_dev, void* stream);

/* a1..a7 for the read-out only (Sec. II.A: the solution is read from the postselected
 * register; App. D: the clock = 0 amplitude after the final Hadamards, U_avg): one whole solve
 * that computes the postselected vector v, its statistics and the dissipation without the
 * rest of the final state. The same circuit, rearranged for its prepared input, in which
 * every clock row of the anc = 0 half holds b / (|b| 2^(n_c/2)):
 *   QPE by doubling - clock rows that agree on bits [0, k) have had the same gates applied,
 *     so rows [2^k, 2^(k+1)) are U_k applied to rows [0, 2^k) (groups of bits at once, with the
 *     plan's per-pattern Strang layer lists; every row still sees its own gate sequence in
 *     circuit order, computed once);
 *   the clock block (inverse QFT, inversion rotation, QFT) as in hhl_apply_circuit;
 *   uncompute, final Hadamards and postselection by halving - the clock = 0 amplitude after
 *     the Hadamards is 2^(-n_c/2) sum_c W_c S1[c] (W_c the product of the U_k^dagger of the set
 *     bits of c), folded from the top clock bit down: row c += U_k^dagger row c + 2^k.
 * Outputs: out_dev (DEVICE, 4 + 2N doubles) in the layout of hhl_measure_async (p_success,
 * p_anc1 = the weight of the anc = 1 half before the uncompute, norm, |b|, xhat); eps_dev
 * (DEVICE, 1 double, may be NULL) as hhl_dissipation_async. b_dev: DEVICE complex128, length N.
 * state_dev is the plan's state buffer used as workspace: afterwards only the clock = 0 row of
 * the anc = 1 half is defined (it holds v, so hhl_dissipation, hhl_sample and
 * hhl_qpp_dissipation may read it; hhl_measure may not). Asynchronous.
 * Dense plans run the two trees as controlled-U products on 2^k rows: tcgen05 GEMMs where
 * 2^k >= 128 (a stream-K grid over the SMs when the product has few tiles, its split tiles added
 * in a fixed order, so results repeat bit for bit), below that on the CUDA cores (for a
 * Toeplitz tridiagonal A with U_k generated on the fly from its eigenbasis; the threshold moves
 * with the environment variable HHL_TOEP_ROWS=<rows>); Strang-Trotter plans as grouped Strang
 * passes.
 * Errors: HHL_ERR_UNSUPPORTED unless full_uncompute = 0 and, for Strang-Trotter plans, every
 * clock bit's layer list fits one pass (2 r_k + 1 <= 17). */
hhl_status hhl_solve_postselected(hhl_plan_t plan, const double* b_dev, void* state_dev, double* out_dev,
                                  double* eps_dev, void* stream);

/* a6 - postselection statistics (Sec. II.A: the end solution read by measurement).
 * Asynchronous form: writes to out_dev (DEVICE, 4 + 2N doubles): [p_success, p_anc1,
 * norm, b_norm, xhat_0.re, xhat_0.im, ...], xhat = v / |v|. */
hhl_status hhl_measure_async(hhl_plan_t plan, const void* state_dev, double* out_dev, void* stream);

/* Synchronous form: fills *out; if x_host != NULL writes xhat (HOST, 2N doubles,
 * re/im interleaved). Synchronises the stream. HHL_ERR_SINGULAR if p_success = 0;
 * HHL_ERR_TIMEOUT / HHL_ERR_NUMERIC as hhl_plan_status. */
hhl_status hhl_measure(hhl_plan_t plan, const void* state_dev, hhl_measurement* out,
                       double* x_host, void* stream);

/* Device-side status of the last circuit on this plan (the bounded waits of Sec. IV's
 * controlled-U_k products on the tensor cores): synchronises the stream and returns HHL_OK,
 * HHL_ERR_TIMEOUT (a bounded wait of the tcgen05 GEMM ran out; its CTAs skipped the rest of
 * their tile after their copies and products in flight had drained, so the state is wrong but
 * the context is intact and the plan usable) or HHL_ERR_NUMERIC (an amplitude of magnitude
 * >= 2 reached the FP16 operands). The flag is cleared when a circuit starts
 * (hhl_apply_circuit, or hhl_apply_stage of HHL_STAGE_QPE_U), on the stream. Plans without
 * tcgen05 operands always report HHL_OK. */
hhl_status hhl_plan_status(hhl_plan_t plan, void* stream);

/* a6 - shots: the system register measured `shots` times after postselection (ancilla 1,
 * clock 0; Sec. II.A reads the solution by repeated measurement): outcome j with probability
 * |v_j|^2 / sum |v|^2, by inverse-transform sampling of the caller's uniforms:
 * shot s lands in the bin j with cdf_{j-1} <= u_s * cdf_{N-1} < cdf_j (cdf = running FP64 sum
 * of |v|^2). uniforms_dev: DEVICE, shots doubles in [0, 1) (the random numbers are inputs, so
 * the outcome is reproducible); counts_dev: DEVICE, N uint64 (overwritten). Asynchronous. */
hhl_status hhl_sample(hhl_plan_t plan, const void* state_dev, const double* uniforms_dev, int64_t shots,
                      uint64_t* counts_dev, void* stream);

/* a7 - in-situ viscous dissipation rate (Sec. VII, App. D: eps = nu <(du/dy)^2>, the
 * same finite-difference post-processing as the classical solution). The velocity is
 * u_i = |b| Re(v_i) / (C lambda_ub) at the N interior nodes, u_0 = wall_lo,
 * u_{N+1} = wall_hi, and eps = nu h sum_{i=0}^{N} ((u_{i+1} - u_i)/h)^2, h = 1/(N+1).
 * Asynchronous form writes eps to eps_dev (DEVICE, 1 double). */
hhl_status hhl_dissipation_async(hhl_plan_t plan, const void* state_dev, double* eps_dev, void* stream);

/* Synchronous form: *eps_out (HOST); if u_host != NULL also the N velocities (HOST). */
hhl_status hhl_dissipation(hhl_plan_t plan, const void* state_dev, double* eps_out,
                           double* u_host, void* stream);

/* ---------------------------------------------------------------------------------- batch
 * Many HHL instances of uneven size in one CUDA graph (growth direction of the path: the
 * paper's sweeps over T0, clock count and system size, Sec. VI, run as one batch). Every
 * instance is the postselected solve of hhl_solve_postselected in its dense form (complex64:
 * QPE by doubling and the uncompute by halving as controlled-U GEMMs on 2^k rows, tcgen05 where
 * 2^k >= 128, the clock block), with the outputs of hhl_measure_async and
 * hhl_dissipation_async; A must be a
 * Toeplitz tridiagonal matrix, because U_k is not stored but expanded from its analytic
 * eigenbasis (U_k[n][m] = g_k(|n-m|) - g_k(n+m)): hhl_batch_create computes the g_k of every
 * instance (an O(N^2) FP64 kernel per k, kept on the device as double-float pairs), and each
 * run generates U_k from them on the fly (tree steps below 128 rows) or expands it into a
 * per-stream GEMM operand right before its product. */
typedef struct hhl_batch_s* hhl_batch_t;

typedef struct hhl_batch_info {
  int32_t count;            /* instances */
  int32_t streams;          /* worker streams of the graph */
  uint64_t state_bytes;     /* all instance states (device) */
  uint64_t workspace_bytes; /* per-stream operand and row buffers (device) */
  double gemm_flops;        /* algorithmic flops of all controlled products of one run */
  uint64_t graph_launches;  /* kernels in the graph (0 before the first run) */
  int64_t b_doubles;        /* length of the packed right-hand-side array */
  int64_t out_doubles;      /* length of the packed measurement array */
} hhl_batch_info;

/* probs[count], params[count] (HOST, read during the call). gemm_choice[count] (HOST, may be
 * NULL): 0 = CUDA-core GEMM, 128 / 256 = tcgen05 GEMM with that tile width (ignored where the
 * tile does not fit); NULL picks by size. streams: worker streams (<= 0: 8). Instances are
 * assigned to streams by decreasing GEMM work. Allocates every state and workspace. */
hhl_status hhl_batch_create(const hhl_problem* probs, const hhl_params* params, int32_t count,
                            const int32_t* gemm_choice, int32_t streams, hhl_batch_t* out);
/* hhl_batch_create with the library's GEMM choice per instance and 8 worker streams, under the
 * name of the hot-path contract. */
hhl_status hhl_batch_plan(const hhl_problem* probs, const hhl_params* params, int32_t count, hhl_batch_t* out);
void hhl_batch_destroy(hhl_batch_t batch);
hhl_status hhl_batch_get_info(hhl_batch_t batch, hhl_batch_info* info);
/* Per instance: register sizes, chosen GEMM, offsets into the packed arrays, T0. */
hhl_status hhl_batch_instance(hhl_batch_t batch, int32_t index, int32_t* n_sys_qubits, int32_t* n_clock,
                              int32_t* gemm, int64_t* b_offset, int64_t* out_offset, double* t0);
/* Run every instance. b_dev: DEVICE packed complex128 right-hand sides (instance i at its
 * b_offset, N_i complex values). out_dev: DEVICE packed blocks of 4 + 2 N_i doubles in the
 * layout of hhl_measure_async; eps_dev: DEVICE count doubles (dissipation). The first call
 * captures the graph (so it must not itself be inside a stream capture); later calls replay
 * it with one launch. Asynchronous on stream. */
hhl_status hhl_batch_run(hhl_batch_t batch, const double* b_dev, double* out_dev, double* eps_dev, void* stream);
/* The same work enqueued launch by launch on the worker streams instead of replaying the
 * graph (for per-kernel timing with hhl_profile_*): reads the right-hand sides already in
 * the batch's device buffer (from the last run) and leaves the results there. */
hhl_status hhl_batch_run_eager(hhl_batch_t batch, void* stream);
/* As hhl_batch_run with HOST arrays (copies in and out on the stream, then synchronises);
 * returns the hhl_batch_status of the run. */
hhl_status hhl_batch_run_host(hhl_batch_t batch, const double* b_host, double* out_host, double* eps_host,
                              void* stream);
/* Device-side status of the last run (hhl_batch_run, _eager or _host), as hhl_plan_status:
 * synchronises the stream; HHL_OK, HHL_ERR_TIMEOUT or HHL_ERR_NUMERIC. Every run clears the
 * flag first, so a status describes that run alone; hhl_batch_run itself does not wait for
 * the GPU, so its results are valid only once this call returns HHL_OK. */
hhl_status hhl_batch_status(hhl_batch_t batch, void* stream);

/* ------------------------------------------------------------------- learned T0 predictor
 * A 6 -> 128 -> 128 -> 2 perceptron (tanh hidden layers) that maps features of the linear
 * system and the clock budget (kappa, N, the eigenvalue bounds and Q_PE that Sec. VI relates
 * to the optimal simulation time T0*) to (log of T0* over the power-law value, recommended
 * clock count), both standardised by the caller. BF16 weights with FP32 accumulation;
 * trained on the GPU by these entry points (forward, mean-squared-error loss, backward,
 * Adam). The parameter vector (HHL_MLP_PARAMS floats, host) is W1[128][6], b1[128],
 * W2[128][128], b2[128], W3[2][128], b3[2]. */
#define HHL_MLP_IN 6
#define HHL_MLP_HIDDEN 128
#define HHL_MLP_OUT 2
#define HHL_MLP_PARAMS 17666
typedef struct hhl_mlp_s* hhl_mlp_t;
hhl_status hhl_mlp_create(hhl_mlp_t* out);  /* parameters zero until hhl_mlp_set_params */
void hhl_mlp_destroy(hhl_mlp_t mlp);
/* Set the FP32 master parameters (HOST), reset the Adam state, refresh the BF16 copy. */
hhl_status hhl_mlp_set_params(hhl_mlp_t mlp, const float* host_params, void* stream);
hhl_status hhl_mlp_get_params(hhl_mlp_t mlp, float* host_params, void* stream);
/* y_dev[rows][2] = network(x_dev[rows][6]) (DEVICE, FP32). */
hhl_status hhl_mlp_forward(hhl_mlp_t mlp, const float* x_dev, int32_t rows, float* y_dev, void* stream);
/* The same network as the T0 predictor of the plan stage (features, outputs as above). */
hhl_status hhl_t0_predict(hhl_mlp_t mlp, const float* features_dev, int32_t rows, float* out_dev, void* stream);
/* Gradient of loss = mean((y - t)^2) over rows and outputs with respect to the parameters
 * (through the BF16 weights): grad_dev[HHL_MLP_PARAMS], loss_dev[1] (DEVICE). */
hhl_status hhl_mlp_gradients(hhl_mlp_t mlp, const float* x_dev, const float* t_dev, int32_t rows, float* grad_dev,
                             float* loss_dev, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on that loss; loss_dev[1]
 * receives the loss before the step. */
hhl_status hhl_mlp_train_step(hhl_mlp_t mlp, const float* x_dev, const float* t_dev, int32_t rows, float lr,
                              float* loss_dev, void* stream);

/* Fused gate block: QFT (inverse = 0) or inverse QFT (inverse = 1) on the m-qubit
 * register of bits [lo, lo + m) of an n-qubit state, in place (the QFT / IQFT subroutine
 * of the algorithm library, App. B; the circuit of the Fig. 1c scaling experiment).
 * precision: HHL_PREC_C64 or HHL_PREC_C128. Requires 1 <= m <= 13, lo + m <= n <= 34. */
hhl_status hhl_apply_qft(void* state_dev, int32_t n_qubits, int32_t lo, int32_t m,
                         int32_t inverse, int32_t precision, void* stream);

/* Whole-register QFT of the Fig. 1c experiment (the QFT-then-inverse-QFT circuit run on
 * random states as the paper's gate benchmark): on each of n_states consecutive n-qubit
 * states (state_dev holds n_states * 2^n amplitudes, n_states a power of two), in place,
 *   direction 0: QFT|x> = 2^(-n/2) sum_y e^{+2 pi i x y / 2^n}|y>, with the result left in
 *                bit-reversed order (amplitude of y at index bitrev_n(y)), i.e. the circuit
 *                without its final swap layer;
 *   direction 1: the inverse QFT reading its input in that bit-reversed order and writing
 *                natural order.
 * Direction 0 followed by direction 1 is the QFT-IQFT circuit (the identity up to rounding).
 * Requires 1 <= n <= 32, n + log2(n_states) <= 34; precision HHL_PREC_C64 or HHL_PREC_C128.
 * Asynchronous on stream; the first call for a given n builds a 48 KiB (c64) twiddle table
 * on the device, kept until exit. */
hhl_status hhl_qft_whole(void* state_dev, int32_t n_qubits, int32_t n_states, int32_t direction, int32_t precision,
                         void* stream);

/* Number of kernels this library has launched since load (all entry points). */
uint64_t hhl_kernel_launch_count(void);

/* Testing the timeout path: with the environment variable HHL_FAULT=tc_wait set when a
 * tcgen05 GEMM is launched (or a batch graph is captured), that GEMM issues no operand copy
 * and bounds its waits by about a millisecond, so it ends with HHL_ERR_TIMEOUT (no copy or
 * product in flight when its waits run out). HHL_FAULT=alloc|plan|launch inject host failures
 * (HHL_ERR_OOM, HHL_ERR_INVALID_ARG, HHL_ERR_CUDA) into allocation, planning and launches. */

/* Clock-controlled U for callers that cannot allocate device memory while they run (the
 * paper has no counterpart; this is an interface convenience). Hosts that hand all device
 * memory to their own pool allocator, or loops that cannot afford the device-wide
 * synchronisation cudaMalloc / cudaFree may cause, call this instead of a plan: it applies
 * r <- U r (adjoint = 0) or r <- U^dagger r (adjoint = 1) to every row r of half_dev whose
 * clock bit k is set, and calls no cudaMalloc, cudaFree or allocating library routine.
 *   u_dev:    DEVICE complex64, N x N row-major, U[n][m] at n*N + m (N = 2^n_sys_qubits).
 *   half_dev: DEVICE complex64, one ancilla half: 2^n_clock rows of N (in place).
 * The product rows are staged in one fixed 8 MiB device array inside the library (held on
 * every GPU that loads it, until exit); requests needing more than 2^20 complex64 values
 * (2^(n_clock-1) * N) are rejected with HHL_ERR_INVALID_ARG. The first call on each device
 * looks up that array's device address (set-up), so make it before any stream capture; the
 * address is kept per device and CUDA context, so after a device reset the next call looks it
 * up again (again before any capture).
 * Each call overwrites the staging space before reading it; calls that may overlap on the
 * GPU (unordered streams) share the array and race. Asynchronous on `stream`. */
hhl_status hhl_controlled_u_noalloc(const void* u_dev, void* half_dev, int32_t n_sys_qubits, int32_t n_clock,
                                    int32_t k, int32_t adjoint, void* stream);

/* Per-kernel device timing (tracing). While enabled, every kernel launch is bracketed by
 * a pair of CUDA events on its stream; reading the profile waits for those events and
 * folds them into per-kernel totals (launch count, summed milliseconds). Process-wide,
 * off by default; enabling adds two event records per launch. */
void hhl_profile_enable(int32_t on);
void hhl_profile_reset(void);
int32_t hhl_profile_count(void);
/* Entry `index` (0 .. count-1, sorted by kernel name): name copied NUL-terminated into
 * name[name_len]; launches and total_ms may be NULL. */
hhl_status hhl_profile_get(int32_t index, char* name, int32_t name_len, uint64_t* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* HHL_H_ */
