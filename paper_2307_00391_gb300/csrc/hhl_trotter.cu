// Controlled exp(i Ahat t_k) as a second-order Strang product of two-level gates, for a
// Toeplitz tridiagonal Ahat (the channel-flow operator of App. A.1 Eq. CDS).
//
// Ahat = E + O: E holds the 2x2 blocks [[d, o], [o, d]] on basis-state pairs (2i, 2i+1),
// O the couplings [[0, o], [o, 0]] on pairs (2i+1, 2i+2). One Strang step is
// S(tau) = E(tau/2) O(tau) E(tau/2) with E(s) = exp(i s E), and r steps merge into the
// layer list E(tau/2), O(tau), [E(tau), O(tau)] x (r-1), E(tau/2) (2r + 1 layers).
//
// Every layer acts inside one system-register row, so a pass applies up to 17 layers to a
// window of the row held in registers (temporal blocking): one warp owns 512 consecutive
// amplitudes, 16 per lane, so E pairs and all but one O pair per lane are in the lane's
// own registers and the remaining O pair crosses to the next lane by a warp shuffle. The
// window has a 16-amplitude halo on each side (lanes 0 and 31), and its 480-amplitude
// interior (lanes 1..30) is written back in place.
// The halos are the edges of the neighbouring interiors, which the same pass overwrites in
// place. Each warp owns a contiguous run of windows and walks it in order, so the left halo
// of a window is the original right end of the interior the warp loaded just before (carried
// in shared memory) and its right halo is the start of the next interior, which no one has
// written yet; only the halos across the boundaries between two warps' runs are saved before
// the pass, by a small kernel, into a side buffer. Each pass moves its rows through HBM once.
//
// A 16-amplitude halo is exact for up to 17 layers when the first layer is an E layer: the
// E pairs never cross the window edge, and each later layer moves the wrong values in from
// the edge by one amplitude. Several clock bits share one pass: the controlled products of
// QPE act on a clock row in bit order, and a row whose bits k1 < k2 < ... (within a group of
// consecutive bits) are set gets U_k1, then U_k2, ..., applied to its system amplitudes, which
// a pass over every row with some bit of the group set can do with the row's own layer list
// (the trailing E(tau_k1 / 2) and leading E(tau_k2 / 2) merge into one E layer, since E
// layers commute). Bits are grouped while the all-bits-set list stays within 17 layers; a
// bit whose own list is longer gets passes over windows of its layers. For the 32-qubit
// Poiseuille case (r_k = 1 for k < 8) 13 single-bit passes over half the rows each become 5
// passes, 3 of them over half the rows.
//
// Warps are persistent: the windows of the pass (rows with a nonzero pattern only, so that
// every window is work) are split into one contiguous run per warp, and the 16-byte copies
// of a warp's next window go into a second staging buffer with cp.async while it computes
// the current one.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kLaneAmps = 16;                 // amplitudes per lane (8 in the double-float kernel)
constexpr int kHalo = 16;                     // halo per side = max layers per pass
constexpr int kWin = 32 * kLaneAmps;          // 512 amplitudes per warp window
constexpr int kInterior = kWin - 2 * kHalo;   // 480 written back per warp
constexpr int kTrotThreads = 256;
constexpr int kMaxPassLayers = kHalo + 1;     // exact with a kHalo halo when layer 0 is E
constexpr int64_t kMaxRuns = 1 << 16;         // warps of one pass (the side buffer holds 32 amplitudes each)

// Window geometry for LA amplitudes per lane: HL = kHalo / LA halo lanes on each side,
// 32 LA amplitudes per window, 32 LA - 2 kHalo of them interior.
template <int LA>
struct Geo {
  static constexpr int HL = kHalo / LA;
  static constexpr int WIN = 32 * LA;
  static constexpr int INTER = WIN - 2 * kHalo;
};

// A layer list also carries each rotation in factored form, used by windows away from the
// row ends: with |cos th| >= |sin th| (form 0)
//   (a, b) <- (a + i w b, b + i w a) = R(th) (a, b) / cos th,        w = tan th,
// else (form 1)
//   (a, b) <- (b + i w a, a + i w b) = R(th) (a, b) / (i sin th),    w = -cot th,
// two FMAs per output component instead of four, |w| <= 1; the product of the factors is
// folded into the end-of-pass scalar (pc2, ps2). (At the row ends an amplitude without an O
// partner would need the inverse factor, so those windows keep the plain rotations.)
struct LayerList {
  int n;                   // layers (<= kMaxPassLayers)
  int first_o;             // 1 if layer 0 is an O layer
  double pc, ps;           // the pattern's summed E phase e^{i d (E time)} in this pass
  double c[kMaxPassLayers], s[kMaxPassLayers];  // cos / sin of each layer's rotation angle
  double w[kMaxPassLayers];                     // factored form
  int form[kMaxPassLayers];
  double pc2, ps2;                              // the phase times the product of the factors
  // the same values rounded to FP32 on the host (GB300's FP64 conversions are slow)
  float pcf, psf, pc2f, ps2f;
  float cf[kMaxPassLayers], sf[kMaxPassLayers], wf[kMaxPassLayers];
  // and the FP32 remainders (value - rounded value) of the double-float complex128 kernel
  float pcl, psl, pc2l, ps2l;
  float cl[kMaxPassLayers], sl[kMaxPassLayers], wl[kMaxPassLayers];
};

// Arithmetic of the pass in registers. V is the amplitude type the layers work on, W its
// real scalar: complex64 amplitudes in float2 / float; complex128 amplitudes either in
// double2 / double (FP64 pipe) or, by default, in double-float dfc / df (FP32 pipe, the
// FP64 amplitudes split on load and rebuilt on store: GB300's FP64 pipe is about 1/32 of
// the FP32 one, so the FP64 form of this pass is compute bound at about ten times its memory
// time).
template <class R, bool DF> struct TrotArith;
template <> struct TrotArith<float, false> {
  using T = float2;
  using V = float2;
  using W = float;
  static __device__ __forceinline__ V load(T t) { return t; }
  static __device__ __forceinline__ T store(V v) { return v; }
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ W coef(const float* f, const float*, const double*, int l) { return f[l]; }
  static __device__ __forceinline__ W coef1(float f, float, double) { return f; }
  static __device__ __forceinline__ V finish(V v) { return v; }
};
template <> struct TrotArith<double, false> {
  using T = double2;
  using V = double2;
  using W = double;
  static __device__ __forceinline__ V load(T t) { return t; }
  static __device__ __forceinline__ T store(V v) { return v; }
  static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ W coef(const float*, const float*, const double* d, int l) { return d[l]; }
  static __device__ __forceinline__ W coef1(float, float, double d) { return d; }
  static __device__ __forceinline__ V finish(V v) { return v; }
};
template <> struct TrotArith<double, true> {
  using T = double2;
  using V = dfc;
  using W = df;
  static __device__ __forceinline__ V load(T t) { return dfc_from(t); }
  static __device__ __forceinline__ T store(V v) { return dfc_to(v); }
  static __device__ __forceinline__ V zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
  static __device__ __forceinline__ W coef(const float* f, const float* fl, const double*, int l) { return {f[l], fl[l]}; }
  static __device__ __forceinline__ W coef1(float f, float fl, double) { return {f, fl}; }
  // (no renormalisation needed: the lazy phase product and the exact FP64 rebuild on the store
  // take any head and tail)
  static __device__ __forceinline__ V finish(V v) { return v; }
};

// p + i w q = (p.x - w q.y, p.y + w q.x): one output of the factored two-FMA rotation
__device__ __forceinline__ float2 fac1(float2 p, float2 q, float w) { return make_float2(p.x - w * q.y, p.y + w * q.x); }
__device__ __forceinline__ double2 fac1(double2 p, double2 q, double w) {
  return make_double2(p.x - w * q.y, p.y + w * q.x);
}
__device__ __forceinline__ dfc fac1(dfc p, dfc q, df w) { return {df_fnma_lazy(w, q.y, p.x), df_fma_lazy(w, q.x, p.y)}; }
// c p + i s q: one output of the plain rotation R(th) = [[c, i s], [i s, c]]
__device__ __forceinline__ float2 rot1(float2 p, float2 q, float c, float s) {
  return make_float2(c * p.x - s * q.y, c * p.y + s * q.x);
}
__device__ __forceinline__ double2 rot1(double2 p, double2 q, double c, double s) {
  return make_double2(c * p.x - s * q.y, c * p.y + s * q.x);
}
__device__ __forceinline__ dfc rot1(dfc p, dfc q, df c, df s) {
  return {df_fnma_lazy(s, q.y, df_mul(c, p.x)), df_fma_lazy(s, q.x, df_mul(c, p.y))};
}
__device__ __forceinline__ float2 phase_mul(float2 a, float2 b) { return cmul(a, b); }
__device__ __forceinline__ double2 phase_mul(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ dfc phase_mul(dfc a, dfc b) { return cmul(a, b); }  // lazy double-float operators

__device__ __forceinline__ int64_t row_with_bit_t(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}

__device__ __forceinline__ float shfl_d(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_d(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ df shfl_d(df v) { return {shfl_d(v.h), shfl_d(v.l)}; }
__device__ __forceinline__ float shfl_u(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_u(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ df shfl_u(df v) { return {shfl_u(v.h), shfl_u(v.l)}; }
template <class V>
__device__ __forceinline__ V shfl_down1(V v) {
  V r;
  r.x = shfl_d(v.x);
  r.y = shfl_d(v.y);
  return r;
}
template <class V>
__device__ __forceinline__ V shfl_up1(V v) {
  V r;
  r.x = shfl_u(v.x);
  r.y = shfl_u(v.y);
  return r;
}

// (a, b) <- (a + i w b, b + i w a), or with SWAP (b + i w a, a + i w b).
template <bool SWAP, class V, class W>
__device__ __forceinline__ void rot_factored(V& a, V& b, W w) {
  const V na = fac1(a, b, w);
  const V nb = fac1(b, a, w);
  a = SWAP ? nb : na;
  b = SWAP ? na : nb;
}

// All layers of a list on a window away from the row ends, in factored form (the result is
// off by the product of the factors, applied with the end-of-pass scalar).
template <bool SWAP, int LA, class V, class W>
__device__ __forceinline__ void layer_factored(V (&x)[LA], bool e_layer, W w) {
  if (e_layer) {
#pragma unroll
    for (int q = 0; q < LA; q += 2) rot_factored<SWAP>(x[q], x[q + 1], w);
  } else {
    const V right = shfl_down1(x[0]);    // next lane's first amplitude
    const V left = shfl_up1(x[LA - 1]);  // previous lane's last amplitude
#pragma unroll
    for (int q = 1; q + 1 < LA; q += 2) rot_factored<SWAP>(x[q], x[q + 1], w);
    const V a = x[LA - 1], b = x[0];
    // (this lane's last a, next lane's first) and (previous lane's last, this lane's first b)
    x[LA - 1] = SWAP ? fac1(right, a, w) : fac1(a, right, w);
    x[0] = SWAP ? fac1(left, b, w) : fac1(b, left, w);
  }
}

// The double-float kernel writes the second form without the exchange of its two outputs:
// R(th) (a, b) / sin th = (v a + i b, v b + i a), v = cot th = -w, so that both forms are one
// fused multiply-add per output component with the operands in place, and its factors are
// sin th instead of i sin th (the end-of-pass scalar is multiplied by (-i)^(number of such
// layers)). One layer per loop iteration with a branch on the form keeps four copies of the
// layer code (E / O, two forms): the fully unrolled double-float arithmetic of the paired
// loop above overflows the instruction cache (measured: issue stalled on instruction fetch).
__device__ __forceinline__ dfc fac2(dfc p, dfc q, df v) {  // v p + i q
  return {df_fma_lazy(v, p.x, df_neg(q.y)), df_fma_lazy(v, p.y, q.x)};
}
template <bool F1>
__device__ __forceinline__ void rot_factored_df(dfc& a, dfc& b, df w) {
  if (F1) {
    const dfc na = fac2(a, b, w), nb = fac2(b, a, w);
    a = na;
    b = nb;
  } else {
    const dfc na = fac1(a, b, w), nb = fac1(b, a, w);
    a = na;
    b = nb;
  }
}
template <bool F1, int LA>
__device__ __forceinline__ void layer_df(dfc (&x)[LA], bool e_layer, df w) {
  if (e_layer) {
#pragma unroll
    for (int q = 0; q < LA; q += 2) rot_factored_df<F1>(x[q], x[q + 1], w);
  } else {
    const dfc right = shfl_down1(x[0]);
    const dfc left = shfl_up1(x[LA - 1]);
#pragma unroll
    for (int q = 1; q + 1 < LA; q += 2) rot_factored_df<F1>(x[q], x[q + 1], w);
    // (this lane's last a, next lane's first) and (previous lane's last, this lane's first b)
    x[LA - 1] = F1 ? fac2(x[LA - 1], right, w) : fac1(x[LA - 1], right, w);
    x[0] = F1 ? fac2(x[0], left, w) : fac1(x[0], left, w);
  }
}

// Rotations R(th) = [[cos th, i sin th], [i sin th, cos th]]: E(s) = exp(i s E) is
// e^{i s d} R(s o) on the E pairs and O(s) = exp(i s O) is R(s o) on the O pairs. A row
// pattern's layers in one pass: their rotations and the summed E phase, applied once at
// the end of the pass (it is a scalar on the row).
// (a, b) <- R(th) (a, b) with c = cos th, s = sin th.
template <class V, class W>
__device__ __forceinline__ void rot_apply(V& a, V& b, W c, W s) {
  const V na = rot1(a, b, c, s);
  const V nb = rot1(b, a, c, s);
  a = na;
  b = nb;
}

// The layer coefficients of the row pattern a warp is on (per warp, in shared memory).
template <class W>
struct LayerCoefs {
  W c[32], s[32], w[32];
  int form[32];
};

// Rows of a pass: single_k >= 0 enumerates the 2^(n_c - 1) rows with clock bit single_k set
// (pattern 1); otherwise the rows whose pattern, clock bits [kb, kb + gbits), is nonzero:
// pass row i = (hi, pattern - 1, lo) in mixed radix (.., 2^gbits - 1, 2^kb).
__device__ __forceinline__ void pass_row(int64_t i, int single_k, int kb, int gbits, int64_t* row, int* pattern) {
  if (single_k >= 0) {
    *row = row_with_bit_t(i, single_k);
    *pattern = 1;
  } else {
    const int64_t M = (1LL << gbits) - 1;
    const int64_t lo = i & ((1LL << kb) - 1), t = i >> kb;
    const int64_t hi = t / M;
    const int pat = (int)(1 + t - hi * M);
    *row = lo | ((int64_t)pat << kb) | (hi << (kb + gbits));
    *pattern = pat;
  }
}

// The run of warp gw < nruns (nruns <= windows, so no run is empty): windows
// [run_start(gw), run_start(gw + 1)) of the pass, window v = i * segs + s (pass row i,
// segment s).
__device__ __forceinline__ int run_start(int gw, int windows, int nruns) {
  return (int)((int64_t)gw * windows / nruns);
}

// side[gw * 32 + q] for the boundary between the runs of warps gw - 1 and gw (window
// v = run_start(gw) and v - 1, when both lie in one row): q < 16 the first 16 interior
// amplitudes of window v (the right halo of v - 1), q >= 16 the last 16 of window v - 1 (the
// left halo of v); zero beyond the row end.
template <class R, int LA>
__global__ void k_trotter_bounds(const typename Cx<R>::T* __restrict__ half, typename Cx<R>::T* __restrict__ side,
                                 int n_s, int segs, int windows, int nruns, int single_k, int kb, int gbits) {
  constexpr int kInterior = Geo<LA>::INTER;
  const int64_t N = 1LL << n_s;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nruns * 32) return;
  const int gw = e >> 5, q = e & 31;
  if (gw == 0) return;
  const int v = run_start(gw, windows, nruns);
  const int i = v / segs;
  const int s = v - i * segs;
  if (s == 0) return;  // a row boundary: the halos are zero
  int64_t row;
  int pattern;
  pass_row(i, single_k, kb, gbits, &row, &pattern);
  const int64_t g = q < 16 ? (int64_t)s * kInterior + q : (int64_t)s * kInterior - 32 + q;
  side[e] = g < N ? half[row * N + g] : mk<R>((R)0, (R)0);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// One warp window: pass row i, segment s; first / last: the first / last window of the
// warp's run (its left / right halo then comes from the side buffer, unless at a row end).
struct Window {
  int i, s;
  int64_t row;
  int pattern;
  bool full;  // the 480-amplitude interior lies inside the row
  bool first, last;
};

// Staging buffer of a warp: 32 x LA amplitudes as 16-byte chunks, window chunk c stored at
// position c ^ ((c / CPL) & 7) (CPL = chunks per lane) so that both the coalesced copy (lane t
// <-> chunk q * 32 + t) and the per-lane gather (lane t <-> its CPL consecutive chunks) spread
// over the banks. The first HL lanes' chunks hold the left halo (16 amplitudes), the last HL
// lanes' the right one. The left halo of a window inside a run is not copied here: the
// previous iteration puts the carried amplitudes there (carry_copy).
template <int CPL>
__device__ __forceinline__ int swz(int c) {
  return c ^ ((c / CPL) & 7);
}
template <class T, int LA>
__device__ __forceinline__ void stage_issue(uint4* stage, const Window& d, const T* half, const T* side, int gw,
                                            int segs, int64_t N, int lane) {
  constexpr int per = 16 / sizeof(T);
  constexpr int CPL = LA / per;
  constexpr int HC = kHalo / per;  // chunks of one halo
  constexpr int kInterior = Geo<LA>::INTER;
  if (!d.full) return;
  const uint4* src = reinterpret_cast<const uint4*>(half + d.row * N + (int64_t)d.s * kInterior);
  constexpr int chunks = kInterior / per;
#pragma unroll
  for (int q = 0; q < (chunks + 31) / 32; ++q) {
    const int c = q * 32 + lane;
    if (c < chunks) cp_async16(&stage[swz<CPL>(c + HC)], src + c);
  }
  if (lane < HC) {  // left halo chunk `lane`
    if (d.s == 0) stage[swz<CPL>(lane)] = make_uint4(0u, 0u, 0u, 0u);
    else if (d.first) cp_async16(&stage[swz<CPL>(lane)], reinterpret_cast<const uint4*>(side + (int64_t)gw * 32 + 16) + lane);
  } else if (lane >= 32 - HC) {  // right halo chunk q
    const int q = lane - (32 - HC);
    const int pos = swz<CPL>(HC + chunks + q);
    if (d.s == segs - 1) {
      stage[pos] = make_uint4(0u, 0u, 0u, 0u);
    } else if (d.last) {
      cp_async16(&stage[pos], reinterpret_cast<const uint4*>(side + (int64_t)(gw + 1) * 32) + q);
    } else {
      // the start of the next interior, unwritten until this warp gets there
      const int64_t a0 = (int64_t)(d.s + 1) * kInterior;
      if (a0 + (int64_t)(q + 1) * per <= N) cp_async16(&stage[pos], reinterpret_cast<const uint4*>(half + d.row * N + a0) + q);
      else stage[pos] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// The left halo of the next window of the run (same row): the original last 16 interior
// amplitudes of the current, full window into the left-halo chunks of the next staging buffer.
template <int CPL, int HC, int CHUNKS>
__device__ __forceinline__ void carry_copy(uint4* next_stage, const uint4* stage, int lane) {
  if (lane < HC) next_stage[swz<CPL>(lane)] = stage[swz<CPL>(CHUNKS + lane)];
}

// The window after d in its run (window v of the pass; the run ends before v1).
template <int LA>
__device__ __forceinline__ Window window_next(Window d, int v, int v1, int segs, int64_t N, int single_k, int kb,
                                              int gbits) {
  constexpr int kInterior = Geo<LA>::INTER;
  d.first = false;
  d.last = v + 2 == v1;
  if (++d.s == segs) {
    d.s = 0;
    ++d.i;
    pass_row(d.i, single_k, kb, gbits, &d.row, &d.pattern);
  }
  d.full = (int64_t)d.s * kInterior + kInterior <= N;
  return d;
}

// Persistent warps: each warp walks its run of windows in order; the copies of its next
// window go to the second staging buffer (cp.async) while it computes the current. (The next
// window is formed again after the current one is done, so that it holds no registers
// during the layers.) 16 warps per SM with up to 128 registers each: the paired layers need
// them (with 24 warps and 80 registers the pass spilled and ran 10% slower).
// The layers of one row pattern and its end-of-pass phase on a window held in registers:
// the factored forms on windows away from the row ends (`away`, warp-uniform), the plain
// rotations with per-pair validity near them. lane0: the row index of this lane's first
// amplitude; coef: the pattern's coefficients (per warp, in shared memory); L: its list.
template <class R, bool DF, int LA>
__device__ __forceinline__ void apply_pattern(typename TrotArith<R, DF>::V (&x)[LA],
                                              const LayerCoefs<typename TrotArith<R, DF>::W>* coef,
                                              const LayerList* L, int n_layers, int first_o, bool away, int64_t lane0,
                                              int64_t N, int lane) {
  using A = TrotArith<R, DF>;
  using V = typename A::V;
  using W = typename A::W;
  int n_f1 = 0;  // double-float kernel: layers in the second form
  if constexpr (DF) {
    if (away) {
      for (int l = 0; l < n_layers; ++l) {
        const bool e_layer = ((l + first_o) & 1) == 0;
        const int f1 = coef->form[l];
        n_f1 += f1;
        if (f1) layer_df<true>(x, e_layer, df_neg(coef->w[l]));
        else layer_df<false>(x, e_layer, coef->w[l]);
      }
    }
  } else if (away) {
    // layers alternate E, O: an O layer first on its own, then (E, O) pairs in one loop
    // body (the pair's second layer writes its outputs back into the registers the loop
    // carries, so no register copies are needed between layers), then a last E layer
    int l = 0;
    if (first_o && n_layers > 0) {
      if (coef->form[0] != 0) layer_factored<true, LA>(x, false, coef->w[0]);
      else layer_factored<false, LA>(x, false, coef->w[0]);
      l = 1;
    }
    for (; l + 1 < n_layers; l += 2) {
      const W we = coef->w[l], wo = coef->w[l + 1];
      if (coef->form[l] != 0) {
        layer_factored<true, LA>(x, true, we);
        if (coef->form[l + 1] != 0) layer_factored<true, LA>(x, false, wo);
        else layer_factored<false, LA>(x, false, wo);
      } else {
        layer_factored<false, LA>(x, true, we);
        if (coef->form[l + 1] != 0) layer_factored<true, LA>(x, false, wo);
        else layer_factored<false, LA>(x, false, wo);
      }
    }
    if (l < n_layers) {
      if (coef->form[l] != 0) layer_factored<true, LA>(x, true, coef->w[l]);
      else layer_factored<false, LA>(x, true, coef->w[l]);
    }
  }
  // per-lane validity of the O pairs (j, j+1), j odd, 1 <= j and j + 1 <= N - 1
  const bool in_ok = lane0 >= 0 && lane0 + LA - 2 <= N - 1;
  const bool right_ok = lane < 31 && lane0 + LA - 1 >= 1 && lane0 + LA <= N - 1;
  const bool left_ok = lane > 0 && lane0 - 1 >= 1 && lane0 <= N - 1;
  for (int l = 0; l < (away ? 0 : n_layers); ++l) {
    const W c = coef->c[l], sn = coef->s[l];
    if (((l + first_o) & 1) == 0) {
      // E layer: pairs (2p, 2p+1) inside each lane; pairs beyond the row are zero.
#pragma unroll
      for (int q = 0; q < LA; q += 2) rot_apply(x[q], x[q + 1], c, sn);
    } else {
      const V right = shfl_down1(x[0]);           // next lane's first amplitude
      const V left = shfl_up1(x[LA - 1]);  // previous lane's last amplitude
      if (in_ok && !DF) {  // (the double-float kernel keeps one copy of this rare path)
#pragma unroll
        for (int q = 1; q + 1 < LA; q += 2) rot_apply(x[q], x[q + 1], c, sn);
      } else {
#pragma unroll
        for (int q = 1; q + 1 < LA; q += 2) {
          const int64_t j = lane0 + q;
          if (j >= 1 && j + 1 <= N - 1) rot_apply(x[q], x[q + 1], c, sn);
        }
      }
      if (right_ok) x[LA - 1] = rot1(x[LA - 1], right, c, sn);  // a <- c a + i s b
      if (left_ok) x[0] = rot1(x[0], left, c, sn);                            // b <- i s a + c b
    }
  }
  {
    V ph;
    if (away) {
      ph.x = A::coef1(L->pc2f, L->pc2l, L->pc2);
      ph.y = A::coef1(L->ps2f, L->ps2l, L->ps2);
      if constexpr (DF) {
        // (-i)^n_f1: the second form's factors are sin th, not i sin th
        for (int j = 0; j < (n_f1 & 3); ++j) {
          const auto t = ph.x;
          ph.x = ph.y;
          ph.y = df_neg(t);
        }
      }
    } else {
      ph.x = A::coef1(L->pcf, L->pcl, L->pc);
      ph.y = A::coef1(L->psf, L->psl, L->ps);
    }
#pragma unroll
    for (int q = 0; q < LA; ++q) x[q] = phase_mul(A::finish(x[q]), ph);
  }
}

// Threads per block: 256. Blocks per SM: 2 for complex64 (128 registers), 1 for the FP64 form
// of complex128, 3 for the double-float form (8 amplitudes per lane: two 4 KiB staging buffers
// per warp, 80 registers, 24 warps per SM to hide its latencies).
template <class R, bool DF>
constexpr int trot_threads() { return kTrotThreads; }
template <class R, bool DF>
constexpr int trot_min_blocks() { return DF ? 3 : (sizeof(R) == 4 ? 2 : 1); }
// Amplitudes per lane: 16; 8 in the double-float kernel (its unrolled layer code for 16 per
// lane, about 60 KB per window, missed the instruction cache: measured, issue stalled on
// instruction fetch; 8 per lane halve the code and the registers at 2 halo lanes per side).
template <class R, bool DF>
constexpr int trot_lane_amps() { return DF ? 8 : kLaneAmps; }

template <class R, bool DF>
__global__ void __launch_bounds__(trot_threads<R, DF>(), trot_min_blocks<R, DF>()) k_trotter_pass(typename Cx<R>::T* __restrict__ half,
                                                              const typename Cx<R>::T* __restrict__ side, int n_s,
                                                              int segs, int windows, int nruns, int single_k,
                                                              int kb, int gbits, const LayerList* __restrict__ lists) {
  using A = TrotArith<R, DF>;
  using T = typename A::T;
  using V = typename A::V;
  using W = typename A::W;
  constexpr int LA = trot_lane_amps<R, DF>();
  constexpr int HL = Geo<LA>::HL;
  constexpr int kInterior = Geo<LA>::INTER;
  constexpr int per = 16 / sizeof(T);  // amplitudes per 16-byte unit
  constexpr int CPL = LA / per;
  constexpr int HC = kHalo / per;
  constexpr int CHUNKS = kInterior / per;
  constexpr int WPB = trot_threads<R, DF>() / 32;  // warps per block
  extern __shared__ __align__(16) unsigned char trot_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint4* stage_w = reinterpret_cast<uint4*>(trot_smem) + (size_t)wid * 2 * 32 * CPL;  // two buffers
  LayerCoefs<W>* coef =
      reinterpret_cast<LayerCoefs<W>*>(reinterpret_cast<uint4*>(trot_smem) + (size_t)WPB * 2 * 32 * CPL) + wid;
  const int64_t N = 1LL << n_s;
  const int gw = (int)blockIdx.x * WPB + wid;
  if (gw >= nruns) return;  // warp-uniform
  const int v0 = run_start(gw, windows, nruns), v1 = run_start(gw + 1, windows, nruns);
  Window cur;
  cur.i = v0 / segs;
  cur.s = v0 - cur.i * segs;
  pass_row(cur.i, single_k, kb, gbits, &cur.row, &cur.pattern);
  cur.full = (int64_t)cur.s * kInterior + kInterior <= N;
  cur.first = true;
  cur.last = v0 + 1 == v1;
  stage_issue<T, LA>(stage_w, cur, half, side, gw, segs, N, lane);
  cp_async_commit();
  int buf = 0;
  int cached = 0, n_layers = 0, first_o = 0;  // the row pattern whose layers coef holds (patterns are >= 1)
  for (int v = v0; v < v1; ++v) {
    const bool more = v + 1 < v1;
    if (more)
      stage_issue<T, LA>(stage_w + (buf ^ 1) * 32 * CPL, window_next<LA>(cur, v, v1, segs, N, single_k, kb, gbits), half, side,
                     gw, segs, N, lane);
    cp_async_commit();
    cp_async_wait1();  // the current window's copies have landed
    __syncwarp();
    {
      uint4* stage = stage_w + buf * 32 * CPL;
      // a full window followed by the next segment of its row: carry the left halo over
      if (more && cur.s + 1 < segs) carry_copy<CPL, HC, CHUNKS>(stage_w + (buf ^ 1) * 32 * CPL, stage, lane);
      const LayerList* L = lists + cur.pattern;
      if (cur.pattern != cached) {  // a new row pattern (runs change rows rarely)
        cached = cur.pattern;
        n_layers = L->n;
        first_o = L->first_o;
        if (lane < n_layers) {
          coef->c[lane] = A::coef(L->cf, L->cl, L->c, lane);
          coef->s[lane] = A::coef(L->sf, L->sl, L->s, lane);
          coef->w[lane] = A::coef(L->wf, L->wl, L->w, lane);
          coef->form[lane] = L->form[lane];
        }
        __syncwarp();
      }
      const int64_t g0 = (int64_t)cur.s * kInterior;        // first interior amplitude
      const int64_t lane0 = g0 - kHalo + (int64_t)lane * LA;  // even
      const bool interior = lane >= HL && lane < 32 - HL;
      T* row = half + cur.row * N;
      V x[LA];
      if (cur.full) {
        T t[LA];
        uint4* d = reinterpret_cast<uint4*>(t);
#pragma unroll
        for (int q = 0; q < CPL; ++q) d[q] = stage[(lane * CPL + q) ^ (lane & 7)];
#pragma unroll
        for (int q = 0; q < LA; ++q) x[q] = A::load(t[q]);
      } else {
        if (interior) {
#pragma unroll
          for (int q = 0; q < LA; ++q) x[q] = lane0 + q < N ? A::load(row[lane0 + q]) : A::zero();
        } else if (lane < HL && cur.s > 0) {
          // the left halo: from the side buffer at the start of the run, else carried
          if (cur.first) {
#pragma unroll
            for (int q = 0; q < LA; ++q) x[q] = A::load(side[(int64_t)gw * 32 + 16 + lane * LA + q]);
          } else {
            T t[LA];
            uint4* d = reinterpret_cast<uint4*>(t);
#pragma unroll
            for (int q = 0; q < CPL; ++q) d[q] = stage[(lane * CPL + q) ^ (lane & 7)];
#pragma unroll
            for (int q = 0; q < LA; ++q) x[q] = A::load(t[q]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < LA; ++q) x[q] = A::zero();  // beyond the row ends
        }
      }
      __syncwarp();
      // warp-uniform: every O pair of the interior lanes lies inside the row (no row end in
      // the window but possibly the halos', whose values do not reach the interior)
      const bool away = cur.full && g0 >= 2 && g0 + kInterior + 1 <= N;
      apply_pattern<R, DF, LA>(x, coef, L, n_layers, first_o, away, lane0, N, lane);
      if (cur.full) {
        if (interior) {
          T t[LA];
#pragma unroll
          for (int q = 0; q < LA; ++q) t[q] = A::store(x[q]);
          const uint4* sx = reinterpret_cast<const uint4*>(t);
#pragma unroll
          for (int q = 0; q < CPL; ++q) stage[(lane * CPL + q) ^ (lane & 7)] = sx[q];
        }
        __syncwarp();
        uint4* dst = reinterpret_cast<uint4*>(row + g0);
#pragma unroll
        for (int q = 0; q < (CHUNKS + 31) / 32; ++q) {
          const int c = q * 32 + lane;
          if (c < CHUNKS) dst[c] = stage[swz<CPL>(c + HC)];
        }
      } else if (interior) {
#pragma unroll
        for (int q = 0; q < LA; ++q)
          if (lane0 + q < N) row[lane0 + q] = A::store(x[q]);
      }
    }
    __syncwarp();  // this buffer is free for the next issue, the coefficients for a new pattern
    if (more) cur = window_next<LA>(cur, v, v1, segs, N, single_k, kb, gbits);
    buf ^= 1;
  }
}

template <class R, bool DF>
size_t trotter_smem() {
  using A = TrotArith<R, DF>;
  constexpr int per = 16 / sizeof(typename A::T);
  constexpr int CPL = trot_lane_amps<R, DF>() / per;
  return (size_t)(trot_threads<R, DF>() / 32) * (2 * 32 * CPL * 16 + sizeof(LayerCoefs<typename A::W>));
}

// ------------------------------------------------------------------------ the tree passes
// The postselected solve (hhl_solve_postselected) replaces the controlled products of QPE and
// of the uncompute by two trees, exact rearrangements of the same circuit for its prepared
// input, in which every clock row of the anc = 0 half holds the same vector.
//
// QPE by doubling (expansion): clock rows that agree on bits [0, kb) have had the same gates
// applied so far, and a row c + p 2^kb (p a pattern of the next group of clock bits) is row c
// with the pattern's products applied next. So, group by group, rows [2^kb, 2^(kb+G)) are
// computed from rows [0, 2^kb) with the groups' per-pattern layer lists: every row still sees
// its own gate sequence in circuit order (the same arithmetic as the in-place passes), each
// computed once; only the clock = 0 row has to be prepared.
//
// Uncompute, final Hadamards and postselection by halving (reduction): after the final
// Hadamard layer the clock = 0 amplitude is 2^(-n_c/2) sum_c W_c S1[c], W_c the product of the
// U_k^dagger of the set bits of c (U_{n_c-1}^dagger first). By linearity the sum folds group by
// group from the top clock bits down: row c (c < 2^kb) accumulates its own value and, for
// every nonzero pattern p of the group, the pattern's adjoint list applied to row c + p 2^kb.
// After the last group row 0 holds the postselected vector (scaled by 2^(-n_c/2) on the store).
//
// A warp takes a window (interior and both halos) of a source row into staging with
// asynchronous copies, double-buffered over its sequence of windows; the halos come straight
// from the source rows, which a tree pass never writes.
template <class R, bool DF, bool RED>
__global__ void __launch_bounds__(kTrotThreads, RED ? (sizeof(R) == 4 || DF ? 2 : 1) : trot_min_blocks<R, DF>())
    k_trotter_tree(typename Cx<R>::T* __restrict__ half, int n_s, int segs, int64_t items, int nwarps, int kb,
                   int gbits, const LayerList* __restrict__ lists, float scale_f, float scale_l, double scale_d) {
  using A = TrotArith<R, DF>;
  using T = typename A::T;
  using V = typename A::V;
  using W = typename A::W;
  constexpr int LA = trot_lane_amps<R, DF>();
  constexpr int HL = Geo<LA>::HL;
  constexpr int kInterior = Geo<LA>::INTER;
  constexpr int per = 16 / sizeof(T);
  constexpr int CPL = LA / per;
  constexpr int HC = kHalo / per;
  constexpr int WCH = 32 * CPL;             // chunks of a window
  constexpr int CHUNKS = kInterior / per;   // of its interior
  constexpr int WPB = kTrotThreads / 32;
  extern __shared__ __align__(16) unsigned char trot_smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint4* stage_w = reinterpret_cast<uint4*>(trot_smem) + (size_t)wid * 2 * WCH;
  LayerCoefs<W>* coef =
      reinterpret_cast<LayerCoefs<W>*>(reinterpret_cast<uint4*>(trot_smem) + (size_t)WPB * 2 * WCH) + wid;
  const int64_t N = 1LL << n_s;
  const int gw = (int)blockIdx.x * WPB + wid;
  if (gw >= nwarps) return;  // warp-uniform
  const int P = RED ? 1 << gbits : 1;  // windows per item
  const int64_t j0 = (int64_t)gw * items / nwarps * P, j1 = (int64_t)(gw + 1) * items / nwarps * P;
  const int64_t kmask = (1LL << kb) - 1;
  // window j of the sequence: source row, destination row, pattern (0: the accumulator's own
  // row in a reduction), segment
  auto decode = [&](int64_t j, int64_t* src, int64_t* dst, int* pat, int* seg) {
    const int64_t item = RED ? j >> gbits : j;
    const int64_t i = item / segs;
    *seg = (int)(item - i * segs);
    if (RED) {
      *pat = (int)(j & (P - 1));
      *dst = i;
      *src = i + ((int64_t)*pat << kb);
    } else {
      *pat = (int)(1 + (i >> kb));
      *src = i & kmask;
      *dst = *src + ((int64_t)*pat << kb);
    }
  };
  auto issue = [&](uint4* stage, int64_t src, int seg) {
    const T* row = half + src * N;
    const int64_t w0 = (int64_t)seg * kInterior - kHalo;  // first amplitude of the window
#pragma unroll
    for (int q = 0; q < WCH / 32; ++q) {
      const int c = q * 32 + lane;
      const int64_t a0 = w0 + (int64_t)c * per;
      if (a0 >= 0 && a0 + per <= N) cp_async16(&stage[swz<CPL>(c)], reinterpret_cast<const uint4*>(row + a0));
      else stage[swz<CPL>(c)] = make_uint4(0u, 0u, 0u, 0u);
    }
  };
  {
    int64_t src, dst;
    int pat, seg;
    decode(j0, &src, &dst, &pat, &seg);
    if (j0 < j1) issue(stage_w, src, seg);
  }
  cp_async_commit();
  int buf = 0, cached = -1, n_layers = 0, first_o = 0;
  const bool interior = lane >= HL && lane < 32 - HL;
  V acc[LA];
  for (int64_t j = j0; j < j1; ++j) {
    if (j + 1 < j1) {
      int64_t src, dst;
      int pat, seg;
      decode(j + 1, &src, &dst, &pat, &seg);
      issue(stage_w + (buf ^ 1) * WCH, src, seg);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    int64_t src, dst;
    int pat, seg;
    decode(j, &src, &dst, &pat, &seg);
    uint4* stage = stage_w + buf * WCH;
    const int64_t g0 = (int64_t)seg * kInterior;
    const int64_t lane0 = g0 - kHalo + (int64_t)lane * LA;
    const bool full = g0 + kInterior <= N;
    V x[LA];
    {
      T t[LA];
      uint4* d = reinterpret_cast<uint4*>(t);
#pragma unroll
      for (int q = 0; q < CPL; ++q) d[q] = stage[(lane * CPL + q) ^ (lane & 7)];
#pragma unroll
      for (int q = 0; q < LA; ++q) x[q] = A::load(t[q]);
    }
    if (RED && pat == 0) {
#pragma unroll
      for (int q = 0; q < LA; ++q) acc[q] = x[q];
    } else {
      const LayerList* L = lists + pat;
      if (pat != cached) {
        cached = pat;
        n_layers = L->n;
        first_o = L->first_o;
        if (lane < n_layers) {
          coef->c[lane] = A::coef(L->cf, L->cl, L->c, lane);
          coef->s[lane] = A::coef(L->sf, L->sl, L->s, lane);
          coef->w[lane] = A::coef(L->wf, L->wl, L->w, lane);
          coef->form[lane] = L->form[lane];
        }
      }
      __syncwarp();
      const bool away = full && g0 >= 2 && g0 + kInterior + 1 <= N;
      apply_pattern<R, DF, LA>(x, coef, L, n_layers, first_o, away, lane0, N, lane);
      if (RED) {
#pragma unroll
        for (int q = 0; q < LA; ++q) acc[q] = cadd(acc[q], x[q]);
      }
    }
    if (!RED || pat == P - 1) {
      V* out = RED ? acc : x;
      if (RED && kb == 0) {  // the postselected vector: 2^(-n_c/2) of the folded sum
        const W sc = A::coef1(scale_f, scale_l, scale_d);
#pragma unroll
        for (int q = 0; q < LA; ++q) out[q] = cscale(out[q], sc);
      }
      T* drow = half + dst * N;
      __syncwarp();  // every lane has read its window out of the staging buffer
      if (full) {
        if (interior) {
          T t[LA];
#pragma unroll
          for (int q = 0; q < LA; ++q) t[q] = A::store(out[q]);
          const uint4* sx = reinterpret_cast<const uint4*>(t);
#pragma unroll
          for (int q = 0; q < CPL; ++q) stage[(lane * CPL + q) ^ (lane & 7)] = sx[q];
        }
        __syncwarp();
        uint4* dptr = reinterpret_cast<uint4*>(drow + g0);
#pragma unroll
        for (int q = 0; q < (CHUNKS + 31) / 32; ++q) {
          const int c = q * 32 + lane;
          if (c < CHUNKS) dptr[c] = stage[swz<CPL>(c + HC)];
        }
      } else if (interior) {
#pragma unroll
        for (int q = 0; q < LA; ++q)
          if (lane0 + q < N) drow[lane0 + q] = A::store(out[q]);
      }
    }
    __syncwarp();  // the buffer is free for the next issue, the coefficients for a new pattern
    buf ^= 1;
  }
}

template <class R, bool DF, bool RED>
hhl_status tree_impl(const Plan& p, void* half, const TrotPassDesc& d, cudaStream_t st) {
  using T = typename Cx<R>::T;
  constexpr int LA = trot_lane_amps<R, DF>();
  const int64_t segs = (p.N + Geo<LA>::INTER - 1) / Geo<LA>::INTER;
  const size_t smem = trotter_smem<R, DF>();
  auto kern = k_trotter_tree<R, DF, RED>;
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  int dev = 0, sms = 0, occ = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  HHL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HHL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTrotThreads, smem));
  if (occ < 1) return fail(HHL_ERR_UNSUPPORTED, "Trotter tree pass does not fit an SM");
  // items: expansion (rows written) x segments; reduction (rows kept) x segments
  const int64_t rows = RED ? (1LL << d.kb) : (1LL << d.kb) * ((1LL << d.gbits) - 1);
  const int64_t items = rows * segs;
  const int64_t max_warps = (int64_t)occ * sms * (kTrotThreads / 32);
  const int nwarps = (int)std::min<int64_t>(items, max_warps);
  const unsigned grid = (unsigned)((nwarps + kTrotThreads / 32 - 1) / (kTrotThreads / 32));
  const double scale = 1.0 / sqrt((double)p.R);
  float sf, sl;
  df_split(scale, &sf, &sl);
  HHL_PROF_BEGIN(st);
  kern<<<grid, kTrotThreads, smem, st>>>((T*)half, p.n_s, (int)segs, items, nwarps, d.kb, d.gbits,
                                        (const LayerList*)p.d_trot_lists + d.list_off, sf, sl, scale);
  HHL_LAUNCH_CHECK(RED ? (DF ? "k_trotter_reduce_df" : "k_trotter_reduce") : (DF ? "k_trotter_expand_df" : "k_trotter_expand"));
  return HHL_OK;
}

__global__ void k_interleave(const double* __restrict__ re, const double* __restrict__ im, int64_t n,
                             double2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(re[i], im ? im[i] : 0.0);
}

template <class R, bool DF>
hhl_status trotter_impl(const Plan& p, void* half, bool adjoint, cudaStream_t st) {
  using T = typename Cx<R>::T;
  constexpr int LA = trot_lane_amps<R, DF>();
  const int64_t segs = (p.N + Geo<LA>::INTER - 1) / Geo<LA>::INTER;
  T* side = (T*)p.d_scratch;  // sized by the planner for min(R * segs, kMaxRuns) * 32 amplitudes
  const LayerList* lists = (const LayerList*)p.d_trot_lists;
  const size_t smem = trotter_smem<R, DF>();
  auto kern = k_trotter_pass<R, DF>;
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  int dev = 0, sms = 0, occ = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  HHL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  constexpr int TH = trot_threads<R, DF>();
  HHL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TH, smem));
  if (occ < 1) return fail(HHL_ERR_UNSUPPORTED, "Trotter pass does not fit an SM");
  for (const TrotPassDesc& d : p.trot_pass[adjoint ? 1 : 0]) {
    // pass rows: those with clock bit single_k set, or with a nonzero pattern of the group
    const int64_t rows = d.single_k >= 0 ? p.R / 2 : p.R - (p.R >> d.gbits);
    const int64_t windows = rows * segs;
    if (windows < 1) continue;
    if (windows > 0x7fffffffLL) return fail(HHL_ERR_UNSUPPORTED, "Trotter pass has too many windows");
    const int64_t max_warps = (int64_t)occ * sms * (TH / 32);
    int64_t runs = std::min<int64_t>(std::min<int64_t>(windows, max_warps), kMaxRuns);  // the side buffer holds them
    if (const char* env = getenv("HHL_TROTTER_RUNS")) {    // testing override: fewer, longer runs
      const long long cap = atoll(env);
      if (cap >= 1) runs = std::min<int64_t>(runs, cap);
    }
    const int nruns = (int)runs;
    const unsigned pgrid = (unsigned)((nruns + TH / 32 - 1) / (TH / 32));
    HHL_PROF_BEGIN(st);
    k_trotter_bounds<R, LA><<<(unsigned)((nruns * 32 + 255) / 256), 256, 0, st>>>((const T*)half, side, p.n_s, (int)segs,
                                                                                (int)windows, nruns, d.single_k, d.kb,
                                                                                d.gbits);
    HHL_LAUNCH_CHECK("k_trotter_bounds");
    HHL_PROF_BEGIN(st);
    kern<<<pgrid, TH, smem, st>>>((T*)half, side, p.n_s, (int)segs, (int)windows, nruns,
                                                         d.single_k, d.kb, d.gbits, lists + d.list_off);
    HHL_LAUNCH_CHECK(DF ? "k_trotter_pass_df" : "k_trotter_pass");
  }
  return HHL_OK;
}

// The layer list of one pass for one row pattern. bits: the set clock bits of the pattern in
// the order the circuit applies them; each contributes E(tau/2) O(tau) [E(tau) O(tau)]^(r-1)
// E(tau/2) (sign -1 and the conjugate phase for the adjoint, whose palindromic Strang product
// is the same list with negated angles), E layers of consecutive bits merged. A window
// [l0, l1) of a single bit's list is taken when win_l1 > 0.
void build_list(const Plan& p, const std::vector<int>& bits, bool adjoint, int win_l0, int win_l1, LayerList* out) {
  const double sg = adjoint ? -1.0 : 1.0;
  std::vector<std::pair<int, double>> layers;  // (is_o, time s): rotation angle s * o
  double pending = 0.0;
  for (size_t b = 0; b < bits.size(); ++b) {
    const int k = bits[b];
    const int r = p.trot_r[k];
    const double tau = p.trot_blocks[(size_t)k * 24 + 4];
    pending += 0.5 * tau;
    layers.push_back({0, pending});
    layers.push_back({1, tau});
    for (int j = 1; j < r; ++j) {
      layers.push_back({0, tau});
      layers.push_back({1, tau});
    }
    pending = 0.5 * tau;
  }
  layers.push_back({0, pending});
  const int l0 = win_l1 > 0 ? win_l0 : 0;
  const int l1 = win_l1 > 0 ? win_l1 : (int)layers.size();
  const double oh_k = p.trot_off_hat, dh = p.trot_diag_hat;
  double e_time = 0.0;
  out->n = l1 - l0;
  out->first_o = layers[l0].first;
  double fr = 1.0, fi = 0.0;  // product of the factored forms' factors
  for (int l = l0; l < l1; ++l) {
    const double th = sg * layers[l].second * oh_k;
    const double c = cos(th), sn = sin(th);
    out->c[l - l0] = c;
    out->s[l - l0] = sn;
    double gr, gi;
    if (fabs(c) >= fabs(sn)) {
      out->w[l - l0] = sn / c;
      out->form[l - l0] = 0;
      gr = c;
      gi = 0.0;
    } else {
      out->w[l - l0] = -c / sn;
      out->form[l - l0] = 1;
      gr = 0.0;
      gi = sn;
    }
    const double nr = fr * gr - fi * gi, ni = fr * gi + fi * gr;
    fr = nr;
    fi = ni;
    if (layers[l].first == 0) e_time += layers[l].second;
  }
  out->pc = cos(e_time * dh);
  out->ps = sg * sin(e_time * dh);
  out->pc2 = out->pc * fr - out->ps * fi;
  out->ps2 = out->pc * fi + out->ps * fr;
  df_split(out->pc2, &out->pc2f, &out->pc2l);
  df_split(out->ps2, &out->ps2f, &out->ps2l);
  df_split(out->pc, &out->pcf, &out->pcl);
  df_split(out->ps, &out->psf, &out->psl);
  for (int l = 0; l < out->n; ++l) {
    df_split(out->c[l], &out->cf[l], &out->cl[l]);
    df_split(out->s[l], &out->sf[l], &out->sl[l]);
    df_split(out->w[l], &out->wf[l], &out->wl[l]);
  }
}

}  // namespace

// Side-buffer amplitudes a Trotter plan needs: 32 per warp of a pass, at most one warp per
// window (the double-float kernel's windows have the smallest interior) and kMaxRuns warps.
int64_t trotter_side_amps(int64_t N, int64_t R) {
  const int64_t segs = (N + Geo<8>::INTER - 1) / Geo<8>::INTER;
  return std::min<int64_t>(R * segs, kMaxRuns) * 32;
}

hhl_status launch_trotter(const Plan& p, void* half, bool adjoint, cudaStream_t st) {
  if (p.d_scratch == nullptr || p.d_trot_lists == nullptr) return fail(HHL_ERR_INVALID_ARG, "Trotter plan without tables");
  if (p.prec == HHL_PREC_C64) return trotter_impl<float, false>(p, half, adjoint, st);
  // complex128: double-float on the FP32 pipe unless HHL_FP64_PIPE=1 (the FP64 form, kept for
  // comparison and tests)
  const char* env = getenv("HHL_FP64_PIPE");
  if (env != nullptr && atoi(env) != 0) return trotter_impl<double, false>(p, half, adjoint, st);
  return trotter_impl<double, true>(p, half, adjoint, st);
}

bool trotter_tree_supported(const Plan& p, std::string* why) {
  if (p.expm_mode != HHL_EXPM_TROTTER || p.d_trot_lists == nullptr) {
    *why = "the postselected solve needs a Strang-Trotter plan";
    return false;
  }
  if (p.full) {
    *why = "the postselected solve needs the postselect-early uncompute (full_uncompute = 0)";
    return false;
  }
  for (int dir = 0; dir < 2; ++dir) {
    int next = dir == 0 ? 0 : p.n_c;  // expansion: groups from bit 0 up; reduction: from the top down
    for (const TrotPassDesc& d : p.trot_pass[dir]) {
      const bool ok = dir == 0 ? d.kb == next : d.kb + d.gbits == next;
      if (!ok) {
        *why = "a clock bit needs more than 17 Strang layers (one bit over several passes)";
        return false;
      }
      next = dir == 0 ? d.kb + d.gbits : d.kb;
    }
  }
  return true;
}

hhl_status launch_trotter_tree(const Plan& p, void* half, bool reduce, cudaStream_t st) {
  const char* env = getenv("HHL_FP64_PIPE");
  const bool fp64 = env != nullptr && atoi(env) != 0;
  for (const TrotPassDesc& d : p.trot_pass[reduce ? 1 : 0]) {
    hhl_status s;
    if (p.prec == HHL_PREC_C64) s = reduce ? tree_impl<float, false, true>(p, half, d, st) : tree_impl<float, false, false>(p, half, d, st);
    else if (fp64) s = reduce ? tree_impl<double, false, true>(p, half, d, st) : tree_impl<double, false, false>(p, half, d, st);
    else s = reduce ? tree_impl<double, true, true>(p, half, d, st) : tree_impl<double, true, false>(p, half, d, st);
    if (s != HHL_OK) return s;
  }
  return HHL_OK;
}

size_t trotter_build_passes(Plan& p, std::vector<unsigned char>* table) {
  std::vector<LayerList> lists;
  for (int dir = 0; dir < 2; ++dir) {
    const bool adjoint = dir == 1;
    p.trot_pass[dir].clear();
    std::vector<int> order(p.n_c);
    for (int j = 0; j < p.n_c; ++j) order[j] = adjoint ? p.n_c - 1 - j : j;
    std::vector<int> group;
    int group_layers = 1;
    auto flush = [&]() {
      if (group.empty()) return;
      TrotPassDesc d;
      d.kb = *std::min_element(group.begin(), group.end());
      d.gbits = (int)group.size();
      d.single_k = d.gbits == 1 ? group[0] : -1;
      d.list_off = (int64_t)lists.size();
      d.max_layers = group_layers;
      const int npat = 1 << d.gbits;
      lists.resize(lists.size() + npat);
      LayerList* L = &lists[d.list_off];
      L[0] = LayerList{};
      for (int pat = 1; pat < npat; ++pat) {
        std::vector<int> bits;
        for (int k : group)
          if ((pat >> (k - d.kb)) & 1) bits.push_back(k);
        build_list(p, bits, adjoint, 0, 0, &L[pat]);
      }
      if (d.single_k >= 0) L[0] = L[1];  // unused: single-bit passes enumerate pattern-1 rows
      p.trot_pass[dir].push_back(d);
      group.clear();
      group_layers = 1;
    };
    for (int k : order) {
      const int lk = 2 * p.trot_r[k];
      if (lk + 1 > kMaxPassLayers) {
        flush();
        // windows of this bit's 2r + 1 layers: 17 from an E layer, then 16 from O layers
        for (int l0 = 0; l0 < lk + 1;) {
          const int cap = (l0 & 1) ? kMaxPassLayers - 1 : kMaxPassLayers;
          const int l1 = std::min(lk + 1, l0 + cap);
          TrotPassDesc d;
          d.kb = k;
          d.gbits = 1;
          d.single_k = k;
          d.list_off = (int64_t)lists.size();
          d.max_layers = l1 - l0;
          lists.resize(lists.size() + 2);
          build_list(p, std::vector<int>{k}, adjoint, l0, l1, &lists[d.list_off + 1]);
          lists[d.list_off] = lists[d.list_off + 1];
          p.trot_pass[dir].push_back(d);
          l0 = l1;
        }
        continue;
      }
      if (group_layers + lk > kMaxPassLayers) flush();
      group.push_back(k);
      group_layers += lk;
    }
    flush();
  }
  table->resize(lists.size() * sizeof(LayerList));
  memcpy(table->data(), lists.data(), table->size());
  return lists.size();
}

hhl_status launch_interleave(const double* re, const double* im, int64_t n, double* out, cudaStream_t st) {
  int g = (int)((n + 255) / 256);
  if (g > 152 * 8) g = 152 * 8;
  HHL_PROF_BEGIN(st);
  k_interleave<<<g, 256, 0, st>>>(re, im, n, (double2*)out);
  HHL_LAUNCH_CHECK("k_interleave");
  return HHL_OK;
}

}  // namespace hhl
