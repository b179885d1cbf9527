// Fused register blocks over the clock register (or any register of <= 13 qubits):
// the clock block of the HHL circuit (inverse QFT + eigenvalue-inversion RY + QFT), the
// Hadamard layer on the clock, and stand-alone QFT / inverse QFT blocks.
//
// A "column" is the 2^m amplitudes that differ only in the register's bits (stride 2^lo
// in the state). A thread-block cluster of C = 2^CB CTAs holds W consecutive columns (so
// every global access covers W contiguous amplitudes, up to 64 bytes): CTA r of the
// cluster keeps the rows whose top CB register bits equal r, 2^m / C rows of W columns,
// in its shared memory. The CB butterfly stages that pair rows held by different CTAs run
// as one radix-C pass that reads the partners through distributed shared memory; the
// other m - CB stages are local and run in passes of up to 4 stages: a thread loads the
// 2^r amplitudes of one group into registers, applies the r radix-2 stages (the Hadamard
// and controlled-phase layers of the QFT circuit, i.e. Cooley-Tukey butterflies), and
// stores them back, so a 12-qubit register costs 3 shared-memory round trips instead of
// 12. Rows are padded by one element per 16 to spread strided accesses over the banks;
// twiddles come from two small tables (exp(-2 pi i q / L) = T1[q >> 6] T0[q & 63]).
//
// Orders: decimation in frequency (DIF) takes natural order and leaves the result in
// bit-reversed order; decimation in time (DIT) takes bit-reversed order and returns natural
// order. The clock block chains DIF (inverse QFT) -> rotation at bit-reversed positions ->
// DIT (QFT), so no explicit bit-reversal permutation (the QFT's swap layer) is applied.
#include <cooperative_groups.h>

#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "hhl_common.cuh"

namespace cg = cooperative_groups;

namespace hhl {

namespace {

constexpr int kFftThreads = 256;
constexpr size_t kFftSmemTarget = 140 * 1024;  // one CTA per SM at most this large
constexpr size_t kFftSmemCap = 200 * 1024;
constexpr int kUnroll = 8;                     // 16-byte loads in flight per thread
constexpr int kCrossK = 4;                     // groups per thread per cross-CTA chunk

__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }
__device__ __forceinline__ int bitrev_m(int x, int m) { return (int)(__brev((unsigned)x) >> (32 - m)); }

template <class T>
struct Twiddle {
  const T* t0;  // exp(-2 pi i j / L), j < 64
  const T* t1;  // exp(-2 pi i 64 j / L)
  __device__ __forceinline__ T operator()(int q, bool conj) const {
    T f = cmul(t1[q >> 6], t0[q & 63]);
    if (conj) f.y = -f.y;
    return f;
  }
};

// Three-level table for transforms of up to 33 bits (global memory, read through L1):
// exp(-2 pi i q / L) = T2[q >> 22] T1[(q >> 11) & 2047] T0[q & 2047].
template <class T>
struct Twiddle3 {
  const T* t0;
  const T* t1;
  const T* t2;
  __device__ __forceinline__ T operator()(int q, bool conj) const {
    T f = cmul(cmul(__ldg(reinterpret_cast<const T*>(t2) + (q >> 22)), __ldg(t1 + ((q >> 11) & 2047))),
               __ldg(t0 + (q & 2047)));
    if (conj) f.y = -f.y;
    return f;
  }
};

// Four-level table in shared memory for the 2^n-point twiddles of a whole-register transform
// (n <= 32): exp(-2 pi i q / 2^n) = T[0][q & 255] T[1][(q >> 8) & 255] T[2][(q >> 16) & 255]
// T[3][q >> 24], level k holding exp(-2 pi i (j 2^(8k) mod 2^n) / 2^n), j < 256, from FP64
// sincospi (8 KiB for complex64: the lookups stay in shared memory instead of reaching L2).
template <class T>
struct Twiddle4 {
  const T* t;  // 4 x 256 entries
  __device__ __forceinline__ T operator()(int q, bool conj) const {
    const unsigned u = (unsigned)q;
    T f = cmul(cmul(t[u & 255], t[256 + ((u >> 8) & 255)]), cmul(t[512 + ((u >> 16) & 255)], t[768 + (u >> 24)]));
    if (conj) f.y = -f.y;
    return f;
  }
};

template <class R>
__device__ void fill_twiddle4(typename Cx<R>::T* t, int n) {
  const double inv = 1.0 / (double)(1ULL << n);
  for (int j = threadIdx.x; j < 1024; j += blockDim.x) {
    const int k = j >> 8;
    const unsigned long long e = ((unsigned long long)(j & 255) << (8 * k)) & ((1ULL << n) - 1);
    double sn = 0.0, cs = 1.0;
    if (e != 0) sincospi(-2.0 * (double)e * inv, &sn, &cs);  // (levels above n bits are all 1)
    t[j] = mk<R>((R)cs, (R)sn);
  }
}

__host__ __device__ constexpr int twiddle_entries(int m) { return 64 + ((1 << m) / 64 > 1 ? (1 << m) / 64 : 1); }

template <class R>
__device__ void fill_twiddles(typename Cx<R>::T* t0, typename Cx<R>::T* t1, int m) {
  const int L = 1 << m;
  const int n1 = twiddle_entries(m) - 64;
  for (int j = threadIdx.x; j < 64 + n1; j += blockDim.x) {
    const int e = j < 64 ? j : 64 * (j - 64);
    if constexpr (std::is_same<R, df>::value) {  // double-float from the FP64 values
      double s, c;
      sincospi(-2.0 * (double)(e & (L - 1)) / (double)L, &s, &c);
      if (j < 64) t0[j] = mk<df>(df_of(c), df_of(s));
      else t1[j - 64] = mk<df>(df_of(c), df_of(s));
    } else {
      R s, c;
      if constexpr (sizeof(R) == 4) {
        sincospif(-2.0f * (float)(e & (L - 1)) / (float)L, &s, &c);
      } else {
        sincospi(-2.0 * (double)(e & (L - 1)) / (double)L, &s, &c);
      }
      if (j < 64) t0[j] = mk<R>(c, s);
      else t1[j - 64] = mk<R>(c, s);
    }
  }
}

// e^{-2 pi i k / 16}, k < 16 (the in-group factors of the twiddles, see butterflies()).
__constant__ double kRoot16[16][2] = {
    {1.0, 0.0}, {0.92387953251128674, -0.38268343236508978}, {0.70710678118654752, -0.70710678118654752},
    {0.38268343236508978, -0.92387953251128674}, {0.0, -1.0}, {-0.38268343236508978, -0.92387953251128674},
    {-0.70710678118654752, -0.70710678118654752}, {-0.92387953251128674, -0.38268343236508978}, {-1.0, 0.0},
    {-0.92387953251128674, 0.38268343236508978}, {-0.70710678118654752, 0.70710678118654752},
    {-0.38268343236508978, 0.92387953251128674}, {0.0, 1.0}, {0.38268343236508978, 0.92387953251128674},
    {0.70710678118654752, 0.70710678118654752}, {0.92387953251128674, 0.38268343236508978}};
__constant__ float kRoot16f[16][2] = {
    {1.0f, 0.0f}, {0.92387953251128674f, -0.38268343236508978f}, {0.70710678118654752f, -0.70710678118654752f},
    {0.38268343236508978f, -0.92387953251128674f}, {0.0f, -1.0f}, {-0.38268343236508978f, -0.92387953251128674f},
    {-0.70710678118654752f, -0.70710678118654752f}, {-0.92387953251128674f, -0.38268343236508978f}, {-1.0f, 0.0f},
    {-0.92387953251128674f, 0.38268343236508978f}, {-0.70710678118654752f, 0.70710678118654752f},
    {-0.38268343236508978f, 0.92387953251128674f}, {0.0f, 1.0f}, {0.38268343236508978f, 0.92387953251128674f},
    {0.70710678118654752f, 0.70710678118654752f}, {0.92387953251128674f, 0.38268343236508978f}};

// The root for the amplitude precision (FP32 kernels read FP32 constants: converting an FP64
// constant costs a pass through GB300's narrow FP64 pipe).
// Double-float remainders of those roots (kRoot16 - kRoot16f, evaluated in FP64 at compile time).
#define HHL_DFL(v) ((float)((v) - (double)(float)(v)))
#define HHL_R16(c, s) {HHL_DFL(c), HHL_DFL(s)}
__constant__ float kRoot16l[16][2] = {
    HHL_R16(1.0, 0.0), HHL_R16(0.92387953251128674, -0.38268343236508978),
    HHL_R16(0.70710678118654752, -0.70710678118654752), HHL_R16(0.38268343236508978, -0.92387953251128674),
    HHL_R16(0.0, -1.0), HHL_R16(-0.38268343236508978, -0.92387953251128674),
    HHL_R16(-0.70710678118654752, -0.70710678118654752), HHL_R16(-0.92387953251128674, -0.38268343236508978),
    HHL_R16(-1.0, 0.0), HHL_R16(-0.92387953251128674, 0.38268343236508978),
    HHL_R16(-0.70710678118654752, 0.70710678118654752), HHL_R16(-0.38268343236508978, 0.92387953251128674),
    HHL_R16(0.0, 1.0), HHL_R16(0.38268343236508978, 0.92387953251128674),
    HHL_R16(0.70710678118654752, 0.70710678118654752), HHL_R16(0.92387953251128674, 0.38268343236508978)};
#undef HHL_R16
#undef HHL_DFL

template <class R>
__device__ __forceinline__ R root16(int k, int part) {
  if constexpr (std::is_same<R, df>::value) return df{kRoot16f[k][part], kRoot16l[k][part]};
  else if constexpr (sizeof(R) == 4) return kRoot16f[k][part];
  else return (R)kRoot16[k][part];
}

// The RB radix-2 stages of one group: v[x] = element lo + x * 2^lo_bits (+ a multiple of
// 2^(lo_bits + RB)); local bit t is global stage s = t + 1 + lo_bits of an m-stage transform.
// MODE 0: DFT butterflies, MODE 1: Hadamard butterflies. DIF runs t from high to low.
// The twiddle of butterfly x at bit t, exp(-2 pi i ((x mod 2^t) 2^lo_bits + lo) 2^(m-s) / L),
// factors into exp(-2 pi i lo 2^(m-s) / L) (one table lookup per stage) times
// exp(-2 pi i (x mod 2^t) / 2^(t+1)) (a sixteenth root of unity, from constant memory).
template <class T, int RB, bool DIT, int MODE>
__device__ __forceinline__ void butterflies(T (&v)[1 << RB], int lo, int lo_bits, int m, const Twiddle<T>& tw,
                                            bool conj) {
  constexpr int G = 1 << RB;
  using R = decltype(T().x);
#pragma unroll
  for (int tt = 0; tt < RB; ++tt) {
    const int t = DIT ? tt : (RB - 1 - tt);
    const int s = t + 1 + lo_bits;
    T base;
    if (MODE == 0) base = tw(lo << (m - s), conj);
#pragma unroll
    for (int x = 0; x < G; ++x) {
      if (x & (1 << t)) continue;
      const int x1 = x | (1 << t);
      T a = v[x], b = v[x1];
      if (MODE == 0) {
        const int xr = x & ((1 << t) - 1);
        T f = base;
        if (xr != 0) {
          const int k16 = xr << (3 - t);
          T w;
          w.x = root16<R>(k16, 0);
          w.y = conj ? -root16<R>(k16, 1) : root16<R>(k16, 1);
          f = cmul(base, w);
        }
        if (DIT) {
          b = cmul(b, f);
          v[x] = cadd(a, b);
          v[x1] = csub(a, b);
        } else {
          v[x] = cadd(a, b);
          v[x1] = cmul(csub(a, b), f);
        }
      } else {
        v[x] = cadd(a, b);
        v[x1] = csub(a, b);
      }
    }
  }
}

// One local pass of RB stages (global stages s0-RB+1 .. s0 <= m_loc) on every group of the
// W local columns of 2^m_loc rows.
template <class T, int RB, bool DIT, int MODE>
__device__ void radix_pass(T* X, int Lp, int W, const Twiddle<T>& tw, int m, int m_loc, int s0, bool conj) {
  constexpr int G = 1 << RB;
  const int lo_bits = s0 - RB;
  const int gpc_bits = m_loc - RB;
  const int total = W << gpc_bits;
  for (int g = threadIdx.x; g < total; g += blockDim.x) {
    const int w = g >> gpc_bits;
    const int gg = g & ((1 << gpc_bits) - 1);
    const int lo = gg & ((1 << lo_bits) - 1);
    const int hi = gg >> lo_bits;
    const int base = (hi << s0) + lo;
    T* col = X + w * Lp;
    T v[G];
#pragma unroll
    for (int x = 0; x < G; ++x) v[x] = col[pad16(base + (x << lo_bits))];
    butterflies<T, RB, DIT, MODE>(v, lo, lo_bits, m, tw, conj);
#pragma unroll
    for (int x = 0; x < G; ++x) col[pad16(base + (x << lo_bits))] = v[x];
  }
}

template <class T, bool DIT, int MODE>
__device__ void local_stages(T* X, int Lp, int W, const Twiddle<T>& tw, int m, int m_loc, bool conj) {
  const int npass = (m_loc + 3) / 4;
  int done = 0;
  for (int p = 0; p < npass; ++p) {
    const int r = (m_loc - done) / (npass - p);  // balanced pass sizes, each <= 4
    const int s0 = DIT ? done + r : m_loc - done;
    switch (r) {
      case 4: radix_pass<T, 4, DIT, MODE>(X, Lp, W, tw, m, m_loc, s0, conj); break;
      case 3: radix_pass<T, 3, DIT, MODE>(X, Lp, W, tw, m, m_loc, s0, conj); break;
      case 2: radix_pass<T, 2, DIT, MODE>(X, Lp, W, tw, m, m_loc, s0, conj); break;
      default: radix_pass<T, 1, DIT, MODE>(X, Lp, W, tw, m, m_loc, s0, conj); break;
    }
    done += r;
    __syncthreads();
  }
}

// The CB stages across the cluster (global stages m_loc+1 .. m): every CTA gathers the C
// partners of each of its groups from all CTAs' shared memory, computes the butterflies
// and keeps the output that belongs to its own rows. Chunks of kCrossK groups per thread;
// a cluster barrier between the gathers and the write-back of each chunk keeps a CTA from
// overwriting values another CTA has yet to read. Every CTA must have finished writing its
// columns (cluster barrier) before this is called. X2 (may be null) is transformed alongside.
template <class T, int CB, bool DIT, int MODE>
__device__ void cross_stages(cg::cluster_group& cl, T* X, T* X2, int Lp, int W, const Twiddle<T>& tw, int m,
                             bool conj) {
  constexpr int C = 1 << CB;
  const int m_loc = m - CB;
  const int rank = (int)cl.block_rank();
  const int total = W << m_loc;
  for (int base = 0; base < total; base += blockDim.x * kCrossK) {
    T keep[kCrossK], keep2[kCrossK];
#pragma unroll
    for (int kk = 0; kk < kCrossK; ++kk) {
      const int g = base + kk * blockDim.x + threadIdx.x;
      if (g < total) {
        const int w = g >> m_loc, p = g & ((1 << m_loc) - 1);
        const int off = w * Lp + pad16(p);
        T v[C];
#pragma unroll
        for (int x = 0; x < C; ++x) v[x] = cl.map_shared_rank(X, x)[off];
        butterflies<T, CB, DIT, MODE>(v, p, m_loc, m, tw, conj);
#pragma unroll
        for (int x = 0; x < C; ++x)
          if (x == rank) keep[kk] = v[x];  // static indexing keeps v in registers
        if (X2 != nullptr) {
#pragma unroll
          for (int x = 0; x < C; ++x) v[x] = cl.map_shared_rank(X2, x)[off];
          butterflies<T, CB, DIT, MODE>(v, p, m_loc, m, tw, conj);
#pragma unroll
          for (int x = 0; x < C; ++x)
            if (x == rank) keep2[kk] = v[x];
        }
      }
    }
    cl.sync();
#pragma unroll
    for (int kk = 0; kk < kCrossK; ++kk) {
      const int g = base + kk * blockDim.x + threadIdx.x;
      if (g < total) {
        const int w = g >> m_loc, p = g & ((1 << m_loc) - 1);
        const int off = w * Lp + pad16(p);
        X[off] = keep[kk];
        if (X2 != nullptr) X2[off] = keep2[kk];
      }
    }
  }
  __syncthreads();
}

// Rows [0, Lc) of a W-column block (row c at src + c * row_stride) -> X[w * Lp + pad16(c)],
// in 16-byte units with kUnroll loads in flight per thread (W * sizeof(T) >= 16), or
// element by element otherwise.
template <class T>
__device__ void load_block(T* X, int Lp, const T* src, int64_t row_stride, int Lc, int W) {
  constexpr int per = 16 / sizeof(T);
  if (W == 1 && row_stride == 1) {
    // one contiguous column (a register at the lowest index bits): 16-byte units of rows
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const int units = Lc / per;
    for (int b = threadIdx.x; b < units; b += blockDim.x * kUnroll) {
      uint4 v[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k)
        if (b + k * blockDim.x < units) v[k] = s4[b + k * blockDim.x];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int u = b + k * blockDim.x;
        if (u < units) {
          const T* t = reinterpret_cast<const T*>(&v[k]);
#pragma unroll
          for (int q = 0; q < per; ++q) X[pad16(u * per + q)] = t[q];
        }
      }
    }
  } else if (W % per == 0) {
    const int upr = W / per;
    const int total = Lc * upr;
    for (int b = threadIdx.x; b < total; b += blockDim.x * kUnroll) {
      uint4 v[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int u = b + k * blockDim.x;
        if (u < total) {
          const int c = u / upr, h = u - c * upr;
          v[k] = *reinterpret_cast<const uint4*>(src + (int64_t)c * row_stride + h * per);
        }
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int u = b + k * blockDim.x;
        if (u < total) {
          const int c = u / upr, h = u - c * upr;
          const T* t = reinterpret_cast<const T*>(&v[k]);
#pragma unroll
          for (int q = 0; q < per; ++q) X[(h * per + q) * Lp + pad16(c)] = t[q];
        }
      }
    }
  } else {
    const int total = Lc * W;
    for (int b = threadIdx.x; b < total; b += blockDim.x * kUnroll) {
      T v[kUnroll];
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int u = b + k * blockDim.x;
        if (u < total) v[k] = src[(int64_t)(u / W) * row_stride + (u % W)];
      }
#pragma unroll
      for (int k = 0; k < kUnroll; ++k) {
        const int u = b + k * blockDim.x;
        if (u < total) X[(u % W) * Lp + pad16(u / W)] = v[k];
      }
    }
  }
}

// dst row row_of(p) (W contiguous amplitudes) = scale * X[w * Lp + pad16(p)], p < Lc;
// row_of(p) = p, or the bit reversal of (rank * Lc + p) over m bits when rev.
template <class T, class S>
__device__ void store_block(T* dst, int64_t row_stride, const T* X, int Lp, int Lc, int W, S scale, bool rev,
                            int rank, int m) {
  constexpr int per = 16 / sizeof(T);
  if (W == 1 && row_stride == 1 && !rev) {
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (int u = threadIdx.x; u < Lc / per; u += blockDim.x) {
      uint4 v;
      T* t = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int q = 0; q < per; ++q) t[q] = cscale(X[pad16(u * per + q)], scale);
      d4[u] = v;
    }
  } else if (W % per == 0) {
    const int upr = W / per;
    for (int u = threadIdx.x; u < Lc * upr; u += blockDim.x) {
      const int p = u / upr, h = u - p * upr;
      const int row = rev ? bitrev_m(rank * Lc + p, m) : p;
      uint4 v;
      T* t = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int q = 0; q < per; ++q) t[q] = cscale(X[(h * per + q) * Lp + pad16(p)], scale);
      *reinterpret_cast<uint4*>(dst + (int64_t)row * row_stride + h * per) = v;
    }
  } else {
    for (int u = threadIdx.x; u < Lc * W; u += blockDim.x) {
      const int p = u / W, w = u % W;
      const int row = rev ? bitrev_m(rank * Lc + p, m) : p;
      dst[(int64_t)row * row_stride + w] = cscale(X[w * Lp + pad16(p)], scale);
    }
  }
}

// Clock block (a3 + a4 + the QFT of a5) on a cluster of 2^CB CTAs.
template <class R, bool FULL, int CB>
__global__ void __launch_bounds__(kFftThreads, 2) k_clock_block(typename Cx<R>::T* __restrict__ S,
                                                             const typename Cx<R>::T* __restrict__ rot, int n_s,
                                                             int n_c, int W) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = CB > 0 ? (int)cl.block_rank() : 0;
  const int m = n_c, m_loc = n_c - CB;
  const int Lc = 1 << m_loc, Lp = Lc + Lc / 16 + 1;
  const int64_t N = 1LL << n_s;
  const int64_t half = (N << n_c);
  T* t0 = reinterpret_cast<T*>(smem_raw);
  T* t1 = t0 + 64;
  T* X = t0 + twiddle_entries(m);
  T* Y = X + (size_t)W * Lp;
  fill_twiddles<R>(t0, t1, m);
  const Twiddle<T> tw{t0, t1};
  const int64_t j0 = (int64_t)(blockIdx.x >> CB) * W;
  const int64_t row0 = (int64_t)rank * Lc;  // first clock row held by this CTA
  T* S0 = S;
  T* S1 = S + half;
  load_block(X, Lp, S0 + row0 * N + j0, N, Lc, W);
  if (CB > 0) {
    cl.sync();
    cross_stages<T, CB, false, 0>(cl, X, (T*)nullptr, Lp, W, tw, m, false);  // inverse QFT, top stages
  } else {
    __syncthreads();
  }
  local_stages<T, false, 0>(X, Lp, W, tw, m, m_loc, false);  // inverse QFT, bit-reversed result
  const R inv = (R)(1.0 / sqrt((double)(1 << m)));
  // rotation at bit-reversed positions, in 16-byte units of W/per consecutive columns
  constexpr int per = 16 / sizeof(T);
  const int upr = W / per;
  for (int u = threadIdx.x; u < Lc * upr; u += blockDim.x) {
    const int p = u / upr, h = u - p * upr;
    const int y = bitrev_m((int)row0 + p, m);
    const T r = rot[y];  // (cos(theta_y/2), sin(theta_y/2))
    uint4 keep;
    T* kt = reinterpret_cast<T*>(&keep);
#pragma unroll
    for (int q = 0; q < per; ++q) {
      const int idx = (h * per + q) * Lp + pad16(p);
      const T x = cscale(X[idx], inv);
      if (FULL) Y[idx] = cscale(x, r.x);
      else kt[q] = cscale(x, r.x);
      X[idx] = cscale(x, r.y);
    }
    if (!FULL) *reinterpret_cast<uint4*>(S0 + (int64_t)y * N + j0 + h * per) = keep;  // anc = 0 half as rotated
  }
  __syncthreads();
  local_stages<T, true, 0>(X, Lp, W, tw, m, m_loc, true);  // QFT, lower stages
  if (FULL) local_stages<T, true, 0>(Y, Lp, W, tw, m, m_loc, true);
  if (CB > 0) {
    cl.sync();
    cross_stages<T, CB, true, 0>(cl, X, FULL ? Y : (T*)nullptr, Lp, W, tw, m, true);  // QFT, top stages
  }
  store_block(S1 + row0 * N + j0, N, X, Lp, Lc, W, inv, false, rank, m);
  if (FULL) store_block(S0 + row0 * N + j0, N, Y, Lp, Lc, W, inv, false, rank, m);
}

// Register transform on bits [lo, lo+m): mode 0 = QFT, 1 = inverse QFT, 2 = Hadamards (DIF,
// natural in; QFT / inverse QFT results are stored from bit-reversed positions), 3 = the QFT's
// DIF stages left in bit-reversed order, 4 = the inverse QFT's DIT stages from bit-reversed
// order (the low register of a whole-register transform: its stages do not depend on the
// bits above). Every output is multiplied by scale.
template <class R, int CB>
__global__ void __launch_bounds__(kFftThreads, 2) k_register_transform(typename Cx<R>::T* __restrict__ S, int lo, int m,
                                                                    int W, int mode, R scale) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = CB > 0 ? (int)cl.block_rank() : 0;
  const int m_loc = m - CB;
  const int Lc = 1 << m_loc, Lp = Lc + Lc / 16 + 1;
  const int64_t inner = 1LL << lo;
  T* t0 = reinterpret_cast<T*>(smem_raw);
  T* t1 = t0 + 64;
  T* X = t0 + twiddle_entries(m);
  if (mode != 2) fill_twiddles<R>(t0, t1, m);
  const Twiddle<T> tw{t0, t1};
  const int64_t groups = inner / W;
  const int64_t col = blockIdx.x >> CB;
  const int64_t o = col / groups, g = col - o * groups;
  T* base = S + o * ((int64_t)1 << (lo + m)) + g * W;
  load_block(X, Lp, base + (int64_t)rank * Lc * inner, inner, Lc, W);
  const bool conj = mode == 0 || mode == 3;  // QFT: exp(+2 pi i x y / L)
  if (mode == 4) {  // DIT: low (local) stages first, then the cluster's top stages
    __syncthreads();
    local_stages<T, true, 0>(X, Lp, W, tw, m, m_loc, false);
    if (CB > 0) {
      cl.sync();
      cross_stages<T, CB, true, 0>(cl, X, (T*)nullptr, Lp, W, tw, m, false);
    }
  } else {
    if (CB > 0) {
      cl.sync();
      if (mode == 2) cross_stages<T, CB, false, 1>(cl, X, (T*)nullptr, Lp, W, tw, m, false);
      else cross_stages<T, CB, false, 0>(cl, X, (T*)nullptr, Lp, W, tw, m, conj);
    } else {
      __syncthreads();
    }
    if (mode == 2) local_stages<T, false, 1>(X, Lp, W, tw, m, m_loc, false);
    else local_stages<T, false, 0>(X, Lp, W, tw, m, m_loc, conj);
  }
  if (mode >= 2) store_block(base + (int64_t)rank * Lc * inner, inner, X, Lp, Lc, W, scale, false, rank, m);
  else store_block(base, inner, X, Lp, Lc, W, scale, true, rank, m);
}

// The low register of a whole-register transform (bits [0, m) of contiguous 2^m-amplitude
// chunks; modes 3 / 4 of k_register_transform) as a persistent kernel: each CTA walks chunks
// with a stride of the grid, and the next chunk is fetched by asynchronous copies straight
// into the second of two padded shared-memory buffers (one copy per amplitude, 8 or 16
// bytes) while the current one is transformed, so loads overlap the radix passes.
__device__ __forceinline__ void cp_async_amp(void* smem, const void* gmem, int bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

template <class R>
__global__ void __launch_bounds__(kFftThreads, 2) k_lowbits_transform(typename Cx<R>::T* __restrict__ S, int m,
                                                                     int mode, R scale, long long chunks) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << m, Lp = L + L / 16 + 1;
  T* t0 = reinterpret_cast<T*>(smem_raw);
  T* t1 = t0 + 64;
  T* Xb = t0 + twiddle_entries(m);
  Xb += (reinterpret_cast<uintptr_t>(Xb) & 15) ? 1 : 0;  // 16-byte aligned buffers for complex128
  const int Lpa = (Lp + 1) & ~1;
  fill_twiddles<R>(t0, t1, m);
  const Twiddle<T> tw{t0, t1};
  long long c = blockIdx.x;
  if (c >= chunks) return;  // block-uniform
  for (int q = threadIdx.x; q < L; q += blockDim.x) cp_async_amp(Xb + pad16(q), S + c * L + q, (int)sizeof(T));
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  int buf = 0;
  for (; c < chunks; c += gridDim.x) {
    const long long cn = c + gridDim.x;
    if (cn < chunks) {
      T* Xn = Xb + (buf ^ 1) * Lpa;
      for (int q = threadIdx.x; q < L; q += blockDim.x) cp_async_amp(Xn + pad16(q), S + cn * L + q, (int)sizeof(T));
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();  // the current chunk has landed (and the twiddles are in place)
    T* X = Xb + buf * Lpa;
    if (mode == 4) local_stages<T, true, 0>(X, Lp, 1, tw, m, m, false);
    else local_stages<T, false, 0>(X, Lp, 1, tw, m, m, true);
    store_block(S + c * L, 1, X, Lp, L, 1, scale, false, 0, m);
    __syncthreads();  // this buffer is read out before it is refilled
    buf ^= 1;
  }
}

template <class R>
hhl_status lowbits_transform(void* state, int n, int m, int mode, R scale, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int L = 1 << m, Lp = L + L / 16 + 1, Lpa = (Lp + 1) & ~1;
  const size_t smem = ((size_t)twiddle_entries(m) + 1 + 2 * (size_t)Lpa) * sizeof(T);
  auto kern = k_lowbits_transform<R>;
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  int dev = 0, sms = 0, occ = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  HHL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HHL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kFftThreads, smem));
  if (occ < 1) return fail(HHL_ERR_UNSUPPORTED, "low-bit transform does not fit an SM");
  const long long chunks = 1LL << (n - m);
  const long long grid = std::min<long long>(chunks, (long long)occ * sms);
  HHL_PROF_BEGIN(st);
  kern<<<(unsigned)grid, kFftThreads, smem, st>>>((T*)state, m, mode, scale, chunks);
  HHL_LAUNCH_CHECK("k_lowbits_transform");
  return HHL_OK;
}

template <class R>
size_t fft_smem(int m, int cb, int W, int buffers) {
  const size_t sz = sizeof(typename Cx<R>::T);
  const size_t Lc = (size_t)1 << (m - cb), Lp = Lc + Lc / 16 + 1;
  return (size_t)twiddle_entries(m) * sz + (size_t)buffers * W * Lp * sz;
}

// Pick the block width W and the smallest cluster (<= 8 CTAs) whose shared memory fits the
// target (else the cap).
template <class R>
bool choose_shape(int m, int64_t limit, int buffers, int* W_out, int* cb_out, size_t* smem_out) {
  // 32-byte row segments (W = 4 complex64 / 2 complex128): measured best on GB300 for the
  // 12- and 13-qubit clocks; wider blocks need larger clusters, whose barriers cost more.
  int W = (int)std::min<int64_t>(32 / (int)sizeof(typename Cx<R>::T), limit);
  // tuning override "W,cb" (W a power of two of at least one 16-byte unit per row, as the
  // rotation of the clock block needs; used when it fits the shared-memory cap)
  if (const char* env = getenv("HHL_FFT_SHAPE")) {
    int w = 0, c = -1;
    if (sscanf(env, "%d,%d", &w, &c) == 2 && w * (int)sizeof(typename Cx<R>::T) >= 16 && w <= W &&
        (w & (w - 1)) == 0 && c >= 0 && c <= 3 && c < m && fft_smem<R>(m, c, w, buffers) <= kFftSmemCap) {
      *W_out = w;
      *cb_out = c;
      *smem_out = fft_smem<R>(m, c, w, buffers);
      return true;
    }
  }
  for (size_t cap : {kFftSmemTarget, kFftSmemCap}) {
    for (int cb = 0; cb <= 3 && cb < m; ++cb) {
      if (fft_smem<R>(m, cb, W, buffers) <= cap) {
        *W_out = W;
        *cb_out = cb;
        *smem_out = fft_smem<R>(m, cb, W, buffers);
        return true;
      }
    }
  }
  return false;
}

template <class Kern>
hhl_status launch_cluster(Kern kernel, int grid, int cb, size_t smem, cudaStream_t st, const char* name,
                          void** args) {
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kernel, smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kFftThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << cb;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HHL_PROF_BEGIN(st);
  cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)kernel, args);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g_prof_on.load(std::memory_order_relaxed)) prof_end(name);
    return cuda_fail(e, name);
  }
  HHL_LAUNCH_CHECK(name);
  return HHL_OK;
}

template <class R, bool FULL>
hhl_status clock_block_impl(const Plan& p, void* state, cudaStream_t st) {
  using T = typename Cx<R>::T;
  int W = 0, cb = 0;
  size_t smem = 0;
  if (!choose_shape<R>(p.n_c, p.N, FULL ? 2 : 1, &W, &cb, &smem))
    return fail(HHL_ERR_UNSUPPORTED, "clock register too large for one cluster");
  constexpr int per = 16 / sizeof(T);
  if (W % per != 0) return fail(HHL_ERR_UNSUPPORTED, "system register narrower than one 16-byte unit");
  const int grid = (int)((p.N / W) << cb);
  T* S = (T*)state;
  const T* rot = (const T*)p.d_rot;
  int n_s = p.n_s, n_c = p.n_c;
  void* args[] = {&S, &rot, &n_s, &n_c, &W};
  switch (cb) {
    case 0: return launch_cluster(k_clock_block<R, FULL, 0>, grid, cb, smem, st, "k_clock_block", args);
    case 1: return launch_cluster(k_clock_block<R, FULL, 1>, grid, cb, smem, st, "k_clock_block", args);
    case 2: return launch_cluster(k_clock_block<R, FULL, 2>, grid, cb, smem, st, "k_clock_block", args);
    default: return launch_cluster(k_clock_block<R, FULL, 3>, grid, cb, smem, st, "k_clock_block", args);
  }
}

template <class R>
hhl_status register_transform_impl(void* state, int n, int lo, int m, int mode, cudaStream_t st,
                                   double scale = 0.0) {
  using T = typename Cx<R>::T;
  int W = 0, cb = 0;
  size_t smem = 0;
  if (!choose_shape<R>(m, 1LL << lo, 1, &W, &cb, &smem))
    return fail(HHL_ERR_UNSUPPORTED, "register too large for one cluster");
  if (lo == 0 && cb == 0 && (mode == 3 || mode == 4) && getenv("HHL_LOWBITS_PLAIN") == nullptr)
    return lowbits_transform<R>(state, n, m, mode, (R)(scale != 0.0 ? scale : 1.0 / sqrt((double)(1LL << m))), st);
  const int64_t cols = (1LL << (n - m)) / W;
  if ((cols << cb) > 0x7fffffffLL) return fail(HHL_ERR_UNSUPPORTED, "too many columns for one launch");
  const int grid = (int)(cols << cb);
  T* S = (T*)state;
  R sc = (R)(scale != 0.0 ? scale : 1.0 / sqrt((double)(1LL << m)));
  void* args[] = {&S, &lo, &m, &W, &mode, &sc};
  switch (cb) {
    case 0: return launch_cluster(k_register_transform<R, 0>, grid, cb, smem, st, "k_register_transform", args);
    case 1: return launch_cluster(k_register_transform<R, 1>, grid, cb, smem, st, "k_register_transform", args);
    case 2: return launch_cluster(k_register_transform<R, 2>, grid, cb, smem, st, "k_register_transform", args);
    default: return launch_cluster(k_register_transform<R, 3>, grid, cb, smem, st, "k_register_transform", args);
  }
}

// ------------------------------------------------------------------ split register passes
// For a large state the clock transforms above are bounded by DRAM efficiency, not by the
// butterflies: a column block of W = 4 complex64 amplitudes is a 32-byte segment per row,
// and row segments that short reach about a quarter of the copy bandwidth on GB300 (128-byte
// segments reach over 90%). A whole 2^13-row column block of 256-byte segments (2 MiB) does
// not fit one SM, so for large states the register transform is split over its bits: the
// register index c = c_lo + 2^m_lo c_hi is transformed by one pass over the m_hi high bits
// (tile: all c_hi rows of W columns at a fixed c_lo) and one over the m_lo low bits (tile:
// all c_lo rows at fixed high bits), each tile at most 128 rows x 256 bytes in shared memory.
// Radix-2 DIF and DIT stages only need the index bits below their own bit for the twiddle,
// so running the high-bit stages in one pass and the low-bit stages in the other is the same
// sequence of butterflies as the single-pass transform.
//
// Clock block (a3 + a4 + the QFT of a5) as three passes:
//   A  inverse-QFT DIF stages on the high bits: anc = 0 half -> anc = 1 half (same rows; the
//      anc = 1 half is overwritten by this stage in every mode, so it serves as scratch),
//   B  inverse-QFT DIF stages on the low bits, the rotation at the bit-reversed frequency,
//      QFT DIT stages on the low bits: reads the anc = 1 half; writes cos(theta_y / 2) x_y to
//      the anc = 0 half at row y (or, when both halves are uncomputed, the cos part after the
//      same low stages at the tile's own rows) and the sin part back in place,
//   C  QFT DIT stages on the high bits, in place (anc = 1 half, or both halves).
// Pass B's write of row y = bitrev(p) goes to the anc = 0 half, which no pass reads after A,
// so the bit-reversed scatter cannot race with another tile's reads.
// kSplitMidSums: pass B of the postselected solve, which needs no anc = 0 half afterwards: the
// cos part is not stored; instead each thread sums cos^2(theta_y/2) |x_y|^2 and
// sin^2(theta_y/2) |x_y|^2, the weights of the anc = 0 and anc = 1 halves after the clock block
// (the QFT of pass C is unitary), and the block totals go to two FP64 accumulators.
enum SplitOp { kSplitDif = 0, kSplitMid = 1, kSplitDit = 2, kSplitHad = 3, kSplitMidSums = 4 };

// Per-thread sums of pass B's weights: compensated (Kahan) in FP32, plain in FP64 and
// double-float.
template <class R>
struct MidSums {
  R s[2], c[2];
  __device__ __forceinline__ void init() {
    s[0] = s[1] = c[0] = c[1] = R(0);
  }
  __device__ __forceinline__ void add(int i, R v) {
    if constexpr (std::is_same<R, float>::value) {
      const float y = v - c[i];
      const float t = s[i] + y;
      c[i] = (t - s[i]) - y;
      s[i] = t;
    } else {
      s[i] = s[i] + v;
    }
  }
  __device__ __forceinline__ double total(int i) const {
    if constexpr (std::is_same<R, float>::value) return (double)s[i] - (double)c[i];
    else if constexpr (std::is_same<R, df>::value) return df_to_double(s[i]);
    else return s[i];
  }
};

constexpr int kSplitThreads = 256;
constexpr int kSplitSegBytes = 256;  // bytes per row segment of a tile
constexpr int kSplitMinBits = 4;     // tile rows >= 16
constexpr int kSplitMaxBits = 7;     // tile rows <= 128

struct SplitArgs {
  double* sums;        // kSplitMidSums: the two weights (accumulated)
  void* src;           // tiles are read here ...
  void* dst;           // ... and written back here at the same rows
  void* dst_cos;       // pass B: cos part (anc = 0 half)
  const void* rot;     // pass B: (cos(theta_y / 2), sin(theta_y / 2)) per y
  long long tiles;     // tiles in the launch
  long long region;    // amplitudes per outer block (2^(lo + m))
  int lo, m, b0, nb;   // register at index bits [lo, lo + m); this pass: register bits [b0, b0 + nb)
  int log_cb;          // 2^log_cb column blocks (tiles) per row
  double scale;        // pass B: 1 / sqrt(2^m); Hadamard pass: final scale
  float scale_f;       // the same in FP32 (GB300's FP64 pipe is narrow: no per-thread conversions)
  float scale_l;       // scale - scale_f (the double-float kernels)
  int scaled;          // scale != 1
};

template <class R>
__device__ __forceinline__ R split_scale(const SplitArgs& a) {
  if constexpr (std::is_same<R, df>::value) return df{a.scale_f, a.scale_l};
  else if constexpr (sizeof(R) == 4) return a.scale_f;
  else return a.scale;
}

// The complex128 passes compute in double-float (dfc in shared memory, the same 16 bytes as the
// double2 it replaces): a landed tile is converted in place once, and converted back as it is
// stored; tables in FP64 (the rotation table) are converted as they are read.
template <class T>
constexpr bool is_dfc() { return std::is_same<T, dfc>::value; }
template <class T>
__device__ __forceinline__ T amp_in(const void* table, long long i) {
  if constexpr (is_dfc<T>()) return dfc_from(static_cast<const double2*>(table)[i]);
  else return static_cast<const T*>(table)[i];
}
template <class T>
__device__ __forceinline__ uint4 unit_out(uint4 v) {
  if constexpr (is_dfc<T>()) {
    const double2 d = dfc_to(*reinterpret_cast<const dfc*>(&v));
    return *reinterpret_cast<const uint4*>(&d);
  } else {
    return v;
  }
}

template <class T>
struct SplitGeom {
  static constexpr int LW = sizeof(T) == 8 ? 5 : 4;  // W = 2^LW amplitudes = kSplitSegBytes
  static constexpr int MR = sizeof(T) == 8 ? 4 : 3;  // radix bits per shared-memory round trip
};

// The RB radix-2 stages of one group (same arithmetic as butterflies() above), with the
// twiddles of each stage formed once per distinct value: stage t needs 2^t factors
// base_t * exp(-2 pi i xr / 2^(t+1)), xr < 2^t.
template <class T, int RB, bool DIT, int MODE, class TW>
__device__ __forceinline__ void group_butterflies(T (&v)[1 << RB], int lo, int lo_bits, int m, const TW& tw,
                                                  bool conj) {
  constexpr int G = 1 << RB;
  using R = decltype(T().x);
#pragma unroll
  for (int tt = 0; tt < RB; ++tt) {
    const int t = DIT ? tt : (RB - 1 - tt);
    T f[1 << (RB - 1)];
    if (MODE == 0) {
      const int s = t + 1 + lo_bits;
      const T base = tw(lo << (m - s), conj);
      f[0] = base;
#pragma unroll
      for (int xr = 1; xr < (1 << t); ++xr) {
        const int k16 = xr << (3 - t);
        T w;
        w.x = root16<R>(k16, 0);
        w.y = conj ? -root16<R>(k16, 1) : root16<R>(k16, 1);
        f[xr] = cmul(base, w);
      }
    }
#pragma unroll
    for (int x = 0; x < G; ++x) {
      if (x & (1 << t)) continue;
      const int x1 = x | (1 << t);
      T a = v[x], b = v[x1];
      if (MODE == 0) {
        const T fx = f[x & ((1 << t) - 1)];
        if (DIT) {
          b = cmul(b, fx);
          v[x] = cadd(a, b);
          v[x1] = csub(a, b);
        } else {
          v[x] = cadd(a, b);
          v[x1] = cmul(csub(a, b), fx);
        }
      } else {
        v[x] = cadd(a, b);
        v[x1] = csub(a, b);
      }
    }
  }
}

// One radix-2^RB pass over tile bits [TB, TB + RB) of the row-major tile X[row * W + w]
// (2^NB rows). Tile row j is register index lo_fixed + (j << b0) + (fixed bits above).
// With a whole-register transform (inner_base >= 0) the tile's columns are register bits
// too: the index below the pass's bits is inner_base + w + ((lo_fixed + (lo << b0)) << shift).
// CV (double-float tiles): the tile still holds the landed FP64 amplitudes, converted as this
// first pass loads them (each element is loaded and stored back by the same thread).
template <class T, int NB, int TB, int RB, bool DIT, int MODE, int LW, bool CV, class TW>
__device__ __forceinline__ void tile_pass(T* X, int b0, int lo_fixed, int m, const TW& tw, bool conj, int inner_base,
                                          int shift) {
  constexpr int W = 1 << LW, G = 1 << RB;
  constexpr int total = W << (NB - RB);
#pragma unroll 1
  for (int g = threadIdx.x; g < total; g += blockDim.x) {
    const int w = g & (W - 1);
    const int gg = g >> LW;
    const int lo = gg & ((1 << TB) - 1);
    const int row0 = ((gg >> TB) << (TB + RB)) + lo;
    T* q = X + (row0 << LW) + w;
    T v[G];
#pragma unroll
    for (int x = 0; x < G; ++x) {
      if constexpr (CV) v[x] = amp_in<T>(q, (long long)x << (TB + LW));
      else v[x] = q[x << (TB + LW)];
    }
    if (inner_base >= 0)
      group_butterflies<T, RB, DIT, MODE>(v, inner_base + w + ((lo_fixed + (lo << b0)) << shift), shift + b0 + TB, m,
                                          tw, conj);
    else
      group_butterflies<T, RB, DIT, MODE>(v, lo_fixed + (lo << b0), b0 + TB, m, tw, conj);
#pragma unroll
    for (int x = 0; x < G; ++x) q[x << (TB + LW)] = v[x];
  }
}

// All NB stages of a tile in passes of at most MR bits (DIF: high bits first), a barrier
// after each pass.
template <class T, int NB, bool DIT, int MODE, int LW = SplitGeom<T>::LW, int Q = 0, int DONE = 0, bool CV = false,
          class TW>
__device__ __forceinline__ void tile_stages(T* X, int b0, int lo_fixed, int m, const TW& tw, bool conj,
                                            int inner_base = -1, int shift = 0) {
  constexpr int MR = SplitGeom<T>::MR;
  constexpr int NPASS = (NB + MR - 1) / MR;
  if constexpr (Q < NPASS) {
    constexpr int RB = (NB - DONE) / (NPASS - Q);
    constexpr int TB = DIT ? DONE : NB - DONE - RB;
    tile_pass<T, NB, TB, RB, DIT, MODE, LW, CV && Q == 0>(X, b0, lo_fixed, m, tw, conj, inner_base, shift);
    __syncthreads();
    tile_stages<T, NB, DIT, MODE, LW, Q + 1, DONE + RB, false>(X, b0, lo_fixed, m, tw, conj, inner_base, shift);
  }
}

__device__ __forceinline__ void split_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void split_cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ void split_cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Tile rows <-> shared memory in 16-byte units. Thread t moves the units t + k * 256: its
// column unit h = t & 15 is fixed and its row advances by 16 per k, so the global address
// advances by a constant stride. Loads are asynchronous copies (cp.async), so a tile can be
// fetched while the previous one is transformed.
template <class T, int NB>
__device__ __forceinline__ void tile_issue(T* X, const T* base, long long row_units, long long row0, int b0) {
  constexpr int upr = kSplitSegBytes / 16;
  constexpr int total = (1 << NB) * upr;
  constexpr int per_thread = total / kSplitThreads;
  static_assert(total % kSplitThreads == 0, "tile units must be a multiple of the block");
  const int h = threadIdx.x & (upr - 1), j0 = threadIdx.x / upr;
  const uint4* src = reinterpret_cast<const uint4*>(base) + (row0 + ((long long)j0 << b0)) * row_units + h;
  const long long step = ((long long)(kSplitThreads / upr) << b0) * row_units;
  uint4* dst = reinterpret_cast<uint4*>(X) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < per_thread; ++k) split_cp_async16(dst + k * kSplitThreads, src + k * step);
}

template <class T, int NB, bool CS = false, class S>
__device__ __forceinline__ void tile_store(T* base, const T* X, long long row_units, long long row0, int b0, S scale,
                                           bool scaled) {
  constexpr int upr = kSplitSegBytes / 16;
  constexpr int per = 16 / sizeof(T);
  constexpr int per_thread = (1 << NB) * upr / kSplitThreads;
  const int h = threadIdx.x & (upr - 1), j0 = threadIdx.x / upr;
  uint4* dst = reinterpret_cast<uint4*>(base) + (row0 + ((long long)j0 << b0)) * row_units + h;
  const long long step = ((long long)(kSplitThreads / upr) << b0) * row_units;
  const uint4* src = reinterpret_cast<const uint4*>(X) + threadIdx.x;
#pragma unroll
  for (int k = 0; k < per_thread; ++k) {
    uint4 v = src[k * kSplitThreads];
    if (scaled) {
      T* t = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int q = 0; q < per; ++q) t[q] = cscale(t[q], scale);
    }
    v = unit_out<T>(v);
    if constexpr (CS) __stcs(dst + k * step, v);  // evict-first in L2
    else dst[k * step] = v;
  }
}

// Position of tile t: column block ib, fixed register bits f, outer block o.
struct TilePos {
  long long row0, base_amp;
  int lo_fixed, hi_fixed;
  int inner_base;  // first inner index of the tile's columns
};

template <int NB, int LW>
__device__ __forceinline__ TilePos tile_pos(const SplitArgs& a, long long t) {
  const int other = a.m - NB;
  const long long ib = t & (((long long)1 << a.log_cb) - 1);
  const long long rest = t >> a.log_cb;
  const int f = (int)(rest & ((1LL << other) - 1));
  const long long o = rest >> other;
  TilePos q;
  q.lo_fixed = f & ((1 << a.b0) - 1);
  q.hi_fixed = f >> a.b0;
  q.row0 = q.lo_fixed + ((long long)q.hi_fixed << (a.b0 + NB));
  q.base_amp = o * a.region + (ib << LW);
  q.inner_base = (int)(ib << LW);
  return q;
}

// The work on one landed tile of a split pass (transform stages, the pass's epilogue and the
// store back), shared by the streaming passes and the L2-staged group passes below.
template <class R, int OP, bool FULL, int NB, bool WHOLE, bool CS = false, class TW>
__device__ __forceinline__ void split_tile(const SplitArgs& a, const TilePos& q, typename Cx<R>::T* X,
                                           typename Cx<R>::T* Y, const TW& tw, int mt, long long row_units,
                                           MidSums<R>* sums = nullptr) {
  using T = typename Cx<R>::T;
  constexpr int upr = kSplitSegBytes / 16;
  constexpr int per = 16 / sizeof(T);
  constexpr int LWT = SplitGeom<T>::LW;
  constexpr bool CVT = is_dfc<T>();  // the landed tile is converted by its first pass
  T* dst = static_cast<T*>(a.dst) + q.base_amp;
  if (WHOLE) {
    // whole-register QFT (DIF, + sign) or inverse QFT (DIT, - sign)
    if (OP == kSplitDif) tile_stages<T, NB, false, 0>(X, a.b0, q.lo_fixed, mt, tw, true, q.inner_base, a.lo);
    else tile_stages<T, NB, true, 0>(X, a.b0, q.lo_fixed, mt, tw, false, q.inner_base, a.lo);
    tile_store<T, NB, CS>(dst, X, row_units, q.row0, a.b0, (R)1, false);
  } else if (OP == kSplitDif) {
    tile_stages<T, NB, false, 0, LWT, 0, 0, CVT>(X, a.b0, q.lo_fixed, a.m, tw, false);
    tile_store<T, NB, CS>(dst, X, row_units, q.row0, a.b0, (R)1, false);
  } else if (OP == kSplitDit) {
    tile_stages<T, NB, true, 0, LWT, 0, 0, CVT>(X, a.b0, q.lo_fixed, a.m, tw, true);
    tile_store<T, NB, CS>(dst, X, row_units, q.row0, a.b0, (R)1, false);
  } else if (OP == kSplitHad) {
    tile_stages<T, NB, false, 1, LWT, 0, 0, CVT>(X, a.b0, q.lo_fixed, a.m, tw, false);
    tile_store<T, NB, CS>(dst, X, row_units, q.row0, a.b0, split_scale<R>(a), a.scaled != 0);
  } else {  // kSplitMid(Sums): b0 = 0, the tile holds every low bit of the rows hi_fixed << NB
    constexpr bool SUMS = OP == kSplitMidSums;
    tile_stages<T, NB, false, 0, LWT, 0, 0, CVT>(X, 0, 0, a.m, tw, false);
    const R s = split_scale<R>(a);
    uint4* cos_out = reinterpret_cast<uint4*>(static_cast<T*>(a.dst_cos) + q.base_amp);
    for (int u = threadIdx.x; u < (upr << NB); u += kSplitThreads) {
      const int j = u / upr, h = u - j * upr;
      const int y = bitrev_m(j + (q.hi_fixed << NB), a.m);
      const T r = amp_in<T>(a.rot, y);
      uint4 xv = reinterpret_cast<uint4*>(X)[u];
      uint4 keep, yv;
      T* xt = reinterpret_cast<T*>(&xv);
      T* kt = reinterpret_cast<T*>(&keep);
      T* yt = reinterpret_cast<T*>(&yv);
#pragma unroll
      for (int e = 0; e < per; ++e) {
        const T x = cscale(xt[e], s);
        if constexpr (SUMS) {
          const R w = x.x * x.x + x.y * x.y;
          sums->add(0, w * (r.x * r.x));
          sums->add(1, w * (r.y * r.y));
        } else if (FULL) {
          yt[e] = cscale(x, r.x * s);
        } else {
          kt[e] = cscale(x, r.x);
        }
        xt[e] = cscale(x, r.y * s);
      }
      reinterpret_cast<uint4*>(X)[u] = xv;
      if constexpr (!SUMS) {
        if (FULL) reinterpret_cast<uint4*>(Y)[u] = yv;
        else cos_out[(long long)y * row_units + h] = unit_out<T>(keep);
      }
    }
    __syncthreads();
    tile_stages<T, NB, true, 0>(X, 0, 0, a.m, tw, true);
    if (FULL) tile_stages<T, NB, true, 0>(Y, 0, 0, a.m, tw, true);
    tile_store<T, NB, CS>(dst, X, row_units, q.row0, 0, (R)1, false);
    if (FULL) tile_store<T, NB, CS>(reinterpret_cast<T*>(cos_out), Y, row_units, q.row0, 0, (R)1, false);
  }
}

// CTAs per SM the register budget is set for: three for complex64 and for the double-float
// passes with one transform per tile (80 registers, no spills; measured faster than two at
// 122-127 registers), two for the FP64-pipe forms and the double-float pass B (two transforms
// and the rotation per tile: measured slower at three).
template <class R, int OP>
constexpr int kSplitMinBlocks =
    (sizeof(R) == 4 || (std::is_same<R, df>::value && OP != kSplitMid && OP != kSplitMidSums)) ? 3 : 2;

// WHOLE: the register is the whole index range [0, lo + m) of each outer block, the tile
// rows are its bits [lo + b0, lo + b0 + NB) and the twiddles are those of the 2^(lo + m) point
// transform (four-level shared-memory tables); only the DIF and DIT passes are used this way.
template <class R, int OP, bool FULL, int NB, bool WHOLE = false>
__global__ void __launch_bounds__(kSplitThreads, kSplitMinBlocks<R, OP>) k_split_pass(SplitArgs a) {
  using T = typename Cx<R>::T;
  constexpr int LW = SplitGeom<T>::LW;
  constexpr int per = 16 / sizeof(T);
  constexpr size_t tile_amps = (size_t)1 << (NB + LW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* t0 = reinterpret_cast<T*>(smem_raw);
  T* t1 = t0 + 64;
  T* Xb = t0 + (WHOLE ? 1024 : twiddle_entries(a.m));  // two tile buffers (double buffering), then Y
  T* Y = Xb + 2 * tile_amps;
  if (!WHOLE && OP != kSplitHad) fill_twiddles<R>(t0, t1, a.m);
  if constexpr (WHOLE) fill_twiddle4<R>(t0, a.lo + a.m);  // first read after the barrier of the first tile
  using TW = typename std::conditional<WHOLE, Twiddle4<T>, Twiddle<T>>::type;
  TW tw;
  if constexpr (WHOLE) {
    tw.t = t0;
  } else {
    tw.t0 = t0;
    tw.t1 = t1;
  }
  const int mt = WHOLE ? a.lo + a.m : a.m;  // bits of the transform the twiddles belong to
  const int rows = 1 << NB;
  const long long row_units = ((long long)1 << a.lo) / per;  // 16-byte units per row
  long long t = blockIdx.x;
  if (t >= a.tiles) return;  // block-uniform
  MidSums<R> sums;
  sums.init();
  {
    const TilePos q = tile_pos<NB, LW>(a, t);
    tile_issue<T, NB>(Xb, static_cast<const T*>(a.src) + q.base_amp, row_units, q.row0, a.b0);
  }
  split_cp_async_commit();
  int buf = 0;
  for (; t < a.tiles; t += gridDim.x) {
    const long long tn = t + gridDim.x;
    if (tn < a.tiles) {
      const TilePos qn = tile_pos<NB, LW>(a, tn);
      tile_issue<T, NB>(Xb + (buf ^ 1) * tile_amps, static_cast<const T*>(a.src) + qn.base_amp, row_units, qn.row0,
                        a.b0);
    }
    split_cp_async_commit();
    split_cp_async_wait1();
    __syncthreads();  // the current tile has landed for every thread
    const TilePos q = tile_pos<NB, LW>(a, t);
    split_tile<R, OP, FULL, NB, WHOLE>(a, q, Xb + buf * tile_amps, Y, tw, mt, row_units, &sums);
    __syncthreads();  // this buffer is read out before it is refilled
    buf ^= 1;
  }
  if constexpr (OP == kSplitMidSums) {  // block totals of the two weights -> FP64 accumulators
    __shared__ double red[2][kSplitThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      double v = sums.total(i);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double v = 0.0;
      for (int w = 0; w < kSplitThreads / 32; ++w) v += red[threadIdx.x][w];
      atomicAdd(a.sums + threadIdx.x, v);
    }
  }
  (void)rows;
}

// The split path serves registers of 8..14 bits whose rows hold at least one 256-byte segment,
// in states too large for L2 (the single-pass kernels are faster on L2-resident states).
template <class R>
bool split_applies(int lo, int m, long long region_amps) {
  const size_t sz = sizeof(typename Cx<R>::T);
  if (m < 2 * kSplitMinBits || (m + 1) / 2 > kSplitMaxBits) return false;
  if (((size_t)1 << lo) * sz < (size_t)kSplitSegBytes) return false;
  if (getenv("HHL_FFT_SPLIT") != nullptr) return atoi(getenv("HHL_FFT_SPLIT")) != 0;  // tuning override
  return (size_t)region_amps * sz > ((size_t)256 << 20);
}

template <class R, int OP, bool FULL, int NB, bool WHOLE = false>
hhl_status launch_split_nb(const SplitArgs& a, cudaStream_t st, const char* name) {
  using T = typename Cx<R>::T;
  const size_t tile = ((size_t)1 << (NB + SplitGeom<T>::LW)) * sizeof(T);
  const size_t smem = (size_t)(WHOLE ? 1024 : twiddle_entries(a.m)) * sizeof(T) + ((OP == kSplitMid && FULL) ? 3 : 2) * tile;
  auto kern = k_split_pass<R, OP, FULL, NB, WHOLE>;
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  int dev = 0, sms = 0, occ = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  HHL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HHL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSplitThreads, smem));
  if (occ < 1) return fail(HHL_ERR_UNSUPPORTED, "split register pass does not fit an SM");
  const long long grid = std::min<long long>(a.tiles, (long long)occ * sms);
  HHL_PROF_BEGIN(st);
  kern<<<(unsigned)grid, kSplitThreads, smem, st>>>(a);
  HHL_LAUNCH_CHECK(name);
  return HHL_OK;
}

template <class R, int OP, bool FULL, bool WHOLE = false>
hhl_status launch_split(SplitArgs a, int outer, cudaStream_t st, const char* name) {
  using T = typename Cx<R>::T;
  a.log_cb = a.lo - SplitGeom<T>::LW;
  a.region = 1LL << (a.lo + a.m);
  a.scale_f = (float)a.scale;
  a.scale_l = (float)(a.scale - (double)a.scale_f);
  a.scaled = a.scale != 1.0;
  a.tiles = ((long long)outer << (a.log_cb + a.m - a.nb));
  switch (a.nb) {
    case 4: return launch_split_nb<R, OP, FULL, 4, WHOLE>(a, st, name);
    case 5: return launch_split_nb<R, OP, FULL, 5, WHOLE>(a, st, name);
    case 6: return launch_split_nb<R, OP, FULL, 6, WHOLE>(a, st, name);
    case 7: return launch_split_nb<R, OP, FULL, 7, WHOLE>(a, st, name);
    default: return fail(HHL_ERR_UNSUPPORTED, "split register pass: tile bits out of range");
  }
}

// ------------------------------------------------------------- L2-staged group passes
// The streaming split passes move the whole half through HBM once per pass. A group pass runs
// every pass of a transform on one 256-byte column block of all 2^m rows of a half (a
// "group": 2^m x 256 B, 2 MiB at m = 13 for complex64) before it moves on to the next: the
// G CTAs of a cluster share the group's tiles in each pass, and a cluster barrier (release /
// acquire at cluster scope, which orders the global stores of one pass before the loads of
// the next) separates the passes. The intermediate results stay in L2 as long as the groups
// in flight fit there, so the launch grid is bounded by an L2 budget, not only by occupancy;
// then the clock block reads the anc = 0 half once and writes both halves once, and the
// Hadamard layer reads and writes its half once. The last pass of a group stores with the
// evict-first cache operator (st.global.cs): its columns are finished, so they should leave
// L2 before the intermediates of the groups still in flight.
struct GroupArgs {
  SplitArgs ph[3];   // the passes, in order (finished by split_finish)
  long long groups;  // column blocks: 2^log_cb
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// One pass over the tiles of group ib: CTA `rank` of the cluster takes the group's tiles
// rank, rank + G, ... (double-buffered as in k_split_pass).
template <class R, int OP, bool FULL, int NB, bool CS = false>
__device__ __forceinline__ void group_phase(const SplitArgs& a, long long ib, int rank, int G,
                                            typename Cx<R>::T* Xb, typename Cx<R>::T* Y,
                                            const Twiddle<typename Cx<R>::T>& tw) {
  using T = typename Cx<R>::T;
  constexpr int LW = SplitGeom<T>::LW;
  constexpr int per = 16 / sizeof(T);
  constexpr size_t tile_amps = (size_t)1 << (NB + LW);
  const long long per_group = a.tiles >> a.log_cb;
  const long long row_units = ((long long)1 << a.lo) / per;
  long long u = rank;
  if (u >= per_group) return;  // block-uniform
  {
    const TilePos q = tile_pos<NB, LW>(a, ib + (u << a.log_cb));
    tile_issue<T, NB>(Xb, static_cast<const T*>(a.src) + q.base_amp, row_units, q.row0, a.b0);
  }
  split_cp_async_commit();
  int buf = 0;
  for (; u < per_group; u += G) {
    const long long un = u + G;
    if (un < per_group) {
      const TilePos qn = tile_pos<NB, LW>(a, ib + (un << a.log_cb));
      tile_issue<T, NB>(Xb + (buf ^ 1) * tile_amps, static_cast<const T*>(a.src) + qn.base_amp, row_units, qn.row0,
                        a.b0);
    }
    split_cp_async_commit();
    split_cp_async_wait1();
    __syncthreads();  // the current tile has landed for every thread
    const TilePos q = tile_pos<NB, LW>(a, ib + (u << a.log_cb));
    split_tile<R, OP, FULL, NB, false, CS>(a, q, Xb + buf * tile_amps, Y, tw, a.m, row_units);
    __syncthreads();  // this buffer is read out before it is refilled
    buf ^= 1;
  }
}

// KIND 0: the clock block (passes A, B, C of clock_block_split); KIND 1: the Hadamard layer
// (high bits, then low bits with the final scale). NBH / NBL: tile bits of the high / low passes.
template <class R, int KIND, bool FULL, int NBH, int NBL>
__global__ void __launch_bounds__(kSplitThreads, 3) k_group_pass(GroupArgs g) {
  using T = typename Cx<R>::T;
  constexpr int LW = SplitGeom<T>::LW;
  constexpr size_t tile_amps = (size_t)1 << (NBH + LW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* t0 = reinterpret_cast<T*>(smem_raw);
  T* t1 = t0 + 64;
  const int m = g.ph[0].m;
  T* Xb = t0 + (KIND == 0 ? twiddle_entries(m) : 0);  // two tile buffers, then Y (full clock block)
  T* Y = Xb + 2 * tile_amps;
  if (KIND == 0) fill_twiddles<R>(t0, t1, m);
  __syncthreads();  // the table is complete before the first butterfly
  Twiddle<T> tw;
  tw.t0 = t0;
  tw.t1 = t1;
  unsigned rank, G;
  asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(G));
  const long long cid = blockIdx.x / G, ncl = gridDim.x / G;
  // every CTA of a cluster runs the same groups, so all of them reach every barrier
  for (long long ib = cid; ib < g.groups; ib += ncl) {
    if constexpr (KIND == 0) {
      group_phase<R, kSplitDif, false, NBH>(g.ph[0], ib, (int)rank, (int)G, Xb, Y, tw);
      cluster_barrier();
      group_phase<R, kSplitMid, FULL, NBL>(g.ph[1], ib, (int)rank, (int)G, Xb, Y, tw);
      cluster_barrier();
      group_phase<R, kSplitDit, false, NBH, true>(g.ph[2], ib, (int)rank, (int)G, Xb, Y, tw);
    } else {
      group_phase<R, kSplitHad, false, NBH>(g.ph[0], ib, (int)rank, (int)G, Xb, Y, tw);
      cluster_barrier();
      group_phase<R, kSplitHad, false, NBL, true>(g.ph[1], ib, (int)rank, (int)G, Xb, Y, tw);
    }
    // the next group touches other columns only: no barrier before its first pass
  }
}

// Derived fields of a split pass over `outer` blocks (as launch_split sets them).
template <class R>
void split_finish(SplitArgs& a, int outer) {
  using T = typename Cx<R>::T;
  a.log_cb = a.lo - SplitGeom<T>::LW;
  a.region = 1LL << (a.lo + a.m);
  a.scale_f = (float)a.scale;
  a.scale_l = (float)(a.scale - (double)a.scale_f);
  a.scaled = a.scale != 1.0;
  a.tiles = ((long long)outer << (a.log_cb + a.m - a.nb));
}

// CTAs per cluster and the L2 budget (MiB) for the groups in flight; HHL_GROUP_SHAPE="G,MiB"
// overrides (tuning).
inline void group_shape(int* G, int* budget_mib) {
  *G = 8;
  *budget_mib = 128;
  if (const char* env = getenv("HHL_GROUP_SHAPE")) {
    int g = 0, b = 0;
    if (sscanf(env, "%d,%d", &g, &b) == 2 && (g == 1 || g == 2 || g == 4 || g == 8 || g == 16) && b >= 1 &&
        b <= 4096) {
      *G = g;
      *budget_mib = b;
    }
  }
}

template <class R, int KIND, bool FULL, int NBH, int NBL>
hhl_status launch_group_nb(const GroupArgs& g, int outer, cudaStream_t st, const char* name) {
  using T = typename Cx<R>::T;
  constexpr int LW = SplitGeom<T>::LW;
  const int m = g.ph[0].m;
  const size_t tile = ((size_t)1 << (NBH + LW)) * sizeof(T);
  const size_t smem = (KIND == 0 ? (size_t)twiddle_entries(m) * sizeof(T) : 0) + 2 * tile +
                      ((KIND == 0 && FULL) ? ((size_t)1 << (NBL + LW)) * sizeof(T) : 0);
  auto kern = k_group_pass<R, KIND, FULL, NBH, NBL>;
  int G = 8, budget = 128;
  group_shape(&G, &budget);
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  if (G > 8) HHL_CUDA_TRY(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(kSplitThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)G;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3((unsigned)G);
  int max_clusters = 0;
  HHL_CUDA_TRY(cudaOccupancyMaxActiveClusters(&max_clusters, (const void*)kern, &cfg));
  if (max_clusters < 1) return fail(HHL_ERR_UNSUPPORTED, "group pass: no cluster fits");
  const long long group_bytes = ((long long)outer << m) * kSplitSegBytes;
  long long n_cl = std::min<long long>(max_clusters, std::max<long long>(1, ((long long)budget << 20) / group_bytes));
  n_cl = std::min<long long>(n_cl, g.groups);
  cfg.gridDim = dim3((unsigned)(n_cl * G));
  GroupArgs ga = g;
  void* args[1] = {&ga};
  HHL_PROF_BEGIN(st);
  cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)kern, args);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g_prof_on.load(std::memory_order_relaxed)) prof_end(name);
    return cuda_fail(e, name);
  }
  HHL_LAUNCH_CHECK(name);
  return HHL_OK;
}

template <class R, int KIND, bool FULL>
hhl_status launch_group(const GroupArgs& g, int outer, cudaStream_t st, const char* name) {
  switch (g.ph[0].m) {
    case 8: return launch_group_nb<R, KIND, FULL, 4, 4>(g, outer, st, name);
    case 9: return launch_group_nb<R, KIND, FULL, 5, 4>(g, outer, st, name);
    case 10: return launch_group_nb<R, KIND, FULL, 5, 5>(g, outer, st, name);
    case 11: return launch_group_nb<R, KIND, FULL, 6, 5>(g, outer, st, name);
    case 12: return launch_group_nb<R, KIND, FULL, 6, 6>(g, outer, st, name);
    case 13: return launch_group_nb<R, KIND, FULL, 7, 6>(g, outer, st, name);
    case 14: return launch_group_nb<R, KIND, FULL, 7, 7>(g, outer, st, name);
    default: return fail(HHL_ERR_UNSUPPORTED, "group pass: register bits out of range");
  }
}

// ------------------------------------------------------------- one-pass clustered clock block
// The clock block of a large state in one HBM pass: a cluster of 8 CTAs holds one 128-byte
// column block of all 2^m clock rows (m <= 13: 1 MiB for complex64), CTA r the rows
// p = 8 j + r. The inverse-QFT DIF stages on the top m - 3 bits are local to each CTA; the
// three stages on bits 2..0 pair rows of different CTAs. For those, CTA r takes the positions
// j in [r J/8, (r+1) J/8) of every CTA (J = 2^(m-3)), gathers the 8 values of a position
// through distributed shared memory, runs the last three DIF stages, the rotation at the
// bit-reversed frequency (storing the cos part to the anc = 0 half) and the first three DIT
// stages of the QFT, and writes the 8 results back to their owners: one exchange, no
// butterfly computed twice. Then each CTA runs the remaining DIT stages locally and stores its
// rows to the anc = 1 half: the half is read once and both halves are written once.
template <class R>
hhl_status whole_tables(int n, const void* out[3]);

constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 256;
constexpr int kClusterSegBytes = 64;  // bytes per row segment: 64 KiB per CTA at m = 13, 2 CTAs per SM

template <class R, int NB>
__global__ void __launch_bounds__(kClusterThreads, 2) k_clock_cluster(typename Cx<R>::T* __restrict__ S,
                                                                    const typename Cx<R>::T* __restrict__ rot,
                                                                    int n_s, int m, R scale, Twiddle3<typename Cx<R>::T> tw) {
  using T = typename Cx<R>::T;
  constexpr int LW = sizeof(T) == 8 ? 3 : 2;  // W = kClusterSegBytes of amplitudes per row
  constexpr int W = 1 << LW;
  constexpr int J = 1 << NB;                  // local rows
  constexpr int per = 16 / sizeof(T);
  constexpr int upr = W / per;                // 16-byte units per row segment
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  T* X = reinterpret_cast<T*>(smem_raw);
  const int64_t N = 1LL << n_s;
  const int64_t half = N << m;
  const int64_t j0 = (int64_t)(blockIdx.x / kClusterCtas) * W;  // first system column
  T* S0 = S;
  T* S1 = S + half;
  const int64_t row_units = N / per;  // 16-byte units per state row
  // load rows p = 8 j + r
  {
    const uint4* src = reinterpret_cast<const uint4*>(S0 + j0);
    uint4* dst = reinterpret_cast<uint4*>(X);
    for (int u0 = threadIdx.x; u0 < J * upr; u0 += kClusterThreads * 4) {
      uint4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = u0 + k * kClusterThreads;
        if (u < J * upr) v[k] = src[((int64_t)kClusterCtas * (u / upr) + r) * row_units + (u % upr)];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int u = u0 + k * kClusterThreads;
        if (u < J * upr) dst[u] = v[k];
      }
    }
  }
  __syncthreads();
  // inverse QFT: DIF stages on register bits 3 .. m-1 (row index p = r + 8 j)
  tile_stages<T, NB, false, 0, LW>(X, 3, r, m, tw, false);
  cl.sync();
  // the three cross-CTA stages, the rotation and the first three QFT stages on this CTA's share
  {
    T* rem[kClusterCtas];
#pragma unroll
    for (int q = 0; q < kClusterCtas; ++q) rem[q] = cl.map_shared_rank(X, q);
    constexpr int share = (J / kClusterCtas) * W;  // positions per CTA
    uint4* cos_out = reinterpret_cast<uint4*>(S0 + j0);
    for (int e = threadIdx.x; e < share; e += kClusterThreads) {
      const int jj = r * (J / kClusterCtas) + (e >> LW), w = e & (W - 1);
      const int off = (jj << LW) + w;
      T v[kClusterCtas];
#pragma unroll
      for (int q = 0; q < kClusterCtas; ++q) v[q] = rem[q][off];
      group_butterflies<T, 3, false, 0>(v, 0, 0, m, tw, false);
#pragma unroll
      for (int q = 0; q < kClusterCtas; ++q) {
        const int y = bitrev_m(kClusterCtas * jj + q, m);
        const T rr = rot[y];
        const T x = cscale(v[q], scale);
        const T c = cscale(x, rr.x);
        v[q] = cscale(x, rr.y * scale);
        if constexpr (sizeof(T) == 8) {
          // pairs of columns make one 16-byte unit: the even lane of each pair stores both
          const T c1 = mk<R>(__shfl_down_sync(0xffffffffu, c.x, 1), __shfl_down_sync(0xffffffffu, c.y, 1));
          if ((w & 1) == 0) {
            uint4 pk;
            T* pt = reinterpret_cast<T*>(&pk);
            pt[0] = c;
            pt[1] = c1;
            cos_out[(int64_t)y * row_units + (w >> 1)] = pk;
          }
        } else {
          reinterpret_cast<T*>(cos_out)[(int64_t)y * N + w] = c;
        }
      }
      group_butterflies<T, 3, true, 0>(v, 0, 0, m, tw, true);
#pragma unroll
      for (int q = 0; q < kClusterCtas; ++q) rem[q][off] = v[q];
    }
  }
  cl.sync();
  // QFT: DIT stages on register bits 3 .. m-1
  tile_stages<T, NB, true, 0, LW>(X, 3, r, m, tw, true);
  // store rows p = 8 j + r of the anc = 1 half
  {
    uint4* dst = reinterpret_cast<uint4*>(S1 + j0);
    const uint4* src = reinterpret_cast<const uint4*>(X);
    for (int u = threadIdx.x; u < J * upr; u += kClusterThreads)
      dst[((int64_t)kClusterCtas * (u / upr) + r) * row_units + (u % upr)] = src[u];
  }
}

// The Hadamard layer on the clock of a large state in one pass, with the same cluster layout:
// the Hadamard stages on bits 3 .. m-1 locally, the three on bits 2..0 through one exchange
// (the stages commute, so their order is free), scaled by 2^(-m/2) on the way.
template <class R, int NB>
__global__ void __launch_bounds__(kClusterThreads, 2) k_hadamard_cluster(typename Cx<R>::T* __restrict__ S, int n_s,
                                                                       int m, R scale) {
  using T = typename Cx<R>::T;
  constexpr int LW = sizeof(T) == 8 ? 3 : 2;
  constexpr int W = 1 << LW;
  constexpr int J = 1 << NB;
  constexpr int per = 16 / sizeof(T);
  constexpr int upr = W / per;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  T* X = reinterpret_cast<T*>(smem_raw);
  const Twiddle<T> tw{X, X};  // unused by the Hadamard butterflies
  const int64_t N = 1LL << n_s;
  const int64_t j0 = (int64_t)(blockIdx.x / kClusterCtas) * W;
  const int64_t row_units = N / per;
  uint4* base = reinterpret_cast<uint4*>(S + j0);
  for (int u0 = threadIdx.x; u0 < J * upr; u0 += kClusterThreads * 4) {
    uint4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int u = u0 + k * kClusterThreads;
      if (u < J * upr) v[k] = base[((int64_t)kClusterCtas * (u / upr) + r) * row_units + (u % upr)];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int u = u0 + k * kClusterThreads;
      if (u < J * upr) reinterpret_cast<uint4*>(X)[u] = v[k];
    }
  }
  __syncthreads();
  tile_stages<T, NB, false, 1, LW>(X, 3, r, m, tw, false);
  cl.sync();
  {
    T* rem[kClusterCtas];
#pragma unroll
    for (int q = 0; q < kClusterCtas; ++q) rem[q] = cl.map_shared_rank(X, q);
    constexpr int share = (J / kClusterCtas) * W;
    for (int e = threadIdx.x; e < share; e += kClusterThreads) {
      const int off = ((r * (J / kClusterCtas) + (e >> LW)) << LW) + (e & (W - 1));
      T v[kClusterCtas];
#pragma unroll
      for (int q = 0; q < kClusterCtas; ++q) v[q] = rem[q][off];
      group_butterflies<T, 3, false, 1>(v, 0, 0, m, tw, false);
#pragma unroll
      for (int q = 0; q < kClusterCtas; ++q) rem[q][off] = cscale(v[q], scale);
    }
  }
  cl.sync();
  for (int u = threadIdx.x; u < J * upr; u += kClusterThreads)
    base[((int64_t)kClusterCtas * (u / upr) + r) * row_units + (u % upr)] = reinterpret_cast<const uint4*>(X)[u];
}

template <class R, int NB>
hhl_status hadamard_cluster_nb(void* half_base, int n_s, int m, int outer, cudaStream_t st) {
  using T = typename Cx<R>::T;
  constexpr int W = kClusterSegBytes / (int)sizeof(T);
  auto kern = k_hadamard_cluster<R, NB>;
  const size_t smem = ((size_t)1 << NB) * kClusterSegBytes;
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  R scale = (R)(1.0 / sqrt((double)(1LL << m)));
  for (int o = 0; o < outer; ++o) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(((1LL << n_s) / W) * kClusterCtas));
    cfg.blockDim = dim3(kClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClusterCtas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    T* S = (T*)half_base + ((size_t)o << (n_s + m));
    int ns = n_s, mm = m;
    void* args[] = {&S, &ns, &mm, &scale};
    HHL_PROF_BEGIN(st);
    cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)kern, args);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (g_prof_on.load(std::memory_order_relaxed)) prof_end("k_hadamard_cluster");
      return cuda_fail(e, "k_hadamard_cluster");
    }
    HHL_LAUNCH_CHECK("k_hadamard_cluster");
  }
  return HHL_OK;
}

template <class R>
hhl_status hadamard_cluster(void* half_base, int n_s, int m, int outer, cudaStream_t st) {
  switch (m - 3) {
    case 5: return hadamard_cluster_nb<R, 5>(half_base, n_s, m, outer, st);
    case 6: return hadamard_cluster_nb<R, 6>(half_base, n_s, m, outer, st);
    case 7: return hadamard_cluster_nb<R, 7>(half_base, n_s, m, outer, st);
    case 8: return hadamard_cluster_nb<R, 8>(half_base, n_s, m, outer, st);
    case 9: return hadamard_cluster_nb<R, 9>(half_base, n_s, m, outer, st);
    default: return hadamard_cluster_nb<R, 10>(half_base, n_s, m, outer, st);
  }
}

template <class R>
bool hadamard_cluster_applies(int n_s, int m, long long region_amps) {  // opt-in, as above
  (void)region_amps;
  if (m < 8 || m > 13) return false;
  if (((size_t)1 << n_s) * sizeof(typename Cx<R>::T) < kClusterSegBytes) return false;
  const char* env = getenv("HHL_CLOCK_CLUSTER");
  return env != nullptr && atoi(env) != 0;
}

template <class R>
size_t clock_cluster_smem(int m) {
  return ((size_t)1 << (m - 3)) * kClusterSegBytes;
}

// The clustered one-pass clock block serves 8 <= m <= 13, postselect-early mode (the cos
// part goes straight to the anc = 0 half) and rows of at least 128 bytes, when
// HHL_CLOCK_CLUSTER=1: measured on GB300 it is slower than the three split passes (one CTA of
// 128 KiB per SM cannot overlap its load, exchange and store phases, and the cluster barrier
// after the exchange waits for the cos-part stores to drain), so it is not the default.
template <class R>
bool clock_cluster_applies(const Plan& p) {
  if (p.full || p.n_c < 8 || p.n_c > 13) return false;
  if ((size_t)p.N * sizeof(typename Cx<R>::T) < kClusterSegBytes) return false;
  const char* env = getenv("HHL_CLOCK_CLUSTER");
  return env != nullptr && atoi(env) != 0;
}

template <class R, int NB>
hhl_status clock_cluster_nb(const Plan& p, void* state, cudaStream_t st) {
  using T = typename Cx<R>::T;
  constexpr int W = kClusterSegBytes / (int)sizeof(T);
  const void* tabs[3];
  hhl_status ts = whole_tables<R>(p.n_c, tabs);
  if (ts != HHL_OK) return ts;
  Twiddle3<T> tw{(const T*)tabs[0], (const T*)tabs[1], (const T*)tabs[2]};
  auto kern = k_clock_cluster<R, NB>;
  const size_t smem = clock_cluster_smem<R>(p.n_c);
  HHL_CUDA_TRY(raise_dyn_smem((const void*)kern, smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((p.N / W) * kClusterCtas));
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kClusterCtas;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  T* S = (T*)state;
  const T* rot = (const T*)p.d_rot;
  int n_s = p.n_s, m = p.n_c;
  R scale = (R)(1.0 / sqrt((double)p.R));
  void* args[] = {&S, &rot, &n_s, &m, &scale, &tw};
  HHL_PROF_BEGIN(st);
  cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)kern, args);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g_prof_on.load(std::memory_order_relaxed)) prof_end("k_clock_cluster");
    return cuda_fail(e, "k_clock_cluster");
  }
  HHL_LAUNCH_CHECK("k_clock_cluster");
  return HHL_OK;
}

template <class R>
hhl_status clock_block_cluster(const Plan& p, void* state, cudaStream_t st) {
  switch (p.n_c - 3) {
    case 5: return clock_cluster_nb<R, 5>(p, state, st);
    case 6: return clock_cluster_nb<R, 6>(p, state, st);
    case 7: return clock_cluster_nb<R, 7>(p, state, st);
    case 8: return clock_cluster_nb<R, 8>(p, state, st);
    case 9: return clock_cluster_nb<R, 9>(p, state, st);
    default: return clock_cluster_nb<R, 10>(p, state, st);
  }
}

// Three-level twiddle tables of the 2^n-point transform, built on the host in FP64 once per
// (device, n, precision) and kept for the process.
template <class R>
hhl_status whole_tables(int n, const void* out[3]) {
  using T = typename Cx<R>::T;
  static std::mutex mu;
  static std::map<std::pair<int, int>, void*> cache;
  int dev = 0;
  HHL_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  void*& ptr = cache[{dev * 64 + n, (int)sizeof(R)}];
  if (ptr == nullptr) {
    std::vector<T> h(3 * 2048);
    const double L = ldexp(1.0, n);
    for (int lvl = 0; lvl < 3; ++lvl)
      for (int j = 0; j < 2048; ++j) {
        const double q = fmod(ldexp((double)j, 11 * lvl), L);  // exact: j 2^(11 lvl) < 2^53
        const double a = -2.0 * q / L;                         // angle / pi in [-2, 0]
        h[lvl * 2048 + j] = mk<R>((R)cospi(a), (R)sinpi(a));
      }
    void* d = nullptr;
    HHL_CUDA_TRY(cudaMalloc(&d, h.size() * sizeof(T)));
    cudaError_t e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return cuda_fail(e, "twiddle tables");
    }
    ptr = d;
  }
  for (int lvl = 0; lvl < 3; ++lvl) out[lvl] = static_cast<const T*>(ptr) + lvl * 2048;
  return HHL_OK;
}

// QFT (direction 0: DIF, natural order in, bit-reversed order out) or inverse QFT (direction
// 1: DIT, bit-reversed in, natural out) on the whole n-qubit register of each of `outer`
// consecutive states. The low g bits (g <= 12) form one pass over contiguous 2^g-amplitude
// chunks (their stages need no higher bits); the other n - g bits are split passes of 4..7
// bits over 256-byte row segments, with the twiddles of the 2^n-point transform.
template <class R>
hhl_status whole_register_impl(void* state, int n, int outer, int direction, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int g = n <= 12 ? n : std::min(12, n - 4);
  const int hbits = n - g;
  const int ngroups = (hbits + kSplitMaxBits - 1) / kSplitMaxBits;
  int logo = 0;
  while ((1 << logo) < outer) ++logo;
  if ((1 << logo) != outer) return fail(HHL_ERR_INVALID_ARG, "state count must be a power of two");
  const double scale = 1.0 / sqrt(ldexp(1.0, n));
  std::vector<std::pair<int, int>> groups;  // (first bit relative to g, bits), low to high
  for (int q = 0, done = 0; q < ngroups; ++q) {
    const int nb = (hbits - done) / (ngroups - q);
    groups.push_back({done, nb});
    done += nb;
  }
  SplitArgs a = {};
  a.src = state;
  a.dst = state;
  a.lo = g;
  a.m = hbits;
  a.scale = 1.0;
  if (direction == 0) {
    for (int q = ngroups - 1; q >= 0; --q) {
      a.b0 = groups[q].first;
      a.nb = groups[q].second;
      hhl_status s = launch_split<R, kSplitDif, false, true>(a, outer, st, "k_whole_pass");
      if (s != HHL_OK) return s;
    }
    return register_transform_impl<R>(state, n + logo, 0, g, 3, st, scale);
  }
  hhl_status s = register_transform_impl<R>(state, n + logo, 0, g, 4, st, scale);
  for (int q = 0; q < ngroups && s == HHL_OK; ++q) {
    a.b0 = groups[q].first;
    a.nb = groups[q].second;
    s = launch_split<R, kSplitDit, false, true>(a, outer, st, "k_whole_pass");
  }
  return s;
}

template <class R, bool FULL>
hhl_status clock_block_split(const Plan& p, void* state, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int m = p.n_c, m_lo = m / 2, m_hi = m - m_lo;
  T* S0 = static_cast<T*>(state);
  T* S1 = S0 + p.R * p.N;
  SplitArgs a = {};
  a.lo = p.n_s;
  a.m = m;
  a.rot = p.d_rot;
  // A: inverse-QFT stages on the high bits, anc = 0 -> anc = 1
  a.src = S0;
  a.dst = S1;
  a.b0 = m_lo;
  a.nb = m_hi;
  hhl_status s = launch_split<R, kSplitDif, false>(a, 1, st, "k_clock_pass_a");
  if (s != HHL_OK) return s;
  // B: low-bit stages, rotation, low-bit QFT stages
  a.src = S1;
  a.dst = S1;
  a.dst_cos = S0;
  a.b0 = 0;
  a.nb = m_lo;
  a.scale = 1.0 / sqrt((double)p.R);
  s = launch_split<R, kSplitMid, FULL>(a, 1, st, "k_clock_pass_b");
  if (s != HHL_OK) return s;
  // C: QFT stages on the high bits, in place (both halves when both are uncomputed)
  a.src = FULL ? S0 : S1;
  a.dst = a.src;
  a.b0 = m_lo;
  a.nb = m_hi;
  return launch_split<R, kSplitDit, false>(a, FULL ? 2 : 1, st, "k_clock_pass_c");
}

// The clock block of the postselected solve: passes A, B (weights summed into sums[0..1], no
// anc = 0 store) and C.
template <class R>
hhl_status clock_block_split_sums(const Plan& p, void* state, double* sums, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int m = p.n_c, m_lo = m / 2, m_hi = m - m_lo;
  T* S0 = static_cast<T*>(state);
  T* S1 = S0 + p.R * p.N;
  SplitArgs a = {};
  a.lo = p.n_s;
  a.m = m;
  a.rot = p.d_rot;
  a.sums = sums;
  a.src = S0;
  a.dst = S1;
  a.b0 = m_lo;
  a.nb = m_hi;
  hhl_status s = launch_split<R, kSplitDif, false>(a, 1, st, "k_clock_pass_a");
  if (s != HHL_OK) return s;
  a.src = S1;
  a.dst = S1;
  a.b0 = 0;
  a.nb = m_lo;
  a.scale = 1.0 / sqrt((double)p.R);
  s = launch_split<R, kSplitMidSums, false>(a, 1, st, "k_clock_pass_b");
  if (s != HHL_OK) return s;
  a.src = S1;
  a.dst = S1;
  a.b0 = m_lo;
  a.nb = m_hi;
  return launch_split<R, kSplitDit, false>(a, 1, st, "k_clock_pass_c");
}

template <class R>
hhl_status hadamard_split(void* base, int lo, int m, int outer, cudaStream_t st) {
  const int m_lo = m / 2, m_hi = m - m_lo;
  SplitArgs a = {};
  a.src = base;
  a.dst = base;
  a.lo = lo;
  a.m = m;
  a.b0 = m_lo;
  a.nb = m_hi;
  a.scale = 1.0;
  hhl_status s = launch_split<R, kSplitHad, false>(a, outer, st, "k_hadamard_pass");
  if (s != HHL_OK) return s;
  a.b0 = 0;
  a.nb = m_lo;
  a.scale = 1.0 / sqrt((double)(1LL << m));
  return launch_split<R, kSplitHad, false>(a, outer, st, "k_hadamard_pass");
}

// The group passes serve complex64 states on the split path: the Hadamard layer by default
// (measured faster than its two streaming passes), the clock block when HHL_GROUP=1 (measured
// slower than its three streaming passes: its groups in flight either overflow L2 or leave
// too few CTAs to hide the latency of the pass-by-pass barriers); HHL_GROUP=0 turns both off.
inline bool group_applies(bool clock) {
  const char* env = getenv("HHL_GROUP");
  if (env != nullptr) return atoi(env) != 0;
  return !clock;
}

// The three passes of clock_block_split as one L2-staged group launch.
template <bool FULL>
hhl_status clock_block_group(const Plan& p, void* state, cudaStream_t st) {
  using T = typename Cx<float>::T;
  const int m = p.n_c, m_lo = m / 2, m_hi = m - m_lo;
  T* S0 = static_cast<T*>(state);
  T* S1 = S0 + p.R * p.N;
  GroupArgs g = {};
  SplitArgs a = {};
  a.lo = p.n_s;
  a.m = m;
  a.rot = p.d_rot;
  a.scale = 1.0;
  a.src = S0;  // A: inverse-QFT stages on the high bits, anc = 0 -> anc = 1
  a.dst = S1;
  a.b0 = m_lo;
  a.nb = m_hi;
  g.ph[0] = a;
  split_finish<float>(g.ph[0], 1);
  a.src = S1;  // B: low-bit stages, rotation, low-bit QFT stages
  a.dst = S1;
  a.dst_cos = S0;
  a.b0 = 0;
  a.nb = m_lo;
  a.scale = 1.0 / sqrt((double)p.R);
  g.ph[1] = a;
  split_finish<float>(g.ph[1], 1);
  a.src = FULL ? S0 : S1;  // C: QFT stages on the high bits, in place (both halves when full)
  a.dst = a.src;
  a.dst_cos = nullptr;
  a.b0 = m_lo;
  a.nb = m_hi;
  a.scale = 1.0;
  g.ph[2] = a;
  split_finish<float>(g.ph[2], FULL ? 2 : 1);
  g.groups = 1LL << g.ph[0].log_cb;
  return launch_group<float, 0, FULL>(g, FULL ? 2 : 1, st, "k_clock_group");
}

// The two passes of hadamard_split as one L2-staged group launch.
inline hhl_status hadamard_group(void* base, int lo, int m, int outer, cudaStream_t st) {
  const int m_lo = m / 2, m_hi = m - m_lo;
  GroupArgs g = {};
  SplitArgs a = {};
  a.src = base;
  a.dst = base;
  a.lo = lo;
  a.m = m;
  a.b0 = m_lo;
  a.nb = m_hi;
  a.scale = 1.0;
  g.ph[0] = a;
  split_finish<float>(g.ph[0], outer);
  a.b0 = 0;
  a.nb = m_lo;
  a.scale = 1.0 / sqrt((double)(1LL << m));
  g.ph[1] = a;
  split_finish<float>(g.ph[1], outer);
  g.groups = 1LL << g.ph[0].log_cb;
  return launch_group<float, 1, false>(g, outer, st, "k_hadamard_group");
}

// Complex128 split passes on the FP64 pipe instead of double-float (HHL_FP64_PIPE=1).
inline bool fp64_pipe() {
  const char* env = getenv("HHL_FP64_PIPE");
  return env != nullptr && atoi(env) != 0;
}

}  // namespace

hhl_status launch_clock_block(const Plan& p, void* state, cudaStream_t st) {
  const long long half = p.R * p.N;
  if (p.prec == HHL_PREC_C64) {
    if (clock_cluster_applies<float>(p)) return clock_block_cluster<float>(p, state, st);
    if (split_applies<float>(p.n_s, p.n_c, half)) {
      if (group_applies(true)) return p.full ? clock_block_group<true>(p, state, st) : clock_block_group<false>(p, state, st);
      return p.full ? clock_block_split<float, true>(p, state, st) : clock_block_split<float, false>(p, state, st);
    }
    return p.full ? clock_block_impl<float, true>(p, state, st) : clock_block_impl<float, false>(p, state, st);
  }
  if (clock_cluster_applies<double>(p)) return clock_block_cluster<double>(p, state, st);
  if (split_applies<double>(p.n_s, p.n_c, half)) {
    if (fp64_pipe()) return p.full ? clock_block_split<double, true>(p, state, st) : clock_block_split<double, false>(p, state, st);
    return p.full ? clock_block_split<df, true>(p, state, st) : clock_block_split<df, false>(p, state, st);
  }
  return p.full ? clock_block_impl<double, true>(p, state, st) : clock_block_impl<double, false>(p, state, st);
}

hhl_status launch_clock_block_sums(const Plan& p, void* state, double* sums, bool* done, cudaStream_t st) {
  *done = false;
  const long long half = p.R * p.N;
  if (p.full) return HHL_OK;
  if (p.prec == HHL_PREC_C64) {
    if (clock_cluster_applies<float>(p) || !split_applies<float>(p.n_s, p.n_c, half) || group_applies(true)) return HHL_OK;
    *done = true;
    return clock_block_split_sums<float>(p, state, sums, st);
  }
  if (clock_cluster_applies<double>(p) || !split_applies<double>(p.n_s, p.n_c, half)) return HHL_OK;
  *done = true;
  return fp64_pipe() ? clock_block_split_sums<double>(p, state, sums, st) : clock_block_split_sums<df>(p, state, sums, st);
}

hhl_status launch_final_h(const Plan& p, void* state, cudaStream_t st) {
  // Hadamards on bits [n_s, n_s + n_c): on the anc = 1 half, or on the whole state (full).
  const int64_t half_amps = p.R * p.N;
  void* base = p.full ? state : (void*)((char*)state + half_amps * p.amp_bytes());
  const int n = p.full ? p.n : p.n - 1;
  const int outer = p.full ? 2 : 1;
  if (p.prec == HHL_PREC_C64) {
    if (hadamard_cluster_applies<float>(p.n_s, p.n_c, half_amps))
      return hadamard_cluster<float>(base, p.n_s, p.n_c, outer, st);
    if (!split_applies<float>(p.n_s, p.n_c, half_amps))
      return register_transform_impl<float>(base, n, p.n_s, p.n_c, 2, st);
    return group_applies(false) ? hadamard_group(base, p.n_s, p.n_c, outer, st)
                           : hadamard_split<float>(base, p.n_s, p.n_c, outer, st);
  }
  if (hadamard_cluster_applies<double>(p.n_s, p.n_c, half_amps))
    return hadamard_cluster<double>(base, p.n_s, p.n_c, outer, st);
  if (!split_applies<double>(p.n_s, p.n_c, half_amps)) return register_transform_impl<double>(base, n, p.n_s, p.n_c, 2, st);
  return fp64_pipe() ? hadamard_split<double>(base, p.n_s, p.n_c, outer, st) : hadamard_split<df>(base, p.n_s, p.n_c, outer, st);
}

hhl_status launch_qft_whole(void* state, int n, int outer, int direction, int prec, cudaStream_t st) {
  return prec == HHL_PREC_C64 ? whole_register_impl<float>(state, n, outer, direction, st)
                              : whole_register_impl<double>(state, n, outer, direction, st);
}

hhl_status launch_qft_register(void* state, int n, int lo, int m, bool inverse, int prec, cudaStream_t st) {
  const int mode = inverse ? 1 : 0;
  return prec == HHL_PREC_C64 ? register_transform_impl<float>(state, n, lo, m, mode, st)
                              : register_transform_impl<double>(state, n, lo, m, mode, st);
}

}  // namespace hhl
