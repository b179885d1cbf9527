// Fused register blocks over the clock register (or any register of <= 13 qubits):
// the clock block of the HHL circuit (inverse QFT + eigenvalue-inversion RY + QFT), the
// Hadamard layer on the clock, and stand-alone QFT / inverse QFT blocks.
//
// A CTA holds W "columns" in shared memory, each the 2^m amplitudes that differ only in
// the register's bits (stride 2^lo in the state), with W consecutive values of the lower
// bits so that each global access covers W contiguous amplitudes. The transform of a
// column is applied in passes of up to 4 qubits: a thread loads the 2^r amplitudes of one
// group into registers, applies the r radix-2 stages (Hadamard + controlled-phase layers
// of the QFT circuit, i.e. Cooley-Tukey butterflies) in registers, and stores them back,
// so a 12-qubit register costs 3 shared-memory round trips instead of 12. Columns are
// padded by one element per 16 to spread the strided group accesses over the banks.
//
// Orders: decimation in frequency (DIF) takes natural order and leaves the result in
// bit-reversed order; decimation in time (DIT) takes bit-reversed order and returns natural
// order. The clock block chains DIF (inverse QFT) -> rotation at bit-reversed positions ->
// DIT (QFT), so no explicit bit-reversal permutation (the QFT's swap layer) is ever applied.
#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kFftThreads = 256;
constexpr size_t kFftSmemCap = 220 * 1024;

__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }
__device__ __forceinline__ int bitrev_m(int x, int m) { return (int)(__brev((unsigned)x) >> (32 - m)); }

// Global <-> shared column blocks in 16-byte units with kUnroll loads in flight per thread.
// Row c of the block holds W contiguous amplitudes at src + c * row_stride; they go to
// X[w * Lp + pad16(pos(c))], pos = identity or bit reversal over m bits.
constexpr int kUnroll = 8;

// Element-wise form for blocks narrower than one 16-byte unit (W * sizeof(T) < 16).
template <class T>
__device__ void load_block_elems(T* X, int Lp, const T* src, int64_t row_stride, int L, int W, int m, bool rev) {
  const int total = L * W;
  for (int b = threadIdx.x; b < total; b += blockDim.x * kUnroll) {
    T v[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int u = b + k * blockDim.x;
      if (u < total) {
        const int c = u / W, w = u - c * W;
        v[k] = src[(int64_t)c * row_stride + w];
      }
    }
#pragma unroll
    for (int k = 0; k < kUnroll; ++k) {
      const int u = b + k * blockDim.x;
      if (u < total) {
        const int c = u / W, w = u - c * W;
        X[w * Lp + pad16(rev ? bitrev_m(c, m) : c)] = v[k];
      }
    }
  }
}

template <class T, class S>
__device__ void store_block_elems(T* dst, int64_t row_stride, const T* X, int Lp, int L, int W, S scale) {
  for (int u = threadIdx.x; u < L * W; u += blockDim.x) {
    const int c = u / W, w = u - c * W;
    dst[(int64_t)c * row_stride + w] = cscale(X[w * Lp + pad16(c)], scale);
  }
}

template <class T>
__device__ void load_block(T* X, int Lp, const T* src, int64_t row_stride, int L, int W, int m, bool rev) {
  constexpr int per = 16 / sizeof(T);
  const int upr = W / per;  // 16-byte units per row (W is a multiple of per)
  const int total = L * upr;
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
        const int pos = pad16(rev ? bitrev_m(c, m) : c);
        const T* t = reinterpret_cast<const T*>(&v[k]);
#pragma unroll
        for (int q = 0; q < per; ++q) X[(h * per + q) * Lp + pos] = t[q];
      }
    }
  }
}

// dst row c (W contiguous amplitudes) = scale * X[w * Lp + pad16(c)].
template <class T, class S>
__device__ void store_block(T* dst, int64_t row_stride, const T* X, int Lp, int L, int W, S scale) {
  constexpr int per = 16 / sizeof(T);
  const int upr = W / per;
  const int total = L * upr;
  for (int u = threadIdx.x; u < total; u += blockDim.x) {
    const int c = u / upr, h = u - c * upr;
    uint4 v;
    T* t = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int q = 0; q < per; ++q) t[q] = cscale(X[(h * per + q) * Lp + pad16(c)], scale);
    *reinterpret_cast<uint4*>(dst + (int64_t)c * row_stride + h * per) = v;
  }
}

template <class R>
__device__ void fill_twiddles(typename Cx<R>::T* tw, int m) {
  const int L = 1 << m;
  for (int j = threadIdx.x; j < L / 2; j += blockDim.x) {
    R s, c;
    if constexpr (sizeof(R) == 4) {
      sincospif(-2.0f * (float)j / (float)L, &s, &c);
    } else {
      sincospi(-2.0 * (double)j / (double)L, &s, &c);
    }
    tw[j] = mk<R>(c, s);
  }
}

// One pass of RB radix-2 stages (global stages s0-RB+1 .. s0) on every group of every column.
// MODE 0: DFT butterflies with twiddles tw[q] = exp(-2 pi i q / L) (conjugated if conj);
// MODE 1: Hadamard butterflies (no twiddles). DIT selects the stage order and twiddle side.
template <class T, int RB, bool DIT, int MODE>
__device__ void radix_pass(T* X, int Lp, int W, const T* tw, int m, int s0, bool conj) {
  constexpr int G = 1 << RB;
  const int lo_bits = s0 - RB;
  const int gpc_bits = m - RB;  // groups per column = 2^(m - RB)
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
#pragma unroll
    for (int tt = 0; tt < RB; ++tt) {
      const int t = DIT ? tt : (RB - 1 - tt);
      const int s = t + 1 + lo_bits;  // global stage of this butterfly layer
#pragma unroll
      for (int x = 0; x < G; ++x) {
        if (x & (1 << t)) continue;
        const int x1 = x | (1 << t);
        T a = v[x], b = v[x1];
        if (MODE == 0) {
          const int j = ((x & ((1 << t) - 1)) << lo_bits) + lo;
          T f = tw[j << (m - s)];
          if (conj) f.y = -f.y;
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
#pragma unroll
    for (int x = 0; x < G; ++x) col[pad16(base + (x << lo_bits))] = v[x];
  }
}

template <class T, bool DIT, int MODE>
__device__ void radix_dispatch(int r, T* X, int Lp, int W, const T* tw, int m, int s0, bool conj) {
  switch (r) {
    case 4: radix_pass<T, 4, DIT, MODE>(X, Lp, W, tw, m, s0, conj); break;
    case 3: radix_pass<T, 3, DIT, MODE>(X, Lp, W, tw, m, s0, conj); break;
    case 2: radix_pass<T, 2, DIT, MODE>(X, Lp, W, tw, m, s0, conj); break;
    default: radix_pass<T, 1, DIT, MODE>(X, Lp, W, tw, m, s0, conj); break;
  }
}

// Full transform of every column: DIF (natural -> bit-reversed) or DIT (bit-reversed ->
// natural), in passes of <= 4 stages.
template <class T, bool DIT, int MODE>
__device__ void column_transform(T* X, int Lp, int W, const T* tw, int m, bool conj) {
  const int npass = (m + 3) / 4;
  int done = 0;
  for (int p = 0; p < npass; ++p) {
    const int r = (m - done) / (npass - p);  // balanced pass sizes, each <= 4
    const int s0 = DIT ? done + r : m - done;
    radix_dispatch<T, DIT, MODE>(r, X, Lp, W, tw, m, s0, conj);
    done += r;
    __syncthreads();
  }
}

// Clock block (a3 + a4 + the QFT of a5).
template <class R, bool FULL>
__global__ void __launch_bounds__(kFftThreads) k_clock_block(typename Cx<R>::T* __restrict__ S,
                                                             const typename Cx<R>::T* __restrict__ rot, int n_s,
                                                             int n_c, int W) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << n_c, Lp = L + L / 16;
  const int64_t N = 1LL << n_s;
  const int64_t half = (int64_t)L * N;
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* X = tw + L / 2;
  T* Y = X + (size_t)W * Lp;
  fill_twiddles<R>(tw, n_c);
  const int64_t j0 = (int64_t)blockIdx.x * W;
  T* S0 = S;
  T* S1 = S + half;
  load_block(X, Lp, S0 + j0, N, L, W, n_c, false);
  __syncthreads();
  column_transform<T, false, 0>(X, Lp, W, tw, n_c, false);  // inverse QFT, bit-reversed result
  const R inv = (R)(1.0 / sqrt((double)L));
  // rotation at bit-reversed positions, in 16-byte units of W/per consecutive columns
  constexpr int per = 16 / sizeof(T);
  const int upr = W / per;
  for (int u = threadIdx.x; u < L * upr; u += blockDim.x) {
    const int p = u / upr, h = u - p * upr;
    const int y = bitrev_m(p, n_c);
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
  column_transform<T, true, 0>(X, Lp, W, tw, n_c, true);  // QFT, natural order
  if (FULL) column_transform<T, true, 0>(Y, Lp, W, tw, n_c, true);
  store_block(S1 + j0, N, X, Lp, L, W, inv);
  if (FULL) store_block(S0 + j0, N, Y, Lp, L, W, inv);
}

// Register transform on bits [lo, lo+m): mode 0 = QFT, 1 = inverse QFT, 2 = Hadamards.
template <class R>
__global__ void __launch_bounds__(kFftThreads) k_register_transform(typename Cx<R>::T* __restrict__ S, int lo, int m,
                                                                    int W, int mode) {
  using T = typename Cx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = 1 << m, Lp = L + L / 16;
  const int64_t inner = 1LL << lo;
  T* tw = reinterpret_cast<T*>(smem_raw);
  T* X = tw + L / 2;
  if (mode != 2) fill_twiddles<R>(tw, m);
  const int64_t groups = inner / W;
  const int64_t o = blockIdx.x / groups, g = blockIdx.x - o * groups;
  T* base = S + o * ((int64_t)L << lo) + g * W;
  constexpr int per = 16 / sizeof(T);
  if (W % per == 0) load_block(X, Lp, base, inner, L, W, m, mode != 2);
  else load_block_elems(X, Lp, base, inner, L, W, m, mode != 2);
  __syncthreads();
  if (mode == 2) column_transform<T, true, 1>(X, Lp, W, tw, m, false);
  else column_transform<T, true, 0>(X, Lp, W, tw, m, mode == 0);
  const R inv = (R)(1.0 / sqrt((double)L));
  if (W % per == 0) store_block(base, inner, X, Lp, L, W, inv);
  else store_block_elems(base, inner, X, Lp, L, W, inv);
}

template <class R>
size_t fft_smem(int m, int W, int buffers) {
  const size_t sz = sizeof(typename Cx<R>::T);
  const size_t L = (size_t)1 << m, Lp = L + L / 16;
  return L / 2 * sz + (size_t)buffers * W * Lp * sz;
}

template <class R>
hhl_status clock_block_impl(const Plan& p, void* state, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int bufs = p.full ? 2 : 1;
  const int per = 16 / (int)sizeof(T);
  int W = 8;
  while (W > per && (W > p.N || fft_smem<R>(p.n_c, W, bufs) > kFftSmemCap)) W >>= 1;
  if (W > p.N) return fail(HHL_ERR_UNSUPPORTED, "system register narrower than one 16-byte unit");
  const size_t smem = fft_smem<R>(p.n_c, W, bufs);
  if (smem > kFftSmemCap) return fail(HHL_ERR_UNSUPPORTED, "clock register too large for one shared-memory block");
  const int grid = (int)(p.N / W);
  if (p.full) {
    HHL_CUDA_TRY(cudaFuncSetAttribute(k_clock_block<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HHL_PROF_BEGIN(st);
    k_clock_block<R, true><<<grid, kFftThreads, smem, st>>>((T*)state, (const T*)p.d_rot, p.n_s, p.n_c, W);
  } else {
    HHL_CUDA_TRY(cudaFuncSetAttribute(k_clock_block<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HHL_PROF_BEGIN(st);
    k_clock_block<R, false><<<grid, kFftThreads, smem, st>>>((T*)state, (const T*)p.d_rot, p.n_s, p.n_c, W);
  }
  HHL_LAUNCH_CHECK("k_clock_block");
  return HHL_OK;
}

template <class R>
hhl_status register_transform_impl(void* state, int n, int lo, int m, int mode, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int64_t inner = 1LL << lo;
  const int per = 16 / (int)sizeof(T);
  int W = 8;
  while (W > 1 && (W > inner || (W > per && fft_smem<R>(m, W, 1) > kFftSmemCap))) W >>= 1;
  (void)per;
  const size_t smem = fft_smem<R>(m, W, 1);
  if (smem > kFftSmemCap) return fail(HHL_ERR_UNSUPPORTED, "register too large for one shared-memory block");
  const int64_t cols = (1LL << (n - m)) / W;
  if (cols > 0x7fffffffLL) return fail(HHL_ERR_UNSUPPORTED, "too many columns for one launch");
  HHL_CUDA_TRY(cudaFuncSetAttribute(k_register_transform<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  HHL_PROF_BEGIN(st);
  k_register_transform<R><<<(int)cols, kFftThreads, smem, st>>>((T*)state, lo, m, W, mode);
  HHL_LAUNCH_CHECK("k_register_transform");
  return HHL_OK;
}

}  // namespace

hhl_status launch_clock_block(const Plan& p, void* state, cudaStream_t st) {
  return p.prec == HHL_PREC_C64 ? clock_block_impl<float>(p, state, st) : clock_block_impl<double>(p, state, st);
}

hhl_status launch_final_h(const Plan& p, void* state, cudaStream_t st) {
  // Hadamards on bits [n_s, n_s + n_c): on the anc = 1 half, or on the whole state (full).
  const int64_t half_amps = p.R * p.N;
  void* base = p.full ? state : (void*)((char*)state + half_amps * p.amp_bytes());
  const int n = p.full ? p.n : p.n - 1;
  return p.prec == HHL_PREC_C64 ? register_transform_impl<float>(base, n, p.n_s, p.n_c, 2, st)
                                : register_transform_impl<double>(base, n, p.n_s, p.n_c, 2, st);
}

hhl_status launch_qft_register(void* state, int n, int lo, int m, bool inverse, int prec, cudaStream_t st) {
  const int mode = inverse ? 1 : 0;
  return prec == HHL_PREC_C64 ? register_transform_impl<float>(state, n, lo, m, mode, st)
                              : register_transform_impl<double>(state, n, lo, m, mode, st);
}

}  // namespace hhl
