// Controlled exp(i Ahat t_k) as a second-order Strang product of two-level gates, for a
// Toeplitz tridiagonal Ahat (the channel-flow operator of App. A.1 Eq. CDS).
//
// Ahat = E + O: E holds the 2x2 blocks [[d, o], [o, d]] on basis-state pairs (2i, 2i+1),
// O the couplings [[0, o], [o, 0]] on pairs (2i+1, 2i+2). One Strang step is
// S(tau) = E(tau/2) O(tau) E(tau/2) with E(s) = exp(i s E), and r steps merge into the
// layer list E(tau/2), O(tau), [E(tau), O(tau)] x (r-1), E(tau/2) (2r + 1 layers).
//
// Every layer acts inside one system-register row, so a pass applies up to 16 layers to a
// window of the row held in registers (temporal blocking): one warp owns 512 consecutive
// amplitudes, 16 per lane, so E pairs and all but one O pair per lane are in the lane's
// own registers and the remaining O pair crosses to the next lane by a warp shuffle. The
// window has a 16-amplitude halo on each side (lanes 0 and 31), as wide as the number of
// layers of a pass, and its 480-amplitude interior (lanes 1..30) is written back in place.
// The halos are the edges of the neighbouring interiors, which the same pass overwrites,
// so a small kernel first saves the 16 leading and 16 trailing amplitudes of every interior
// into a side buffer and the pass reads its halos from there: each pass moves the rows
// through HBM once (plus about 7% for the edges), in place.
#include <math.h>

#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kLaneAmps = 16;                 // amplitudes per lane
constexpr int kHalo = 16;                     // halo per side = max layers per pass
constexpr int kWin = 32 * kLaneAmps;          // 512 amplitudes per warp window
constexpr int kInterior = kWin - 2 * kHalo;   // 480 written back per warp
constexpr int kTrotThreads = 256;

__device__ __forceinline__ int64_t row_with_bit_t(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}

template <class T>
__device__ __forceinline__ T shfl_down1(T v) {
  T r;
  r.x = __shfl_down_sync(0xffffffffu, v.x, 1);
  r.y = __shfl_down_sync(0xffffffffu, v.y, 1);
  return r;
}

template <class T>
__device__ __forceinline__ T shfl_up1(T v) {
  T r;
  r.x = __shfl_up_sync(0xffffffffu, v.x, 1);
  r.y = __shfl_up_sync(0xffffffffu, v.y, 1);
  return r;
}

// Rotations R(th) = [[cos th, i sin th], [i sin th, cos th]] of one pass: the half-step
// E layers use th = (tau/2) o, the full E layers and the O layers th = tau o; the E-layer
// phases e^{i s d} are scalars on the row and are applied once, summed, at the pass end.
struct TrotBlocks {
  double ch, sh, cf, sf;   // cos / sin of (tau/2) o and tau o
  double pc, ps;           // cos / sin of the summed E phase of this pass
};

// (a, b) <- R(th) (a, b) with c = cos th, s = sin th.
template <class T, class R>
__device__ __forceinline__ void rot_apply(T& a, T& b, R c, R s) {
  const T na = mk<R>(c * a.x - s * b.y, c * a.y + s * b.x);
  const T nb = mk<R>(c * b.x - s * a.y, c * b.y + s * a.x);
  a = na;
  b = nb;
}

// side[(i * segs + s) * 32 + q]: q < 16 the first 16 interior amplitudes of segment s of
// subset row i, q >= 16 its last 16 (zero beyond the row end).
template <class R>
__global__ void k_trotter_edges(const typename Cx<R>::T* __restrict__ half, typename Cx<R>::T* __restrict__ side,
                                int n_s, int k, int64_t segs, int64_t m_sub) {
  const int64_t N = 1LL << n_s;
  const int64_t total = m_sub * segs * 32;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rs = e >> 5;
    const int q = (int)(e & 31);
    const int64_t i = rs / segs, s = rs - i * segs;
    const int64_t g = s * kInterior + (q < 16 ? q : kInterior - 32 + q);
    side[e] = g < N ? half[row_with_bit_t(i, k) * N + g] : mk<R>((R)0, (R)0);
  }
}

template <class R>
__global__ void __launch_bounds__(kTrotThreads) k_trotter_pass(typename Cx<R>::T* __restrict__ half,
                                                              const typename Cx<R>::T* __restrict__ side, int n_s,
                                                              int k, int64_t segs, int64_t m_sub, int l0, int l1,
                                                              int n_layers_total, TrotBlocks blk, int adjoint) {
  using T = typename Cx<R>::T;
  constexpr int per = 16 / sizeof(T);  // amplitudes per 16-byte unit
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (kTrotThreads / 32) + (threadIdx.x >> 5);
  if (gw >= m_sub * segs) return;  // warp-uniform: whole warps leave together
  const int64_t N = 1LL << n_s;
  const int64_t i = gw / segs, s = gw - i * segs;
  const int64_t g0 = s * kInterior;             // first interior amplitude
  const int64_t lane0 = g0 - kHalo + (int64_t)lane * kLaneAmps;  // even
  T* row = half + row_with_bit_t(i, k) * N;

  // Staging buffer of this warp: 32 x kLaneAmps amplitudes as 16-byte chunks, chunk c of
  // the window stored at position c ^ ((c / CPL) & 7) (CPL = chunks per lane) so that both
  // the coalesced pass (lane t <-> chunk q * 32 + t) and the blocked pass (lane t <-> its
  // CPL consecutive chunks) spread over the banks.
  constexpr int CPL = kLaneAmps / per;
  __shared__ uint4 stage_all[kTrotThreads / 32][32 * CPL];
  uint4* stage = stage_all[threadIdx.x >> 5];
  T x[kLaneAmps];
  const bool full_interior = (g0 + kInterior <= N);  // warp-uniform
  if (full_interior) {
    // lanes 1..30 of the window = the 480 interior amplitudes: coalesced 16-byte loads
    const uint4* src = reinterpret_cast<const uint4*>(row + g0);
    constexpr int chunks = kInterior / per;  // 30 * CPL
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = q * 32 + lane;
      if (c < chunks) {
        const int wc = c + CPL;  // window chunk (lane 0 holds the left halo)
        stage[wc ^ ((wc / CPL) & 7)] = src[c];
      }
    }
    __syncwarp();
    if (lane > 0 && lane < 31) {
      uint4* d = reinterpret_cast<uint4*>(x);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int wc = lane * CPL + q;
        d[q] = stage[wc ^ (lane & 7)];
      }
    }
  } else if (lane > 0 && lane < 31) {
#pragma unroll
    for (int q = 0; q < kLaneAmps; ++q) x[q] = lane0 + q < N ? row[lane0 + q] : mk<R>((R)0, (R)0);
  }
  if (lane == 0 || lane == 31) {
    const int64_t ns = lane == 0 ? s - 1 : s + 1;
    const int off = lane == 0 ? 16 : 0;  // the neighbour's last 16 / first 16
#pragma unroll
    for (int q = 0; q < kLaneAmps; ++q)
      x[q] = (ns >= 0 && ns < segs) ? side[(i * segs + ns) * 32 + off + q] : mk<R>((R)0, (R)0);
  }

  const R sg = adjoint ? (R)-1 : (R)1;  // the adjoint uses R(-th) and the conjugate phase
  const R ch = (R)blk.ch, sh = sg * (R)blk.sh, cf = (R)blk.cf, sf = sg * (R)blk.sf;
  // per-lane validity of the O pairs (j, j+1), j odd, 1 <= j and j + 1 <= N - 1
  const bool in_ok = lane0 >= 0 && lane0 + kLaneAmps - 2 <= N - 1;
  const bool right_ok = lane < 31 && lane0 + kLaneAmps - 1 >= 1 && lane0 + kLaneAmps <= N - 1;
  const bool left_ok = lane > 0 && lane0 - 1 >= 1 && lane0 <= N - 1;
  for (int l = l0; l < l1; ++l) {
    if ((l & 1) == 0) {
      // E layer: pairs (2p, 2p+1) inside each lane; pairs beyond the row are zero.
      const bool halfstep = (l == 0 || l == n_layers_total - 1);
      const R c = halfstep ? ch : cf, sn = halfstep ? sh : sf;
#pragma unroll
      for (int q = 0; q < kLaneAmps; q += 2) rot_apply(x[q], x[q + 1], c, sn);
    } else {
      const T right = shfl_down1(x[0]);           // next lane's first amplitude
      const T left = shfl_up1(x[kLaneAmps - 1]);  // previous lane's last amplitude
      if (in_ok) {
#pragma unroll
        for (int q = 1; q + 1 < kLaneAmps; q += 2) rot_apply(x[q], x[q + 1], cf, sf);
      } else {
#pragma unroll
        for (int q = 1; q + 1 < kLaneAmps; q += 2) {
          const int64_t j = lane0 + q;
          if (j >= 1 && j + 1 <= N - 1) rot_apply(x[q], x[q + 1], cf, sf);
        }
      }
      if (right_ok) {  // (this lane's last a, next lane's first b): a <- c a + i s b
        const T a = x[kLaneAmps - 1];
        x[kLaneAmps - 1] = mk<R>(cf * a.x - sf * right.y, cf * a.y + sf * right.x);
      }
      if (left_ok) {  // (previous lane's last a, this lane's first b): b <- i s a + c b
        const T b = x[0];
        x[0] = mk<R>(cf * b.x - sf * left.y, cf * b.y + sf * left.x);
      }
    }
  }
  {
    const T ph = mk<R>((R)blk.pc, sg * (R)blk.ps);
#pragma unroll
    for (int q = 0; q < kLaneAmps; ++q) x[q] = cmul(x[q], ph);
  }
  if (full_interior) {
    __syncwarp();
    if (lane > 0 && lane < 31) {
      const uint4* sx = reinterpret_cast<const uint4*>(x);
#pragma unroll
      for (int q = 0; q < CPL; ++q) {
        const int wc = lane * CPL + q;
        stage[wc ^ (lane & 7)] = sx[q];
      }
    }
    __syncwarp();
    uint4* dst = reinterpret_cast<uint4*>(row + g0);
    constexpr int chunks = kInterior / per;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      const int c = q * 32 + lane;
      if (c < chunks) {
        const int wc = c + CPL;
        dst[c] = stage[wc ^ ((wc / CPL) & 7)];
      }
    }
  } else if (lane > 0 && lane < 31) {
#pragma unroll
    for (int q = 0; q < kLaneAmps; ++q)
      if (lane0 + q < N) row[lane0 + q] = x[q];
  }
}

__global__ void k_interleave(const double* __restrict__ re, const double* __restrict__ im, int64_t n,
                             double2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_double2(re[i], im ? im[i] : 0.0);
}

template <class R>
hhl_status trotter_impl(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st) {
  using T = typename Cx<R>::T;
  const int r = p.trot_r[k];
  const int n_layers = 2 * r + 1;
  const double* b = &p.trot_blocks[(size_t)k * 24];
  const double tau = b[4], dh = b[5];
  const int64_t m_sub = p.R / 2;
  const int64_t segs = trotter_segments(p.N);
  const int64_t warps = m_sub * segs;
  const int64_t grid = (warps + kTrotThreads / 32 - 1) / (kTrotThreads / 32);
  if (grid > 0x7fffffffLL) return fail(HHL_ERR_UNSUPPORTED, "Trotter grid too large");
  T* side = (T*)p.d_scratch;  // sized by the planner for m_sub * segs * 32 amplitudes
  const int64_t edge_total = m_sub * segs * 32;
  int eg = (int)((edge_total + 255) / 256);
  if (eg > 152 * 16) eg = 152 * 16;
  for (int l0 = 0; l0 < n_layers; l0 += kHalo) {
    const int l1 = l0 + kHalo < n_layers ? l0 + kHalo : n_layers;
    double steps = 0.0;  // E-layer time in this pass
    for (int l = l0; l < l1; ++l)
      if ((l & 1) == 0) steps += (l == 0 || l == n_layers - 1) ? 0.5 : 1.0;
    TrotBlocks blk;
    blk.ch = b[0];
    blk.sh = b[1];
    blk.cf = b[2];
    blk.sf = b[3];
    blk.pc = cos(steps * tau * dh);
    blk.ps = sin(steps * tau * dh);
    HHL_PROF_BEGIN(st);
    k_trotter_edges<R><<<eg, 256, 0, st>>>((const T*)half, side, p.n_s, k, segs, m_sub);
    HHL_LAUNCH_CHECK("k_trotter_edges");
    HHL_PROF_BEGIN(st);
    k_trotter_pass<R><<<(unsigned)grid, kTrotThreads, 0, st>>>((T*)half, side, p.n_s, k, segs, m_sub, l0, l1,
                                                               n_layers, blk, adjoint ? 1 : 0);
    HHL_LAUNCH_CHECK("k_trotter_pass");
  }
  return HHL_OK;
}

}  // namespace

int64_t trotter_segments(int64_t N) { return (N + kInterior - 1) / kInterior; }

hhl_status launch_trotter(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st) {
  if (p.d_scratch == nullptr) return fail(HHL_ERR_INVALID_ARG, "Trotter plan without scratch");
  return p.prec == HHL_PREC_C64 ? trotter_impl<float>(p, half, k, adjoint, st)
                                : trotter_impl<double>(p, half, k, adjoint, st);
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
