// Controlled exp(i Ahat t_k) as a second-order Strang product of two-level gates, for a
// Toeplitz tridiagonal Ahat (the channel-flow operator of App. A.1 Eq. CDS).
//
// Ahat = E + O: E holds the 2x2 blocks [[d, o], [o, d]] on basis-state pairs (2i, 2i+1),
// O the couplings [[0, o], [o, 0]] on pairs (2i+1, 2i+2). One Strang step is
// S(tau) = E(tau/2) O(tau) E(tau/2) with E(s) = exp(i s E), and r steps merge into the
// layer list E(tau/2), O(tau), [E(tau), O(tau)] x (r-1), E(tau/2) (2r + 1 layers).
// Every layer acts inside one system-register row, so a pass applies several layers to a
// tile of a row held in shared memory (temporal blocking): the tile is loaded with a halo
// as wide as the number of layers of the pass, and only its interior is written back.
// Passes read one buffer and write another (state rows with clock bit k set <-> scratch
// rows), so that no tile reads a halo another tile has already overwritten.
#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kTile = 2048;        // interior amplitudes per CTA
constexpr int kMaxLayers = 16;     // layers per pass (halo width)
constexpr int kTrotThreads = 256;

__device__ __forceinline__ int64_t row_with_bit_t(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}

// blocks: E_half (a00, a01), E_full (a00, a01), O (a00, a01) as complex doubles.
struct TrotBlocks {
  double2 eh0, eh1, ef0, ef1, o0, o1;
};

template <class R>
__global__ void __launch_bounds__(kTrotThreads) k_trotter_pass(const typename Cx<R>::T* __restrict__ src,
                                                              typename Cx<R>::T* __restrict__ dst, int n_s, int k,
                                                              int src_is_state, int dst_is_state, int l0, int l1,
                                                              int n_layers_total, TrotBlocks blk, int adjoint) {
  using T = typename Cx<R>::T;
  __shared__ T buf[kTile + 2 * kMaxLayers];
  const int64_t N = 1LL << n_s;
  const int64_t i = blockIdx.y;  // subset row
  const int64_t g0 = (int64_t)blockIdx.x * kTile;
  const int H = kMaxLayers;
  const int64_t ws = (g0 - H) < 0 ? 0 : (g0 - H);
  const int64_t we = (g0 + kTile + H) > N ? N : (g0 + kTile + H);
  const int wn = (int)(we - ws);
  const int64_t srow = src_is_state ? row_with_bit_t(i, k) : i;
  const int64_t drow = dst_is_state ? row_with_bit_t(i, k) : i;
  const T* s = src + srow * N;
  T* d = dst + drow * N;
  for (int e = threadIdx.x; e < wn; e += blockDim.x) buf[e] = s[ws + e];
  __syncthreads();

  const R sg = adjoint ? (R)-1 : (R)1;
  const T eh0 = mk<R>((R)blk.eh0.x, sg * (R)blk.eh0.y), eh1 = mk<R>((R)blk.eh1.x, sg * (R)blk.eh1.y);
  const T ef0 = mk<R>((R)blk.ef0.x, sg * (R)blk.ef0.y), ef1 = mk<R>((R)blk.ef1.x, sg * (R)blk.ef1.y);
  const T o0 = mk<R>((R)blk.o0.x, sg * (R)blk.o0.y), o1 = mk<R>((R)blk.o1.x, sg * (R)blk.o1.y);
  for (int l = l0; l < l1; ++l) {
    const bool odd = (l & 1) != 0;
    T a00, a01;
    if (odd) {
      a00 = o0;
      a01 = o1;
    } else if (l == 0 || l == n_layers_total - 1) {
      a00 = eh0;
      a01 = eh1;
    } else {
      a00 = ef0;
      a01 = ef1;
    }
    // E: local pairs (2p, 2p+1) (ws is even); O: global pairs (2j+1, 2j+2) with 2j+2 < N.
    const int first = odd ? 1 : 0;
    const int npairs = (wn - first) / 2;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
      const int a = first + 2 * p, b = a + 1;
      if (odd && ws + b >= N) continue;
      const T xa = buf[a], xb = buf[b];
      buf[a] = cadd(cmul(a00, xa), cmul(a01, xb));
      buf[b] = cadd(cmul(a01, xa), cmul(a00, xb));
    }
    __syncthreads();
  }
  const int off = (int)(g0 - ws);
  const int cnt = (int)((g0 + kTile > N ? N : g0 + kTile) - g0);
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) d[g0 + e] = buf[off + e];
}

template <class R>
__global__ void k_rows_copy_back(typename Cx<R>::T* __restrict__ state, const typename Cx<R>::T* __restrict__ scratch,
                                 int n_s, int k, int64_t m_sub) {
  const int64_t N = 1LL << n_s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m_sub * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e >> n_s, m = e & (N - 1);
    state[row_with_bit_t(i, k) * N + m] = scratch[e];
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
  TrotBlocks blk;
  blk.eh0 = make_double2(b[0], b[1]);
  blk.eh1 = make_double2(b[2], b[3]);
  blk.ef0 = make_double2(b[8], b[9]);
  blk.ef1 = make_double2(b[10], b[11]);
  blk.o0 = make_double2(b[16], b[17]);
  blk.o1 = make_double2(b[18], b[19]);
  const int64_t m_sub = p.R / 2;
  if (m_sub > 65535) return fail(HHL_ERR_UNSUPPORTED, "too many clock rows for the Trotter grid");
  dim3 grid((unsigned)((p.N + kTile - 1) / kTile), (unsigned)m_sub);
  T* state = (T*)half;
  T* scratch = (T*)p.d_scratch;
  bool in_state = true;
  for (int l0 = 0; l0 < n_layers; l0 += kMaxLayers) {
    const int l1 = l0 + kMaxLayers < n_layers ? l0 + kMaxLayers : n_layers;
    const T* src = in_state ? state : scratch;
    T* dst = in_state ? scratch : state;
    HHL_PROF_BEGIN(st);
    k_trotter_pass<R><<<grid, kTrotThreads, 0, st>>>(src, dst, p.n_s, k, in_state ? 1 : 0, in_state ? 0 : 1, l0, l1,
                                                     n_layers, blk, adjoint ? 1 : 0);
    HHL_LAUNCH_CHECK("k_trotter_pass");
    in_state = !in_state;
  }
  if (!in_state) {
    const int64_t total = m_sub * p.N;
    int g = (int)((total + 255) / 256);
    if (g > 152 * 32) g = 152 * 32;
    HHL_PROF_BEGIN(st);
    k_rows_copy_back<R><<<g, 256, 0, st>>>(state, scratch, p.n_s, k, m_sub);
    HHL_LAUNCH_CHECK("k_rows_copy_back");
  }
  return HHL_OK;
}

}  // namespace

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
