// CUDA kernels of the HHL state-vector path (sm_103a): state preparation, the SIMT
// controlled-U GEMM, postselection / dissipation reductions, and the plan-time exponential
// exp(i Ahat t) from an eigendecomposition. (Register blocks over the clock are in
// hhl_fft.cu, the tensor-core GEMM in hhl_gemm_tc.cu, the Trotter passes in hhl_trotter.cu.)
//
// State layout: S[anc][clk][sys] row-major, complex64 or complex128 interleaved; the
// "active half" of a stage is S[0] or S[1], a row-major (2^n_c x N) matrix whose row c is
// the system register for clock value c.
#include <math.h>

#include <type_traits>

#include <stdlib.h>

#include <cooperative_groups.h>

#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV per-thread values over the block and add them to dst[0..NV) with one atomic each.
template <int NV>
__device__ void block_sum_atomic(const double (&v)[NV], double* dst) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = warp_sum(v[i]);
    if (lane == 0) sh[i][wid] = s;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = lane < nw ? sh[i][lane] : 0.0;
      s = warp_sum(s);
      if (lane == 0) atomicAdd(dst + i, s);
    }
  }
}

int grid_for(int64_t n, int threads, int cap = 152 * 16) {
  int64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Subset index i -> row c of the 2^n_c rows whose bit k is 1.
__device__ __forceinline__ int64_t row_with_bit(int64_t i, int k) {
  return ((i >> k) << (k + 1)) | (1LL << k) | (i & ((1LL << k) - 1));
}

// ------------------------------------------------------------------------------ prep

__global__ void k_bnorm(const double2* __restrict__ b, int64_t n, double* acc) {
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 z = b[i];
    s[0] += z.x * z.x + z.y * z.y;
  }
  block_sum_atomic<1>(s, acc);
}

// bs = b / (|b| 2^(n_c/2)) in the amplitude precision (one row of the anc = 0 half).
template <class R>
__global__ void k_prep_scale(const double2* __restrict__ b, const double* __restrict__ acc,
                             typename Cx<R>::T* __restrict__ bs, int64_t N, int n_c) {
  const double nb2 = acc[0];
  const double scale = nb2 > 0.0 ? 1.0 / sqrt(nb2 * (double)(1LL << n_c)) : 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 z = b[i];
    bs[i] = mk<R>((R)(z.x * scale), (R)(z.y * scale));
  }
}

// Every clock row of the anc = 0 half gets bs, the anc = 1 half is zeroed: 16-byte stores.
__global__ void k_prep_fill(const uint4* __restrict__ bs, uint4* __restrict__ st, int64_t row_units,
                            int64_t half_units) {
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < 2 * half_units;
       u += (int64_t)gridDim.x * blockDim.x)
    st[u] = u < half_units ? bs[u & (row_units - 1)] : zero;
}

// ------------------------------------------------------------------------------ SIMT GEMM
// out[i][n] = sum_m S[row(i)][m] * B[m][n] for the M_sub = 2^(n_c-1) rows with clock bit k
// set; B = U_k^T (forward) or conj(U_k) (adjoint) so that out row = U row.
template <class R, int BM, int BN, int BK>
__global__ void __launch_bounds__(256) k_ctrl_gemm_simt(const typename Cx<R>::T* __restrict__ S,
                                                        typename Cx<R>::T* __restrict__ out,
                                                        const typename Cx<R>::T* __restrict__ B,
                                                        int n_s, RowMap rows, int64_t m_sub) {
  using T = typename Cx<R>::T;
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int64_t N = 1LL << n_s;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t i0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  R accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int c = 0; c < TN; ++c) { accr[a][c] = 0; acci[a][c] = 0; }

  for (int64_t m0 = 0; m0 < N; m0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int r = e / BK, kk = e % BK;
      const int64_t i = i0 + r, m = m0 + kk;
      T v = mk<R>((R)0, (R)0);
      if (i < m_sub && m < N) v = S[rowmap_in(rows, i) * N + m];
      As[kk][r] = v;
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int kk = e / BN, c = e % BN;
      const int64_t m = m0 + kk, n = n0 + c;
      T v = mk<R>((R)0, (R)0);
      if (m < N && n < N) v = B[m * N + n];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], bb[TN];
#pragma unroll
      for (int x = 0; x < TM; ++x) a[x] = As[kk][ty + 16 * x];
#pragma unroll
      for (int y = 0; y < TN; ++y) bb[y] = Bs[kk][tx + 16 * y];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) {
          accr[x][y] = fma(a[x].x, bb[y].x, accr[x][y]);
          accr[x][y] = fma(-a[x].y, bb[y].y, accr[x][y]);
          acci[x][y] = fma(a[x].x, bb[y].y, acci[x][y]);
          acci[x][y] = fma(a[x].y, bb[y].x, acci[x][y]);
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
      if (n < N) out[i * N + n] = mk<R>(accr[x][y], acci[x][y]);
    }
  }
}

// S[row(i)][:] = out[i][:] (the rows with clock bit k set, or a tree's mapped rows, where the
// reduction adds out[i][:] to the row and its last step scales the sum).
template <class R>
__global__ void k_rows_scatter(typename Cx<R>::T* __restrict__ S, const typename Cx<R>::T* __restrict__ out,
                               int n_s, RowMap rows, int64_t m_sub) {
  const int64_t N = 1LL << n_s;
  const int64_t total = m_sub * N;
  const R sc = (R)rows.scale;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e >> n_s, m = e & (N - 1);
    typename Cx<R>::T* d = S + rowmap_out(rows, i) * N + m;
    if (rows.accumulate) {
      const typename Cx<R>::T v = cadd(*d, out[e]);
      *d = rows.scale != 1.0 ? cscale(v, sc) : v;
    } else {
      *d = out[e];
    }
  }
}

// ------------------------------------------------------------------------------ readout

// FP64 sums of |S0|^2, |S1|^2 and |v|^2 (v = first row of S1), read in 16-byte units; the
// squares of one unit are added in the amplitude precision, the running sums are FP64.
// s - c <- s - c + p (compensated summation; c holds the negated lost low-order part)
template <class R>
__device__ __forceinline__ void kahan_add(R& s, R& c, R p) {
  const R y = p - c;
  const R t = s + y;
  c = (t - s) - y;
  s = t;
}

// Complex128 form on the FP32 pipe: the FP64 amplitudes split into double-float with integer
// operations, |z|^2 and the running sums in double-float (about 48 significant bits per
// partial; the block and grid totals in FP64).
__global__ void k_measure_sums_df(const double2* __restrict__ S, int64_t half, int64_t N, double* acc) {
  const int64_t units = 2 * half;
  constexpr int U = 4;  // loads in flight per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  df s[3] = {df(0), df(0), df(0)};
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < units; i0 += U * stride) {
    double2 z[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i0 + k * stride < units) z[k] = S[i0 + k * stride];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t i = i0 + k * stride;
      if (i >= units) break;
      const df re = df_from_double(z[k].x), im = df_from_double(z[k].y);
      const df p = df_add(df_mul(re, re), df_mul(im, im));
      if (i < half) {
        s[0] = df_add(s[0], p);
      } else {
        s[1] = df_add(s[1], p);
        if (i - half < N) s[2] = df_add(s[2], p);
      }
    }
  }
  double a[3] = {df_to_double(s[0]), df_to_double(s[1]), df_to_double(s[2])};
  block_sum_atomic<3>(a, acc);
}

template <class R>
__global__ void k_measure_sums(const typename Cx<R>::T* __restrict__ S, int64_t half, int64_t N, double* acc) {
  constexpr int per = 16 / sizeof(typename Cx<R>::T);  // amplitudes per 16-byte unit
  using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  const V* u = reinterpret_cast<const V*>(S);
  const int64_t units = 2 * half / per, half_u = half / per, v_u = N / per;
  constexpr int U = 4;  // loads in flight per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // Each thread sums its squares in the amplitude precision with compensated (Kahan)
  // summation, so the partial carries about one rounding error whatever its length, and
  // converts it to FP64 once; the block and grid totals are FP64. (GB300's FP64 pipe is far
  // narrower than its FP32 pipe: an FP64 conversion and add per amplitude would bound the pass.)
  R s[3] = {(R)0, (R)0, (R)0}, c[3] = {(R)0, (R)0, (R)0};
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < units; i0 += U * stride) {
    V z[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (i0 + k * stride < units) z[k] = u[i0 + k * stride];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t i = i0 + k * stride;
      if (i >= units) break;
      R p;
      if constexpr (sizeof(R) == 4) {
        p = fmaf(z[k].x, z[k].x, fmaf(z[k].y, z[k].y, fmaf(z[k].z, z[k].z, z[k].w * z[k].w)));
      } else {
        p = z[k].x * z[k].x + z[k].y * z[k].y;
      }
      if (i < half_u) {
        kahan_add(s[0], c[0], p);
      } else {
        kahan_add(s[1], c[1], p);
        if (i - half_u < v_u) kahan_add(s[2], c[2], p);
      }
    }
  }
  double a[3] = {(double)s[0] - (double)c[0], (double)s[1] - (double)c[1], (double)s[2] - (double)c[2]};
  block_sum_atomic<3>(a, acc);
}

// |v|^2 of one row of N amplitudes (the postselected row), FP64.
template <class R>
__global__ void k_row_norm(const typename Cx<R>::T* __restrict__ v, int64_t N, double* acc) {
  double s[1] = {0.0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const double re = (double)v[j].x, im = (double)v[j].y;
    s[0] += re * re + im * im;
  }
  block_sum_atomic<1>(s, acc);
}

// out = [p_success, p_anc1, norm, |b|, xhat (2N doubles)]
template <class R>
__global__ void k_measure_finish(const typename Cx<R>::T* __restrict__ S, int64_t half, int64_t N,
                                 const double* __restrict__ scal, double* __restrict__ out) {
  const double ps = scal[3];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i == 0) {
    out[0] = ps;
    out[1] = scal[2];
    out[2] = scal[1] + scal[2];
    out[3] = sqrt(scal[0]);
  }
  const double inv = ps > 0.0 ? 1.0 / sqrt(ps) : 0.0;
  for (int64_t j = i; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const typename Cx<R>::T z = S[half + j];
    out[4 + 2 * j] = (double)z.x * inv;
    out[5 + 2 * j] = (double)z.y * inv;
  }
}

// QSP-1 (App. C): the system register prepared from |0> by a binary tree of uniformly
// controlled RY rotations. tree[(1 << l) + i] holds the probability mass of node i of level l
// (level n_s: the leaves |b_i|^2); level l rotates qubit n_s-1-l, conditioned on the l more
// significant qubits holding node i, by R_y(theta) in the paper's convention (our RY(2 theta)),
// theta = arccos sqrt(p(zero child) / p(node)).
__global__ void k_qsp_leaves(const double* __restrict__ b, int64_t N, double* __restrict__ tree) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    tree[N + i] = b[i] * b[i];
}

__global__ void k_qsp_sum(int l, double* __restrict__ tree) {
  const int64_t n = 1LL << l;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    tree[n + i] = tree[2 * n + 2 * i] + tree[2 * n + 2 * i + 1];
}

__global__ void k_qsp_level(int l, int n_s, const double* __restrict__ tree, double2* __restrict__ psi) {
  const int t = n_s - 1 - l;
  const int64_t pairs = 1LL << (n_s - 1);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < pairs; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = ((q >> t) << (t + 1)) | (q & ((1LL << t) - 1));
    const int64_t i1 = i0 | (1LL << t);
    const int64_t node = i0 >> (t + 1);
    const double parent = tree[(1LL << l) + node];
    const double child0 = tree[(2LL << l) + 2 * node];
    const double th = parent > 0.0 ? acos(sqrt(fmin(1.0, child0 / parent))) : 0.0;
    const double c = cos(th), s = sin(th);
    const double2 a0 = psi[i0], a1 = psi[i1];
    psi[i0] = make_double2(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
    psi[i1] = make_double2(s * a0.x + c * a1.x, s * a0.y + c * a1.y);
  }
}

// QSP-2 (Sec. III, App. C): the same tree, but only the nodes on a path to one of the
// nonzero entries (idx strictly increasing, values val) get a rotation, so the work is
// O(count n_s) instead of O(N). Level l: the first entry of each run of entries sharing the
// l top bits (the node's prefix) sums the node's and its zero child's probability over the
// run and rotates the node's amplitude, which still sits at prefix << (n_s - l) (the lower
// qubits are |0>), into the pair (zero child, one child). Entries outside [0, N) are ignored
// (they match no prefix). Negative values get their sign at the end (a Z on the leaf's path).
// One block; acc = |val|^2 for the dissipation read-out.
__global__ void __launch_bounds__(1024) k_qsp2_tree(const int64_t* __restrict__ idx, const double* __restrict__ val,
                                                    int64_t count, int n_s, double2* __restrict__ psi,
                                                    double* __restrict__ acc) {
  const int64_t N = 1LL << n_s;
  for (int l = 0; l < n_s; ++l) {
    const int shift = n_s - l;
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) {
      const int64_t i = idx[k];
      if (i < 0 || i >= N) continue;
      const int64_t pre = i >> shift;
      if (k > 0 && (idx[k - 1] >> shift) == pre) continue;  // not the first entry of its node
      double p_node = 0.0, p_zero = 0.0;
      for (int64_t j = k; j < count && (idx[j] >> shift) == pre; ++j) {
        const double w = val[j] * val[j];
        p_node += w;
        if (((idx[j] >> (shift - 1)) & 1) == 0) p_zero += w;
      }
      const double th = p_node > 0.0 ? acos(sqrt(fmin(1.0, p_zero / p_node))) : 0.0;
      const double c = cos(th), s = sin(th);
      const int64_t i0 = pre << shift, i1 = i0 | (1LL << (shift - 1));
      const double2 a0 = psi[i0], a1 = psi[i1];
      psi[i0] = make_double2(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
      psi[i1] = make_double2(s * a0.x + c * a1.x, s * a0.y + c * a1.y);
    }
    __syncthreads();  // the next level rotates the children this level wrote
  }
  __shared__ double part[1024];
  double w = 0.0;
  for (int64_t k = threadIdx.x; k < count; k += blockDim.x) {
    const int64_t i = idx[k];
    if (i < 0 || i >= N) continue;
    w += val[k] * val[k];
    if (val[k] < 0.0) psi[i] = make_double2(-psi[i].x, -psi[i].y);
  }
  part[threadIdx.x] = w;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) acc[0] = part[0];
}

// psi = |0>, then (after the tree) bs = psi / 2^(n_c/2) in the amplitude precision.
__global__ void k_qsp_init(double2* __restrict__ psi, int64_t N) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    psi[i] = make_double2(i == 0 ? 1.0 : 0.0, 0.0);
}

template <class R>
__global__ void k_qsp_scale(const double2* __restrict__ psi, int64_t N, int n_c, typename Cx<R>::T* __restrict__ bs) {
  const double sc = 1.0 / sqrt((double)(1LL << n_c));
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    bs[i] = mk<R>((R)(psi[i].x * sc), (R)(psi[i].y * sc));
}

// Shots (inverse-transform sampling of the postselected outcome distribution): running sum
// cdf_j = sum_{i <= j} |v_i|^2 in FP64 by one block (contiguous chunks per thread, then a scan
// of the chunk totals), then per shot the bin j with cdf_{j-1} <= u total < cdf_j.
template <class R>
__global__ void __launch_bounds__(1024) k_sample_cdf(const typename Cx<R>::T* __restrict__ v, int64_t N,
                                                     double* __restrict__ cdf) {
  __shared__ double part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (N + blockDim.x - 1) / blockDim.x;
  const int64_t a = t * chunk, b = a + chunk < N ? a + chunk : N;
  double sum = 0.0;
  for (int64_t j = a; j < b; ++j) sum += (double)v[j].x * (double)v[j].x + (double)v[j].y * (double)v[j].y;
  part[t] = sum;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive Hillis-Steele scan
    const double add = t >= off ? part[t - off] : 0.0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  double run = t > 0 ? part[t - 1] : 0.0;
  for (int64_t j = a; j < b; ++j) {
    run += (double)v[j].x * (double)v[j].x + (double)v[j].y * (double)v[j].y;
    cdf[j] = run;
  }
}

__global__ void k_sample_bins(const double* __restrict__ cdf, int64_t N, const double* __restrict__ u, int64_t shots,
                              unsigned long long* __restrict__ counts) {
  const double total = cdf[N - 1];
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < shots; s += (int64_t)gridDim.x * blockDim.x) {
    const double x = u[s] * total;
    int64_t lo = 0, hi = N - 1;  // smallest j with x < cdf[j] (the last bin if none)
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (x < cdf[mid]) hi = mid;
      else lo = mid + 1;
    }
    atomicAdd(counts + lo, 1ULL);
  }
}

// Dissipation: sum over the N+1 cells of (u_{i+1} - u_i)^2 with walls at both ends.
template <class R>
__global__ void k_diss_sum(const typename Cx<R>::T* __restrict__ S, int64_t half, int64_t N,
                           const double* __restrict__ scal, double inv_c_lam, double wlo, double whi,
                           double* acc, double* __restrict__ u_out) {
  const double scale = sqrt(scal[0]) * inv_c_lam;
  double s[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= N; i += (int64_t)gridDim.x * blockDim.x) {
    const double left = (i == 0) ? wlo : scale * (double)S[half + i - 1].x;
    const double right = (i == N) ? whi : scale * (double)S[half + i].x;
    const double d = right - left;
    s[0] += d * d;
    if (u_out != nullptr && i < N) u_out[i] = right;
  }
  block_sum_atomic<1>(s, acc);
}

__global__ void k_diss_finish(const double* __restrict__ acc, double nu_over_h, double* eps) {
  if (threadIdx.x == 0 && blockIdx.x == 0) eps[0] = nu_over_h * acc[0];
}

// ------------------------------------------------------------------------------ QPP (LCU)
// Post-processing of the dissipation rate by a linear combination of unitaries (App. D):
// the register [ancilla | data of 2N points] holds w = (u_1 .. u_N, u_{N+1} (wall), 0 ..., u_0
// (wall)) normalised in its ancilla-0 half; H on the ancilla, Z on it (the coefficient -1),
// the cyclic increment P of the data controlled by it, H again; P(ancilla = 0) =
// ||(w - P w) / 2||^2 / |w|^2 holds every forward difference of u. One kernel per gate, FP64.
template <class R>
__global__ void k_qpp_load(const typename Cx<R>::T* __restrict__ S, int64_t half, int64_t N,
                           const double* __restrict__ scal, double inv_c_lam, double wlo, double whi,
                           double2* __restrict__ reg0, double2* __restrict__ reg1, double* acc) {
  const double scale = sqrt(scal[0]) * inv_c_lam;
  double s[1] = {0.0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < 2 * N; j += (int64_t)gridDim.x * blockDim.x) {
    const double w = j < N ? scale * (double)S[half + j].x : (j == N ? whi : (j == 2 * N - 1 ? wlo : 0.0));
    reg0[j] = make_double2(w, 0.0);
    reg1[j] = make_double2(0.0, 0.0);
    s[0] += w * w;
  }
  block_sum_atomic<1>(s, acc);
}

__global__ void k_qpp_normalize(double2* __restrict__ reg0, int64_t L, const double* __restrict__ acc) {
  const double inv = acc[0] > 0.0 ? 1.0 / sqrt(acc[0]) : 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x)
    reg0[j] = make_double2(reg0[j].x * inv, reg0[j].y * inv);
}

// H on the ancilla (the most significant qubit): (a, b) -> ((a + b), (a - b)) / sqrt 2.
__global__ void k_qpp_h(double2* __restrict__ reg0, double2* __restrict__ reg1, int64_t L) {
  const double r = 0.70710678118654752;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = reg0[j], b = reg1[j];
    reg0[j] = make_double2(r * (a.x + b.x), r * (a.y + b.y));
    reg1[j] = make_double2(r * (a.x - b.x), r * (a.y - b.y));
  }
}

// Z on the ancilla, then the cyclic increment of the data controlled by it: out[(j+1) mod L] =
// -reg1[j] (the ancilla-1 half only; out is a separate buffer, the halves are swapped after).
__global__ void k_qpp_z_ctrl_inc(const double2* __restrict__ reg1, double2* __restrict__ out, int64_t L) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = reg1[j];
    out[j + 1 == L ? 0 : j + 1] = make_double2(-a.x, -a.y);
  }
}

__global__ void k_qpp_p0(const double2* __restrict__ reg0, int64_t L, double* acc) {
  double s[1] = {0.0};
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < L; j += (int64_t)gridDim.x * blockDim.x)
    s[0] += reg0[j].x * reg0[j].x + reg0[j].y * reg0[j].y;
  block_sum_atomic<1>(s, acc);
}

// ------------------------------------------------------------------------------ plan kernels
// U[n][m] = wgt sum_j e^{i phi_j} (Vr + i Vi)[n][j] conj((Vr + i Vi)[m][j]), FP64.
__global__ void __launch_bounds__(256) k_expm_eigen(int N, int J, const double* __restrict__ vr,
                                                    const double* __restrict__ vi, const double* __restrict__ cph,
                                                    const double* __restrict__ sph, double wgt, double2* __restrict__ U) {
  __shared__ double ar[16][17], ai[16][17], br[16][17], bi[16][17], pc[16], ps[16];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n = blockIdx.y * 16 + ty, m = blockIdx.x * 16 + tx;
  double accr = 0.0, acci = 0.0;
  for (int j0 = 0; j0 < J; j0 += 16) {
    {
      const int rn = blockIdx.y * 16 + ty, rm = blockIdx.x * 16 + ty, jj = j0 + tx;
      ar[ty][tx] = (rn < N && jj < J) ? vr[(size_t)rn * J + jj] : 0.0;
      ai[ty][tx] = (vi != nullptr && rn < N && jj < J) ? vi[(size_t)rn * J + jj] : 0.0;
      br[ty][tx] = (rm < N && jj < J) ? vr[(size_t)rm * J + jj] : 0.0;
      bi[ty][tx] = (vi != nullptr && rm < N && jj < J) ? vi[(size_t)rm * J + jj] : 0.0;
      if (ty == 0) {
        pc[tx] = jj < J ? cph[jj] : 0.0;
        ps[tx] = jj < J ? sph[jj] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      // p = (ar + i ai)(br - i bi)
      const double pr = ar[ty][jj] * br[tx][jj] + ai[ty][jj] * bi[tx][jj];
      const double pi = ai[ty][jj] * br[tx][jj] - ar[ty][jj] * bi[tx][jj];
      accr += pc[jj] * pr - ps[jj] * pi;
      acci += pc[jj] * pi + ps[jj] * pr;
    }
    __syncthreads();
  }
  if (n < N && m < N) U[(size_t)n * N + m] = make_double2(wgt * accr, wgt * acci);
}

// B_fwd[m][n] = U[n][m], B_adj[m][n] = conj(U[m][n]) in the amplitude precision.
template <class R>
__global__ void k_store_operands(const double2* __restrict__ U, int64_t N, typename Cx<R>::T* __restrict__ bf,
                                 typename Cx<R>::T* __restrict__ ba) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / N, n = e - m * N;
    const double2 ut = U[n * N + m];
    const double2 u = U[e];
    bf[e] = mk<R>((R)ut.x, (R)ut.y);
    ba[e] = mk<R>((R)u.x, (R)(-u.y));
  }
}

}  // namespace

// ================================================================================ launchers

hhl_status launch_bnorm(const double* b, int64_t N, double* acc, cudaStream_t st) {
  HHL_PROF_BEGIN(st);
  k_bnorm<<<grid_for(N, kThreads, 152), kThreads, 0, st>>>((const double2*)b, N, acc);
  HHL_LAUNCH_CHECK("k_bnorm");
  return HHL_OK;
}

hhl_status launch_prep_fill(const Plan& p, const double* b, void* state, cudaStream_t st) {
  const int gs = grid_for(p.N, kThreads, 152);
  if (p.prec == HHL_PREC_C64) {
    HHL_PROF_BEGIN(st);
    k_prep_scale<float><<<gs, kThreads, 0, st>>>((const double2*)b, p.d_scal, (float2*)p.d_bs, p.N, p.n_c);
  } else {
    HHL_PROF_BEGIN(st);
    k_prep_scale<double><<<gs, kThreads, 0, st>>>((const double2*)b, p.d_scal, (double2*)p.d_bs, p.N, p.n_c);
  }
  HHL_LAUNCH_CHECK("k_prep_scale");
  const int64_t row_units = p.N * (int64_t)p.amp_bytes() / 16;
  const int64_t half_units = p.R * row_units;
  const int g = grid_for(2 * half_units, kThreads, 152 * 16);
  HHL_PROF_BEGIN(st);
  k_prep_fill<<<g, kThreads, 0, st>>>((const uint4*)p.d_bs, (uint4*)state, row_units, half_units);
  HHL_LAUNCH_CHECK("k_prep_fill");
  return HHL_OK;
}

hhl_status launch_ctrl_u_dense(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st) {
  const size_t mat = (size_t)p.N * p.N;
  const size_t off = (size_t)k * mat * p.amp_bytes();
  const void* B = (const char*)(adjoint ? p.d_badj : p.d_bfwd) + off;
  return launch_ctrl_u_simt(p, half, k, B, st);
}

hhl_status launch_ctrl_u_tree(const Plan& p, void* half, int k, bool reduce, cudaStream_t st) {
  RowMap rows;
  const int64_t m = 1LL << k;
  if (reduce) {
    rows.in_off = m;
    rows.out_off = 0;
    rows.accumulate = 1;
    if (k == 0) rows.scale = 1.0 / sqrt((double)p.R);
  } else {
    rows.in_off = 0;
    rows.out_off = m;
  }
  if (p.d_gdf != nullptr && m < toeplitz_rows_limit())  // few rows: U_k generated on the fly from its g table
    return launch_toeplitz_rows((float2*)half, p.n_s, p.d_gdf + (size_t)k * (2 * p.N + 2), reduce ? 1 : 0, rows, m, st);
  if (p.gemm_impl == HHL_GEMM_TCGEN05 && m >= 128 && rows.scale == 1.0)
    return launch_ctrl_u_tc_map(p, half, rows, m, k, reduce, st);
  if (p.d_gdf != nullptr && m < 128)
    return launch_toeplitz_rows((float2*)half, p.n_s, p.d_gdf + (size_t)k * (2 * p.N + 2), reduce ? 1 : 0, rows, m, st);
  if (p.d_bfwd == nullptr) {  // a tcgen05 plan keeps no CUDA-core operands
    return fail(HHL_ERR_UNSUPPORTED, "tree step below 128 rows on a tcgen05-only plan");
  }
  const size_t mat = (size_t)p.N * p.N;
  const void* B = (const char*)(reduce ? p.d_badj : p.d_bfwd) + (size_t)k * mat * p.amp_bytes();
  return launch_ctrl_u_simt_map(p, half, rows, m, B, st);
}

hhl_status launch_ctrl_u_simt(const Plan& p, void* half, int k, const void* B, cudaStream_t st) {
  return launch_ctrl_u_simt_map(p, half, circuit_rows(k), p.R / 2, B, st);
}

hhl_status launch_ctrl_u_simt_map(const Plan& p, void* half, const RowMap& k, int64_t m_sub, const void* B,
                                  cudaStream_t st) {
  const int64_t N = p.N;
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((m_sub + 63) / 64));
  const int sg = grid_for(m_sub * N, kThreads, 152 * 32);
  if (p.prec == HHL_PREC_C64) {
    HHL_PROF_BEGIN(st);
    k_ctrl_gemm_simt<float, 64, 64, 16><<<grid, 256, 0, st>>>((const float2*)half, (float2*)p.d_scratch,
                                                              (const float2*)B, p.n_s, k, m_sub);
    HHL_LAUNCH_CHECK("k_ctrl_gemm_simt<f32>");
    HHL_PROF_BEGIN(st);
    k_rows_scatter<float><<<sg, kThreads, 0, st>>>((float2*)half, (const float2*)p.d_scratch, p.n_s, k, m_sub);
  } else {
    HHL_PROF_BEGIN(st);
    k_ctrl_gemm_simt<double, 64, 64, 8><<<grid, 256, 0, st>>>((const double2*)half, (double2*)p.d_scratch,
                                                              (const double2*)B, p.n_s, k, m_sub);
    HHL_LAUNCH_CHECK("k_ctrl_gemm_simt<f64>");
    HHL_PROF_BEGIN(st);
    k_rows_scatter<double><<<sg, kThreads, 0, st>>>((double2*)half, (const double2*)p.d_scratch, p.n_s, k, m_sub);
  }
  HHL_LAUNCH_CHECK("k_rows_scatter");
  return HHL_OK;
}

hhl_status launch_measure_sums(const Plan& p, const void* state, cudaStream_t st) {
  const int64_t half = p.R * p.N;
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal + 1, 0, 3 * sizeof(double), st));
  const int g = grid_for(2 * half, kThreads, 152 * 8);
  const char* env = getenv("HHL_FP64_PIPE");
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64)
    k_measure_sums<float><<<g, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal + 1);
  else if (env != nullptr && atoi(env) != 0)
    k_measure_sums<double><<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal + 1);
  else
    k_measure_sums_df<<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal + 1);
  HHL_LAUNCH_CHECK("k_measure_sums");
  return HHL_OK;
}

hhl_status launch_measure_row(const Plan& p, const void* state, double* out, cudaStream_t st) {
  const int64_t half = p.R * p.N;
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal + 3, 0, sizeof(double), st));
  const int gf = grid_for(p.N, kThreads, 152 * 4);
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64)
    k_row_norm<float><<<gf, kThreads, 0, st>>>((const float2*)state + half, p.N, p.d_scal + 3);
  else
    k_row_norm<double><<<gf, kThreads, 0, st>>>((const double2*)state + half, p.N, p.d_scal + 3);
  HHL_LAUNCH_CHECK("k_row_norm");
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64)
    k_measure_finish<float><<<gf, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal, out);
  else
    k_measure_finish<double><<<gf, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal, out);
  HHL_LAUNCH_CHECK("k_measure_finish");
  return HHL_OK;
}

hhl_status launch_prep_row(const Plan& p, const double* b, void* state, cudaStream_t st) {
  const int gs = grid_for(p.N, kThreads, 152);
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64)
    k_prep_scale<float><<<gs, kThreads, 0, st>>>((const double2*)b, p.d_scal, (float2*)p.d_bs, p.N, p.n_c);
  else
    k_prep_scale<double><<<gs, kThreads, 0, st>>>((const double2*)b, p.d_scal, (double2*)p.d_bs, p.N, p.n_c);
  HHL_LAUNCH_CHECK("k_prep_scale");
  HHL_CUDA_TRY(cudaMemcpyAsync(state, p.d_bs, (size_t)p.N * p.amp_bytes(), cudaMemcpyDeviceToDevice, st));
  return HHL_OK;
}

hhl_status launch_measure(const Plan& p, const void* state, double* out, cudaStream_t st) {
  const int64_t half = p.R * p.N;
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal + 1, 0, 3 * sizeof(double), st));
  const int g = grid_for(2 * half, kThreads, 152 * 8);
  const int gf = grid_for(p.N, kThreads, 152 * 4);
  if (p.prec == HHL_PREC_C64) {
    HHL_PROF_BEGIN(st);
    k_measure_sums<float><<<g, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal + 1);
    HHL_LAUNCH_CHECK("k_measure_sums");
    HHL_PROF_BEGIN(st);
    k_measure_finish<float><<<gf, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal, out);
  } else {
    const char* env = getenv("HHL_FP64_PIPE");
    HHL_PROF_BEGIN(st);
    if (env != nullptr && atoi(env) != 0)
      k_measure_sums<double><<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal + 1);
    else
      k_measure_sums_df<<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal + 1);
    HHL_LAUNCH_CHECK("k_measure_sums");
    HHL_PROF_BEGIN(st);
    k_measure_finish<double><<<gf, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal, out);
  }
  HHL_LAUNCH_CHECK("k_measure_finish");
  return HHL_OK;
}

hhl_status launch_prep_qsp1(const Plan& p, const double* b, double* tree, double2* psi, void* state,
                            cudaStream_t st) {
  const int g = grid_for(p.N, kThreads, 152 * 4);
  HHL_PROF_BEGIN(st);
  k_qsp_leaves<<<g, kThreads, 0, st>>>(b, p.N, tree);
  HHL_LAUNCH_CHECK("k_qsp_leaves");
  for (int l = p.n_s - 1; l >= 0; --l) {
    HHL_PROF_BEGIN(st);
    k_qsp_sum<<<grid_for(1LL << l, kThreads, 152 * 4), kThreads, 0, st>>>(l, tree);
    HHL_LAUNCH_CHECK("k_qsp_sum");
  }
  // the root holds |b|^2: recorded for the read-outs, as hhl_prepare_rhs does
  HHL_CUDA_TRY(cudaMemcpyAsync(p.d_scal, tree + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
  HHL_PROF_BEGIN(st);
  k_qsp_init<<<g, kThreads, 0, st>>>(psi, p.N);
  HHL_LAUNCH_CHECK("k_qsp_init");
  for (int l = 0; l < p.n_s; ++l) {
    HHL_PROF_BEGIN(st);
    k_qsp_level<<<grid_for(p.N / 2, kThreads, 152 * 4), kThreads, 0, st>>>(l, p.n_s, tree, psi);
    HHL_LAUNCH_CHECK("k_qsp_level");
  }
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64) k_qsp_scale<float><<<g, kThreads, 0, st>>>(psi, p.N, p.n_c, (float2*)p.d_bs);
  else k_qsp_scale<double><<<g, kThreads, 0, st>>>(psi, p.N, p.n_c, (double2*)p.d_bs);
  HHL_LAUNCH_CHECK("k_qsp_scale");
  // H on every clock qubit of |0>: every clock row holds the prepared system state
  const int64_t row_units = p.N * (int64_t)p.amp_bytes() / 16;
  const int64_t half_units = p.R * row_units;
  HHL_PROF_BEGIN(st);
  k_prep_fill<<<grid_for(2 * half_units, kThreads, 152 * 16), kThreads, 0, st>>>((const uint4*)p.d_bs, (uint4*)state,
                                                                                row_units, half_units);
  HHL_LAUNCH_CHECK("k_prep_fill");
  return HHL_OK;
}

hhl_status launch_qpp_dissipation(const Plan& p, const void* state, double2* reg, double* acc, cudaStream_t st) {
  const int64_t half = p.R * p.N, L = 2 * p.N;
  double2 *r0 = reg, *r1 = reg + L, *tmp = reg + 2 * L;
  const int g = grid_for(L, kThreads, 152 * 4);
  HHL_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  const double inv_c_lam = 1.0 / (p.C * p.lam_ub);
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64)
    k_qpp_load<float><<<g, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal, inv_c_lam, p.wall_lo,
                                              p.wall_hi, r0, r1, acc);
  else
    k_qpp_load<double><<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal, inv_c_lam, p.wall_lo,
                                               p.wall_hi, r0, r1, acc);
  HHL_LAUNCH_CHECK("k_qpp_load");
  HHL_PROF_BEGIN(st);
  k_qpp_normalize<<<g, kThreads, 0, st>>>(r0, L, acc);
  HHL_LAUNCH_CHECK("k_qpp_normalize");
  HHL_PROF_BEGIN(st);
  k_qpp_h<<<g, kThreads, 0, st>>>(r0, r1, L);
  HHL_LAUNCH_CHECK("k_qpp_h");
  HHL_PROF_BEGIN(st);
  k_qpp_z_ctrl_inc<<<g, kThreads, 0, st>>>(r1, tmp, L);
  HHL_LAUNCH_CHECK("k_qpp_z_ctrl_inc");
  HHL_PROF_BEGIN(st);
  k_qpp_h<<<g, kThreads, 0, st>>>(r0, tmp, L);
  HHL_LAUNCH_CHECK("k_qpp_h");
  HHL_PROF_BEGIN(st);
  k_qpp_p0<<<g, kThreads, 0, st>>>(r0, L, acc + 1);
  HHL_LAUNCH_CHECK("k_qpp_p0");
  return HHL_OK;
}

hhl_status launch_prep_qsp2(const Plan& p, const int64_t* idx, const double* val, int64_t count, double2* psi,
                            void* state, cudaStream_t st) {
  const int g = grid_for(p.N, kThreads, 152 * 4);
  HHL_PROF_BEGIN(st);
  k_qsp_init<<<g, kThreads, 0, st>>>(psi, p.N);
  HHL_LAUNCH_CHECK("k_qsp_init");
  HHL_PROF_BEGIN(st);
  k_qsp2_tree<<<1, 1024, 0, st>>>(idx, val, count, p.n_s, psi, p.d_scal);
  HHL_LAUNCH_CHECK("k_qsp2_tree");
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64) k_qsp_scale<float><<<g, kThreads, 0, st>>>(psi, p.N, p.n_c, (float2*)p.d_bs);
  else k_qsp_scale<double><<<g, kThreads, 0, st>>>(psi, p.N, p.n_c, (double2*)p.d_bs);
  HHL_LAUNCH_CHECK("k_qsp_scale");
  const int64_t row_units = p.N * (int64_t)p.amp_bytes() / 16;
  const int64_t half_units = p.R * row_units;
  HHL_PROF_BEGIN(st);
  k_prep_fill<<<grid_for(2 * half_units, kThreads, 152 * 16), kThreads, 0, st>>>((const uint4*)p.d_bs, (uint4*)state,
                                                                                row_units, half_units);
  HHL_LAUNCH_CHECK("k_prep_fill");
  return HHL_OK;
}

hhl_status launch_sample(const Plan& p, const void* state, const double* uniforms, int64_t shots, uint64_t* counts,
                         double* cdf, cudaStream_t st) {
  const int64_t half = p.R * p.N;
  HHL_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)p.N * sizeof(uint64_t), st));
  HHL_PROF_BEGIN(st);
  if (p.prec == HHL_PREC_C64) k_sample_cdf<float><<<1, 1024, 0, st>>>((const float2*)state + half, p.N, cdf);
  else k_sample_cdf<double><<<1, 1024, 0, st>>>((const double2*)state + half, p.N, cdf);
  HHL_LAUNCH_CHECK("k_sample_cdf");
  if (shots > 0) {
    HHL_PROF_BEGIN(st);
    k_sample_bins<<<grid_for(shots, kThreads, 152 * 4), kThreads, 0, st>>>(cdf, p.N, uniforms, shots,
                                                                          (unsigned long long*)counts);
    HHL_LAUNCH_CHECK("k_sample_bins");
  }
  return HHL_OK;
}

hhl_status launch_dissipation(const Plan& p, const void* state, double* eps, double* u_dev, cudaStream_t st) {
  const int64_t half = p.R * p.N;
  HHL_CUDA_TRY(cudaMemsetAsync(p.d_scal + 4, 0, sizeof(double), st));
  const int g = grid_for(p.N + 1, kThreads, 152 * 4);
  const double inv_c_lam = 1.0 / (p.C * p.lam_ub);
  if (p.prec == HHL_PREC_C64) {
    HHL_PROF_BEGIN(st);
    k_diss_sum<float><<<g, kThreads, 0, st>>>((const float2*)state, half, p.N, p.d_scal, inv_c_lam, p.wall_lo,
                                              p.wall_hi, p.d_scal + 4, u_dev);
  } else {
    HHL_PROF_BEGIN(st);
    k_diss_sum<double><<<g, kThreads, 0, st>>>((const double2*)state, half, p.N, p.d_scal, inv_c_lam, p.wall_lo,
                                               p.wall_hi, p.d_scal + 4, u_dev);
  }
  HHL_LAUNCH_CHECK("k_diss_sum");
  HHL_PROF_BEGIN(st);
  k_diss_finish<<<1, 32, 0, st>>>(p.d_scal + 4, p.nu * (double)(p.N + 1), eps);
  HHL_LAUNCH_CHECK("k_diss_finish");
  return HHL_OK;
}

hhl_status launch_expm_eigen(int N, int J, const double* d_vr, const double* d_vi, const double* d_cos,
                             const double* d_sin, double wgt, double2* d_u, cudaStream_t st) {
  dim3 grid((unsigned)((N + 15) / 16), (unsigned)((N + 15) / 16));
  HHL_PROF_BEGIN(st);
  k_expm_eigen<<<grid, 256, 0, st>>>(N, J, d_vr, d_vi, d_cos, d_sin, wgt, d_u);
  HHL_LAUNCH_CHECK("k_expm_eigen");
  return HHL_OK;
}

// Toeplitz tridiagonal A = tridiag(o, d, o): eigenpairs lambda_j = d + 2 o cos(j pi/(N+1)),
// v_j(i) = sqrt(2/(N+1)) sin(i j pi/(N+1)) (i, j = 1..N), so with sin a sin b =
// (cos(a-b) - cos(a+b))/2,
//   U[n][m] = sum_j v_j(n) v_j(m) e^{i lambdahat_j t} = g(n-m) - g(n+m)   (1-based n, m),
//   g(q) = 1/(N+1) sum_j cos(q j pi/(N+1)) e^{i lambdahat_j t}.
// g for q in [0, 2N+2) (cos(q j pi/(N+1)) read from a table by (q j) mod (2N+2)), FP64.
__global__ void __launch_bounds__(256) k_toeplitz_g(int N, const double* __restrict__ cph,
                                                    const double* __restrict__ sph,
                                                    const double* __restrict__ ctab, double2* __restrict__ g) {
  const int M = 2 * N + 2;
  const double inv = 1.0 / (double)(N + 1);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < M; q += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    int r = 0;  // (q j) mod M
    for (int j = 1; j <= N; ++j) {
      r += q;
      if (r >= M) r -= M;
      const double c = ctab[r];
      re = fma(c, cph[j - 1], re);
      im = fma(c, sph[j - 1], im);
    }
    g[q] = make_double2(re * inv, im * inv);
  }
}

// U[n][m] = g(|n - m|) - g(n + m + 2), 0-based n, m.
__global__ void k_toeplitz_u(int N, const double2* __restrict__ g, double2* __restrict__ U) {
  const int64_t total = (int64_t)N * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / N), m = (int)(e - (int64_t)n * N);
    const double2 a = g[n > m ? n - m : m - n], b = g[n + m + 2];
    U[e] = make_double2(a.x - b.x, a.y - b.y);
  }
}

hhl_status launch_toeplitz_expm(int N, const double* d_c, const double* d_s, const double* d_ctab, double2* d_g,
                                double2* d_u, cudaStream_t st) {
  const int M = 2 * N + 2;
  HHL_PROF_BEGIN(st);
  k_toeplitz_g<<<(M + 255) / 256, 256, 0, st>>>(N, d_c, d_s, d_ctab, d_g);
  HHL_LAUNCH_CHECK("k_toeplitz_g");
  HHL_PROF_BEGIN(st);
  k_toeplitz_u<<<grid_for((int64_t)N * N, kThreads, 152 * 16), kThreads, 0, st>>>(N, d_g, d_u);
  HHL_LAUNCH_CHECK("k_toeplitz_u");
  return HHL_OK;
}

__global__ void k_g_to_df(int M, const double2* __restrict__ g, float4* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < M; q += gridDim.x * blockDim.x) {
    const double2 v = g[q];
    const float rh = (float)v.x, ih = (float)v.y;
    out[q] = make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  }
}

hhl_status launch_g_to_df(int N, const double2* d_g, float4* gdf, cudaStream_t st) {
  const int M = 2 * N + 2;
  HHL_PROF_BEGIN(st);
  k_g_to_df<<<(M + 255) / 256, 256, 0, st>>>(M, d_g, gdf);
  HHL_LAUNCH_CHECK("k_g_to_df");
  return HHL_OK;
}

// A controlled product on few rows (the small steps of the postselected solve's trees, 2^k < 128
// rows): y[i][n] = sum_m U'[n][m] x[i][m] with U' = U_k or U_k^dagger = conj(U_k) generated on
// the fly from the double-float g table (U[n][m] = g(|n - m|) - g(n + m + 2)), so no N x N
// operand is written or read. A block owns TN output columns n of MT rows (MT = min(16, rows
// of the step); TN = 8, 16 or 32, the largest that still gives two blocks per SM) and splits
// the sum over m in 256 / TN parts: thread t takes n = n0 + t % TN and every (256 / TN)-th
// column of each chunk of CH columns (1024 for blocks of up to 4 rows, whose chunks are
// latency-bound round trips with little arithmetic, else 256). Per chunk the block stages the
// x rows and the g entries the chunk needs (its TN + CH - 1 differences n - m and sums
// n + m + 2) in shared memory, the loads of a thread issued together; the parts of each output
// are added by shuffles inside the warp, then across the 8 warps in shared memory (reusing the
// x buffer). Output rows are mapped as the GEMMs' (write, or add to the row and scale). At
// N >= 512 blocks of 4-16 rows take k_toeplitz_rows_ks below instead (the sum over m split
// across a cluster of 4 CTAs); this kernel serves the 1- and 2-row steps and small N.
template <int MT> constexpr int toep_chunk() { return MT <= 4 ? 1024 : 256; }
template <int MT, int TN> constexpr int toep_smem() {
  return MT * toep_chunk<MT>() * (int)sizeof(float2) + 2 * (TN + toep_chunk<MT>()) * (int)sizeof(float4);
}

// Tree steps on fewer rows than this take the on-the-fly Toeplitz product instead of a GEMM
// (128 by default: the tensor-core tiles start at 128 rows); HHL_TOEP_ROWS=<power of two>
// moves the threshold.
int64_t toeplitz_rows_limit() {
  static const int64_t lim = [] {
    const char* e = getenv("HHL_TOEP_ROWS");
    const long long v = e != nullptr ? atoll(e) : 0;
    return v >= 1 ? (int64_t)v : (int64_t)128;
  }();
  return lim;
}

template <int MT, int TN>
__global__ void __launch_bounds__(256) k_toeplitz_rows(float2* __restrict__ half, int n_s, const float4* __restrict__ g,
                                                       int adjoint, RowMap rows, int64_t m_rows) {
  constexpr int P = 256 / TN;                      // parts of each output
  constexpr int CH = toep_chunk<MT>();             // columns per chunk
  constexpr int kXs = MT * CH;                     // staged x values per chunk
  constexpr int kLd = (kXs + 255) / 256;           // x loads per thread per chunk
  constexpr int kGl = (TN + CH + 255) / 256;       // g entries per thread per chunk
  static_assert(8 * MT * TN <= kXs, "partials reuse the x buffer");
  extern __shared__ __align__(16) unsigned char toep_smem_raw[];
  float2* xs = reinterpret_cast<float2*>(toep_smem_raw);   // [kXs]
  float4* gd = reinterpret_cast<float4*>(xs + kXs);        // [TN + CH]: g(|n - m|)
  float4* gs = gd + (TN + CH);                             // [TN + CH]: g(n + m + 2)
  const int N = 1 << n_s;
  const int gmax = 2 * N + 1;  // last entry of the g table
  const int nl = threadIdx.x % TN, cs = threadIdx.x / TN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * TN, n = n0 + nl;
  const int64_t i0 = (int64_t)blockIdx.y * MT;
  const int64_t left = m_rows - i0;
  const int nr = left < MT ? (int)left : MT;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 acc[MT];
#pragma unroll
  for (int r = 0; r < MT; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int c0 = 0; c0 < N; c0 += CH) {
    const int cw = min(CH, N - c0);
    // differences n - m = (n0 - c0 - cw + 1) + j and sums n + m + 2 = (n0 + c0 + 2) + j
    const int dlo = n0 - c0 - cw + 1, slo = n0 + c0 + 2;
    float2 v[kLd];
    float4 ga[kGl], gb[kGl];
#pragma unroll
    for (int j = 0; j < kLd; ++j) {
      const int e = threadIdx.x + j * 256;
      const int r = e / CH, c = e % CH;
      v[j] = (e < kXs && r < nr && c < cw) ? half[rowmap_in(rows, i0 + r) * N + c0 + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < kGl; ++q) {
      const int j = threadIdx.x + q * 256;
      const int ia = abs(dlo + j), is = slo + j;
      const bool in = j < TN + cw - 1;
      ga[q] = in && ia <= gmax ? g[ia] : z4;
      gb[q] = in && is <= gmax ? g[is] : z4;
    }
    __syncthreads();  // the previous chunk's readers are done
#pragma unroll
    for (int j = 0; j < kLd; ++j) {
      const int e = threadIdx.x + j * 256;
      if (e < kXs) xs[e] = v[j];
    }
#pragma unroll
    for (int q = 0; q < kGl; ++q) {
      const int j = threadIdx.x + q * 256;
      if (j < TN + CH) {
        gd[j] = ga[q];
        gs[j] = gb[q];
      }
    }
    __syncthreads();
    if (n < N) {
#pragma unroll 4
      for (int c = cs; c < cw; c += P) {
        const float4 a = gd[nl - c + cw - 1], b = gs[nl + c];
        float2 u = make_float2((a.x - b.x) + (a.y - b.y), (a.z - b.z) + (a.w - b.w));
        if (adjoint) u.y = -u.y;
#pragma unroll
        for (int r = 0; r < MT; ++r) {
          const float2 x = xs[r * CH + c];
          acc[r].x = fmaf(u.x, x.x, fmaf(-u.y, x.y, acc[r].x));
          acc[r].y = fmaf(u.x, x.y, fmaf(u.y, x.x, acc[r].y));
        }
      }
    }
  }
  // the parts of one output inside a warp sit on lanes nl, nl + TN, ...
#pragma unroll
  for (int off = TN; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < MT; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
    }
  }
  __syncthreads();  // every reader of xs is done: it now holds the partials
  float2* part = xs;  // [warp][r][o]
  if (lane < TN) {
#pragma unroll
    for (int r = 0; r < MT; ++r) part[(warp * MT + r) * TN + lane] = acc[r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < MT * TN; e += 256) {
    const int r = e / TN, o = e % TN;
    const int no = n0 + o;
    if (r < nr && no < N) {
      float2 y = part[r * TN + o];
#pragma unroll
      for (int w = 1; w < 8; ++w) {
        y.x += part[(w * MT + r) * TN + o].x;
        y.y += part[(w * MT + r) * TN + o].y;
      }
      float2* d = half + rowmap_out(rows, i0 + r) * N + no;
      if (rows.accumulate) {
        y.x += d->x;
        y.y += d->y;
        if (rows.scale != 1.0) {
          const float sc = (float)rows.scale;
          y.x *= sc;
          y.y *= sc;
        }
      }
      *d = y;
    }
  }
}

// Blocks of MT = 4, 8 or 16 rows with the sum over m split across a cluster of 4 CTAs: CTA q of
// the cluster takes the columns [q N / 4, (q + 1) N / 4) for the same TN outputs and MT rows (the
// direct product above on a quarter of the columns, chunks of 256), so each CTA stages a quarter
// of the x rows for TN outputs, and TN can be 32 with as many blocks as 8 outputs per block
// give without the split. The CTAs' partial tiles (16 x TN, in shared memory) are added through
// distributed shared memory in the order of the cluster ranks (the same sum on every run),
// CTA q writing a quarter of the outputs; a second cluster barrier keeps every tile alive
// until its readers are done.
constexpr int kToepKs = 4;

template <int MT, int TN>
__global__ void __launch_bounds__(256) k_toeplitz_rows_ks(float2* __restrict__ half, int n_s, const float4* __restrict__ g,
                                                          int adjoint, RowMap rows, int64_t m_rows) {
  namespace cg = cooperative_groups;
  constexpr int P = 256 / TN, CH = 256;
  constexpr int kXs = MT * CH, kLd = kXs / 256, kGl = (TN + CH + 255) / 256;
  static_assert(8 * MT * TN <= kXs, "partials reuse the x buffer");
  __shared__ float2 xs[kXs];
  __shared__ float4 gd[TN + CH], gs[TN + CH];
  __shared__ float2 red[MT * TN];  // this CTA's partial tile
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int N = 1 << n_s;
  const int gmax = 2 * N + 1;
  const int nl = threadIdx.x % TN, cs = threadIdx.x / TN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = (int)(blockIdx.x / kToepKs) * TN, n = n0 + nl;
  const int64_t i0 = (int64_t)blockIdx.y * MT;
  const int64_t left = m_rows - i0;
  const int nr = left < MT ? (int)left : MT;
  const int kq = N / kToepKs, k_begin = q * kq, k_end = k_begin + kq;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float2 acc[MT];
#pragma unroll
  for (int r = 0; r < MT; ++r) acc[r] = make_float2(0.f, 0.f);
  for (int c0 = k_begin; c0 < k_end; c0 += CH) {
    const int cw = min(CH, k_end - c0);
    const int dlo = n0 - c0 - cw + 1, slo = n0 + c0 + 2;
    float2 v[kLd];
    float4 ga[kGl], gb[kGl];
#pragma unroll
    for (int j = 0; j < kLd; ++j) {
      const int e = threadIdx.x + j * 256;
      const int r = e / CH, c = e % CH;
      v[j] = (r < nr && c < cw) ? half[rowmap_in(rows, i0 + r) * N + c0 + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int qq = 0; qq < kGl; ++qq) {
      const int j = threadIdx.x + qq * 256;
      const int ia = abs(dlo + j), is = slo + j;
      const bool in = j < TN + cw - 1;
      ga[qq] = in && ia <= gmax ? g[ia] : z4;
      gb[qq] = in && is <= gmax ? g[is] : z4;
    }
    __syncthreads();  // the previous chunk's readers are done
#pragma unroll
    for (int j = 0; j < kLd; ++j) xs[threadIdx.x + j * 256] = v[j];
#pragma unroll
    for (int qq = 0; qq < kGl; ++qq) {
      const int j = threadIdx.x + qq * 256;
      if (j < TN + CH) {
        gd[j] = ga[qq];
        gs[j] = gb[qq];
      }
    }
    __syncthreads();
    if (n < N) {
#pragma unroll 4
      for (int c = cs; c < cw; c += P) {
        const float4 a = gd[nl - c + cw - 1], b = gs[nl + c];
        float2 u = make_float2((a.x - b.x) + (a.y - b.y), (a.z - b.z) + (a.w - b.w));
        if (adjoint) u.y = -u.y;
#pragma unroll
        for (int r = 0; r < MT; ++r) {
          const float2 x = xs[r * CH + c];
          acc[r].x = fmaf(u.x, x.x, fmaf(-u.y, x.y, acc[r].x));
          acc[r].y = fmaf(u.x, x.y, fmaf(u.y, x.x, acc[r].y));
        }
      }
    }
  }
#pragma unroll
  for (int off = TN; off < 32; off <<= 1) {
#pragma unroll
    for (int r = 0; r < MT; ++r) {
      acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
      acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
    }
  }
  __syncthreads();
  float2* part = xs;  // [warp][r][o]
  if (lane < TN) {
#pragma unroll
    for (int r = 0; r < MT; ++r) part[(warp * MT + r) * TN + lane] = acc[r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < MT * TN; e += 256) {
    float2 y = part[e];  // e = r * TN + o
#pragma unroll
    for (int w = 1; w < 8; ++w) {
      y.x += part[w * MT * TN + e].x;
      y.y += part[w * MT * TN + e].y;
    }
    red[e] = y;
  }
  cl.sync();  // every CTA's partial tile is complete
  constexpr int kOut = MT * TN / kToepKs;  // outputs this CTA writes (MT * TN divides by 4)
  for (int e = q * kOut + threadIdx.x; e < (q + 1) * kOut; e += 256) {
    const int r = e / TN, o = e % TN;
    const int no = n0 + o;
    float2 y = make_float2(0.f, 0.f);
#pragma unroll
    for (int rr = 0; rr < kToepKs; ++rr) {
      const float2 p = cl.map_shared_rank(red, rr)[e];
      y.x += p.x;
      y.y += p.y;
    }
    if (r < nr && no < N) {
      float2* d = half + rowmap_out(rows, i0 + r) * N + no;
      if (rows.accumulate) {
        y.x += d->x;
        y.y += d->y;
        if (rows.scale != 1.0) {
          const float sc = (float)rows.scale;
          y.x *= sc;
          y.y *= sc;
        }
      }
      *d = y;
    }
  }
  cl.sync();  // the partial tiles stay until every reader is done
}

template <int MT, int TN>
cudaError_t toeplitz_rows_ks_launch(dim3 grid, cudaStream_t st, float2* half, int n_s, const float4* g, int adjoint,
                                    const RowMap& rows, int64_t m) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kToepKs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_toeplitz_rows_ks<MT, TN>, half, n_s, g, adjoint, rows, m);
}

template <int MT>
cudaError_t toeplitz_rows_ks_tn(int tk, dim3 grid, cudaStream_t st, float2* half, int n_s, const float4* g,
                                int adjoint, const RowMap& rows, int64_t m) {
  if (tk == 32) return toeplitz_rows_ks_launch<MT, 32>(grid, st, half, n_s, g, adjoint, rows, m);
  if (tk == 16) return toeplitz_rows_ks_launch<MT, 16>(grid, st, half, n_s, g, adjoint, rows, m);
  return toeplitz_rows_ks_launch<MT, 8>(grid, st, half, n_s, g, adjoint, rows, m);
}

template <int MT, int TN>
cudaError_t toeplitz_rows_launch(dim3 grid, cudaStream_t st, float2* half, int n_s, const float4* g, int adjoint,
                                 const RowMap& rows, int64_t m) {
  constexpr int smem = toep_smem<MT, TN>();
  cudaError_t e = raise_dyn_smem((const void*)k_toeplitz_rows<MT, TN>, smem);
  if (e != cudaSuccess) return e;
  k_toeplitz_rows<MT, TN><<<grid, 256, smem, st>>>(half, n_s, g, adjoint, rows, m);
  return cudaSuccess;
}

template <int MT>
cudaError_t toeplitz_rows_tn(int tn, dim3 grid, cudaStream_t st, float2* half, int n_s, const float4* g, int adjoint,
                             const RowMap& rows, int64_t m) {
  if (tn == 32) return toeplitz_rows_launch<MT, 32>(grid, st, half, n_s, g, adjoint, rows, m);
  if (tn == 16) return toeplitz_rows_launch<MT, 16>(grid, st, half, n_s, g, adjoint, rows, m);
  return toeplitz_rows_launch<MT, 8>(grid, st, half, n_s, g, adjoint, rows, m);
}

hhl_status launch_toeplitz_rows(float2* half, int n_s, const float4* g, int adjoint, const RowMap& rows, int64_t m,
                                cudaStream_t st) {
  const int64_t N = 1LL << n_s;
  const int mt = m >= 16 ? 16 : (int)m;  // m is a power of two here
  const int64_t groups = (m + mt - 1) / mt;
  if (mt >= 4 && N >= 512) {  // the sum over m split across clusters of 4 CTAs
    int tk = 32;
    while (tk > 8 && ((N + tk - 1) / tk) * groups * kToepKs < 2 * 152) tk /= 2;
    dim3 gk((unsigned)(((N + tk - 1) / tk) * kToepKs), (unsigned)groups);
    HHL_PROF_BEGIN(st);
    cudaError_t e = mt == 16  ? toeplitz_rows_ks_tn<16>(tk, gk, st, half, n_s, g, adjoint, rows, m)
                    : mt == 8 ? toeplitz_rows_ks_tn<8>(tk, gk, st, half, n_s, g, adjoint, rows, m)
                              : toeplitz_rows_ks_tn<4>(tk, gk, st, half, n_s, g, adjoint, rows, m);
    if (e != cudaSuccess) return cuda_fail(e, "k_toeplitz_rows_ks");
    HHL_LAUNCH_CHECK("k_toeplitz_rows");
    return HHL_OK;
  }
  int tn = 32;  // outputs per block: the widest that still gives two blocks per SM
  while (tn > 8 && ((N + tn - 1) / tn) * groups < 2 * 152) tn /= 2;
  dim3 grid((unsigned)((N + tn - 1) / tn), (unsigned)groups);
  HHL_PROF_BEGIN(st);
  cudaError_t e;
  switch (mt) {
    case 1: e = toeplitz_rows_tn<1>(tn, grid, st, half, n_s, g, adjoint, rows, m); break;
    case 2: e = toeplitz_rows_tn<2>(tn, grid, st, half, n_s, g, adjoint, rows, m); break;
    case 4: e = toeplitz_rows_tn<4>(tn, grid, st, half, n_s, g, adjoint, rows, m); break;
    case 8: e = toeplitz_rows_tn<8>(tn, grid, st, half, n_s, g, adjoint, rows, m); break;
    default: e = toeplitz_rows_tn<16>(tn, grid, st, half, n_s, g, adjoint, rows, m); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "k_toeplitz_rows (shared-memory limit)");
  HHL_LAUNCH_CHECK("k_toeplitz_rows");
  return HHL_OK;
}

hhl_status launch_store_operands(const Plan& p, const double2* d_u, int k, cudaStream_t st) {
  const size_t mat = (size_t)p.N * p.N;
  const int g = grid_for((int64_t)mat, kThreads, 152 * 16);
  if (p.prec == HHL_PREC_C64) {
    HHL_PROF_BEGIN(st);
    k_store_operands<float><<<g, kThreads, 0, st>>>(d_u, p.N, (float2*)p.d_bfwd + k * mat, (float2*)p.d_badj + k * mat);
  } else {
    HHL_PROF_BEGIN(st);
    k_store_operands<double><<<g, kThreads, 0, st>>>(d_u, p.N, (double2*)p.d_bfwd + k * mat, (double2*)p.d_badj + k * mat);
  }
  HHL_LAUNCH_CHECK("k_store_operands");
  return HHL_OK;
}

}  // namespace hhl
