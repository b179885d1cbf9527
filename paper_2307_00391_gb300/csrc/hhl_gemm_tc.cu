// Controlled-U_k GEMM on the 5th-generation tensor cores (tcgen05, sm_103a), complex64.
//
// The controlled U_k multiplies every system-register row r (length N, complex) whose
// clock bit k is set: r <- U_k r. In real arithmetic on interleaved (re, im) floats this is
// one real GEMM  Y (M x 2N) = X (M x 2N) * E^T, with M = 2^(n_c-1) rows and the real
// embedding E (2N x 2N):  E[2n][2m] = Re U[n][m], E[2n][2m+1] = -Im U[n][m],
// E[2n+1][2m] = Im U[n][m], E[2n+1][2m+1] = Re U[n][m]. Its flops equal the complex GEMM's
// 8 M N N.
//
// FP32 accuracy from FP16 tensor cores (split FP16): both operands are scaled by 2^15
// (|amplitude| <= 1 in a normalised state and |U entry| <= 1, so the scaled values stay
// below the FP16 maximum 65504) and split as v ~ hi + lo, hi = v rounded to the nearest FP16,
// lo = (v - hi) rounded to the nearest FP16 (round to nearest keeps the splitting error
// unbiased, so the norm does not drift over the 2 n_c controlled products). The product is
// X_hi E_hi + X_hi E_lo + X_lo E_hi, accumulated in FP32 in tensor memory (three kind::f16
// MMAs per K step, A and B both FP16), and the epilogue multiplies by 2^-30. Each part carries
// 11 significant bits, so the represented operands hold about 22 bits, as split TF32 does, at
// twice the TF32 tensor rate and with half the operand bytes. The row gather flags any
// amplitude of magnitude >= 2 (outside the scaled FP16 range) as a numeric error.
// The plan stores E_hi and E_lo (forward and adjoint) for every k; the gather kernel copies
// the rows with bit k set into compact X_hi / X_lo arrays, so the GEMM may write its result
// straight back into those state rows.
//
// Kernel (persistent, stream-K): the work is the list of (output tile, K step) units, tile-major,
// 128 x BN tiles of K / 32 steps each; the grid has one CTA per SM (fewer when there are few
// units, every CTA keeping at least a quarter of a tile's steps) and CTA b takes the contiguous
// units [b U / G, (b + 1) U / G), so every SM does the same number of MMAs whatever the number
// of rows (a 128-row product no longer runs on 8 SMs only). When the tiles alone fill most of
// the SMs the grid is one CTA per tile instead (each range is one whole tile): a large product
// is bound by the operand bytes each SM takes in per stage (48 KiB of A and B for six MMAs),
// which a finer split does not reduce, and the split tiles' partials would cost a second pass.
// One CTA per tile also lets clusters of four CTAs (four consecutive row tiles of one column
// tile) share the B operand: each loads a quarter of every B stage and multicasts it to all
// four, which cuts the L2 reads by 43% (the SM intake stays the same). Its range is a sequence of tile
// segments. Roles: warp 0 (one lane) issues the TMA loads (64-byte swizzle, 32 K elements per
// stage: four stages at BN = 256, six at 128) into a ring of
// shared-memory stages, across segment boundaries; warp 1 (one lane) issues the MMAs
// (M = 128, N = BN, K = 16) into one of two BN-column TMEM accumulators, alternating per
// segment, so that the epilogue of one segment overlaps the MMAs of the next; warps 2-5 drain
// TMEM with tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) .. + 31, i.e. output rows). A
// segment that covers its whole tile is written straight to the state rows. A tile split over
// several CTAs needs no wait between CTAs: each contributor stores its FP32 partial in a
// workspace slot of its own (two per CTA: its range's first and last segment), and a second
// launch on the same stream, k_tc_fixup, adds each split tile's partials in the order of the
// CTAs (the same sum on every run) and writes the rows. Every mbarrier wait is
// bounded (wait_cycles, a kernel argument) and gives up early once another role has given up;
// on expiry the CTA records an error flag (read back as HHL_ERR_TIMEOUT) and skips the
// remaining work, but before it frees its TMEM and exits it drains what it started: the
// producer waits (bounded) for every bulk copy it issued to land, and the MMA lane always
// commits its issued MMAs to the final barrier, which the whole CTA waits on (bounded) before
// the dealloc (and k_tc_fixup does nothing once the flag is set).
// Fault injection for the error path (fault = 1): the producer issues no copy at all, so the
// MMA lane's first wait runs out with nothing in flight.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <stdlib.h>
#include <string.h>

#include "hhl_common.cuh"

namespace hhl {

namespace {

constexpr int kBM = 128;           // output rows per CTA (MMA M)
constexpr int kBN = 256;           // output real columns per CTA (MMA N), plan path
constexpr int kBK = 32;            // fp16 K elements per stage (64 bytes: one swizzle row)
constexpr int kTileA = kBM * kBK * 2;   // 8 KiB
constexpr int kThreadsTc = 192;    // producer warp, MMA warp, four epilogue warps
constexpr float kOpScale = 32768.0f;    // 2^15 on each operand
constexpr float kUnscale = 1.0f / (32768.0f * 32768.0f);  // 2^-30 on the product
template <int BN> struct TcShape {
  static constexpr int kTileB = BN * kBK * 2;                     // 16 KiB at BN = 256
  static constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;     // A_hi, A_lo, B_hi, B_lo
  static constexpr int kStages = BN == 256 ? 4 : 6;               // 192 KiB of stages either way
  static constexpr int kSmemBytes = kStages * kStageBytes + 1024;  // + alignment slack
  static constexpr int kTmemCols = 2 * BN;                        // two fp32 accumulators
};
constexpr long long kWaitCycles = 4000000000LL;      // default bound of a wait: ~2 s at 2 GHz
constexpr long long kFaultWaitCycles = 2000000LL;    // injected timeout: ~1 ms

struct TcState {
  __half* a_hi = nullptr;  // M_sub x 2N
  __half* a_lo = nullptr;
  __half* b = nullptr;     // n_c x {fwd_hi, fwd_lo, adj_hi, adj_lo} x (2N x 2N)
  int* err = nullptr;      // device error flag
  TcWork work;             // stream-K partials and tile counters
  int bn = kBN;           // output tile width (128 or 256)
  std::vector<CUtensorMap> maps;  // [0] A_hi, [1] A_lo, then per k: fwd_hi, fwd_lo, adj_hi, adj_lo
  std::vector<CUtensorMap> smaps; // per k the same four with a quarter-height box (cluster slices)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false (and the error flag set) after
// `limit` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err, int code, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// The same, also giving up (without a flag of its own) once another role of the CTA has set
// *abort; on its own expiry it sets *abort.
__device__ __forceinline__ bool mbar_wait_role(uint64_t* bar, uint32_t parity, int* err, int code, long long limit,
                                               volatile int* abort) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > limit) {
      atomicExch(err, code);
      *abort = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Barrier 1 over the four epilogue warps (128 threads).
__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// Stream-K partition: CTA b of G takes units [b U / G, (b + 1) U / G); the CTA holding unit x.
__device__ __forceinline__ int64_t sk_start(int64_t b, int64_t units, int64_t G) { return b * units / G; }
__device__ __forceinline__ int64_t sk_owner(int64_t x, int64_t units, int64_t G) { return ((x + 1) * G - 1) / units; }
// End (exclusive K step) of the segment that starts at step kb of a tile with `left` units left.
__device__ __forceinline__ int seg_end(int kb, int k_iters, int64_t left) {
  return left < (int64_t)(k_iters - kb) ? kb + (int)left : k_iters;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// The same box delivered to the same shared-memory offset of every CTA in `mask` (this GPU's
// own memory; each destination's mbarrier at the same offset receives the bytes it got).
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(dst),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle (rows of 32 FP16), 8-row
// atoms 512 B apart.
__device__ __forceinline__ uint64_t desc_sw64(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;          // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)4 << 61;                   // 64-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16, D = F32, A = B = F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int m, int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Arrive on the mbarrier at the same offset in every CTA of `mask` once this thread's MMAs so
// far have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void tmem_ld_32cols(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// v (already scaled by 2^15) -> (hi, lo): hi = nearest FP16, lo = nearest FP16 of v - hi.
__device__ __forceinline__ void split_f16(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}


template <int BN, int CL>
__global__ void __launch_bounds__(kThreadsTc, 1)
    k_ctrl_gemm_tc(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
                   const __grid_constant__ CUtensorMap map_bhi, const __grid_constant__ CUtensorMap map_blo,
                   float* __restrict__ state_half, int n_s, RowMap rows, int k_iters, int tiles_n, int64_t units,
                   float* __restrict__ ws, int* err, long long wait_cycles, int fault) {
  constexpr int S = TcShape<BN>::kStages;
  constexpr int kTileB = TcShape<BN>::kTileB, kStageBytes = TcShape<BN>::kStageBytes;
  constexpr int kTmemCols = TcShape<BN>::kTmemCols;
  constexpr int kPart = kBM * BN;  // floats of one partial tile
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int s_go[2];  // by segment parity: rewritten only two barriers later

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const int64_t G = gridDim.x, cta = blockIdx.x;
  int64_t u_begin = sk_start(cta, units, G), u_end = sk_start(cta + 1, units, G);
  const int crank = (int)(cta % CL);  // rank in the cluster (clusters of CL consecutive CTAs)
  constexpr uint16_t kMask = (uint16_t)((1u << CL) - 1u);
  if (CL > 1) {
    // one whole tile per CTA: the cluster's CL CTAs take CL consecutive row tiles of one column
    // tile and share its B operand, each loading 1 / CL of it for all of them
    const int64_t rest = cta / CL;
    const int64_t t = ((rest / tiles_n) * CL + crank) * tiles_n + rest % tiles_n;
    u_begin = t * k_iters;
    u_end = u_begin + k_iters;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], CL);  // a stage is free once every CTA it is delivered to has read it
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&tfull_bar[s], 1);
      mbar_init(&tempty_bar[s], 128);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (CL > 1) cluster_sync_all();  // every CTA's barriers are initialised before any remote signal
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer: TMA loads of the four operand tiles of each K step, segment after segment
      int64_t gi = 0, issued = 0;
      for (int64_t u = u_begin; u < u_end && !fault && !abort_flag;) {
        const int64_t t = u / k_iters;
        const int kb = (int)(u - t * k_iters);
        const int ke = seg_end(kb, k_iters, u_end - u);
        const int m0 = (int)(t / tiles_n) * kBM, n0 = (int)(t % tiles_n) * BN;
        for (int it = kb; it < ke; ++it, ++gi) {
          const int s = (int)(gi % S);
          if (!mbar_wait_role(&empty_bar[s], (uint32_t)((gi / S) & 1) ^ 1u, err, 1, wait_cycles, &abort_flag)) break;
          const uint32_t st = base + s * kStageBytes;
          mbar_expect_tx(&full_bar[s], kStageBytes);
          const int kx = it * kBK;
          tma_load_2d(st, &map_ahi, &full_bar[s], kx, m0);
          tma_load_2d(st + kTileA, &map_alo, &full_bar[s], kx, m0);
          if (CL > 1) {  // this CTA's slice of B (BN / CL rows; the maps' box), to every CTA of the cluster
            const uint32_t so = (uint32_t)crank * (kTileB / CL);
            tma_load_2d_mc(st + 2 * kTileA + so, &map_bhi, &full_bar[s], kx, n0 + crank * (BN / CL), kMask);
            tma_load_2d_mc(st + 2 * kTileA + kTileB + so, &map_blo, &full_bar[s], kx, n0 + crank * (BN / CL), kMask);
          } else {
            tma_load_2d(st + 2 * kTileA, &map_bhi, &full_bar[s], kx, n0);
            tma_load_2d(st + 2 * kTileA + kTileB, &map_blo, &full_bar[s], kx, n0);
          }
          issued = gi + 1;
        }
        u += ke - kb;
      }
      // drain: the last copy issued into each stage has landed before shared memory is released
      // (on the normal path the MMA lane has already consumed them, so these return at once)
      for (int64_t g2 = issued > S ? issued - S : 0; g2 < issued; ++g2)
        mbar_wait_bounded(&full_bar[g2 % S], (uint32_t)((g2 / S) & 1), err, 5, wait_cycles);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: one accumulator per segment, alternating between the two
      constexpr uint32_t idesc = idesc_f16(kBM, BN);
      int64_t gi = 0;
      int j = 0;
      bool ok = true;
      for (int64_t u = u_begin; u < u_end && ok; ++j) {
        const int64_t t = u / k_iters;
        const int kb = (int)(u - t * k_iters);
        const int ke = seg_end(kb, k_iters, u_end - u);
        const int buf = j & 1;
        // the epilogue has read this accumulator's previous segment (free at first use)
        if (!mbar_wait_role(&tempty_bar[buf], (uint32_t)((j >> 1) & 1) ^ 1u, err, 3, wait_cycles, &abort_flag)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(buf * BN);
        for (int it = kb; it < ke; ++it, ++gi) {
          const int s = (int)(gi % S);
          if (!mbar_wait_role(&full_bar[s], (uint32_t)((gi / S) & 1), err, 2, wait_cycles, &abort_flag)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = base + s * kStageBytes;
          const uint32_t a_hi = st, a_lo = st + kTileA, b_hi = st + 2 * kTileA, b_lo = st + 2 * kTileA + kTileB;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 fp16 = 32 bytes along K inside the swizzled row
            const uint32_t acc0 = (it > kb || kk > 0) ? 1u : 0u;
            mma_f16(d, desc_sw64(a_hi + off), desc_sw64(b_hi + off), idesc, acc0);
            mma_f16(d, desc_sw64(a_hi + off), desc_sw64(b_lo + off), idesc, 1u);
            mma_f16(d, desc_sw64(a_lo + off), desc_sw64(b_hi + off), idesc, 1u);
          }
          if (CL > 1)
            mma_commit_mc(&empty_bar[s], kMask);  // every CTA that delivers into this stage waits on it
          else
            mma_commit(&empty_bar[s]);  // stage free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&tfull_bar[buf]);  // the segment's accumulator is complete
        u += ke - kb;
      }
      // always commit: done_bar completes once every MMA this lane issued has finished (at once
      // when none was), so the wait below also drains an aborted accumulation before the dealloc
      mma_commit(&done_bar);
    }
  } else {
    // epilogue: warps 2-5, thread row = its TMEM lane
    const int q = warp & 3;
    const int row = q * 32 + lane;
    const bool leader = threadIdx.x == 64;
    const int64_t N2 = 2LL << n_s;  // floats per state row
    int j = 0;
    for (int64_t u = u_begin; u < u_end; ++j) {
      const int64_t t = u / k_iters;
      const int kb = (int)(u - t * k_iters);
      const int ke = seg_end(kb, k_iters, u_end - u);
      const int buf = j & 1;
      if (leader) s_go[j & 1] = mbar_wait_role(&tfull_bar[buf], (uint32_t)((j >> 1) & 1), err, 3, wait_cycles, &abort_flag);
      epilogue_sync();
      if (!s_go[j & 1]) break;  // uniform: read after the barrier
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
      const int m0 = (int)(t / tiles_n) * kBM, n0 = (int)(t % tiles_n) * BN;
      float* dst = state_half + rowmap_out(rows, m0 + row) * N2 + n0;
      if (kb == 0 && ke == k_iters) {
        // the whole tile is this CTA's: straight to the state row
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          float v[32];
          tmem_ld_32cols(taddr + c, v);
          float4* d4 = reinterpret_cast<float4*>(dst + c);
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float4 o = make_float4(v[4 * e] * kUnscale, v[4 * e + 1] * kUnscale, v[4 * e + 2] * kUnscale,
                                   v[4 * e + 3] * kUnscale);
            if (rows.accumulate) {  // a reduction step of the postselected solve: the row keeps its value
              const float4 prev = d4[e];
              o = make_float4(prev.x + o.x, prev.y + o.y, prev.z + o.z, prev.w + o.w);
            }
            d4[e] = o;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty_bar[buf]);
      } else {
        // a split tile: this CTA's FP32 partial goes to its slot (row-major 128 x BN; slot 0 when
        // the segment starts the CTA's range inside the tile, else slot 1), added up by
        // k_tc_fixup after the launch
        float* wp = ws + (size_t)(2 * cta + (u_begin > t * k_iters ? 0 : 1)) * kPart + (size_t)row * BN;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
          float v[32];
          tmem_ld_32cols(taddr + c, v);
          float4* w4 = reinterpret_cast<float4*>(wp + c);
#pragma unroll
          for (int e = 0; e < 8; ++e) __stcg(w4 + e, make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&tempty_bar[buf]);  // the accumulator is free for the segment after next
      }
      u += ke - kb;
    }
  }
  __syncwarp();
  __syncthreads();  // every role has left its (bounded) loop

  if (!mbar_wait_bounded(&done_bar, 0, err, 3, wait_cycles)) abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  // no CTA leaves while a partner may still signal its barriers or deliver into its stages
  if (CL > 1) cluster_sync_all();
}

// The tiles the stream-K GEMM split over several CTAs: one thread per 4 output columns adds
// the contributors' partials in CTA order (the same sum on every run), scales by 2^-30 and
// writes (or adds to) the state row. Tiles held whole by one CTA were written by the GEMM.
template <int BN>
__global__ void __launch_bounds__(256) k_tc_fixup(const float4* __restrict__ ws, float* __restrict__ state_half,
                                                  int n_s, RowMap rows, int k_iters, int tiles_n, int64_t units,
                                                  int64_t G, int* err) {
  constexpr int kQ = BN / 4;  // float4 per tile row
  const int64_t t = blockIdx.y;
  const int64_t t0u = t * k_iters;
  const int64_t first = ((t0u + 1) * G - 1) / units, last = ((t0u + k_iters) * G - 1) / units;
  if (first == last || *err != 0) return;  // whole tile, or the GEMM gave up
  const int e = blockIdx.x * 256 + threadIdx.x;  // < 128 * kQ by the grid
  const int row = e / kQ, q = e % kQ;
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t b = first; b <= last; ++b) {
    const int64_t slot = 2 * b + (b * units / G > t0u ? 0 : 1);
    const float4 v = __ldcg(ws + slot * (kBM * kQ) + (int64_t)row * kQ + q);
    o = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
  }
  const int m0 = (int)(t / tiles_n) * kBM, n0 = (int)(t % tiles_n) * BN;
  float4* d4 = reinterpret_cast<float4*>(state_half + rowmap_out(rows, m0 + row) * (2LL << n_s) + n0) + q;
  o = make_float4(o.x * kUnscale, o.y * kUnscale, o.z * kUnscale, o.w * kUnscale);
  if (rows.accumulate) {
    const float4 prev = *d4;
    o = make_float4(prev.x + o.x, prev.y + o.y, prev.z + o.z, prev.w + o.w);
  }
  *d4 = o;
}

// The mapped rows (those with clock bit k set, or a tree step's source rows) -> compact FP16
// hi / lo arrays (M_sub x 2N), scaled by 2^15.
// An amplitude component of magnitude >= 2 cannot be represented: error flag 4.
__global__ void k_tc_split_rows(const float4* __restrict__ half, uint2* __restrict__ a_hi, uint2* __restrict__ a_lo,
                                int n_s, RowMap rows, int64_t m_sub, int* err) {
  const int row4_bits = n_s - 1;  // float4 per row = 2N/4 = 2^(n_s-1)
  const int64_t total = m_sub << row4_bits;
  constexpr int U = 4;  // loads in flight per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < total; e0 += U * stride) {
    float4 v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t e = e0 + q * stride;
      if (e < total) {
        const int64_t i = e >> row4_bits, c = e & ((1LL << row4_bits) - 1);
        v[q] = half[(rowmap_in(rows, i) << row4_bits) + c];
      }
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int64_t e = e0 + q * stride;
      if (e < total) {
        const float x[4] = {v[q].x * kOpScale, v[q].y * kOpScale, v[q].z * kOpScale, v[q].w * kOpScale};
        __half h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          split_f16(x[j], h[j], l[j]);
          bad |= !(fabsf(x[j]) < 2.0f * kOpScale);
        }
        a_hi[e] = make_uint2((uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16),
                             (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16));
        a_lo[e] = make_uint2((uint32_t)__half_as_ushort(l[0]) | ((uint32_t)__half_as_ushort(l[1]) << 16),
                             (uint32_t)__half_as_ushort(l[2]) | ((uint32_t)__half_as_ushort(l[3]) << 16));
      }
    }
  }
  if (bad) atomicExch(err, 4);
}

// Real embeddings of U_k (forward) and U_k^dagger (adjoint), scaled by 2^15 and split into
// FP16 hi / lo. out layout: [fwd_hi | fwd_lo | adj_hi | adj_lo], each (2N x 2N) row-major with
// rows = output real column, columns = input real index (K-major B operand).
__global__ void k_tc_prep_b(const double2* __restrict__ U, int64_t N, __half* __restrict__ out) {
  const int64_t N2 = 2 * N, sz = N2 * N2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < sz; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t nr = e / N2, kr = e - nr * N2;
    const int64_t n = nr >> 1, m = kr >> 1;
    const int s = (int)(nr & 1), t = (int)(kr & 1);
    const double2 uf = U[n * N + m];
    const double2 ua = U[m * N + n];
    const double ar = ua.x, ai = -ua.y;  // (U^dagger)[n][m] = conj(U[m][n])
    const double vf = (s == 0 ? (t == 0 ? uf.x : -uf.y) : (t == 0 ? uf.y : uf.x)) * (double)kOpScale;
    const double va = (s == 0 ? (t == 0 ? ar : -ai) : (t == 0 ? ai : ar)) * (double)kOpScale;
    const __half hf = __float2half_rn((float)vf), ha = __float2half_rn((float)va);
    out[e] = hf;
    out[sz + e] = __float2half_rn((float)(vf - (double)__half2float(hf)));
    out[2 * sz + e] = ha;
    out[3 * sz + e] = __float2half_rn((float)(va - (double)__half2float(ha)));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

hhl_status make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (fn == nullptr) return fail(HHL_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * sizeof(__half)};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(HHL_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return HHL_OK;
}

}  // namespace

bool tc_supported(const Plan& p) {
  if (p.prec != HHL_PREC_C64 || p.expm_mode != HHL_EXPM_DENSE) return false;
  if (p.N < 128 || p.R / 2 < kBM) return false;  // at least one full 128 x 256 tile
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

hhl_status tc_prepare_operands(Plan& p, const double2* d_u, int k, cudaStream_t st) {
  TcState* t = static_cast<TcState*>(p.d_tc);
  const int64_t N2 = 2 * p.N;
  const size_t mat = (size_t)N2 * N2;
  if (t == nullptr) {
    t = new TcState();
    p.d_tc = t;
    const size_t abytes = (size_t)(p.R / 2) * N2 * sizeof(__half);
    if (cudaMalloc(&t->a_hi, abytes) != cudaSuccess || cudaMalloc(&t->a_lo, abytes) != cudaSuccess ||
        cudaMalloc(&t->b, (size_t)p.n_c * 4 * mat * sizeof(__half)) != cudaSuccess ||
        cudaMalloc(&t->err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(HHL_ERR_OOM, "tcgen05 operand allocation failed");
    }
    hhl_status ws = tc_work_alloc(t->work, &p.workspace_bytes);
    if (ws != HHL_OK) return ws;
    p.workspace_bytes += 2 * abytes;
    p.table_bytes += (size_t)p.n_c * 4 * mat * sizeof(__half);
    HHL_CUDA_TRY(cudaMemsetAsync(t->err, 0, sizeof(int), st));
    // tile width: 256 unless HHL_TC_BN=128 (tuning) or the operand is narrower
    if (const char* env = getenv("HHL_TC_BN")) t->bn = atoi(env) == 128 ? 128 : 256;
    if (N2 < t->bn) t->bn = 128;
    t->maps.resize(2 + 4 * (size_t)p.n_c);
    hhl_status s = make_map(&t->maps[0], t->a_hi, N2, p.R / 2, kBM);
    if (s == HHL_OK) s = make_map(&t->maps[1], t->a_lo, N2, p.R / 2, kBM);
    for (int kk = 0; kk < p.n_c && s == HHL_OK; ++kk)
      for (int j = 0; j < 4 && s == HHL_OK; ++j)
        s = make_map(&t->maps[2 + 4 * kk + j], t->b + ((size_t)kk * 4 + j) * mat, N2, N2, t->bn);
    t->smaps.resize(4 * (size_t)p.n_c);
    for (int kk = 0; kk < p.n_c && s == HHL_OK; ++kk)
      for (int j = 0; j < 4 && s == HHL_OK; ++j)
        s = make_map(&t->smaps[4 * kk + j], t->b + ((size_t)kk * 4 + j) * mat, N2, N2, t->bn / 4);
    if (s != HHL_OK) return s;
    s = tc_init_kernels();
    if (s != HHL_OK) return s;
  }
  int g = (int)((mat + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  HHL_PROF_BEGIN(st);
  k_tc_prep_b<<<g, 256, 0, st>>>(d_u, p.N, t->b + (size_t)k * 4 * mat);
  HHL_LAUNCH_CHECK("k_tc_prep_b");
  return HHL_OK;
}

hhl_status launch_ctrl_u_tc(const Plan& p, void* half, int k, bool adjoint, cudaStream_t st) {
  return launch_ctrl_u_tc_map(p, half, circuit_rows(k), p.R / 2, k, adjoint, st);
}

hhl_status launch_ctrl_u_tc_map(const Plan& p, void* half, const RowMap& rows, int64_t m_sub, int k, bool adjoint,
                                cudaStream_t st) {
  const TcState* t = static_cast<const TcState*>(p.d_tc);
  if (t == nullptr) return fail(HHL_ERR_INVALID_ARG, "tcgen05 operands not prepared");
  const CUtensorMap* mb = &t->maps[2 + 4 * (size_t)k + (adjoint ? 2 : 0)];
  const CUtensorMap* ms = &t->smaps[4 * (size_t)k + (adjoint ? 2 : 0)];
  return launch_tc_gemm_map(p.n_s, m_sub, rows, half, t->a_hi, t->a_lo, t->maps[0], t->maps[1], mb[0], mb[1], t->bn,
                            t->err, t->work, 1, st, ms);
}

int tc_num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 152;
    return v > 0 ? v : 152;
  }();
  return n;
}

hhl_status tc_work_alloc(TcWork& w, size_t* bytes) {
  w.grid_cap = tc_num_sms();
  const size_t wsb = (size_t)2 * w.grid_cap * kBM * kBN * sizeof(float);  // two partial tiles per CTA
  if (cudaMalloc(&w.ws, wsb) != cudaSuccess) {
    cudaGetLastError();
    return fail(HHL_ERR_OOM, "tcgen05 stream-K workspace allocation failed");
  }
  if (bytes) *bytes += wsb;
  return HHL_OK;
}

void tc_work_free(TcWork& w) {
  if (w.ws) cudaFree(w.ws);
  w.ws = nullptr;
}

hhl_status launch_tc_gemm_map(int n_s, int64_t m_sub, const RowMap& k, void* half, void* a_hi, void* a_lo,
                              const CUtensorMap& map_ahi, const CUtensorMap& map_alo, const CUtensorMap& map_bhi,
                              const CUtensorMap& map_blo, int bn, int* err, const TcWork& w, int streamk,
                              cudaStream_t st, const CUtensorMap* slice4) {
  const int64_t N2 = 2LL << n_s;
  if (m_sub < kBM || m_sub % kBM != 0) return fail(HHL_ERR_INVALID_ARG, "tcgen05 GEMM rows must be a multiple of 128");
  if (bn != 128 && bn != 256) return fail(HHL_ERR_INVALID_ARG, "tcgen05 tile width must be 128 or 256");
  const int64_t tiles_n = N2 / bn, tiles = (m_sub / kBM) * tiles_n;
  if (streamk && w.ws == nullptr) return fail(HHL_ERR_INVALID_ARG, "tcgen05 stream-K workspace missing");
  // HHL_FAULT=tc_wait (testing the timeout path): no operand copy is issued and every wait is
  // bounded by about a millisecond, so the MMA lane's first wait runs out with nothing in flight
  const char* fenv = getenv("HHL_FAULT");
  const int fault = (fenv != nullptr && strcmp(fenv, "tc_wait") == 0) ? 1 : 0;
  const long long wait_cycles = fault ? kFaultWaitCycles : kWaitCycles;
  const int64_t total4 = m_sub * N2 / 4;
  int g = (int)((total4 + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  HHL_PROF_BEGIN(st);
  k_tc_split_rows<<<g, 256, 0, st>>>((const float4*)half, (uint2*)a_hi, (uint2*)a_lo, n_s, k, m_sub, err);
  HHL_LAUNCH_CHECK("k_tc_split_rows");
  // grid: one CTA per tile when the tiles fill at least three quarters of the SMs (or the
  // caller asks for it: the batch, whose streams fill the GPU together); otherwise stream-K,
  // one CTA per SM, fewer when a CTA would get under a quarter of a tile
  const int k_iters = (int)(N2 / kBK);
  const int64_t units = tiles * k_iters;
  int64_t G = tiles;
  if (streamk && 4 * tiles < 3 * (int64_t)w.grid_cap) {
    const int64_t min_units = k_iters >= 4 ? k_iters / 4 : 1;
    G = units / min_units;
    if (G < 1) G = 1;
    if (G > w.grid_cap) G = w.grid_cap;
  }
  // one CTA per tile with quarter-height B maps: clusters of 4 consecutive row tiles share the
  // B operand (HHL_TC_CLUSTER=1 turns the sharing off)
  static const int cl_env = [] {
    const char* e = getenv("HHL_TC_CLUSTER");
    return e != nullptr ? atoi(e) : 4;
  }();
  const int64_t tiles_m = m_sub / kBM;
  const int cl = (G == tiles && slice4 != nullptr && cl_env == 4 && tiles_m % 4 == 0) ? 4 : 1;
  HHL_PROF_BEGIN(st);
  if (cl == 4) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G);
    cfg.blockDim = dim3(kThreadsTc);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 4;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    float* sh = (float*)half;
    float* wsp = w.ws;
    const int ti = (int)tiles_n;
    cudaError_t e;
    if (bn == 256) {
      cfg.dynamicSmemBytes = TcShape<256>::kSmemBytes;
      e = cudaLaunchKernelEx(&cfg, k_ctrl_gemm_tc<256, 4>, map_ahi, map_alo, slice4[0], slice4[1], sh, n_s, k, k_iters,
                             ti, units, wsp, err, wait_cycles, fault);
    } else {
      cfg.dynamicSmemBytes = TcShape<128>::kSmemBytes;
      e = cudaLaunchKernelEx(&cfg, k_ctrl_gemm_tc<128, 4>, map_ahi, map_alo, slice4[0], slice4[1], sh, n_s, k, k_iters,
                             ti, units, wsp, err, wait_cycles, fault);
    }
    if (e != cudaSuccess) return cuda_fail(e, "k_ctrl_gemm_tc (cluster launch)");
  } else if (bn == 256) {
    k_ctrl_gemm_tc<256, 1><<<(unsigned)G, kThreadsTc, TcShape<256>::kSmemBytes, st>>>(
        map_ahi, map_alo, map_bhi, map_blo, (float*)half, n_s, k, k_iters, (int)tiles_n, units, w.ws, err,
        wait_cycles, fault);
  } else {
    k_ctrl_gemm_tc<128, 1><<<(unsigned)G, kThreadsTc, TcShape<128>::kSmemBytes, st>>>(
        map_ahi, map_alo, map_bhi, map_blo, (float*)half, n_s, k, k_iters, (int)tiles_n, units, w.ws, err,
        wait_cycles, fault);
  }
  HHL_LAUNCH_CHECK("k_ctrl_gemm_tc");
  // the split tiles, if any (a range boundary inside a tile): partials added in CTA order
  bool split = false;
  for (int64_t b = 1; b < G && !split; ++b) split = (b * units / G) % k_iters != 0;
  if (!split) return HHL_OK;
  const dim3 fgrid((unsigned)(kBM * (bn / 4) / 256), (unsigned)tiles);
  HHL_PROF_BEGIN(st);
  if (bn == 256)
    k_tc_fixup<256><<<fgrid, 256, 0, st>>>((const float4*)w.ws, (float*)half, n_s, k, k_iters, (int)tiles_n, units, G,
                                           err);
  else
    k_tc_fixup<128><<<fgrid, 256, 0, st>>>((const float4*)w.ws, (float*)half, n_s, k, k_iters, (int)tiles_n, units, G,
                                           err);
  HHL_LAUNCH_CHECK("k_tc_fixup");
  return HHL_OK;
}

hhl_status tc_init_kernels() {
  HHL_CUDA_TRY(cudaFuncSetAttribute(k_ctrl_gemm_tc<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcShape<256>::kSmemBytes));
  HHL_CUDA_TRY(cudaFuncSetAttribute(k_ctrl_gemm_tc<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcShape<128>::kSmemBytes));
  HHL_CUDA_TRY(cudaFuncSetAttribute(k_ctrl_gemm_tc<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcShape<256>::kSmemBytes));
  HHL_CUDA_TRY(cudaFuncSetAttribute(k_ctrl_gemm_tc<128, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    TcShape<128>::kSmemBytes));
  return HHL_OK;
}

hhl_status tc_make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  return make_map(map, base, cols, rows, box_rows);
}

int* tc_error_flag(const Plan& p) {
  const TcState* t = static_cast<const TcState*>(p.d_tc);
  return t ? t->err : nullptr;
}

hhl_status tc_flag_status(int flag) {
  if (flag == 0) return HHL_OK;
  if (flag == 4) return fail(HHL_ERR_NUMERIC, "an amplitude of magnitude >= 2 reached the FP16 tensor-core operands");
  static const char* const where[] = {"", "producer (free stage)", "MMA issuer (operands)", "epilogue (accumulator)", "",
                                      "producer (copies in flight)"};
  return fail(HHL_ERR_TIMEOUT, std::string("a bounded wait in the tcgen05 GEMM ran out: ") +
                                   (flag > 0 && flag <= 5 ? where[flag] : "unknown"));
}

hhl_status tc_reset_error(const Plan& p, cudaStream_t st) {
  const TcState* t = static_cast<const TcState*>(p.d_tc);
  if (t == nullptr || t->err == nullptr) return HHL_OK;
  HHL_CUDA_TRY(cudaMemsetAsync(t->err, 0, sizeof(int), st));
  return HHL_OK;
}

void tc_free(Plan& p) {
  TcState* t = static_cast<TcState*>(p.d_tc);
  if (t == nullptr) return;
  if (t->a_hi) cudaFree(t->a_hi);
  if (t->a_lo) cudaFree(t->a_lo);
  if (t->b) cudaFree(t->b);
  if (t->err) cudaFree(t->err);
  tc_work_free(t->work);
  delete t;
  p.d_tc = nullptr;
}

}  // namespace hhl
