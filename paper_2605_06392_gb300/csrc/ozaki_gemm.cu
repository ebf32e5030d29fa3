// FP64 GEMM emulated on BF16 tensor cores by error-free operand splitting
// (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012; the fixed-point slice form
// follows Mukunoki, Ozaki, Ogita and Imamura, "DGEMM using Tensor Cores,
// and its accurate and reproducible versions", ISC 2020):
//
//   C = alpha op(A) op(B) + beta C,   FP64 in and out.
//
// Splitting.  Row i of op(A) is scaled by a power of two 2^(e_i) with
// |a_ik| < 2^(e_i + 7) and written in S signed base-128 digits:
//     a_ik = 2^(e_i) * sum_j d_j(a_ik) * 2^(-7(j-1)),   |d_1| <= 128, |d_j| <= 64,
// each digit rounded to nearest from the fixed-point value of a_ik with
// 7S fractional bits (S = 8: 56 bits, one more than the 53 of an FP64
// significand).  Column n of op(B) likewise with 2^(f_n).  Every digit
// times its power of two is exact in BF16 (<= 8 significant bits), so each
// slice A_j, B_l is a BF16 matrix and each slice product A_j B_l is exact
// in its terms.
//
// Products.  C = 2^(e_i + f_n) sum over pairs (j, l) with j + l <= S + 1 of
// A_j B_l (the pairs beyond are below the 7S-bit truncation).  The pairs
// of one level L = j + l share the scale 2^(-7(L-2)), so their sum over
// k is an integer multiple of it; with the digit bounds above it stays
// within 2^24 units over 512 consecutive k for L <= 7, so an FP32
// accumulator holds it exactly.  Levels 2..7 therefore run on tcgen05
// (kind::f16, BF16 operands, FP32 accumulator in tensor memory) into one
// accumulator per level, drained into 64-bit integers every 512 of K;
// levels 8..S+1 (relative weight <= 2^-42) share one FP32 accumulator over
// the whole K, whose rounding (2^-24 of it) stays far below the FP64 unit.
// The FP64 result is assembled from the integer sum and that accumulator
// with integer operations (GB300's FP64 pipe runs more than 1000x slower than
// its BF16 tensor cores, so the epilogue avoids it except for the beta C add).
//
// Kernel: one 128 x 64 output tile per CTA (1 CTA per SM), 192 threads.
//   * warp 4 streams 32-wide K slabs of the S A-slices and S B-slices into a
//     2-stage shared-memory ring with TMA (64-byte swizzle);
//   * warp 5 issues the S(S+1)/2 slice-pair MMAs (M=128, N=64, K=16) per 16
//     of K into the seven TMEM accumulators (7 x 64 columns), from lane 0
//     of the converged warp;
//   * warps 0-3 drain the exact accumulators (one TMEM lane quarter each)
//     every 512 of K and write the tile.
// Every mbarrier wait is bounded: on expiry the kernel records
// BTA_ERR_TIMEOUT in the status word, stops issuing work, waits (bounded)
// for the loads and MMAs it issued and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>

#include "common.cuh"
#include "ozaki_digits.cuh"
#include "tma.cuh"

// Timeline hooks of ozaki_gemm128_kernel (producer, MMA issuer, drain):
// empty in the library; a measurement harness that includes this file may
// define OZ_TRACE(event, value) before the include to record them.
#ifndef OZ_TRACE
#define OZ_TRACE(event, value) ((void)0)
#endif

namespace bta {
namespace {
using oz::compose;
using oz::digits;

using namespace tc;

constexpr int OM = 128;                 // tile rows = TMEM lanes
constexpr int OBN = 64;                 // tile columns
constexpr int OK16 = 32;                // bf16 per K slab: 64-byte rows
constexpr int kOzStages = 2;
constexpr int kChunkSlabs = 16;         // exact accumulators drained every 512 of K
constexpr int kOzThreads = 192;   // warps 0-3 drain, 4 loads, 5 issues MMAs
constexpr int kMaxOzK = kOzakiMaxK;
constexpr long long kOzWaitLimit = 1ll << 21;
constexpr int kATile = OM * OK16 * 2;   // 8 KB
constexpr int kBTile = OBN * OK16 * 2;  // 4 KB

template <int S>
struct OzCfg {
  static_assert(S >= 6 && S <= 8, "levels 2..7 exact, 8..S+1 in one rounded accumulator");
  static constexpr bool kRounded = S >= 7;   // some pair has level >= 8
  static constexpr int kStage = S * (kATile + kBTile);
  static constexpr int kSmem = kOzStages * kStage + 1024 + 512;
  static constexpr uint32_t kTmemCols = 512;
  // kind::f16: FP32 accumulator, A and B BF16, both K-major, N = 64, M = 128
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     ((uint32_t)(OBN >> 3) << 17) | ((uint32_t)(OM >> 4) << 24);
};

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, 8-row
// groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                     // leading-dimension offset (unused)
  d |= (uint64_t)(512 >> 4) << 32;            // stride between 8-row groups
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)4 << 61;                     // 64-byte swizzle
  return d;
}

// The MMA of slice pair (J, LL) (0-based digits of A and B, level
// L = J + LL + 2) for the 16-wide K step KK of the stage whose descriptor
// base is dst; issued by one lane (leader != 0) of a converged warp.  The
// operand offsets are immediates, so no descriptor lives in a register.
// The first MMA of a level in a slab overwrites its accumulator when the
// slab opens a 512-wide K chunk (exact levels) or the whole K range (the
// rounded accumulator of levels >= 8).
template <int S, int J, int LL, int KK>
__device__ __forceinline__ void issue_pair(uint32_t tmem, uint64_t dst, uint32_t chunk_first,
                                           uint32_t kernel_first, uint32_t leader) {
  constexpr int L = J + LL + 2;
  constexpr int kAccIdx = L <= 7 ? L - 2 : 6;
  constexpr bool kFirstInSlab = KK == 0 && J == 0 && L <= 8;
  const uint32_t accumulate =
      kFirstInSlab ? ((L <= 7 ? chunk_first : kernel_first) ? 0u : 1u) : 1u;
  constexpr unsigned long long kAo = (unsigned long long)(J * kATile + KK * 32) >> 4;
  constexpr unsigned long long kBo =
      (unsigned long long)(S * kATile + LL * kBTile + KK * 32) >> 4;
  asm volatile(
      "{\n .reg .b64 da, db;\n .reg .pred p, e;\n"
      " add.s64 da, %1, %2;\n add.s64 db, %1, %3;\n"
      " setp.ne.b32 p, %5, 0;\n setp.ne.b32 e, %6, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n" ::"r"(
          tmem + (uint32_t)(kAccIdx * OBN)),
      "l"(dst), "n"(kAo), "n"(kBo), "r"(OzCfg<S>::kIdesc), "r"(accumulate), "r"(leader)
      : "memory");
}

template <int S, int J, int LL, int KK>
__device__ __forceinline__ void issue_row(uint32_t tmem, uint64_t dst, uint32_t cf, uint32_t kf,
                                          uint32_t leader) {
  if constexpr (J + LL < S) {
    issue_pair<S, J, LL, KK>(tmem, dst, cf, kf, leader);
    issue_row<S, J, LL + 1, KK>(tmem, dst, cf, kf, leader);
  }
}

template <int S, int J, int KK>
__device__ __forceinline__ void issue_step(uint32_t tmem, uint64_t dst, uint32_t cf, uint32_t kf,
                                           uint32_t leader) {
  if constexpr (J < S) {
    issue_row<S, J, 0, KK>(tmem, dst, cf, kf, leader);
    issue_step<S, J + 1, KK>(tmem, dst, cf, kf, leader);
  }
}

__device__ __forceinline__ void mma_commit_if(uint32_t mbar, uint32_t leader) {
  asm volatile(
      "{\n .reg .pred e;\n setp.ne.b32 e, %1, 0;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
          mbar),
      "r"(leader)
      : "memory");
}

// Bounded wait by lane 0, result broadcast: a warp-uniform decision.
__device__ __forceinline__ bool warp_wait(uint32_t addr, uint32_t parity, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait(addr, parity, kOzWaitLimit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// A shared flag read by lane 0 and broadcast.
__device__ __forceinline__ bool warp_flag(const int* f, int lane) {
  int v = 0;
  if (lane == 0) v = *(const volatile int*)f;
  return __shfl_sync(0xffffffffu, v, 0) != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// OR of v over the 128 threads of warps 0-3 (named barrier 1).
__device__ __forceinline__ int bar_or_128(int v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n"
      " barrier.cta.red.or.pred q, 1, 128, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v)
      : "memory");
  return r;
}

// alpha and beta as integer modes (decided on the host: comparisons of
// doubles would run on the FP64 pipe once per element): alpha 0 -> +1,
// 1 -> -1, 2 -> general; beta 0 -> 0, 1 -> +1, 2 -> general.
inline int alpha_mode(double a) { return a == 1.0 ? 0 : a == -1.0 ? 1 : 2; }
inline int beta_mode(double b) { return b == 0.0 ? 0 : b == 1.0 ? 1 : 2; }

__device__ __forceinline__ double scale_add(double out, int am, double alpha, int bm, double beta,
                                            const double* cin) {
  if (am == 1) out = -out;
  else if (am == 2) out *= alpha;
  if (bm == 1) out += *cin;
  else if (bm == 2) out = fma(beta, *cin, out);
  return out;
}

struct OzArgs {
  int M, N, Kp, Mp, Np;
  double alpha, beta;
  int amode, bmode;
  double* C;
  int ldc;
  const double* Cin;
  int ldcin;
  int out_lower;
  const int* exA;   // [Mp] biased exponent bound of each row of op(A)
  const int* exB;   // [Np] biased exponent bound of each column of op(B)
  long long* partial;   // [Np][Mp] integer sums between K chunks (K > 512 only)
  int32_t* status;
};

// At most 248 registers a thread: with a task-graph factor CTA of the other
// sweep (256 threads x 68 registers, ~26 KB) the CTA still fits on one SM
// (64 K registers, 228 KB), so the two overlap on the FP64 and tensor pipes.
template <int S>
__global__ void __maxnreg__(248)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap mA,
                      const __grid_constant__ CUtensorMap mB, OzArgs g) {
  using Cfg = OzCfg<S>;
  const int m0 = blockIdx.x * OM, n0 = blockIdx.y * OBN;
  if (g.out_lower && n0 > m0 + OM - 1) return;   // whole CTA exits before any set-up
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOzStages * Cfg::kStage);
  // bars: full[stages], empty[stages], accumulators full, accumulators drained, final
  const int kFull = 0, kEmpty = kOzStages, kAccFull = 2 * kOzStages,
            kAccEmpty = 2 * kOzStages + 1, kFinal = 2 * kOzStages + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kOzStages + 3);
  int* s_exB = reinterpret_cast<int*>(tmem_slot + 4);   // [OBN]
  __shared__ int s_abort, s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = g.Kp / OK16;
  const int nchunks = (nk + kChunkSlabs - 1) / kChunkSlabs;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(smem_u32(&bars[kFull + s]), 1);
      mbar_init(smem_u32(&bars[kEmpty + s]), 1);
    }
    mbar_init(smem_u32(&bars[kAccFull]), 1);
    mbar_init(smem_u32(&bars[kAccEmpty]), 128);
    mbar_init(smem_u32(&bars[kFinal]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  for (int i = threadIdx.x; i < OBN; i += kOzThreads) s_exB[i] = g.exB[n0 + i];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---- TMA producer: slab kt of every slice into stage kt % stages
    const uint32_t leader = lane == 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % kOzStages;
      if (kt >= kOzStages &&
          !warp_wait(smem_u32(&bars[kEmpty + s]), (uint32_t)((kt / kOzStages - 1) & 1), lane)) {
        if (leader) atomicExch(&s_abort, 1);
        break;
      }
      if (warp_flag(&s_abort, lane)) break;
      if (leader) {
        const uint32_t full = smem_u32(&bars[kFull + s]);
        mbar_expect_tx(full, Cfg::kStage);
        uint8_t* st = smem + s * Cfg::kStage;
        const int k0 = kt * OK16;
#pragma unroll
        for (int j = 0; j < S; ++j) {
          tma_load_2d(smem_u32(st + j * kATile), &mA, full, k0, j * g.Mp + m0);
          tma_load_2d(smem_u32(st + S * kATile + j * kBTile), &mB, full, k0, j * g.Np + n0);
        }
        *(volatile int*)&s_issued = kt + 1;
      }
      __syncwarp();
    }
  } else if (warp == 5) {
    // ---- MMA issuer: the whole warp runs the loop, lane 0 issues
    const uint32_t leader = lane == 0;
    const uint64_t dbase = sdesc64(smem_u32(smem));   // + (byte offset >> 4) per operand tile
    bool stop = false;
    for (int c = 0; c < nchunks && !stop; ++c) {
      if (c > 0 && !warp_wait(smem_u32(&bars[kAccEmpty]), (uint32_t)((c - 1) & 1), lane)) {
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int kt1 = min(nk, (c + 1) * kChunkSlabs);
      for (int kt = c * kChunkSlabs; kt < kt1; ++kt) {
        const int s = kt % kOzStages;
        if (warp_flag(&s_abort, lane) ||
            !warp_wait(smem_u32(&bars[kFull + s]), (uint32_t)((kt / kOzStages) & 1), lane)) {
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t dst = dbase + (uint64_t)((s * Cfg::kStage) >> 4);
        const uint32_t cf = kt == c * kChunkSlabs, kf = kt == 0;
        issue_step<S, 0, 0>(tmem, dst, cf, kf, leader);   // 16 bf16 = 32 bytes along K
        issue_step<S, 0, 1>(tmem, dst, cf, kf, leader);
        mma_commit_if(smem_u32(&bars[kEmpty + s]), leader);   // slab free once these finish
        if (leader) *(volatile int*)&s_consumed = kt + 1;
        __syncwarp();
      }
      mma_commit_if(smem_u32(&bars[kAccFull]), leader);        // this chunk's sums ready
    }
    if (stop) {
      if (leader) atomicExch(&s_abort, 1);
      // wait (bounded) for the MMAs this warp issued before leaving
      mma_commit_if(smem_u32(&bars[kFinal]), leader);
      warp_wait(smem_u32(&bars[kFinal]), 0, lane);
    }
  } else {
    // ---- warps 0-3: drain the exact accumulators every 512 of K into 64-bit
    // integer sums (kept in a workspace between chunks), and after the last
    // chunk assemble and store the tile.  Thread = output row, 32 columns at
    // a time.
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const int m = m0 + warp * 32 + lane;
    const int ea = g.exA[m];   // exA has Mp entries
    int failed = 0;
    for (int c = 0; c < nchunks; ++c) {
      const bool ok = mbar_wait(smem_u32(&bars[kAccFull]), (uint32_t)(c & 1), kOzWaitLimit);
      if (bar_or_128(!ok || *(volatile int*)&s_abort)) {
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const bool last = c == nchunks - 1;
#pragma unroll 1
      for (int cc = 0; cc < OBN / 32; ++cc) {
        long long* part = g.partial + m + (int64_t)(n0 + cc * 32) * g.Mp;
        long long acc[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = c > 0 ? part[(int64_t)q * g.Mp] : 0ll;
        // levels 2..7 in units of level 7 (2^-35)
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const float up = __int_as_float((127 + 7 * a) << 23);   // level a+2 in integer units
          const long long sc = 1ll << (7 * (5 - a));
          float v[32];
          tmem_ld32(tmem + lane_off + (uint32_t)(a * OBN + cc * 32), v);
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[q] += (long long)__float2int_rn(v[q] * up) * sc;
        }
        if (!last) {
#pragma unroll
          for (int q = 0; q < 32; ++q) part[(int64_t)q * g.Mp] = acc[q];
          continue;
        }
        // the rounded accumulator, assemble, alpha / beta, store
        float v[32];
        if (Cfg::kRounded) {
          tmem_ld32(tmem + lane_off + (uint32_t)(6 * OBN + cc * 32), v);
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = 0.f;
        }
        if (m < g.M) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int n = n0 + cc * 32 + q;
            if (n >= g.N || (g.out_lower && m < n)) continue;
            // sum = (acc + v 2^35) 2^-35
            const long long X = acc[q] + __float2ll_rn(v[q] * 34359738368.0f);
            // a = 2^(exA - 1029) sum_j A_j, b likewise: C = X 2^(exA + exB - 2058 - 35)
            double out = compose(X, ea + s_exB[cc * 32 + q] - 2093);
            out = scale_add(out, g.amode, g.alpha, g.bmode, g.beta,
                            g.Cin + m + (int64_t)n * g.ldcin);
            g.C[m + (int64_t)n * g.ldc] = out;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bars[kAccEmpty]));
    }
    if (failed && threadIdx.x == 0) atomicExch(&s_abort, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && s_abort) {
    // loads issued but never consumed: wait (bounded) for them to land
    for (int kt = s_consumed; kt < s_issued; ++kt)
      mbar_wait(smem_u32(&bars[kFull + kt % kOzStages]), (uint32_t)((kt / kOzStages) & 1),
                kOzWaitLimit);
    if (g.status) atomicExch(g.status, (int)BTA_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cfg::kTmemCols)
                 : "memory");
  }
}

// ---- 128 x 128 tiles (S = 8) ----------------------------------------------------
//
// The same products with N = 128 MMAs, which take as long as N = 64 ones: a
// 128 x 128 tile per CTA doubles the work per MMA.  Tensor memory (512
// columns) then holds four 128-column accumulators, not seven, so every
// 512-wide K chunk runs four sub-passes over its 16 slabs, each streaming
// four A and four B slices (64 KB a slab, a 3-stage ring):
//   P0  levels 2..5   A1..4 x B1..4, j + l <= 5      4 exact accumulators
//   P1  levels 6..9   A1..4 x B5..8                  levels 6, 7 exact + rounded
//   P2  levels 6..8   A1..4 x B1..4, 6 <= j + l <= 8 (the same three)
//   P3  levels 6..9   A5..8 x B1..4                  (the same three)
// (10 + 10 + 6 + 10 = 36 pairs).  The accumulators are drained after P0 and
// after P3 into the 64-bit integer sum of the tile, kept in the workspace;
// the rounded one is drained per chunk too (one rounding to 2^-35 of the
// level-2 unit per chunk).  K chunks may be split over several CTAs (grid
// z), each with its own integer sums; ozaki_compose_kernel adds them and
// assembles C.  576 threads: warps 0-15 drain (four per TMEM lane quarter,
// 32 columns each, the tile's 64-bit sums held in their registers across
// the chunks, so a drain is TMEM loads and integer adds only), warp 16
// loads, warp 17 issues MMAs.
constexpr int QN = 128;
constexpr int kQThreads = 576;
constexpr int kQDrain = 512;
constexpr int kQTile = 128 * OK16 * 2;    // one slice slab: 128 rows x 32 of K, 8 KB
constexpr int kQStage = 8 * kQTile;       // 4 A slots + 4 B slots: 64 KB
constexpr int kQStages = 3;
constexpr int kQPasses = 4;
constexpr int kQSmem = kQStages * kQStage + 1024 + 256;
constexpr uint32_t kQIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(QN >> 3) << 17) |
                             ((uint32_t)(OM >> 4) << 24);

// First A and B slice (0-based) a sub-pass streams.
__host__ __device__ constexpr int q_a0(int P) { return P == 3 ? 4 : 0; }
__host__ __device__ constexpr int q_b0(int P) { return P == 1 ? 4 : 0; }

// CTA-pair variant (ozaki_gemm_pair_kernel below): M = 256 over two CTAs,
// each holding 128 A rows and 64 of the 128 B columns (4 KB a B slot).
constexpr int kPM = 256;
constexpr int kPBRows = 64;
constexpr int kPBTile = kPBRows * OK16 * 2;       // 4 KB
constexpr int kPStage = 4 * kQTile + 4 * kPBTile;  // 48 KB
constexpr int kPStages = 4;
// ring, barriers, and 8 KB of slack past the ring: every operand read an MMA
// can make from a slot stays inside the allocation
constexpr int kPSmem = kPStages * kPStage + 1024 + 256 + 8192;
constexpr uint32_t kPIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(QN >> 3) << 17) |
                             ((uint32_t)(kPM >> 4) << 24);

// MMA of A slot I and B slot LL in sub-pass P for the 16-wide K step KK:
// one CTA (PAIR = false, M = 128) or a CTA pair (PAIR = true, M = 256, issued
// by the pair's leader; the descriptors name the same offsets in both CTAs).
template <bool PAIR, int P, int I, int LL, int KK>
__device__ __forceinline__ void q_pair(uint32_t tmem, uint64_t dst, uint32_t first,
                                       uint32_t leader) {
  constexpr int L = q_a0(P) + I + q_b0(P) + LL + 2;   // level
  constexpr bool kValid = P == 0 ? L <= 5 : (P == 2 ? (L >= 6 && L <= 8) : L <= 9);
  if constexpr (kValid) {
    constexpr int kAcc = P == 0 ? L - 2 : (L <= 7 ? L - 6 : 2);
    // P0 and P1 open their accumulator set (P1's levels 6, 7, 8 come first)
    constexpr bool kMayOpen = KK == 0 && I == 0 && (P == 0 || (P == 1 && L <= 8));
    const uint32_t accumulate = kMayOpen ? (first ? 0u : 1u) : 1u;
    constexpr unsigned long long kAo = (unsigned long long)(I * kQTile + KK * 32) >> 4;
    constexpr unsigned long long kBo =
        PAIR ? (unsigned long long)(4 * kQTile + LL * kPBTile + KK * 32) >> 4
             : (unsigned long long)((4 + LL) * kQTile + KK * 32) >> 4;
    if constexpr (PAIR) {
      asm volatile(
          "{\n .reg .b64 da, db;\n .reg .pred p, e;\n"
          " add.s64 da, %1, %2;\n add.s64 db, %1, %3;\n"
          " setp.ne.b32 p, %5, 0;\n setp.ne.b32 e, %6, 0;\n"
          " @e tcgen05.mma.cta_group::2.kind::f16 [%0], da, db, %4, p;\n}\n" ::"r"(
              tmem + (uint32_t)(kAcc * QN)),
          "l"(dst), "n"(kAo), "n"(kBo), "r"(kPIdesc), "r"(accumulate), "r"(leader)
          : "memory");
    } else {
      asm volatile(
          "{\n .reg .b64 da, db;\n .reg .pred p, e;\n"
          " add.s64 da, %1, %2;\n add.s64 db, %1, %3;\n"
          " setp.ne.b32 p, %5, 0;\n setp.ne.b32 e, %6, 0;\n"
          " @e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n" ::"r"(
              tmem + (uint32_t)(kAcc * QN)),
          "l"(dst), "n"(kAo), "n"(kBo), "r"(kQIdesc), "r"(accumulate), "r"(leader)
          : "memory");
    }
  }
}

// One slab of sub-pass P in level-major order: for each level, its pairs
// (A slot ascending) and both 16-wide K steps back to back, so consecutive
// MMAs accumulate into the same TMEM accumulator.  A level's first MMA is
// its pair with A slot 0 at K step 0 (present in every level of P0 and P1),
// which opens the accumulator in the first slab of a chunk.
template <bool PAIR, int P, int L, int I>
__device__ __forceinline__ void q_level(uint32_t tmem, uint64_t dst, uint32_t first,
                                        uint32_t leader) {
  if constexpr (I < 4) {
    constexpr int LL = L - 2 - q_a0(P) - q_b0(P) - I;
    if constexpr (LL >= 0 && LL < 4) {
      q_pair<PAIR, P, I, LL, 0>(tmem, dst, first, leader);
      q_pair<PAIR, P, I, LL, 1>(tmem, dst, first, leader);
    }
    q_level<PAIR, P, L, I + 1>(tmem, dst, first, leader);
  }
}

template <bool PAIR, int P, int L>
__device__ __forceinline__ void q_levels(uint32_t tmem, uint64_t dst, uint32_t first,
                                         uint32_t leader) {
  if constexpr (L <= 9) {
    q_level<PAIR, P, L, 0>(tmem, dst, first, leader);
    q_levels<PAIR, P, L + 1>(tmem, dst, first, leader);
  }
}

template <bool PAIR, int P>
__device__ __forceinline__ void q_slab(uint32_t tmem, uint64_t dst, uint32_t first,
                                       uint32_t leader) {
  q_levels<PAIR, P, 2>(tmem, dst, first, leader);
}

// OR of v over the 512 threads of warps 0-15 (named barrier 1).
__device__ __forceinline__ int bar_or_512(int v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n"
      " barrier.cta.red.or.pred q, 1, 512, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v)
      : "memory");
  return r;
}

struct OzqArgs {
  int Mp, Np, Bp, nk, splits;   // nk: 32-wide K slabs; Bp: rows per B slice in its array
  int group;                             // tile rows per group of the launch order
  int out_lower;
  int tri_a, tri_b;     // triangle of op(A) / op(B) (Tri): their zero K ranges are skipped
  int reverse;          // take the tiles in reverse launch order (longest K ranges first)
  long long* partial;   // [splits][Np][Mp] integer sums, units 2^-35 of level 2
  int32_t* status;
  // Compose in the epilogue (one split, one-CTA kernel): each drain thread
  // turns its row's integer sums into C itself, as ozaki_compose_kernel would
  // (same operations, same bits), instead of writing them to `partial`.
  int fuse;
  int M, N;             // rows / columns of C (the padding is not written)
  int amode, bmode;
  double alpha, beta;
  double* C;
  int ldc;
  const double* Cin;
  int ldcin;
  int c_rows;           // rows m >= c_rows go to C2 / Cin2 (INT_MAX: none)
  double* C2;
  int ldc2;
  const double* Cin2;
  int ldcin2;
  const int* exA;
  const int* exB;
};

// The 32-wide K slabs [kb, ke) of a tile with output rows m0 .. m0 + rows - 1
// and columns n0 .. n0 + cols - 1 on which op(A) and op(B) can be nonzero: a
// lower op(A) has a_mk = 0 for k > m, an upper one for k < m; a lower op(B)
// has b_kn = 0 for k < n, an upper one for k > n.  The slices hold exact zeros
// there (the split masks the triangles), so leaving those slabs out changes
// no level sum.  Split z of `splits` takes its share of [kb, ke).
__device__ __forceinline__ void tile_slabs(const OzqArgs& g, int m0, int rows, int n0, int cols,
                                           int z, int& ks0, int& ks1) {
  int kb = 0, ke = g.nk;
  if (g.tri_a == TRI_LOWER) ke = min(ke, (m0 + rows + OK16 - 1) / OK16);
  if (g.tri_a == TRI_UPPER) kb = max(kb, m0 / OK16);
  if (g.tri_b == TRI_LOWER) kb = max(kb, n0 / OK16);
  if (g.tri_b == TRI_UPPER) ke = min(ke, (n0 + cols + OK16 - 1) / OK16);
  if (ke < kb) ke = kb;
  ks0 = kb + (int)((int64_t)z * (ke - kb) / g.splits);
  ks1 = kb + (int)((int64_t)(z + 1) * (ke - kb) / g.splits);
}

// 8 columns at each of two TMEM addresses, one wait for both.
__device__ __forceinline__ void tmem_ld8x2(uint32_t a0, uint32_t a1, float (&v0)[8],
                                           float (&v1)[8]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
      " tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
      " tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(a0), "r"(a1)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v0[j] = __uint_as_float(r[j]);
    v1[j] = __uint_as_float(r[8 + j]);
  }
}

// 8 columns at each of three TMEM addresses, one wait for all three.
__device__ __forceinline__ void tmem_ld8x3(uint32_t a0, uint32_t a1, uint32_t a2, float (&v0)[8],
                                           float (&v1)[8], float (&v2)[8]) {
  uint32_t r[24];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n"
      " tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n"
      " tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n"
      " tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
      : "r"(a0), "r"(a1), "r"(a2)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    v0[j] = __uint_as_float(r[j]);
    v1[j] = __uint_as_float(r[8 + j]);
    v2[j] = __uint_as_float(r[16 + j]);
  }
}

// 18 warps: an SM sub-partition hosts five of them, so at most 96
// registers a thread (5 x 32 x 96 <= 16 K).
__global__ void __launch_bounds__(kQThreads, 1)
    ozaki_gemm128_kernel(const __grid_constant__ CUtensorMap mA,
                         const __grid_constant__ CUtensorMap mB, OzqArgs g) {
  // Tile order: groups of `group` tile rows, column by column inside a
  // group, so that the CTAs resident together share few A and B row blocks.
  const int mt_all = g.Mp / OM, nt_all = g.Np / QN;
  const int bx = g.reverse ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
  const int grp = bx / (g.group * nt_all);
  const int gm = min(g.group, mt_all - grp * g.group);
  const int in = bx - grp * g.group * nt_all;
  const int m0 = (grp * g.group + in % gm) * OM, n0 = (in / gm) * QN, z = blockIdx.z;
  if (g.out_lower && n0 > m0 + OM - 1) return;   // whole CTA exits before any set-up
  // this CTA's slabs of K: split z of `splits` near-equal ranges, taken in
  // chunks of at most 16 slabs (512 of K: the exactness limit of a level sum)
  int ks0, ks1;
  tile_slabs(g, m0, OM, n0, QN, z, ks0, ks1);
  const int nc = (ks1 - ks0 + kChunkSlabs - 1) / kChunkSlabs;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kQStages * kQStage);
  const int kFull = 0, kEmpty = kQStages, kAccFull = 2 * kQStages,
            kAccEmpty = 2 * kQStages + 1, kFinal = 2 * kQStages + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kQStages + 3);
  __shared__ int s_abort, s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kQStages; ++s) {
      mbar_init(smem_u32(&bars[kFull + s]), 1);
      mbar_init(smem_u32(&bars[kEmpty + s]), 1);
    }
    mbar_init(smem_u32(&bars[kAccFull]), 1);
    mbar_init(smem_u32(&bars[kAccEmpty]), kQDrain);
    mbar_init(smem_u32(&bars[kFinal]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 16) {
    // ---- TMA producer: for each chunk and sub-pass, the chunk's slabs of the
    // sub-pass's slices; ring position r = running slab count.  Lane 0 alone
    // runs the loop (no warp-wide step between slabs).
    if (lane == 0) {
      int r = 0;
      bool stop = false;
      for (int c = 0; c < nc && !stop; ++c) {
        const int kt0 = ks0 + c * kChunkSlabs, kt1 = min(ks1, kt0 + kChunkSlabs);
        for (int P = 0; P < kQPasses && !stop; ++P) {
          const int aj0 = q_a0(P), bl0 = q_b0(P);
          for (int kt = kt0; kt < kt1; ++kt, ++r) {
            const int s = r % kQStages;
            if (r >= kQStages && !mbar_wait(smem_u32(&bars[kEmpty + s]),
                                            (uint32_t)((r / kQStages - 1) & 1), kOzWaitLimit)) {
              atomicExch(&s_abort, 1);
              stop = true;
              break;
            }
            if (*(volatile int*)&s_abort) {
              stop = true;
              break;
            }
            OZ_TRACE(1, r);                                   // slab r's loads issued
            const uint32_t full = smem_u32(&bars[kFull + s]);
            mbar_expect_tx(full, (uint32_t)kQStage);
            uint8_t* st = smem + s * kQStage;
            const int k0 = kt * OK16;
            for (int i = 0; i < 4; ++i)
              tma_load_2d(smem_u32(st + i * kQTile), &mA, full, k0, (aj0 + i) * g.Mp + m0);
            for (int l = 0; l < 4; ++l)
              tma_load_2d(smem_u32(st + (4 + l) * kQTile), &mB, full, k0, (bl0 + l) * g.Bp + n0);
            *(volatile int*)&s_issued = r + 1;
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 17) {
    // ---- MMA issuer: lane 0 alone runs the loop and issues every MMA, with
    // no warp-wide step between slabs (each would leave the tensor pipe idle
    // while the next slab's MMAs wait behind it)
    if (lane == 0) {
      const uint64_t dbase = sdesc64(smem_u32(smem));
      bool stop = false;
      int r = 0, e = 0;   // slabs consumed, accumulator sets handed to the drain
      for (int c = 0; c < nc && !stop; ++c) {
        const int kt0 = ks0 + c * kChunkSlabs, kt1 = min(ks1, kt0 + kChunkSlabs);
        for (int P = 0; P < kQPasses && !stop; ++P) {
          // P0 and P1 open an accumulator set: wait until the previous one is drained
          OZ_TRACE(2, 4 * c + P);                            // sub-pass P wants its set
          if (P <= 1 && e > 0 &&
              !mbar_wait(smem_u32(&bars[kAccEmpty]), (uint32_t)((e - 1) & 1), kOzWaitLimit)) {
            stop = true;
            break;
          }
          OZ_TRACE(3, 4 * c + P);                            // ... and starts
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int kt = kt0; kt < kt1; ++kt, ++r) {
            const int s = r % kQStages;
            // a producer that gave up issues nothing more, so this wait runs out
            if (!mbar_wait(smem_u32(&bars[kFull + s]), (uint32_t)((r / kQStages) & 1),
                           kOzWaitLimit)) {
              stop = true;
              break;
            }
            OZ_TRACE(4, r);                                  // slab r in place: MMAs go
            // (no tcgen05 fence here: the slab arrives by TMA, whose mbarrier
            // completion already orders it before the MMAs that read it)
            const uint64_t dst = dbase + (uint64_t)((s * kQStage) >> 4);
            const uint32_t first = kt == kt0;
            if (P == 0) q_slab<false, 0>(tmem, dst, first, 1u);
            else if (P == 1) q_slab<false, 1>(tmem, dst, first, 1u);
            else if (P == 2) q_slab<false, 2>(tmem, dst, first, 1u);
            else q_slab<false, 3>(tmem, dst, first, 1u);
            mma_commit_if(smem_u32(&bars[kEmpty + s]), 1u);   // slab free once these finish
            *(volatile int*)&s_consumed = r + 1;
          }
          if (!stop && (P == 0 || P == kQPasses - 1)) {
            mma_commit_if(smem_u32(&bars[kAccFull]), 1u);     // this set's sums ready
            ++e;
          }
        }
      }
      if (stop) {
        atomicExch(&s_abort, 1);
        mma_commit_if(smem_u32(&bars[kFinal]), 1u);
        mbar_wait(smem_u32(&bars[kFinal]), 0, kOzWaitLimit);
      }
    }
    __syncwarp();
  } else {
    // ---- warps 0-15: thread = output row (TMEM lane) x 32 columns; the
    // tile's integer sums (units 2^-35 of the level-2 unit) stay in registers
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const int row = (warp & 3) * 32 + lane, col0 = (warp >> 2) * 32;
    long long acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0ll;
    int failed = 0, e = 0;
    for (int c = 0; c < nc && !failed; ++c) {
      for (int set = 0; set < 2; ++set, ++e) {
        const bool ok = mbar_wait(smem_u32(&bars[kAccFull]), (uint32_t)(e & 1), kOzWaitLimit);
        if (bar_or_512(!ok || *(volatile int*)&s_abort)) {
          failed = 1;
          break;
        }
        if (threadIdx.x == 0) OZ_TRACE(5, e);                // set e drain starts
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (set == 0) {
          // levels 2..5 in pairs: over 512 of K |sum_2|, |sum_3| <= 2^23, |sum_4| <= 5 2^21,
          // |sum_5| <= 6 2^21 (digit bounds), so x_2 128 + x_3 and x_4 128 + x_5 are exact
          // in 32 bits; 8 columns of two levels per TMEM round trip
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            const float up0 = __int_as_float((127 + 14 * pr) << 23);       // level 2 + 2 pr
            const float up1 = __int_as_float((127 + 14 * pr + 7) << 23);   // level 3 + 2 pr
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
              float va[8], vb[8];
              const uint32_t base = tmem + lane_off + (uint32_t)(2 * pr * QN + col0 + 8 * hh);
              tmem_ld8x2(base, base + QN, va, vb);
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int c = __float2int_rn(va[q] * up0) * 128 + __float2int_rn(vb[q] * up1);
                acc[8 * hh + q] += (long long)c << (pr == 0 ? 28 : 14);
              }
            }
          }
        } else {
          // levels 6, 7 (|sum_6| <= 7 2^21, |sum_7| <= 2^24) and the rounded 8..9
          // (|sum| 2^35 < 9.1 2^14 over 512 of K: 9 2^12 digit units per k at level 8,
          // 10 2^12 at level 9), all three in one exact 32-bit integer; 8 columns of
          // each per round trip
#pragma unroll
          for (int hh = 0; hh < 4; ++hh) {
            float v6[8], v7[8], vr[8];
            const uint32_t base = tmem + lane_off + (uint32_t)(col0 + 8 * hh);
            tmem_ld8x3(base, base + QN, base + 2 * QN, v6, v7, vr);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int c = __float2int_rn(v6[q] * 268435456.0f) * 128 +
                            __float2int_rn(v7[q] * 34359738368.0f) +
                            __float2int_rn(vr[q] * 34359738368.0f);
              acc[8 * hh + q] += (long long)c;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) OZ_TRACE(6, e);                // ... and ends
        mbar_arrive(smem_u32(&bars[kAccEmpty]));
      }
    }
    if (!failed && g.fuse) {
      // a warp's lanes are 32 consecutive rows: each column's stores coalesce
      const int m = m0 + row;
      if (m < g.M) {
        const bool top = m < g.c_rows;
        double* const Cm = top ? g.C + m : g.C2 + (m - g.c_rows);
        const double* const Cinm = top ? g.Cin + m : g.Cin2 + (m - g.c_rows);
        const int ldc = top ? g.ldc : g.ldc2, ldcin = top ? g.ldcin : g.ldcin2;
        const bool lower = g.out_lower && top;
        const int ea = g.exA[m] - 2093;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int n = n0 + col0 + q;
          if (n >= g.N || (lower && m < n)) continue;
          double out = compose(acc[q], ea + g.exB[n]);
          out = scale_add(out, g.amode, g.alpha, g.bmode, g.beta, Cinm + (int64_t)n * ldcin);
          Cm[(int64_t)n * ldc] = out;
        }
      }
    } else if (!failed) {
      long long* part = g.partial + (int64_t)z * g.Mp * g.Np + (m0 + row) +
                        (int64_t)(n0 + col0) * g.Mp;
#pragma unroll
      for (int q = 0; q < 32; ++q) part[(int64_t)q * g.Mp] = acc[q];
    }
    if (failed && threadIdx.x == 0) atomicExch(&s_abort, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && s_abort) {
    for (int r = s_consumed; r < s_issued; ++r)
      mbar_wait(smem_u32(&bars[kFull + r % kQStages]), (uint32_t)((r / kQStages) & 1),
                kOzWaitLimit);
    if (g.status) atomicExch(g.status, (int)BTA_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// ---- 256 x 128 tiles on a CTA pair (S = 8) ---------------------------------
//
// The products of ozaki_gemm128_kernel with M = 256 MMAs over a pair of CTAs
// on two SMs (a thread-block cluster of 2, tcgen05 cta_group::2).  CTA r of
// the pair loads rows r*128 .. r*128+127 of the pair's A rows and B rows
// (columns of op(B)) r*64 .. r*64+63 of its 128; one MMA, issued by the
// leader (r = 0), reads both CTAs' shared memory and accumulates each CTA's
// 128 output rows in that CTA's tensor memory.  Per 128 x 128 x 16 of work an
// SM then reads 4 KB of A and 2 KB of B (8 KB in the one-CTA kernel) and its
// TMA writes 48 KB per slab (64 KB), which relieves the shared-memory port
// that bounds the one-CTA kernel.  Sub-passes, accumulator sets, drains and
// integer sums are those of ozaki_gemm128_kernel, per CTA.
//
// Across the pair: each CTA's loads complete on its own `loaded` barrier, so
// each can account for its own copies; the peer's warp 17 relays every
// completed slab to the leader's `peer` barrier (a remote arrive), and the
// leader's MMA warp starts a slab once both halves are in.  The leader's
// commits arrive on both CTAs' `empty` and `accfull` barriers (multicast);
// each CTA's drain warps, when done with a set, arrive once on the leader's
// `accempty`.  Before releasing tensor memory the two CTAs exchange `done`
// arrivals, so neither deallocates or exits while the other may still touch
// its shared or tensor memory.  Every wait is bounded; on expiry a CTA records
// BTA_ERR_TIMEOUT, stops issuing, waits (bounded) for its own loads and MMAs
// and still takes part in the exchange.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// The shared::cluster address of the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr)
               : "memory");
}

// Bounded wait with cluster-scope acquire (the barrier receives arrivals from
// the peer CTA or the leader's tensor-core commits).
__device__ __forceinline__ bool mbar_wait_cl(uint32_t addr, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ bool warp_wait_cl(uint32_t addr, uint32_t parity, int lane) {
  int ok = 0;
  if (lane == 0) ok = mbar_wait_cl(addr, parity, kOzWaitLimit) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Commit of the leader's pair MMAs: arrive on the barrier at this offset in
// both CTAs once they complete.
__device__ __forceinline__ void pair_commit_both(uint32_t mbar, uint32_t leader) {
  const uint16_t mask = 3;
  asm volatile(
      "{\n .reg .pred e;\n setp.ne.b32 e, %1, 0;\n"
      " @e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %2;\n}\n" ::"r"(mbar),
      "r"(leader), "h"(mask)
      : "memory");
}

// ... on the leader's barrier only.
__device__ __forceinline__ void pair_commit_own(uint32_t mbar, uint32_t leader) {
  asm volatile(
      "{\n .reg .pred e;\n setp.ne.b32 e, %1, 0;\n"
      " @e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
          mbar),
      "r"(leader)
      : "memory");
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kQThreads, 1)
    ozaki_gemm_pair_kernel(const __grid_constant__ CUtensorMap mA,
                           const __grid_constant__ CUtensorMap mB, OzqArgs g) {
  // Pair-tile order: groups of `group` pair rows, column by column inside a
  // group (as ozaki_gemm128_kernel, in units of 256 x 128 tiles).
  const uint32_t rank = cluster_rank();
  const int pt = g.reverse ? (int)(gridDim.x >> 1) - 1 - ((int)blockIdx.x >> 1)
                           : (int)blockIdx.x >> 1;
  const int mt_all = g.Mp / kPM, nt_all = g.Np / QN;
  const int grp = pt / (g.group * nt_all);
  const int gm = min(g.group, mt_all - grp * g.group);
  const int in = pt - grp * g.group * nt_all;
  const int pm0 = (grp * g.group + in % gm) * kPM, n0 = (in / gm) * QN, z = blockIdx.z;
  // the same decision in both CTAs of the pair: the pair exits before any set-up
  if (g.out_lower && n0 > pm0 + kPM - 1) return;
  const int m0 = pm0 + (int)rank * OM;                 // this CTA's A rows / output rows
  const int nb0 = n0 + (int)rank * kPBRows;            // this CTA's B rows (columns of C)
  // the pair's K range (the same in both CTAs: it depends on the pair tile)
  int ks0, ks1;
  tile_slabs(g, pm0, kPM, n0, QN, z, ks0, ks1);
  const int nc = (ks1 - ks0 + kChunkSlabs - 1) / kChunkSlabs;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kPStages * kPStage);
  const int kLoaded = 0, kPeer = kPStages, kEmpty = 2 * kPStages, kAccFull = 3 * kPStages,
            kAccEmpty = 3 * kPStages + 1, kFinal = 3 * kPStages + 2, kDone = 3 * kPStages + 3;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kPStages + 4);
  __shared__ int s_abort, s_issued, s_waited;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) {
      mbar_init(smem_u32(&bars[kLoaded + s]), 1);
      mbar_init(smem_u32(&bars[kPeer + s]), 1);
      mbar_init(smem_u32(&bars[kEmpty + s]), 1);
    }
    mbar_init(smem_u32(&bars[kAccFull]), 1);
    mbar_init(smem_u32(&bars[kAccEmpty]), 2);   // one arrival per CTA of the pair
    mbar_init(smem_u32(&bars[kFinal]), 1);
    mbar_init(smem_u32(&bars[kDone]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
    s_issued = 0;
    s_waited = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  // both CTAs' barriers and tensor memory are set up before either touches the other's
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 16) {
    // ---- TMA producer (both CTAs): this CTA's halves of every slab; lane 0
    // alone runs the loop
    if (lane == 0) {
      int r = 0;
      bool stop = false;
      for (int c = 0; c < nc && !stop; ++c) {
        const int kt0 = ks0 + c * kChunkSlabs, kt1 = min(ks1, kt0 + kChunkSlabs);
        for (int P = 0; P < kQPasses && !stop; ++P) {
          const int aj0 = q_a0(P), bl0 = q_b0(P);
          for (int kt = kt0; kt < kt1; ++kt, ++r) {
            const int s = r % kPStages;
            if (r >= kPStages && !mbar_wait_cl(smem_u32(&bars[kEmpty + s]),
                                               (uint32_t)((r / kPStages - 1) & 1), kOzWaitLimit)) {
              atomicExch(&s_abort, 1);
              stop = true;
              break;
            }
            if (*(volatile int*)&s_abort) {
              stop = true;
              break;
            }
            const uint32_t full = smem_u32(&bars[kLoaded + s]);
            mbar_expect_tx(full, (uint32_t)kPStage);
            uint8_t* st = smem + s * kPStage;
            const int k0 = kt * OK16;
            for (int i = 0; i < 4; ++i)
              tma_load_2d(smem_u32(st + i * kQTile), &mA, full, k0, (aj0 + i) * g.Mp + m0);
            for (int l = 0; l < 4; ++l)
              tma_load_2d(smem_u32(st + 4 * kQTile + l * kPBTile), &mB, full, k0,
                          (bl0 + l) * g.Bp + nb0);
            *(volatile int*)&s_issued = r + 1;
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 17 && rank != 0) {
    // ---- relay (peer CTA): each slab of this CTA in place -> the leader's `peer`
    if (lane == 0) {
      int r = 0;
      bool stop = false;
      for (int c = 0; c < nc && !stop; ++c) {
        const int kt0 = ks0 + c * kChunkSlabs, kt1 = min(ks1, kt0 + kChunkSlabs);
        for (int P = 0; P < kQPasses && !stop; ++P) {
          for (int kt = kt0; kt < kt1; ++kt, ++r) {
            const int s = r % kPStages;
            if (!mbar_wait(smem_u32(&bars[kLoaded + s]), (uint32_t)((r / kPStages) & 1),
                           kOzWaitLimit)) {
              atomicExch(&s_abort, 1);
              stop = true;
              break;
            }
            mbar_arrive_remote(cluster_addr(smem_u32(&bars[kPeer + s]), 0));
            *(volatile int*)&s_waited = r + 1;
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == 17) {
    // ---- MMA issuer (leader CTA): lane 0 alone runs the loop and issues
    if (lane == 0) {
      const uint64_t dbase = sdesc64(smem_u32(smem));
      bool stop = false;
      int r = 0, e = 0;   // slabs consumed, accumulator sets handed to the drains
      for (int c = 0; c < nc && !stop; ++c) {
        const int kt0 = ks0 + c * kChunkSlabs, kt1 = min(ks1, kt0 + kChunkSlabs);
        for (int P = 0; P < kQPasses && !stop; ++P) {
          // P0 and P1 open an accumulator set: wait until both CTAs drained the last one
          if (P <= 1 && e > 0 &&
              !mbar_wait_cl(smem_u32(&bars[kAccEmpty]), (uint32_t)((e - 1) & 1), kOzWaitLimit)) {
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          for (int kt = kt0; kt < kt1; ++kt, ++r) {
            const int s = r % kPStages;
            const uint32_t par = (uint32_t)((r / kPStages) & 1);
            if (!mbar_wait(smem_u32(&bars[kLoaded + s]), par, kOzWaitLimit)) {
              stop = true;
              break;
            }
            *(volatile int*)&s_waited = r + 1;
            if (!mbar_wait_cl(smem_u32(&bars[kPeer + s]), par, kOzWaitLimit)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t dst = dbase + (uint64_t)((s * kPStage) >> 4);
            const uint32_t first = kt == kt0;
            if (P == 0) q_slab<true, 0>(tmem, dst, first, 1u);
            else if (P == 1) q_slab<true, 1>(tmem, dst, first, 1u);
            else if (P == 2) q_slab<true, 2>(tmem, dst, first, 1u);
            else q_slab<true, 3>(tmem, dst, first, 1u);
            pair_commit_both(smem_u32(&bars[kEmpty + s]), 1u);   // both halves free
          }
          if (!stop && (P == 0 || P == kQPasses - 1)) {
            pair_commit_both(smem_u32(&bars[kAccFull]), 1u);     // this set's sums ready
            ++e;
          }
        }
      }
      if (stop) {
        atomicExch(&s_abort, 1);
        // wait (bounded) for the MMAs this thread issued before leaving
        pair_commit_own(smem_u32(&bars[kFinal]), 1u);
        mbar_wait(smem_u32(&bars[kFinal]), 0, kOzWaitLimit);
      }
    }
    __syncwarp();
  } else if (warp < 16) {
    // ---- warps 0-15 (both CTAs): thread = output row (TMEM lane) x 32
    // columns; the tile's integer sums (units 2^-35 of the level-2 unit) stay
    // in registers
    const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
    const int row = (warp & 3) * 32 + lane, col0 = (warp >> 2) * 32;
    const uint32_t acc_empty = cluster_addr(smem_u32(&bars[kAccEmpty]), 0);
    long long acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0ll;
    int failed = 0, e = 0;
    for (int c = 0; c < nc && !failed; ++c) {
      for (int set = 0; set < 2; ++set, ++e) {
        const bool ok = mbar_wait_cl(smem_u32(&bars[kAccFull]), (uint32_t)(e & 1), kOzWaitLimit);
        if (bar_or_512(!ok || *(volatile int*)&s_abort)) {
          failed = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (set == 0) {
          // levels 2..5 in pairs: over 512 of K |sum_2|, |sum_3| <= 2^23, |sum_4| <= 5 2^21,
          // |sum_5| <= 6 2^21 (digit bounds), so x_2 128 + x_3 and x_4 128 + x_5 are exact
          // in 32 bits; 8 columns of two levels per TMEM round trip
#pragma unroll
          for (int pr = 0; pr < 2; ++pr) {
            const float up0 = __int_as_float((127 + 14 * pr) << 23);       // level 2 + 2 pr
            const float up1 = __int_as_float((127 + 14 * pr + 7) << 23);   // level 3 + 2 pr
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
              float va[8], vb[8];
              const uint32_t base = tmem + lane_off + (uint32_t)(2 * pr * QN + col0 + 8 * hh);
              tmem_ld8x2(base, base + QN, va, vb);
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int c = __float2int_rn(va[q] * up0) * 128 + __float2int_rn(vb[q] * up1);
                acc[8 * hh + q] += (long long)c << (pr == 0 ? 28 : 14);
              }
            }
          }
        } else {
          // levels 6, 7 (|sum_6| <= 7 2^21, |sum_7| <= 2^24) and the rounded 8..9
          // (|sum| 2^35 < 9.1 2^14 over 512 of K: 9 2^12 digit units per k at level 8,
          // 10 2^12 at level 9), all three in one exact 32-bit integer; 8 columns of
          // each per round trip
#pragma unroll
          for (int hh = 0; hh < 4; ++hh) {
            float v6[8], v7[8], vr[8];
            const uint32_t base = tmem + lane_off + (uint32_t)(col0 + 8 * hh);
            tmem_ld8x3(base, base + QN, base + 2 * QN, v6, v7, vr);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int c = __float2int_rn(v6[q] * 268435456.0f) * 128 +
                            __float2int_rn(v7[q] * 34359738368.0f) +
                            __float2int_rn(vr[q] * 34359738368.0f);
              acc[8 * hh + q] += (long long)c;
            }
          }
        }
        // every drain thread's loads are done before the one arrival on the leader
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        bar_or_512(0);
        if (threadIdx.x == 0) mbar_arrive_remote(acc_empty);
      }
    }
    if (!failed) {
      long long* part = g.partial + (int64_t)z * g.Mp * g.Np + (m0 + row) +
                        (int64_t)(n0 + col0) * g.Mp;
#pragma unroll
      for (int q = 0; q < 32; ++q) part[(int64_t)q * g.Mp] = acc[q];
    }
    if (failed && threadIdx.x == 0) atomicExch(&s_abort, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_abort) {
      // this CTA's loads issued but not seen complete: wait (bounded) for them
      for (int r = s_waited; r < s_issued; ++r)
        mbar_wait(smem_u32(&bars[kLoaded + r % kPStages]), (uint32_t)((r / kPStages) & 1),
                  kOzWaitLimit);
    }
    // the exchange: the peer arrives, then waits; the leader waits, then arrives
    bool ok;
    if (rank != 0) {
      mbar_arrive_remote(cluster_addr(smem_u32(&bars[kDone]), 0));
      ok = mbar_wait_cl(smem_u32(&bars[kDone]), 0, kOzWaitLimit);
    } else {
      ok = mbar_wait_cl(smem_u32(&bars[kDone]), 0, kOzWaitLimit);
      mbar_arrive_remote(cluster_addr(smem_u32(&bars[kDone]), 1));
    }
    if ((s_abort || !ok) && g.status) atomicExch(g.status, (int)BTA_ERR_TIMEOUT);
  }
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// C = alpha * (sum over the splits of the integer tile sums) * 2^(exA + exB - 2093)
// + beta * Cin; one thread per element, m fastest.
struct ComposeArgs {
  int M, N, Mp, Np, splits, out_lower;
  double alpha, beta;
  int amode, bmode;
  double* C;
  int ldc;
  const double* Cin;
  int ldcin;
  // rows m >= c_rows (INT_MAX: none) go to C2 / Cin2, without the lower mask
  int c_rows;
  double* C2;
  int ldc2;
  const double* Cin2;
  int ldcin2;
  const int* exA;
  const int* exB;
  const long long* partial;
};

// Thread: row m and kComposeCols consecutive columns, every load issued
// before the first store (several independent loads in flight per thread).
constexpr int kComposeCols = 4;

__global__ void ozaki_compose_kernel(ComposeArgs g) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.M) return;
  const bool top = m < g.c_rows;
  double* const Cm = top ? g.C + m : g.C2 + (m - g.c_rows);
  const double* const Cinm = top ? g.Cin + m : g.Cin2 + (m - g.c_rows);
  const int ldc = top ? g.ldc : g.ldc2, ldcin = top ? g.ldcin : g.ldcin2;
  const bool lower = g.out_lower && top;
  const int64_t zstride = (int64_t)g.Mp * g.Np;
  for (int n0 = blockIdx.y * kComposeCols; n0 < g.N; n0 += gridDim.y * kComposeCols) {
    if (lower && m < n0) break;
    long long X[kComposeCols];
    double cin[kComposeCols];
#pragma unroll
    for (int c = 0; c < kComposeCols; ++c) {
      const int n = n0 + c;
      X[c] = 0;
      cin[c] = 0.0;
      if (n >= g.N || (lower && m < n)) continue;
      const long long* p = g.partial + m + (int64_t)n * g.Mp;
      for (int z = 0; z < g.splits; ++z) X[c] += p[(int64_t)z * zstride];
      if (g.bmode) cin[c] = Cinm[(int64_t)n * ldcin];
    }
#pragma unroll
    for (int c = 0; c < kComposeCols; ++c) {
      const int n = n0 + c;
      if (n >= g.N || (lower && m < n)) continue;
      double out = compose(X[c], g.exA[m] + g.exB[n] - 2093);
      out = scale_add(out, g.amode, g.alpha, g.bmode, g.beta, &cin[c]);
      Cm[(int64_t)n * ldc] = out;
    }
  }
}

// ---- splitting ---------------------------------------------------------------

// Element (r, k) of op(X) masked to its triangle (0 outside).
__device__ __forceinline__ double op_elem(const double* X, int ldx, int trans, int tri, int r,
                                          int k) {
  if ((tri == TRI_LOWER && k > r) || (tri == TRI_UPPER && k < r)) return 0.0;
  return trans ? X[k + (int64_t)r * ldx] : X[r + (int64_t)k * ldx];
}

// One operand to split: rows of op(X) (op(B)^T for the B side), their
// exponent bounds ex[rowsP] and slices Y[S][rowsP][Kp].  op(X) may be a 2 x 2
// block matrix cut after row rc and column kc: the leading block is (X, ldx,
// trans, tri), the others P[0] (rows < rc, k >= kc), P[1] (rows >= rc,
// k < kc) and P[2] (rows >= rc, k >= kc), each untriangular, zero when its
// pointer is null.  An operand without cuts has rc = kc = INT_MAX.  The
// leading block's trans also fixes the order in which the kernels read.
struct SplitPart {
  const double* X;
  int ld, trans;
};
struct SplitOp {
  const double* X;
  int ldx, trans, tri, rows, rowsP;
  int* ex;
  __nv_bfloat16* Y;
  int rc, kc;
  SplitPart P[3];
};

// Element (r, k) of a block part (r, k within op(X) as a whole).
__device__ __forceinline__ double op_part(const SplitOp& o, int r, int k) {
  const bool rb = r >= o.rc, kb = k >= o.kc;
  const SplitPart& q = !rb ? o.P[0] : !kb ? o.P[1] : o.P[2];
  if (!q.X) return 0.0;
  if (rb) r -= o.rc;
  if (kb) k -= o.kc;
  return q.trans ? q.X[k + (int64_t)r * q.ld] : q.X[r + (int64_t)k * q.ld];
}

// Element (r, k) of op(X): the leading block inline with its memory order
// TR known at compile time, then the other parts.
template <int TR>
__device__ __forceinline__ double op_get(const SplitOp& o, int r, int k) {
  if (r < o.rc && k < o.kc) return op_elem(o.X, o.ldx, TR, o.tri, r, k);
  return op_part(o, r, k);
}
struct SplitArgs {
  SplitOp op[2];   // blockIdx.z selects the operand
  int K, Kp;
};

// ex[r] = max over k of the biased exponent field of op(X)[r][k] (ex zeroed
// beforehand).  Block 256 threads over 32 rows x 64 columns of op(X), read
// in the memory order of X, 8 independent loads per thread.
__global__ void ozaki_exp_kernel(SplitArgs a) {
  const SplitOp o = blockIdx.z == 0 ? a.op[0] : a.op[1];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  if (r0 >= o.rows) return;
  __shared__ int smax[32];
  const int t = threadIdx.x;
  if (t < 32) smax[t] = 0;
  __syncthreads();
  int e = 0;
  if (!o.trans) {
    const int rr = t & 31, r = r0 + rr;   // consecutive threads: consecutive rows
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + (t >> 5) + 8 * i;
      if (r < o.rows && k < a.K) {
        const double v = op_get<0>(o, r, k);
        e = max(e, (int)((__double_as_longlong(v) >> 52) & 0x7FF));
      }
    }
    atomicMax(&smax[rr], e);
  } else {
    const int kk = t & 63, k = k0 + kk;   // consecutive threads: consecutive k
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int rr = (t >> 6) + 4 * i, r = r0 + rr;
      int ei = 0;
      if (r < o.rows && k < a.K) {
        const double v = op_get<1>(o, r, k);
        ei = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
      }
      ei = (int)__reduce_max_sync(0xffffffffu, (unsigned)ei);   // a warp shares rr
      if ((t & 31) == 0) atomicMax(&smax[rr], ei);
    }
  }
  __syncthreads();
  if (t < 32 && r0 + t < o.rows && smax[t] > 0) atomicMax(&o.ex[r0 + t], smax[t]);
}

// Y[j][r][k] (j < S, r < rowsP, k < Kp; K contiguous) = digit j of
// op(X)[r][k] times 2^(-7j); zero in the padding.  Block 256 threads over
// 32 rows x 64 columns, staged through a swizzled shared tile: column c of
// row q sits at c ^ ((q ^ (c >> 3)) & 15), which keeps both the transposing
// writes (16 rows, one column) and the digit reads (2 rows x 8 column groups)
// of every half-warp on 16 distinct 8-byte banks.
__device__ __forceinline__ int split_swz(int q, int c) { return c ^ ((q ^ (c >> 3)) & 15); }

template <int S>
__global__ void ozaki_split_kernel(SplitArgs a) {
  const SplitOp o = blockIdx.z == 0 ? a.op[0] : a.op[1];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  if (r0 >= o.rowsP) return;
  __shared__ double tile[32][64];   // tile[r - r0][split_swz(r - r0, k - k0)]
  const int t = threadIdx.x;
  if (!o.trans) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int idx = t + 256 * i, rr = idx & 31, kk = idx >> 5;
      const int r = r0 + rr, k = k0 + kk;
      tile[rr][split_swz(rr, kk)] =
          (r < o.rows && k < a.K) ? op_get<0>(o, r, k) : 0.0;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int idx = t + 256 * i, kk = idx & 63, rr = idx >> 6;
      const int r = r0 + rr, k = k0 + kk;
      tile[rr][split_swz(rr, kk)] =
          (r < o.rows && k < a.K) ? op_get<1>(o, r, k) : 0.0;
    }
  }
  __syncthreads();
  const size_t plane = (size_t)o.rowsP * a.Kp;
  // thread: row q = t >> 3 and columns 8 g .. 8 g + 7, g = t & 7, so that a
  // warp writes 4 rows x 128 contiguous bytes of each slice, one 16-byte
  // store per thread and slice.  A digit times its power of two has at most
  // 8 significant bits, so its BF16 pattern is the upper half of its FP32 one.
  const int q = t >> 3, g = t & 7, r = r0 + q, k = k0 + 8 * g;
  if (k >= a.Kp) return;   // Kp is a multiple of 32 and k of 8: k + 7 < Kp too
  const int er = r < o.rows ? o.ex[r] : 0;
  uint32_t w[S][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    float d0[S], d1[S];
    digits<S>(tile[q][split_swz(q, 8 * g + e)], er, d0);
    digits<S>(tile[q][split_swz(q, 8 * g + e + 1)], er, d1);
#pragma unroll
    for (int j = 0; j < S; ++j)
      w[j][e / 2] = __byte_perm(__float_as_uint(d0[j]), __float_as_uint(d1[j]), 0x7632);
  }
  uint4* y = reinterpret_cast<uint4*>(o.Y + (size_t)r * a.Kp + k);
#pragma unroll
  for (int j = 0; j < S; ++j) y[j * plane / 8] = make_uint4(w[j][0], w[j][1], w[j][2], w[j][3]);
}

// 2D map over Y viewed as (S * rowsP) x Kp BF16, box 32 (K) x boxRows.
bta_status make_map_bf16(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* map,
                         const __nv_bfloat16* base, int rowsAll, int Kp, int boxRows) {
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rowsAll};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)OK16, (cuuint32_t)boxRows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base),
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BTA_OK : BTA_ERR_ARG;
}

// Which kernel a product takes: 128 x 64 tiles, or (S = 8) 128 x 128 tiles
// with the K slabs split over `splits` CTAs per tile.  A wave model in units
// of one slab's MMAs (about the same time in either kernel) plus a fixed cost
// of ~4 slabs a CTA (set-up, drains, store): the time goes as (waves of CTAs)
// x (slabs per CTA + 4); the 128 x 128 kernel is taken when that is smaller
// (BTA_OZAKI_N128 = 0 / 1 forces the choice).
struct OzPlan {
  bool n128 = false;
  bool pair = false;   // 256 x 128 tiles on CTA pairs (implies n128)
  int splits = 1;
};
constexpr int kMaxSplits = 16;
constexpr int kCtaFixedSlabs = 4;
constexpr int kPairSlab = 13;   // a pair's slab time in sixteenths of the one-CTA kernel's

// CTA pairs of the pair kernel that fit on the GPU at once (1 CTA per SM;
// a pair needs two SMs of one cluster-capable group), queried once per device.
int pair_slots() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  int* slot = dev >= 0 && dev < 64 ? &cache[dev] : nullptr;
  if (slot && *slot > 0) return *slot;
  int n = 0;
  if (cudaFuncSetAttribute(ozaki_gemm_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           kPSmem) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * 512);
    cfg.blockDim = dim3(kQThreads);
    cfg.dynamicSmemBytes = kPSmem;
    if (cudaOccupancyMaxActiveClusters(&n, ozaki_gemm_pair_kernel, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  if (n < 1) n = std::max(1, sm_count() / 2);
  if (slot) *slot = n;
  return n;
}

// need128: the product writes a two-part C, which only the 128 x 128
// kernel's compose pass does (S = 8).
OzPlan oz_plan(int M, int N, int K, int S, bool need128 = false) {
  static const int force = [] {
    const char* v = std::getenv("BTA_OZAKI_N128");
    return v && *v ? std::atoi(v) : -1;
  }();
  // BTA_OZAKI_PAIR = 1 selects the pair kernel (otherwise the one-CTA kernels)
  static const int force_pair = [] {
    const char* v = std::getenv("BTA_OZAKI_PAIR");
    return v && *v ? std::atoi(v) : -1;
  }();
  OzPlan p;
  if (S != 8 || (force == 0 && !need128)) return p;
  const int kSmCount = sm_count();
  const int64_t nk = cdiv(K, OK16);
  const int64_t t64 = (int64_t)cdiv(M, OM) * cdiv(N, OBN);
  const int64_t t128 = (int64_t)cdiv(M, OM) * cdiv(N, QN);
  const int64_t est64 = cdiv(t64, kSmCount) * (nk + kCtaFixedSlabs);
  int64_t best = -1;
  for (int sp = 1; sp <= kMaxSplits && sp <= nk; ++sp) {
    if (sp > 1 && t128 * sp > kSmCount) break;   // keeps the split sums small
    const int64_t est = cdiv(t128 * sp, kSmCount) * (cdiv(nk, sp) + kCtaFixedSlabs);
    if (best < 0 || est < best) {
      best = est;
      p.splits = sp;
    }
  }
  p.n128 = force == 1 || need128 || best < est64;
  if (!p.n128) p.splits = 1;
  // Opt-in (BTA_OZAKI_PAIR = 1): measured on GB300 it is slower than the
  // one-CTA 128 x 128 kernel (4096^3: 4.37 vs 3.78 ms; 4800^3: 7.34 vs
  // 6.35 ms), so the plan keeps the one-CTA kernels unless asked.
  if (force_pair != 1) return p;
  // The pair kernel: a 256 x 128 tile per pair in about the time the one-CTA
  // kernel spends on a 128 x 128 tile per SM, with its slabs ~kPairSlab as
  // long (the MMAs read less shared memory).  Same wave model.
  const int pairs = pair_slots();
  const int64_t tp = (int64_t)cdiv(M, kPM) * cdiv(N, QN);
  int64_t bestp = -1;
  int sp_best = 1;
  for (int sp = 1; sp <= kMaxSplits && sp <= nk; ++sp) {
    if (sp > 1 && tp * sp > pairs) break;
    const int64_t est = cdiv(tp * sp, pairs) * (cdiv(nk, sp) * kPairSlab / 16 + kCtaFixedSlabs);
    if (bestp < 0 || est < bestp) {
      bestp = est;
      sp_best = sp;
    }
  }
  const int64_t cur = p.n128 ? best : est64;
  if (force_pair == 1 || bestp < cur) {
    p.pair = true;
    p.n128 = true;
    p.splits = sp_best;
  }
  return p;
}

struct OzLayout {
  int Mp, Np, Kp;
  size_t a_off, b_off, ea_off, eb_off, p_off, total;
  OzLayout(int M, int N, int K, int S, const OzPlan& plan) {
    Mp = plan.pair ? cdiv(M, kPM) * kPM : cdiv(M, OM) * OM;
    Np = plan.n128 ? cdiv(N, QN) * QN : cdiv(N, OBN) * OBN;
    Kp = cdiv(K, OK16) * OK16;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    a_off = 0;
    b_off = up((size_t)S * Mp * Kp * 2);
    ea_off = b_off + up((size_t)S * Np * Kp * 2);
    eb_off = ea_off + up((size_t)Mp * 4);
    p_off = eb_off + up((size_t)Np * 4);
    const size_t part = plan.n128 ? (size_t)plan.splits * Mp * Np * 8
                                  : (Kp > kChunkSlabs * OK16 ? (size_t)Mp * Np * 8 : 0);
    total = p_off + up(part) + 256;
  }
};

// marks (optional): two events recorded on s around the tensor-core product
// kernel's launch alone (the measurement entry point bta_gemm_emulated_timed).
template <int S>
bta_status launch_ozaki(const Gemm& g, uint8_t* ws, int32_t* status, cudaStream_t s,
                        const cudaEvent_t* marks) {
  using Cfg = OzCfg<S>;
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  BTA_TRY(tensor_map_encoder(&enc));
  const int M = g.M, N = g.N, K = g.K;
  if (g.C2 && S != 8) return BTA_ERR_ARG;
  const OzPlan plan = oz_plan(M, N, K, S, g.C2 != nullptr);
  const OzLayout L(M, N, K, S, plan);
  __nv_bfloat16* YA = reinterpret_cast<__nv_bfloat16*>(ws + L.a_off);
  __nv_bfloat16* YB = reinterpret_cast<__nv_bfloat16*>(ws + L.b_off);
  int* exA = reinterpret_cast<int*>(ws + L.ea_off);
  int* exB = reinterpret_cast<int*>(ws + L.eb_off);
  // rows of op(B)^T: Y[n][k] = op(B)[k][n]; the triangle flips with the transpose
  const int trib = g.triB == TRI_LOWER ? TRI_UPPER : g.triB == TRI_UPPER ? TRI_LOWER : TRI_NONE;
  // op(B)^T == the first N rows of op(A) (the symmetric update L L^T, with
  // or without extra rows of A below): one set of slices serves both
  const bool b_parts = g.B12.X || g.B21.X || g.B22.X || g.b_k || g.b_cols;
  const bool a_kparts = g.A12.X || g.A22.X || g.a_k;
  const bool same = g.A == g.B && g.lda == g.ldb && g.transA == !g.transB && g.triA == trib &&
                    !b_parts && !a_kparts && N <= (g.a_rows ? g.a_rows : M);
  SplitArgs sa;
  sa.K = K;
  sa.Kp = L.Kp;
  auto cut = [](int c) { return c > 0 ? c : INT_MAX; };
  sa.op[0] = {g.A, g.lda, g.transA, g.triA, M, L.Mp, exA, YA, cut(g.a_rows), cut(g.a_k),
              {{g.A12.X, g.A12.ld, g.A12.trans},
               {g.A21.X, g.A21.ld, g.A21.trans},
               {g.A22.X, g.A22.ld, g.A22.trans}}};
  // the B side holds op(B)^T: its row cut is op(B)'s column cut and each
  // part is the transpose of the matching block of op(B)
  sa.op[1] = {g.B, g.ldb, !g.transB, trib, N, L.Np, exB, YB, cut(g.b_cols), cut(g.b_k),
              {{g.B21.X, g.B21.ld, !g.B21.trans},
               {g.B12.X, g.B12.ld, !g.B12.trans},
               {g.B22.X, g.B22.ld, !g.B22.trans}}};
  const int nops = same ? 1 : 2;
  BTA_CUDA_TRY(cudaMemsetAsync(exA, 0, (size_t)L.Mp * 4, s));
  if (!same) BTA_CUDA_TRY(cudaMemsetAsync(exB, 0, (size_t)L.Np * 4, s));
  ozaki_exp_kernel<<<dim3(cdiv(K, 64), cdiv(std::max(M, N), 32), nops), 256, 0, s>>>(sa);
  BTA_LAUNCHED();
  ozaki_split_kernel<S><<<dim3(cdiv(L.Kp, 64), std::max(L.Mp, L.Np) / 32, nops), 256, 0, s>>>(sa);
  BTA_LAUNCHED();
  const __nv_bfloat16* YBm = same ? YA : YB;
  const int bpitch = same ? L.Mp : L.Np;   // rows per B slice in its array
  CUtensorMap mA, mB;
  BTA_TRY(make_map_bf16(enc, &mA, YA, S * L.Mp, L.Kp, OM));
  BTA_TRY(make_map_bf16(enc, &mB, YBm, S * bpitch, L.Kp,
                        plan.pair ? kPBRows : plan.n128 ? QN : OBN));
  long long* partial = reinterpret_cast<long long*>(ws + L.p_off);
  if (plan.pair) {
    static bool attrp = false;
    if (!attrp) {
      BTA_CUDA_TRY(cudaFuncSetAttribute(ozaki_gemm_pair_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kPSmem));
      attrp = true;
    }
    OzqArgs q{};
    q.Mp = L.Mp; q.Np = L.Np; q.Bp = bpitch;
    q.nk = L.Kp / OK16;
    q.splits = plan.splits;
    q.out_lower = g.out_lower;
    q.tri_a = g.triA;
    q.tri_b = g.triB;
    // the K range of a tile grows with its row under a lower op(A) and with
    // its column under an upper op(B), the ends of the launch order: start
    // those first (the CTAs then finish closer together)
    q.reverse = (g.triA == TRI_LOWER || g.triB == TRI_UPPER) &&
                !(g.triA == TRI_UPPER || g.triB == TRI_LOWER);
    q.partial = partial;
    q.status = status;
    // a wave of pairs spans a near-square patch of 256 x 128 tiles
    q.group = std::min(L.Mp / kPM,
                       std::max(1, (int)std::lround(std::sqrt(pair_slots() / 2.0))));
    if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[0], s));
    ozaki_gemm_pair_kernel<<<dim3(2 * (L.Mp / kPM) * (L.Np / QN), 1, plan.splits), kQThreads,
                             kPSmem, s>>>(mA, mB, q);
    BTA_LAUNCHED();
    if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[1], s));
  }
  if (plan.n128) {
    static bool attr128 = false;
    if (!attr128) {
      BTA_CUDA_TRY(cudaFuncSetAttribute(ozaki_gemm128_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, kQSmem));
      attr128 = true;
    }
    OzqArgs q{};
    q.Mp = L.Mp; q.Np = L.Np; q.Bp = bpitch;
    q.nk = L.Kp / OK16;
    q.splits = plan.splits;
    q.out_lower = g.out_lower;
    q.tri_a = g.triA;
    q.tri_b = g.triB;
    // the K range of a tile grows with its row under a lower op(A) and with
    // its column under an upper op(B), the ends of the launch order: start
    // those first (the CTAs then finish closer together)
    q.reverse = (g.triA == TRI_LOWER || g.triB == TRI_UPPER) &&
                !(g.triA == TRI_UPPER || g.triB == TRI_LOWER);
    q.partial = partial;
    q.status = status;
    // ~sqrt(SMs) tile rows a group: a wave of CTAs spans a near-square patch
    q.group = std::min(L.Mp / OM, std::max(1, (int)std::lround(std::sqrt((double)sm_count()))));
    q.fuse = 0;
    if (!plan.pair && plan.splits == 1) {   // C composed in the kernel's epilogue
      q.fuse = 1;
      q.M = M; q.N = N;
      q.amode = alpha_mode(g.alpha); q.bmode = beta_mode(g.beta);
      q.alpha = g.alpha; q.beta = g.beta;
      q.C = g.C; q.ldc = g.ldc;
      q.Cin = g.Cin ? g.Cin : g.C; q.ldcin = g.Cin ? g.ldcin : g.ldc;
      q.c_rows = g.C2 ? g.c_rows : INT_MAX;
      q.C2 = g.C2; q.ldc2 = g.ldc2;
      q.Cin2 = g.Cin2 ? g.Cin2 : g.C2; q.ldcin2 = g.Cin2 ? g.ldcin2 : g.ldc2;
      q.exA = exA; q.exB = same ? exA : exB;
    }
    if (!plan.pair) {
      if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[0], s));
      ozaki_gemm128_kernel<<<dim3((L.Mp / OM) * (L.Np / QN), 1, plan.splits), kQThreads,
                             kQSmem, s>>>(mA, mB, q);
      BTA_LAUNCHED();
      if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[1], s));
      if (q.fuse) return BTA_OK;
    }
    ComposeArgs c;
    c.M = M; c.N = N; c.Mp = L.Mp; c.Np = L.Np; c.splits = plan.splits;
    c.out_lower = g.out_lower;
    c.alpha = g.alpha; c.beta = g.beta; c.C = g.C; c.ldc = g.ldc;
    c.amode = alpha_mode(g.alpha); c.bmode = beta_mode(g.beta);
    c.Cin = g.Cin ? g.Cin : g.C; c.ldcin = g.Cin ? g.ldcin : g.ldc;
    c.c_rows = g.C2 ? g.c_rows : INT_MAX;
    c.C2 = g.C2; c.ldc2 = g.ldc2;
    c.Cin2 = g.Cin2 ? g.Cin2 : g.C2; c.ldcin2 = g.Cin2 ? g.ldcin2 : g.ldc2;
    c.exA = exA; c.exB = same ? exA : exB; c.partial = partial;
    ozaki_compose_kernel<<<dim3(cdiv(M, 256), std::min(cdiv(N, kComposeCols), 65535)), 256, 0, s>>>(c);
    BTA_LAUNCHED();
    return BTA_OK;
  }
  static bool attr_set = false;
  if (!attr_set) {
    BTA_CUDA_TRY(cudaFuncSetAttribute(ozaki_gemm_kernel<S>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::kSmem));
    attr_set = true;
  }
  OzArgs a;
  a.M = M; a.N = N; a.Kp = L.Kp; a.Mp = L.Mp; a.Np = bpitch;
  a.alpha = g.alpha; a.beta = g.beta; a.C = g.C; a.ldc = g.ldc;
  a.amode = alpha_mode(g.alpha); a.bmode = beta_mode(g.beta);
  a.Cin = g.Cin ? g.Cin : g.C; a.ldcin = g.Cin ? g.ldcin : g.ldc;
  a.out_lower = g.out_lower; a.exA = exA; a.exB = same ? exA : exB; a.status = status;
  a.partial = partial;
  if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[0], s));
  ozaki_gemm_kernel<S><<<dim3(L.Mp / OM, L.Np / OBN), kOzThreads, Cfg::kSmem, s>>>(mA, mB, a);
  BTA_LAUNCHED();
  if (marks) BTA_CUDA_TRY(cudaEventRecord(marks[1], s));
  return BTA_OK;
}

}  // namespace

// An upper bound over every product of at most M x N x K (either kernel):
// a sweep sizes one workspace for all of its products.
size_t ozaki_ws_bytes(int M, int N, int K, int slices) {
  const size_t t64 = OzLayout(M, N, K, slices, OzPlan()).total;
  if (slices != 8) return t64;
  const size_t Mq = (size_t)cdiv(M, OM) * OM, Nq = (size_t)cdiv(N, QN) * QN;
  const size_t Kp = (size_t)cdiv(K, OK16) * OK16;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t part = std::max(Mq * Nq, (size_t)sm_count() * OM * QN) * 8;
  const size_t t128 = up(8 * Mq * Kp * 2) + up(8 * Nq * Kp * 2) + up(Mq * 4) + up(Nq * 4) +
                      up(part) + 256;
  // pair kernel: rows padded to 256, at most one pair per two SMs per split
  const size_t Mr = (size_t)cdiv(M, kPM) * kPM;
  const size_t partp = std::max(Mr * Nq, (size_t)sm_count() * kPM * QN) * 8;
  const size_t tpair = up(8 * Mr * Kp * 2) + up(8 * Nq * Kp * 2) + up(Mr * 4) + up(Nq * 4) +
                       up(partp) + 256;
  return std::max(t64, std::max(t128, tpair));
}

bool ozaki_supported(const Gemm& g) {
  if (!(g.batch == 1 && !g.Ab && g.A && g.B && g.C && g.K >= 1 && g.K <= kMaxOzK && g.M >= 1 &&
        g.N >= 1))
    return false;
  if (!g.blocked()) return true;
  // block operands: cuts inside the matrix, parts only where a cut makes
  // room for them, no triangle in an operand with parts, C2 with its cut
  auto in = [](int c, int n) { return c == 0 || (c > 0 && c < n); };
  auto ok = [](const Gemm::Part& q) { return !q.X || q.ld >= 1; };
  if (!in(g.a_rows, g.M) || !in(g.a_k, g.K) || !in(g.b_k, g.K) || !in(g.b_cols, g.N) ||
      !in(g.c_rows, g.M))
    return false;
  if (!ok(g.A12) || !ok(g.A21) || !ok(g.A22) || !ok(g.B12) || !ok(g.B21) || !ok(g.B22))
    return false;
  if ((g.A21.X || g.A22.X) && !g.a_rows) return false;
  if ((g.A12.X || g.A22.X) && !g.a_k) return false;
  if ((g.B21.X || g.B22.X) && !g.b_k) return false;
  if ((g.B12.X || g.B22.X) && !g.b_cols) return false;
  if ((g.a_rows || g.a_k) && g.triA != TRI_NONE) return false;
  if ((g.b_k || g.b_cols) && g.triB != TRI_NONE) return false;
  if ((g.C2 != nullptr) != (g.c_rows > 0) || (g.C2 && g.ldc2 < 1)) return false;
  if (g.Cin2 && g.ldcin2 < 1) return false;
  return true;
}

bta_status ozaki_gemm(const Gemm& g, void* ws, int32_t* status, int slices, cudaStream_t s,
                      const cudaEvent_t* marks) {
  if (g.M <= 0 || g.N <= 0) return BTA_OK;
  if (!ozaki_supported(g) || !ws) return BTA_ERR_ARG;
  uint8_t* w = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ws) + 255) &
                                          ~(uintptr_t)255);
  switch (slices) {
    case 6: return launch_ozaki<6>(g, w, status, s, marks);
    case 7: return launch_ozaki<7>(g, w, status, s, marks);
    case 8: return launch_ozaki<8>(g, w, status, s, marks);
    default: return BTA_ERR_ARG;
  }
}

}  // namespace bta
