// Split-precision tensor-core GEMM for the mixed-precision sweeps (sm_103a):
//   C = alpha op(A) op(B) + beta C,  FP64 in and out,
// computed on tcgen05 tensor cores with TF32 operands and FP32 accumulation
// in tensor memory, each FP64 operand carried as a pair hi + lo of TF32
// values ("3xTF32": hi*hi + hi*lo + lo*hi, about 22 significant bits per
// product, against 11 for one TF32 product).
//
// Pipeline per 128 x 128 output tile (one CTA, 128 threads):
//   * a split kernel writes op(A) and op(B)^T as K-major FP32 hi/lo arrays;
//   * warp 0 lane 0 streams 32-wide K slabs of the four operand tiles into a
//     3-stage shared-memory ring with TMA (128-byte swizzle), signalling a
//     "full" mbarrier with the transaction byte count;
//   * warp 1 lane 0 issues 12 tcgen05.mma (kind::tf32, M=128, N=128, K=8) per
//     slab into one TMEM accumulator and releases the slab with
//     tcgen05.commit on its "empty" mbarrier;
//   * all four warps read the accumulator back with tcgen05.ld (one warp per
//     32 TMEM lanes) and apply alpha / beta in FP64.
// Every mbarrier wait is bounded: on expiry the kernel records
// BTA_ERR_TIMEOUT in a status word, stops issuing work, still waits (bounded)
// for the MMAs it issued and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tma.cuh"

namespace bta {
namespace {

using namespace tc;

constexpr int TM = 128, TN = 128, TK = 32;          // tile rows, cols, fp32 per K slab
constexpr int kStages = 3;
constexpr int kTileBytes = TM * TK * 4;             // 16 KB: one operand tile of one slab
constexpr int kStageBytes = 4 * kTileBytes;         // Ahi, Alo, Bhi, Blo
constexpr int kTcThreads = 128;
constexpr int kSmemBytes = kStages * kStageBytes + 1024 + 128;
constexpr uint32_t kTmemCols = 128;                 // 128 lanes x 128 fp32 columns
constexpr long long kWaitLimit = 1ll << 21;          // bounded mbarrier polls (~1 s)

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);     // start address
  d |= (uint64_t)1 << 16;                       // leading-dimension offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;             // stride between 8-row groups
  d |= (uint64_t)1 << 46;                       // descriptor version
  d |= (uint64_t)2 << 61;                       // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::tf32, FP32 accumulator, both operands
// K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

// FP32 accumulator value widened to FP64 with integer operations (GB300's
// FP64 pipe, conversions included, runs one warp instruction per ~64
// cycles); zero and subnormal inputs take the conversion.
__device__ __forceinline__ double widen(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xFF;
  if (e == 0 || e == 0xFF) return (double)x;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(e - 127 + 1023) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

struct TcArgs {
  int M, N, K;
  int amode, bmode;   // alpha: 0 -> 1, 1 -> -1, 2 -> general; beta: 0 -> 0, 1 -> 1, 2 -> general
  double alpha, beta;
  double* C;
  int ldc;
  const double* Cin;
  int ldcin;
  int out_lower;
  int32_t* status;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap mAhi,
                          const __grid_constant__ CUtensorMap mAlo,
                          const __grid_constant__ CUtensorMap mBhi,
                          const __grid_constant__ CUtensorMap mBlo, TcArgs g) {
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  if (g.out_lower && n0 > m0 + TM - 1) return;   // whole CTA exits before any set-up
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  // bars[0..S): full, bars[S..2S): empty, bars[2S]: done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (g.K + TK - 1) / TK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[kStages + s]), 1);
    }
    mbar_init(smem_u32(&bars[2 * kStages]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % kStages;
      if (kt >= kStages &&
          !mbar_wait(smem_u32(&bars[kStages + s]), (uint32_t)((kt / kStages - 1) & 1), kWaitLimit)) {
        s_abort = 1;
        break;
      }
      if (*(volatile int*)&s_abort) break;
      const uint32_t full = smem_u32(&bars[s]);
      mbar_expect_tx(full, kStageBytes);
      uint8_t* st = smem + s * kStageBytes;
      const int k0 = kt * TK;
      tma_load_2d(smem_u32(st), &mAhi, full, k0, m0);
      tma_load_2d(smem_u32(st + kTileBytes), &mAlo, full, k0, m0);
      tma_load_2d(smem_u32(st + 2 * kTileBytes), &mBhi, full, k0, n0);
      tma_load_2d(smem_u32(st + 3 * kTileBytes), &mBlo, full, k0, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    int issued = 0;
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)((kt / kStages) & 1), kWaitLimit)) {
        s_abort = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < TK / 8; ++kk) {
        const uint32_t off = kk * 32;   // 8 fp32 = 32 bytes along K inside the swizzle atom
        const uint64_t ahi = sdesc(base + off), alo = sdesc(base + kTileBytes + off);
        const uint64_t bhi = sdesc(base + 2 * kTileBytes + off);
        const uint64_t blo = sdesc(base + 3 * kTileBytes + off);
        mma_tf32(tmem, ahi, bhi, issued++ > 0);
        mma_tf32(tmem, ahi, blo, 1);
        mma_tf32(tmem, alo, bhi, 1);
      }
      mma_commit(smem_u32(&bars[kStages + s]));   // slab s free once these MMAs finish
    }
    mma_commit(smem_u32(&bars[2 * kStages]));     // accumulator complete
  }
  __syncwarp();
  // ---- epilogue: all four warps (the decision below is uniform per CTA)
  const bool done = mbar_wait(smem_u32(&bars[2 * kStages]), 0, kWaitLimit);
  const int failed = __syncthreads_or(!done || s_abort);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (failed) {
    if (threadIdx.x == 0 && g.status) atomicExch(g.status, (int)BTA_ERR_TIMEOUT);
  } else {
    const int m = m0 + warp * 32 + lane;
    for (int c = 0; c < TN; c += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c + j;
          if (n >= g.N || (g.out_lower && m < n)) continue;
          double out = widen(v[j]);
          if (g.amode == 1) out = -out;
          else if (g.amode == 2) out *= g.alpha;
          if (g.bmode == 1) out += g.Cin[m + (int64_t)n * g.ldcin];
          else if (g.bmode == 2) out = fma(g.beta, g.Cin[m + (int64_t)n * g.ldcin], out);
          g.C[m + (int64_t)n * g.ldc] = out;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

// Y (rows x Kp, row-major fp32 hi/lo) = split(op(X)) with
// op(X)[r][k] = trans ? X[k + r*ldx] : X[r + k*ldx], masked to its triangle.
// v = hi + lo + O(2^-22 |v|) with hi, lo TF32 (10 stored mantissa bits):
// hi is v rounded to nearest (ties away from zero) at its 10th mantissa bit,
// lo = v - hi (exact, at most 42 significant bits) rounded the same way.
// Both come from v's bit pattern with integer operations; exponents outside
// [2^-70, 2^100] (zero included) take FP32 conversions instead.
__device__ __forceinline__ void tf32_split(double v, float& h, float& l) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 1023 - 70 || e > 1023 + 100) {
    uint32_t hb, lb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"((float)v));
    h = __uint_as_float(hb);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lb) : "f"((float)(v - (double)h)));
    l = __uint_as_float(lb);
    return;
  }
  const unsigned long long sgn = b & (1ull << 63);
  const unsigned long long mag = b ^ sgn;
  const unsigned long long hmag = (mag + (1ull << 41)) & ~((1ull << 42) - 1);
  const int he = (int)(hmag >> 52);   // e, or e + 1 when the rounding carried
  const uint32_t s32 = (uint32_t)(sgn >> 32);
  h = __uint_as_float(s32 | ((uint32_t)(he - 1023 + 127) << 23) |
                      (uint32_t)((hmag >> 29) & 0x7FFFFFu));
  // lo in units of 2^(e - 1075): significand of v minus that of hi
  const long long vs = (long long)((mag & ((1ull << 52) - 1)) | (1ull << 52));
  const long long hs = he == e ? (long long)((hmag & ((1ull << 52) - 1)) | (1ull << 52))
                               : (long long)(1ull << 53);
  const long long d = vs - hs;   // |d| <= 2^41
  if (d == 0) {
    l = __uint_as_float(s32);    // signed zero
    return;
  }
  const unsigned long long ad = (unsigned long long)(d < 0 ? -d : d);
  const int nb = 64 - __clzll((long long)ad);   // significant bits of |d|
  unsigned long long q = ad;
  int ex = 0;
  if (nb > 11) {   // keep 11 significant bits, nearest, ties away from zero
    const int sh = nb - 11;
    q = (ad + (1ull << (sh - 1))) >> sh;
    ex = sh;
    if (q >> 11) {
      q >>= 1;
      ++ex;
    }
  }
  const int qb = 63 - __clzll((long long)q);    // leading-one position of q
  const int fe = qb + ex + e - 1075 + 127;        // >= 5 for e >= 1023 - 70
  l = __uint_as_float((s32 ^ (d < 0 ? 0x80000000u : 0u)) | ((uint32_t)fe << 23) |
                      (uint32_t)((q << (23 - qb)) & 0x7FFFFFu));
}

__global__ void split_tf32_kernel(int rows, int K, int Kp, const double* __restrict__ X, int ldx,
                                  int trans, int tri, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  __shared__ double t[32][33];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    // coalesced read: consecutive tx walk the contiguous index of X
    int r, k;
    if (!trans) { r = r0 + tx; k = k0 + yy; } else { k = k0 + tx; r = r0 + yy; }
    double v = 0.0;
    if (r < rows && k < K) {
      const bool zero = (tri == TRI_LOWER && k > r) || (tri == TRI_UPPER && k < r);
      if (!zero) v = trans ? X[k + (int64_t)r * ldx] : X[r + (int64_t)k * ldx];
    }
    if (!trans) t[tx][yy] = v; else t[yy][tx] = v;   // t[r - r0][k - k0]
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int r = r0 + yy, k = k0 + tx;
    if (r >= rows || k >= Kp) continue;
    float h, l;
    tf32_split(t[yy][tx], h, l);
    hi[(int64_t)r * Kp + k] = h;
    lo[(int64_t)r * Kp + k] = l;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bta_status get_encode() { return tensor_map_encoder(&g_encode); }

// 2D map over a row-major fp32 array rows x Kp, box 32 (K) x 128 (rows).
bta_status make_map(CUtensorMap* map, const float* base, int rows, int Kp) {
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  cuuint32_t box[2] = {TK, TM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BTA_OK : BTA_ERR_ARG;
}

}  // namespace

bta_status tensor_map_encoder(PFN_cuTensorMapEncodeTiled_v12000* out) {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return BTA_ERR_CUDA;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  *out = fn;
  return BTA_OK;
}

size_t tc_gemm_ws_bytes(int M, int N, int K) {
  const size_t Kp = (size_t)(K + 3) / 4 * 4;
  return 2 * ((size_t)M + N) * Kp * sizeof(float) + 256;
}

bta_status tc_gemm_mixed(const Gemm& g, void* ws, int32_t* status, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return BTA_OK;
  if (g.batch != 1 || g.Ab || !g.A || !g.B || !g.C || g.K < 1 || !ws) return BTA_ERR_ARG;
  if (g.blocked()) return BTA_ERR_ARG;   // block operands: emulated products only
  BTA_TRY(get_encode());
  const int M = g.M, N = g.N, K = g.K;
  const int Kp = (K + 3) / 4 * 4;
  float* Ahi = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(ws) + 255) & ~(uintptr_t)255);
  float* Alo = Ahi + (size_t)M * Kp;
  float* Bhi = Alo + (size_t)M * Kp;
  float* Blo = Bhi + (size_t)N * Kp;
  {
    dim3 grid(cdiv(Kp, 32), cdiv(M, 32));
    split_tf32_kernel<<<grid, dim3(32, 8), 0, s>>>(M, K, Kp, g.A, g.lda, g.transA, g.triA, Ahi,
                                                   Alo);
    BTA_LAUNCHED();
  }
  {
    // rows of op(B)^T: Y[n][k] = op(B)[k][n]; the mask flips with the transpose
    const int trib = g.triB == TRI_LOWER ? TRI_UPPER : g.triB == TRI_UPPER ? TRI_LOWER : TRI_NONE;
    dim3 grid(cdiv(Kp, 32), cdiv(N, 32));
    split_tf32_kernel<<<grid, dim3(32, 8), 0, s>>>(N, K, Kp, g.B, g.ldb, !g.transB, trib, Bhi,
                                                   Blo);
    BTA_LAUNCHED();
  }
  CUtensorMap mAhi, mAlo, mBhi, mBlo;
  BTA_TRY(make_map(&mAhi, Ahi, M, Kp));
  BTA_TRY(make_map(&mAlo, Alo, M, Kp));
  BTA_TRY(make_map(&mBhi, Bhi, N, Kp));
  BTA_TRY(make_map(&mBlo, Blo, N, Kp));
  static bool attr_set = false;
  if (!attr_set) {
    BTA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_tf32x3_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr_set = true;
  }
  TcArgs a;
  a.M = M; a.N = N; a.K = K; a.alpha = g.alpha; a.beta = g.beta; a.C = g.C; a.ldc = g.ldc;
  a.amode = g.alpha == 1.0 ? 0 : g.alpha == -1.0 ? 1 : 2;
  a.bmode = g.beta == 0.0 ? 0 : g.beta == 1.0 ? 1 : 2;
  a.Cin = g.Cin ? g.Cin : g.C; a.ldcin = g.Cin ? g.ldcin : g.ldc; a.out_lower = g.out_lower;
  a.status = status;
  dim3 grid(cdiv(M, TM), cdiv(N, TN));
  tc_gemm_tf32x3_kernel<<<grid, kTcThreads, kSmemBytes, s>>>(mAhi, mAlo, mBhi, mBlo, a);
  BTA_LAUNCHED();
  return BTA_OK;
}

}  // namespace bta
