// FP64 dense tile contractions for the BTA sweeps (sm_103a).
//
// On GB300 the FP64 rate is about two DFMA per clock per SM (a DFMA-chain
// probe reaches ~1.19 TFLOP/s over 152 SMs, while mma.sync .f64 reaches only
// ~1.05), so these kernels are FP64-pipe bound at any reasonable tiling: the
// design goal is to keep every SM's FP64 pipe fed (many resident CTAs, no
// idle tails), not to save bandwidth.  A 16x16 thread grid computes a
// BM x BN tile with DFMA from shared-memory stages of BK = 16, prefetching
// the next stage into registers while the current one is consumed.
#include <algorithm>

#include "common.cuh"

namespace bta {

int64_t g_launches = 0;

namespace {

constexpr int BK = 16;
constexpr int NT = 256;

struct GemmDev {
  int M, N, K;
  const double* A; int lda, transA, triA;
  const double* B; int ldb, transB, triB;
  double* C; int ldc;
  const double* Cin; int ldcin;
  double alpha, beta;
  int out_lower;
  int64_t strideA, strideB, strideC, strideCin;
};

__device__ __forceinline__ bool a_zero(int tri, int m, int k) {
  return (tri == TRI_LOWER && k > m) || (tri == TRI_UPPER && k < m);
}
// op(B) is K x N; lower means nonzero only for k >= n.
__device__ __forceinline__ bool b_zero(int tri, int k, int n) {
  return (tri == TRI_LOWER && n > k) || (tri == TRI_UPPER && k > n);
}

template <int BM, int BN>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(GemmDev g) {
  constexpr int TM = BM / 16, TN = BN / 16;
  constexpr int LA = BM * BK / NT;   // A elements loaded per thread per stage
  constexpr int LB = BN * BK / NT;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];

  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (g.out_lower && n0 > m0 + BM - 1) return;
  const double* A = g.A + (int64_t)blockIdx.z * g.strideA;
  const double* B = g.B + (int64_t)blockIdx.z * g.strideB;
  double* C = g.C + (int64_t)blockIdx.z * g.strideC;
  const double* Cin = g.Cin ? g.Cin + (int64_t)blockIdx.z * g.strideCin : nullptr;

  // K range that can hold nonzeros for this tile.
  int kbeg = 0, kend = g.K;
  if (g.triA == TRI_LOWER) kend = min(kend, m0 + BM);
  if (g.triA == TRI_UPPER) kbeg = max(kbeg, m0);
  if (g.triB == TRI_LOWER) kbeg = max(kbeg, n0);
  if (g.triB == TRI_UPPER) kend = min(kend, n0 + BN);
  kbeg = kbeg / BK * BK;

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  double ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      int idx = tid + NT * r;
      int m, k;
      if (!g.transA) { m = idx % BM; k = idx / BM; } else { k = idx % BK; m = idx / BK; }
      int gm = m0 + m, gk = k0 + k;
      double v = 0.0;
      if (gm < g.M && gk < kend && !a_zero(g.triA, gm, gk))
        v = g.transA ? A[gk + (int64_t)gm * g.lda] : A[gm + (int64_t)gk * g.lda];
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      int idx = tid + NT * r;
      int n, k;
      if (!g.transB) { k = idx % BK; n = idx / BK; } else { n = idx % BN; k = idx / BN; }
      int gn = n0 + n, gk = k0 + k;
      double v = 0.0;
      if (gn < g.N && gk < kend && !b_zero(g.triB, gk, gn))
        v = g.transB ? B[gn + (int64_t)gk * g.ldb] : B[gk + (int64_t)gn * g.ldb];
      rb[r] = v;
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < LA; ++r) {
      int idx = tid + NT * r;
      int m, k;
      if (!g.transA) { m = idx % BM; k = idx / BM; } else { k = idx % BK; m = idx / BK; }
      As[k][m] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < LB; ++r) {
      int idx = tid + NT * r;
      int n, k;
      if (!g.transB) { k = idx % BK; n = idx / BK; } else { n = idx % BN; k = idx / BN; }
      Bs[k][n] = rb[r];
    }
  };

  if (kbeg < kend) {
    load(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      __syncthreads();
      store();
      __syncthreads();
      if (k0 + BK < kend) load(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][ty + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
    }
  }

#pragma unroll
  for (int j = 0; j < TN; ++j) {
    int gn = n0 + ty + 16 * j;
    if (gn >= g.N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int gm = m0 + tx + 16 * i;
      if (gm >= g.M) continue;
      if (g.out_lower && gm < gn) continue;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, Cin[gm + (int64_t)gn * g.ldcin], v);
      C[gm + (int64_t)gn * g.ldc] = v;
    }
  }
}

// ----------------------------------------------------------------------------
// GEMV with a deterministic split over K.
// ----------------------------------------------------------------------------
__global__ void gemv_n_partial(int M, int K, const double* __restrict__ A, int lda, int triA,
                               const double* __restrict__ x, double* __restrict__ part) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int split = blockIdx.y;
  int kc = (K + gridDim.y - 1) / gridDim.y;
  int kb = split * kc, ke = min(K, kb + kc);
  if (triA == TRI_LOWER) ke = min(ke, m + 1);
  if (triA == TRI_UPPER) kb = max(kb, m);
  double s = 0.0;
  if (m < M)
    for (int k = kb; k < ke; ++k) s = fma(A[m + (int64_t)k * lda], x[k], s);
  if (m < M) part[(int64_t)split * M + m] = s;
}

// y[m] = sum_k A[k, m] x[k] (op(A) = A^T), one warp per output, lanes over K.
__global__ void gemv_t_partial(int M, int K, const double* __restrict__ A, int lda, int triA,
                               const double* __restrict__ x, double* __restrict__ part) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int split = blockIdx.y;
  int m = warp;
  if (m >= M) return;
  int kc = (K + gridDim.y - 1) / gridDim.y;
  int kb = split * kc, ke = min(K, kb + kc);
  // op(A)[m,k] = A[k,m]; op(A) lower -> zero for k > m
  if (triA == TRI_LOWER) ke = min(ke, m + 1);
  if (triA == TRI_UPPER) kb = max(kb, m);
  double s = 0.0;
  for (int k = kb + lane; k < ke; k += 32) s = fma(A[k + (int64_t)m * lda], x[k], s);
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) part[(int64_t)split * M + m] = s;
}

__global__ void gemv_finish(int M, int nsplit, const double* __restrict__ part, double alpha,
                            double beta, const double* yin, double* y) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  double s = 0.0;
  for (int j = 0; j < nsplit; ++j) s += part[(int64_t)j * M + m];
  double v = alpha * s;
  if (beta != 0.0) v = fma(beta, yin[m], v);
  y[m] = v;
}

}  // namespace

bta_status gemm_f64(const Gemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0) return BTA_OK;
  GemmDev d{g.M, g.N, g.K, g.A, g.lda, g.transA, g.triA, g.B, g.ldb, g.transB, g.triB,
            g.C, g.ldc, g.Cin ? g.Cin : g.C, g.Cin ? g.ldcin : g.ldc, g.alpha, g.beta,
            g.out_lower, g.strideA, g.strideB, g.strideC, g.strideCin};
  if (g.K <= 0) { d.K = 0; }
  // Tile choice.  Every tile is FP64-pipe bound and the hardware spreads
  // tiles evenly over the 152 SMs, so an op takes about
  // ceil(tiles / 152) x (BM x BN x K) / rate: pick the shape minimising that
  // (16 x 16 tiles pay ~5 % more for their shared-memory traffic per FMA).
  constexpr int kSMs = 152;
  auto units = [&](int bm, int bn) -> int64_t {
    const int tm = cdiv(g.M, bm), tn = cdiv(g.N, bn);
    int64_t u = 0;
    if (!g.out_lower) {
      u = (int64_t)tm * tn;
    } else {
      for (int r = 0; r < tm; ++r) u += std::min(tn, (r * bm + bm - 1) / bn + 1);
    }
    return u * g.batch;
  };
  auto cost = [&](int t, double pen) {
    const int64_t u = units(t, t);
    return (double)((u + kSMs - 1) / kSMs) * t * t * (1.0 + pen);
  };
  int bm = 0;   // 0: 16 x 64 tiles for M <= 16
  if (g.M > 16) {
    const double c64 = cost(64, 0.0), c32 = cost(32, 0.0), c16 = cost(16, 0.05);
    bm = 64;
    double best = c64;
    if (c32 < best) { bm = 32; best = c32; }
    if (c16 < best) { bm = 16; best = c16; }
  }
  if (bm == 0) {
    dim3 grid(cdiv(g.M, 16), cdiv(g.N, 64), g.batch);
    gemm_f64_kernel<16, 64><<<grid, NT, 0, s>>>(d);
  } else if (bm == 64) {
    dim3 grid(cdiv(g.M, 64), cdiv(g.N, 64), g.batch);
    gemm_f64_kernel<64, 64><<<grid, NT, 0, s>>>(d);
  } else if (bm == 32) {
    dim3 grid(cdiv(g.M, 32), cdiv(g.N, 32), g.batch);
    gemm_f64_kernel<32, 32><<<grid, NT, 0, s>>>(d);
  } else {
    dim3 grid(cdiv(g.M, 16), cdiv(g.N, 16), g.batch);
    gemm_f64_kernel<16, 16><<<grid, NT, 0, s>>>(d);
  }
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status gemv_f64(const Gemv& g, double* work, cudaStream_t s) {
  if (g.M <= 0) return BTA_OK;
  int nsplit = g.K >= 512 ? kGemvSplit : 1;
  if (g.K <= 0) nsplit = 1;
  if (!g.transA) {
    dim3 grid(cdiv(g.M, 128), nsplit);
    gemv_n_partial<<<grid, 128, 0, s>>>(g.M, g.K, g.A, g.lda, g.triA, g.x, work);
  } else {
    dim3 grid(cdiv((int64_t)g.M * 32, 256), nsplit);
    gemv_t_partial<<<grid, 256, 0, s>>>(g.M, g.K, g.A, g.lda, g.triA, g.x, work);
  }
  BTA_LAUNCHED();
  gemv_finish<<<cdiv(g.M, 256), 256, 0, s>>>(g.M, nsplit, work, g.alpha, g.beta,
                                               g.yin ? g.yin : g.y, g.y);
  BTA_LAUNCHED();
  return BTA_OK;
}

}  // namespace bta
