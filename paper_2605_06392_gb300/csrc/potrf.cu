// Cholesky factor and its inverse for one dense SPD diagonal block (FP64).
//
// The BTA sweeps use L_Di only through L_Di^{-1}: the off-diagonal factors
// L_Bi = B_i L_Di^{-T} and L_Ci, the lower and upper solves (Algorithm 1,
// Eqs. 3-5) and the selected inversion all become products with L_Di^{-1},
// which parallelise over every output tile instead of running as
// column-sequential triangular solves.  This routine therefore overwrites
// the lower triangle of A with L^{-1} (A = L L^T) and records log|A|.
//
// Recursive formulation on a 2 x 2 split (n1 + n2), all big steps being
// tile-parallel products:
//     [A11      ]   L11 = chol(A11),         W = L11^{-1} (recursive)
//     [A21  A22 ]   L21 = A21 L11^{-T}
//                   A22 <- A22 - L21 L21^T,  L22^{-1} (recursive)
//                   (L^{-1})21 = -L22^{-1} L21 L11^{-1}
// with a single-CTA shared-memory kernel for 32 x 32 leaves.
#include <cmath>

#include "common.cuh"

namespace bta {
namespace {

constexpr int T = kPad;   // leaf size

// 32 x 32 leaf: A = L1 D L1^T (unit-lower L1) by right-looking elimination,
// with the inverse X = L1^{-1} built in the same steps (Gauss-Jordan on the
// unit factor), then L^{-1} = D^{-1/2} X and log|A| = sum log D_j.  Step j
// reads only column j of the trailing matrix and row j of X, both final at
// the end of step j-1, and writes only positions right of column j or below
// row j, so one barrier per step suffices.  Each of the 128 threads owns a
// fixed set of lower-triangle positions (i, k) and updates each of them once
// per step while i > j: the trailing matrix if k > j, X if k <= j.
constexpr int kLeafThreads = 128;
constexpr int kLeafPos = T * (T + 1) / 2;
constexpr int kLeafPer = (kLeafPos + kLeafThreads - 1) / kLeafThreads;

__global__ void __launch_bounds__(kLeafThreads) potrf_inv_leaf(double* A, int ld,
                                                               double* logdet_slot, int32_t* fail,
                                                               int32_t fail_code) {
  __shared__ double S[T][T + 1];
  __shared__ double X[T][T + 1];
  const int tid = threadIdx.x;
  int pi[kLeafPer], pk[kLeafPer];
#pragma unroll
  for (int r = 0; r < kLeafPer; ++r) {
    int p = tid + kLeafThreads * r;
    if (p < kLeafPos) {
      int i = 0;
      while ((i + 1) * (i + 2) / 2 <= p) ++i;
      pi[r] = i;
      pk[r] = p - i * (i + 1) / 2;
    } else {
      pi[r] = -1;
      pk[r] = 0;
    }
  }
  for (int e = tid; e < T * T; e += kLeafThreads) {
    int i = e % T, j = e / T;
    S[i][j] = (i >= j) ? A[i + (int64_t)j * ld] : 0.0;
    X[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < T; ++j) {
    const double invd = 1.0 / S[j][j];
#pragma unroll
    for (int r = 0; r < kLeafPer; ++r) {
      const int i = pi[r], k = pk[r];
      if (i > j) {
        const double lij = S[i][j] * invd;
        if (k > j) S[i][k] = fma(-lij, S[k][j], S[i][k]);
        else X[i][k] = fma(-lij, X[j][k], X[i][k]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kLeafPer; ++r) {
    const int i = pi[r], k = pk[r];
    if (i >= 0) A[i + (int64_t)k * ld] = X[i][k] / sqrt(S[i][i]);
  }
  if (tid < 32) {
    const double dj = S[tid][tid];
    const bool bad = !(dj > 0.0) || !isfinite(dj);
    double l = bad ? 0.0 : log(dj);
#pragma unroll
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (tid == 0) {
      *logdet_slot = l;
      if (anybad) atomicCAS(fail, -1, fail_code);
    }
  }
}

bta_status rec(double* A, int n, int ld, double* scratch, double* slots, int32_t* fail,
               int32_t fail_code, cudaStream_t s) {
  if (n == T) {
    potrf_inv_leaf<<<1, kLeafThreads, 0, s>>>(A, ld, slots, fail, fail_code);
    BTA_LAUNCHED();
    return BTA_OK;
  }
  int p = n / T;
  int n1 = (p / 2) * T, n2 = n - n1;
  double* A11 = A;
  double* A21 = A + n1;
  double* A22 = A + n1 + (int64_t)n1 * ld;
  double* W1 = scratch;                       // n2 x n1, ld n2 : L21
  double* W2 = scratch + (int64_t)n2 * n1;    // n2 x n1        : L21 L11^{-1}
  double* sub = W2 + (int64_t)n2 * n1;        // scratch for the recursion on A22
  BTA_TRY(rec(A11, n1, ld, sub, slots, fail, fail_code, s));
  {  // L21 = A21 * (L11^{-1})^T
    Gemm g; g.M = n2; g.N = n1; g.K = n1;
    g.A = A21; g.lda = ld;
    g.B = A11; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;   // (lower W)^T is upper
    g.C = W1; g.ldc = n2;
    BTA_TRY(gemm_f64(g, s));
  }
  {  // A22 -= L21 L21^T (lower)
    Gemm g; g.M = n2; g.N = n2; g.K = n1;
    g.A = W1; g.lda = n2;
    g.B = W1; g.ldb = n2; g.transB = 1;
    g.C = A22; g.ldc = ld; g.Cin = A22; g.ldcin = ld;
    g.alpha = -1.0; g.beta = 1.0; g.out_lower = 1;
    BTA_TRY(gemm_f64(g, s));
  }
  BTA_TRY(rec(A22, n2, ld, sub, slots + n1 / T, fail, fail_code, s));
  {  // W2 = L21 * L11^{-1}
    Gemm g; g.M = n2; g.N = n1; g.K = n1;
    g.A = W1; g.lda = n2;
    g.B = A11; g.ldb = ld; g.triB = TRI_LOWER;
    g.C = W2; g.ldc = n2;
    BTA_TRY(gemm_f64(g, s));
  }
  {  // (L^{-1})21 = -L22^{-1} W2
    Gemm g; g.M = n2; g.N = n1; g.K = n2;
    g.A = A22; g.lda = ld; g.triA = TRI_LOWER;
    g.B = W2; g.ldb = n2;
    g.C = A21; g.ldc = ld; g.alpha = -1.0;
    BTA_TRY(gemm_f64(g, s));
  }
  return BTA_OK;
}

}  // namespace

int potrf_inv_slots(int n) { return n / T; }

bta_status potrf_inv(double* A, int n, int ld, double* scratch, double* logdet_parts,
                     int32_t* fail, int32_t fail_code, cudaStream_t s) {
  if (n <= 0 || n % T) return BTA_ERR_ARG;
  return rec(A, n, ld, scratch, logdet_parts, fail, fail_code, s);
}

}  // namespace bta
