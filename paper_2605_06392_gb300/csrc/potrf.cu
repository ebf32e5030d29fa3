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
#include <cstdlib>

#include "common.cuh"

namespace bta {
namespace {

constexpr int T = kPad;   // leaf size

// 32 x 32 leaf: A = L1 D L1^T (unit-lower L1) by right-looking elimination,
// with the inverse X = L1^{-1} built in the same steps (Gauss-Jordan on the
// unit factor), then L^{-1} = D^{-1/2} X and log|A| = sum log D_j.
//
// On GB300 every warp-wide FP64 instruction occupies its SM sub-partition's
// FP64 pipe for ~64 cycles, so the leaf is written to issue as few FP64
// instructions as possible on its serial chain: per step j,
//   (a) warp 0 scales column j once, l_ij = S_ij / D_j (one multiply per row,
//       with 1 / D_j computed once, by the thread that last updated D_j);
//   (b) every owned lower-triangle position (i, k), i > j, does one FMA:
//       the trailing matrix if k > j (S_ik -= l_ij S_kj), X otherwise
//       (X_ik -= l_ij X_jk).
// Step j reads only column j / row j, final after step j-1, so two
// barriers per step suffice.
constexpr int kLeafThreads = 128;
constexpr int kLeafPos = T * (T + 1) / 2;
constexpr int kLeafPer = (kLeafPos + kLeafThreads - 1) / kLeafThreads;

struct LeafDev {
  int ld;
  double* A[kMaxBatch];
  double* slot[kMaxBatch];
  int32_t* fail[kMaxBatch];
  int32_t code[kMaxBatch];
};

// One CTA per block of the batch (blockIdx.x).
__global__ void __launch_bounds__(kLeafThreads) potrf_inv_leaf(LeafDev dv) {
  double* A = dv.A[blockIdx.x];
  const int ld = dv.ld;
  __shared__ double S[T][T + 1];
  __shared__ double X[T][T + 1];
  __shared__ double lcol[T];
  __shared__ double rinv[T];   // 1 / D_j
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
  if (tid == 0) rinv[0] = 1.0 / S[0][0];
  __syncthreads();
  for (int j = 0; j < T; ++j) {
    if (tid > j && tid < T) lcol[tid] = S[tid][j] * rinv[j];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kLeafPer; ++r) {
      const int i = pi[r], k = pk[r];
      if (i > j) {
        const double lij = lcol[i];
        if (k > j) {
          const double v = fma(-lij, S[k][j], S[i][k]);
          S[i][k] = v;
          if (i == j + 1 && k == j + 1) rinv[j + 1] = 1.0 / v;   // D_{j+1} is final now
        } else {
          X[i][k] = fma(-lij, X[j][k], X[i][k]);
        }
      }
    }
    __syncthreads();
  }
  if (tid < T) rinv[tid] = 1.0 / sqrt(S[tid][tid]);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kLeafPer; ++r) {
    const int i = pi[r], k = pk[r];
    if (i >= 0) A[i + (int64_t)k * ld] = X[i][k] * rinv[i];
  }
  if (tid < 32) {
    const double dj = S[tid][tid];
    const bool bad = !(dj > 0.0) || !isfinite(dj);
    double l = bad ? 0.0 : log(dj);
#pragma unroll
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    const unsigned anybad = __ballot_sync(0xffffffffu, bad);
    if (tid == 0) {
      *dv.slot[blockIdx.x] = l;
      if (anybad) atomicCAS(dv.fail[blockIdx.x], -1, dv.code[blockIdx.x]);
    }
  }
}

// A batch of same-sized diagonal blocks factored together: every step of
// the recursion is one launch over all of them.
struct PB {
  int cnt;
  double* A[kMaxBatch];
  double* W[kMaxBatch];
  double* slots[kMaxBatch];
  int32_t* fail[kMaxBatch];
  int32_t code[kMaxBatch];
};

bta_status rec(const PB& b, int64_t aoff, int n, int ld, int64_t woff, int soff,
               cudaStream_t s) {
  const int cnt = b.cnt;
  if (n == T) {
    LeafDev dv;
    dv.ld = ld;
    for (int z = 0; z < cnt; ++z) {
      dv.A[z] = b.A[z] + aoff;
      dv.slot[z] = b.slots[z] + soff;
      dv.fail[z] = b.fail[z];
      dv.code[z] = b.code[z];
    }
    launch_prio(potrf_inv_leaf, dim3(cnt), dim3(kLeafThreads), s, dv);
    BTA_LAUNCHED();
    return BTA_OK;
  }
  const int p = n / T;
  const int n1 = (p / 2) * T, n2 = n - n1;
  const int64_t o11 = aoff, o21 = aoff + n1, o22 = aoff + n1 + (int64_t)n1 * ld;
  const int64_t w1 = woff, w2 = woff + (int64_t)n2 * n1;   // L21, L21 L11^{-1}
  const int64_t wsub = w2 + (int64_t)n2 * n1;              // scratch of the recursion
  const double* A11[kMaxBatch];
  const double* A21c[kMaxBatch];
  const double* A22c[kMaxBatch];
  double* A21[kMaxBatch];
  double* A22[kMaxBatch];
  double* W1[kMaxBatch];
  double* W2[kMaxBatch];
  const double* W1c[kMaxBatch];
  const double* W2c[kMaxBatch];
  for (int z = 0; z < cnt; ++z) {
    A11[z] = b.A[z] + o11;
    A21[z] = b.A[z] + o21;
    A21c[z] = A21[z];
    A22[z] = b.A[z] + o22;
    A22c[z] = A22[z];
    W1[z] = b.W[z] + w1;
    W2[z] = b.W[z] + w2;
    W1c[z] = W1[z];
    W2c[z] = W2[z];
  }
  BTA_TRY(rec(b, o11, n1, ld, wsub, soff, s));
  {  // L21 = A21 * (L11^{-1})^T
    Gemm g; g.M = n2; g.N = n1; g.K = n1; g.batch = cnt;
    g.Ab = A21c; g.lda = ld;
    g.Bb = A11; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;   // (lower W)^T is upper
    g.Cb = W1; g.ldc = n2;
    BTA_TRY(gemm_f64(g, s));
  }
  {  // A22 -= L21 L21^T (lower)
    Gemm g; g.M = n2; g.N = n2; g.K = n1; g.batch = cnt;
    g.Ab = W1c; g.lda = n2;
    g.Bb = W1c; g.ldb = n2; g.transB = 1;
    g.Cb = A22; g.ldc = ld; g.Cinb = A22c; g.ldcin = ld;
    g.alpha = -1.0; g.beta = 1.0; g.out_lower = 1;
    BTA_TRY(gemm_f64(g, s));
  }
  BTA_TRY(rec(b, o22, n2, ld, wsub, soff + n1 / T, s));
  {  // W2 = L21 * L11^{-1}
    Gemm g; g.M = n2; g.N = n1; g.K = n1; g.batch = cnt;
    g.Ab = W1c; g.lda = n2;
    g.Bb = A11; g.ldb = ld; g.triB = TRI_LOWER;
    g.Cb = W2; g.ldc = n2;
    BTA_TRY(gemm_f64(g, s));
  }
  {  // (L^{-1})21 = -L22^{-1} W2
    Gemm g; g.M = n2; g.N = n1; g.K = n2; g.batch = cnt;
    g.Ab = A22c; g.lda = ld; g.triA = TRI_LOWER;
    g.Bb = W2c; g.ldb = n2;
    g.Cb = A21; g.ldc = ld; g.alpha = -1.0;
    BTA_TRY(gemm_f64(g, s));
  }
  return BTA_OK;
}

// The products of one recursion level: batched FP64 (precision 0) or one
// emulated-FP64 product per block (8 BF16 slices; FP64 accuracy).
struct ProdCfg {
  int precision = 0;
  void* const* tcws = nullptr;
  int32_t* const* tcstat = nullptr;
  int leaf_ctas = 0;   // cap on the task-graph grid of the leaves (0: one CTA per SM)
};

bta_status level_product(const Gemm& g, const ProdCfg& c, cudaStream_t s) {
  if (c.precision == 0) return gemm_f64(g, s);
  for (int z = 0; z < g.batch; ++z) {
    Gemm one = g;
    one.batch = 1;
    one.Ab = nullptr; one.Bb = nullptr; one.Cb = nullptr; one.Cinb = nullptr;
    one.A = g.Ab[z]; one.B = g.Bb[z]; one.C = g.Cb[z];
    one.Cin = g.Cinb ? g.Cinb[z] : g.Cb[z];
    BTA_TRY(ozaki_gemm(one, c.tcws[z], c.tcstat[z], 8, s));
  }
  return BTA_OK;
}

// The 2 x 2 recursion of rec() above, stopped at blocks of at most `leaf`
// rows, which the task-graph kernel factors and inverts.  Those blocks hold
// a fraction (leaf / n)^2 of the b^3 / 3 + b^3 / 3 flops of the factor and
// the inverse; the rest are the four products of each level.
bta_status rec_hybrid(const PB& b, int64_t aoff, int n, int ld, int64_t woff, int soff,
                      int leaf, const ProdCfg& pc, cudaStream_t s, bool top = false) {
  const int cnt = b.cnt;
  if (n <= leaf && !top) {
    double* A[kMaxBatch];
    double* W[kMaxBatch];
    double* sl[kMaxBatch];
    for (int z = 0; z < cnt; ++z) {
      A[z] = b.A[z] + aoff;
      W[z] = b.W[z] + woff;
      sl[z] = b.slots[z] + soff;
    }
    return potrf_dag_batch(cnt, A, n, ld, W, sl, b.fail, b.code, s, pc.leaf_ctas,
                           pc.precision != 0);
  }
  const int p = n / T;
  const int n1 = (p / 2) * T, n2 = n - n1;
  const int64_t o11 = aoff, o21 = aoff + n1, o22 = aoff + n1 + (int64_t)n1 * ld;
  const int64_t w1 = woff, w2 = woff + (int64_t)n2 * n1;   // L21, L21 L11^{-1}
  const int64_t wsub = w2 + (int64_t)n2 * n1;              // scratch of the recursion
  const double* A11[kMaxBatch];
  const double* A22c[kMaxBatch];
  const double* A21c[kMaxBatch];
  double* A21[kMaxBatch];
  double* A22[kMaxBatch];
  double* W1[kMaxBatch];
  double* W2[kMaxBatch];
  const double* W1c[kMaxBatch];
  const double* W2c[kMaxBatch];
  for (int z = 0; z < cnt; ++z) {
    A11[z] = b.A[z] + o11;
    A21[z] = b.A[z] + o21;
    A21c[z] = A21[z];
    A22[z] = b.A[z] + o22;
    A22c[z] = A22[z];
    W1[z] = b.W[z] + w1;
    W2[z] = b.W[z] + w2;
    W1c[z] = W1[z];
    W2c[z] = W2[z];
  }
  BTA_TRY(rec_hybrid(b, o11, n1, ld, wsub, soff, leaf, pc, s));
  {  // L21 = A21 * (L11^{-1})^T
    Gemm g; g.M = n2; g.N = n1; g.K = n1; g.batch = cnt;
    g.Ab = A21c; g.lda = ld;
    g.Bb = A11; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
    g.Cb = W1; g.ldc = n2;
    BTA_TRY(level_product(g, pc, s));
  }
  {  // A22 -= L21 L21^T (lower)
    Gemm g; g.M = n2; g.N = n2; g.K = n1; g.batch = cnt;
    g.Ab = W1c; g.lda = n2;
    g.Bb = W1c; g.ldb = n2; g.transB = 1;
    g.Cb = A22; g.ldc = ld; g.Cinb = A22c; g.ldcin = ld;
    g.alpha = -1.0; g.beta = 1.0; g.out_lower = 1;
    BTA_TRY(level_product(g, pc, s));
  }
  BTA_TRY(rec_hybrid(b, o22, n2, ld, wsub, soff + n1 / T, leaf, pc, s));
  {  // W2 = L21 * L11^{-1}
    Gemm g; g.M = n2; g.N = n1; g.K = n1; g.batch = cnt;
    g.Ab = W1c; g.lda = n2;
    g.Bb = A11; g.ldb = ld; g.triB = TRI_LOWER;
    g.Cb = W2; g.ldc = n2;
    BTA_TRY(level_product(g, pc, s));
  }
  {  // (L^{-1})21 = -L22^{-1} W2
    Gemm g; g.M = n2; g.N = n1; g.K = n2; g.batch = cnt;
    g.Ab = A22c; g.lda = ld; g.triA = TRI_LOWER;
    g.Bb = W2c; g.ldb = n2;
    g.Cb = A21; g.ldc = ld; g.alpha = -1.0;
    BTA_TRY(level_product(g, pc, s));
  }
  return BTA_OK;
}

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

int potrf_hybrid_leaf(int precision) {
  // Largest block the task-graph kernel factors whole below the top level
  // (0: always whole).  Up to 1024 rows its serial chain of 32-row pivots
  // costs about as much as the split's extra products; above, the split wins
  // (measured on GB300: b = 2025 1.6x (emulated) and 1.9x (mixed) faster per
  // gradient, b = 4800 2.2x; FP64 b = 2025 1.4 %).
  static const int fp64 = env_int("BTA_POTRF_LEAF_FP64", 1024);
  static const int tc = env_int("BTA_POTRF_LEAF_TC", 1024);
  return precision == 0 ? fp64 : tc;
}

namespace {
// Blocks above this many rows are split at least once (tensor-core modes):
// with the emulated products a 1024-row block is faster as two 512-row
// task graphs (GB300: 157 -> 154 ms emulated, 142 -> 130 ms mixed per
// gradient of the b = 1024 model), while deeper splits of larger blocks lose.
int potrf_hybrid_top(int precision) {
  static const int tc = env_int("BTA_POTRF_SPLIT_TC", 512);
  return precision == 0 ? 0 : tc;
}
}  // namespace

bta_status potrf_inv_batch_prec(int count, double* const* A, int n, int ld,
                                double* const* scratch, double* const* logdet_parts,
                                int32_t* const* fail, const int32_t* fail_code, int precision,
                                void* const* tcws, int32_t* const* tcstat, cudaStream_t s) {
  if (n <= 0 || n % T || count < 0) return BTA_ERR_ARG;
  const int leaf = potrf_hybrid_leaf(precision);
  int top = potrf_hybrid_top(precision);
  if (top <= 0 || top > leaf) top = leaf;   // the top-level split threshold
  bool tc_ok = precision == 0 || (tcws && tcstat && n <= 5120);
  for (int z = 0; tc_ok && precision != 0 && z < count; ++z) tc_ok = tcws[z] && tcstat[z];
  if (leaf < T || top < T || n <= top || n < 2 * T || !tc_ok || n / T > 160 || g_potrf_recursive)
    return potrf_inv_batch(count, A, n, ld, scratch, logdet_parts, fail, fail_code, s);
  PriorityScope prio(highest_priority());
  ProdCfg pc;
  pc.precision = precision;
  // In the tensor-core modes the other sweep's products run on the SMs the
  // leaves leave free: ~3/7 of the SMs keep the leaves' bulk tasks off their
  // chain (GB300, b = 1024: mixed 126 -> 114 ms, emulated 134 -> 127 ms per
  // gradient; the FP64 mode, whose bulk tasks need the SMs, keeps them all).
  pc.leaf_ctas = precision ? std::max(2, sm_count() * 3 / 7) : 0;
  for (int z0 = 0; z0 < count; z0 += kMaxBatch) {
    PB b;
    b.cnt = count - z0 < kMaxBatch ? count - z0 : kMaxBatch;
    for (int z = 0; z < b.cnt; ++z) {
      b.A[z] = A[z0 + z];
      b.W[z] = scratch[z0 + z];
      b.slots[z] = logdet_parts[z0 + z];
      b.fail[z] = fail[z0 + z];
      b.code[z] = fail_code[z0 + z];
    }
    pc.tcws = tcws ? tcws + z0 : nullptr;
    pc.tcstat = tcstat ? tcstat + z0 : nullptr;
    BTA_TRY(rec_hybrid(b, 0, n, ld, 0, 0, (leaf / T) * T, pc, s, /*top=*/true));
  }
  return BTA_OK;
}

int potrf_inv_slots(int n) { return n / T; }

int g_potrf_recursive = 0;

bta_status potrf_inv_batch(int count, double* const* A, int n, int ld, double* const* scratch,
                           double* const* logdet_parts, int32_t* const* fail,
                           const int32_t* fail_code, cudaStream_t s) {
  if (n <= 0 || n % T || count < 0) return BTA_ERR_ARG;
  PriorityScope prio(highest_priority());   // the sweep's critical path
  if (count > 0 && n / T <= 160 && !g_potrf_recursive)
    return potrf_dag_batch(count, A, n, ld, scratch, logdet_parts, fail, fail_code, s);
  for (int z0 = 0; z0 < count; z0 += kMaxBatch) {
    PB b;
    b.cnt = count - z0 < kMaxBatch ? count - z0 : kMaxBatch;
    for (int z = 0; z < b.cnt; ++z) {
      b.A[z] = A[z0 + z];
      b.W[z] = scratch[z0 + z];
      b.slots[z] = logdet_parts[z0 + z];
      b.fail[z] = fail[z0 + z];
      b.code[z] = fail_code[z0 + z];
    }
    BTA_TRY(rec(b, 0, n, ld, 0, 0, s));
  }
  return BTA_OK;
}

bta_status potrf_inv(double* A, int n, int ld, double* scratch, double* logdet_parts,
                     int32_t* fail, int32_t fail_code, cudaStream_t s) {
  return potrf_inv_batch(1, &A, n, ld, &scratch, &logdet_parts, &fail, &fail_code, s);
}

}  // namespace bta
