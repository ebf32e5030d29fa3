// Shared definitions for the BTA / INLA CUDA library (sm_103a, FP64 path).
#pragma once

#include <cstdint>
#include <cstdio>
#include <utility>
#include <cuda_runtime.h>

#include "../../include/bta.h"

namespace bta {

// All block sizes are padded to a multiple of this tile (the padding holds the
// identity on diagonal blocks and zeros elsewhere).
constexpr int kPad = 32;

// Number of kernels launched by this library (process-wide and per model).
extern int64_t g_launches;

#define BTA_CUDA_TRY(expr)                                                    \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) {                                                  \
      fprintf(stderr, "[bta] %s failed: %s (%s:%d)\n", #expr,                 \
              cudaGetErrorString(_e), __FILE__, __LINE__);                    \
      return _e == cudaErrorMemoryAllocation ? BTA_ERR_NOMEM : BTA_ERR_CUDA;  \
    }                                                                         \
  } while (0)

#define BTA_TRY(expr)                                                         \
  do {                                                                        \
    bta_status _s = (expr);                                                   \
    if (_s != BTA_OK) return _s;                                              \
  } while (0)

// After a kernel launch: count it and surface launch-configuration errors.
#define BTA_LAUNCHED()                                                        \
  do {                                                                        \
    ++::bta::g_launches;                                                      \
    cudaError_t _e = cudaPeekAtLastError();                                   \
    if (_e != cudaSuccess) {                                                  \
      fprintf(stderr, "[bta] launch failed: %s (%s:%d)\n",                    \
              cudaGetErrorString(_e), __FILE__, __LINE__);                    \
      return BTA_ERR_CUDA;                                                    \
    }                                                                         \
  } while (0)

// Launch priority for the kernels on the sweeps' critical path (the
// diagonal-block factorisation): while set (PriorityScope), launches carry
// the device's highest stream priority as a launch attribute, so the
// scheduler places them ahead of the wide products of a concurrent sweep.
extern int g_launch_priority;   // 0: default priority
struct PriorityScope {
  int saved;
  explicit PriorityScope(int prio) : saved(g_launch_priority) { g_launch_priority = prio; }
  ~PriorityScope() { g_launch_priority = saved; }
};
int highest_priority();

// Launch a kernel with the current launch priority (cudaLaunchKernelEx) and
// `smem` bytes of dynamic shared memory.
template <class... KArgs, class... Args>
cudaError_t launch_prio_smem(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = g_launch_priority;
  cfg.attrs = attr;
  cfg.numAttrs = g_launch_priority ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
template <class... KArgs, class... Args>
cudaError_t launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                        Args&&... args) {
  return launch_prio_smem(kernel, grid, block, 0, s, std::forward<Args>(args)...);
}

inline int pad_ld(int b) { return (b + kPad - 1) / kPad * kPad; }

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount,
// queried once per device): grids and tile plans are sized in waves of it.
int sm_count();

// Bound of every globaltimer wait in the task-graph factor (ns; 2 s unless a
// test lowered it with bta_set_wait_limit), and the test switch that makes its
// chain wait on a counter nothing sets.
extern unsigned long long g_dag_wait_ns;
extern int g_dag_stall;
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ----------------------------------------------------------------------------
// Dense FP64 tile GEMM (gemm_f64.cu)
// C[M x N] = alpha * op(A) * op(B) + beta * Cin, column-major.
// tri flags mask the operand outside its triangle (the stored values there
// are ignored) and skip the all-zero K ranges.
// ----------------------------------------------------------------------------
enum Tri : int { TRI_NONE = 0, TRI_LOWER = 1, TRI_UPPER = 2 };

// Problems per batched launch (pointer arrays travel in the kernel parameters).
constexpr int kMaxBatch = 32;

struct Gemm {
  int M = 0, N = 0, K = 0;
  const double* A = nullptr; int lda = 0; int transA = 0; int triA = TRI_NONE;
  const double* B = nullptr; int ldb = 0; int transB = 0; int triB = TRI_NONE;
  double* C = nullptr; int ldc = 0;
  const double* Cin = nullptr; int ldcin = 0;   // may alias C; ignored when beta == 0
  double alpha = 1.0, beta = 0.0;
  int out_lower = 0;   // write only C[i][j] with i >= j (tiles above the diagonal skipped)
  // Batched: `batch` problems of the same shape; when batch > 1 the pointers
  // come from these host arrays (Cinb may be null: Cin = C) and A..Cin are
  // ignored.  Larger batches are split into launches of kMaxBatch.
  int batch = 1;
  const double* const* Ab = nullptr;
  const double* const* Bb = nullptr;
  double* const* Cb = nullptr;
  const double* const* Cinb = nullptr;
  // Optional split-K workspace (per problem, sk_cap doubles each): products
  // with too few output tiles then run as K chunks plus an ordered sum.
  double* sk_ws = nullptr;
  double* const* sk_wsb = nullptr;
  size_t sk_cap = 0;
  // Emulated products only (ozaki_gemm, batch 1; the other GEMMs refuse a
  // Gemm that sets any of these).  op(A) (M x K) and op(B) (K x N) as 2 x 2
  // block matrices: op(A) = [A, A12; A21, A22] with A's block a_rows x a_k,
  // op(B) = [B, B12; B21, B22] with B's block b_k x b_cols.  Each extra part
  // is a plain column-major matrix (op(part) = part, or its transpose when
  // trans is set); a null part is zero.  Only the leading blocks may be
  // triangular (triA / triB), and only in an operand without other parts.
  // C likewise in two row blocks: rows m < c_rows go to C / Cin (out_lower
  // applies there), rows m >= c_rows to C2 / Cin2 (ldc2, ldcin2; full).
  struct Part {
    const double* X = nullptr;
    int ld = 0, trans = 0;
  };
  Part A12, A21, A22, B12, B21, B22;
  int a_rows = 0, a_k = 0, b_k = 0, b_cols = 0;   // 0: the whole of M / K / N
  double* C2 = nullptr; int ldc2 = 0;
  const double* Cin2 = nullptr; int ldcin2 = 0;
  int c_rows = 0;
  bool blocked() const {
    return A12.X || A21.X || A22.X || B12.X || B21.X || B22.X || C2 || a_rows || a_k || b_k ||
           b_cols || c_rows;
  }
};
bta_status gemm_f64(const Gemm& g, cudaStream_t s);

// y[M] = alpha * op(A) x + beta * yin ; A column-major lda; tri masks A.
// Batched like Gemm: per-problem A, x, y, yin and GEMV work areas.
struct Gemv {
  int M = 0, K = 0;
  const double* A = nullptr; int lda = 0; int transA = 0; int triA = TRI_NONE;
  const double* x = nullptr;
  double* y = nullptr;
  const double* yin = nullptr;    // may alias y
  double alpha = 1.0, beta = 0.0;
  int batch = 1;
  const double* const* Ab = nullptr;
  const double* const* xb = nullptr;
  double* const* yb = nullptr;
  const double* const* yinb = nullptr;   // null: yin = y
  double* const* workb = nullptr;
};
bta_status gemv_f64(const Gemv& g, double* work, cudaStream_t s);
constexpr int kGemvSplit = 16;      // K splits; work needs kGemvSplit * M doubles

// Split-precision (3xTF32) tensor-core GEMM (tc_gemm.cu): same contract as
// gemm_f64 for a single problem; ws holds tc_gemm_ws_bytes(M, N, K) bytes;
// *status (device, may be null) receives BTA_ERR_TIMEOUT if a bounded wait
// inside the kernel expired.
// While one is open on this thread, gemm_f64 times each not yet measured
// product shape's tile candidates on scratch operands and keeps the fastest
// (outside stream capture only).
struct TuneScope {
  TuneScope();
  ~TuneScope();
};

bta_status tc_gemm_mixed(const Gemm& g, void* ws, int32_t* status, cudaStream_t s);
size_t tc_gemm_ws_bytes(int M, int N, int K);
// FP64 GEMM emulated on BF16 tensor cores with `slices` (6..8) base-128
// digits per operand (ozaki_gemm.cu); single problem, K <= kOzakiMaxK.
constexpr int kOzakiMaxK = 5120;   // keeps the 64-bit integer sums below 2^62.4
// marks (optional): events recorded around the tensor-core product kernel.
bta_status ozaki_gemm(const Gemm& g, void* ws, int32_t* status, int slices, cudaStream_t s,
                      const cudaEvent_t* marks = nullptr);
size_t ozaki_ws_bytes(int M, int N, int K, int slices);
bool ozaki_supported(const Gemm& g);

// ----------------------------------------------------------------------------
// Diagonal-block Cholesky + inverse (potrf.cu)
// On return the lower triangle of A (n x n, ld) holds L^{-1} where A = L L^T;
// logdet_parts[slot0 + j] receives 2 sum log diag over base tile j;
// *fail receives `fail_code` if a pivot was not positive.
// scratch: at least n*n doubles.
// ----------------------------------------------------------------------------
bta_status potrf_inv(double* A, int n, int ld, double* scratch, double* logdet_parts,
                     int32_t* fail, int32_t fail_code, cudaStream_t s);
// The same on `count` blocks of one size at once (host arrays of per-block
// pointers and failure codes).
bta_status potrf_inv_batch(int count, double* const* A, int n, int ld, double* const* scratch,
                           double* const* logdet_parts, int32_t* const* fail,
                           const int32_t* fail_code, cudaStream_t s);
int potrf_inv_slots(int n);   // number of logdet slots potrf_inv writes
// The same with the precision of the sweep: above potrf_hybrid_leaf(precision)
// rows the block is split 2 x 2 recursively, the diagonal sub-blocks factored
// by the task-graph kernel and the products of each level run in FP64
// (precision 0) or emulated FP64 (precision 1, 2; per-block workspace tcws of
// ozaki_ws_bytes(n, n, n, 8) bytes and status words tcstat).
bta_status potrf_inv_batch_prec(int count, double* const* A, int n, int ld,
                                double* const* scratch, double* const* logdet_parts,
                                int32_t* const* fail, const int32_t* fail_code, int precision,
                                void* const* tcws, int32_t* const* tcstat, cudaStream_t s);
int potrf_hybrid_leaf(int precision);
// The task-graph kernel (potrf_dag.cu) used by potrf_inv_batch for n <= 5120;
// g_potrf_recursive = 1 selects the recursive launch sequence instead.
// max_ctas > 0 caps the persistent grid (at least 2: the chain and a bulk CTA).
// tc = 1: the 32 x 32 tile products emulated in FP64 from BF16 slices on the
// tensor cores (the tensor-core modes); 0: FP64 FMAs.
bta_status potrf_dag_batch(int count, double* const* A, int n, int ld, double* const* scratch,
                           double* const* logdet_parts, int32_t* const* fail,
                           const int32_t* fail_code, cudaStream_t s, int max_ctas = 0,
                           int tc = 0);
extern int g_potrf_recursive;

// Small helpers (sweep.cu)
bta_status copy_block(const double* src, int lds, double* dst, int ldd, int rows, int cols,
                      double alpha, int mode, cudaStream_t s);  // mode 0 copy, 1 mirror lower->full
bta_status copy_block_batch(int count, const double* const* src, int lds, double* const* dst,
                            int ldd, int rows, int cols, double alpha, int mode, cudaStream_t s);
bta_status fill_value(double* p, int64_t n, double v, cudaStream_t s);
bta_status sum_slots(const double* parts, int nparts, double* out, int accumulate,
                     cudaStream_t s);

}  // namespace bta
