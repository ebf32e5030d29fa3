// Block sweeps over a BTA descriptor (sweep.cu).
#pragma once

#include "model.cuh"

namespace bta {

// Scratch for one sweep: three ld x ld blocks, the diagonal-factor scratch,
// two a x ld arrow blocks, GEMV partials and the arrow accumulator v_T.
struct SweepWs {
  double *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *pot = nullptr;
  double *Wc1 = nullptr, *Wc2 = nullptr, *gv = nullptr, *vT = nullptr;
  // mixed precision only: operand copies of the tensor-core products and
  // their status word (set by the owner, not by carve)
  void* tc = nullptr;
  int32_t* tcstat = nullptr;
  static size_t bytes(int ld, int a);
  void carve(double* base, int ld, int a);
};

// Fused Eq. 7 reductions for the selected-inversion sweep.
struct SelinvFuse {
  const ModelDev* md = nullptr;
  int counts = 0;          // add the observation-count diagonal (Q_c)
  double* PD = nullptr;    // [nt][kk][pchunks][kNP]
  double* PB = nullptr;    // [nt-1][kk][pchunks][kNP]
  double* PC = nullptr;    // [nt][k][achunks] or null
};

int logdet_slots(int n, int ld);   // n * (ld / 32) + 1 (tip)

// Emulated FP64 (precision 2) carries the arrow through the b x b products
// of both sweeps: its a rows ride along the rows of the product that shares
// their right-hand operand (in the row padding when b is not a multiple of
// 128), and its rank-a terms extend K, so that no FP64 product of the a x b
// arrow blocks with a b x b block is left per block step.
bool arrow_fused(int ld, int a, int precision);
// Bytes of the tensor-core workspace (SweepWs::tc) of a sweep of block size
// ld and arrow a in any precision, the arrow-extended products included.
size_t sweep_tc_ws_bytes(int ld, int a);

// One matrix of a set swept together.  All matrices of a set share n and ld;
// the arrow width may differ (Q_c with a > 0 next to the block-tridiagonal
// Q_p).  Every block step of the sweep is then one launch over the set.
struct SweepItem {
  bta_desc q{};
  double* vec = nullptr;           // factor: rhs -> z (or null); solves: z -> x
  double* slots = nullptr;         // factor: log-det slots
  int32_t* fail = nullptr;         // factor: failure flag (first failing block)
  SweepWs ws;
  const SelinvFuse* fuse = nullptr;   // selected inversion: fused Eq. 7 sums (or null)
  // Low-memory sweeps (q.B == nullptr): the off-diagonal factors L_Bi are not
  // kept; B_i is assembled from the model when a step needs it and L_Bi =
  // B_i L_Di^{-T} recomputed.  W4 (ld x ld) holds every other L_Bi of the
  // factor sweep.
  const ModelDev* md = nullptr;
  const CoefLayout* lay = nullptr;
  const double* coef = nullptr;
  double* W4 = nullptr;
};
// mark (optional): recorded on s right after block 0's diagonal factor, so a
// concurrent sweep can start one diagonal step behind this one.
// precision 0: every product in FP64; 1: the b x b off-diagonal Schur
// products (and the selected-inversion products) in split precision on the
// tensor cores, the diagonal-block factorisation, arrow and log-det in FP64.
// Block range (optional): blocks i0 <= i < i1 of the factor sweep (i1 < 0:
// to the end) and i_hi >= i >= i_lo of the selected inversion (i_hi < 0:
// from the last block), the set-up with the first block and the tip with
// the last, so that consecutive ranges issue exactly the whole sweep.  A
// caller interleaves two sweeps' ranges to create their operations (and the
// nodes of a captured graph) in alternation.
bta_status factor_sweep_multi(const SweepItem* items, int m, cudaStream_t s,
                              cudaEvent_t mark = nullptr, int precision = 0, int i0 = 0,
                              int i1 = -1);
bta_status upper_solve_multi(const SweepItem* items, int m, cudaStream_t s);
bta_status selinv_sweep_multi(const SweepItem* items, int m, cudaStream_t s, int precision = 0,
                              int i_hi = -1, int i_lo = 0);

bta_status factor_sweep(const bta_desc& q, double* rhs, double* slots, int32_t* fail,
                        const SweepWs& ws, cudaStream_t s, int precision = 0);
// d <- d - Q x for an assembled BTA matrix Q (D lower triangle referenced, B,
// C, T as in bta_desc); x, d: n*ld + a.  gv: GEMV work of kGemvSplit * ld.
bta_status bta_residual(const bta_desc& q, const double* x, double* d, double* gv,
                        cudaStream_t s);
bta_status lower_solve(const bta_desc& q, double* z, const SweepWs& ws, cudaStream_t s);
bta_status upper_solve(const bta_desc& q, double* z, const SweepWs& ws, cudaStream_t s);
bta_status tip_forward(const bta_desc& q, double* rT, const double* vT, cudaStream_t s);
bta_status selinv_sweep(const bta_desc& q, const SweepWs& ws, const SelinvFuse* fuse,
                        cudaStream_t s);

}  // namespace bta
