// Device-side model data and the internal kernels' entry points.
#pragma once

#include <vector>

#include "common.cuh"

namespace bta {

constexpr int kMaxK = 4;           // response variables supported
constexpr int kMaxD = 4 * kMaxK + kMaxK * (kMaxK - 1) / 2;
constexpr int kNS = 3;             // spatial base matrices: Cm, G, GG
constexpr int kNJ = 3;             // temporal base matrices: M0, M1, M2
constexpr int kNP = kNS + 1;       // pattern sums per variable pair: Cm, G, GG, counts

// Offsets (in doubles) inside the per-evaluation coefficient buffer.
struct CoefLayout {
  int k, d, nt;
  int theta, tau, coef, dcoef, alphaD, alphaB, total;
  void init(int k_, int d_, int nt_) {
    k = k_; d = d_; nt = nt_;
    int kk = k * k;
    theta = 0;
    tau = theta + d;
    coef = tau + k;                          // [kk][kNJ][kNS]
    dcoef = coef + kk * kNJ * kNS;           // [d][kk][kNJ][kNS]
    alphaD = dcoef + d * kk * kNJ * kNS;     // [nt][kk][kNS]
    alphaB = alphaD + nt * kk * kNS;         // [nt-1][kk][kNS]
    total = alphaB + (nt > 1 ? nt - 1 : 0) * kk * kNS;
  }
};

// Theta-independent model data resident on the device.
struct ModelDev {
  int k = 0, ns = 0, nt = 0, a = 0, a_r = 0, b = 0, ld = 0, d = 0, nnz = 0;
  int64_t n_obs = 0;
  double tip_prior = 1e-3, theta_prior_var = 100.0;
  int32_t* row_ptr = nullptr;   // [ns+1]
  int32_t* col = nullptr;       // [nnz]
  int32_t* row_of = nullptr;    // [nnz] CSR row of each entry
  double* val = nullptr;        // [kNS][nnz]
  double* m_diag = nullptr;     // [kNJ][nt]
  double* m_sub = nullptr;      // [kNJ][nt-1]
  double* cnt = nullptr;        // [nt*ld]   observations per latent node
  double* craw = nullptr;       // [nt][a x ld] covariate sums per latent node
  double* traw = nullptr;       // [k][a x a] covariate Gram per response
  double* rraw = nullptr;       // [nt*ld + a] A^T y (unscaled by tau)
  int32_t* obs_lat = nullptr;   // [n_obs] padded latent index t*ld + v*ns + s
  int32_t* obs_v = nullptr;     // [n_obs]
  double* obs_cov = nullptr;    // [n_obs * a_r]
  double* y = nullptr;          // [n_obs]
  std::vector<double> n_per_var;   // host
  std::vector<double> m_diag_h, m_sub_h;
};

// --- assemble.cu ------------------------------------------------------------
// Coefficients of the block expansion and their theta derivatives.
bta_status launch_coef(const ModelDev& md, const CoefLayout& L, double* coefbuf, cudaStream_t s);
// Dense BTA blocks of Q_p (cond = 0) or Q_c (cond = 1); rhs optional (cond only).
bta_status launch_assemble(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                           int cond, const bta_desc& q, double* rhs, cudaStream_t s);

// The one off-diagonal block B_i (= Q[i+1, i]) of Q_p, which Q_c shares, into
// dst (ld x ld); for sweeps that do not keep the B blocks.
bta_status launch_assemble_b(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                             int i, double* dst, cudaStream_t s);

// --- reduce.cu --------------------------------------------------------------
// Sizes of the per-block partial-sum arrays.
int pattern_chunks(const ModelDev& md);
int arrow_chunks(const ModelDev& md);
// Pattern inner products <Z^(pq), S> of one dense b x b block (Phase A/C).
// out: [k*k][chunks][kNP]
bta_status launch_pattern_dot(const ModelDev& md, const double* Z, int with_counts, int t,
                              double* out, cudaStream_t s);
// <Z_C, craw_t restricted to variable m> for all m.  out: [k][achunks]
bta_status launch_arrow_dot(const ModelDev& md, const double* ZC, int t, double* out,
                            cudaStream_t s);
// Stencil quadratic forms x_t^(p)T S x_u^(q).  out: [k*k][chunks][kNP]
bta_status launch_pattern_quad(const ModelDev& md, const double* xr, const double* xc,
                               double* out, cudaStream_t s);
// All of them for one mode x: QD[t] = x_t x_t forms, QB[t] = x_{t+1} x_t forms.
bta_status launch_pattern_quad_all(const ModelDev& md, const double* x, double* QD, double* QB,
                                  cudaStream_t s);
// Squared residuals per response.  out: [k][rchunks]
int resid_chunks(const ModelDev& md);
bta_status launch_residual(const ModelDev& md, const double* x, double* out, cudaStream_t s);

// Refinement of x*: r <- r - Q_c x in FP64 from the stencil form (no dense
// blocks: the factor has overwritten them), and y += alpha x.
bta_status launch_qc_residual(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                              const double* x, double* r, cudaStream_t s);
bta_status launch_axpy(int64_t n, double alpha, const double* x, double* y, cudaStream_t s);
// r = sum_m tau_m A_m^T y_m alone (n*ld + a).
bta_status launch_rhs(const ModelDev& md, const CoefLayout& L, const double* coefbuf, double* rhs,
                      cudaStream_t s);

// Everything the final combination reads.
struct Reductions {
  const double* PDc;   // [nt][kk][pchunks][kNP]     Z_D of Q_c
  const double* PBc;   // [nt-1][kk][pchunks][kNP]   Z_B of Q_c
  const double* PCc;   // [nt][k][achunks]           Z_C of Q_c against craw
  const double* ZTc;   // a x a (Z_T of Q_c, full)
  const double* PDp;   // [nt][kk][pchunks][kNP]     Z_D of Q_p
  const double* PBp;   // [nt-1][kk][pchunks][kNP]
  const double* QD;    // [nt][kk][pchunks][kNP]     x quad forms, same block
  const double* QB;    // [nt-1][kk][pchunks][kNP]   x_{t+1}, x_t
  const double* RS;    // [k][rchunks]               residual sums of squares
  const double* ldc;   // log|Q_c| partial slots
  int nldc;
  const double* ldp;   // log|Q_st| partial slots
  int nldp;
  const int32_t* failc;
  const int32_t* failp;
  const double* x;     // mode (for beta part of x^T Q_p x)
  int grad;
};
// out: [0] f, [1..d] grad, then parts (8) and phases (4*d).
bta_status launch_finalize(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                           const Reductions& r, double* out, cudaStream_t s);
constexpr int kOutParts = 8;
inline int out_size(int d) { return 1 + d + kOutParts + 4 * d; }

}  // namespace bta
