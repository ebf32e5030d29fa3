// The three block sweeps over a BTA matrix (FP64):
//   factor_sweep  -- Algorithm 1, fused block Cholesky + lower solve
//   upper_solve   -- Eqs. 3-5
//   selinv_sweep  -- selected inversion with the Eq. 7 traces fused in
// Each step is a handful of tile-parallel products on the whole GPU; the
// diagonal factor is kept as L_Di^{-1} (see potrf.cu).
#include <algorithm>
#include <cmath>

#include "sweep.cuh"

namespace bta {
namespace {

// Tip block (a x a, a <= kMaxTip) in one CTA: Cholesky, solves, inverse.
constexpr int kMaxTip = 32;

// mode 0: factor T in place (lower L_T, upper zeroed), logdet slot, and if
//         r != null: z_T = L_T^{-1} (r_T - v_T)  (written to r)
// mode 1: x_T = L_T^{-T} z_T in place (z)
// mode 2: T <- Z_T = L_T^{-T} L_T^{-1} (full)
__global__ void tip_kernel(int mode, int a, double* T, double* r, const double* vT,
                           double* logdet_slot, int32_t* fail, int32_t fail_code) {
  __shared__ double L[kMaxTip][kMaxTip + 1];
  __shared__ double v[kMaxTip];
  __shared__ int bad;
  if (threadIdx.x != 0) return;   // a is small; one thread keeps it exact and simple
  for (int j = 0; j < a; ++j)
    for (int i = 0; i < a; ++i) L[i][j] = T[i + j * a];
  bad = 0;
  if (mode == 0) {
    double ld = 0.0;
    for (int j = 0; j < a; ++j) {
      double dsum = L[j][j];
      for (int k = 0; k < j; ++k) dsum -= L[j][k] * L[j][k];
      if (!(dsum > 0.0) || !isfinite(dsum)) { bad = 1; dsum = 1.0; }
      double piv = sqrt(dsum);
      L[j][j] = piv;
      ld += log(piv);
      for (int i = j + 1; i < a; ++i) {
        double s = L[i][j];
        for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
        L[i][j] = s / piv;
      }
    }
    for (int j = 0; j < a; ++j)
      for (int i = 0; i < a; ++i) T[i + j * a] = i >= j ? L[i][j] : 0.0;
    *logdet_slot = 2.0 * ld;
    if (bad) atomicCAS(fail, -1, fail_code);
    if (r) {
      for (int i = 0; i < a; ++i) {
        double s = r[i] - vT[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * v[k];
        v[i] = s / L[i][i];
      }
      for (int i = 0; i < a; ++i) r[i] = v[i];
    }
  } else if (mode == 1) {
    for (int i = a - 1; i >= 0; --i) {
      double s = r[i];
      for (int k = i + 1; k < a; ++k) s -= L[k][i] * v[k];
      v[i] = s / L[i][i];
    }
    for (int i = 0; i < a; ++i) r[i] = v[i];
  } else {
    // W = L^{-1} (lower), then Z = W^T W
    __shared__ double W[kMaxTip][kMaxTip + 1];
    for (int c = 0; c < a; ++c) {
      for (int i = 0; i < c; ++i) W[i][c] = 0.0;
      W[c][c] = 1.0 / L[c][c];
      for (int i = c + 1; i < a; ++i) {
        double s = 0.0;
        for (int k = c; k < i; ++k) s += L[i][k] * W[k][c];
        W[i][c] = -s / L[i][i];
      }
    }
    for (int j = 0; j < a; ++j)
      for (int i = 0; i < a; ++i) {
        double s = 0.0;
        for (int k = (i > j ? i : j); k < a; ++k) s += W[k][i] * W[k][j];
        T[i + j * a] = s;
      }
  }
}

__global__ void copy_kernel(const double* __restrict__ src, int lds, double* __restrict__ dst,
                            int ldd, int rows, int cols, double alpha, int mode) {
  int64_t n = (int64_t)rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % rows), j = (int)(e / rows);
    double v;
    if (mode == 1 && i < j) v = src[j + (int64_t)i * lds];
    else v = src[i + (int64_t)j * lds];
    dst[i + (int64_t)j * ldd] = alpha * v;
  }
}

__global__ void fill_kernel(double* p, int64_t n, double v) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    p[e] = v;
}

__global__ void sum_kernel(const double* parts, int n, double* out, int acc) {
  if (threadIdx.x || blockIdx.x) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += parts[i];
  *out = acc ? *out + s : s;
}

}  // namespace

bta_status copy_block(const double* src, int lds, double* dst, int ldd, int rows, int cols,
                      double alpha, int mode, cudaStream_t s) {
  int64_t n = (int64_t)rows * cols;
  if (n <= 0) return BTA_OK;
  int grid = (int)std::min<int64_t>(cdiv(n, 256), 4 * 152 * 8);
  copy_kernel<<<grid, 256, 0, s>>>(src, lds, dst, ldd, rows, cols, alpha, mode);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status fill_value(double* p, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return BTA_OK;
  int grid = (int)std::min<int64_t>(cdiv(n, 256), 4 * 152 * 8);
  fill_kernel<<<grid, 256, 0, s>>>(p, n, v);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status sum_slots(const double* parts, int nparts, double* out, int accumulate,
                     cudaStream_t s) {
  sum_kernel<<<1, 32, 0, s>>>(parts, nparts, out, accumulate);
  BTA_LAUNCHED();
  return BTA_OK;
}

size_t SweepWs::bytes(int ld, int a) {
  size_t m = (size_t)ld * ld;
  return sizeof(double) * (4 * m + 2 * (size_t)a * ld + (size_t)kGemvSplit * ld + a + 64);
}

void SweepWs::carve(double* base, int ld, int a) {
  size_t m = (size_t)ld * ld;
  W1 = base;
  W2 = W1 + m;
  W3 = W2 + m;
  pot = W3 + m;
  Wc1 = pot + m;
  Wc2 = Wc1 + (size_t)a * ld;
  gv = Wc2 + (size_t)a * ld;
  vT = gv + (size_t)kGemvSplit * ld;
}

int logdet_slots(int n, int ld) { return n * potrf_inv_slots(ld) + 1; }

// ----------------------------------------------------------------------------
// Algorithm 1
// ----------------------------------------------------------------------------
bta_status factor_sweep(const bta_desc& q, double* rhs, double* slots, int32_t* fail,
                        const SweepWs& ws, cudaStream_t s) {
  const int n = q.n, ld = q.ld, a = q.a;
  const int64_t blk = (int64_t)ld * ld;
  const int p = potrf_inv_slots(ld);
  if (a > kMaxTip) return BTA_ERR_ARG;
  if (a > 0 && rhs) BTA_TRY(fill_value(ws.vT, a, 0.0, s));
  if (a > 0) BTA_TRY(fill_value(slots + (int64_t)n * p, 1, 0.0, s));
  else BTA_TRY(fill_value(slots + (int64_t)n * p, 1, 0.0, s));
  for (int i = 0; i < n; ++i) {
    double* Di = q.D + i * blk;
    double* Ci = a > 0 ? q.C + (int64_t)i * a * ld : nullptr;
    if (i > 0) {
      const double* Bp = q.B + (i - 1) * blk;
      {  // D_i -= S_{i-1} = L_B,i-1 L_B,i-1^T (lower)
        Gemm g; g.M = ld; g.N = ld; g.K = ld;
        g.A = Bp; g.lda = ld; g.B = Bp; g.ldb = ld; g.transB = 1;
        g.C = Di; g.ldc = ld; g.Cin = Di; g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
        g.out_lower = 1;
        BTA_TRY(gemm_f64(g, s));
      }
      if (a > 0) {  // C_i -= L_C,i-1 L_B,i-1^T
        Gemm g; g.M = a; g.N = ld; g.K = ld;
        g.A = q.C + (int64_t)(i - 1) * a * ld; g.lda = a;
        g.B = Bp; g.ldb = ld; g.transB = 1;
        g.C = Ci; g.ldc = a; g.Cin = Ci; g.ldcin = a; g.alpha = -1.0; g.beta = 1.0;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    // L_Di^{-1} in place, log-det slots
    BTA_TRY(potrf_inv(Di, ld, ld, ws.pot, slots + (int64_t)i * p, fail, i, s));
    if (a > 0) {  // L_Ci = C_i L_Di^{-T};  T -= L_Ci L_Ci^T
      Gemm g; g.M = a; g.N = ld; g.K = ld;
      g.A = Ci; g.lda = a; g.B = Di; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
      g.C = ws.Wc1; g.ldc = a;
      BTA_TRY(gemm_f64(g, s));
      BTA_TRY(copy_block(ws.Wc1, a, Ci, a, a, ld, 1.0, 0, s));
      Gemm h; h.M = a; h.N = a; h.K = ld;
      h.A = Ci; h.lda = a; h.B = Ci; h.ldb = a; h.transB = 1;
      h.C = q.T; h.ldc = a; h.Cin = q.T; h.ldcin = a; h.alpha = -1.0; h.beta = 1.0;
      BTA_TRY(gemm_f64(h, s));
    }
    if (i < n - 1) {  // L_Bi = B_i L_Di^{-T}
      double* Bi = q.B + i * blk;
      Gemm g; g.M = ld; g.N = ld; g.K = ld;
      g.A = Bi; g.lda = ld; g.B = Di; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
      g.C = ws.W1; g.ldc = ld;
      BTA_TRY(gemm_f64(g, s));
      BTA_TRY(copy_block(ws.W1, ld, Bi, ld, ld, ld, 1.0, 0, s));
    }
    if (rhs) {  // z_i = L_Di^{-1} (r_i - L_B,i-1 z_{i-1});  v_T += L_Ci z_i
      double* ri = rhs + (int64_t)i * ld;
      if (i > 0) {
        Gemv g; g.M = ld; g.K = ld; g.A = q.B + (i - 1) * blk; g.lda = ld;
        g.x = ri - ld; g.y = ri; g.yin = ri; g.alpha = -1.0; g.beta = 1.0;
        BTA_TRY(gemv_f64(g, ws.gv, s));
      }
      Gemv g; g.M = ld; g.K = ld; g.A = Di; g.lda = ld; g.triA = TRI_LOWER;
      g.x = ri; g.y = ri;
      BTA_TRY(gemv_f64(g, ws.gv, s));
      if (a > 0) {
        Gemv h; h.M = a; h.K = ld; h.A = Ci; h.lda = a; h.x = ri; h.y = ws.vT; h.yin = ws.vT;
        h.beta = 1.0;
        BTA_TRY(gemv_f64(h, ws.gv, s));
      }
    }
  }
  if (a > 0) {
    tip_kernel<<<1, 32, 0, s>>>(0, a, q.T, rhs ? rhs + (int64_t)n * ld : nullptr, ws.vT,
                                slots + (int64_t)n * p, fail, n);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

// ----------------------------------------------------------------------------
// Eqs. 3-5 (optionally preceded by the lower solve)
// ----------------------------------------------------------------------------
bta_status lower_solve(const bta_desc& q, double* z, const SweepWs& ws, cudaStream_t s) {
  const int n = q.n, ld = q.ld, a = q.a;
  const int64_t blk = (int64_t)ld * ld;
  if (a > 0) BTA_TRY(fill_value(ws.vT, a, 0.0, s));
  for (int i = 0; i < n; ++i) {
    double* ri = z + (int64_t)i * ld;
    if (i > 0) {
      Gemv g; g.M = ld; g.K = ld; g.A = q.B + (i - 1) * blk; g.lda = ld;
      g.x = ri - ld; g.y = ri; g.yin = ri; g.alpha = -1.0; g.beta = 1.0;
      BTA_TRY(gemv_f64(g, ws.gv, s));
    }
    Gemv g; g.M = ld; g.K = ld; g.A = q.D + i * blk; g.lda = ld; g.triA = TRI_LOWER;
    g.x = ri; g.y = ri;
    BTA_TRY(gemv_f64(g, ws.gv, s));
    if (a > 0) {
      Gemv h; h.M = a; h.K = ld; h.A = q.C + (int64_t)i * a * ld; h.lda = a; h.x = ri;
      h.y = ws.vT; h.yin = ws.vT; h.beta = 1.0;
      BTA_TRY(gemv_f64(h, ws.gv, s));
    }
  }
  if (a > 0) {
    // z_T = L_T^{-1}(r_T - v_T): reuse the tip kernel's solve on an already
    // factored tip by running the forward substitution alone.
    BTA_TRY(tip_forward(q, z + (int64_t)n * ld, ws.vT, s));
  }
  return BTA_OK;
}

namespace {
__global__ void tip_fwd_kernel(int a, const double* T, double* r, const double* vT) {
  if (threadIdx.x || blockIdx.x) return;
  double v[kMaxTip];
  for (int i = 0; i < a; ++i) {
    double s = r[i] - vT[i];
    for (int k = 0; k < i; ++k) s -= T[i + k * a] * v[k];
    v[i] = s / T[i + i * a];
  }
  for (int i = 0; i < a; ++i) r[i] = v[i];
}
}  // namespace

bta_status tip_forward(const bta_desc& q, double* rT, const double* vT, cudaStream_t s) {
  tip_fwd_kernel<<<1, 32, 0, s>>>(q.a, q.T, rT, vT);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status upper_solve(const bta_desc& q, double* z, const SweepWs& ws, cudaStream_t s) {
  const int n = q.n, ld = q.ld, a = q.a;
  const int64_t blk = (int64_t)ld * ld;
  double* xT = z + (int64_t)n * ld;
  if (a > 0) {
    tip_kernel<<<1, 32, 0, s>>>(1, a, q.T, xT, nullptr, nullptr, nullptr, 0);
    BTA_LAUNCHED();
  }
  for (int i = n - 1; i >= 0; --i) {
    double* zi = z + (int64_t)i * ld;
    if (a > 0) {  // z_i -= L_Ci^T x_T
      Gemv g; g.M = ld; g.K = a; g.A = q.C + (int64_t)i * a * ld; g.lda = a; g.transA = 1;
      g.x = xT; g.y = zi; g.yin = zi; g.alpha = -1.0; g.beta = 1.0;
      BTA_TRY(gemv_f64(g, ws.gv, s));
    }
    if (i < n - 1) {  // z_i -= L_Bi^T x_{i+1}
      Gemv g; g.M = ld; g.K = ld; g.A = q.B + i * blk; g.lda = ld; g.transA = 1;
      g.x = zi + ld; g.y = zi; g.yin = zi; g.alpha = -1.0; g.beta = 1.0;
      BTA_TRY(gemv_f64(g, ws.gv, s));
    }
    // x_i = L_Di^{-T} z_i
    Gemv g; g.M = ld; g.K = ld; g.A = q.D + i * blk; g.lda = ld; g.transA = 1;
    g.triA = TRI_UPPER; g.x = zi; g.y = zi;
    BTA_TRY(gemv_f64(g, ws.gv, s));
  }
  return BTA_OK;
}

// ----------------------------------------------------------------------------
// Selected inversion, in place, with the fused Eq. 7 reductions.
// With F_Bi = L_Bi L_Di^{-1}, F_Ci = L_Ci L_Di^{-1}:
//   Z_Ci = -Z_T F_Ci - Z_C,i+1 F_Bi
//   Z_Bi = -Z_D,i+1 F_Bi - Z_C,i+1^T F_Ci
//   Z_Di = L_Di^{-T} L_Di^{-1} - Z_Bi^T F_Bi - Z_Ci^T F_Ci
// ----------------------------------------------------------------------------
bta_status selinv_sweep(const bta_desc& q, const SweepWs& ws, const SelinvFuse* fuse,
                        cudaStream_t s) {
  const int n = q.n, ld = q.ld, a = q.a;
  const int64_t blk = (int64_t)ld * ld;
  if (a > 0) {
    tip_kernel<<<1, 32, 0, s>>>(2, a, q.T, nullptr, nullptr, nullptr, nullptr, 0);
    BTA_LAUNCHED();
  }
  for (int i = n - 1; i >= 0; --i) {
    double* Di = q.D + i * blk;
    double* Bi = i < n - 1 ? q.B + i * blk : nullptr;
    double* Ci = a > 0 ? q.C + (int64_t)i * a * ld : nullptr;
    const double* Dn = i < n - 1 ? q.D + (i + 1) * blk : nullptr;      // Z_D,i+1
    const double* Cn = (a > 0 && i < n - 1) ? q.C + (int64_t)(i + 1) * a * ld : nullptr;
    if (Bi) {  // W1 = F_B = L_Bi L_Di^{-1}
      Gemm g; g.M = ld; g.N = ld; g.K = ld;
      g.A = Bi; g.lda = ld; g.B = Di; g.ldb = ld; g.triB = TRI_LOWER;
      g.C = ws.W1; g.ldc = ld;
      BTA_TRY(gemm_f64(g, s));
    }
    if (a > 0) {
      {  // Wc1 = F_C = L_Ci L_Di^{-1}
        Gemm g; g.M = a; g.N = ld; g.K = ld;
        g.A = Ci; g.lda = a; g.B = Di; g.ldb = ld; g.triB = TRI_LOWER;
        g.C = ws.Wc1; g.ldc = a;
        BTA_TRY(gemm_f64(g, s));
      }
      {  // Wc2 = -Z_T F_C
        Gemm g; g.M = a; g.N = ld; g.K = a;
        g.A = q.T; g.lda = a; g.B = ws.Wc1; g.ldb = a;
        g.C = ws.Wc2; g.ldc = a; g.alpha = -1.0;
        BTA_TRY(gemm_f64(g, s));
      }
      if (Bi) {  // Wc2 -= Z_C,i+1 F_B
        Gemm g; g.M = a; g.N = ld; g.K = ld;
        g.A = Cn; g.lda = a; g.B = ws.W1; g.ldb = ld;
        g.C = ws.Wc2; g.ldc = a; g.Cin = ws.Wc2; g.ldcin = a; g.alpha = -1.0; g.beta = 1.0;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    if (Bi) {
      {  // W2 = Z_B = -Z_D,i+1 F_B
        Gemm g; g.M = ld; g.N = ld; g.K = ld;
        g.A = Dn; g.lda = ld; g.B = ws.W1; g.ldb = ld;
        g.C = ws.W2; g.ldc = ld; g.alpha = -1.0;
        BTA_TRY(gemm_f64(g, s));
      }
      if (a > 0) {  // W2 -= Z_C,i+1^T F_C
        Gemm g; g.M = ld; g.N = ld; g.K = a;
        g.A = Cn; g.lda = a; g.transA = 1; g.B = ws.Wc1; g.ldb = a;
        g.C = ws.W2; g.ldc = ld; g.Cin = ws.W2; g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    {  // W3 = L_Di^{-T} L_Di^{-1} (lower part)
      Gemm g; g.M = ld; g.N = ld; g.K = ld;
      g.A = Di; g.lda = ld; g.transA = 1; g.triA = TRI_UPPER;
      g.B = Di; g.ldb = ld; g.triB = TRI_LOWER;
      g.C = ws.W3; g.ldc = ld; g.out_lower = 1;
      BTA_TRY(gemm_f64(g, s));
    }
    if (Bi) {  // W3 -= Z_B^T F_B
      Gemm g; g.M = ld; g.N = ld; g.K = ld;
      g.A = ws.W2; g.lda = ld; g.transA = 1; g.B = ws.W1; g.ldb = ld;
      g.C = ws.W3; g.ldc = ld; g.Cin = ws.W3; g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
      g.out_lower = 1;
      BTA_TRY(gemm_f64(g, s));
    }
    if (a > 0) {  // W3 -= Z_C^T F_C
      Gemm g; g.M = ld; g.N = ld; g.K = a;
      g.A = ws.Wc2; g.lda = a; g.transA = 1; g.B = ws.Wc1; g.ldb = a;
      g.C = ws.W3; g.ldc = ld; g.Cin = ws.W3; g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
      g.out_lower = 1;
      BTA_TRY(gemm_f64(g, s));
    }
    BTA_TRY(copy_block(ws.W3, ld, Di, ld, ld, ld, 1.0, 1, s));       // Z_D (full)
    if (Bi) BTA_TRY(copy_block(ws.W2, ld, Bi, ld, ld, ld, 1.0, 0, s));
    if (a > 0) BTA_TRY(copy_block(ws.Wc2, a, Ci, a, a, ld, 1.0, 0, s));
    if (fuse) {
      const ModelDev& md = *fuse->md;
      const int kk = md.k * md.k, pch = pattern_chunks(md);
      BTA_TRY(launch_pattern_dot(md, Di, fuse->counts, i, fuse->PD + (int64_t)i * kk * pch * kNP,
                                 s));
      if (Bi)
        BTA_TRY(launch_pattern_dot(md, Bi, 0, i, fuse->PB + (int64_t)i * kk * pch * kNP, s));
      if (a > 0 && fuse->PC)
        BTA_TRY(launch_arrow_dot(md, Ci, i, fuse->PC + (int64_t)i * md.k * arrow_chunks(md), s));
    }
  }
  return BTA_OK;
}

}  // namespace bta
