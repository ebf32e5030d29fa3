// Assembly of the BTA blocks of Q_p(theta) and Q_c(theta) (Section II-A,
// computational structure; Eq. 10 for the coregionalised super-blocks) and
// the closed-form theta-derivatives of their Kronecker coefficients
// (Eqs. 11-12), all on the device.
//
// Block expansion used everywhere:  for time blocks (t, t') with t' in
// {t, t-1} and variable pair (p, q),
//     Q^(pq)(t, t') = sum_j Mj[t, t'] sum_s coef[pq][j][s] S_s,
// with S_s in {Cm, G, GG} and, per variable m with unit scale,
//     u_m[0] = (kappa^4, 2 kappa^2, 1)        (M0 (x) K0)
//     u_m[1] = (2 kappa^3 gamma, 2 kappa gamma, 0)   (2 kappa gamma M1 (x) K1)
//     u_m[2] = (1, 0, 0)                      (M2 (x) Cm)
//     coef[pq][j][s] = sum_m W_pq^(m) u_m[j][s]   (k > 1),  e^{theta_1} u[j][s] (k = 1),
// W_pq^(m) = (Lambda^{-1})_{mp} (Lambda^{-1})_{mq}.
#include "model.cuh"

namespace bta {
namespace {

__device__ void unit_terms(double kap, double gam, double u[kNJ][kNS], double dk[kNJ][kNS],
                           double dg[kNJ][kNS]) {
  double k2 = kap * kap, k3 = k2 * kap, k4 = k2 * k2;
  for (int j = 0; j < kNJ; ++j)
    for (int s = 0; s < kNS; ++s) u[j][s] = dk[j][s] = dg[j][s] = 0.0;
  u[0][0] = k4;            dk[0][0] = 4 * k4;
  u[0][1] = 2 * k2;        dk[0][1] = 4 * k2;
  u[0][2] = 1.0;
  u[1][0] = 2 * k3 * gam;  dk[1][0] = 6 * k3 * gam;  dg[1][0] = 2 * k3 * gam;
  u[1][1] = 2 * kap * gam; dk[1][1] = 2 * kap * gam; dg[1][1] = 2 * kap * gam;
  u[2][0] = 1.0;
}

struct CoefArgs {
  int k, d, nt;
  const double* m_diag;
  const double* m_sub;
  CoefLayout L;
};

__global__ void coef_kernel(CoefArgs a, double* buf) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int k = a.k, d = a.d, kk = k * k;
  const CoefLayout& L = a.L;
  const double* th = buf + L.theta;
  double* tau = buf + L.tau;
  double* coef = buf + L.coef;
  double* dcoef = buf + L.dcoef;
  for (int i = 0; i < kk * kNJ * kNS; ++i) coef[i] = 0.0;
  for (int i = 0; i < d * kk * kNJ * kNS; ++i) dcoef[i] = 0.0;
  double u[kNJ][kNS], dk[kNJ][kNS], dg[kNJ][kNS];
  auto C = [&](int pq, int j, int s) -> double& { return coef[(pq * kNJ + j) * kNS + s]; };
  auto dC = [&](int p, int pq, int j, int s) -> double& {
    return dcoef[((p * kk + pq) * kNJ + j) * kNS + s];
  };
  if (k == 1) {
    double sc = exp(th[0]);
    unit_terms(exp(th[1]), exp(th[2]), u, dk, dg);
    for (int j = 0; j < kNJ; ++j)
      for (int s = 0; s < kNS; ++s) {
        C(0, j, s) = sc * u[j][s];
        dC(0, 0, j, s) = sc * u[j][s];
        dC(1, 0, j, s) = sc * dk[j][s];
        dC(2, 0, j, s) = sc * dg[j][s];
      }
    tau[0] = exp(th[3]);
  } else {
    const int nc = k * (k - 1) / 2;
    // Lambda (lower) and its inverse by forward substitution.
    double Lam[kMaxK][kMaxK], Li[kMaxK][kMaxK];
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Lam[i][j] = 0.0;
    for (int m = 0; m < k; ++m) Lam[m][m] = exp(th[2 * k + m]);
    {
      int c = 0;
      for (int p = 0; p < k; ++p)
        for (int q = 0; q < p; ++q) Lam[p][q] = th[3 * k + c++];
    }
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < k; ++i) Li[i][j] = 0.0;
      Li[j][j] = 1.0 / Lam[j][j];
      for (int i = j + 1; i < k; ++i) {
        double s = 0.0;
        for (int r = j; r < i; ++r) s += Lam[i][r] * Li[r][j];
        Li[i][j] = -s / Lam[i][i];
      }
    }
    for (int m = 0; m < k; ++m) {
      unit_terms(exp(th[m]), exp(th[k + m]), u, dk, dg);
      for (int p = 0; p < k; ++p)
        for (int q = 0; q < k; ++q) {
          double w = Li[m][p] * Li[m][q];
          int pq = p * k + q;
          for (int j = 0; j < kNJ; ++j)
            for (int s = 0; s < kNS; ++s) {
              C(pq, j, s) += w * u[j][s];
              dC(m, pq, j, s) += w * dk[j][s];        // d / d log kappa_m (Eq. 11)
              dC(k + m, pq, j, s) += w * dg[j][s];    // d / d log gamma_m (Eq. 11)
            }
        }
      // coupling-type parameters (Eq. 12): dLambda^{-1} = -Li E Li
      for (int c = 0; c < k + nc; ++c) {
        int er, ec;
        double ew;
        if (c < k) { er = ec = c; ew = Lam[c][c]; }
        else {
          int idx = c - k, cc = 0;
          er = ec = 0;
          for (int p = 0; p < k; ++p)
            for (int q = 0; q < p; ++q) {
              if (cc == idx) { er = p; ec = q; }
              ++cc;
            }
          ew = 1.0;
        }
        for (int p = 0; p < k; ++p)
          for (int q = 0; q < k; ++q) {
            double dLp = -ew * Li[m][er] * Li[ec][p];
            double dLq = -ew * Li[m][er] * Li[ec][q];
            double dw = dLp * Li[m][q] + Li[m][p] * dLq;
            int pq = p * k + q;
            for (int j = 0; j < kNJ; ++j)
              for (int s = 0; s < kNS; ++s) dC(2 * k + c, pq, j, s) += dw * u[j][s];
          }
      }
    }
    for (int m = 0; m < k; ++m) tau[m] = exp(th[3 * k + nc + m]);
  }
  // Per-block expansion coefficients.
  double* aD = buf + L.alphaD;
  double* aB = buf + L.alphaB;
  for (int t = 0; t < a.nt; ++t)
    for (int pq = 0; pq < kk; ++pq)
      for (int s = 0; s < kNS; ++s) {
        double vd = 0.0, vb = 0.0;
        for (int j = 0; j < kNJ; ++j) {
          vd += a.m_diag[j * a.nt + t] * C(pq, j, s);
          if (t + 1 < a.nt) vb += a.m_sub[j * (a.nt - 1) + t] * C(pq, j, s);
        }
        aD[(t * kk + pq) * kNS + s] = vd;
        if (t + 1 < a.nt) aB[(t * kk + pq) * kNS + s] = vb;
      }
}

struct AsmArgs {
  int k, ns, b, ld, nnz, cond, diag;
  int t0;                 // time block of output block 0 (coefficients, counts)
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;      // [kNS][nnz]
  const double* alpha;    // [nblk][kk][kNS]
  const double* tau;
  const double* cnt;      // [nt*ld]
};

// One CTA per column c of output block blockIdx.y (time block t0 + blockIdx.y):
// zero-fill, then scatter the stencil.
__global__ void __launch_bounds__(256) assemble_kernel(AsmArgs a, double* out) {
  const int c = blockIdx.x, t = a.t0 + blockIdx.y;
  const int ld = a.ld;
  double* colp = out + ((int64_t)blockIdx.y * ld + c) * ld;
  double2* col2 = reinterpret_cast<double2*>(colp);
  for (int r = threadIdx.x; r < ld / 2; r += blockDim.x) col2[r] = make_double2(0.0, 0.0);
  __syncthreads();
  if (c >= a.b) {
    if (a.diag && threadIdx.x == 0) colp[c] = 1.0;
    return;
  }
  const int q = c / a.ns, s2 = c % a.ns;
  const int e0 = a.row_ptr[s2], e1 = a.row_ptr[s2 + 1];
  const int kk = a.k * a.k;
  const double* al = a.alpha + (int64_t)t * kk * kNS;
  const int len = e1 - e0;
  for (int w = threadIdx.x; w < len * a.k; w += blockDim.x) {
    int p = w / len, e = e0 + w % len;
    int s1 = a.col[e];
    const double* ap = al + (p * a.k + q) * kNS;
    double v = ap[0] * a.val[e] + ap[1] * a.val[a.nnz + e] + ap[2] * a.val[2 * a.nnz + e];
    int r = p * a.ns + s1;
    if (a.cond && a.diag && r == c) v += a.tau[p] * a.cnt[(int64_t)t * ld + r];
    colp[r] = v;
  }
}

__global__ void assemble_arrow(int nt, int a, int ld, int ns, int a_r, const double* tau,
                               const double* craw, double* C) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t total = (int64_t)nt * a * ld;
  if (i >= total) return;
  int f = (int)(i % a);
  C[i] = tau[f / a_r] * craw[i];
}

__global__ void assemble_tip(int a, int k, double tip, const double* tau, const double* traw,
                             double* T) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a * a) return;
  double v = (i % a == i / a) ? tip : 0.0;
  for (int m = 0; m < k; ++m) v += tau[m] * traw[(int64_t)m * a * a + i];
  T[i] = v;
}

__global__ void assemble_rhs(int nt, int ld, int ns, int b, int a, int a_r, const double* tau,
                             const double* rraw, double* r) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t lat = (int64_t)nt * ld;
  if (i >= lat + a) return;
  int v;
  if (i < lat) {
    int row = (int)(i % ld);
    if (row >= b) { r[i] = 0.0; return; }
    v = row / ns;
  } else {
    v = (int)(i - lat) / a_r;
  }
  r[i] = tau[v] * rraw[i];
}

}  // namespace

bta_status launch_coef(const ModelDev& md, const CoefLayout& L, double* coefbuf, cudaStream_t s) {
  CoefArgs a{md.k, md.d, md.nt, md.m_diag, md.m_sub, L};
  coef_kernel<<<1, 32, 0, s>>>(a, coefbuf);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_rhs(const ModelDev& md, const CoefLayout& L, const double* coefbuf, double* rhs,
                      cudaStream_t s) {
  const int64_t tot = (int64_t)md.nt * md.ld + md.a;
  assemble_rhs<<<cdiv(tot, 256), 256, 0, s>>>(md.nt, md.ld, md.ns, md.b, md.a, md.a_r,
                                               coefbuf + L.tau, md.rraw, rhs);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_assemble(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                           int cond, const bta_desc& q, double* rhs, cudaStream_t s) {
  const int ld = md.ld;
  AsmArgs a{md.k, md.ns, md.b, ld, md.nnz, cond, 1, 0, md.row_ptr, md.col, md.val,
            coefbuf + L.alphaD, coefbuf + L.tau, md.cnt};
  assemble_kernel<<<dim3(ld, md.nt), 256, 0, s>>>(a, q.D);
  BTA_LAUNCHED();
  if (md.nt > 1 && q.B) {   // no B storage: the sweeps assemble B_i per step
    a.diag = 0;
    a.alpha = coefbuf + L.alphaB;
    assemble_kernel<<<dim3(ld, md.nt - 1), 256, 0, s>>>(a, q.B);
    BTA_LAUNCHED();
  }
  if (cond && md.a > 0) {
    int64_t tot = (int64_t)md.nt * md.a * ld;
    assemble_arrow<<<cdiv(tot, 256), 256, 0, s>>>(md.nt, md.a, ld, md.ns, md.a_r,
                                                  coefbuf + L.tau, md.craw, q.C);
    BTA_LAUNCHED();
    assemble_tip<<<cdiv(md.a * md.a, 256), 256, 0, s>>>(md.a, md.k, md.tip_prior,
                                                        coefbuf + L.tau, md.traw, q.T);
    BTA_LAUNCHED();
  }
  if (cond && rhs) {
    int64_t tot = (int64_t)md.nt * ld + md.a;
    assemble_rhs<<<cdiv(tot, 256), 256, 0, s>>>(md.nt, ld, md.ns, md.b, md.a, md.a_r,
                                                 coefbuf + L.tau, md.rraw, rhs);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

bta_status launch_assemble_b(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                             int i, double* dst, cudaStream_t s) {
  if (i < 0 || i >= md.nt - 1) return BTA_ERR_ARG;
  AsmArgs a{md.k, md.ns, md.b, md.ld, md.nnz, 0, 0, i, md.row_ptr, md.col, md.val,
            coefbuf + L.alphaB, coefbuf + L.tau, md.cnt};
  assemble_kernel<<<dim3(md.ld, 1), 256, 0, s>>>(a, dst);
  BTA_LAUNCHED();
  return BTA_OK;
}

}  // namespace bta
