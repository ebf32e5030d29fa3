// Reductions of the gradient phases (Eq. 6) and of f (Eq. 1).
//
//  * Phase A / C (Eq. 7): every block Jacobian is a combination of the few
//    base stencils, dD_t/dth_k = sum_{pq,s} d alpha^D_{t,pq,s} S_s (plus the
//    count diagonal and the arrow for log tau), so tr(Z_D dD) reduces to the
//    stencil inner products <Z_D^(pq), S_s>, read only on the stencil
//    pattern (O(nnz) per block, independent of d).
//  * Phase B (Eq. 8): the same expansion turns x^T dQ_p x into stencil
//    quadratic forms x_t^(p)T S_s x_u^(q).
//  * log l: squared residuals y - A x* per response.
// All partial sums are written to fixed slots and summed in a fixed order,
// so results are bit-reproducible run to run.
#include <algorithm>
#include <cmath>

#include "model.cuh"

namespace bta {
namespace {

constexpr int RT = 256;

template <int NV>
__device__ void block_sum(double (&v)[NV], double* out, int stride) {
  __shared__ double sh[NV][RT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[i][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int j = 0; j < RT / 32; ++j) s += sh[threadIdx.x][j];
    out[threadIdx.x * stride] = s;
  }
}

struct PatArgs {
  int k, ns, ld, nnz;
  const int32_t* row_of;
  const int32_t* col;
  const double* val;
  const double* cnt;   // [ld] of this block, or null
};

// out[((pq * chunks) + chunk) * kNP + s]
__global__ void __launch_bounds__(RT) pattern_dot_kernel(PatArgs a, const double* __restrict__ Z,
                                                         double* out) {
  const int chunk = blockIdx.x, pq = blockIdx.y;
  const int p = pq / a.k, q = pq % a.k;
  const int e = chunk * RT + threadIdx.x;
  double v[kNP] = {0.0, 0.0, 0.0, 0.0};
  if (e < a.nnz) {
    int s2 = a.row_of[e], s1 = a.col[e];
    int r = p * a.ns + s1, c = q * a.ns + s2;
    double z = Z[r + (int64_t)c * a.ld];
    v[0] = z * a.val[e];
    v[1] = z * a.val[a.nnz + e];
    v[2] = z * a.val[2 * a.nnz + e];
    if (a.cnt && p == q && s1 == s2) v[3] = z * a.cnt[r];
  }
  block_sum<kNP>(v, out + ((int64_t)pq * gridDim.x + chunk) * kNP, 1);
}

__global__ void __launch_bounds__(RT) pattern_quad_kernel(PatArgs a, const double* __restrict__ xr,
                                                          const double* __restrict__ xc,
                                                          double* out) {
  const int chunk = blockIdx.x, pq = blockIdx.y;
  const int p = pq / a.k, q = pq % a.k;
  const int e = chunk * RT + threadIdx.x;
  double v[kNP] = {0.0, 0.0, 0.0, 0.0};
  if (e < a.nnz) {
    int s2 = a.row_of[e], s1 = a.col[e];
    double z = xr[p * a.ns + s1] * xc[q * a.ns + s2];
    v[0] = z * a.val[e];
    v[1] = z * a.val[a.nnz + e];
    v[2] = z * a.val[2 * a.nnz + e];
  }
  block_sum<kNP>(v, out + ((int64_t)pq * gridDim.x + chunk) * kNP, 1);
}

// All stencil quadratic forms of one mode x in one launch: blockIdx.z < n
// gives x_t^(p)T S x_t^(q) (into QD[t]), blockIdx.z = n + t gives
// x_{t+1}^(p)T S x_t^(q) (into QB[t]).
__global__ void __launch_bounds__(RT) pattern_quad_all_kernel(PatArgs a,
                                                              const double* __restrict__ x,
                                                              int ld, int n, double* QD,
                                                              double* QB) {
  const int chunk = blockIdx.x, pq = blockIdx.y;
  const int z = blockIdx.z;
  const bool diag = z < n;
  const int t = diag ? z : z - n;
  const double* xc = x + (int64_t)t * ld;
  const double* xr = diag ? xc : xc + ld;
  const int p = pq / a.k, q = pq % a.k;
  const int e = chunk * RT + threadIdx.x;
  double v[kNP] = {0.0, 0.0, 0.0, 0.0};
  if (e < a.nnz) {
    int s2 = a.row_of[e], s1 = a.col[e];
    double w = xr[p * a.ns + s1] * xc[q * a.ns + s2];
    v[0] = w * a.val[e];
    v[1] = w * a.val[a.nnz + e];
    v[2] = w * a.val[2 * a.nnz + e];
  }
  const int64_t per = (int64_t)a.k * a.k * gridDim.x * kNP;
  double* out = (diag ? QD : QB) + (int64_t)t * per;
  block_sum<kNP>(v, out + ((int64_t)pq * gridDim.x + chunk) * kNP, 1);
}

// <Z_C, craw> restricted to variable m: rows m*a_r.., columns m*ns..
__global__ void __launch_bounds__(RT) arrow_dot_kernel(int ns, int a, int a_r,
                                                       const double* __restrict__ ZC,
                                                       const double* __restrict__ craw,
                                                       double* out) {
  const int chunk = blockIdx.x, m = blockIdx.y;
  const int i = chunk * RT + threadIdx.x;
  double v[1] = {0.0};
  if (i < a_r * ns) {
    int f = m * a_r + i % a_r;
    int c = m * ns + i / a_r;
    int64_t idx = f + (int64_t)c * a;
    v[0] = ZC[idx] * craw[idx];
  }
  block_sum<1>(v, out + (int64_t)m * gridDim.x + chunk, 1);
}

__global__ void __launch_bounds__(RT) residual_kernel(int64_t n_obs, int per, int k, int a_r,
                                                      int64_t fe0, const int32_t* __restrict__ lat,
                                                      const int32_t* __restrict__ var,
                                                      const double* __restrict__ cov,
                                                      const double* __restrict__ y,
                                                      const double* __restrict__ x, double* out) {
  double v[kMaxK] = {0.0, 0.0, 0.0, 0.0};
  int64_t beg = (int64_t)blockIdx.x * per, end = min(n_obs, beg + per);
  for (int64_t j = beg + threadIdx.x; j < end; j += RT) {
    int m = var[j];
    double r = y[j] - x[lat[j]];
    const double* cj = cov + j * a_r;
    const double* beta = x + fe0 + (int64_t)m * a_r;
    for (int c = 0; c < a_r; ++c) r -= cj[c] * beta[c];
#pragma unroll
    for (int mm = 0; mm < kMaxK; ++mm)
      if (mm == m) v[mm] = fma(r, r, v[mm]);
  }
  block_sum<kMaxK>(v, out + blockIdx.x, gridDim.x);
}

struct FinArgs {
  int k, d, nt, a, a_r, ld, kk, pch, ach, rch, nldc, nldp, grad;
  double tip, pvar;
  const double* m_diag;
  const double* m_sub;
  const double* traw;
  double n_var[kMaxK];
  CoefLayout L;
  Reductions r;
};

// Sum over a warp (every lane gets the total).
__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kFinThreads = 1024;

// The combination of Eq. 1 and Eq. 6 from the per-block partial sums.  On
// GB300 every dependent FP64 add costs ~64 cycles, so each sum is split over
// the lanes of a warp (fixed order: the result is deterministic) and the
// warps take different sums.
__global__ void __launch_bounds__(kFinThreads) finalize_kernel(FinArgs a, const double* coefbuf,
                                                               double* out) {
  // R[j][pq][s] sums for Q_c (RDc), Q_p (RDp) and the mode's quadratic form (RX).
  __shared__ double RDc[kNJ][kMaxK * kMaxK][kNS], RDp[kNJ][kMaxK * kMaxK][kNS],
      RX[kNJ][kMaxK * kMaxK][kNS];
  __shared__ double CNT[kMaxK], PC[kMaxK], TT[kMaxK], RS[kMaxK], SL[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kk = a.kk, nt = a.nt, pch = a.pch, k = a.k;
  const Reductions& r = a.r;
  // (1) pattern sums: one warp per (array, pq, s), lanes over (block, chunk)
  for (int w = warp; w < 3 * kk * kNS; w += nw) {
    const int which = w / (kk * kNS), pq = (w / kNS) % kk, s = w % kNS;
    const double* PD = which == 0 ? r.PDc : which == 1 ? r.PDp : r.QD;
    const double* PB = which == 0 ? r.PBc : which == 1 ? r.PBp : r.QB;
    double acc[kNJ] = {0.0, 0.0, 0.0};
    if (which == 2 || a.grad) {
      const int nd = nt * pch, nb = (nt - 1) * pch;
      for (int u = lane; u < nd + nb; u += 32) {
        const bool isb = u >= nd;
        const int uu = isb ? u - nd : u, t = uu / pch, c = uu % pch;
        const double v = (isb ? PB : PD)[(((int64_t)t * kk + pq) * pch + c) * kNP + s];
#pragma unroll
        for (int j = 0; j < kNJ; ++j) {
          const double m = isb ? 2.0 * a.m_sub[j * (nt - 1) + t] : a.m_diag[j * nt + t];
          acc[j] = fma(m, v, acc[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kNJ; ++j) acc[j] = warp_total(acc[j]);
    }
    if (lane == 0)
      for (int j = 0; j < kNJ; ++j) {
        if (which == 0) RDc[j][pq][s] = acc[j];
        else if (which == 1) RDp[j][pq][s] = acc[j];
        else RX[j][pq][s] = acc[j];
      }
  }
  // (2) per response: counts, arrow and tip traces, residual sums; the two
  // log-determinant slot sums
  for (int w = warp; w < 4 * k + 2; w += nw) {
    double v = 0.0;
    if (w < 4 * k) {
      const int q = w / k, m = w % k;
      if (q == 0 && a.grad) {          // sum of the count-diagonal pattern term
        const int mm = m * k + m;
        for (int u = lane; u < nt * pch; u += 32) {
          const int t = u / pch, c = u % pch;
          v += r.PDc[(((int64_t)t * kk + mm) * pch + c) * kNP + 3];
        }
      } else if (q == 1 && a.grad && a.a > 0) {
        for (int u = lane; u < nt * a.ach; u += 32) {
          const int t = u / a.ach, c = u % a.ach;
          v += r.PCc[((int64_t)t * k + m) * a.ach + c];
        }
      } else if (q == 2 && a.grad && a.a > 0) {
        const double* tr = a.traw + (int64_t)m * a.a * a.a;
        for (int i = lane; i < a.a * a.a; i += 32) v = fma(r.ZTc[i], tr[i], v);
      } else if (q == 3) {
        for (int c = lane; c < a.rch; c += 32) v += r.RS[(int64_t)m * a.rch + c];
      }
      v = warp_total(v);
      if (lane == 0) {
        if (q == 0) CNT[m] = v;
        else if (q == 1) PC[m] = v;
        else if (q == 2) TT[m] = v;
        else RS[m] = v;
      }
    } else {
      const bool cond = w == 4 * k;
      const double* sl = cond ? r.ldc : r.ldp;
      const int ns = cond ? a.nldc : a.nldp;
      for (int i = lane; i < ns; i += 32) v += sl[i];
      v = warp_total(v);
      if (lane == 0) SL[cond ? 0 : 1] = v;
    }
  }
  __syncthreads();
  const CoefLayout& L = a.L;
  const double* th = coefbuf + L.theta;
  const double* tau = coefbuf + L.tau;
  const double* coef = coefbuf + L.coef;
  const double* dcoef = coefbuf + L.dcoef;
  const int d = a.d;
  double* parts = out + 1 + d;
  double* ph = parts + kOutParts;
  const int tau0 = d - k;
  const int nterm = kk * kNJ * kNS;
  if (warp == 0) {
    // (3) f of Eq. 1
    double quad = 0.0;
    for (int i = lane; i < nterm; i += 32) {
      const int pq = i / (kNJ * kNS), j = (i / kNS) % kNJ, s = i % kNS;
      quad = fma(coef[i], RX[j][pq][s], quad);
    }
    const double* beta = r.x + (int64_t)nt * a.ld;
    for (int i = lane; i < a.a; i += 32) quad += a.tip * beta[i] * beta[i];
    quad = warp_total(quad);
    if (lane == 0) {
      const double ldc = SL[0], ldp = SL[1] + a.a * log(a.tip);
      double ll = 0.0, lp = 0.0;
      for (int m = 0; m < k; ++m) ll += 0.5 * a.n_var[m] * log(tau[m]) - 0.5 * tau[m] * RS[m];
      for (int i = 0; i < d; ++i) lp -= th[i] * th[i] / (2.0 * a.pvar);
      const double f = 0.5 * ldp - 0.5 * ldc - 0.5 * quad + ll + lp;
      out[0] = f;
      parts[0] = ldp; parts[1] = ldc; parts[2] = quad; parts[3] = ll; parts[4] = lp;
      parts[5] = f;
      parts[6] = *r.failc; parts[7] = *r.failp;
    }
  } else {
    // (4) the gradient components of Eq. 6: one warp per component
    for (int kp = warp - 1; kp < d; kp += nw - 1) {
    double trc = 0.0, trp = 0.0, qx = 0.0;
    if (a.grad) {
      const double* dc = dcoef + (int64_t)kp * nterm;
      for (int i = lane; i < nterm; i += 32) {
        const int pq = i / (kNJ * kNS), j = (i / kNS) % kNJ, s = i % kNS;
        const double w = dc[i];
        trc = fma(w, RDc[j][pq][s], trc);
        trp = fma(w, RDp[j][pq][s], trp);
        qx = fma(w, RX[j][pq][s], qx);
      }
      trc = warp_total(trc);
      trp = warp_total(trp);
      qx = warp_total(qx);
    }
    if (lane == 0) {
      double expl = -th[kp] / a.pvar;
      if (kp >= tau0) {
        const int m = kp - tau0;
        trc += tau[m] * (CNT[m] + 2.0 * PC[m] + TT[m]);
        expl += 0.5 * a.n_var[m] - 0.5 * tau[m] * RS[m];
      }
      const double pa = -0.5 * trc, pb = -0.5 * qx, pcc = 0.5 * trp;
      ph[kp] = pa;
      ph[d + kp] = pb;
      ph[2 * d + kp] = pcc;
      ph[3 * d + kp] = expl;
      out[1 + kp] = a.grad ? pa + pb + pcc + expl : 0.0;
    }
    }
  }
}

}  // namespace

int pattern_chunks(const ModelDev& md) { return cdiv(md.nnz, RT); }
int arrow_chunks(const ModelDev& md) { return cdiv((int64_t)md.a_r * md.ns, RT); }
int resid_chunks(const ModelDev& md) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(2048, (md.n_obs + RT - 1) / RT));
}

bta_status launch_pattern_dot(const ModelDev& md, const double* Z, int with_counts, int t,
                              double* out, cudaStream_t s) {
  PatArgs a{md.k, md.ns, md.ld, md.nnz, md.row_of, md.col, md.val,
            with_counts ? md.cnt + (int64_t)t * md.ld : nullptr};
  pattern_dot_kernel<<<dim3(pattern_chunks(md), md.k * md.k), RT, 0, s>>>(a, Z, out);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_pattern_quad(const ModelDev& md, const double* xr, const double* xc,
                               double* out, cudaStream_t s) {
  PatArgs a{md.k, md.ns, md.ld, md.nnz, md.row_of, md.col, md.val, nullptr};
  pattern_quad_kernel<<<dim3(pattern_chunks(md), md.k * md.k), RT, 0, s>>>(a, xr, xc, out);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_pattern_quad_all(const ModelDev& md, const double* x, double* QD, double* QB,
                                  cudaStream_t s) {
  PatArgs a{md.k, md.ns, md.ld, md.nnz, md.row_of, md.col, md.val, nullptr};
  pattern_quad_all_kernel<<<dim3(pattern_chunks(md), md.k * md.k, 2 * md.nt - 1), RT, 0, s>>>(
      a, x, md.ld, md.nt, QD, QB);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_arrow_dot(const ModelDev& md, const double* ZC, int t, double* out,
                            cudaStream_t s) {
  arrow_dot_kernel<<<dim3(arrow_chunks(md), md.k), RT, 0, s>>>(
      md.ns, md.a, md.a_r, ZC, md.craw + (int64_t)t * md.a * md.ld, out);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_residual(const ModelDev& md, const double* x, double* out, cudaStream_t s) {
  int ch = resid_chunks(md);
  int per = (int)((md.n_obs + ch - 1) / ch);
  residual_kernel<<<ch, RT, 0, s>>>(md.n_obs, per, md.k, md.a_r, (int64_t)md.nt * md.ld,
                                    md.obs_lat, md.obs_v, md.obs_cov, md.y, x, out);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status launch_finalize(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                           const Reductions& r, double* out, cudaStream_t s) {
  FinArgs a{};
  a.k = md.k; a.d = md.d; a.nt = md.nt; a.a = md.a; a.a_r = md.a_r; a.ld = md.ld;
  a.kk = md.k * md.k; a.pch = pattern_chunks(md); a.ach = arrow_chunks(md);
  a.rch = resid_chunks(md); a.nldc = r.nldc; a.nldp = r.nldp; a.grad = r.grad;
  a.tip = md.tip_prior; a.pvar = md.theta_prior_var;
  a.m_diag = md.m_diag; a.m_sub = md.m_sub; a.traw = md.traw;
  for (int m = 0; m < kMaxK; ++m) a.n_var[m] = m < md.k ? md.n_per_var[m] : 0.0;
  a.L = L; a.r = r;
  finalize_kernel<<<1, kFinThreads, 0, s>>>(a, coefbuf, out);
  BTA_LAUNCHED();
  return BTA_OK;
}



// ----------------------------------------------------------------------------
// FP64 product with Q_c straight from its Kronecker/stencil form (no dense
// blocks), for the refinement of x* in the mixed-precision mode:
//   d = r - Q_c x.
// Block row t of Q_c x:  sum over t' in {t-1, t, t+1} of
//   sum_q sum_s alpha_{pq,s}(t, t') S_s x_t'^(q)  (+ tau_p cnt x_t on t' = t)
//   + C_t^T x_T;   tip row:  sum_t C_t x_t + T x_T.
// The temporal matrices are symmetric, so block (t, t+1) uses B_t's
// coefficients with p and q exchanged.
// ----------------------------------------------------------------------------
namespace {

struct QmvArgs {
  int k, ns, nt, ld, b, a, a_r, nnz;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* alphaD;   // [nt][kk][kNS]
  const double* alphaB;   // [nt-1][kk][kNS]
  const double* tau;
  const double* cnt;
  const double* craw;     // [nt][a x ld]
  const double* traw;     // [k][a x a]
  double tip;
};

__global__ void qc_residual_lat_kernel(QmvArgs g, const double* __restrict__ x, double* r) {
  const int t = blockIdx.y;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= g.ld) return;
  double* rt = r + (int64_t)t * g.ld;
  if (row >= g.b) { rt[row] = 0.0; return; }
  const int p = row / g.ns, s1 = row % g.ns;
  const int kk = g.k * g.k;
  double acc = 0.0;
  const int e0 = g.row_ptr[s1], e1 = g.row_ptr[s1 + 1];
  for (int dt = -1; dt <= 1; ++dt) {
    const int u = t + dt;
    if (u < 0 || u >= g.nt) continue;
    const double* xu = x + (int64_t)u * g.ld;
    for (int q = 0; q < g.k; ++q) {
      const double* al;
      if (dt == 0) al = g.alphaD + ((int64_t)t * kk + p * g.k + q) * kNS;
      else if (dt == -1) al = g.alphaB + ((int64_t)u * kk + p * g.k + q) * kNS;   // B_{t-1}
      else al = g.alphaB + ((int64_t)t * kk + q * g.k + p) * kNS;                  // B_t^T
      double sq = 0.0;
      for (int e = e0; e < e1; ++e) {
        const double w = al[0] * g.val[e] + al[1] * g.val[g.nnz + e] + al[2] * g.val[2 * g.nnz + e];
        sq = fma(w, xu[q * g.ns + g.col[e]], sq);
      }
      acc += sq;
    }
  }
  acc = fma(g.tau[p] * g.cnt[(int64_t)t * g.ld + row], x[(int64_t)t * g.ld + row], acc);
  if (g.a > 0) {
    const double* xT = x + (int64_t)g.nt * g.ld;
    const double* cr = g.craw + (int64_t)t * g.a * g.ld + (int64_t)row * g.a;
    for (int f = 0; f < g.a; ++f) acc = fma(g.tau[f / g.a_r] * cr[f], xT[f], acc);
  }
  rt[row] -= acc;
}

// Tip rows: one CTA per fixed effect f, deterministic block reduction.
__global__ void __launch_bounds__(RT) qc_residual_tip_kernel(QmvArgs g, const double* __restrict__ x,
                                                             double* r) {
  const int f = blockIdx.x;
  const double tf = g.tau[f / g.a_r];
  double v[1] = {0.0};
  const int64_t tot = (int64_t)g.nt * g.ld;
  for (int64_t i = threadIdx.x; i < tot; i += RT) {
    const int t = (int)(i / g.ld), row = (int)(i % g.ld);
    if (row >= g.b) continue;
    v[0] = fma(tf * g.craw[(int64_t)t * g.a * g.ld + (int64_t)row * g.a + f], x[i], v[0]);
  }
  __shared__ double res[1];
  block_sum<1>(v, res, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double* xT = x + tot;
    double acc = res[0];
    for (int h = 0; h < g.a; ++h) {
      double th = f == h ? g.tip : 0.0;   // T = tip I + sum_m tau_m traw_m
      for (int m = 0; m < g.k; ++m) th = fma(g.tau[m], g.traw[(int64_t)m * g.a * g.a + f + h * g.a], th);
      acc = fma(th, xT[h], acc);
    }
    r[tot + f] -= acc;
  }
}

__global__ void axpy_kernel(int64_t n, double alpha, const double* __restrict__ x, double* y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(alpha, x[i], y[i]);
}

}  // namespace

bta_status launch_qc_residual(const ModelDev& md, const CoefLayout& L, const double* coefbuf,
                              const double* x, double* r, cudaStream_t s) {
  QmvArgs g{md.k, md.ns, md.nt, md.ld, md.b, md.a, md.a_r, md.nnz, md.row_ptr, md.col, md.val,
            coefbuf + L.alphaD, coefbuf + L.alphaB, coefbuf + L.tau, md.cnt, md.craw, md.traw,
            md.tip_prior};
  qc_residual_lat_kernel<<<dim3(cdiv(md.ld, 128), md.nt), 128, 0, s>>>(g, x, r);
  BTA_LAUNCHED();
  if (md.a > 0) {
    qc_residual_tip_kernel<<<md.a, RT, 0, s>>>(g, x, r);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

bta_status launch_axpy(int64_t n, double alpha, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<(int)std::min<int64_t>(cdiv(n, 256), 1216), 256, 0, s>>>(n, alpha, x, y);
  BTA_LAUNCHED();
  return BTA_OK;
}

}  // namespace bta
