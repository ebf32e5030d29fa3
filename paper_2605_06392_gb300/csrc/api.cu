// C ABI: model set-up, the bta_* descriptor calls and inla_value_and_grad.
//
// inla_value_and_grad runs, for one theta (Eq. 1 and Eq. 6):
//   stream 0 : theta -> coefficients (closed-form Kronecker coefficients and
//              their theta-derivatives)
//   stream 1 : assemble Q_c, r -> Algorithm 1 with fused lower solve ->
//              Eqs. 3-5 -> x*, residuals ->  [grad] selected inversion of Q_c
//              with Phase A fused
//   stream 2 : assemble Q_p -> block Cholesky -> (after x*) stencil quadratic
//              forms (Phase B, x*^T Q_p x*) -> [grad] selected inversion of Q_p
//              with Phase C fused
//   stream 0 : join, final combination into f and grad.
// The two factorisations and the two selected inversions are independent, so
// they run concurrently and fill each other's idle SMs.  The whole evaluation
// is captured once into a CUDA graph per (value / value+grad) and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sweep.cuh"

using namespace bta;

struct inla_model {
  ModelDev md;
  CoefLayout L;
  int n = 0, b = 0, ld = 0, a = 0, d = 0;
  int nslots = 0, nslots_p = 0;
  // device buffers (model-owned)
  double* coefbuf = nullptr;
  bta_desc qc{}, qp{};
  double* x = nullptr;          // r -> z -> x*  (n*ld + a)
  double* slots_c = nullptr;
  double* slots_p = nullptr;
  int32_t* fail = nullptr;      // [2]
  double *PDc = nullptr, *PBc = nullptr, *PCc = nullptr, *PDp = nullptr, *PBp = nullptr;
  double *QD = nullptr, *QB = nullptr, *RS = nullptr;
  double* out = nullptr;
  double* wsbuf = nullptr;
  SweepWs wsc, wsp;
  std::vector<void*> allocs;
  // host
  double* hout = nullptr;       // pinned
  double* htheta = nullptr;     // pinned
  std::vector<double> last;
  // concurrency
  cudaStream_t s1 = nullptr, s2 = nullptr;
  cudaEvent_t ev0 = nullptr, evx = nullptr, ev1 = nullptr, ev2 = nullptr;
  cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};   // value, value+grad, backward
  int64_t graph_kernels[3] = {0, 0, 0};
  int have_factors = 0;         // last evaluation was value-only: factors still held
  int64_t launched = 0;         // kernels this model ran (graph replays included)
};

namespace {

template <class T>
bta_status dmalloc(inla_model* m, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) { *p = nullptr; return BTA_OK; }
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BTA_ERR_NOMEM;
  }
  m->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return BTA_OK;
}

template <class T>
bta_status upload(inla_model* m, T** p, const T* host, size_t count) {
  BTA_TRY(dmalloc(m, p, count));
  if (count) BTA_CUDA_TRY(cudaMemcpy(*p, host, count * sizeof(T), cudaMemcpyHostToDevice));
  return BTA_OK;
}

bool finite_theta(const double* th, int d) {
  for (int i = 0; i < d; ++i)
    if (!std::isfinite(th[i])) return false;
  return true;
}

// Record one evaluation (grad = 0/1) on stream s0; theta already in coefbuf.
bta_status record_eval(inla_model* m, int grad, cudaStream_t s0) {
  const ModelDev& md = m->md;
  const int n = m->n, ld = m->ld, kk = md.k * md.k, pch = pattern_chunks(md);
  BTA_TRY(launch_coef(md, m->L, m->coefbuf, s0));
  BTA_CUDA_TRY(cudaMemsetAsync(m->fail, 0xff, 2 * sizeof(int32_t), s0));
  BTA_CUDA_TRY(cudaEventRecord(m->ev0, s0));
  // ---- stream 1: Q_c
  BTA_CUDA_TRY(cudaStreamWaitEvent(m->s1, m->ev0, 0));
  m->qc.state = BTA_STATE_EMPTY;
  BTA_TRY(launch_assemble(md, m->L, m->coefbuf, 1, m->qc, m->x, m->s1));
  BTA_TRY(factor_sweep(m->qc, m->x, m->slots_c, m->fail, m->wsc, m->s1));
  BTA_TRY(upper_solve(m->qc, m->x, m->wsc, m->s1));
  BTA_CUDA_TRY(cudaEventRecord(m->evx, m->s1));
  BTA_TRY(launch_residual(md, m->x, m->RS, m->s1));
  if (grad) {
    SelinvFuse fz;
    fz.md = &md; fz.counts = 1; fz.PD = m->PDc; fz.PB = m->PBc; fz.PC = m->PCc;
    BTA_TRY(selinv_sweep(m->qc, m->wsc, &fz, m->s1));
  }
  BTA_CUDA_TRY(cudaEventRecord(m->ev1, m->s1));
  // ---- stream 2: Q_p
  BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->ev0, 0));
  BTA_TRY(launch_assemble(md, m->L, m->coefbuf, 0, m->qp, nullptr, m->s2));
  BTA_TRY(factor_sweep(m->qp, nullptr, m->slots_p, m->fail + 1, m->wsp, m->s2));
  BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->evx, 0));
  for (int t = 0; t < n; ++t) {
    const double* xt = m->x + (int64_t)t * ld;
    BTA_TRY(launch_pattern_quad(md, xt, xt, m->QD + (int64_t)t * kk * pch * kNP, m->s2));
    if (t + 1 < n)
      BTA_TRY(launch_pattern_quad(md, xt + ld, xt, m->QB + (int64_t)t * kk * pch * kNP, m->s2));
  }
  if (grad) {
    SelinvFuse fz;
    fz.md = &md; fz.counts = 0; fz.PD = m->PDp; fz.PB = m->PBp; fz.PC = nullptr;
    BTA_TRY(selinv_sweep(m->qp, m->wsp, &fz, m->s2));
  }
  BTA_CUDA_TRY(cudaEventRecord(m->ev2, m->s2));
  // ---- join
  BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev1, 0));
  BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev2, 0));
  Reductions r{};
  r.PDc = m->PDc; r.PBc = m->PBc; r.PCc = m->PCc; r.ZTc = m->qc.T;
  r.PDp = m->PDp; r.PBp = m->PBp; r.QD = m->QD; r.QB = m->QB; r.RS = m->RS;
  r.ldc = m->slots_c; r.nldc = m->nslots; r.ldp = m->slots_p; r.nldp = m->nslots_p;
  r.failc = m->fail; r.failp = m->fail + 1; r.x = m->x; r.grad = grad;
  BTA_TRY(launch_finalize(md, m->L, m->coefbuf, r, m->out, s0));
  return BTA_OK;
}

// Backward only: the two selected inversions on the factors a value-only
// evaluation left in place, then the final combination with grad on.
bta_status record_backward(inla_model* m, cudaStream_t s0) {
  const ModelDev& md = m->md;
  BTA_CUDA_TRY(cudaEventRecord(m->ev0, s0));
  BTA_CUDA_TRY(cudaStreamWaitEvent(m->s1, m->ev0, 0));
  SelinvFuse fc;
  fc.md = &md; fc.counts = 1; fc.PD = m->PDc; fc.PB = m->PBc; fc.PC = m->PCc;
  BTA_TRY(selinv_sweep(m->qc, m->wsc, &fc, m->s1));
  BTA_CUDA_TRY(cudaEventRecord(m->ev1, m->s1));
  BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->ev0, 0));
  SelinvFuse fp;
  fp.md = &md; fp.counts = 0; fp.PD = m->PDp; fp.PB = m->PBp; fp.PC = nullptr;
  BTA_TRY(selinv_sweep(m->qp, m->wsp, &fp, m->s2));
  BTA_CUDA_TRY(cudaEventRecord(m->ev2, m->s2));
  BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev1, 0));
  BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev2, 0));
  Reductions r{};
  r.PDc = m->PDc; r.PBc = m->PBc; r.PCc = m->PCc; r.ZTc = m->qc.T;
  r.PDp = m->PDp; r.PBp = m->PBp; r.QD = m->QD; r.QB = m->QB; r.RS = m->RS;
  r.ldc = m->slots_c; r.nldc = m->nslots; r.ldp = m->slots_p; r.nldp = m->nslots_p;
  r.failc = m->fail; r.failp = m->fail + 1; r.x = m->x; r.grad = 1;
  BTA_TRY(launch_finalize(md, m->L, m->coefbuf, r, m->out, s0));
  return BTA_OK;
}

// mode 0: value, 1: value + grad, 2: backward of the last value-only call.
bta_status run_eval(inla_model* m, const double* theta, int mode, int use_graph,
                    cudaStream_t stream) {
  const int d = m->d;
  const int grad = mode;
  if (mode < 2) {
    std::memcpy(m->htheta, theta, d * sizeof(double));
    BTA_CUDA_TRY(cudaMemcpyAsync(m->coefbuf + m->L.theta, m->htheta, d * sizeof(double),
                                 cudaMemcpyHostToDevice, stream));
  }
  auto rec = [&](cudaStream_t s0) {
    return mode < 2 ? record_eval(m, mode, s0) : record_backward(m, s0);
  };
  if (use_graph) {
    if (!m->gexec[grad]) {
      const int64_t before = g_launches;
      cudaStream_t cap;
      BTA_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      BTA_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      bta_status st = rec(cap);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap, &graph);
      if (st != BTA_OK) { if (graph) cudaGraphDestroy(graph); cudaStreamDestroy(cap); return st; }
      BTA_CUDA_TRY(e);
      e = cudaGraphInstantiate(&m->gexec[grad], graph, 0);
      cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      BTA_CUDA_TRY(e);
      m->graph_kernels[grad] = g_launches - before;
    }
    BTA_CUDA_TRY(cudaGraphLaunch(m->gexec[grad], stream));
    m->launched += m->graph_kernels[grad];
  } else {
    const int64_t before = g_launches;
    BTA_TRY(rec(stream));
    m->launched += g_launches - before;
  }
  const int no = out_size(d);
  BTA_CUDA_TRY(cudaMemcpyAsync(m->hout, m->out, no * sizeof(double), cudaMemcpyDeviceToHost,
                               stream));
  BTA_CUDA_TRY(cudaStreamSynchronize(stream));
  m->last.assign(m->hout, m->hout + no);
  m->have_factors = mode == 0;
  const double* parts = m->hout + 1 + d;
  if (parts[6] >= 0 || parts[7] >= 0) return BTA_ERR_NOT_SPD;
  return BTA_OK;
}

}  // namespace

extern "C" {

const char* bta_status_string(bta_status s) {
  switch (s) {
    case BTA_OK: return "ok";
    case BTA_ERR_ARG: return "invalid argument";
    case BTA_ERR_NOT_SPD: return "matrix not positive definite";
    case BTA_ERR_CUDA: return "CUDA error";
    case BTA_ERR_NOMEM: return "out of device memory";
    case BTA_ERR_TIMEOUT: return "bounded device wait timed out";
    case BTA_ERR_STATE: return "descriptor in the wrong state";
  }
  return "unknown status";
}

void inla_model_destroy(inla_model* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  for (int g = 0; g < 3; ++g)
    if (m->gexec[g]) cudaGraphExecDestroy(m->gexec[g]);
  for (void* p : m->allocs) cudaFree(p);
  if (m->hout) cudaFreeHost(m->hout);
  if (m->htheta) cudaFreeHost(m->htheta);
  if (m->s1) cudaStreamDestroy(m->s1);
  if (m->s2) cudaStreamDestroy(m->s2);
  for (cudaEvent_t e : {m->ev0, m->evx, m->ev1, m->ev2})
    if (e) cudaEventDestroy(e);
  delete m;
}

static bta_status model_create_impl(const inla_model_spec* sp, inla_model* m) {
  ModelDev& md = m->md;
  const int k = sp->k, ns = sp->ns, nt = sp->nt, a = sp->a;
  if (k < 1 || k > kMaxK || ns < 1 || nt < 1 || a < 0 || a % k || a > 32 || sp->nnz < 1 ||
      !sp->row_ptr || !sp->col || !sp->val_C || !sp->val_G || !sp->val_GG || !sp->m_diag ||
      (nt > 1 && !sp->m_sub) || sp->n_obs < 0 || (sp->n_obs > 0 && (!sp->obs_t || !sp->obs_s ||
      !sp->obs_v || !sp->y || (a > 0 && !sp->obs_cov))))
    return BTA_ERR_ARG;
  md.k = k; md.ns = ns; md.nt = nt; md.a = a; md.a_r = a / k; md.b = k * ns;
  md.ld = pad_ld(md.b); md.d = 4 * k + k * (k - 1) / 2; md.nnz = sp->nnz; md.n_obs = sp->n_obs;
  md.tip_prior = sp->tip_prior > 0 ? sp->tip_prior : 1e-3;
  md.theta_prior_var = sp->theta_prior_var > 0 ? sp->theta_prior_var : 100.0;
  if (md.d > kMaxD) return BTA_ERR_ARG;
  const int ld = md.ld, b = md.b, a_r = md.a_r;
  m->n = nt; m->b = b; m->ld = ld; m->a = a; m->d = md.d;
  // --- spatial pattern
  if (sp->row_ptr[0] != 0 || sp->row_ptr[ns] != sp->nnz) return BTA_ERR_ARG;
  std::vector<int32_t> row_of(sp->nnz);
  for (int s = 0; s < ns; ++s) {
    bool diag = false;
    for (int e = sp->row_ptr[s]; e < sp->row_ptr[s + 1]; ++e) {
      if (sp->col[e] < 0 || sp->col[e] >= ns) return BTA_ERR_ARG;
      row_of[e] = s;
      diag |= sp->col[e] == s;
    }
    if (!diag) return BTA_ERR_ARG;   // the pattern must hold the diagonal
  }
  std::vector<double> val(3 * (size_t)sp->nnz);
  std::memcpy(val.data(), sp->val_C, sp->nnz * sizeof(double));
  std::memcpy(val.data() + sp->nnz, sp->val_G, sp->nnz * sizeof(double));
  std::memcpy(val.data() + 2 * (size_t)sp->nnz, sp->val_GG, sp->nnz * sizeof(double));
  BTA_TRY(upload(m, &md.row_ptr, sp->row_ptr, ns + 1));
  BTA_TRY(upload(m, &md.col, sp->col, sp->nnz));
  BTA_TRY(upload(m, &md.row_of, row_of.data(), sp->nnz));
  BTA_TRY(upload(m, &md.val, val.data(), val.size()));
  md.m_diag_h.assign(sp->m_diag, sp->m_diag + 3 * nt);
  md.m_sub_h.assign(std::max(3 * (nt - 1), 1), 0.0);
  if (nt > 1) std::memcpy(md.m_sub_h.data(), sp->m_sub, 3 * (nt - 1) * sizeof(double));
  BTA_TRY(upload(m, &md.m_diag, md.m_diag_h.data(), md.m_diag_h.size()));
  BTA_TRY(upload(m, &md.m_sub, md.m_sub_h.data(), md.m_sub_h.size()));
  // --- observation-derived, theta-independent pieces (fixed accumulation order)
  std::vector<double> cnt((size_t)nt * ld, 0.0), craw((size_t)nt * a * ld, 0.0),
      traw((size_t)k * a * a, 0.0), rraw((size_t)nt * ld + a, 0.0);
  std::vector<int32_t> lat(std::max<int64_t>(sp->n_obs, 1));
  md.n_per_var.assign(k, 0.0);
  for (int64_t j = 0; j < sp->n_obs; ++j) {
    int t = sp->obs_t[j], s = sp->obs_s[j], v = sp->obs_v[j];
    if (t < 0 || t >= nt || s < 0 || s >= ns || v < 0 || v >= k) return BTA_ERR_ARG;
    int c = v * ns + s;
    int64_t li = (int64_t)t * ld + c;
    lat[j] = (int32_t)li;
    cnt[li] += 1.0;
    rraw[li] += sp->y[j];
    md.n_per_var[v] += 1.0;
    const double* cv = sp->obs_cov + j * a_r;
    for (int i = 0; i < a_r; ++i) {
      int f = v * a_r + i;
      craw[(size_t)t * a * ld + f + (size_t)c * a] += cv[i];
      rraw[(size_t)nt * ld + f] += cv[i] * sp->y[j];
      for (int i2 = 0; i2 < a_r; ++i2)
        traw[(size_t)v * a * a + f + (size_t)(v * a_r + i2) * a] += cv[i] * cv[i2];
    }
  }
  BTA_TRY(upload(m, &md.cnt, cnt.data(), cnt.size()));
  BTA_TRY(upload(m, &md.craw, craw.data(), std::max<size_t>(craw.size(), 1)));
  BTA_TRY(upload(m, &md.traw, traw.data(), std::max<size_t>(traw.size(), 1)));
  BTA_TRY(upload(m, &md.rraw, rraw.data(), rraw.size()));
  BTA_TRY(upload(m, &md.obs_lat, lat.data(), lat.size()));
  BTA_TRY(upload(m, &md.obs_v, sp->n_obs ? sp->obs_v : lat.data(), lat.size()));
  std::vector<double> covv((size_t)std::max<int64_t>(sp->n_obs, 1) * std::max(a_r, 1), 0.0),
      yv(std::max<int64_t>(sp->n_obs, 1), 0.0);
  if (sp->n_obs) {
    if (a_r) std::memcpy(covv.data(), sp->obs_cov, sp->n_obs * a_r * sizeof(double));
    std::memcpy(yv.data(), sp->y, sp->n_obs * sizeof(double));
  }
  BTA_TRY(upload(m, &md.obs_cov, covv.data(), covv.size()));
  BTA_TRY(upload(m, &md.y, yv.data(), yv.size()));
  // --- evaluation buffers
  m->L.init(k, md.d, nt);
  BTA_TRY(dmalloc(m, &m->coefbuf, m->L.total));
  const size_t blk = (size_t)ld * ld;
  m->qc.n = nt; m->qc.b = b; m->qc.a = a; m->qc.ld = ld;
  BTA_TRY(dmalloc(m, &m->qc.D, nt * blk));
  BTA_TRY(dmalloc(m, &m->qc.B, std::max(nt - 1, 1) * blk));
  BTA_TRY(dmalloc(m, &m->qc.C, std::max<size_t>((size_t)nt * a * ld, 1)));
  BTA_TRY(dmalloc(m, &m->qc.T, std::max(a * a, 1)));
  m->qp = m->qc;
  m->qp.a = 0; m->qp.C = nullptr; m->qp.T = nullptr;
  BTA_TRY(dmalloc(m, &m->qp.D, nt * blk));
  BTA_TRY(dmalloc(m, &m->qp.B, std::max(nt - 1, 1) * blk));
  BTA_TRY(dmalloc(m, &m->x, (size_t)nt * ld + a));
  m->nslots = logdet_slots(nt, ld);
  m->nslots_p = m->nslots;
  BTA_TRY(dmalloc(m, &m->slots_c, m->nslots));
  BTA_TRY(dmalloc(m, &m->slots_p, m->nslots_p));
  BTA_TRY(dmalloc(m, &m->fail, 2));
  const size_t pblk = (size_t)k * k * pattern_chunks(md) * kNP;
  BTA_TRY(dmalloc(m, &m->PDc, nt * pblk));
  BTA_TRY(dmalloc(m, &m->PBc, std::max(nt - 1, 1) * pblk));
  BTA_TRY(dmalloc(m, &m->PCc, std::max<size_t>((size_t)nt * k * arrow_chunks(md), 1)));
  BTA_TRY(dmalloc(m, &m->PDp, nt * pblk));
  BTA_TRY(dmalloc(m, &m->PBp, std::max(nt - 1, 1) * pblk));
  BTA_TRY(dmalloc(m, &m->QD, nt * pblk));
  BTA_TRY(dmalloc(m, &m->QB, std::max(nt - 1, 1) * pblk));
  BTA_TRY(dmalloc(m, &m->RS, (size_t)kMaxK * resid_chunks(md)));   // residual_kernel writes kMaxK rows
  BTA_TRY(dmalloc(m, &m->out, out_size(md.d)));
  size_t wsb = SweepWs::bytes(ld, a) / sizeof(double);
  BTA_TRY(dmalloc(m, &m->wsbuf, 2 * wsb));
  m->wsc.carve(m->wsbuf, ld, a);
  m->wsp.carve(m->wsbuf + wsb, ld, a);
  BTA_CUDA_TRY(cudaMallocHost(&m->hout, out_size(md.d) * sizeof(double)));
  BTA_CUDA_TRY(cudaMallocHost(&m->htheta, kMaxD * sizeof(double)));
  BTA_CUDA_TRY(cudaStreamCreateWithFlags(&m->s1, cudaStreamNonBlocking));
  BTA_CUDA_TRY(cudaStreamCreateWithFlags(&m->s2, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&m->ev0, &m->evx, &m->ev1, &m->ev2})
    BTA_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  BTA_CUDA_TRY(cudaDeviceSynchronize());
  return BTA_OK;
}

bta_status inla_model_create(const inla_model_spec* spec, inla_model** out) {
  if (!spec || !out) return BTA_ERR_ARG;
  *out = nullptr;
  inla_model* m = new (std::nothrow) inla_model();
  if (!m) return BTA_ERR_NOMEM;
  bta_status st = model_create_impl(spec, m);
  if (st != BTA_OK) {
    inla_model_destroy(m);
    return st;
  }
  *out = m;
  return BTA_OK;
}

bta_status inla_model_dims(const inla_model* m, int32_t* d, int32_t* b, int32_t* ld, int32_t* n,
                           int32_t* a) {
  if (!m) return BTA_ERR_ARG;
  if (d) *d = m->d;
  if (b) *b = m->b;
  if (ld) *ld = m->ld;
  if (n) *n = m->n;
  if (a) *a = m->a;
  return BTA_OK;
}

static bool desc_ok(const bta_desc* q, int need_arrow) {
  if (!q || q->n < 1 || q->b < 1 || q->ld < q->b || q->ld % kPad || q->a < 0 || q->a > 32 ||
      !q->D || (q->n > 1 && !q->B))
    return false;
  if (q->a > 0 && (!q->C || !q->T)) return false;
  (void)need_arrow;
  return true;
}

bta_status bta_assemble(inla_model* m, const double* theta, int32_t which, bta_desc* out,
                        double* rhs, cudaStream_t stream) {
  if (!m || !theta || !out || (which != 0 && which != 1)) return BTA_ERR_ARG;
  if (!finite_theta(theta, m->d)) return BTA_ERR_ARG;
  if (out->n != m->n || out->b != m->b || out->ld != m->ld ||
      out->a != (which ? m->a : 0) || !desc_ok(out, which))
    return BTA_ERR_ARG;
  double* cb = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&cb, m->L.total * sizeof(double), stream));
  BTA_CUDA_TRY(cudaMemcpyAsync(cb + m->L.theta, theta, m->d * sizeof(double),
                               cudaMemcpyHostToDevice, stream));
  bta_status st = launch_coef(m->md, m->L, cb, stream);
  if (st == BTA_OK) st = launch_assemble(m->md, m->L, cb, which, *out, which ? rhs : nullptr,
                                         stream);
  cudaFreeAsync(cb, stream);
  if (st == BTA_OK) out->state = BTA_STATE_ASSEMBLED;
  return st;
}

bta_status bta_factor(bta_desc* q, double* rhs_inout, double* logdet, int32_t* fail_block,
                      int32_t precision, cudaStream_t stream) {
  if (!desc_ok(q, 0) || !logdet || !fail_block || precision != 0) return BTA_ERR_ARG;
  if (q->state != BTA_STATE_ASSEMBLED) return BTA_ERR_STATE;
  const int nsl = logdet_slots(q->n, q->ld);
  size_t wsb = SweepWs::bytes(q->ld, q->a);
  double* buf = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&buf, wsb + nsl * sizeof(double), stream));
  SweepWs ws;
  ws.carve(buf, q->ld, q->a);
  double* slots = buf + wsb / sizeof(double);
  BTA_CUDA_TRY(cudaMemsetAsync(fail_block, 0xff, sizeof(int32_t), stream));
  bta_status st = factor_sweep(*q, rhs_inout, slots, fail_block, ws, stream);
  if (st == BTA_OK) st = sum_slots(slots, nsl, logdet, 0, stream);
  cudaFreeAsync(buf, stream);
  if (st == BTA_OK) q->state = BTA_STATE_FACTORED;
  return st;
}

bta_status bta_solve(const bta_desc* L, double* z_inout, int32_t lower, int32_t refine,
                     const bta_desc* Q_or_null, cudaStream_t stream) {
  (void)Q_or_null;
  if (!desc_ok(L, 0) || !z_inout || refine != 0) return BTA_ERR_ARG;
  if (L->state != BTA_STATE_FACTORED) return BTA_ERR_STATE;
  size_t wsb = SweepWs::bytes(L->ld, L->a);
  double* buf = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&buf, wsb, stream));
  SweepWs ws;
  ws.carve(buf, L->ld, L->a);
  bta_status st = BTA_OK;
  if (lower) st = lower_solve(*L, z_inout, ws, stream);
  if (st == BTA_OK) st = upper_solve(*L, z_inout, ws, stream);
  cudaFreeAsync(buf, stream);
  return st;
}

bta_status bta_selinv(bta_desc* L, inla_model* m, const double* theta, int32_t which,
                      double* trace_terms, cudaStream_t stream) {
  if (!desc_ok(L, 0)) return BTA_ERR_ARG;
  if (L->state != BTA_STATE_FACTORED) return BTA_ERR_STATE;
  const bool fused = m && trace_terms;
  if (fused) {
    if (!theta || !finite_theta(theta, m->d) || (which != 0 && which != 1)) return BTA_ERR_ARG;
    if (L->n != m->n || L->ld != m->ld || L->a != (which ? m->a : 0)) return BTA_ERR_ARG;
  }
  size_t wsb = SweepWs::bytes(L->ld, L->a);
  double* buf = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&buf, wsb, stream));
  SweepWs ws;
  ws.carve(buf, L->ld, L->a);
  bta_status st = BTA_OK;
  if (!fused) {
    st = selinv_sweep(*L, ws, nullptr, stream);
  } else {
    const ModelDev& md = m->md;
    const size_t pblk = (size_t)md.k * md.k * pattern_chunks(md) * kNP;
    const size_t nPD = md.nt * pblk, nPB = std::max(md.nt - 1, 1) * pblk;
    const size_t nPC = std::max<size_t>((size_t)md.nt * md.k * arrow_chunks(md), 1);
    const size_t nRS = (size_t)kMaxK * resid_chunks(md);
    double* rb = nullptr;
    const size_t nZ0 = std::max(nPD + nPB, (size_t)md.nt * md.ld + md.a);
    size_t total = m->L.total + nPD + nPB + nPC + nZ0 + nRS + out_size(md.d) + 4;
    BTA_CUDA_TRY(cudaMallocAsync(&rb, total * sizeof(double), stream));
    double* cb = rb;
    double* PD = cb + m->L.total;
    double* PB = PD + nPD;
    double* PC = PB + nPB;
    double* Z0 = PC + nPC;           // zero reductions for the other matrix / quad forms
    double* RS = Z0 + nZ0;
    double* o = RS + nRS;
    int32_t* fl = reinterpret_cast<int32_t*>(o + out_size(md.d));
    BTA_CUDA_TRY(cudaMemsetAsync(rb, 0, total * sizeof(double), stream));
    BTA_CUDA_TRY(cudaMemsetAsync(fl, 0xff, 2 * sizeof(int32_t), stream));
    BTA_CUDA_TRY(cudaMemcpyAsync(cb + m->L.theta, theta, md.d * sizeof(double),
                                 cudaMemcpyHostToDevice, stream));
    st = launch_coef(md, m->L, cb, stream);
    SelinvFuse fz;
    fz.md = &md; fz.counts = which; fz.PD = PD; fz.PB = PB; fz.PC = which ? PC : nullptr;
    if (st == BTA_OK) st = selinv_sweep(*L, ws, &fz, stream);
    if (st == BTA_OK) {
      // Reuse the final combination with the other matrix's sums at zero:
      // Phase A = -1/2 tr(Q_c^-1 dQ_c), Phase C = +1/2 tr(Q_p^-1 dQ_p).
      Reductions r{};
      r.PDc = which ? PD : Z0; r.PBc = which ? PB : Z0 + nPD; r.PCc = which ? PC : Z0;
      r.ZTc = which ? L->T : Z0;
      r.PDp = which ? Z0 : PD; r.PBp = which ? Z0 + nPD : PB;
      r.QD = Z0; r.QB = Z0 + nPD; r.RS = RS;
      r.ldc = Z0; r.nldc = 1; r.ldp = Z0; r.nldp = 1; r.failc = fl; r.failp = fl + 1;
      r.x = Z0; r.grad = 1;
      ModelDev mz = md;
      mz.a = which ? md.a : 0;
      st = launch_finalize(mz, m->L, cb, r, o, stream);
      if (st == BTA_OK) {
        // phases at o + 1 + d + kOutParts: A (d), B (d), C (d)
        const double* ph = o + 1 + md.d + kOutParts;
        st = copy_block(which ? ph : ph + 2 * md.d, md.d, trace_terms, md.d, md.d, 1,
                        which ? -2.0 : 2.0, 0, stream);
      }
    }
    cudaFreeAsync(rb, stream);
  }
  cudaFreeAsync(buf, stream);
  if (st == BTA_OK) L->state = BTA_STATE_SELINV;
  return st;
}

bta_status inla_value_and_grad(inla_model* m, const double* theta, int32_t batch, double* f,
                               double* grad, const inla_opts* opts, cudaStream_t stream) {
  if (!m || !theta || !f || batch < 1) return BTA_ERR_ARG;
  if (opts && opts->precision != 0) return BTA_ERR_ARG;
  for (int i = 0; i < batch; ++i)
    if (!finite_theta(theta + (size_t)i * m->d, m->d)) return BTA_ERR_ARG;
  const int use_graph = opts ? opts->use_graph : 1;
  const int g = grad ? 1 : 0;
  for (int i = 0; i < batch; ++i) {
    bta_status st = run_eval(m, theta + (size_t)i * m->d, g, use_graph, stream);
    f[i] = m->last[0];
    if (grad)
      for (int j = 0; j < m->d; ++j) grad[(size_t)i * m->d + j] = m->last[1 + j];
    if (st != BTA_OK) return st;
  }
  return BTA_OK;
}

bta_status inla_backward(inla_model* m, double* grad, int32_t use_graph, cudaStream_t stream) {
  if (!m || !grad) return BTA_ERR_ARG;
  if (!m->have_factors) return BTA_ERR_STATE;
  bta_status st = run_eval(m, nullptr, 2, use_graph, stream);
  for (int j = 0; j < m->d; ++j) grad[j] = m->last[1 + j];
  return st;
}

bta_status bta_gemm(int32_t M, int32_t N, int32_t K, double alpha, const double* A, int32_t lda,
                    int32_t transA, const double* B, int32_t ldb, int32_t transB, double beta,
                    double* Cm, int32_t ldc, cudaStream_t stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !Cm) return BTA_ERR_ARG;
  Gemm g;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.transA = transA ? 1 : 0;
  g.B = B; g.ldb = ldb; g.transB = transB ? 1 : 0;
  g.C = Cm; g.ldc = ldc; g.Cin = Cm; g.ldcin = ldc;
  return gemm_f64(g, stream);
}

bta_status inla_last_parts(const inla_model* m, double* parts, double* phases) {
  if (!m || m->last.empty()) return BTA_ERR_STATE;
  const double* p = m->last.data() + 1 + m->d;
  if (parts)
    for (int i = 0; i < kOutParts; ++i) parts[i] = p[i];
  if (phases)
    for (int i = 0; i < 4 * m->d; ++i) phases[i] = p[kOutParts + i];
  return BTA_OK;
}

bta_status inla_copy_mode(const inla_model* m, double* dst, cudaStream_t stream) {
  if (!m || !dst) return BTA_ERR_ARG;
  BTA_CUDA_TRY(cudaMemcpyAsync(dst, m->x, ((size_t)m->n * m->ld + m->a) * sizeof(double),
                               cudaMemcpyDeviceToDevice, stream));
  return BTA_OK;
}

int64_t inla_kernel_launches(const inla_model* m) { return m ? m->launched : g_launches; }

}  // extern "C"
