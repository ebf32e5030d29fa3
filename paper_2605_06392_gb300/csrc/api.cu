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
#include <functional>
#include <memory>
#include <new>
#include <vector>

#include "sweep.cuh"

using namespace bta;

// One evaluation context: everything a single theta's evaluation writes.
struct EvalCtx {
  double* coefbuf = nullptr;
  bta_desc qc{}, qp{};
  double* x = nullptr;          // r -> z -> x*  (n*ld + a)
  double* slots_c = nullptr;
  double* slots_p = nullptr;
  int32_t* fail = nullptr;      // [2]
  double *PDc = nullptr, *PBc = nullptr, *PCc = nullptr, *PDp = nullptr, *PBp = nullptr;
  double *QD = nullptr, *QB = nullptr, *RS = nullptr;
  double* out = nullptr;
  SweepWs wsc, wsp;
  SelinvFuse fc, fp;
  double* dr = nullptr;         // mixed mode: refinement residual / correction
  double *w4c = nullptr, *w4p = nullptr;   // low memory: second L_B buffer per sweep
  int have_factors = 0;         // last evaluation was value-only: factors still held
};

struct GraphKey {
  int mode, count, precision;
  cudaGraphExec_t exec;
  int64_t kernels;
};

struct inla_model {
  ModelDev md;
  CoefLayout L;
  int n = 0, b = 0, ld = 0, a = 0, d = 0;
  int nslots = 0;
  int lowmem = 0;               // keep only the diagonal factors (see inla_model_spec)
  std::vector<EvalCtx> ctx;     // grown on demand (batched evaluations)
  std::vector<void*> allocs;
  // host
  double* hout = nullptr;       // pinned, kMaxBatch outputs
  double* htheta = nullptr;     // pinned, kMaxBatch thetas
  std::vector<double> last;     // output of the last single evaluation
  std::vector<GraphKey> graphs;
  int64_t launched = 0;         // kernels this model ran (graph replays included)
  // the Q_c set and the Q_p set are swept on two streams (fork/join by events)
  cudaStream_t s1 = nullptr, s2 = nullptr;
  cudaStream_t s0 = nullptr;    // the model's own root stream inside a multi-model graph
  cudaEvent_t ev0 = nullptr, evx = nullptr, ev1 = nullptr, ev2 = nullptr, evd = nullptr;
  cudaEvent_t evj = nullptr;    // join event of a multi-model graph
};

// Several models evaluated by one CUDA graph (see inla_batch_value_and_grad).
struct inla_batch {
  std::vector<inla_model*> models;
  cudaGraphExec_t exec[2][3] = {};   // [grad][precision]
  int64_t kernels[2][3] = {};
  cudaEvent_t fork = nullptr;
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

// Allocate evaluation context c (buffers for Q_c, Q_p, x*, reductions).
bta_status ctx_alloc(inla_model* m, EvalCtx& c) {
  const ModelDev& md = m->md;
  const int nt = md.nt, ld = md.ld, a = md.a, k = md.k;
  const size_t blk = (size_t)ld * ld;
  BTA_TRY(dmalloc(m, &c.coefbuf, m->L.total));
  c.qc.n = nt; c.qc.b = md.b; c.qc.a = a; c.qc.ld = ld;
  BTA_TRY(dmalloc(m, &c.qc.D, nt * blk));
  if (!m->lowmem) BTA_TRY(dmalloc(m, &c.qc.B, std::max(nt - 1, 1) * blk));
  BTA_TRY(dmalloc(m, &c.qc.C, std::max<size_t>((size_t)nt * a * ld, 1)));
  BTA_TRY(dmalloc(m, &c.qc.T, std::max(a * a, 1)));
  c.qp = c.qc;
  c.qp.a = 0; c.qp.C = nullptr; c.qp.T = nullptr;
  BTA_TRY(dmalloc(m, &c.qp.D, nt * blk));
  if (!m->lowmem) {
    BTA_TRY(dmalloc(m, &c.qp.B, std::max(nt - 1, 1) * blk));
  } else {
    c.qp.B = nullptr;
    BTA_TRY(dmalloc(m, &c.w4c, blk));
    BTA_TRY(dmalloc(m, &c.w4p, blk));
  }
  BTA_TRY(dmalloc(m, &c.x, (size_t)nt * ld + a));
  BTA_TRY(dmalloc(m, &c.slots_c, m->nslots));
  BTA_TRY(dmalloc(m, &c.slots_p, m->nslots));
  BTA_TRY(dmalloc(m, &c.fail, 4));   // [0] Q_c pivot, [1] Q_p pivot, [2] tensor-core status
  const size_t pblk = (size_t)k * k * pattern_chunks(md) * kNP;
  BTA_TRY(dmalloc(m, &c.PDc, nt * pblk));
  BTA_TRY(dmalloc(m, &c.PBc, std::max(nt - 1, 1) * pblk));
  BTA_TRY(dmalloc(m, &c.PCc, std::max<size_t>((size_t)nt * k * arrow_chunks(md), 1)));
  BTA_TRY(dmalloc(m, &c.PDp, nt * pblk));
  BTA_TRY(dmalloc(m, &c.PBp, std::max(nt - 1, 1) * pblk));
  BTA_TRY(dmalloc(m, &c.QD, nt * pblk));
  BTA_TRY(dmalloc(m, &c.QB, std::max(nt - 1, 1) * pblk));
  // residual_kernel writes kMaxK rows
  BTA_TRY(dmalloc(m, &c.RS, (size_t)kMaxK * resid_chunks(md)));
  BTA_TRY(dmalloc(m, &c.out, out_size(md.d)));
  const size_t wsb = SweepWs::bytes(ld, a) / sizeof(double);
  double* wsbuf = nullptr;
  BTA_TRY(dmalloc(m, &wsbuf, 2 * wsb));
  c.wsc.carve(wsbuf, ld, a);
  c.wsp.carve(wsbuf + wsb, ld, a);
  // tensor-core modes: operand copies of the tensor-core products, one per sweep
  const size_t tcb = sweep_tc_ws_bytes(ld, a);
  uint8_t* tcbuf = nullptr;
  BTA_TRY(dmalloc(m, &tcbuf, 2 * tcb));
  c.wsc.tc = tcbuf;
  c.wsp.tc = tcbuf + tcb;
  c.wsc.tcstat = c.fail + 2;
  c.wsp.tcstat = c.fail + 2;
  BTA_TRY(dmalloc(m, &c.dr, (size_t)nt * ld + a));
  c.fc.md = &m->md; c.fc.counts = 1; c.fc.PD = c.PDc; c.fc.PB = c.PBc; c.fc.PC = c.PCc;
  c.fp.md = &m->md; c.fp.counts = 0; c.fp.PD = c.PDp; c.fp.PB = c.PBp; c.fp.PC = nullptr;
  return BTA_OK;
}

bta_status ensure_ctx(inla_model* m, int count) {
  if ((int)m->ctx.size() >= count) return BTA_OK;
  cudaDeviceSynchronize();
  m->ctx.reserve(count);
  while ((int)m->ctx.size() < count) {
    m->ctx.emplace_back();
    bta_status st = ctx_alloc(m, m->ctx.back());
    if (st != BTA_OK) {
      m->ctx.pop_back();
      return st;
    }
  }
  // contexts hold pointers to the model: the fuse blocks refer to m->md (stable)
  return BTA_OK;
}

// The evaluation of contexts 0..cnt-1 as a list of issue steps.
//   mode 0: f only; 1: f and gradient; 2: reverse pass of a preceding mode-0
//   evaluation (the factors are still in place).
// The conditional matrices Q_c of all contexts form one set and the priors
// Q_p another; each set is swept with one batched launch per block step, and
// the two sets run on two streams.  They are independent until the final
// combination (the stencil quadratic forms on the Q_p stream wait for x*), so
// the serial diagonal steps of one set overlap the wide products of the other.
// Each step issues one block of both sweeps (Q_c's, then Q_p's), so the two
// streams' operations, and the nodes of a captured graph, are created in
// alternation: the driver submits a graph's kernels in creation order into a
// bounded queue, and a whole Q_c sweep created first (~1600 launches a block)
// held the Q_p stream back until the GPU had drained most of it.
using IssueStep = std::function<bta_status()>;

struct GroupSets {
  std::vector<SweepItem> ic, ip;
};

bta_status group_program(inla_model* m, int mode, int cnt, int prec, cudaStream_t s0,
                         std::vector<IssueStep>& steps) {
  const ModelDev& md = m->md;
  const int grad = mode >= 1, nt = md.nt;
  auto sets = std::make_shared<GroupSets>();
  sets->ic.resize(cnt);
  sets->ip.resize(cnt);
  for (int e = 0; e < cnt; ++e) {
    EvalCtx& c = m->ctx[e];
    SweepItem& ic = sets->ic[e];
    SweepItem& ip = sets->ip[e];
    ic.q = c.qc; ic.vec = c.x; ic.slots = c.slots_c; ic.fail = c.fail;
    ic.ws = c.wsc; ic.fuse = &c.fc;
    ip.q = c.qp; ip.vec = nullptr; ip.slots = c.slots_p; ip.fail = c.fail + 1;
    ip.ws = c.wsp; ip.fuse = &c.fp;
    ic.md = ip.md = &md;
    ic.lay = ip.lay = &m->L;
    ic.coef = ip.coef = c.coefbuf;
    ic.W4 = c.w4c;
    ip.W4 = c.w4p;
  }
  // set-up on s0, the fork, and (mode < 2) the assembly of both sets
  steps.push_back([=]() -> bta_status {
    if (mode < 2) {
      for (int e = 0; e < cnt; ++e) {
        EvalCtx& c = m->ctx[e];
        BTA_TRY(launch_coef(md, m->L, c.coefbuf, s0));
        BTA_CUDA_TRY(cudaMemsetAsync(c.fail, 0xff, 2 * sizeof(int32_t), s0));
        BTA_CUDA_TRY(cudaMemsetAsync(c.fail + 2, 0, sizeof(int32_t), s0));
      }
    }
    BTA_CUDA_TRY(cudaEventRecord(m->ev0, s0));
    BTA_CUDA_TRY(cudaStreamWaitEvent(m->s1, m->ev0, 0));
    BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->ev0, 0));
    if (mode < 2)
      for (int e = 0; e < cnt; ++e) {
        BTA_TRY(launch_assemble(md, m->L, m->ctx[e].coefbuf, 1, m->ctx[e].qc, m->ctx[e].x,
                                m->s1));
        BTA_TRY(launch_assemble(md, m->L, m->ctx[e].coefbuf, 0, m->ctx[e].qp, nullptr, m->s2));
      }
    return BTA_OK;
  });
  if (mode < 2) {
    for (int i = 0; i < nt; ++i)
      steps.push_back([=]() -> bta_status {
        BTA_TRY(factor_sweep_multi(sets->ic.data(), cnt, m->s1, m->evd, prec, i, i + 1));
        // the Q_p sweep starts one diagonal step behind the Q_c sweep: the two
        // then alternate their latency-bound diagonal factors with wide products
        if (i == 0) BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->evd, 0));
        return factor_sweep_multi(sets->ip.data(), cnt, m->s2, nullptr, prec, i, i + 1);
      });
    steps.push_back([=]() -> bta_status {
      BTA_TRY(upper_solve_multi(sets->ic.data(), cnt, m->s1));
      if (prec == 1) {
        // one step of iterative refinement in FP64: x += Q_c^{-1} (r - Q_c x)
        for (int e = 0; e < cnt; ++e) {
          EvalCtx& c = m->ctx[e];
          BTA_TRY(launch_rhs(md, m->L, c.coefbuf, c.dr, m->s1));
          BTA_TRY(launch_qc_residual(md, m->L, c.coefbuf, c.x, c.dr, m->s1));
          BTA_TRY(lower_solve(c.qc, c.dr, c.wsc, m->s1));
          BTA_TRY(upper_solve(c.qc, c.dr, c.wsc, m->s1));
          BTA_TRY(launch_axpy((int64_t)md.nt * md.ld + md.a, 1.0, c.dr, c.x, m->s1));
        }
      }
      BTA_CUDA_TRY(cudaEventRecord(m->evx, m->s1));
      for (int e = 0; e < cnt; ++e)
        BTA_TRY(launch_residual(md, m->ctx[e].x, m->ctx[e].RS, m->s1));
      BTA_CUDA_TRY(cudaStreamWaitEvent(m->s2, m->evx, 0));
      for (int e = 0; e < cnt; ++e)
        BTA_TRY(launch_pattern_quad_all(md, m->ctx[e].x, m->ctx[e].QD, m->ctx[e].QB, m->s2));
      return BTA_OK;
    });
  }
  if (grad)
    for (int i = nt - 1; i >= 0; --i)
      steps.push_back([=]() -> bta_status {
        BTA_TRY(selinv_sweep_multi(sets->ic.data(), cnt, m->s1, prec, i, i));
        return selinv_sweep_multi(sets->ip.data(), cnt, m->s2, prec, i, i);
      });
  // join and combine
  steps.push_back([=]() -> bta_status {
    BTA_CUDA_TRY(cudaEventRecord(m->ev1, m->s1));
    BTA_CUDA_TRY(cudaEventRecord(m->ev2, m->s2));
    BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev1, 0));
    BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->ev2, 0));
    for (int e = 0; e < cnt; ++e) {
      EvalCtx& c = m->ctx[e];
      Reductions r{};
      r.PDc = c.PDc; r.PBc = c.PBc; r.PCc = c.PCc; r.ZTc = c.qc.T;
      r.PDp = c.PDp; r.PBp = c.PBp; r.QD = c.QD; r.QB = c.QB; r.RS = c.RS;
      r.ldc = c.slots_c; r.nldc = m->nslots; r.ldp = c.slots_p; r.nldp = m->nslots;
      r.failc = c.fail; r.failp = c.fail + 1; r.x = c.x; r.grad = grad;
      BTA_TRY(launch_finalize(md, m->L, c.coefbuf, r, c.out, s0));
    }
    return BTA_OK;
  });
  return BTA_OK;
}

// Record (issue, or capture) the evaluation of contexts 0..cnt-1.
bta_status record_group(inla_model* m, int mode, int cnt, int prec, cudaStream_t s0) {
  std::vector<IssueStep> steps;
  BTA_TRY(group_program(m, mode, cnt, prec, s0, steps));
  for (auto& st : steps) BTA_TRY(st());
  return BTA_OK;
}

// Status of one evaluation from its two failure words (parts[6], parts[7]:
// -1, a failing block, or BTA_ERR_TIMEOUT from the task-graph factor) and the
// tensor-core status word: a timeout outranks a non-positive pivot.
bta_status eval_status(const double* parts, int32_t tcs) {
  const double fc = parts[6], fp = parts[7];
  if (tcs == BTA_ERR_TIMEOUT || fc == BTA_ERR_TIMEOUT || fp == BTA_ERR_TIMEOUT)
    return BTA_ERR_TIMEOUT;
  if (fc >= 0 || fp >= 0) return BTA_ERR_NOT_SPD;
  return BTA_OK;
}

bta_status worse(bta_status a, bta_status b) {
  if (a == BTA_ERR_TIMEOUT || b == BTA_ERR_TIMEOUT) return BTA_ERR_TIMEOUT;
  return a != BTA_OK ? a : b;
}

// Run one group (thetas for contexts 0..cnt-1 already in htheta for mode < 2);
// outputs land in hout[e * out_size(d)].
bta_status run_group(inla_model* m, int mode, int cnt, int prec, int use_graph,
                     cudaStream_t stream) {
  const int d = m->d, no = out_size(d);
  if (mode < 2)
    for (int e = 0; e < cnt; ++e)
      BTA_CUDA_TRY(cudaMemcpyAsync(m->ctx[e].coefbuf + m->L.theta, m->htheta + (size_t)e * d,
                                   d * sizeof(double), cudaMemcpyHostToDevice, stream));
  if (use_graph) {
    GraphKey* gk = nullptr;
    for (auto& g : m->graphs)
      if (g.mode == mode && g.count == cnt && g.precision == prec) gk = &g;
    if (!gk) {
      if (mode < 2) {
        // one eager evaluation first: it times the tile shapes of the
        // products the graph will hold, which then replays those choices
        TuneScope tune;
        BTA_TRY(record_group(m, mode, cnt, prec, stream));
        BTA_CUDA_TRY(cudaStreamSynchronize(stream));
      }
      const int64_t before = g_launches;
      cudaStream_t cap;
      BTA_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
      BTA_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
      bta_status st = record_group(m, mode, cnt, prec, cap);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(cap, &graph);
      if (st != BTA_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cap);
        return st;
      }
      BTA_CUDA_TRY(e);
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      BTA_CUDA_TRY(e);
      m->graphs.push_back({mode, cnt, prec, exec, g_launches - before});
      gk = &m->graphs.back();
    }
    BTA_CUDA_TRY(cudaGraphLaunch(gk->exec, stream));
    m->launched += gk->kernels;
  } else {
    const int64_t before = g_launches;
    BTA_TRY(record_group(m, mode, cnt, prec, stream));
    m->launched += g_launches - before;
  }
  for (int e = 0; e < cnt; ++e)
    BTA_CUDA_TRY(cudaMemcpyAsync(m->hout + (size_t)e * no, m->ctx[e].out, no * sizeof(double),
                                 cudaMemcpyDeviceToHost, stream));
  BTA_CUDA_TRY(cudaStreamSynchronize(stream));
  bta_status st = BTA_OK;
  for (int e = 0; e < cnt; ++e) {
    int32_t tcs = 0;   // the tensor-core kernels' status word
    BTA_CUDA_TRY(cudaMemcpy(&tcs, m->ctx[e].fail + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
    const double* parts = m->hout + (size_t)e * no + 1 + d;
    st = worse(st, eval_status(parts, tcs));
    m->ctx[e].have_factors = mode == 0 ? 1 + prec : 0;   // remembers the factor's precision
  }
  m->last.assign(m->hout + (size_t)(cnt - 1) * no, m->hout + (size_t)cnt * no);
  return st;
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
  for (auto& g : m->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  for (void* p : m->allocs) cudaFree(p);
  if (m->hout) cudaFreeHost(m->hout);
  if (m->htheta) cudaFreeHost(m->htheta);
  if (m->s1) cudaStreamDestroy(m->s1);
  if (m->s2) cudaStreamDestroy(m->s2);
  if (m->s0) cudaStreamDestroy(m->s0);
  for (cudaEvent_t e : {m->ev0, m->evx, m->ev1, m->ev2, m->evd, m->evj})
    if (e) cudaEventDestroy(e);
  delete m;
}

static bta_status model_create_impl(const inla_model_spec* sp, inla_model* m) {
  ModelDev& md = m->md;
  m->lowmem = sp->low_memory != 0;
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
  // with no fixed effects (a = 0) the arrow arrays are empty: keep one zero
  // element so that every device array exists
  if (craw.empty()) craw.assign(1, 0.0);
  if (traw.empty()) traw.assign(1, 0.0);
  BTA_TRY(upload(m, &md.cnt, cnt.data(), cnt.size()));
  BTA_TRY(upload(m, &md.craw, craw.data(), craw.size()));
  BTA_TRY(upload(m, &md.traw, traw.data(), traw.size()));
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
  // --- evaluation buffers: one context up front, more on demand
  m->L.init(k, md.d, nt);
  m->nslots = logdet_slots(nt, ld);
  BTA_TRY(ensure_ctx(m, 1));
  BTA_CUDA_TRY(cudaMallocHost(&m->hout, (size_t)kMaxBatch * out_size(md.d) * sizeof(double)));
  BTA_CUDA_TRY(cudaMallocHost(&m->htheta, (size_t)kMaxBatch * kMaxD * sizeof(double)));
  BTA_CUDA_TRY(cudaStreamCreateWithFlags(&m->s1, cudaStreamNonBlocking));
  BTA_CUDA_TRY(cudaStreamCreateWithFlags(&m->s2, cudaStreamNonBlocking));
  BTA_CUDA_TRY(cudaStreamCreateWithFlags(&m->s0, cudaStreamNonBlocking));
  for (cudaEvent_t* e : {&m->ev0, &m->evx, &m->ev1, &m->ev2, &m->evd, &m->evj})
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
  if (!desc_ok(q, 0) || !logdet || !fail_block || precision < 0 || precision > 2)
    return BTA_ERR_ARG;
  if (q->state != BTA_STATE_ASSEMBLED) return BTA_ERR_STATE;
  const int nsl = logdet_slots(q->n, q->ld);
  const size_t wsb = SweepWs::bytes(q->ld, q->a);
  const int ld = q->ld;
  // tensor-core modes: operand copies of the b x b products (split TF32
  // planes or BF16 slices, whichever is larger), 256-byte aligned
  const size_t tcb = precision ? sweep_tc_ws_bytes(ld, q->a) : 0;
  const size_t head = (wsb + nsl * sizeof(double) + 255) / 256 * 256;
  uint8_t* buf = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&buf), head + tcb, stream));
  SweepWs ws;
  ws.carve(reinterpret_cast<double*>(buf), ld, q->a);
  double* slots = reinterpret_cast<double*>(buf) + wsb / sizeof(double);
  if (precision) {
    ws.tc = buf + head;
    ws.tcstat = fail_block;   // a tensor-core timeout lands in the failure word
  }
  BTA_CUDA_TRY(cudaMemsetAsync(fail_block, 0xff, sizeof(int32_t), stream));
  bta_status st = factor_sweep(*q, rhs_inout, slots, fail_block, ws, stream, precision);
  if (st == BTA_OK) st = sum_slots(slots, nsl, logdet, 0, stream);
  cudaFreeAsync(buf, stream);
  if (st == BTA_OK) q->state = BTA_STATE_FACTORED;
  return st;
}

bta_status bta_solve(const bta_desc* L, double* z_inout, int32_t lower, int32_t refine,
                     const bta_desc* Q_or_null, cudaStream_t stream) {
  if (!desc_ok(L, 0) || !z_inout || refine < 0 || refine > 1) return BTA_ERR_ARG;
  if (refine) {   // needs r (lower = 1) and the assembled matrix of the same shape
    const bta_desc* Q = Q_or_null;
    if (!lower || !desc_ok(Q, 0) || Q->n != L->n || Q->b != L->b || Q->ld != L->ld ||
        Q->a != L->a || Q->D == L->D)
      return BTA_ERR_ARG;
    if (Q->state != BTA_STATE_ASSEMBLED) return BTA_ERR_STATE;
  }
  if (L->state != BTA_STATE_FACTORED) return BTA_ERR_STATE;
  const size_t wsb = SweepWs::bytes(L->ld, L->a);
  const size_t nv = (size_t)L->n * L->ld + L->a;
  double* buf = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&buf, wsb + (refine ? 2 * nv * sizeof(double) : 0), stream));
  SweepWs ws;
  ws.carve(buf, L->ld, L->a);
  double* r = buf + wsb / sizeof(double);   // refinement: r, then the correction
  double* dx = r + nv;
  bta_status st = BTA_OK;
  if (refine)
    st = copy_block(z_inout, (int)nv, r, (int)nv, (int)nv, 1, 1.0, 0, stream);
  if (st == BTA_OK && lower) st = lower_solve(*L, z_inout, ws, stream);
  if (st == BTA_OK) st = upper_solve(*L, z_inout, ws, stream);
  if (st == BTA_OK && refine) {
    // one step of iterative refinement in FP64 (Eqs. 3-5 on the residual):
    // x += Q^{-1} (r - Q x) with the factor L of Q
    st = copy_block(r, (int)nv, dx, (int)nv, (int)nv, 1, 1.0, 0, stream);
    if (st == BTA_OK) st = bta_residual(*Q_or_null, z_inout, dx, ws.gv, stream);
    if (st == BTA_OK) st = lower_solve(*L, dx, ws, stream);
    if (st == BTA_OK) st = upper_solve(*L, dx, ws, stream);
    if (st == BTA_OK) st = launch_axpy((int64_t)nv, 1.0, dx, z_inout, stream);
  }
  cudaFreeAsync(buf, stream);
  return st;
}

bta_status bta_set_wait_limit(int64_t limit_ns, int32_t stall) {
  if (limit_ns < 0 || (limit_ns > 0 && limit_ns < 1000000) || limit_ns > 60000000000ll ||
      (stall != 0 && stall != 1))
    return BTA_ERR_ARG;
  g_dag_wait_ns = limit_ns ? (unsigned long long)limit_ns : 2000000000ull;
  g_dag_stall = stall;
  return BTA_OK;
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
  const int prec = opts ? opts->precision : 0;
  if (prec < 0 || prec > 2) return BTA_ERR_ARG;
  if (prec == 1 && m->lowmem) return BTA_ERR_ARG;   // its refinement solves read the B blocks
  for (int i = 0; i < batch; ++i)
    if (!finite_theta(theta + (size_t)i * m->d, m->d)) return BTA_ERR_ARG;
  const int use_graph = opts ? opts->use_graph : 1;
  int group = opts && opts->streams > 1 ? opts->streams : 1;
  group = std::min(group, std::min<int>(batch, kMaxBatch / 2));
  BTA_TRY(ensure_ctx(m, group));
  const int mode = grad ? 1 : 0;
  const int d = m->d, no = out_size(d);
  bta_status st = BTA_OK;
  for (int i0 = 0; i0 < batch; i0 += group) {
    const int cnt = std::min(group, batch - i0);
    std::memcpy(m->htheta, theta + (size_t)i0 * d, (size_t)cnt * d * sizeof(double));
    bta_status s1 = run_group(m, mode, cnt, prec, use_graph, stream);
    if (s1 != BTA_OK && s1 != BTA_ERR_NOT_SPD && s1 != BTA_ERR_TIMEOUT) return s1;
    st = worse(st, s1);
    for (int e = 0; e < cnt; ++e) {
      const double* o = m->hout + (size_t)e * no;
      f[i0 + e] = o[0];
      if (grad)
        for (int j = 0; j < d; ++j) grad[(size_t)(i0 + e) * d + j] = o[1 + j];
    }
  }
  return st;
}

bta_status inla_backward(inla_model* m, double* grad, int32_t use_graph, cudaStream_t stream) {
  if (!m || !grad) return BTA_ERR_ARG;
  if (m->ctx.empty() || !m->ctx[0].have_factors) return BTA_ERR_STATE;
  for (size_t e = 1; e < m->ctx.size(); ++e) m->ctx[e].have_factors = 0;
  bta_status st = run_group(m, 2, 1, m->ctx[0].have_factors - 1, use_graph, stream);
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

bta_status bta_gemm_mixed(int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                          int32_t lda, int32_t transA, const double* B, int32_t ldb,
                          int32_t transB, double beta, double* Cm, int32_t ldc, int32_t* status,
                          cudaStream_t stream) {
  if (M < 0 || N < 0 || K < 1 || !A || !B || !Cm) return BTA_ERR_ARG;
  Gemm g;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.transA = transA ? 1 : 0;
  g.B = B; g.ldb = ldb; g.transB = transB ? 1 : 0;
  g.C = Cm; g.ldc = ldc; g.Cin = Cm; g.ldcin = ldc;
  void* ws = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&ws, tc_gemm_ws_bytes(M, N, K), stream));
  bta_status st = tc_gemm_mixed(g, ws, status, stream);
  cudaFreeAsync(ws, stream);
  return st;
}

bta_status bta_gemm_emulated(int32_t M, int32_t N, int32_t K, double alpha, const double* A,
                             int32_t lda, int32_t transA, const double* B, int32_t ldb,
                             int32_t transB, double beta, double* Cm, int32_t ldc,
                             int32_t slices, int32_t* status, cudaStream_t stream) {
  if (M < 0 || N < 0 || K < 1 || K > 5120 || !A || !B || !Cm || slices < 6 || slices > 8)
    return BTA_ERR_ARG;
  Gemm g;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.transA = transA ? 1 : 0;
  g.B = B; g.ldb = ldb; g.transB = transB ? 1 : 0;
  g.C = Cm; g.ldc = ldc; g.Cin = Cm; g.ldcin = ldc;
  void* ws = nullptr;
  BTA_CUDA_TRY(cudaMallocAsync(&ws, ozaki_ws_bytes(M, N, K, slices), stream));
  bta_status st = ozaki_gemm(g, ws, status, slices, stream);
  cudaFreeAsync(ws, stream);
  return st;
}

bta_status bta_gemm_emulated_timed(int32_t M, int32_t N, int32_t K, double alpha,
                                   const double* A, int32_t lda, int32_t transA, const double* B,
                                   int32_t ldb, int32_t transB, double beta, double* Cm,
                                   int32_t ldc, int32_t slices, int32_t* status,
                                   float* kernel_ms, cudaStream_t stream) {
  if (M < 1 || N < 1 || K < 1 || K > 5120 || !A || !B || !Cm || slices < 6 || slices > 8 ||
      !kernel_ms)
    return BTA_ERR_ARG;
  Gemm g;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
  g.A = A; g.lda = lda; g.transA = transA ? 1 : 0;
  g.B = B; g.ldb = ldb; g.transB = transB ? 1 : 0;
  g.C = Cm; g.ldc = ldc; g.Cin = Cm; g.ldcin = ldc;
  cudaEvent_t marks[2] = {nullptr, nullptr};
  BTA_CUDA_TRY(cudaEventCreate(&marks[0]));
  BTA_CUDA_TRY(cudaEventCreate(&marks[1]));
  void* ws = nullptr;
  bta_status st = BTA_OK;
  if (cudaMallocAsync(&ws, ozaki_ws_bytes(M, N, K, slices), stream) != cudaSuccess) {
    cudaGetLastError();
    st = BTA_ERR_NOMEM;
  }
  if (st == BTA_OK) st = ozaki_gemm(g, ws, status, slices, stream, marks);
  if (ws) cudaFreeAsync(ws, stream);
  if (st == BTA_OK && cudaEventSynchronize(marks[1]) == cudaSuccess &&
      cudaEventElapsedTime(kernel_ms, marks[0], marks[1]) != cudaSuccess)
    st = BTA_ERR_CUDA;
  cudaEventDestroy(marks[0]);
  cudaEventDestroy(marks[1]);
  return st;
}

bta_status inla_batch_create(inla_model* const* models, int32_t count, inla_batch** out) {
  if (!models || !out || count < 1) return BTA_ERR_ARG;
  *out = nullptr;
  inla_batch* b = new (std::nothrow) inla_batch();
  if (!b) return BTA_ERR_NOMEM;
  for (int i = 0; i < count; ++i) {
    if (!models[i]) { delete b; return BTA_ERR_ARG; }
    for (int j = 0; j < i; ++j)
      if (models[j] == models[i]) { delete b; return BTA_ERR_ARG; }
    b->models.push_back(models[i]);
  }
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    delete b;
    return BTA_ERR_CUDA;
  }
  *out = b;
  return BTA_OK;
}

void inla_batch_destroy(inla_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (auto& row : b->exec)
    for (auto& e : row)
      if (e) cudaGraphExecDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  delete b;
}

// Record every model's evaluation (theta upload, sweeps, result download)
// as branches forked from s0.  The models' issue steps are taken round-robin
// (step j of every model, then step j + 1), so their operations are created
// interleaved and every model's streams start together.
static bta_status record_batch(inla_batch* b, int grad, int prec, cudaStream_t s0) {
  BTA_CUDA_TRY(cudaEventRecord(b->fork, s0));
  const size_t nm = b->models.size();
  std::vector<std::vector<IssueStep>> progs(nm);
  size_t longest = 0;
  for (size_t k = 0; k < nm; ++k) {
    inla_model* m = b->models[k];
    BTA_CUDA_TRY(cudaStreamWaitEvent(m->s0, b->fork, 0));
    BTA_CUDA_TRY(cudaMemcpyAsync(m->ctx[0].coefbuf + m->L.theta, m->htheta,
                                 m->d * sizeof(double), cudaMemcpyHostToDevice, m->s0));
    BTA_TRY(group_program(m, grad, 1, prec, m->s0, progs[k]));
    longest = std::max(longest, progs[k].size());
  }
  for (size_t j = 0; j < longest; ++j)
    for (size_t k = 0; k < nm; ++k)
      if (j < progs[k].size()) BTA_TRY(progs[k][j]());
  for (inla_model* m : b->models) {
    BTA_CUDA_TRY(cudaMemcpyAsync(m->hout, m->ctx[0].out, out_size(m->d) * sizeof(double),
                                 cudaMemcpyDeviceToHost, m->s0));
    BTA_CUDA_TRY(cudaEventRecord(m->evj, m->s0));
    BTA_CUDA_TRY(cudaStreamWaitEvent(s0, m->evj, 0));
  }
  return BTA_OK;
}

bta_status inla_batch_value_and_grad(inla_batch* b, const double* theta, int32_t ldt, double* f,
                                     double* grad, const inla_opts* opts, cudaStream_t stream) {
  if (!b || !theta || !f || ldt < 1) return BTA_ERR_ARG;
  const int prec = opts ? opts->precision : 0;
  if (prec < 0 || prec > 2) return BTA_ERR_ARG;
  const int g = grad ? 1 : 0;
  const int nm = (int)b->models.size();
  for (int i = 0; i < nm; ++i)   // mixed mode's refinement solves read the B blocks
    if (prec == 1 && b->models[i]->lowmem) return BTA_ERR_ARG;
  for (int i = 0; i < nm; ++i) {
    inla_model* m = b->models[i];
    if (m->d > ldt || !finite_theta(theta + (size_t)i * ldt, m->d)) return BTA_ERR_ARG;
    std::memcpy(m->htheta, theta + (size_t)i * ldt, m->d * sizeof(double));
  }
  if (!b->exec[g][prec]) {
    {  // an eager run first times the products' tile shapes (see run_group)
      TuneScope tune;
      BTA_TRY(record_batch(b, g, prec, stream));
      BTA_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    const int64_t before = g_launches;
    cudaStream_t cap;
    BTA_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    BTA_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    bta_status st = record_batch(b, g, prec, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    if (st != BTA_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
      return st;
    }
    BTA_CUDA_TRY(e);
    e = cudaGraphInstantiate(&b->exec[g][prec], graph, 0);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    BTA_CUDA_TRY(e);
    b->kernels[g][prec] = g_launches - before;
  }
  BTA_CUDA_TRY(cudaGraphLaunch(b->exec[g][prec], stream));
  BTA_CUDA_TRY(cudaStreamSynchronize(stream));
  bta_status st = BTA_OK;
  for (int i = 0; i < nm; ++i) {
    inla_model* m = b->models[i];
    const int no = out_size(m->d);
    int32_t tcs = 0;
    BTA_CUDA_TRY(cudaMemcpy(&tcs, m->ctx[0].fail + 2, sizeof(int32_t), cudaMemcpyDeviceToHost));
    m->last.assign(m->hout, m->hout + no);
    m->ctx[0].have_factors = g ? 0 : 1 + prec;
    m->launched += b->kernels[g][prec] / nm;
    f[i] = m->hout[0];
    if (grad)
      for (int j = 0; j < m->d; ++j) grad[(size_t)i * ldt + j] = m->hout[1 + j];
    st = worse(st, eval_status(m->hout + 1 + m->d, tcs));
  }
  return st;
}

bta_status inla_hessian(inla_model* m, const double* theta, double h, double* H, double* grad0,
                        const inla_opts* opts, cudaStream_t stream) {
  if (!m || !theta || !H || !(h > 0.0) || !finite_theta(theta, m->d)) return BTA_ERR_ARG;
  const int d = m->d;
  // rows: theta, then theta + h e_j, theta - h e_j for every j (Eq. 13)
  std::vector<double> pts((size_t)(2 * d + 1) * d), f(2 * d + 1), g((size_t)(2 * d + 1) * d);
  for (int r = 0; r < 2 * d + 1; ++r)
    for (int j = 0; j < d; ++j) pts[(size_t)r * d + j] = theta[j];
  for (int j = 0; j < d; ++j) {
    pts[(size_t)(1 + 2 * j) * d + j] += h;
    pts[(size_t)(2 + 2 * j) * d + j] -= h;
  }
  inla_opts o = opts ? *opts : inla_opts{0, 1, 1, 0};
  if (o.streams < 1) o.streams = 1;
  bta_status st = inla_value_and_grad(m, pts.data(), 2 * d + 1, f.data(), g.data(), &o, stream);
  if (st != BTA_OK) return st;
  for (int j = 0; j < d; ++j)
    for (int i = 0; i < d; ++i)   // column j: central difference of the gradient along e_j
      H[(size_t)i * d + j] = (g[(size_t)(1 + 2 * j) * d + i] - g[(size_t)(2 + 2 * j) * d + i]) /
                             (2.0 * h);
  if (grad0)
    for (int i = 0; i < d; ++i) grad0[i] = g[i];
  return BTA_OK;
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
  if (m->ctx.empty()) return BTA_ERR_STATE;
  BTA_CUDA_TRY(cudaMemcpyAsync(dst, m->ctx[0].x, ((size_t)m->n * m->ld + m->a) * sizeof(double),
                               cudaMemcpyDeviceToDevice, stream));
  return BTA_OK;
}

int64_t inla_kernel_launches(const inla_model* m) { return m ? m->launched : g_launches; }

}  // extern "C"
