// The three block sweeps over a BTA matrix (FP64):
//   factor_sweep  -- Algorithm 1, fused block Cholesky + lower solve
//   upper_solve   -- Eqs. 3-5
//   selinv_sweep  -- selected inversion with the Eq. 7 traces fused in
// Each step is a handful of tile-parallel products on the whole GPU; the
// diagonal factor is kept as L_Di^{-1} (see potrf.cu).
#include <algorithm>
#include <cmath>
#include <vector>

#include "sweep.cuh"

// Phase marks of the sweeps for timeline measurements: compile-time empty in
// the library.  A measurement build defines BTA_SWEEP_MARK(stream, tag, block)
// to stamp the time at which the stream's work reaches that point.  Tags:
// 0 / 3 a factor step's start / end, 1 / 2 around its diagonal factor, 4 / 5 a
// selected-inversion step's start / end.
#ifndef BTA_SWEEP_MARK
#define BTA_SWEEP_MARK(s, tag, i) ((void)0)
#endif

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

struct CopyDev {
  int lds, ldd, rows, cols, mode;
  double alpha;
  const double* src[kMaxBatch];
  double* dst[kMaxBatch];
};

__global__ void copy_batch_kernel(CopyDev d) {
  const double* __restrict__ src = d.src[blockIdx.y];
  double* __restrict__ dst = d.dst[blockIdx.y];
  const int64_t n = (int64_t)d.rows * d.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e % d.rows), j = (int)(e / d.rows);
    double v;
    if (d.mode == 1 && i < j) v = src[j + (int64_t)i * d.lds];
    else v = src[i + (int64_t)j * d.lds];
    dst[i + (int64_t)j * d.ldd] = d.alpha * v;
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

int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  int* slot = dev >= 0 && dev < 64 ? &cache[dev] : nullptr;
  if (slot && *slot > 0) return *slot;
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();
    v = 1;
  }
  if (slot) *slot = v;
  return v;
}

bta_status copy_block(const double* src, int lds, double* dst, int ldd, int rows, int cols,
                      double alpha, int mode, cudaStream_t s) {
  int64_t n = (int64_t)rows * cols;
  if (n <= 0) return BTA_OK;
  int grid = (int)std::min<int64_t>(cdiv(n, 256), 32 * sm_count());
  copy_kernel<<<grid, 256, 0, s>>>(src, lds, dst, ldd, rows, cols, alpha, mode);
  BTA_LAUNCHED();
  return BTA_OK;
}

bta_status copy_block_batch(int count, const double* const* src, int lds, double* const* dst,
                            int ldd, int rows, int cols, double alpha, int mode, cudaStream_t s) {
  const int64_t n = (int64_t)rows * cols;
  if (n <= 0 || count <= 0) return BTA_OK;
  CopyDev d;
  d.lds = lds; d.ldd = ldd; d.rows = rows; d.cols = cols; d.mode = mode; d.alpha = alpha;
  for (int z0 = 0; z0 < count; z0 += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, count - z0);
    for (int z = 0; z < cnt; ++z) {
      d.src[z] = src[z0 + z];
      d.dst[z] = dst[z0 + z];
    }
    int gx = (int)std::min<int64_t>(cdiv(n, 256), std::max(1, 32 * sm_count() / cnt));
    copy_batch_kernel<<<dim3(gx, cnt), 256, 0, s>>>(d);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

bta_status fill_value(double* p, int64_t n, double v, cudaStream_t s) {
  if (n <= 0) return BTA_OK;
  int grid = (int)std::min<int64_t>(cdiv(n, 256), 32 * sm_count());
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
  // a multiple of 256 bytes: a second workspace carved right after this one
  // keeps its blocks aligned for vector access
  const size_t d = 4 * m + 2 * (size_t)a * ld + (size_t)kGemvSplit * ld + a + 64;
  return sizeof(double) * ((d + 31) / 32 * 32);
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

bool arrow_fused(int ld, int a, int precision) {
  return precision == 2 && a > 0 && ld + a <= kOzakiMaxK;
}

size_t sweep_tc_ws_bytes(int ld, int a) {
  const int e = a > 0 && ld + a <= kOzakiMaxK ? a : 0;
  return std::max(tc_gemm_ws_bytes(ld, ld, ld),
                  ld <= kOzakiMaxK ? ozaki_ws_bytes(ld + e, ld, ld + e, 8) : (size_t)0);
}


namespace {

// Index groups of a set: all items, items with an arrow (grouped by a),
// items with a vector.
struct Groups {
  std::vector<int> all;
  std::vector<std::vector<int>> arrow;   // one group per distinct a > 0
  std::vector<int> vec;
};

Groups make_groups(const SweepItem* it, int m) {
  Groups g;
  for (int z = 0; z < m; ++z) {
    g.all.push_back(z);
    if (it[z].vec) g.vec.push_back(z);
    if (it[z].q.a > 0) {
      bool placed = false;
      for (auto& grp : g.arrow)
        if (it[grp[0]].q.a == it[z].q.a) { grp.push_back(z); placed = true; break; }
      if (!placed) g.arrow.push_back({z});
    }
  }
  return g;
}

// Gather per-item pointers for a batched launch.
template <class F>
std::vector<double*> ptrs(const std::vector<int>& idx, F f) {
  std::vector<double*> v;
  v.reserve(idx.size());
  for (int z : idx) v.push_back(f(z));
  return v;
}

inline const double* const* cp(const std::vector<double*>& v) {
  return reinterpret_cast<const double* const*>(v.data());
}

// A b x b product of the sweep over the items idx: batched FP64
// (precision 0), or one tensor-core product per matrix: split TF32
// (precision 1) or FP64 emulated from 8 BF16 slices (precision 2).
bta_status big_product(const Gemm& g, const SweepItem* it, const std::vector<int>& idx,
                       int precision, cudaStream_t s) {
  if (precision == 0 || (precision == 2 && g.K > 5120)) return gemm_f64(g, s);
  for (size_t z = 0; z < idx.size(); ++z) {
    const SweepWs& ws = it[idx[z]].ws;
    if (!ws.tc) return BTA_ERR_ARG;
    Gemm one = g;
    one.batch = 1;
    one.Ab = nullptr; one.Bb = nullptr; one.Cb = nullptr; one.Cinb = nullptr;
    one.A = g.Ab[z]; one.B = g.Bb[z]; one.C = g.Cb[z];
    one.Cin = g.Cinb ? g.Cinb[z] : g.Cb[z];
    if (precision == 2) {
      BTA_TRY(ozaki_gemm(one, ws.tc, ws.tcstat, 8, s));
    } else {
      BTA_TRY(tc_gemm_mixed(one, ws.tc, ws.tcstat, s));
    }
  }
  return BTA_OK;
}

bta_status check_set(const SweepItem* it, int m) {
  if (m < 1) return BTA_ERR_ARG;
  const bool low = it[0].q.B == nullptr;
  for (int z = 0; z < m; ++z) {
    if (it[z].q.n != it[0].q.n || it[z].q.ld != it[0].q.ld) return BTA_ERR_ARG;
    if (it[z].q.a > kMaxTip) return BTA_ERR_ARG;
    if ((it[z].q.B == nullptr) != low) return BTA_ERR_ARG;
    if (low && it[z].q.n > 1 && (!it[z].md || !it[z].lay || !it[z].coef || !it[z].W4))
      return BTA_ERR_ARG;
  }
  return BTA_OK;
}

// Low-memory sweeps: B_i of every item of idx into the item's W2.
bta_status assemble_b_items(const SweepItem* it, const std::vector<int>& idx, int i,
                            cudaStream_t s) {
  for (int z : idx)
    BTA_TRY(launch_assemble_b(*it[z].md, *it[z].lay, it[z].coef, i, it[z].ws.W2, s));
  return BTA_OK;
}

}  // namespace

// ----------------------------------------------------------------------------
// Algorithm 1 on a set of matrices
// ----------------------------------------------------------------------------
bta_status factor_sweep_multi(const SweepItem* it, int m, cudaStream_t s, cudaEvent_t mark,
                              int precision, int i0, int i1) {
  BTA_TRY(check_set(it, m));
  const int n = it[0].q.n, ld = it[0].q.ld;
  if (i1 < 0) i1 = n;
  if (i0 < 0 || i0 > i1 || i1 > n) return BTA_ERR_ARG;
  const int64_t blk = (int64_t)ld * ld;
  const int p = potrf_inv_slots(ld);
  const Groups G = make_groups(it, m);
  const int M = (int)G.all.size();
  if (i0 == 0)
    for (int z = 0; z < m; ++z) {
      if (it[z].q.a > 0 && it[z].vec) BTA_TRY(fill_value(it[z].ws.vT, it[z].q.a, 0.0, s));
      BTA_TRY(fill_value(it[z].slots + (int64_t)n * p, 1, 0.0, s));
    }
  auto D = [&](int z, int i) { return it[z].q.D + i * blk; };
  auto B = [&](int z, int i) { return it[z].q.B + i * blk; };
  auto Cb = [&](int z, int i) { return it[z].q.C + (int64_t)i * it[z].q.a * ld; };
  const bool low = it[0].q.B == nullptr;
  // where L_Bi lives: in place of B_i, or (low memory) in W1 / W4 by parity
  auto LB = [&](int z, int i) {
    return low ? ((i & 1) ? it[z].W4 : it[z].ws.W1) : B(z, i);
  };
  // Emulated FP64: one product per matrix; the arrow rides along (arrow_fused).
  const bool emu = precision == 2 && ld <= kOzakiMaxK;
  auto fused = [&](int z) { return emu && arrow_fused(ld, it[z].q.a, precision); };
  auto emulate = [&](int z, const Gemm& g) -> bta_status {
    if (!it[z].ws.tc) return BTA_ERR_ARG;
    return ozaki_gemm(g, it[z].ws.tc, it[z].ws.tcstat, 8, s);
  };
  // L_Ci (in Wc1) into C_i, then T -= L_Ci L_Ci^T
  auto arrow_tail = [&](const std::vector<int>& grp, int i) -> bta_status {
    const int a = it[grp[0]].q.a, c = (int)grp.size();
    auto Ci = ptrs(grp, [&](int z) { return Cb(z, i); });
    auto W = ptrs(grp, [&](int z) { return it[z].ws.Wc1; });
    auto T = ptrs(grp, [&](int z) { return it[z].q.T; });
    auto SK = ptrs(grp, [&](int z) { return it[z].ws.W3; });
    BTA_TRY(copy_block_batch(c, cp(W), a, Ci.data(), a, a, ld, 1.0, 0, s));
    Gemm h; h.M = a; h.N = a; h.K = ld; h.batch = c;
    h.Ab = cp(Ci); h.lda = a; h.Bb = cp(Ci); h.ldb = a; h.transB = 1;
    h.Cb = T.data(); h.ldc = a; h.Cinb = cp(T); h.ldcin = a; h.alpha = -1.0; h.beta = 1.0;
    h.sk_wsb = SK.data(); h.sk_cap = blk;
    return gemm_f64(h, s);
  };
  for (int i = i0; i < i1; ++i) {
    BTA_SWEEP_MARK(s, 0, i);
    if (i > 0) {
      if (emu) {  // D_i -= L_B,i-1 L_B,i-1^T (lower); rows below: C_i -= L_C,i-1 L_B,i-1^T
        for (int z : G.all) {
          Gemm g; g.M = ld; g.N = ld; g.K = ld;
          g.A = LB(z, i - 1); g.lda = ld; g.B = g.A; g.ldb = ld; g.transB = 1;
          g.C = D(z, i); g.ldc = ld; g.Cin = g.C; g.ldcin = ld;
          g.alpha = -1.0; g.beta = 1.0; g.out_lower = 1;
          if (fused(z)) {
            const int a = it[z].q.a;
            g.M = ld + a; g.a_rows = ld; g.A21 = {Cb(z, i - 1), a, 0};
            g.c_rows = ld; g.C2 = Cb(z, i); g.ldc2 = a; g.Cin2 = g.C2; g.ldcin2 = a;
          }
          BTA_TRY(emulate(z, g));
        }
      } else {  // D_i -= S_{i-1} = L_B,i-1 L_B,i-1^T (lower)
        auto Bp = ptrs(G.all, [&](int z) { return LB(z, i - 1); });
        auto Di = ptrs(G.all, [&](int z) { return D(z, i); });
        Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
        g.Ab = cp(Bp); g.lda = ld; g.Bb = cp(Bp); g.ldb = ld; g.transB = 1;
        g.Cb = Di.data(); g.ldc = ld; g.Cinb = cp(Di); g.ldcin = ld;
        g.alpha = -1.0; g.beta = 1.0; g.out_lower = 1;
        BTA_TRY(big_product(g, it, G.all, precision, s));
      }
      for (const auto& grp : G.arrow) {  // C_i -= L_C,i-1 L_B,i-1^T
        if (fused(grp[0])) continue;      // carried by the product above
        const int a = it[grp[0]].q.a;
        auto Cp = ptrs(grp, [&](int z) { return Cb(z, i - 1); });
        auto Bp = ptrs(grp, [&](int z) { return LB(z, i - 1); });
        auto Ci = ptrs(grp, [&](int z) { return Cb(z, i); });
        auto SK = ptrs(grp, [&](int z) { return it[z].ws.W3; });   // W3 is free here
        Gemm g; g.M = a; g.N = ld; g.K = ld; g.batch = (int)grp.size();
        g.Ab = cp(Cp); g.lda = a; g.Bb = cp(Bp); g.ldb = ld; g.transB = 1;
        g.Cb = Ci.data(); g.ldc = a; g.Cinb = cp(Ci); g.ldcin = a; g.alpha = -1.0; g.beta = 1.0;
        g.sk_wsb = SK.data(); g.sk_cap = blk;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    {  // L_Di^{-1} in place, log-det slots
      auto Di = ptrs(G.all, [&](int z) { return D(z, i); });
      auto W = ptrs(G.all, [&](int z) { return it[z].ws.pot; });
      auto sl = ptrs(G.all, [&](int z) { return it[z].slots + (int64_t)i * p; });
      std::vector<int32_t*> fl;
      std::vector<int32_t> code(M, i);
      for (int z : G.all) fl.push_back(it[z].fail);
      std::vector<void*> tw;
      std::vector<int32_t*> ts;
      for (int z : G.all) {
        tw.push_back(it[z].ws.tc);
        ts.push_back(it[z].ws.tcstat);
      }
      BTA_SWEEP_MARK(s, 1, i);
      BTA_TRY(potrf_inv_batch_prec(M, Di.data(), ld, ld, W.data(), sl.data(), fl.data(),
                                   code.data(), precision, tw.data(), ts.data(), s));
      BTA_SWEEP_MARK(s, 2, i);
      if (i == 0 && mark) BTA_CUDA_TRY(cudaEventRecord(mark, s));
    }
    const bool with_b = emu && i < n - 1;   // L_Ci as extra rows of L_Bi's product
    for (const auto& grp : G.arrow) {  // L_Ci = C_i L_Di^{-T};  T -= L_Ci L_Ci^T
      if (with_b && fused(grp[0])) continue;
      const int a = it[grp[0]].q.a, c = (int)grp.size();
      auto Ci = ptrs(grp, [&](int z) { return Cb(z, i); });
      auto Di = ptrs(grp, [&](int z) { return D(z, i); });
      auto W = ptrs(grp, [&](int z) { return it[z].ws.Wc1; });
      auto SK = ptrs(grp, [&](int z) { return it[z].ws.W3; });
      Gemm g; g.M = a; g.N = ld; g.K = ld; g.batch = c;
      g.Ab = cp(Ci); g.lda = a; g.Bb = cp(Di); g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
      g.Cb = W.data(); g.ldc = a;
      g.sk_wsb = SK.data(); g.sk_cap = blk;
      BTA_TRY(gemm_f64(g, s));
      BTA_TRY(arrow_tail(grp, i));
    }
    if (i < n - 1) {  // L_Bi = B_i L_Di^{-T}
      if (low) BTA_TRY(assemble_b_items(it, G.all, i, s));
      auto Bi = ptrs(G.all, [&](int z) { return low ? it[z].ws.W2 : B(z, i); });
      auto Di = ptrs(G.all, [&](int z) { return D(z, i); });
      auto W = ptrs(G.all, [&](int z) { return low ? LB(z, i) : it[z].ws.W1; });
      if (emu) {  // rows below: L_Ci = C_i L_Di^{-T} into Wc1
        for (size_t q = 0; q < G.all.size(); ++q) {
          const int z = G.all[q];
          Gemm g; g.M = ld; g.N = ld; g.K = ld;
          g.A = Bi[q]; g.lda = ld; g.B = Di[q]; g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
          g.C = W[q]; g.ldc = ld;
          if (fused(z)) {
            const int a = it[z].q.a;
            g.M = ld + a; g.a_rows = ld; g.A21 = {Cb(z, i), a, 0};
            g.c_rows = ld; g.C2 = it[z].ws.Wc1; g.ldc2 = a;
          }
          BTA_TRY(emulate(z, g));
        }
      } else {
        Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
        g.Ab = cp(Bi); g.lda = ld; g.Bb = cp(Di); g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
        g.Cb = W.data(); g.ldc = ld;
        BTA_TRY(big_product(g, it, G.all, precision, s));
      }
      if (!low) BTA_TRY(copy_block_batch(M, cp(W), ld, Bi.data(), ld, ld, ld, 1.0, 0, s));
      if (with_b)
        for (const auto& grp : G.arrow)
          if (fused(grp[0])) BTA_TRY(arrow_tail(grp, i));
    }
    if (!G.vec.empty()) {  // z_i = L_Di^{-1} (r_i - L_B,i-1 z_{i-1});  v_T += L_Ci z_i
      const int c = (int)G.vec.size();
      auto ri = ptrs(G.vec, [&](int z) { return it[z].vec + (int64_t)i * ld; });
      auto gv = ptrs(G.vec, [&](int z) { return it[z].ws.gv; });
      if (i > 0) {
        auto Bp = ptrs(G.vec, [&](int z) { return LB(z, i - 1); });
        auto rp = ptrs(G.vec, [&](int z) { return it[z].vec + (int64_t)(i - 1) * ld; });
        Gemv g; g.M = ld; g.K = ld; g.lda = ld; g.alpha = -1.0; g.beta = 1.0; g.batch = c;
        g.Ab = cp(Bp); g.xb = cp(rp); g.yb = ri.data(); g.yinb = cp(ri); g.workb = gv.data();
        BTA_TRY(gemv_f64(g, nullptr, s));
      }
      auto Di = ptrs(G.vec, [&](int z) { return D(z, i); });
      Gemv g; g.M = ld; g.K = ld; g.lda = ld; g.triA = TRI_LOWER; g.batch = c;
      g.Ab = cp(Di); g.xb = cp(ri); g.yb = ri.data(); g.workb = gv.data();
      BTA_TRY(gemv_f64(g, nullptr, s));
      for (int z : G.vec) {
        if (it[z].q.a == 0) continue;
        Gemv h; h.M = it[z].q.a; h.K = ld; h.A = Cb(z, i); h.lda = it[z].q.a;
        h.x = it[z].vec + (int64_t)i * ld; h.y = it[z].ws.vT; h.yin = it[z].ws.vT; h.beta = 1.0;
        BTA_TRY(gemv_f64(h, it[z].ws.gv, s));
      }
    }
    BTA_SWEEP_MARK(s, 3, i);
  }
  if (i1 < n) return BTA_OK;
  for (int z = 0; z < m; ++z) {
    const int a = it[z].q.a;
    if (a == 0) continue;
    tip_kernel<<<1, 32, 0, s>>>(0, a, it[z].q.T, it[z].vec ? it[z].vec + (int64_t)n * ld : nullptr,
                                it[z].ws.vT, it[z].slots + (int64_t)n * p, it[z].fail, n);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

bta_status factor_sweep(const bta_desc& q, double* rhs, double* slots, int32_t* fail,
                        const SweepWs& ws, cudaStream_t s, int precision) {
  SweepItem item;
  item.q = q; item.vec = rhs; item.slots = slots; item.fail = fail; item.ws = ws;
  return factor_sweep_multi(&item, 1, s, nullptr, precision);
}

// ----------------------------------------------------------------------------
// Residual d - Q x of an assembled BTA matrix (the refinement step of
// bta_solve), as GEMVs on its blocks.  D_i is stored as its lower triangle:
// D_i x = L x + L^T x - diag(D_i) x with L the stored lower part.
// ----------------------------------------------------------------------------
namespace {
__global__ void diag_axpy_kernel(const double* __restrict__ D, int ld, const double* x,
                                 double* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ld) y[i] = fma(D[i + (int64_t)i * ld], x[i], y[i]);
}
}  // namespace

bta_status bta_residual(const bta_desc& q, const double* x, double* d, double* gv,
                        cudaStream_t s) {
  const int n = q.n, ld = q.ld, a = q.a;
  const int64_t blk = (int64_t)ld * ld;
  const double* xT = x + (int64_t)n * ld;
  double* dT = d + (int64_t)n * ld;
  for (int i = 0; i < n; ++i) {
    const double* xi = x + (int64_t)i * ld;
    double* di = d + (int64_t)i * ld;
    const double* Di = q.D + i * blk;
    auto minus = [&](const double* A, int lda, int M, int K, int trans, int tri,
                     const double* v, double* y) {
      Gemv g; g.M = M; g.K = K; g.A = A; g.lda = lda; g.transA = trans; g.triA = tri;
      g.x = v; g.y = y; g.yin = y; g.alpha = -1.0; g.beta = 1.0;
      return gemv_f64(g, gv, s);
    };
    BTA_TRY(minus(Di, ld, ld, ld, 0, TRI_LOWER, xi, di));          // - L x
    BTA_TRY(minus(Di, ld, ld, ld, 1, TRI_UPPER, xi, di));          // - L^T x
    diag_axpy_kernel<<<cdiv(ld, 256), 256, 0, s>>>(Di, ld, xi, di);   // + diag x
    BTA_LAUNCHED();
    if (i > 0) BTA_TRY(minus(q.B + (i - 1) * blk, ld, ld, ld, 0, TRI_NONE, xi - ld, di));
    if (i < n - 1) BTA_TRY(minus(q.B + i * blk, ld, ld, ld, 1, TRI_NONE, xi + ld, di));
    if (a > 0) {
      const double* Ci = q.C + (int64_t)i * a * ld;
      BTA_TRY(minus(Ci, a, ld, a, 1, TRI_NONE, xT, di));           // - C_i^T x_T
      BTA_TRY(minus(Ci, a, a, ld, 0, TRI_NONE, xi, dT));           // tip row: - C_i x_i
    }
  }
  if (a > 0) {   // - T x_T (lower triangle referenced, as D)
    Gemv g; g.M = a; g.K = a; g.A = q.T; g.lda = a; g.triA = TRI_LOWER;
    g.x = xT; g.y = dT; g.yin = dT; g.alpha = -1.0; g.beta = 1.0;
    BTA_TRY(gemv_f64(g, gv, s));
    g.transA = 1; g.triA = TRI_UPPER;
    BTA_TRY(gemv_f64(g, gv, s));
    diag_axpy_kernel<<<1, 32, 0, s>>>(q.T, a, xT, dT);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

// ----------------------------------------------------------------------------
// Lower solve alone (L z = r) on one matrix, for bta_solve(lower = 1)
// ----------------------------------------------------------------------------
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
  if (a > 0) BTA_TRY(tip_forward(q, z + (int64_t)n * ld, ws.vT, s));
  return BTA_OK;
}

// ----------------------------------------------------------------------------
// Eqs. 3-5 on a set of matrices (items with a vector)
// ----------------------------------------------------------------------------
bta_status upper_solve_multi(const SweepItem* it, int m, cudaStream_t s) {
  BTA_TRY(check_set(it, m));
  const int n = it[0].q.n, ld = it[0].q.ld;
  const int64_t blk = (int64_t)ld * ld;
  const Groups G = make_groups(it, m);
  if (G.vec.empty()) return BTA_OK;
  const int c = (int)G.vec.size();
  for (int z : G.vec) {
    const int a = it[z].q.a;
    if (a == 0) continue;
    tip_kernel<<<1, 32, 0, s>>>(1, a, it[z].q.T, it[z].vec + (int64_t)n * ld, nullptr, nullptr,
                                nullptr, 0);
    BTA_LAUNCHED();
  }
  auto gv = ptrs(G.vec, [&](int z) { return it[z].ws.gv; });
  for (int i = n - 1; i >= 0; --i) {
    auto zi = ptrs(G.vec, [&](int z) { return it[z].vec + (int64_t)i * ld; });
    for (int z : G.vec) {  // z_i -= L_Ci^T x_T
      const int a = it[z].q.a;
      if (a == 0) continue;
      double* zz = it[z].vec + (int64_t)i * ld;
      Gemv g; g.M = ld; g.K = a; g.A = it[z].q.C + (int64_t)i * a * ld; g.lda = a; g.transA = 1;
      g.x = it[z].vec + (int64_t)n * ld; g.y = zz; g.yin = zz; g.alpha = -1.0; g.beta = 1.0;
      BTA_TRY(gemv_f64(g, it[z].ws.gv, s));
    }
    if (i < n - 1 && it[0].q.B) {  // z_i -= L_Bi^T x_{i+1}
      auto Bi = ptrs(G.vec, [&](int z) { return it[z].q.B + i * blk; });
      auto xn = ptrs(G.vec, [&](int z) { return it[z].vec + (int64_t)(i + 1) * ld; });
      Gemv g; g.M = ld; g.K = ld; g.lda = ld; g.transA = 1; g.alpha = -1.0; g.beta = 1.0;
      g.batch = c; g.Ab = cp(Bi); g.xb = cp(xn); g.yb = zi.data(); g.yinb = cp(zi);
      g.workb = gv.data();
      BTA_TRY(gemv_f64(g, nullptr, s));
    } else if (i < n - 1) {
      // low memory: L_Bi^T x_{i+1} = L_Di^{-1} (B_i^T x_{i+1}), B_i assembled into W2,
      // the product into W3's first ld entries
      BTA_TRY(assemble_b_items(it, G.vec, i, s));
      auto W2 = ptrs(G.vec, [&](int z) { return it[z].ws.W2; });
      auto t = ptrs(G.vec, [&](int z) { return it[z].ws.W3; });
      auto xn = ptrs(G.vec, [&](int z) { return it[z].vec + (int64_t)(i + 1) * ld; });
      Gemv g; g.M = ld; g.K = ld; g.lda = ld; g.transA = 1; g.batch = c;
      g.Ab = cp(W2); g.xb = cp(xn); g.yb = t.data(); g.workb = gv.data();
      BTA_TRY(gemv_f64(g, nullptr, s));
      auto Di = ptrs(G.vec, [&](int z) { return it[z].q.D + i * blk; });
      Gemv h; h.M = ld; h.K = ld; h.lda = ld; h.triA = TRI_LOWER; h.alpha = -1.0; h.beta = 1.0;
      h.batch = c; h.Ab = cp(Di); h.xb = cp(t); h.yb = zi.data(); h.yinb = cp(zi);
      h.workb = gv.data();
      BTA_TRY(gemv_f64(h, nullptr, s));
    }
    {  // x_i = L_Di^{-T} z_i
      auto Di = ptrs(G.vec, [&](int z) { return it[z].q.D + i * blk; });
      Gemv g; g.M = ld; g.K = ld; g.lda = ld; g.transA = 1; g.triA = TRI_UPPER;
      g.batch = c; g.Ab = cp(Di); g.xb = cp(zi); g.yb = zi.data(); g.workb = gv.data();
      BTA_TRY(gemv_f64(g, nullptr, s));
    }
  }
  return BTA_OK;
}

bta_status upper_solve(const bta_desc& q, double* z, const SweepWs& ws, cudaStream_t s) {
  SweepItem item;
  item.q = q; item.vec = z; item.ws = ws;
  return upper_solve_multi(&item, 1, s);
}

// ----------------------------------------------------------------------------
// Selected inversion, in place, on a set of matrices, with the fused Eq. 7
// reductions.  With F_Bi = L_Bi L_Di^{-1}, F_Ci = L_Ci L_Di^{-1}:
//   Z_Ci = -Z_T F_Ci - Z_C,i+1 F_Bi
//   Z_Bi = -Z_D,i+1 F_Bi - Z_C,i+1^T F_Ci
//   Z_Di = L_Di^{-T} L_Di^{-1} - Z_Bi^T F_Bi - Z_Ci^T F_Ci
// ----------------------------------------------------------------------------
bta_status selinv_sweep_multi(const SweepItem* it, int m, cudaStream_t s, int precision,
                              int i_hi, int i_lo) {
  BTA_TRY(check_set(it, m));
  const int n = it[0].q.n, ld = it[0].q.ld;
  if (i_hi < 0) i_hi = n - 1;
  if (i_lo < 0 || i_hi >= n || i_lo > i_hi + 1) return BTA_ERR_ARG;
  const int64_t blk = (int64_t)ld * ld;
  const Groups G = make_groups(it, m);
  const int M = (int)G.all.size();
  auto D = [&](int z, int i) { return it[z].q.D + i * blk; };
  auto B = [&](int z, int i) { return it[z].q.B + i * blk; };
  auto Cb = [&](int z, int i) { return it[z].q.C + (int64_t)i * it[z].q.a * ld; };
  if (i_hi == n - 1)
    for (int z = 0; z < m; ++z) {
      if (it[z].q.a == 0) continue;
      tip_kernel<<<1, 32, 0, s>>>(2, it[z].q.a, it[z].q.T, nullptr, nullptr, nullptr, nullptr, 0);
      BTA_LAUNCHED();
    }
  auto W1 = ptrs(G.all, [&](int z) { return it[z].ws.W1; });
  auto W2 = ptrs(G.all, [&](int z) { return it[z].ws.W2; });
  auto W3 = ptrs(G.all, [&](int z) { return it[z].ws.W3; });
  const bool low = it[0].q.B == nullptr;
  // Emulated FP64: one product per matrix; the arrow rides along (arrow_fused).
  const bool emu = precision == 2 && ld <= kOzakiMaxK;
  auto fused = [&](int z) { return emu && arrow_fused(ld, it[z].q.a, precision); };
  auto emulate = [&](int z, const Gemm& g) -> bta_status {
    if (!it[z].ws.tc) return BTA_ERR_ARG;
    return ozaki_gemm(g, it[z].ws.tc, it[z].ws.tcstat, 8, s);
  };
  for (int i = i_hi; i >= i_lo; --i) {
    BTA_SWEEP_MARK(s, 4, i);
    const bool hasB = i < n - 1;
    auto Di = ptrs(G.all, [&](int z) { return D(z, i); });
    if (hasB && low) {  // low memory: W3 = L_Bi = B_i L_Di^{-T}, B_i assembled into W2
      BTA_TRY(assemble_b_items(it, G.all, i, s));
      Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
      g.Ab = cp(W2); g.lda = ld; g.Bb = cp(Di); g.ldb = ld; g.transB = 1; g.triB = TRI_UPPER;
      g.Cb = W3.data(); g.ldc = ld;
      BTA_TRY(big_product(g, it, G.all, precision, s));
    }
    if (hasB) {  // W1 = F_B = L_Bi L_Di^{-1}
      auto Bi = ptrs(G.all, [&](int z) { return low ? it[z].ws.W3 : B(z, i); });
      if (emu) {  // rows below: Wc1 = F_C = L_Ci L_Di^{-1}
        for (size_t q = 0; q < G.all.size(); ++q) {
          const int z = G.all[q];
          Gemm g; g.M = ld; g.N = ld; g.K = ld;
          g.A = Bi[q]; g.lda = ld; g.B = Di[q]; g.ldb = ld; g.triB = TRI_LOWER;
          g.C = W1[q]; g.ldc = ld;
          if (fused(z)) {
            const int a = it[z].q.a;
            g.M = ld + a; g.a_rows = ld; g.A21 = {Cb(z, i), a, 0};
            g.c_rows = ld; g.C2 = it[z].ws.Wc1; g.ldc2 = a;
          }
          BTA_TRY(emulate(z, g));
        }
      } else {
        Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
        g.Ab = cp(Bi); g.lda = ld; g.Bb = cp(Di); g.ldb = ld; g.triB = TRI_LOWER;
        g.Cb = W1.data(); g.ldc = ld;
        BTA_TRY(big_product(g, it, G.all, precision, s));
      }
    }
    for (const auto& grp : G.arrow) {
      // with B_i, an arrow carried by the products (arrow_fused) gets F_C above
      // and Z_C with Z_B below
      if (hasB && fused(grp[0])) continue;
      const int a = it[grp[0]].q.a, c = (int)grp.size();
      auto Ci = ptrs(grp, [&](int z) { return Cb(z, i); });
      auto Dg = ptrs(grp, [&](int z) { return D(z, i); });
      auto Wc1 = ptrs(grp, [&](int z) { return it[z].ws.Wc1; });
      auto Wc2 = ptrs(grp, [&](int z) { return it[z].ws.Wc2; });
      auto T = ptrs(grp, [&](int z) { return it[z].q.T; });
      auto SK = ptrs(grp, [&](int z) { return it[z].ws.W3; });   // W3 is free until LAUUM
      {  // Wc1 = F_C = L_Ci L_Di^{-1}
        Gemm g; g.M = a; g.N = ld; g.K = ld; g.batch = c;
        g.Ab = cp(Ci); g.lda = a; g.Bb = cp(Dg); g.ldb = ld; g.triB = TRI_LOWER;
        g.Cb = Wc1.data(); g.ldc = a;
        g.sk_wsb = SK.data(); g.sk_cap = blk;
        BTA_TRY(gemm_f64(g, s));
      }
      {  // Wc2 = -Z_T F_C
        Gemm g; g.M = a; g.N = ld; g.K = a; g.batch = c;
        g.Ab = cp(T); g.lda = a; g.Bb = cp(Wc1); g.ldb = a;
        g.Cb = Wc2.data(); g.ldc = a; g.alpha = -1.0;
        BTA_TRY(gemm_f64(g, s));
      }
      if (hasB) {  // Wc2 -= Z_C,i+1 F_B
        auto Cn = ptrs(grp, [&](int z) { return Cb(z, i + 1); });
        auto W1g = ptrs(grp, [&](int z) { return it[z].ws.W1; });
        Gemm g; g.M = a; g.N = ld; g.K = ld; g.batch = c;
        g.Ab = cp(Cn); g.lda = a; g.Bb = cp(W1g); g.ldb = ld;
        g.Cb = Wc2.data(); g.ldc = a; g.Cinb = cp(Wc2); g.ldcin = a; g.alpha = -1.0;
        g.beta = 1.0;
        g.sk_wsb = SK.data(); g.sk_cap = blk;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    if (hasB) {
      auto Dn = ptrs(G.all, [&](int z) { return D(z, i + 1); });
      if (emu) {
        // W2 = Z_B = -Z_D,i+1 F_B; an arrow carried along as a 2 x 2 block
        // product: [W2; Wc2] = -[Z_D,i+1, Z_C,i+1^T; Z_C,i+1, Z_T] [F_B; F_C],
        // i.e. also W2 -= Z_C,i+1^T F_C and Wc2 = Z_C = -Z_C,i+1 F_B - Z_T F_C
        for (size_t q = 0; q < G.all.size(); ++q) {
          const int z = G.all[q];
          Gemm g; g.M = ld; g.N = ld; g.K = ld;
          g.A = Dn[q]; g.lda = ld; g.B = W1[q]; g.ldb = ld;
          g.C = W2[q]; g.ldc = ld; g.alpha = -1.0;
          if (fused(z)) {
            const int a = it[z].q.a;
            const double* Cn = Cb(z, i + 1);
            g.M = ld + a; g.K = ld + a; g.a_rows = ld; g.a_k = ld;
            g.A12 = {Cn, a, 1}; g.A21 = {Cn, a, 0}; g.A22 = {it[z].q.T, a, 0};
            g.b_k = ld; g.B21 = {it[z].ws.Wc1, a, 0};
            g.c_rows = ld; g.C2 = it[z].ws.Wc2; g.ldc2 = a;
          }
          BTA_TRY(emulate(z, g));
        }
      } else {  // W2 = Z_B = -Z_D,i+1 F_B
        Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
        g.Ab = cp(Dn); g.lda = ld; g.Bb = cp(W1); g.ldb = ld;
        g.Cb = W2.data(); g.ldc = ld; g.alpha = -1.0;
        BTA_TRY(big_product(g, it, G.all, precision, s));
      }
      for (const auto& grp : G.arrow) {  // W2 -= Z_C,i+1^T F_C
        if (fused(grp[0])) continue;
        const int a = it[grp[0]].q.a, c = (int)grp.size();
        auto Cn = ptrs(grp, [&](int z) { return Cb(z, i + 1); });
        auto Wc1 = ptrs(grp, [&](int z) { return it[z].ws.Wc1; });
        auto W2g = ptrs(grp, [&](int z) { return it[z].ws.W2; });
        Gemm g; g.M = ld; g.N = ld; g.K = a; g.batch = c;
        g.Ab = cp(Cn); g.lda = a; g.transA = 1; g.Bb = cp(Wc1); g.ldb = a;
        g.Cb = W2g.data(); g.ldc = ld; g.Cinb = cp(W2g); g.ldcin = ld; g.alpha = -1.0;
        g.beta = 1.0;
        BTA_TRY(gemm_f64(g, s));
      }
    }
    {  // W3 = L_Di^{-T} L_Di^{-1} (lower part)
      Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
      g.Ab = cp(Di); g.lda = ld; g.transA = 1; g.triA = TRI_UPPER;
      g.Bb = cp(Di); g.ldb = ld; g.triB = TRI_LOWER;
      g.Cb = W3.data(); g.ldc = ld; g.out_lower = 1;
      BTA_TRY(big_product(g, it, G.all, precision, s));
    }
    if (hasB) {  // W3 -= Z_B^T F_B
      if (emu) {  // an arrow carried along extends K: W3 -= [Z_B; Z_C]^T [F_B; F_C]
        for (size_t q = 0; q < G.all.size(); ++q) {
          const int z = G.all[q];
          Gemm g; g.M = ld; g.N = ld; g.K = ld;
          g.A = W2[q]; g.lda = ld; g.transA = 1; g.B = W1[q]; g.ldb = ld;
          g.C = W3[q]; g.ldc = ld; g.Cin = W3[q]; g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
          g.out_lower = 1;
          if (fused(z)) {
            const int a = it[z].q.a;
            g.K = ld + a; g.a_k = ld; g.A12 = {it[z].ws.Wc2, a, 1};
            g.b_k = ld; g.B21 = {it[z].ws.Wc1, a, 0};
          }
          BTA_TRY(emulate(z, g));
        }
      } else {
        Gemm g; g.M = ld; g.N = ld; g.K = ld; g.batch = M;
        g.Ab = cp(W2); g.lda = ld; g.transA = 1; g.Bb = cp(W1); g.ldb = ld;
        g.Cb = W3.data(); g.ldc = ld; g.Cinb = cp(W3); g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
        g.out_lower = 1;
        BTA_TRY(big_product(g, it, G.all, precision, s));
      }
    }
    for (const auto& grp : G.arrow) {  // W3 -= Z_C^T F_C
      if (hasB && fused(grp[0])) continue;
      const int a = it[grp[0]].q.a, c = (int)grp.size();
      auto Wc1 = ptrs(grp, [&](int z) { return it[z].ws.Wc1; });
      auto Wc2 = ptrs(grp, [&](int z) { return it[z].ws.Wc2; });
      auto W3g = ptrs(grp, [&](int z) { return it[z].ws.W3; });
      Gemm g; g.M = ld; g.N = ld; g.K = a; g.batch = c;
      g.Ab = cp(Wc2); g.lda = a; g.transA = 1; g.Bb = cp(Wc1); g.ldb = a;
      g.Cb = W3g.data(); g.ldc = ld; g.Cinb = cp(W3g); g.ldcin = ld; g.alpha = -1.0; g.beta = 1.0;
      g.out_lower = 1;
      BTA_TRY(gemm_f64(g, s));
    }
    BTA_TRY(copy_block_batch(M, cp(W3), ld, Di.data(), ld, ld, ld, 1.0, 1, s));   // Z_D (full)
    if (hasB && !low) {   // Z_B in place of L_Bi (low memory: reduced from W2 below)
      auto Bi = ptrs(G.all, [&](int z) { return B(z, i); });
      BTA_TRY(copy_block_batch(M, cp(W2), ld, Bi.data(), ld, ld, ld, 1.0, 0, s));
    }
    for (const auto& grp : G.arrow) {
      const int a = it[grp[0]].q.a, c = (int)grp.size();
      auto Wc2 = ptrs(grp, [&](int z) { return it[z].ws.Wc2; });
      auto Ci = ptrs(grp, [&](int z) { return Cb(z, i); });
      BTA_TRY(copy_block_batch(c, cp(Wc2), a, Ci.data(), a, a, ld, 1.0, 0, s));
    }
    for (int z = 0; z < m; ++z) {
      const SelinvFuse* fz = it[z].fuse;
      if (!fz) continue;
      const ModelDev& md = *fz->md;
      const int kk = md.k * md.k, pch = pattern_chunks(md);
      BTA_TRY(launch_pattern_dot(md, D(z, i), fz->counts, i,
                                 fz->PD + (int64_t)i * kk * pch * kNP, s));
      if (hasB)
        BTA_TRY(launch_pattern_dot(md, low ? it[z].ws.W2 : B(z, i), 0, i,
                                   fz->PB + (int64_t)i * kk * pch * kNP, s));
      if (it[z].q.a > 0 && fz->PC)
        BTA_TRY(launch_arrow_dot(md, Cb(z, i), i, fz->PC + (int64_t)i * md.k * arrow_chunks(md),
                                 s));
    }
    BTA_SWEEP_MARK(s, 5, i);
  }
  return BTA_OK;
}

bta_status selinv_sweep(const bta_desc& q, const SweepWs& ws, const SelinvFuse* fuse,
                        cudaStream_t s) {
  SweepItem item;
  item.q = q; item.ws = ws; item.fuse = fuse;
  return selinv_sweep_multi(&item, 1, s);
}

}  // namespace bta
