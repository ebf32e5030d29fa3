// Diagonal-block Cholesky factor and inverse as one persistent kernel over a
// tile task graph (FP64, 32 x 32 tiles, p = n / 32 tile rows).
//
// Same contract as the recursive potrf_inv: on return the lower triangle of
// A holds L^{-1} (A = L L^T), one log-det slot per diagonal tile, the failure
// code on a non-positive pivot.  The recursion issues ~5 p dependent
// launches per block, each using a sliver of the GPU; here the whole block
// is one launch whose CTAs pull tasks from a list in topological order and
// start each as soon as the tiles it reads are final.
//
// Tasks, for step k = 0..p-1 (A's lower tiles are reused in place: first the
// trailing matrix W, then the inverse's accumulator R, then the inverse X):
//   F(k)      leaf on W_kk: D / unit-L elimination with its inverse
//             -> X_kk = L_kk^{-1} into A_kk, log-det slot k
//   S(i,k)    L_ik = W_ik X_kk^T                     (into the scratch Lt)
//   G(k,j)    X_kj = X_kk R_kj            (j < k; R_kj = -sum_m L_km X_mj)
//   U(i,j,k)  W_ij -= L_ik L_jk^T         (k < j <= i; column k+1 first)
//   V(i,j,k)  R_ij -= L_ik X_kj           (k < i, j <= k; R_ij = -L_ij X_jj at k = j)
// A task waits only for tasks earlier in the list, which running CTAs hold,
// so the graph always drains.  Per-tile counters (W updates applied, R
// updates applied, F/S/G done) are published with release stores after the
// tile is written and read with acquire loads; tile data are read through
// L2 (ld.global.cg).  Every wait is bounded by a 2 s globaltimer limit; on
// expiry the CTA raises a shared abort flag, records the timeout code in the
// block's failure word and returns, and every other CTA returns at its next
// wait.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "common.cuh"

namespace bta {
namespace {

constexpr int T = kPad;                 // tile size
constexpr int kDagThreads = 256;
constexpr int kMaxP = 160;              // tile rows supported (ld <= 5120)
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr int32_t kFailTimeout = 0x40000000;

enum : int { TK_F = 0, TK_S = 1, TK_G = 2, TK_U = 3, TK_V = 4, TK_C = 5 };

struct DagInst {
  double* A;       // n x n block, ld
  double* Lt;      // scratch: L tiles (i > k), tile (i,k) at Lt + (i(i-1)/2 + k)*T*T
  int* st;         // counters: cntW[p*p], cntR[p*p], doneF[p], doneS[p*p], doneG[p*p]
  double* slots;   // log-det slots (p)
  int32_t* fail;
  int32_t code;
};

struct DagArgs {
  int p, ld, cnt;
  int total;                // tasks over all instances
  int* counter;             // global task ticket
  int* abort;               // shared abort flag
  int* smbusy;              // per SM: chain tasks running there (see TK_C)
  int yield;                // bulk tasks wait while a chain task holds their SM
  int off[kMaxP + 1];       // task offset of each step within one instance
  DagInst inst[kMaxBatch];
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int sm_id() {
  int v;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
  return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *p >= need (bounded); false on timeout / abort.
__device__ bool wait_ge(const int* p, int need, int* abort) {
  if (ld_acquire(p) >= need) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    __nanosleep(64);
    if (ld_acquire(p) >= need) return true;
    if (ld_acquire(abort)) return false;
    if (now_ns() - t0 > kWaitNs) {
      atomicExch(abort, 1);
      return false;
    }
  }
}

// Tile (r, c) of the n x n block, column-major with leading dimension ld.
__device__ __forceinline__ double* tile(double* A, int ld, int r, int c) {
  return A + (int64_t)c * T * ld + (int64_t)r * T;
}

// Load a 32 x 32 tile (column-major, ld) into smem S[row][col] through L2.
__device__ __forceinline__ void load_tile(double (*S)[T + 1], const double* src, int ld) {
  for (int e = threadIdx.x; e < T * T; e += kDagThreads) {
    const int r = e % T, c = e / T;
    S[r][c] = __ldcg(src + (int64_t)c * ld + r);
  }
}

__device__ __forceinline__ void store_tile(double* dst, int ld, double (*S)[T + 1], bool lower) {
  for (int e = threadIdx.x; e < T * T; e += kDagThreads) {
    const int r = e % T, c = e / T;
    if (!lower || r >= c) dst[(int64_t)c * ld + r] = S[r][c];
  }
}

// out[r][c] (+)= sign * sum_m X[r][m] * Y'[m][c], with Y' = Y^T when ytrans.
// 256 threads, each 2 x 2 outputs.
__device__ __forceinline__ void tile_mm(double (*X)[T + 1], double (*Y)[T + 1], bool ytrans,
                                        double (*out)[T + 1], double sign, bool accumulate) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
#pragma unroll 8
  for (int m = 0; m < T; ++m) {
    const double x0 = X[tx][m], x1 = X[tx + 16][m];
    const double y0 = ytrans ? Y[ty][m] : Y[m][ty];
    const double y1 = ytrans ? Y[ty + 16][m] : Y[m][ty + 16];
    a00 = fma(x0, y0, a00); a01 = fma(x0, y1, a01);
    a10 = fma(x1, y0, a10); a11 = fma(x1, y1, a11);
  }
  if (accumulate) {
    out[tx][ty] += sign * a00; out[tx][ty + 16] += sign * a01;
    out[tx + 16][ty] += sign * a10; out[tx + 16][ty + 16] += sign * a11;
  } else {
    out[tx][ty] = sign * a00; out[tx][ty + 16] = sign * a01;
    out[tx + 16][ty] = sign * a10; out[tx + 16][ty + 16] = sign * a11;
  }
}

struct Task {
  int type, i, j, k;
};

// Number of tasks of step k (see potrf_dag_batch for the list order).
__host__ __device__ inline int step_tasks(int p, int k) {
  const int nS = p - 2 - k > 0 ? p - 2 - k : 0;
  const int nC = k + 1 < p ? 1 : 0;
  const int nU = (p - 1 - k) * (p - k) / 2 - nC;
  const int nV = (p - 1 - k) * (k + 1);
  return nS + nC + k + nU + nV;
}

// Decode task index l of one instance.  Index 0 is F(0); then for each step
// k: S(i,k) for i >= k+2, the fused chain task C(k+1) = S(k+1,k) +
// U(k+1,k+1,k) + F(k+1), G(k,j), the remaining U(i,j,k) (column k+1 first),
// and V(i,j,k).
__device__ Task decode(const DagArgs& g, int l) {
  const int p = g.p;
  Task t{TK_F, 0, 0, 0};
  if (l == 0) return t;
  l -= 1;
  int lo = 0, hi = p - 1;
  while (lo < hi) {   // largest k with off[k] <= l
    const int mid = (lo + hi + 1) >> 1;
    if (g.off[mid] <= l) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  int r = l - g.off[k];
  t.k = k;
  const int nS = p - 2 - k > 0 ? p - 2 - k : 0;
  if (r < nS) { t.type = TK_S; t.i = k + 2 + r; t.j = k; return t; }
  r -= nS;
  if (k + 1 < p) {
    if (r == 0) { t.type = TK_C; t.i = k + 1; t.j = k + 1; return t; }
    r -= 1;
  }
  if (r < k) { t.type = TK_G; t.i = k; t.j = r; return t; }
  r -= k;
  const int nU = (p - 1 - k) * (p - k) / 2 - (k + 1 < p ? 1 : 0);
  if (r < nU) {   // columns j = k+1.. in order, rows i = j..p-1, skipping (k+1, k+1)
    int j = k + 1;
    int len = p - j - 1;            // column k+1 without its diagonal tile
    while (r >= len) { r -= len; ++j; len = p - j; }
    t.type = TK_U; t.j = j; t.i = (j == k + 1 ? j + 1 : j) + r; return t;
  }
  r -= nU;
  t.type = TK_V;   // rows i = k+1.. in order, columns j = 0..k
  t.i = k + 1 + r / (k + 1);
  t.j = r % (k + 1);
  return t;
}

// 1 / v by Newton-Raphson (r <- r + r (1 - v r), each step doubling the
// correct bits) from the FP32 reciprocal: two steps reach FP64 accuracy with
// 4 dependent FP64 operations, where a division costs about ten on the
// leaf's serial chain.  Values outside FP32's range use the division.
__device__ __forceinline__ double recip(double v) {
  const double av = fabs(v);
  if (!(av > 1e-30 && av < 1e30)) return 1.0 / v;
  double r = (double)__frcp_rn((float)v);
  double e = fma(-v, r, 1.0);
  r = fma(r, e, r);
  e = fma(-v, r, 1.0);
  return fma(r, e, r);
}

// Leaf on smem tile S (lower, W_kk): writes X_kk = L_kk^{-1} into Xo, returns
// log det in *ld (thread 0) and a bad-pivot flag.  (Same elimination as the
// standalone leaf kernel, with 256 threads.)
__device__ void leaf(double (*S)[T + 1], double (*X)[T + 1], double* lcol, double* rinv,
                     double* logdet, int* bad) {
  constexpr int kPos = T * (T + 1) / 2;
  constexpr int kPer = (kPos + kDagThreads - 1) / kDagThreads;
  const int tid = threadIdx.x;
  int pi[kPer], pk[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int q = tid + kDagThreads * r;
    if (q < kPos) {
      int i = 0;
      while ((i + 1) * (i + 2) / 2 <= q) ++i;
      pi[r] = i;
      pk[r] = q - i * (i + 1) / 2;
    } else {
      pi[r] = -1;
      pk[r] = 0;
    }
  }
  for (int e = tid; e < T * T; e += kDagThreads) X[e % T][e / T] = (e % T == e / T) ? 1.0 : 0.0;
  if (tid == 0) rinv[0] = recip(S[0][0]);
  __syncthreads();
  for (int j = 0; j < T; ++j) {
    if (tid > j && tid < T) lcol[tid] = S[tid][j] * rinv[j];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int i = pi[r], k = pk[r];
      if (i > j) {
        const double lij = lcol[i];
        if (k > j) {
          const double v = fma(-lij, S[k][j], S[i][k]);
          S[i][k] = v;
          if (i == j + 1 && k == j + 1) rinv[j + 1] = recip(v);
        } else {
          X[i][k] = fma(-lij, X[j][k], X[i][k]);
        }
      }
    }
    __syncthreads();
  }
  if (tid < T) rinv[tid] = 1.0 / sqrt(S[tid][tid]);
  __syncthreads();
  for (int e = tid; e < T * T; e += kDagThreads) {
    const int i = e % T, k = e / T;
    X[i][k] = i >= k ? X[i][k] * rinv[i] : 0.0;
  }
  if (tid < 32) {
    const double dj = S[tid][tid];
    const bool b = !(dj > 0.0) || !isfinite(dj);
    double l = b ? 0.0 : log(dj);
#pragma unroll
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    const unsigned anyb = __ballot_sync(0xffffffffu, b);
    if (tid == 0) {
      *logdet = l;
      *bad = anyb != 0;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kDagThreads) potrf_dag_kernel(DagArgs g) {
  __shared__ double S0[T][T + 1], S1[T][T + 1], S2[T][T + 1], S3[T][T + 1];
  __shared__ double lcol[T], rinv[T];
  __shared__ int s_task, s_ok;
  __shared__ double s_logdet;
  __shared__ int s_bad;
  const int p = g.p, ld = g.ld, pp = p * p;
  while (true) {
    if (threadIdx.x == 0) s_task = atomicAdd(g.counter, 1);
    __syncthreads();
    const int tg = s_task;
    __syncthreads();
    if (tg >= g.total) return;
    const int z = tg % g.cnt;
    const Task t = decode(g, tg / g.cnt);
    const DagInst& I = g.inst[z];
    int* cntW = I.st;
    int* cntR = I.st + pp;
    int* doneF = I.st + 2 * pp;
    int* doneS = doneF + p;
    int* doneG = doneS + pp;
    auto Lt = [&](int i, int k) { return I.Lt + ((int64_t)i * (i - 1) / 2 + k) * T * T; };
    // ---- wait for the tiles this task reads
    if (threadIdx.x == 0) {
      bool ok = true;
      switch (t.type) {
        case TK_F: ok = wait_ge(&cntW[t.k * p + t.k], t.k, g.abort); break;
        case TK_C:   // t.i = k + 1 = c: W_{c,c-1} and W_cc up to step c-2 here;
                     // F(c-1) is awaited after these tiles are loaded
          ok = wait_ge(&cntW[t.i * p + t.i - 1], t.i - 1, g.abort) &&
               wait_ge(&cntW[t.i * p + t.i], t.i - 1, g.abort);
          break;
        case TK_S:
          ok = wait_ge(&doneF[t.k], 1, g.abort) && wait_ge(&cntW[t.i * p + t.k], t.k, g.abort);
          break;
        case TK_G:
          ok = wait_ge(&doneF[t.i], 1, g.abort) &&
               wait_ge(&cntR[t.i * p + t.j], t.i - t.j, g.abort);
          break;
        case TK_U:
          ok = wait_ge(&doneS[t.i * p + t.k], 1, g.abort) &&
               wait_ge(&doneS[t.j * p + t.k], 1, g.abort) &&
               wait_ge(&cntW[t.i * p + t.j], t.k, g.abort);
          break;
        default:   // TK_V
          ok = wait_ge(&doneS[t.i * p + t.k], 1, g.abort) &&
               (t.j == t.k ? wait_ge(&doneF[t.k], 1, g.abort)
                           : wait_ge(&doneG[t.k * p + t.j], 1, g.abort)) &&
               wait_ge(&cntR[t.i * p + t.j], t.k - t.j, g.abort);
      }
      // A bulk task starts only when no chain task holds this SM, so the chain
      // (the latency-critical path) gets the SM's whole FP64 pipe.
      if (ok && g.yield && t.type != TK_C && t.type != TK_F) {
        const int* busy = &g.smbusy[sm_id() & 255];
        if (ld_acquire(busy) > 0) {
          const unsigned long long t0 = now_ns();
          while (ld_acquire(busy) > 0) {
            __nanosleep(128);
            if (ld_acquire(g.abort)) { ok = false; break; }
            if (now_ns() - t0 > kWaitNs) { atomicExch(g.abort, 1); ok = false; break; }
          }
        }
      }
      if (ok && t.type == TK_C && g.yield) atomicAdd(&g.smbusy[sm_id() & 255], 1);
      s_ok = ok;
      if (!ok) atomicCAS(I.fail, -1, kFailTimeout);
    }
    __syncthreads();
    if (!s_ok) return;
    // ---- execute
    switch (t.type) {
      case TK_F: {
        load_tile(S0, tile(I.A, ld, t.k, t.k), ld);
        __syncthreads();
        leaf(S0, S1, lcol, rinv, &s_logdet, &s_bad);
        store_tile(tile(I.A, ld, t.k, t.k), ld, S1, true);
        if (threadIdx.x == 0) {
          I.slots[t.k] = s_logdet;
          if (s_bad) atomicCAS(I.fail, -1, I.code);
        }
        __syncthreads();
        if (threadIdx.x == 0) { __threadfence(); st_release(&doneF[t.k], 1); }
        break;
      }
      case TK_C: {   // c = t.i: L_{c,c-1}, W_cc -= L L^T, then the leaf of W_cc
        const int c = t.i;
        load_tile(S0, tile(I.A, ld, c, c - 1), ld);
        load_tile(S3, tile(I.A, ld, c, c), ld);
        if (threadIdx.x == 0) s_ok = wait_ge(&doneF[c - 1], 1, g.abort);
        __syncthreads();
        if (!s_ok) {
          if (threadIdx.x == 0) {
            atomicCAS(I.fail, -1, kFailTimeout);
            if (g.yield) atomicSub(&g.smbusy[sm_id() & 255], 1);
          }
          return;
        }
        load_tile(S1, tile(I.A, ld, c - 1, c - 1), ld);
        __syncthreads();
        for (int e = threadIdx.x; e < T * T; e += kDagThreads)
          if (e % T < e / T) S1[e % T][e / T] = 0.0;
        __syncthreads();
        tile_mm(S0, S1, true, S2, 1.0, false);            // S2 = L_{c,c-1}
        __syncthreads();
        store_tile(Lt(c, c - 1), T, S2, false);
        __syncthreads();
        if (threadIdx.x == 0) { __threadfence(); st_release(&doneS[c * p + c - 1], 1); }
        tile_mm(S2, S2, true, S3, -1.0, true);            // W_cc -= L L^T
        __syncthreads();
        leaf(S3, S1, lcol, rinv, &s_logdet, &s_bad);
        store_tile(tile(I.A, ld, c, c), ld, S1, true);
        if (threadIdx.x == 0) {
          I.slots[c] = s_logdet;
          if (s_bad) atomicCAS(I.fail, -1, I.code);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          __threadfence();
          st_release(&cntW[c * p + c], c);
          st_release(&doneF[c], 1);
          if (g.yield) atomicSub(&g.smbusy[sm_id() & 255], 1);
        }
        break;
      }
      case TK_S: {   // L_ik = W_ik X_kk^T
        load_tile(S0, tile(I.A, ld, t.i, t.k), ld);
        load_tile(S1, tile(I.A, ld, t.k, t.k), ld);
        __syncthreads();
        // X_kk is lower: zero its upper part before use
        for (int e = threadIdx.x; e < T * T; e += kDagThreads)
          if (e % T < e / T) S1[e % T][e / T] = 0.0;
        __syncthreads();
        tile_mm(S0, S1, true, S2, 1.0, false);
        __syncthreads();
        store_tile(Lt(t.i, t.k), T, S2, false);
        __syncthreads();
        if (threadIdx.x == 0) { __threadfence(); st_release(&doneS[t.i * p + t.k], 1); }
        break;
      }
      case TK_G: {   // X_kj = X_kk R_kj  (t.i = k)
        load_tile(S0, tile(I.A, ld, t.i, t.i), ld);
        load_tile(S1, tile(I.A, ld, t.i, t.j), ld);
        __syncthreads();
        // X_kk is lower: zero its upper part before use
        for (int e = threadIdx.x; e < T * T; e += kDagThreads)
          if (e % T < e / T) S0[e % T][e / T] = 0.0;
        __syncthreads();
        tile_mm(S0, S1, false, S2, 1.0, false);
        __syncthreads();
        store_tile(tile(I.A, ld, t.i, t.j), ld, S2, false);
        __syncthreads();
        if (threadIdx.x == 0) { __threadfence(); st_release(&doneG[t.i * p + t.j], 1); }
        break;
      }
      case TK_U: {   // W_ij -= L_ik L_jk^T
        load_tile(S0, Lt(t.i, t.k), T);
        load_tile(S1, Lt(t.j, t.k), T);
        load_tile(S2, tile(I.A, ld, t.i, t.j), ld);
        __syncthreads();
        tile_mm(S0, S1, true, S2, -1.0, true);
        __syncthreads();
        store_tile(tile(I.A, ld, t.i, t.j), ld, S2, t.i == t.j);
        __syncthreads();
        if (threadIdx.x == 0) { __threadfence(); st_release(&cntW[t.i * p + t.j], t.k + 1); }
        break;
      }
      default: {     // TK_V: R_ij -= L_ik X_kj
        load_tile(S0, Lt(t.i, t.k), T);
        load_tile(S1, tile(I.A, ld, t.k, t.j), ld);
        const bool first = t.k == t.j;
        if (!first) load_tile(S2, tile(I.A, ld, t.i, t.j), ld);
        __syncthreads();
        if (first)   // X_jj is lower: zero its upper part
          for (int e = threadIdx.x; e < T * T; e += kDagThreads)
            if (e % T < e / T) S1[e % T][e / T] = 0.0;
        __syncthreads();
        tile_mm(S0, S1, false, S2, -1.0, !first);
        __syncthreads();
        store_tile(tile(I.A, ld, t.i, t.j), ld, S2, false);
        __syncthreads();
        if (threadIdx.x == 0) {
          __threadfence();
          st_release(&cntR[t.i * p + t.j], t.k - t.j + 1);
        }
      }
    }
    __syncthreads();
  }
}

// Resident CTAs per SM of the persistent grid: more CTAs keep SMs busy while
// some wait on dependencies, fewer give the critical-path tiles a larger share
// of each SM's FP64 pipe.  BTA_DAG_CTAS_PER_SM overrides the default.
int dag_ctas_per_sm() {
  static int v = [] {
    const char* e = getenv("BTA_DAG_CTAS_PER_SM");
    int x = e ? atoi(e) : 2;
    return x < 1 ? 1 : (x > 8 ? 8 : x);
  }();
  return v;
}

// Whether bulk tasks yield the SM to chain tasks (BTA_DAG_YIELD=0 disables).
int dag_yield() {
  static int v = [] {
    const char* e = getenv("BTA_DAG_YIELD");
    return e ? (atoi(e) != 0) : 1;
  }();
  return v;
}

}  // namespace

int potrf_dag_tasks(int p) {
  int tot = 1;
  for (int k = 0; k < p; ++k) tot += step_tasks(p, k);
  return tot;
}

size_t potrf_dag_state_ints(int p) { return (size_t)4 * p * p + p + 64 + 256; }

// scratch[z] holds the packed L tiles (p(p-1)/2 tiles) followed by the
// counters; n*n doubles are enough.
bta_status potrf_dag_batch(int count, double* const* A, int n, int ld, double* const* scratch,
                           double* const* logdet_parts, int32_t* const* fail,
                           const int32_t* fail_code, cudaStream_t s) {
  const int p = n / T;
  if (n <= 0 || n % T || p > kMaxP || count < 1) return BTA_ERR_ARG;
  const size_t lt_doubles = (size_t)p * (p - 1) / 2 * T * T;
  for (int z0 = 0; z0 < count; z0 += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, count - z0);
    DagArgs g;
    g.p = p; g.ld = ld; g.cnt = cnt;
    int acc = 0;
    for (int k = 0; k < p; ++k) {
      g.off[k] = acc;
      acc += step_tasks(p, k);
    }
    g.off[p] = acc;
    g.total = (acc + 1) * cnt;
    for (int z = 0; z < cnt; ++z) {
      DagInst& I = g.inst[z];
      I.A = A[z0 + z];
      I.Lt = scratch[z0 + z];
      I.st = reinterpret_cast<int*>(scratch[z0 + z] + lt_doubles);
      I.slots = logdet_parts[z0 + z];
      I.fail = fail[z0 + z];
      I.code = fail_code[z0 + z];
      BTA_CUDA_TRY(cudaMemsetAsync(I.st, 0, potrf_dag_state_ints(p) * sizeof(int), s));
    }
    // ticket counter and abort flag live after instance 0's counters
    g.counter = g.inst[0].st + 4 * p * p + p + 8;
    g.abort = g.counter + 16;
    g.smbusy = g.inst[0].st + 4 * p * p + p + 64;
    g.yield = cnt <= 2 ? dag_yield() : 0;
    const int grid = std::min(g.total, 152 * dag_ctas_per_sm());
    launch_prio(potrf_dag_kernel, dim3(grid), dim3(kDagThreads), s, g);
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

}  // namespace bta
