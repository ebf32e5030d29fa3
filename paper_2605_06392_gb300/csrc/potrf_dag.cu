// Diagonal-block Cholesky factor and inverse as one persistent kernel over a
// tile task graph (FP64 results, 32 x 32 tiles, p = n / 32 tile rows).  Its
// tile products run as FP64 FMAs, or (the tensor-core modes, kernel
// instance TC) emulated in FP64 from BF16 slices on warp-level tensor-core
// MMAs (tile_mm_oz); pivots, reciprocals and log-dets stay in FP64.
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
//   H         the chain, one task per block run by one CTA: for c = 0..p-1,
//             L_{c,c-1} = W_{c,c-1} X_{c-1,c-1}^T, W_cc -= L L^T, and the leaf
//             on W_cc (D / unit-L elimination with its inverse) -> X_cc =
//             L_cc^{-1} into A_cc, log-det slot c; X_cc stays in shared
//             memory for the next step
//   S(i,k)    L_ik = W_ik X_kk^T, i >= k+2           (into the scratch Lt)
//   G(k,j)    X_kj = X_kk R_kj            (j < k; R_kj = -sum_m L_km X_mj)
//   U(i,j,k)  W_ij -= L_ik L_jk^T         (k < j <= i, not (k+1,k+1); column k+1 first)
//   V(i,j,k)  R_ij -= L_ik X_kj           (k < i, j <= k; R_ij = -L_ij X_jj at k = j)
// A task waits only for tasks earlier in the list, which running CTAs hold,
// so the graph always drains.  Per-tile counters (W updates applied, R
// updates applied, F/S/G done) are published with release stores after the
// tile is written and read with acquire loads; tile data are read through
// L2 (ld.global.cg).  Every wait is bounded by a globaltimer limit (2 s); on
// expiry the CTA raises a shared abort flag, writes BTA_ERR_TIMEOUT into the
// block's failure word (which otherwise holds -1 or the index of a block with
// a non-positive pivot) and returns, and every other CTA returns at its next
// wait.  A test switch (bta_set_wait_limit) lowers the limit and makes the
// chain wait on a counter nothing sets, so that this path runs without a fault.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "ozaki_digits.cuh"

// Timeline hooks of the chain (compile-time empty in the library): a
// measurement build that includes this file may define DAG_TRACE(event, step)
// before the include to stamp the chain's phases of each diagonal step:
// 0 the step's inputs are final (waits done), 1 the triangular product done,
// 2 the symmetric update done, 3 the leaf done, 4 the step published.
#ifndef DAG_TRACE
#define DAG_TRACE(event, step) ((void)0)
#endif

namespace bta {
namespace {

constexpr int T = kPad;                 // tile size
constexpr int kDagThreads = 256;
constexpr int kMaxP = 160;              // tile rows supported (ld <= 5120)

enum : int { TK_H = 0, TK_S = 1, TK_G = 2, TK_U = 3, TK_V = 4 };

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
  int* smbusy;              // per SM: chain tasks running there (see TK_H)
  int yield;                // bulk tasks wait while a chain task holds their SM
  int stall;                // test switch: the chain waits on a counter nothing sets
  unsigned long long wait_ns;   // bound of every wait
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

// Thread 0 waits until *p >= need (bounded by wait_ns); false on timeout / abort.
__device__ bool wait_ge(const int* p, int need, int* abort, unsigned long long wait_ns) {
  if (ld_acquire(p) >= need) return true;
  const unsigned long long t0 = now_ns();
  while (true) {
    __nanosleep(64);
    if (ld_acquire(p) >= need) return true;
    if (ld_acquire(abort)) return false;
    if (now_ns() - t0 > wait_ns) {
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

// out[r][c] = sum_{m <= c} W[r][m] Y[c][m] = (W Y^T)[r][c] for lower-triangular Y
// (its upper part is not read).  Same thread layout as tile_mm; the m range
// of a thread's columns (ty, ty + 16) is uniform within a warp, so the
// skipped half of the products issues no instructions.
__device__ __forceinline__ void tile_mm_lt(double (*W)[T + 1], double (*Y)[T + 1],
                                           double (*out)[T + 1]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
  for (int m = 0; m <= ty; ++m) {
    const double x0 = W[tx][m], x1 = W[tx + 16][m];
    const double y0 = Y[ty][m], y1 = Y[ty + 16][m];
    a00 = fma(x0, y0, a00); a01 = fma(x0, y1, a01);
    a10 = fma(x1, y0, a10); a11 = fma(x1, y1, a11);
  }
  for (int m = ty + 1; m <= ty + 16; ++m) {
    const double y1 = Y[ty + 16][m];
    a01 = fma(W[tx][m], y1, a01);
    a11 = fma(W[tx + 16][m], y1, a11);
  }
  out[tx][ty] = a00; out[tx][ty + 16] = a01;
  out[tx + 16][ty] = a10; out[tx + 16][ty + 16] = a11;
}

// W[r][c] -= sum_m L[r][m] L[c][m] on the lower triangle (r >= c): threads
// 0..135 each own one 2 x 2 block of the 16 x 16 block triangle, so only 5
// of the 8 warps issue FMAs.  Upper entries of diagonal blocks get the same
// update (W is symmetric; only its lower part is read afterwards).
__device__ __forceinline__ void tile_syrk_lower(double (*L)[T + 1], double (*W)[T + 1]) {
  const int b = threadIdx.x;
  if (b >= 136) return;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= b) ++bi;
  const int bj = b - bi * (bi + 1) / 2;
  const int r = 2 * bi, c = 2 * bj;
  double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
#pragma unroll 8
  for (int m = 0; m < T; ++m) {
    const double x0 = L[r][m], x1 = L[r + 1][m], y0 = L[c][m], y1 = L[c + 1][m];
    a00 = fma(x0, y0, a00); a01 = fma(x0, y1, a01);
    a10 = fma(x1, y0, a10); a11 = fma(x1, y1, a11);
  }
  W[r][c] -= a00; W[r][c + 1] -= a01;
  W[r + 1][c] -= a10; W[r + 1][c + 1] -= a11;
}

// ---- emulated-FP64 tile products (tensor-core modes) -----------------------
// out (+)= sign * X op(Y) on 32 x 32 tiles, op(Y) = Y^T (ytrans) or Y, to FP64
// accuracy from 8 BF16 digit slices per operand on warp-level tensor-core
// MMAs (mma.sync m16n8k16): on GB300 these run ~1900 BF16 flop per clock per
// SM against ~1.6 FP64 FMAs, so the 36 slice-pair products of a tile cost
// ~1.2 k clocks where its 32^3 FP64 FMAs cost ~20 k.  The digits are those
// of the emulated GEMM (fixed point on each row's exponent bound, 7 bits a
// digit); a level L = i + j of slice pairs sums to |S_L| < 2^21 digit units
// over K = 32, exact in FP32; levels 0..5 are added as 64-bit integers in
// units of 2^-35 of level 0, levels 6 and 7 rounded to that unit, and the
// FP64 result assembled by integer operations.  Levels from 8 on are dropped,
// the bound of the emulated GEMM with K = 32.  ylower: Y is lower triangular
// (its upper part is not read).
constexpr int kOzPitch = 40;                      // bf16 a slice row: 80 bytes, conflict-free ldmatrix
constexpr int kOzPlane = T * kOzPitch;            // one 32 x 32 slice
constexpr int kOzTileSmem = 2 * 8 * kOzPlane * 2 + 2 * T * 4;   // both operands' slices, exponents

struct OzTile {
  __nv_bfloat16* xp;   // [8][32][kOzPitch]: slices of the rows of X
  __nv_bfloat16* yp;   // [8][32][kOzPitch]: slices of the rows of op(Y)^T
  int* ex;             // [32] row exponents of X
  int* ey;             // [32] row exponents of op(Y)^T
};

// Slices of a 32 x 32 matrix (element (r, k) = get(r, k)) into planes[8][r][k]
// and its row exponent bounds e[r]: warp w takes rows w, w + 8, w + 16, w + 24.
template <class Get>
__device__ __forceinline__ void oz_split(Get get, __nv_bfloat16* planes, int* e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double v[4];
  int er[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = get(warp + 8 * q, lane);
    const int ef = (int)((__double_as_longlong(v[q]) >> 52) & 0x7FF);
    er[q] = (int)__reduce_max_sync(0xffffffffu, (unsigned)ef);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = warp + 8 * q;
    float d[8];
    oz::digits<8>(v[q], er[q], d);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      planes[j * kOzPlane + r * kOzPitch + lane] = __float2bfloat16_rn(d[j]);
    if (lane == 0) e[r] = er[q];
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t (&r)[2]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// All 256 threads; out must not alias X or Y.  Warp w computes the 16 x 8
// output block (rows 16 (w / 4).., columns 8 (w % 4)..).
__device__ void tile_mm_oz(double (*X)[T + 1], double (*Y)[T + 1], bool ytrans, bool ylower,
                           double (*out)[T + 1], double sign, bool accumulate,
                           const OzTile& z) {
  const bool same = X == Y && ytrans && !ylower;   // X op(Y) = X X^T: one split
  oz_split([&](int r, int k) { return X[r][k]; }, z.xp, z.ex);
  if (!same)
    oz_split(
        [&](int n, int k) {
          const double v = ytrans ? Y[n][k] : Y[k][n];
          return ylower && (ytrans ? k > n : n > k) ? 0.0 : v;
        },
        z.yp, z.ey);
  __syncthreads();
  const __nv_bfloat16* yp = same ? z.xp : z.yp;
  const int* ey = same ? z.ex : z.ey;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mt = warp >> 2, nt = warp & 3;
  uint32_t a[8][2][4], b[8][2][2];
  {
    const uint32_t xb = (uint32_t)__cvta_generic_to_shared(z.xp);
    const uint32_t yb = (uint32_t)__cvta_generic_to_shared(yp);
    // ldmatrix rows: A's four 8 x 8 blocks (rows 0-7 / 8-15 by k 0-7 / 8-15),
    // B's two (columns 0-7 by k 0-7 / 8-15), from lanes 0-31 / 0-15
    const int ar = 16 * mt + (lane & 7) + ((lane >> 3) & 1) * 8, ac = (lane >> 4) * 8;
    const int br = 8 * nt + (lane & 7), bc = ((lane >> 3) & 1) * 8;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        ldsm_x4(xb + 2u * (uint32_t)(j * kOzPlane + ar * kOzPitch + 16 * ks + ac), a[j][ks]);
        ldsm_x2(yb + 2u * (uint32_t)(j * kOzPlane + br * kOzPitch + 16 * ks + bc), b[j][ks]);
      }
  }
  // one accumulator per level, the pairs issued slice by slice of A so that
  // consecutive MMAs go to different accumulators (no dependent chain)
  float c[8][4];
#pragma unroll
  for (int L = 0; L < 8; ++L)
#pragma unroll
    for (int q = 0; q < 4; ++q) c[L][q] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; i + j < 8; ++j) mma_bf16(c[i + j], a[i][ks], b[j][ks]);
  // S_L = c[L] 2^(7 L), |S_L| < 2^21: to integers by the exact FP32 rounding
  // against 1.5 2^23 (no 64-bit conversions, which GB300 runs at its FP64
  // rate); two levels 7 bits apart share one 32-bit integer, then
  // tot = S_0 2^35 + S_1 2^28 + ... + S_5 + round(S_6 2^-7 + S_7 2^-14).
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int sl[6];
#pragma unroll
    for (int L = 0; L < 6; ++L) sl[L] = oz::f2i_small(c[L][q] * __int_as_float((127 + 7 * L) << 23));
    const int r67 = oz::f2i_small((c[6][q] + c[7][q]) * 34359738368.0f);
    const long long tot = ((long long)(sl[0] * 128 + sl[1]) << 28) +
                          ((long long)(sl[2] * 128 + sl[3]) << 14) + (sl[4] * 128 + sl[5]) + r67;
    const int r = 16 * mt + g + (q >> 1) * 8, c = 8 * nt + 2 * t + (q & 1);
    const double v = oz::compose(tot, z.ex[r] + ey[c] - 2093);
    out[r][c] = accumulate ? fma(sign, v, out[r][c]) : sign * v;
  }
}

struct Task {
  int type, i, j, k;
};

// Number of tasks of step k (see potrf_dag_batch for the list order).
__host__ __device__ inline int step_tasks(int p, int k) {
  const int nS = p - 2 - k > 0 ? p - 2 - k : 0;
  const int nU = (p - 1 - k) * (p - k) / 2 - (k + 1 < p ? 1 : 0);
  const int nV = (p - 1 - k) * (k + 1);
  return nS + k + nU + nV;
}

// Decode task index l of one instance.  Index 0 is the chain H; then for
// each step k: S(i,k) for i >= k+2, G(k,j), U(i,j,k) (column k+1 first,
// without (k+1,k+1), which the chain applies) and V(i,j,k).
__device__ Task decode(const DagArgs& g, int l) {
  const int p = g.p;
  Task t{TK_H, 0, 0, 0};
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

// 1 / v to FP64 accuracy.  Seed: the FP32 reciprocal of v's leading bits,
// with v narrowed and the result widened by integer operations (a GB300 FP64
// instruction, conversions included, has ~64 clock cycles of latency).  With
// r = (1 + eps) / v, e = 1 - v r = -eps, the correction r (1 + e + e^2) has
// relative error eps^3 (~2^-66) plus rounding: three dependent FP64 FMAs.
// Values outside the seed's exponent range use the division.
__device__ __forceinline__ double recip(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 1023 - 100 || e > 1023 + 100) return 1.0 / v;
  const unsigned f = (unsigned)((b >> 32) & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) |
                     (unsigned)((b >> 29) & 0x7FFFFFu);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(f)));
  const unsigned rb = __float_as_uint(rf);
  const unsigned long long db = ((unsigned long long)(rb & 0x80000000u) << 32) |
                                ((unsigned long long)(((rb >> 23) & 0xFF) - 127 + 1023) << 52) |
                                ((unsigned long long)(rb & 0x7FFFFFu) << 29);
  const double r = __longlong_as_double((long long)db);
  const double err = fma(-v, r, 1.0);
  return fma(r, fma(err, err, err), r);
}

// d^{-1/2} to FP64 accuracy: FP32 seed of the narrowed value widened by
// integer operations, then y (1 + e/2 + 3e^2/8) with e = 1 - d y^2 (relative
// error ~e^3): five dependent FP64 operations.  Outside the seed's range the
// library square root and division.
__device__ __forceinline__ double rsqrt_fp64(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (!(d > 0.0) || e < 1023 - 100 || e > 1023 + 100) return 1.0 / sqrt(d);
  const unsigned f = ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(__uint_as_float(f)));
  const unsigned rb = __float_as_uint(yf);
  const unsigned long long db = ((unsigned long long)(((rb >> 23) & 0xFF) - 127 + 1023) << 52) |
                                ((unsigned long long)(rb & 0x7FFFFFu) << 29);
  const double y = __longlong_as_double((long long)db);
  const double err = fma(-d, y * y, 1.0);
  return fma(y, fma(0.375, err, 0.5) * err, y);
}

// Leaf on smem tile S (lower, W_kk): D / unit-L elimination carrying the
// inverse of the unit-L factor in X, then X = D^{-1/2} (unit L)^{-1} =
// L_kk^{-1}; the pivots d_i stay in piv[] (leaf_logdet sums their logs, off
// the critical path).
//
// Pivot j eliminates column j with the multipliers l_ij = S_ij / d_j:
// S_ik -= l_ij S_kj (j < k <= i) and X_ik -= l_ij X_jk (k <= j < i).  Warp 0
// runs one pivot ahead: while warps 1-3 and 5-7 apply pivot j to columns
// k >= j+2 and to X, it applies pivot j to column j+1, takes d_{j+1}, its
// reciprocal and the next multipliers, so each pivot costs one barrier and
// the serial chain per pivot is one FMA, the reciprocal and one multiply.
// Warp 4 shares warp 0's scheduler and FP64 unit and stays idle, so the
// chain's instructions do not queue behind bulk ones.
__device__ void leaf(double (*S)[T + 1], double (*X)[T + 1], double (*lcol)[T], double* piv,
                     double* rs) {
  constexpr int kPos = T * (T + 1) / 2;   // lower-triangle positions, row by row
  constexpr int kBulk = kDagThreads - 64;   // warps 1-3 and 5-7
  constexpr int kPer = (kPos + kBulk - 1) / kBulk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool bulk = warp != 0 && warp != 4;
  const int bt = warp < 4 ? tid - 32 : tid - 64;   // 0..kBulk-1 over the bulk warps
  int pi[kPer], pk[kPer];
  if (bulk) {
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int q = bt + kBulk * r;
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
  }
  for (int e = tid; e < T * T; e += kDagThreads) X[e % T][e / T] = (e % T == e / T) ? 1.0 : 0.0;
  if (tid < 32) {   // pivot 0 and its multipliers
    const double d = S[0][0];
    const double r = recip(d);
    if (lane > 0) lcol[0][lane] = S[lane][0] * r;
    if (lane == 0) piv[0] = d;
  }
  __syncthreads();
  for (int j = 0; j < T - 1; ++j) {
    const double* lj = lcol[j & 1];
    if (tid < 32) {
      // column j+1 with pivot j, then pivot j+1 and its multipliers
      const int c = j + 1;
      double v = 0.0;
      if (lane >= c) {
        v = fma(-lj[lane], S[c][j], S[lane][c]);
        S[lane][c] = v;
      }
      const double d = __shfl_sync(0xffffffffu, v, c);
      const double r = recip(d);
      if (lane > c) lcol[c & 1][lane] = v * r;
      if (lane == 0) piv[c] = d;
    } else if (bulk) {
      // k > j+1: trailing S_ik -= l_ij S_kj; k <= j: X_ik -= l_ij X_jk.  The
      // positions are distinct and none is a source of this pivot (column j of
      // S, row j of X), so all loads go first and the FMAs overlap.
      double* dst[kPer];
      double dv[kPer], sv[kPer], lv[kPer];
      bool act[kPer];
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int i = pi[q], k = pk[q];
        act[q] = i > j && k != j + 1;
        if (act[q]) {
          dst[q] = k > j ? &S[i][k] : &X[i][k];
          sv[q] = k > j ? S[k][j] : X[j][k];
          dv[q] = *dst[q];
          lv[q] = lj[i];
        }
      }
#pragma unroll
      for (int q = 0; q < kPer; ++q)
        if (act[q]) *dst[q] = fma(-lv[q], sv[q], dv[q]);
    }
    __syncthreads();
  }
  if (tid < 32) rs[tid] = rsqrt_fp64(piv[tid]);   // rows scale by d_i^{-1/2}
  __syncthreads();
  for (int e = tid; e < T * T; e += kDagThreads) {
    const int i = e % T, k = e / T;
    X[i][k] = i >= k ? X[i][k] * rs[i] : 0.0;
  }
  __syncthreads();
}

// Log-det slot of a leaf: sum of log d_i over its pivots, and the failure
// code on a non-positive or non-finite pivot (warp 0).
__device__ __forceinline__ void leaf_logdet(const double* piv, double* slot, int32_t* fail,
                                            int32_t code) {
  if (threadIdx.x < 32) {
    const double dj = piv[threadIdx.x];
    const bool b = !(dj > 0.0) || !isfinite(dj);
    double l = b ? 0.0 : log(dj);
#pragma unroll
    for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    const unsigned anyb = __ballot_sync(0xffffffffu, b);
    if (threadIdx.x == 0) {
      *slot = l;
      if (anyb) atomicCAS(fail, -1, code);
    }
  }
}

// TC: the tile products emulated in FP64 on the tensor cores (tile_mm_oz,
// the tensor-core modes); otherwise FP64 FMAs.
template <bool TC>
__global__ void __launch_bounds__(kDagThreads) potrf_dag_kernel(DagArgs g) {
  // three tiles (~26 KB with the leaf's vectors); TC adds the slices of two
  // tiles (40 KB of dynamic shared memory)
  __shared__ double S0[T][T + 1], S1[T][T + 1], S2[T][T + 1];
  extern __shared__ __align__(16) unsigned char dsm[];
  OzTile ozs;
  ozs.xp = reinterpret_cast<__nv_bfloat16*>(dsm);
  ozs.yp = ozs.xp + 8 * kOzPlane;
  ozs.ex = reinterpret_cast<int*>(ozs.yp + 8 * kOzPlane);
  ozs.ey = ozs.ex + T;
  // out (+)= sign X op(Y), and the product with a lower-triangular Y^T
  auto mm = [&](double (*X)[T + 1], double (*Y)[T + 1], bool ytrans, double (*o)[T + 1],
                double sign, bool acc) {
    if constexpr (TC) tile_mm_oz(X, Y, ytrans, false, o, sign, acc, ozs);
    else tile_mm(X, Y, ytrans, o, sign, acc);
  };
  auto mm_lt = [&](double (*W)[T + 1], double (*Y)[T + 1], double (*o)[T + 1]) {
    if constexpr (TC) tile_mm_oz(W, Y, true, true, o, 1.0, false, ozs);
    else tile_mm_lt(W, Y, o);
  };
  __shared__ double lcol[2][T], piv[T], rs[T];
  __shared__ int s_task, s_ok;
  const int p = g.p, ld = g.ld, pp = p * p;
  int* busy = &g.smbusy[sm_id() & 255];
  while (true) {
    if (threadIdx.x == 0) {
      // On an SM that runs a chain, take no task while the chain is there: it
      // gets the SM's whole FP64 pipe.  Waiting before taking a ticket holds
      // nothing another task needs.
      if (g.yield && ld_acquire(busy) > 0) {
        const unsigned long long t0 = now_ns();
        while (ld_acquire(busy) > 0 && ld_acquire(g.counter) < g.total && !ld_acquire(g.abort)) {
          __nanosleep(256);
          if (now_ns() - t0 > g.wait_ns) {
            atomicExch(g.abort, 1);
            break;
          }
        }
      }
      s_task = atomicAdd(g.counter, 1);
    }
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
    if (t.type == TK_H) {
      // ---- the chain: every diagonal step of this block on this CTA
      if (threadIdx.x == 0 && g.yield) atomicAdd(busy, 1);
      for (int c = 0; c < p; ++c) {
        if (c > 0 || g.stall) {
          // W_{c,c-1} and W_cc updated through step c-2 by the U tasks (the
          // test switch instead waits for a count no task reaches)
          if (threadIdx.x == 0)
            s_ok = g.stall ? wait_ge(&cntW[c * p + c], 0x7fffffff, g.abort, g.wait_ns)
                           : wait_ge(&cntW[c * p + c - 1], c - 1, g.abort, g.wait_ns) &&
                             wait_ge(&cntW[c * p + c], c - 1, g.abort, g.wait_ns);
          __syncthreads();
          if (!s_ok) {
            if (threadIdx.x == 0) {
              atomicExch(I.fail, (int32_t)BTA_ERR_TIMEOUT);
              if (g.yield) atomicSub(busy, 1);
            }
            return;
          }
        }
        if (threadIdx.x == 0 && z == 0) DAG_TRACE(0, c);
        if (c > 0) {
          load_tile(S0, tile(I.A, ld, c, c - 1), ld);
          // W_cc into registers now, into S0 once the product has read it
          double wcc[T * T / kDagThreads];
          {
            const double* src = tile(I.A, ld, c, c);
#pragma unroll
            for (int q = 0; q < T * T / kDagThreads; ++q) {
              const int e = threadIdx.x + kDagThreads * q;
              wcc[q] = __ldcg(src + (int64_t)(e / T) * ld + e % T);
            }
          }
          __syncthreads();
          mm_lt(S0, S1, S2);                      // L_{c,c-1} = W X_{c-1,c-1}^T (S1)
          __syncthreads();
          if (threadIdx.x == 0 && z == 0) DAG_TRACE(1, c);
#pragma unroll
          for (int q = 0; q < T * T / kDagThreads; ++q) {
            const int e = threadIdx.x + kDagThreads * q;
            S0[e % T][e / T] = wcc[q];
          }
          store_tile(Lt(c, c - 1), T, S2, false);
          __syncthreads();
          if (threadIdx.x == 0) { __threadfence(); st_release(&doneS[c * p + c - 1], 1); }
          if constexpr (TC) tile_mm_oz(S2, S2, true, false, S0, -1.0, true, ozs);   // W_cc -= L L^T
          else tile_syrk_lower(S2, S0);           // W_cc -= L L^T (lower)
          __syncthreads();
          if (threadIdx.x == 0 && z == 0) DAG_TRACE(2, c);
        } else {
          load_tile(S0, tile(I.A, ld, 0, 0), ld);
          __syncthreads();
        }
        leaf(S0, S1, lcol, piv, rs);              // S1 = X_cc = L_cc^{-1}
        if (threadIdx.x == 0 && z == 0) DAG_TRACE(3, c);
        store_tile(tile(I.A, ld, c, c), ld, S1, true);
        __syncthreads();
        if (threadIdx.x == 0) {
          __threadfence();
          st_release(&cntW[c * p + c], c);
          st_release(&doneF[c], 1);
          if (z == 0) DAG_TRACE(4, c);
        }
        leaf_logdet(piv, &I.slots[c], I.fail, I.code);   // after the release: off the chain
        __syncthreads();
      }
      if (threadIdx.x == 0 && g.yield) atomicSub(busy, 1);
      continue;
    }
    // ---- bulk task: wait for the tiles it reads
    if (threadIdx.x == 0) {
      bool ok = true;
      switch (t.type) {
        case TK_S:
          ok = wait_ge(&doneF[t.k], 1, g.abort, g.wait_ns) &&
               wait_ge(&cntW[t.i * p + t.k], t.k, g.abort, g.wait_ns);
          break;
        case TK_G:
          ok = wait_ge(&doneF[t.i], 1, g.abort, g.wait_ns) &&
               wait_ge(&cntR[t.i * p + t.j], t.i - t.j, g.abort, g.wait_ns);
          break;
        case TK_U:
          ok = wait_ge(&doneS[t.i * p + t.k], 1, g.abort, g.wait_ns) &&
               wait_ge(&doneS[t.j * p + t.k], 1, g.abort, g.wait_ns) &&
               wait_ge(&cntW[t.i * p + t.j], t.k, g.abort, g.wait_ns);
          break;
        default:   // TK_V
          ok = wait_ge(&doneS[t.i * p + t.k], 1, g.abort, g.wait_ns) &&
               (t.j == t.k ? wait_ge(&doneF[t.k], 1, g.abort, g.wait_ns)
                           : wait_ge(&doneG[t.k * p + t.j], 1, g.abort, g.wait_ns)) &&
               wait_ge(&cntR[t.i * p + t.j], t.k - t.j, g.abort, g.wait_ns);
      }
      s_ok = ok;
      if (!ok) atomicExch(I.fail, (int32_t)BTA_ERR_TIMEOUT);
    }
    __syncthreads();
    if (!s_ok) return;
    // ---- execute
    switch (t.type) {
      case TK_S: {   // L_ik = W_ik X_kk^T
        load_tile(S0, tile(I.A, ld, t.i, t.k), ld);
        load_tile(S1, tile(I.A, ld, t.k, t.k), ld);
        __syncthreads();
        mm_lt(S0, S1, S2);                        // X_kk lower: its upper part is not read
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
        mm(S0, S1, false, S2, 1.0, false);
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
        mm(S0, S1, true, S2, -1.0, true);
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
        mm(S0, S1, false, S2, -1.0, !first);
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

// Resident CTAs per SM of the persistent grid.  The kernel is bound by its
// chain, and one CTA per SM (as fast as two, measured) leaves room on every
// SM for a tensor-core GEMM CTA of the other sweep.  BTA_DAG_CTAS_PER_SM
// overrides the default.
int dag_ctas_per_sm() {
  static int v = [] {
    const char* e = getenv("BTA_DAG_CTAS_PER_SM");
    int x = e ? atoi(e) : 1;
    return x < 1 ? 1 : (x > 8 ? 8 : x);
  }();
  return v;
}

// Most CTAs of the persistent grid (BTA_DAG_MAX_CTAS, overriding the caller's
// cap; 0: the caller's cap, or one per SM).  A leaf's critical path is its
// chain on one CTA; CTAs beyond what keeps its bulk tasks off that path only
// hold SMs that a concurrent sweep's products could use.
int dag_max_ctas() {
  static int v = [] {
    const char* e = getenv("BTA_DAG_MAX_CTAS");
    return e ? atoi(e) : 0;
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

__global__ void pivot_reciprocals_kernel(const double* __restrict__ v, int64_t n,
                                         double* __restrict__ r, double* __restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    if (r) r[i] = recip(v[i]);
    if (q) q[i] = rsqrt_fp64(v[i]);
  }
}

}  // namespace

unsigned long long g_dag_wait_ns = 2000000000ull;
int g_dag_stall = 0;

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
                           const int32_t* fail_code, cudaStream_t s, int max_ctas, int tc) {
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
    g.stall = g_dag_stall;
    g.wait_ns = g_dag_wait_ns;
    int grid = std::min(g.total, sm_count() * dag_ctas_per_sm());
    const int cap = dag_max_ctas() > 0 ? dag_max_ctas() : max_ctas;
    if (cap > 0) grid = std::min(grid, std::max(2, cap));   // the chain and a bulk CTA
    if (tc) {
      static bool attr = false;   // the slices take the dynamic shared memory above 48 KB
      if (!attr) {
        BTA_CUDA_TRY(cudaFuncSetAttribute(potrf_dag_kernel<true>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kOzTileSmem));
        attr = true;
      }
      launch_prio_smem(potrf_dag_kernel<true>, dim3(grid), dim3(kDagThreads), kOzTileSmem, s, g);
    } else {
      launch_prio(potrf_dag_kernel<false>, dim3(grid), dim3(kDagThreads), s, g);
    }
    BTA_LAUNCHED();
  }
  return BTA_OK;
}

}  // namespace bta

extern "C" bta_status bta_pivot_reciprocals(const double* v, int64_t n, double* recip_out,
                                            double* rsqrt_out, cudaStream_t stream) {
  if (n < 0 || (n > 0 && !v) || (!recip_out && !rsqrt_out)) return BTA_ERR_ARG;
  if (n == 0) return BTA_OK;
  const int64_t blocks = (n + 255) / 256;
  if (blocks > 0x7fffffff) return BTA_ERR_ARG;
  bta::pivot_reciprocals_kernel<<<(unsigned)blocks, 256, 0, stream>>>(v, n, recip_out, rsqrt_out);
  BTA_LAUNCHED();
  return BTA_OK;
}
