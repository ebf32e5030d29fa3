// Measurement build: chain timeline of the task-graph factor.  Includes the
// library's source with DAG_TRACE stamping %globaltimer at each phase of each
// diagonal step (instance 0, thread 0), factors one SPD block of n rows with
// potrf_dag_batch and prints one JSON line: the factor's time (best of four
// runs after two warm-ups) and the chain's average step, phase by phase.
// Built and run by `python -m paper_2605_06392_gb300.trace chain`.
#include <cstdio>
#include <cstdlib>
#include <vector>
#include <cuda_runtime.h>
__device__ unsigned long long g_dt[5][256];
__device__ __forceinline__ void dag_trace_rec(int ev, int c) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  if (c >= 0 && c < 256) g_dt[ev][c] = t;
}
#define DAG_TRACE(e, c) dag_trace_rec((e), (c))
#include "../csrc/potrf_dag.cu"

__global__ void fill_spd(double* A, int n, unsigned seed) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  const int r = (int)(i % n), c = (int)(i / n);
  const int lo = r < c ? r : c, hi = r < c ? c : r;
  unsigned x = (unsigned)(lo * 2654435761u) ^ (unsigned)(hi * 40503u) ^ seed;
  x ^= x >> 13; x *= 0x5bd1e995u; x ^= x >> 15;
  A[i] = r == c ? (double)n : ((double)(x & 0xFFFF) / 65536.0 - 0.5);
}

int main(int argc, char** argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 608;   // a multiple of 32, 64 .. 5120
  const int tc = argc > 2 ? atoi(argv[2]) : 1;
  const int cap = argc > 3 ? atoi(argv[3]) : 65;
  const int p = n / 32;
  if (n % 32 || p < 2 || p > 160) { printf("n must be a multiple of 32 in 64..5120\n"); return 2; }
  double *A, *W, *sl; int32_t* fl;
  cudaMalloc(&A, (size_t)n * n * 8); cudaMalloc(&W, (size_t)n * n * 8 + 4096 * 8);
  cudaMalloc(&sl, 4096 * 8); cudaMalloc(&fl, 4);
  int32_t code = 0;
  cudaStream_t s; cudaStreamCreate(&s);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  void* dt = nullptr; cudaGetSymbolAddress(&dt, g_dt);
  float best = 1e30f;
  std::vector<unsigned long long> h(5 * 256);
  for (int it = 0; it < 6; ++it) {
    fill_spd<<<(unsigned)(((int64_t)n * n + 255) / 256), 256, 0, s>>>(A, n, 7);
    cudaMemsetAsync(fl, 0xff, 4, s);
    cudaMemsetAsync(dt, 0, sizeof(unsigned long long) * 5 * 256, s);
    cudaEventRecord(e0, s);
    bta_status st = bta::potrf_dag_batch(1, &A, n, n, &W, &sl, &fl, &code, s, cap, tc);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st != BTA_OK || e != cudaSuccess) { printf("fail %d %s\n", (int)st, cudaGetErrorString(e)); return 1; }
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    if (it >= 2 && ms < best) {
      best = ms;
      cudaMemcpy(h.data(), dt, h.size() * 8, cudaMemcpyDeviceToHost);
    }
  }
  int f = 0; cudaMemcpy(&f, fl, 4, cudaMemcpyDeviceToHost);
  auto T = [&](int ev, int c) { return (double)h[ev * 256 + c]; };
  double sw = 0, sp1 = 0, sp2 = 0, sl2 = 0, spub = 0; int ns = 0;
  for (int c = 1; c < p; ++c) {
    sw += T(0, c) - T(4, c - 1);
    sp1 += T(1, c) - T(0, c);
    sp2 += T(2, c) - T(1, c);
    sl2 += T(3, c) - T(2, c);
    spub += T(4, c) - T(3, c);
    ++ns;
  }
  printf("{\"n\": %d, \"tc\": %d, \"ctas\": %d, \"factor_ms\": %.4f, \"fail\": %d, "
         "\"step_us\": {\"wait\": %.3f, \"triangular_product\": %.3f, \"symmetric_update\": %.3f, "
         "\"leaf\": %.3f, \"publish\": %.3f, \"total\": %.3f}, \"chain_ms\": %.4f}\n",
         n, tc, cap, best, f, sw / ns / 1e3, sp1 / ns / 1e3, sp2 / ns / 1e3, sl2 / ns / 1e3,
         spub / ns / 1e3, (sw + sp1 + sp2 + sl2 + spub) / ns / 1e3, (T(4, p - 1) - T(0, 0)) / 1e6);
  return 0;
}
