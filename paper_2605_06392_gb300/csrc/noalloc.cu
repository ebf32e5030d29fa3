// bta_factor_noalloc: the block factorisation of bta_factor, run out of a
// fixed scratch area in the library's device memory (a static __device__
// array), so the call itself never allocates.
//
// Who needs this: callers that cannot allocate device memory while they run
// the factorisation.  Examples are a serving process that has handed the
// whole device to its own allocator or fixed memory budget, a host framework
// that forbids allocation calls on its hot path, and code that cannot
// afford the device-wide synchronisation that freeing memory may imply.
// They pass in their inputs and outputs as usual; the temporary blocks the
// sweep needs (three ld x ld work blocks, the diagonal-factor scratch, arrow
// blocks, GEMV partials and the per-leaf log-determinant slots) live in the
// static array below instead of a per-call allocation.
//
// Limits (checked, BTA_ERR_ARG beyond them): ld <= 256, a <= 32, and
// n * (ld / 32) + 1 <= 16384 log-determinant slots (n <= 2047 at ld = 256).
// The array holds 2.4 MB and, once reserved on a GPU, stays there until the
// process exits.
//
// Sharing: all calls on a device use the same array.  Calls that overlap on
// the GPU (different streams, or different host threads without ordering)
// race on it and give wrong results; order them on one stream.  The array
// keeps the previous call's contents; nothing in it needs to start at zero
// (every work block and slot is written before it is read, and the sweep
// clears its arrow accumulator itself).
//
// Set-up: every call looks up the device address of the array on the
// current device (cudaGetSymbolAddress), so a device reset cannot leave a
// stale address behind.  Under CUDA's lazy module loading the first lookup on
// a device loads this file's device code and reserves the array there: that
// first call can itself allocate device memory and synchronise.  Callers on a
// strict budget should therefore make one call at set-up time, before any
// stream capture; later calls find the array in place and allocate nothing.
#include "sweep.cuh"

namespace {

using namespace bta;

constexpr int kNoAllocMaxLd = 256;
constexpr int kNoAllocMaxA = 32;
constexpr int kNoAllocMaxSlots = 16384;
// Work area of one sweep at the maximum sizes, in doubles (see SweepWs):
// 4 ld^2 + 2 a ld + kGemvSplit ld + a + 64.
constexpr size_t kWorkDoubles = 4 * (size_t)kNoAllocMaxLd * kNoAllocMaxLd +
                                2 * (size_t)kNoAllocMaxA * kNoAllocMaxLd +
                                (size_t)kGemvSplit * kNoAllocMaxLd + kNoAllocMaxA + 64;
constexpr size_t kScratchDoubles = kWorkDoubles + kNoAllocMaxSlots;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side stand-in, never the device memory; only
// this lookup gives the address a kernel may use.
bta_status scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    fprintf(stderr, "[bta] bta_factor_noalloc: cudaGetSymbolAddress failed: %s\n",
            cudaGetErrorString(e));
    return BTA_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return BTA_OK;
}

}  // namespace

extern "C" bta_status bta_factor_noalloc(bta_desc* q, double* rhs_inout, double* logdet,
                                         int32_t* fail_block, cudaStream_t stream) {
  if (!q || !logdet || !fail_block || q->n < 1 || q->b < 1 || q->ld < q->b || q->ld % kPad ||
      q->a < 0 || !q->D || (q->n > 1 && !q->B) || (q->a > 0 && (!q->C || !q->T)))
    return BTA_ERR_ARG;
  if (q->state != BTA_STATE_ASSEMBLED) return BTA_ERR_STATE;
  const int nsl = logdet_slots(q->n, q->ld);
  if (q->ld > kNoAllocMaxLd || q->a > kNoAllocMaxA || nsl > kNoAllocMaxSlots) {
    fprintf(stderr,
            "[bta] bta_factor_noalloc: size beyond the fixed scratch (ld %d of max %d, a %d of "
            "max %d, %d log-det slots of max %d); use bta_factor\n",
            q->ld, kNoAllocMaxLd, q->a, kNoAllocMaxA, nsl, kNoAllocMaxSlots);
    return BTA_ERR_ARG;
  }
  const size_t wsd = SweepWs::bytes(q->ld, q->a) / sizeof(double);
  if (wsd + (size_t)nsl > kScratchDoubles) return BTA_ERR_ARG;
  double* base = nullptr;
  BTA_TRY(scratch_address(&base));
  SweepWs ws;
  ws.carve(base, q->ld, q->a);
  double* slots = base + wsd;
  BTA_CUDA_TRY(cudaMemsetAsync(fail_block, 0xff, sizeof(int32_t), stream));
  bta_status st = factor_sweep(*q, rhs_inout, slots, fail_block, ws, stream);
  if (st == BTA_OK) st = sum_slots(slots, nsl, logdet, 0, stream);
  if (st == BTA_OK) q->state = BTA_STATE_FACTORED;
  return st;
}
