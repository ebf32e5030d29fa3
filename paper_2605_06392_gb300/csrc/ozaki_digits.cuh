// Digit split and integer-to-FP64 composition of the emulated FP64 products
// (Ozaki scheme, fixed-point slices): shared by the emulated GEMM
// (ozaki_gemm.cu) and the task-graph leaves' 32 x 32 tile products
// (potrf_dag.cu).
#pragma once

#include <cstdint>

namespace bta {
namespace oz {

// Conversions between FP32 and 32-bit integers of magnitude below 2^22 by
// FP32 arithmetic against 1.5 2^23 (the FP32 adder's round to nearest even,
// exact for integers): one add and one integer operation each, on the
// full-rate pipes instead of the conversion unit.
__device__ __forceinline__ int f2i_small(float x) {
  return __float_as_int(x + 12582912.0f) - 0x4B400000;
}
__device__ __forceinline__ float i2f_small(int d) {
  return __int_as_float(d + 0x4B400000) - 12582912.0f;
}

// X * 2^E rounded to the nearest double, from the integer X by integer
// operations (the usual case); out-of-range exponents take ldexp.
__device__ __forceinline__ double compose(long long X, int E) {
  if (X == 0) return 0.0;
  const unsigned long long sgn = X < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = X < 0 ? 0ull - (unsigned long long)X : (unsigned long long)X;
  int lz = __clzll((long long)u);
  u <<= lz;                                   // leading one at bit 63
  unsigned long long m = u >> 11;             // 53 significant bits
  const unsigned long long rem = u & 0x7FFull;
  if (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) {
    ++m;
    if (m >> 53) { m >>= 1; --lz; }
  }
  const int be = 1023 + (63 - lz) + E;
  if (be <= 0 || be >= 2047) return ldexp((double)X, E);
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) |
                                          (m & ((1ull << 52) - 1))));
}

// The S signed base-128 digits of v for the row exponent bound er, each
// times its power of two (exact in BF16).
template <int S>
__device__ __forceinline__ void digits(double v, int er, float (&out)[S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long F = 0;   // v 2^(1078 - er): |F| < 2^56
  if (E != 0) {
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = E - er + 3;   // <= 3
    if (sh >= 0) {
      F = (long long)(mant << sh);
    } else if (sh > -54) {
      F = (long long)((mant + (1ull << (-sh - 1))) >> (-sh));
    }
    if (bits >> 63) F = -F;
  }
  // F = G 2^28 + R, R in [-2^27, 2^27): digits 1..4 from G, 5..8 from R,
  // each taken with round-half-up so that every remainder stays within
  // half a digit (|d_1| <= 128, |d_j| <= 64 otherwise); 32-bit arithmetic.
  const int G0 = (int)((F + (1ll << 27)) >> 28);
  const int R0 = (int)(F - (long long)G0 * (1ll << 28));
  int parts[2] = {G0, R0};
#pragma unroll
  for (int hpart = 0; hpart < 2; ++hpart) {
    int x = parts[hpart];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = 4 * hpart + jj;
      if (j >= S) break;
      int d;
      if (jj < 3) {
        const int sh = 21 - 7 * jj;
        d = (x + (1 << (sh - 1))) >> sh;
        x -= d * (1 << sh);
      } else {
        d = x;
      }
      out[j] = i2f_small(d) * __int_as_float((127 - 7 * j) << 23);
    }
  }
}

}  // namespace oz
}  // namespace bta
