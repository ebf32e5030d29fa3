"""Arithmetic of the emulated-FP64 products, checked on the CPU with exact
integer and rational arithmetic, independent of the CUDA kernels.

The scheme is error-free splitting into BF16 slices (Ozaki, Ogita, Oishi and
Rump 2012; fixed-point slices as in Mukunoki et al. 2020).  These tests pin
the facts the kernels rely on:

* Digits.  Row i of op(A) is scaled by 2^e_i, the smallest power of two with
  max_k |a_ik| < 2^(e_i + 7).  Each entry then becomes F = a_ik 2^(49 - e_i)
  rounded to an integer, so |F| <= 2^56.  F is written as 8 signed base-128
  digits, d_1 2^49 + d_2 2^42 + ... + d_8, each taken with round-half-up of
  the remainder.  The representation is exact, with |d_1| <= 128 and
  |d_j| <= 64 for j >= 2, so every d_j 2^(-7(j-1)) is exact in BF16.
* Level sums.  The pairs (j, l) of one level L = j + l, summed over 512
  consecutive k, stay within 2^24 in magnitude for L <= 7.  FP32 therefore
  accumulates them exactly, and only levels >= 8 need a rounded accumulator.
* Truncation.  Keeping the pairs with j + l <= 9 gives op(A) op(B) to within
  (S + 4) 2^(-7S) K max_k|a_ik| max_k|b_kn| with S = 8.  That is the bound
  the GPU tests apply before the FP32 and FP64 roundings.
"""
import math
from fractions import Fraction

import numpy as np

S = 8


def _row_scale(row):
    """e with max |row| < 2^(e + 7) (smallest such integer); None for a zero row."""
    m = max(abs(x) for x in row)
    if m == 0.0:
        return None
    _, ex = math.frexp(m)          # m = f 2^ex, 0.5 <= f < 1, so m < 2^ex
    return ex - 7


def _fixed(v, e):
    """round(v 2^(49 - e)) as an exact integer (half away from zero)."""
    q = Fraction(v) * Fraction(2) ** (49 - e)
    n = abs(q.numerator) * 2 + q.denominator
    r = n // (2 * q.denominator)
    return r if q >= 0 else -r


def _digits(F):
    """8 signed base-128 digits of F, most significant first, round half up."""
    out = []
    for j in range(S):
        sh = 49 - 7 * j
        if sh > 0:
            d = (F + (1 << (sh - 1))) >> sh
            F -= d << sh
        else:
            d = F
        out.append(d)
    return out


def test_digits_exact_and_bounded():
    rng = np.random.default_rng(3)
    vals = np.concatenate([
        rng.standard_normal(2000) * 10.0 ** rng.uniform(-300, 300, 2000),
        rng.standard_normal(2000),
        [0.0, 1.0, -1.0, 2.0 ** -1074, 1.7976931348623157e308, -2.0 ** 60, 0.5 - 2 ** -54]])
    for v in vals:
        e = _row_scale([v])
        if e is None:
            continue
        # a row's own largest entry gives the tightest case; smaller entries
        # of the same row only shrink F
        for x in (v, v * 0.75, v * 2.0 ** -30):
            F = _fixed(x, e)
            assert abs(F) <= 1 << 56
            d = _digits(F)
            assert sum(dj << (49 - 7 * j) for j, dj in enumerate(d)) == F
            assert abs(d[0]) <= 128 and all(abs(dj) <= 64 for dj in d[1:])
            # d_j 2^(-7j) in BF16: at most 8 significant bits
            assert all(abs(dj) <= 256 for dj in d)


def test_level_sums_fit_fp32_over_512():
    """Worst case over the digit bounds: |d_1| = 128, |d_j| = 64 otherwise,
    all signs aligned, 512 terms per level sum."""
    bound = [128] + [64] * (S - 1)
    for L in range(2, 2 * S + 1):
        per_k = sum(bound[j] * bound[L - 2 - j] for j in range(S) if 0 <= L - 2 - j < S)
        total = 512 * per_k
        if L <= 7:
            assert total <= 2 ** 24, (L, total)      # exact in FP32
        if L == 8:
            assert total > 2 ** 24                   # hence the rounded accumulator


def _emulated(A, B):
    """What the kernels compute before their FP32 / FP64 roundings: the
    digit-pair products with j + l <= S + 1 (1-based), exactly."""
    M, K = A.shape
    _, N = B.shape
    ea = [_row_scale(A[i]) for i in range(M)]
    fb = [_row_scale(B[:, n]) for n in range(N)]
    da = [[_digits(_fixed(A[i, k], ea[i])) if ea[i] is not None else [0] * S
           for k in range(K)] for i in range(M)]
    db = [[_digits(_fixed(B[k, n], fb[n])) if fb[n] is not None else [0] * S
           for k in range(K)] for n in range(N)]
    C = [[Fraction(0)] * N for _ in range(M)]
    for i in range(M):
        for n in range(N):
            if ea[i] is None or fb[n] is None:
                continue
            acc = 0            # in units of 2^-98 (both digits' weights)
            for k in range(K):
                a, b = da[i][k], db[n][k]
                for j in range(S):
                    for l in range(S - j):   # j + l <= S - 1 (0-based): levels <= S + 1
                        acc += (a[j] * b[l]) << (98 - 7 * (j + l))
            C[i][n] = Fraction(acc, 1 << 98) * Fraction(2) ** (ea[i] + fb[n])
    return C


def test_truncated_product_within_bound():
    rng = np.random.default_rng(7)
    for M, N, K, wide in [(3, 2, 40, False), (2, 3, 513, False), (2, 2, 64, True)]:
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((K, N))
        if wide:   # entries of a row spread over 6 decades, rows over 12
            A *= 10.0 ** rng.uniform(-3, 3, (M, K)) * 10.0 ** rng.uniform(-6, 6, (M, 1))
            B *= 10.0 ** rng.uniform(-3, 3, (K, N)) * 10.0 ** rng.uniform(-6, 6, (1, N))
        C = _emulated(A, B)
        for i in range(M):
            for n in range(N):
                exact = sum(Fraction(A[i, k]) * Fraction(B[k, n]) for k in range(K))
                bound = (Fraction(S + 4) * Fraction(2) ** (-7 * S) * K
                         * Fraction(float(np.max(np.abs(A[i])))) * Fraction(float(np.max(np.abs(B[:, n])))))
                assert abs(C[i][n] - exact) <= bound, (M, N, K, i, n)
