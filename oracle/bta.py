"""Banded BTA oracle: block sweep for f(theta) and its gradient (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's steps in its own order and notation, one block at a
time, with SciPy's dense Cholesky and triangular solves as the only
library primitives:

  * Section II-B: BTA blocks D_i (b x b), B_i = Q[i+1, i] (b x b),
    C_i = Q[T, i] (a x b), tip T (a x a).
  * Algorithm 1: fused block Cholesky and lower solve, producing L_Di,
    L_Bi, L_Ci, z_i, the carries S_i = L_Bi L_Bi^T, the updated tip and
    L_T, z_T.  log|Q| = 2 sum log diag(L).
  * Eqs. 3-5: upper solve x* from z.
  * Selected inversion (Section III-A, Phase A; the recurrences are not
    printed in the paper).  They follow from Z L = L^{-T}, read block
    column by block column from the bottom (L^{-T} is upper triangular with
    diagonal blocks L_Di^{-T}, L_T^{-T}):
        Z_T  = L_T^{-T} L_T^{-1}
        F_Bi = L_Bi L_Di^{-1},  F_Ci = L_Ci L_Di^{-1}
        Z_Ci = -Z_C,i+1 F_Bi - Z_T F_Ci                 (first term absent at i = n)
        Z_Bi = -Z_D,i+1 F_Bi - Z_C,i+1^T F_Ci           (i < n)
        Z_Di = L_Di^{-T} L_Di^{-1} - Z_Bi^T F_Bi - Z_Ci^T F_Ci
  * Eq. 7: Phase A trace as a sum of per-block traces.
  * Eq. 8: Phase B quadratic form with x* held fixed (x_i^T dB_i^T x_{i+1};
    Eq. 9 drops the transpose, which is immaterial for the symmetric B
    blocks of these models).
  * Section III-A, Phase C: the same selected-inversion trace on the BT
    prior Q_p (no arrowhead; the fixed-effect tip of Q_p is a constant).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as la

from . import model as M


# ----------------------------------------------------------------------------
# Block extraction (Section II-B)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Blocks:
    n: int
    b: int
    a: int
    D: list      # n dense b x b
    B: list      # n-1 dense b x b, block (i+1, i)
    C: list      # n dense a x b, block (T, i)
    T: np.ndarray  # a x a


def extract(Q, n, b, a) -> Blocks:
    Q = Q.tocsr()
    D = [Q[i * b:(i + 1) * b, i * b:(i + 1) * b].toarray() for i in range(n)]
    B = [Q[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b].toarray() for i in range(n - 1)]
    C = [Q[n * b:n * b + a, i * b:(i + 1) * b].toarray() for i in range(n)]
    T = Q[n * b:, n * b:].toarray()
    return Blocks(n, b, a, D, B, C, T)


def split_vec(v, n, b):
    return [v[i * b:(i + 1) * b].copy() for i in range(n)], v[n * b:].copy()


def join_vec(parts, tail):
    return np.concatenate(list(parts) + [tail])


# ----------------------------------------------------------------------------
# Algorithm 1: fused BTA Cholesky with lower triangular solve
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Factor:
    n: int
    b: int
    a: int
    LD: list
    LB: list
    LC: list
    LT: np.ndarray
    S: list          # carries S_1..S_{n-1}
    z: list
    zT: np.ndarray
    logdet: float


def _chol(A):
    return la.cholesky(A, lower=True)


def _trsm_right_lt(X, L):
    """X L^{-T}: solve Y L^T = X for Y."""
    return la.solve_triangular(L, X.T, lower=True).T


def factor(blk: Blocks, r=None) -> Factor:
    n, b, a = blk.n, blk.b, blk.a
    if r is None:
        r = np.zeros(n * b + a)
    rb, rT = split_vec(r, n, b)
    S_prev = np.zeros((b, b))
    Ttil = blk.T.copy()
    CL_prev = np.zeros((a, b))
    LB_prev = np.zeros((b, b))
    z_prev = np.zeros(b)
    vT = np.zeros(a)
    LD, LB, LC, S, z = [], [], [], [], []
    logdet = 0.0
    for i in range(n):
        Ld = _chol(blk.D[i] - S_prev)
        Lc = _trsm_right_lt(blk.C[i] - CL_prev @ LB_prev.T, Ld)
        zi = la.solve_triangular(Ld, rb[i] - LB_prev @ z_prev, lower=True)
        vT = vT + Lc @ zi
        if i < n - 1:
            Lb = _trsm_right_lt(blk.B[i], Ld)
            S_prev = Lb @ Lb.T
            S.append(S_prev)
            LB.append(Lb)
            LB_prev = Lb
        Ttil = Ttil - Lc @ Lc.T
        CL_prev = Lc
        z_prev = zi
        LD.append(Ld)
        LC.append(Lc)
        z.append(zi)
        logdet += 2.0 * float(np.sum(np.log(np.diag(Ld))))
    if a > 0:
        LT = _chol(Ttil)
        zT = la.solve_triangular(LT, rT - vT, lower=True)
        logdet += 2.0 * float(np.sum(np.log(np.diag(LT))))
    else:
        LT = np.zeros((0, 0))
        zT = np.zeros(0)
    return Factor(n, b, a, LD, LB, LC, LT, S, z, zT, logdet)


# ----------------------------------------------------------------------------
# Eqs. 3-5: upper triangular solve
# ----------------------------------------------------------------------------
def upper_solve(F: Factor):
    n = F.n
    if F.a > 0:
        xT = la.solve_triangular(F.LT, F.zT, lower=True, trans="T")
    else:
        xT = np.zeros(0)
    x = [None] * n
    for i in range(n - 1, -1, -1):
        rhs = F.z[i] - F.LC[i].T @ xT
        if i < n - 1:
            rhs = rhs - F.LB[i].T @ x[i + 1]
        x[i] = la.solve_triangular(F.LD[i], rhs, lower=True, trans="T")
    return join_vec(x, xT)


# ----------------------------------------------------------------------------
# Selected inversion
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class SelInv:
    ZD: list
    ZB: list
    ZC: list
    ZT: np.ndarray


def _inv_lower(L):
    return la.solve_triangular(L, np.eye(L.shape[0]), lower=True)


def selinv(F: Factor) -> SelInv:
    n, b, a = F.n, F.b, F.a
    if a > 0:
        LTi = _inv_lower(F.LT)
        ZT = LTi.T @ LTi
    else:
        ZT = np.zeros((0, 0))
    ZD = [None] * n
    ZB = [None] * (n - 1)
    ZC = [None] * n
    for i in range(n - 1, -1, -1):
        Li = _inv_lower(F.LD[i])
        FC = F.LC[i] @ Li
        ZCi = -ZT @ FC
        if i < n - 1:
            FB = F.LB[i] @ Li
            ZCi = ZCi - ZC[i + 1] @ FB
            ZBi = -ZD[i + 1] @ FB - ZC[i + 1].T @ FC
            ZDi = Li.T @ Li - ZBi.T @ FB - ZCi.T @ FC
            ZB[i] = ZBi
        else:
            ZDi = Li.T @ Li - ZCi.T @ FC
        ZD[i] = ZDi
        ZC[i] = ZCi
    return SelInv(ZD, ZB, ZC, ZT)


# ----------------------------------------------------------------------------
# Phase traces (Eq. 7) and quadratic form (Eq. 8)
# ----------------------------------------------------------------------------
def _sparse_block(Qs, r0, r1, c0, c1):
    return Qs[r0:r1, c0:c1]


def trace_eq7(Z: SelInv, dQ, n, b, a) -> float:
    """sum_i tr(Z_Di dD_i) + 2 sum_i tr(Z_Bi^T dB_i) + 2 sum_i tr(Z_Ci^T dC_i)
    + tr(Z_T dT), with the block Jacobians read from the sparse dQ."""
    dQ = dQ.tocsr()
    tot = 0.0
    for i in range(n):
        dD = _sparse_block(dQ, i * b, (i + 1) * b, i * b, (i + 1) * b)
        tot += float(dD.multiply(Z.ZD[i]).sum())
        if i < n - 1:
            dB = _sparse_block(dQ, (i + 1) * b, (i + 2) * b, i * b, (i + 1) * b)
            tot += 2.0 * float(dB.multiply(Z.ZB[i]).sum())
        if a > 0:
            dC = _sparse_block(dQ, n * b, n * b + a, i * b, (i + 1) * b)
            tot += 2.0 * float(dC.multiply(Z.ZC[i]).sum())
    if a > 0:
        dT = _sparse_block(dQ, n * b, n * b + a, n * b, n * b + a)
        tot += float(dT.multiply(Z.ZT).sum())
    return tot


def quad_eq8(x, dQ, n, b) -> float:
    """sum_i x_i^T dD_i x_i + 2 sum_i x_i^T dB_i^T x_{i+1} (latent part)."""
    dQ = dQ.tocsr()
    xs = [x[i * b:(i + 1) * b] for i in range(n)]
    tot = 0.0
    for i in range(n):
        dD = _sparse_block(dQ, i * b, (i + 1) * b, i * b, (i + 1) * b)
        tot += float(xs[i] @ (dD @ xs[i]))
        if i < n - 1:
            dB = _sparse_block(dQ, (i + 1) * b, (i + 2) * b, i * b, (i + 1) * b)
            tot += 2.0 * float(xs[i] @ (dB.T @ xs[i + 1]))
    return tot


# ----------------------------------------------------------------------------
# f and gradient by the block sweep
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class BTAResult:
    f: float
    grad: np.ndarray
    logdet_p: float
    logdet_c: float
    x: np.ndarray
    quad: float
    loglik: float
    logprior: float
    phase_a: np.ndarray
    phase_b: np.ndarray
    phase_c: np.ndarray
    explicit: np.ndarray


def quad_form_blocks(blk: Blocks, x) -> float:
    """x^T Q x over the latent BT part (Eq. 8 with Q in place of dQ)."""
    n, b = blk.n, blk.b
    xs = [x[i * b:(i + 1) * b] for i in range(n)]
    tot = 0.0
    for i in range(n):
        tot += float(xs[i] @ (blk.D[i] @ xs[i]))
        if i < n - 1:
            tot += 2.0 * float(xs[i] @ (blk.B[i].T @ xs[i + 1]))
    return tot


def evaluate(prob, theta=None, grad: bool = True) -> BTAResult:
    mdl = M.build_model(prob, theta)
    n, b, a = prob.nt, prob.b, prob.a
    # Q_c: full BTA (Algorithm 1 with the right-hand side r)
    blk_c = extract(mdl.Qc, n, b, a)
    Fc = factor(blk_c, mdl.r)
    x = upper_solve(Fc)
    # Q_p: BT latent part; the fixed-effect tip 1e-3 I_a is a constant block
    blk_p = extract(mdl.Qst, n, b, 0)
    Fp = factor(blk_p)
    logdet_p = Fp.logdet + a * np.log(M.TIP_PRIOR)
    beta = x[n * b:]
    quad = quad_form_blocks(blk_p, x) + M.TIP_PRIOR * float(beta @ beta)
    ll, dll = M.log_lik(mdl, x)
    lp, dlp = M.log_prior(mdl.theta)
    f = 0.5 * logdet_p - 0.5 * Fc.logdet - 0.5 * quad + ll + lp
    d = mdl.theta.shape[0]
    pa = np.zeros(d)
    pb = np.zeros(d)
    pc = np.zeros(d)
    if grad:
        Zc = selinv(Fc)
        Zp = selinv(Fp)
        for j in range(d):
            pa[j] = -0.5 * trace_eq7(Zc, mdl.dQc[j], n, b, a)
            pb[j] = -0.5 * quad_eq8(x, mdl.dQp[j], n, b)
            dQst = mdl.dQp[j][:n * b, :n * b]
            pc[j] = 0.5 * trace_eq7(Zp, dQst, n, b, 0)
    expl = dlp + dll
    g = pa + pb + pc + expl
    return BTAResult(f, g, logdet_p, Fc.logdet, x, quad, ll, lp, pa, pb, pc, expl)


def value(prob, theta=None) -> float:
    return evaluate(prob, theta, grad=False).f
