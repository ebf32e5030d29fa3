"""Dense FP64 oracle for f(theta) and its gradient (small N only).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is the plain definition written out with dense linear algebra:
  * Eq. 1: f = 1/2 log|Q_p| - 1/2 log|Q_c| - 1/2 x*^T Q_p x* + log l + log p.
    log|Q| comes from a dense Cholesky (2 sum log diag L).
  * Eq. 6 (Section III-A): with x* held fixed (envelope theorem),
        df/dth_k = -1/2 tr(Q_c^{-1} dQ_c) - 1/2 x*^T dQ_p x*
                   + 1/2 tr(Q_p^{-1} dQ_p) + d log p + d log l,
    the traces taken with the dense inverses.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as la

from . import model as M


@dataclasses.dataclass
class DenseResult:
    f: float
    grad: np.ndarray
    logdet_p: float
    logdet_c: float
    x: np.ndarray
    quad: float          # x*^T Q_p x*
    loglik: float
    logprior: float
    phase_a: np.ndarray  # -1/2 tr(Qc^-1 dQc_k)
    phase_b: np.ndarray  # -1/2 x*^T dQp_k x*
    phase_c: np.ndarray  # +1/2 tr(Qp^-1 dQp_k)
    explicit: np.ndarray  # d log p + d log l


def logdet_chol(Q: np.ndarray) -> float:
    L = la.cholesky(Q, lower=True)
    return 2.0 * float(np.sum(np.log(np.diag(L))))


def value(prob, theta=None):
    """f only (the finite-difference baseline's evaluation)."""
    return evaluate(prob, theta, grad=False).f


def evaluate(prob, theta=None, grad: bool = True) -> DenseResult:
    mdl = M.build_model(prob, theta)
    Qp = mdl.Qp.toarray()
    Qc = mdl.Qc.toarray()
    ld_p = logdet_chol(Qp)
    ld_c = logdet_chol(Qc)
    cf = la.cho_factor(Qc, lower=True)
    x = la.cho_solve(cf, mdl.r)
    quad = float(x @ (Qp @ x))
    ll, dll = M.log_lik(mdl, x)
    lp, dlp = M.log_prior(mdl.theta)
    f = 0.5 * ld_p - 0.5 * ld_c - 0.5 * quad + ll + lp
    d = mdl.theta.shape[0]
    pa = np.zeros(d)
    pb = np.zeros(d)
    pc = np.zeros(d)
    if grad:
        Zc = la.cho_solve(cf, np.eye(Qc.shape[0]))
        Zp = la.cho_solve(la.cho_factor(Qp, lower=True), np.eye(Qp.shape[0]))
        for j in range(d):
            dQc = mdl.dQc[j].toarray()
            dQp = mdl.dQp[j].toarray()
            pa[j] = -0.5 * float(np.sum(Zc * dQc))      # tr(Z dQ), both symmetric
            pb[j] = -0.5 * float(x @ (dQp @ x))
            pc[j] = 0.5 * float(np.sum(Zp * dQp))
    expl = dlp + dll
    g = pa + pb + pc + expl
    return DenseResult(f, g, ld_p, ld_c, x, quad, ll, lp, pa, pb, pc, expl)


def selected_inverse_dense(Q: np.ndarray) -> np.ndarray:
    """Full dense inverse; tests read the BTA-pattern entries out of it."""
    return la.cho_solve(la.cho_factor(Q, lower=True), np.eye(Q.shape[0]))
