"""Hyperparameter optimisation driver over the library's exact gradients.

The INLA pipeline maximises f(theta) with a quasi-Newton method (Section II-A
and II-D, the L-BFGS-B loop; Section IV-C, the convergence study).  This is
a plain L-BFGS (two-loop recursion, memory ``m``) on -f.  Its line search
tries several step lengths at once: the candidate thetas are evaluated
together in one batched call (their matrices swept in the same launches),
and the longest step meeting the Armijo condition is taken.  All
arithmetic on the objective happens in the library; this module only
combines gradient vectors into search directions.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class LbfgsResult:
    theta: np.ndarray
    f: float                 # f(theta) (the objective of Eq. 1, maximised)
    grad: np.ndarray
    iterations: int
    evaluations: int
    converged: bool
    history: list            # (f, ||grad||) per iteration


def lbfgs(model, theta0, *, m: int = 10, gtol: float = 1e-5, max_iter: int = 200,
          steps=(1.0, 0.5, 0.25, 0.1), c1: float = 1e-4, precision: int = 0,
          max_step: float = 1.0) -> LbfgsResult:
    """Maximise f over theta starting at theta0.  Stops when
    ||grad f||_inf <= gtol * max(1, |f|) or after max_iter iterations."""
    theta = np.asarray(theta0, dtype=np.float64).copy()
    f, g = model.value_and_grad(theta, precision=precision)
    # minimise phi = -f
    phi, dphi = -f, -g
    S, Y = [], []
    hist = [(f, float(np.linalg.norm(g)))]
    nev = 1
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        if np.max(np.abs(dphi)) <= gtol * max(1.0, abs(phi)):
            converged = True
            break
        # two-loop recursion: direction = -H dphi
        q = dphi.copy()
        alphas = []
        for s, y in reversed(list(zip(S, Y))):
            rho = 1.0 / float(y @ s)
            a = rho * float(s @ q)
            alphas.append((a, rho, s, y))
            q -= a * y
        if S:
            gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
        else:
            gamma = 1.0 / max(1.0, float(np.linalg.norm(dphi)))
        r = gamma * q
        for a, rho, s, y in reversed(alphas):
            b = rho * float(y @ r)
            r += (a - b) * s
        p = -r
        slope = float(dphi @ p)
        if slope >= 0.0:             # not a descent direction: restart
            S, Y = [], []
            p = -dphi / max(1.0, float(np.linalg.norm(dphi)))
            slope = float(dphi @ p)
        pn = float(np.max(np.abs(p)))
        if pn > max_step:
            p *= max_step / pn
            slope = float(dphi @ p)
        cands = np.array([theta + t * p for t in steps])
        fc, gc = model.value_and_grad(cands, precision=precision, concurrent=len(steps))
        nev += len(steps)
        accepted = None
        for idx, t in enumerate(steps):
            if -fc[idx] <= phi + c1 * t * slope and np.isfinite(fc[idx]):
                accepted = idx
                break
        if accepted is None:         # shrink further, one candidate at a time
            t = steps[-1]
            while accepted is None and t > 1e-8:
                t *= 0.25
                fn, gn = model.value_and_grad(theta + t * p, precision=precision)
                nev += 1
                if -fn <= phi + c1 * t * slope:
                    cands = np.array([theta + t * p])
                    fc, gc = np.array([fn]), np.array([gn])
                    accepted = 0
            if accepted is None:
                break
        new_theta = cands[accepted]
        new_phi, new_dphi = -fc[accepted], -gc[accepted]
        s_vec, y_vec = new_theta - theta, new_dphi - dphi
        if float(s_vec @ y_vec) > 1e-12 * float(np.linalg.norm(s_vec) * np.linalg.norm(y_vec)):
            S.append(s_vec)
            Y.append(y_vec)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
        theta, phi, dphi = new_theta, new_phi, new_dphi
        hist.append((-phi, float(np.linalg.norm(dphi))))
    return LbfgsResult(theta, -phi, -dphi, it, nev, converged, hist)
