"""Central finite differences of the oracle objective (Eq. 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

df/dth_j ~ (f(th + h e_j) - f(th - h e_j)) / (2 h), 2d + 1 evaluations when
f(th) itself is included.
"""
from __future__ import annotations

import numpy as np

from . import bta, dense


def gradient(prob, theta=None, h: float = 1e-5, path: str = "dense") -> np.ndarray:
    theta = np.asarray(prob.theta if theta is None else theta, dtype=np.float64)
    fval = dense.value if path == "dense" else bta.value
    g = np.zeros_like(theta)
    for j in range(theta.shape[0]):
        tp = theta.copy()
        tm = theta.copy()
        tp[j] += h
        tm[j] -= h
        g[j] = (fval(prob, tp) - fval(prob, tm)) / (2 * h)
    return g
