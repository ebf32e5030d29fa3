"""Seeded synthetic inputs for the spatio-temporal INLA objective.

This module is shared by the FP64 CPU oracle (``oracle/``) and by the GPU
library's tests and benchmark.  It draws *inputs only*: grid sizes, the
observation design (which latent node each observation row touches, its
covariates, its response variable), the observations ``y`` and the
hyperparameter points ``theta``.  It holds none of the method's arithmetic:
no precision matrix, stencil, factorisation or objective is formed here, so
neither consumer can inherit a mistake from the other through it.

Shapes follow the paper's benchmark family (Table I, Section IV-A): a
regular ``nx x ny`` spatial grid per variable, ``n_t`` time steps, ``k``
response variables (block size ``b = k * nx * ny``), ``a`` fixed effects
forming the arrowhead, and ``n_obs`` point observations drawn uniformly over
(time, node, variable).  The observations are not drawn from the GMRF prior
(doing so needs a factorisation, i.e. the method itself); instead each
variable's latent field is a smooth random superposition of space-time
Fourier modes, plus fixed effects and Gaussian noise of precision tau.  The
objective is defined for any ``y``; ``y`` only sets the conditioning.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["Problem", "WORKLOADS", "make_problem", "theta_dim", "fd_stencil",
           "make_batch"]


@dataclasses.dataclass(frozen=True)
class Problem:
    """One synthetic dataset plus a hyperparameter point.

    Latent ordering (used by every consumer): time-major blocks
    ``x = [x_1 .. x_nt, beta]``; inside a time block the ``k`` variables are
    stacked (variable-major), inside a variable the grid node is
    ``s = iy * nx + ix``.  ``b = k * nx * ny`` and ``N = nt * b + a``.
    """

    name: str
    k: int              # number of response variables
    nx: int
    ny: int
    nt: int
    a: int              # number of fixed effects (arrowhead width)
    a_r: int            # fixed effects per response (a == k * a_r)
    intercept: bool     # first fixed effect of every response is a constant 1
    obs_t: np.ndarray   # int32 [n_obs]  time index of each observation row
    obs_s: np.ndarray   # int32 [n_obs]  grid node of each row
    obs_v: np.ndarray   # int32 [n_obs]  response variable of each row
    obs_cov: np.ndarray  # float64 [n_obs, a_r] covariates of the row's response
    y: np.ndarray       # float64 [n_obs]
    theta: np.ndarray   # float64 [d]     evaluation point
    theta_true: np.ndarray  # float64 [d] point used to draw y
    seed: int

    @property
    def ns(self) -> int:
        return self.nx * self.ny

    @property
    def b(self) -> int:
        return self.k * self.nx * self.ny

    @property
    def N(self) -> int:
        return self.nt * self.b + self.a

    @property
    def n_obs(self) -> int:
        return int(self.y.shape[0])

    @property
    def d(self) -> int:
        return theta_dim(self.k)

    def with_theta(self, theta) -> "Problem":
        return dataclasses.replace(self, theta=np.asarray(theta, dtype=np.float64).copy())


def theta_dim(k: int) -> int:
    """Hyperparameter count: 4 per variable plus one coupling per pair
    (Section II-B: d = 4k + C(k,2)).  Univariate layout is
    (log scale, log kappa, log gamma, log tau); multivariate layout is
    (log kappa_1..k, log gamma_1..k, log sigma_1..k, lambda_21, lambda_31,
    lambda_32, ..., log tau_1..k)."""
    return 4 * k + k * (k - 1) // 2


# Workload table.  Sizes mirror the paper's model family; theta_true values
# for the univariate models are the ones the benchmark definitions fix.
WORKLOADS = {
    # 8x8 grid, b=64, 4 time steps, 4 covariates, 512 rows (GST-S-like).
    "st_tiny": dict(k=1, nx=8, ny=8, nt=4, a=4, n_obs=512,
                    theta_true=(0.0, 0.5, 0.0, 2.0), seed=0),
    # 32x32 grid, b=1024, 50 time steps, 6 covariates, 1e5 rows (GST-M-like).
    "st_medium": dict(k=1, nx=32, ny=32, nt=50, a=6, n_obs=100_000,
                      theta_true=(0.3, 1.0, -0.5, 1.5), seed=1),
    # The same model cut to 6 time steps and 12 500 rows.
    "st_medium_nt6": dict(k=1, nx=32, ny=32, nt=6, a=6, n_obs=12_500,
                          theta_true=(0.3, 1.0, -0.5, 1.5), seed=1),
    # 45x45 grid, b=2025, 100 time steps, 8 covariates, 4e5 rows (GST-T scale).
    "st_large": dict(k=1, nx=45, ny=45, nt=100, a=8, n_obs=400_000,
                     theta_true=(0.3, 1.0, -0.5, 1.5), seed=2),
    # Three coregionalised responses on a 40x40 grid, b=4800, 192 steps,
    # 4 fixed effects per response (intercept + 3 covariates), 2e6 rows (SA1-like).
    "coreg_production": dict(k=3, nx=40, ny=40, nt=192, a=12, n_obs=2_000_000,
                             intercept=True, seed=3),
    # Small coregionalised models used for parity at several tiles.
    "coreg_tiny": dict(k=3, nx=4, ny=4, nt=3, a=6, n_obs=300, seed=4),
    "coreg_small": dict(k=3, nx=8, ny=8, nt=5, a=9, n_obs=3000, seed=5),
    "coreg_k2_small": dict(k=2, nx=6, ny=5, nt=4, a=4, n_obs=800, seed=6),
}


def _default_theta_true(k: int) -> np.ndarray:
    if k == 1:
        return np.array([0.0, 0.5, 0.0, 2.0])
    # log kappa, log gamma, log sigma, couplings, log tau
    lk = np.full(k, 0.4)
    lg = np.full(k, -0.3)
    ls = np.zeros(k)
    lam = np.full(k * (k - 1) // 2, 0.3)
    lt = np.full(k, 1.5)
    return np.concatenate([lk, lg, ls, lam, lt])


def _latent_field(rng, nx, ny, nt, n_modes=8):
    """Smooth random space-time field on the grid, values at all (t, iy, ix)."""
    amp = rng.standard_normal(n_modes) / math.sqrt(n_modes)
    fx = rng.integers(0, 3, n_modes)
    fy = rng.integers(0, 3, n_modes)
    ft = rng.integers(0, 3, n_modes)
    ph = rng.uniform(0, 2 * math.pi, n_modes)
    t = np.arange(nt)[:, None, None] / max(nt, 1)
    yy = np.arange(ny)[None, :, None] / ny
    xx = np.arange(nx)[None, None, :] / nx
    out = np.zeros((nt, ny, nx))
    for m in range(n_modes):
        out += amp[m] * np.sin(2 * math.pi * (fx[m] * xx + fy[m] * yy + ft[m] * t) + ph[m])
    return out.reshape(nt, ny * nx)


def _tau_of(theta_true: np.ndarray, k: int) -> np.ndarray:
    # observation precision sits in the last k entries in both layouts
    return np.exp(np.asarray(theta_true[-k:], dtype=np.float64))


def make_problem(name: str = "st_tiny", *, seed: int | None = None,
                 theta=None, theta_perturb: float = 0.1, **overrides) -> Problem:
    """Draw one workload.  ``theta`` defaults to ``theta_true`` plus a seeded
    N(0, theta_perturb^2) perturbation, so gradients are evaluated away from
    the data-generating point."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    k, nx, ny, nt, a = spec["k"], spec["nx"], spec["ny"], spec["nt"], spec["a"]
    n_obs = int(spec["n_obs"])
    intercept = bool(spec.get("intercept", False))
    seed = spec["seed"] if seed is None else seed
    if a % k:
        raise ValueError("a must be a multiple of k")
    a_r = a // k
    rng = np.random.default_rng(seed)
    tt = spec.get("theta_true")
    theta_true = np.asarray(tt if tt is not None else _default_theta_true(k), dtype=np.float64)
    if theta_true.shape != (theta_dim(k),):
        raise ValueError("theta_true has the wrong length")
    ns = nx * ny
    # Observation design: variable, time and node uniformly at random.
    obs_v = (np.arange(n_obs) % k).astype(np.int32)
    rng.shuffle(obs_v)
    obs_t = rng.integers(0, nt, n_obs).astype(np.int32)
    obs_s = rng.integers(0, ns, n_obs).astype(np.int32)
    cov = rng.standard_normal((n_obs, a_r))
    if intercept:
        cov[:, 0] = 1.0
    # Data: smooth latent field per variable + fixed effects + noise.
    beta = rng.standard_normal(a)
    fields = [_latent_field(rng, nx, ny, nt) for _ in range(k)]
    tau = _tau_of(theta_true, k)
    lat = np.empty(n_obs)
    for m in range(k):
        sel = obs_v == m
        lat[sel] = fields[m][obs_t[sel], obs_s[sel]]
    fe = np.einsum("ij,ij->i", cov, beta.reshape(k, a_r)[obs_v])
    noise = rng.standard_normal(n_obs) / np.sqrt(tau[obs_v])
    y = lat + fe + noise
    if theta is None:
        theta = theta_true + theta_perturb * rng.standard_normal(theta_true.shape)
    return Problem(name=name, k=k, nx=nx, ny=ny, nt=nt, a=a, a_r=a_r,
                   intercept=intercept, obs_t=obs_t, obs_s=obs_s, obs_v=obs_v,
                   obs_cov=np.ascontiguousarray(cov), y=y,
                   theta=np.asarray(theta, dtype=np.float64).copy(),
                   theta_true=theta_true, seed=seed)


def fd_stencil(theta, h: float = 1e-3) -> np.ndarray:
    """The 2d+1 points of the central finite-difference gradient (Eq. 2):
    row 0 is theta, rows 1+2j and 2+2j are theta +/- h e_j."""
    theta = np.asarray(theta, dtype=np.float64)
    d = theta.shape[0]
    pts = np.repeat(theta[None, :], 2 * d + 1, axis=0)
    for j in range(d):
        pts[1 + 2 * j, j] += h
        pts[2 + 2 * j, j] -= h
    return pts


def make_batch(n_instances: int = 31, *, k: int = 3, nt: int = 40, a: int = 9,
               n_obs: int = 50_000, grids=(16, 24, 32), seed: int = 0):
    """Independent coregionalised instances of uneven block size: instance j
    draws its grid side from ``grids`` with seed j; its theta is the j-th
    point of the 2d+1 FD stencil around theta0 ~ N(0, 0.25 I) (seed ``seed``)."""
    d = theta_dim(k)
    theta0 = 0.5 * np.random.default_rng(seed).standard_normal(d)
    pts = fd_stencil(theta0, 1e-3)
    out = []
    for j in range(n_instances):
        g = int(np.random.default_rng(1000 + j).choice(grids))
        p = make_problem("coreg_small", seed=1000 + j, k=k, nx=g, ny=g, nt=nt, a=a,
                         n_obs=n_obs, theta=pts[j % pts.shape[0]])
        out.append(p)
    return out
