"""Oracle model construction: sparse precision matrices and their exact
theta-derivatives, in plain SciPy sparse algebra (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.

Definitions followed:
  * Eq. 1 (Section II-A): Q_c = Q_p + tau A^T A, r = tau A^T y, x* = Q_c^{-1} r.
  * Section II-A, computational structure: Q_p is built from Kronecker
    products of temporal and spatial base matrices,
        Q_st = e^{th1} [M0 (x) K0 + 2 kappa gamma M1 (x) K1 + M2 (x) C],
        K0 = kappa^4 C + 2 kappa^2 G + GG,  K1 = kappa^2 C + G,
    with C = I, G the 5-point grid-graph Laplacian (Neumann), GG = G G,
    M0 = M2 = I and M1 = tridiag(-1, 2, -1) over the time steps.
  * Section II-B: BTA layout, N = n b + a; fixed effects form the arrowhead
    (their prior precision 1e-3 I sits in the tip of Q_p).
  * Section III-B, Eq. 10: multivariate super-blocks
        Q^(pq)(t, t') = sum_m W_pq^(m) Q_m(t, t'),
    read as the linear model of coregionalisation: u = (Lambda (x) I) w with
    independent w_m of precision Q_m (unit scale), Lambda lower-triangular
    with diagonal sigma_m = e^{theta_sd,m} and sub-diagonal couplings
    lambda_pq; then W_pq^(m) = (Lambda^{-1})_{mp} (Lambda^{-1})_{mq}.
  * Eqs. 11-12: per-variable parameters differentiate Q_m only, coupling
    parameters differentiate W only.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

TIP_PRIOR = 1e-3          # prior precision of every fixed effect
PRIOR_VAR = 100.0         # log p(theta) = -sum theta^2 / (2 * 100)


# ----------------------------------------------------------------------------
# Base matrices
# ----------------------------------------------------------------------------
def grid_laplacian(nx: int, ny: int) -> sp.csr_matrix:
    """5-point graph Laplacian of an nx-by-ny grid with natural (Neumann)
    boundary: degree on the diagonal, -1 for each horizontal/vertical
    neighbour.  Node s = iy * nx + ix."""
    def path(m):
        if m == 1:
            return sp.csr_matrix((1, 1))
        main = np.full(m, 2.0)
        main[0] = main[-1] = 1.0
        off = -np.ones(m - 1)
        return sp.diags([off, main, off], [-1, 0, 1], format="csr")
    return (sp.kron(sp.identity(ny), path(nx)) + sp.kron(path(ny), sp.identity(nx))).tocsr()


def temporal_matrices(nt: int):
    """M0 = I, M1 = tridiag(-1, 2, -1), M2 = I (all nt x nt)."""
    I = sp.identity(nt, format="csr")
    M1 = sp.diags([-np.ones(nt - 1), np.full(nt, 2.0), -np.ones(nt - 1)], [-1, 0, 1],
                  format="csr")
    return I, M1, I


@dataclasses.dataclass
class Params:
    """Unpacked hyperparameters.  For k == 1 the objective's univariate
    layout (log scale, log kappa, log gamma, log tau) is used; for k > 1 the
    layout (log kappa_m, log gamma_m, log sigma_m, lambda_pq (p>q, row order),
    log tau_m)."""
    k: int
    scale: float                 # e^{theta_1} (univariate only, else 1)
    kappa: np.ndarray            # [k]
    gamma: np.ndarray            # [k]
    sigma: np.ndarray            # [k]  (univariate: unused, 1)
    lam: np.ndarray              # [k(k-1)/2]
    tau: np.ndarray              # [k]


def coupling_pairs(k: int):
    """(p, q) index pairs of the coupling parameters, p > q, row order."""
    return [(p, q) for p in range(k) for q in range(p)]


def unpack(theta: np.ndarray, k: int) -> Params:
    theta = np.asarray(theta, dtype=np.float64)
    if k == 1:
        return Params(1, float(np.exp(theta[0])), np.exp(theta[1:2]), np.exp(theta[2:3]),
                      np.ones(1), np.zeros(0), np.exp(theta[3:4]))
    nc = k * (k - 1) // 2
    return Params(k, 1.0, np.exp(theta[0:k]), np.exp(theta[k:2 * k]),
                  np.exp(theta[2 * k:3 * k]), theta[3 * k:3 * k + nc].copy(),
                  np.exp(theta[3 * k + nc:]))


def lambda_matrix(sigma, lam, k):
    L = np.diag(np.asarray(sigma, dtype=np.float64))
    for c, (p, q) in enumerate(coupling_pairs(k)):
        L[p, q] = lam[c]
    return L


def coregional_weights(sigma, lam, k):
    """W[m, p, q] = (Lambda^{-1})_{mp} (Lambda^{-1})_{mq} (Eq. 10, LMC reading)."""
    Li = np.linalg.inv(lambda_matrix(sigma, lam, k))
    return np.einsum("mp,mq->mpq", Li, Li)


def coregional_weight_derivs(sigma, lam, k):
    """dW[j] for each coupling-type parameter j (log sigma_1..k, then lambda_pq):
    d(Lambda^{-1}) = -Lambda^{-1} dLambda Lambda^{-1}, product rule on W."""
    Lam = lambda_matrix(sigma, lam, k)
    Li = np.linalg.inv(Lam)
    dLams = []
    for m in range(k):
        E = np.zeros((k, k))
        E[m, m] = sigma[m]           # d sigma / d log sigma
        dLams.append(E)
    for (p, q) in coupling_pairs(k):
        E = np.zeros((k, k))
        E[p, q] = 1.0
        dLams.append(E)
    out = []
    for dL in dLams:
        dLi = -Li @ dL @ Li
        out.append(np.einsum("mp,mq->mpq", dLi, Li) + np.einsum("mp,mq->mpq", Li, dLi))
    return out


# ----------------------------------------------------------------------------
# Spatio-temporal precision of one variable and its derivatives
# ----------------------------------------------------------------------------
def st_precision_terms(nx, ny, nt):
    """The six Kronecker terms T_j (x) S_j of Q_st."""
    G = grid_laplacian(nx, ny)
    C = sp.identity(nx * ny, format="csr")
    GG = (G @ G).tocsr()
    M0, M1, M2 = temporal_matrices(nt)
    return dict(C=C, G=G, GG=GG, M0=M0, M1=M1, M2=M2)


def q_st(base, kappa, gamma, scale=1.0):
    """Q_st = scale [M0 (x) K0 + 2 kappa gamma M1 (x) K1 + M2 (x) C]."""
    C, G, GG = base["C"], base["G"], base["GG"]
    K0 = kappa ** 4 * C + 2 * kappa ** 2 * G + GG
    K1 = kappa ** 2 * C + G
    Q = sp.kron(base["M0"], K0) + 2 * kappa * gamma * sp.kron(base["M1"], K1) \
        + sp.kron(base["M2"], C)
    return (scale * Q).tocsr()


def dq_st_dlogkappa(base, kappa, gamma, scale=1.0):
    """d Q_st / d log kappa:  dK0 = 4 k^4 C + 4 k^2 G;  d(2 k g K1) = 2 k g K1 + 4 k^3 g C."""
    C, G = base["C"], base["G"]
    dK0 = 4 * kappa ** 4 * C + 4 * kappa ** 2 * G
    K1 = kappa ** 2 * C + G
    Q = sp.kron(base["M0"], dK0) + sp.kron(base["M1"], 2 * kappa * gamma * K1
                                          + 4 * kappa ** 3 * gamma * C)
    return (scale * Q).tocsr()


def dq_st_dloggamma(base, kappa, gamma, scale=1.0):
    """d Q_st / d log gamma = 2 kappa gamma M1 (x) K1."""
    C, G = base["C"], base["G"]
    K1 = kappa ** 2 * C + G
    return (scale * 2 * kappa * gamma * sp.kron(base["M1"], K1)).tocsr()


# ----------------------------------------------------------------------------
# Full model
# ----------------------------------------------------------------------------
def _perm_var_major_to_time_major(k, nt, ns):
    """Index map: position in (var, time, node) order for each position of
    the (time, var, node) latent order."""
    t, v, s = np.meshgrid(np.arange(nt), np.arange(k), np.arange(ns), indexing="ij")
    return (v * nt * ns + t * ns + s).reshape(-1)


def embed_multivariate(blocks_by_var_pair, k, nt, ns):
    """Place per-variable-pair spatio-temporal matrices (each nt*ns square,
    time-major) into the (time, var, node) ordering."""
    big = sp.bmat([[blocks_by_var_pair[p][q] for q in range(k)] for p in range(k)],
                  format="csr")
    perm = _perm_var_major_to_time_major(k, nt, ns)
    return big[perm][:, perm].tocsr()


@dataclasses.dataclass
class Model:
    prob: object
    theta: np.ndarray
    par: Params
    Qst: sp.csr_matrix          # prior precision of the latent field (n b)
    Qp: sp.csr_matrix           # blkdiag(Qst, 1e-3 I_a)
    A: sp.csr_matrix            # n_obs x N
    tau_row: np.ndarray         # tau of each observation row
    AtA_by_var: list            # per response m: A_m^T A_m (N x N)
    Qc: sp.csr_matrix
    r: np.ndarray
    dQp: list                   # d Qp / d theta_k (N x N), k = 0..d-1
    dQc: list                   # d Qc / d theta_k


def projection(prob) -> sp.csr_matrix:
    """A: row j has 1 at latent (t_j, v_j, s_j) and the row's covariates in its
    response's fixed-effect columns."""
    n_obs, b, nt = prob.n_obs, prob.b, prob.nt
    lat = prob.obs_t.astype(np.int64) * b + prob.obs_v.astype(np.int64) * prob.ns + prob.obs_s
    rows = [np.arange(n_obs)]
    cols = [lat]
    vals = [np.ones(n_obs)]
    for c in range(prob.a_r):
        rows.append(np.arange(n_obs))
        cols.append(nt * b + prob.obs_v.astype(np.int64) * prob.a_r + c)
        vals.append(prob.obs_cov[:, c])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n_obs, prob.N))


def build_model(prob, theta=None) -> Model:
    theta = np.asarray(prob.theta if theta is None else theta, dtype=np.float64)
    k, nt, ns, a = prob.k, prob.nt, prob.ns, prob.a
    par = unpack(theta, k)
    base = st_precision_terms(prob.nx, prob.ny, nt)
    d = theta.shape[0]
    dQst = [None] * d
    if k == 1:
        Qst = q_st(base, par.kappa[0], par.gamma[0], par.scale)
        dQst[0] = Qst.copy()                                        # d/d log scale
        dQst[1] = dq_st_dlogkappa(base, par.kappa[0], par.gamma[0], par.scale)
        dQst[2] = dq_st_dloggamma(base, par.kappa[0], par.gamma[0], par.scale)
        dQst[3] = sp.csr_matrix(Qst.shape)                          # log tau: none
    else:
        W = coregional_weights(par.sigma, par.lam, k)
        dW = coregional_weight_derivs(par.sigma, par.lam, k)
        Qm = [q_st(base, par.kappa[m], par.gamma[m]) for m in range(k)]

        def combine(weights, mats):
            # weights[m, p, q]; mats[m] or None
            pairs = [[sum(weights[m, p, q] * mats[m] for m in range(k) if mats[m] is not None)
                      for q in range(k)] for p in range(k)]
            return embed_multivariate(pairs, k, nt, ns)

        Qst = combine(W, Qm)
        nc = k * (k - 1) // 2
        for m in range(k):
            sel = [None] * k
            sel[m] = dq_st_dlogkappa(base, par.kappa[m], par.gamma[m])
            dQst[m] = combine(W, sel)                              # Eq. 11
            sel = [None] * k
            sel[m] = dq_st_dloggamma(base, par.kappa[m], par.gamma[m])
            dQst[k + m] = combine(W, sel)                          # Eq. 11
        for j in range(k + nc):
            dQst[2 * k + j] = combine(dW[j], Qm)                   # Eq. 12
        for m in range(k):
            dQst[3 * k + nc + m] = sp.csr_matrix(Qst.shape)
    tip = TIP_PRIOR * sp.identity(a, format="csr")
    Qp = sp.block_diag([Qst, tip], format="csr")
    dQp = [sp.block_diag([dq, sp.csr_matrix((a, a))], format="csr") for dq in dQst]
    A = projection(prob)
    tau_row = par.tau[prob.obs_v]
    AtA = []
    for m in range(k):
        Am = A[np.flatnonzero(prob.obs_v == m)]
        AtA.append((Am.T @ Am).tocsr())
    Qc = (Qp + sum(par.tau[m] * AtA[m] for m in range(k))).tocsr()
    r = A.T @ (tau_row * prob.y)
    dQc = list(dQp)
    for m in range(k):
        j = d - k + m                                              # log tau_m
        dQc[j] = (dQp[j] + par.tau[m] * AtA[m]).tocsr()
    return Model(prob, theta, par, Qst, Qp, A, tau_row, AtA, Qc, r, dQp, dQc)


def log_prior(theta):
    """Reading of the unspecified hyperprior: independent N(0, 10^2)."""
    theta = np.asarray(theta, dtype=np.float64)
    return -float(theta @ theta) / (2 * PRIOR_VAR), -theta / PRIOR_VAR


def log_lik(model: Model, x):
    """Gaussian log-likelihood without the 2 pi constant:
    sum_m [(n_m/2) log tau_m - (tau_m/2) ||y_m - A_m x||^2], and its exact
    partial derivative in each log tau_m with x held fixed."""
    prob, par = model.prob, model.par
    res = prob.y - model.A @ x
    k = prob.k
    val = 0.0
    grad = np.zeros(model.theta.shape[0])
    for m in range(k):
        sel = prob.obs_v == m
        nm = int(sel.sum())
        ss = float(res[sel] @ res[sel])
        val += 0.5 * nm * np.log(par.tau[m]) - 0.5 * par.tau[m] * ss
        grad[grad.shape[0] - k + m] = 0.5 * nm - 0.5 * par.tau[m] * ss
    return val, grad
