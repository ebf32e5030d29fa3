"""Pins for the FP64 oracle: checks against facts fixed by the mathematics,
not by the oracle itself.

* Spectral closed form.  With C = I every spatial factor is a polynomial in
  the grid Laplacian G, and M0, M1, M2 are polynomials in M1, so Q_st is
  diagonalised by the Kronecker product of their eigenbases.  The Neumann
  path Laplacian on m nodes has eigenvalues 2 - 2 cos(pi p / m), p = 0..m-1;
  tridiag(-1, 2, -1) on n nodes has 2 - 2 cos(pi j / (n + 1)), j = 1..n.
  Each eigenvalue of Q_st is s[(k^2+mu)^2 + 2 k g nu (k^2+mu) + 1], which
  fixes log|Q_p| and every Phase C term (1/2 sum dlambda/lambda) exactly.
* Multivariate: log|Q| = sum_m log|Q_m| - 2 nt ns sum_m log sigma_m because
  Lambda is triangular; the couplings lambda leave log|Q_p| unchanged.
* Brute force on tiny inputs: dense inverse / slogdet against the block
  sweep's selected inverse and log-determinant.
* Finite differences of f (Eq. 2) at h = 1e-5; envelope-theorem check.
* Identities: Phase A(th1) + Phase A(log tau) = -1/2 (N - 1e-3 tr Z_T);
  Phase B(th1) = -1/2 x_st^T Q_st x_st; [Q Z]_ii = I using selected blocks only.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads
from oracle import bta, dense, model as M


def _path_eigs(m):
    return 2.0 - 2.0 * np.cos(np.pi * np.arange(m) / m)


def _grid_eigs(nx, ny):
    return (_path_eigs(nx)[None, :] + _path_eigs(ny)[:, None]).reshape(-1)


def _m1_eigs(n):
    return 2.0 - 2.0 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1))


def _spectral_univariate(nx, ny, nt, scale, kappa, gamma):
    mu = _grid_eigs(nx, ny)[None, :]
    nu = _m1_eigs(nt)[:, None]
    u = kappa ** 2 + mu
    lam = scale * (u ** 2 + 2 * kappa * gamma * nu * u + 1.0)
    dk = scale * (4 * kappa ** 2 * u + 2 * kappa * gamma * nu * u + 4 * kappa ** 3 * gamma * nu)
    dg = scale * (2 * kappa * gamma * nu * u)
    return lam, dk, dg


@pytest.mark.parametrize("name,theta", [
    ("st_tiny", None),
    ("st_tiny", [0.7, -0.4, 0.9, 1.0]),
    ("st_tiny", [-1.2, 1.3, -0.8, 0.0]),
])
def test_prior_logdet_and_phase_c_spectral(name, theta):
    p = workloads.make_problem(name)
    if theta is not None:
        p = p.with_theta(theta)
    th = p.theta
    lam, dk, dg = _spectral_univariate(p.nx, p.ny, p.nt, np.exp(th[0]), np.exp(th[1]), np.exp(th[2]))
    ld_exact = float(np.sum(np.log(lam))) + p.a * np.log(1e-3)
    pc_exact = np.array([0.5 * lam.size, 0.5 * np.sum(dk / lam), 0.5 * np.sum(dg / lam), 0.0])
    d = dense.evaluate(p)
    b = bta.evaluate(p)
    assert abs(d.logdet_p - ld_exact) <= 1e-11 * abs(ld_exact)
    assert abs(b.logdet_p - ld_exact) <= 1e-11 * abs(ld_exact)
    np.testing.assert_allclose(d.phase_c, pc_exact, rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(b.phase_c, pc_exact, rtol=1e-11, atol=1e-9)


def test_prior_logdet_scale_shift_closed_form():
    # d/dth1 log|Q_st| = N_st exactly: log|Q_st(th1)| - log|Q_st(0)| = N_st th1
    p = workloads.make_problem("st_tiny")
    t0 = p.theta.copy()
    t1 = t0.copy()
    t1[0] += 0.37
    l0 = bta.evaluate(p, t0, grad=False).logdet_p
    l1 = bta.evaluate(p, t1, grad=False).logdet_p
    assert abs((l1 - l0) - p.nt * p.b * 0.37) < 1e-9


@pytest.mark.parametrize("name", ["coreg_tiny", "coreg_k2_small"])
def test_multivariate_logdet_and_phase_c_closed_form(name):
    p = workloads.make_problem(name)
    k = p.k
    nc = k * (k - 1) // 2
    th = p.theta
    kap, gam, sig = np.exp(th[:k]), np.exp(th[k:2 * k]), np.exp(th[2 * k:3 * k])
    ld = 0.0
    pc = np.zeros(p.d)
    nst = p.nt * p.ns
    for m in range(k):
        lam, dk, dg = _spectral_univariate(p.nx, p.ny, p.nt, 1.0, kap[m], gam[m])
        ld += float(np.sum(np.log(lam)))
        pc[m] = 0.5 * np.sum(dk / lam)
        pc[k + m] = 0.5 * np.sum(dg / lam)
        pc[2 * k + m] = -nst           # 1/2 d/dlog sigma of (-2 nst log sigma)
    ld += -2.0 * nst * float(np.sum(np.log(sig))) + p.a * np.log(1e-3)
    # couplings (indices 3k .. 3k+nc-1) and log tau: zero
    b = bta.evaluate(p)
    assert abs(b.logdet_p - ld) <= 1e-11 * abs(ld)
    np.testing.assert_allclose(b.phase_c, pc, rtol=1e-10, atol=1e-8)
    assert np.all(np.abs(b.phase_c[3 * k:3 * k + nc]) < 1e-8)


@pytest.mark.parametrize("name", ["st_tiny", "coreg_tiny"])
def test_bta_logdet_and_selinv_brute_force(name):
    p = workloads.make_problem(name)
    mdl = M.build_model(p)
    n, b, a = p.nt, p.b, p.a
    Qc = mdl.Qc.toarray()
    Zd = np.linalg.inv(Qc)
    blk = bta.extract(mdl.Qc, n, b, a)
    F = bta.factor(blk, mdl.r)
    sign, ld = np.linalg.slogdet(Qc)
    assert sign > 0 and abs(F.logdet - ld) <= 1e-12 * abs(ld)
    Z = bta.selinv(F)
    for i in range(n):
        np.testing.assert_allclose(Z.ZD[i], Zd[i * b:(i + 1) * b, i * b:(i + 1) * b],
                                   rtol=1e-10, atol=1e-13)
        np.testing.assert_allclose(Z.ZC[i], Zd[n * b:, i * b:(i + 1) * b], rtol=1e-10, atol=1e-13)
        if i < n - 1:
            np.testing.assert_allclose(Z.ZB[i], Zd[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b],
                                       rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(Z.ZT, Zd[n * b:, n * b:], rtol=1e-10, atol=1e-13)
    # the mode: plain dense solve
    x_dense = np.linalg.solve(Qc, mdl.r)
    np.testing.assert_allclose(bta.upper_solve(F), x_dense, rtol=1e-10, atol=1e-12)


def test_selinv_identities_from_selected_blocks_only():
    # [QZ]_ii = B_{i-1} Z_{i-1,i} + D_i Z_ii + B_i^T Z_{i+1,i} + C_i^T Z_{T,i} = I
    # [QZ]_TT = sum_i C_i Z_Ci^T + T Z_T = I
    p = workloads.make_problem("st_medium_nt6", nx=12, ny=10, n_obs=2000)
    mdl = M.build_model(p)
    n, b, a = p.nt, p.b, p.a
    blk = bta.extract(mdl.Qc, n, b, a)
    Z = bta.selinv(bta.factor(blk, mdl.r))
    I = np.eye(b)
    for i in range(n):
        acc = blk.D[i] @ Z.ZD[i] + blk.C[i].T @ Z.ZC[i]
        if i > 0:
            acc += blk.B[i - 1] @ Z.ZB[i - 1].T
        if i < n - 1:
            acc += blk.B[i].T @ Z.ZB[i]
        np.testing.assert_allclose(acc, I, atol=1e-10)
    accT = blk.T @ Z.ZT + sum(blk.C[i] @ Z.ZC[i].T for i in range(n))
    np.testing.assert_allclose(accT, np.eye(a), atol=1e-10)


@pytest.mark.parametrize("name,over", [("st_tiny", {}), ("coreg_tiny", {}),
                                       ("st_tiny", {"a": 0})])   # no fixed effects: no arrow
def test_gradient_matches_central_fd(name, over):
    p = workloads.make_problem(name, **over)
    g = dense.evaluate(p).grad
    gfd = oracle.fd.gradient(p, h=1e-5, path="dense")
    scale = np.maximum(np.abs(g), 1.0)
    assert np.max(np.abs(g - gfd) / scale) < 1e-7


@pytest.mark.parametrize("name,over", [("st_tiny", {}), ("coreg_tiny", {}),
                                       ("st_tiny", {"a": 0}), ("st_tiny", {"n_obs": 0}),
                                       ("st_tiny", {"nx": 1, "ny": 1}),
                                       ("st_tiny", {"nx": 3, "ny": 1, "nt": 2, "n_obs": 30})])
def test_bta_path_equals_dense_path(name, over):
    p = workloads.make_problem(name, **over)
    d = dense.evaluate(p)
    b = bta.evaluate(p)
    assert abs(d.f - b.f) <= 1e-12 * abs(d.f)
    np.testing.assert_allclose(b.grad, d.grad, rtol=1e-11, atol=1e-9)
    for attr in ("phase_a", "phase_b", "phase_c"):
        np.testing.assert_allclose(getattr(b, attr), getattr(d, attr), rtol=1e-11, atol=1e-9)


def test_mode_residual_and_envelope():
    p = workloads.make_problem("st_tiny")
    mdl = M.build_model(p)
    r = dense.evaluate(p)
    x = r.x
    res = np.linalg.norm(mdl.Qc @ x - mdl.r) / np.linalg.norm(mdl.r)
    assert res < 1e-12

    # f's x-dependent part g(x) = -1/2 x^T Qp x + log l(y | x) is stationary at x*.
    def gx(xx):
        return -0.5 * float(xx @ (mdl.Qp @ xx)) + M.log_lik(mdl, xx)[0]
    rng = np.random.default_rng(7)
    dx = rng.standard_normal(x.shape)
    dx /= np.linalg.norm(dx)
    g0 = gx(x)
    d1 = gx(x + 1e-3 * dx) - g0
    d2 = gx(x + 2e-3 * dx) - g0
    # second order: doubling the step quadruples the change
    assert abs(d2 / d1 - 4.0) < 1e-3


def test_phase_identities_univariate():
    p = workloads.make_problem("st_tiny")
    r = bta.evaluate(p)
    mdl = M.build_model(p)
    n, b, a = p.nt, p.b, p.a
    Z = bta.selinv(bta.factor(bta.extract(mdl.Qc, n, b, a), mdl.r))
    N = p.N
    np.testing.assert_allclose(r.phase_a[0] + r.phase_a[3], -0.5 * (N - 1e-3 * np.trace(Z.ZT)),
                               rtol=1e-12)
    xs = r.x[:n * b]
    np.testing.assert_allclose(r.phase_b[0], -0.5 * float(xs @ (mdl.Qst @ xs)), rtol=1e-12)


def test_matrix_derivatives_match_fd_of_matrices():
    # dQ/dth_k against central differences of the assembled matrices
    for name in ("st_tiny", "coreg_tiny"):
        p = workloads.make_problem(name)
        mdl = M.build_model(p)
        h = 1e-6
        for j in range(p.d):
            tp = p.theta.copy()
            tm = p.theta.copy()
            tp[j] += h
            tm[j] -= h
            fd = (M.build_model(p, tp).Qc - M.build_model(p, tm).Qc) / (2 * h)
            diff = abs(fd - mdl.dQc[j]).max()
            scale = max(abs(mdl.dQc[j]).max(), 1.0)
            assert diff / scale < 1e-7, (name, j)


def test_b_blocks_symmetric_so_eq8_and_eq9_agree():
    for name in ("st_tiny", "coreg_tiny"):
        p = workloads.make_problem(name)
        mdl = M.build_model(p)
        blk = bta.extract(mdl.Qc, p.nt, p.b, p.a)
        for B in blk.B:
            np.testing.assert_array_equal(B, B.T)


def test_coregional_weights_definition():
    # Q^(pq) = sum_m W_pq^(m) Q_m must equal (Lambda^-T (x) I) blkdiag(Q_m) (Lambda^-1 (x) I)
    rng = np.random.default_rng(3)
    k = 3
    sig = np.exp(rng.standard_normal(k))
    lam = rng.standard_normal(3)
    W = M.coregional_weights(sig, lam, k)
    Lam = M.lambda_matrix(sig, lam, k)
    mats = [np.diag(rng.uniform(1, 2, 4)) for _ in range(k)]
    Li = np.linalg.inv(Lam)
    big = np.kron(Li.T, np.eye(4)) @ sp.block_diag([sp.csr_matrix(m_) for m_ in mats]).toarray() @ np.kron(Li, np.eye(4))
    for pp in range(k):
        for q in range(k):
            blkpq = sum(W[m, pp, q] * mats[m] for m in range(k))
            np.testing.assert_allclose(big[pp * 4:(pp + 1) * 4, q * 4:(q + 1) * 4], blkpq, atol=1e-12)


def _coreg_scaling_sums(p, res):
    """The scaling identities of the coregionalised prior.  With
    Lambda -> e^t Lambda (log sigma_m += t, lambda_pq *= e^t) the weights
    (Lambda^-1)_mp (Lambda^-1)_mq, and so Q_st, scale by e^-2t:
      sum_m A_{log sigma_m} + sum lambda_pq A_{lambda_pq} - 2 sum_m A_{log tau_m}
          = N - 1e-3 tr(Z_T)
      sum_m B_{log sigma_m} + sum lambda_pq B_{lambda_pq} = x*' Q_st x*
    (A, B: the Phase A and Phase B terms; Z_T the tip block of Q_c^-1).
    Returns the two left-hand sides."""
    k = p.k
    nc = k * (k - 1) // 2
    th = p.theta
    lam = th[3 * k:3 * k + nc]
    pa, pb = np.asarray(res.phase_a), np.asarray(res.phase_b)
    sa = (pa[2 * k:3 * k].sum() + float(lam @ pa[3 * k:3 * k + nc])
          - 2.0 * pa[3 * k + nc:].sum())
    sb = pb[2 * k:3 * k].sum() + float(lam @ pb[3 * k:3 * k + nc])
    return sa, sb


@pytest.mark.parametrize("name", ["coreg_tiny", "coreg_k2_small"])
def test_multivariate_scaling_identities(name):
    from oracle import dense
    from oracle import model as M
    p = workloads.make_problem(name)
    res = bta.evaluate(p)
    sa, sb = _coreg_scaling_sums(p, res)
    mdl = M.build_model(p)
    Z = np.linalg.inv(mdl.Qc.toarray())
    N = Z.shape[0]
    trzt = float(np.trace(Z[N - p.a:, N - p.a:]))
    assert abs(sa - (N - 1e-3 * trzt)) <= 1e-9 * N
    x = res.x
    nst = N - p.a
    xst = x[:nst]
    assert abs(sb - float(xst @ (mdl.Qst @ xst))) <= 1e-9 * abs(sb)
    # the same from the dense definition of every phase term
    d = dense.evaluate(p)
    sa2, sb2 = _coreg_scaling_sums(p, d)
    assert abs(sa2 - sa) <= 1e-9 * N and abs(sb2 - sb) <= 1e-9 * abs(sb)
