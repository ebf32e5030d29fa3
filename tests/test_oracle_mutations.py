"""Planted mistakes in the oracle must be caught by its pins.

Each test plants one plausible error in a copy of an oracle function (on
the CPU, via monkeypatch) and checks that the independent pin it targets
no longer holds.  This guards the pins themselves against being too weak.
"""
import numpy as np
import scipy.linalg as la

import workloads
from oracle import bta, dense, fd, model as M
from test_oracle_pins import _spectral_univariate


def test_wrong_laplacian_boundary_is_caught(monkeypatch):
    orig = M.grid_laplacian

    def dirichlet_like(nx, ny):
        G = orig(nx, ny).tolil()
        for s in range(nx * ny):
            G[s, s] = 4.0          # boundary degree not reduced
        return G.tocsr()
    monkeypatch.setattr(M, "grid_laplacian", dirichlet_like)
    p = workloads.make_problem("st_tiny")
    th = p.theta
    lam, _, _ = _spectral_univariate(p.nx, p.ny, p.nt, np.exp(th[0]), np.exp(th[1]), np.exp(th[2]))
    exact = float(np.sum(np.log(lam))) + p.a * np.log(1e-3)
    assert abs(bta.evaluate(p, grad=False).logdet_p - exact) > 1e-6 * abs(exact)


def test_dropped_selinv_term_is_caught(monkeypatch):
    def bad_selinv(F):
        n = F.n
        LTi = la.solve_triangular(F.LT, np.eye(F.a), lower=True)
        ZT = LTi.T @ LTi
        ZD, ZB, ZC = [None] * n, [None] * (n - 1), [None] * n
        for i in range(n - 1, -1, -1):
            Li = la.solve_triangular(F.LD[i], np.eye(F.b), lower=True)
            FC = F.LC[i] @ Li
            ZCi = -ZT @ FC
            if i < n - 1:
                FB = F.LB[i] @ Li
                ZCi = ZCi - ZC[i + 1] @ FB
                ZBi = -ZD[i + 1] @ FB          # arrow term dropped
                ZDi = Li.T @ Li - ZBi.T @ FB - ZCi.T @ FC
                ZB[i] = ZBi
            else:
                ZDi = Li.T @ Li - ZCi.T @ FC
            ZD[i], ZC[i] = ZDi, ZCi
        return bta.SelInv(ZD, ZB, ZC, ZT)
    p = workloads.make_problem("st_tiny")
    mdl = M.build_model(p)
    F = bta.factor(bta.extract(mdl.Qc, p.nt, p.b, p.a), mdl.r)
    Zd = np.linalg.inv(mdl.Qc.toarray())
    Z = bad_selinv(F)
    b = p.b
    assert not np.allclose(Z.ZD[0], Zd[:b, :b], rtol=1e-10, atol=1e-13)


def test_phase_b_factor_error_is_caught(monkeypatch):
    orig = bta.quad_eq8

    def half_offdiag(x, dQ, n, b):
        return 0.5 * (orig(x, dQ, n, b) + sum(
            float(x[i * b:(i + 1) * b] @ (dQ.tocsr()[i * b:(i + 1) * b, i * b:(i + 1) * b]
                                         @ x[i * b:(i + 1) * b])) for i in range(n)))
    monkeypatch.setattr(bta, "quad_eq8", half_offdiag)
    p = workloads.make_problem("st_tiny")
    g = bta.evaluate(p).grad
    gfd = fd.gradient(p, h=1e-5, path="dense")
    assert np.max(np.abs(g - gfd) / np.maximum(np.abs(gfd), 1.0)) > 1e-4


def test_model_blocks_match_neighbour_loop_construction():
    # D_t and B_t built from an explicit neighbour loop (not scipy kron):
    # D = s[(k^2 I + G)^2 + 4 k g (k^2 I + G) + I], B = -2 s k g (k^2 I + G)
    p = workloads.make_problem("st_tiny", nx=3, ny=4, nt=3, n_obs=50)
    nx, ny = p.nx, p.ny
    ns = nx * ny
    G = np.zeros((ns, ns))
    for iy in range(ny):
        for ix in range(nx):
            s = iy * nx + ix
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                jx, jy = ix + dx, iy + dy
                if 0 <= jx < nx and 0 <= jy < ny:
                    G[s, jy * nx + jx] -= 1.0
                    G[s, s] += 1.0
    s_, kap, gam = np.exp(p.theta[:3])
    K1 = kap ** 2 * np.eye(ns) + G
    D = s_ * (K1 @ K1 + 4 * kap * gam * K1 + np.eye(ns))
    B = -2 * s_ * kap * gam * K1
    blk = bta.extract(M.build_model(p).Qst, p.nt, ns, 0)
    for t in range(p.nt):
        np.testing.assert_allclose(blk.D[t], D, rtol=1e-13, atol=1e-12)
    for t in range(p.nt - 1):
        np.testing.assert_allclose(blk.B[t], B, rtol=1e-13, atol=1e-12)


def test_likelihood_normalisation_error_is_caught(monkeypatch):
    # n log tau in place of (n/2) log tau in log l (Eq. 1): the value and the
    # explicit gradient term both move, and both pins on log l see it
    from test_oracle_likelihood_pins import closed_form_gaps, loglik_density_gap, scalar_problem

    def doubled(model, x):
        val, grad = orig(model, x)
        prob, k = model.prob, model.prob.k
        for m in range(k):
            nm = int(np.sum(prob.obs_v == m))
            val += 0.5 * nm * np.log(model.par.tau[m])
            grad[grad.shape[0] - k + m] += 0.5 * nm
        return val, grad
    orig = M.log_lik
    monkeypatch.setattr(M, "log_lik", doubled)
    p = workloads.make_problem("coreg_tiny")
    gap, gerr = loglik_density_gap(p, np.zeros(p.N))
    assert gap > 1e-3 and gerr > 1e-3
    worst_val, worst_grad = closed_form_gaps(scalar_problem(1))
    assert worst_val > 1e-3 and worst_grad > 1e-3


def test_fixed_effect_column_offset_is_caught(monkeypatch):
    # the covariates of response v written into response (v + 1) mod k's
    # fixed-effect columns: the hand-typed projection pin fails
    from test_oracle_likelihood_pins import projection_gaps, two_response_problem
    import scipy.sparse as sp

    def shifted(prob):
        A = orig(prob).tolil()
        nb, ar, k = prob.nt * prob.b, prob.a_r, prob.k
        for j in range(prob.n_obs):
            v = int(prob.obs_v[j])
            for c in range(ar):
                A[j, nb + v * ar + c] = 0.0
                A[j, nb + ((v + 1) % k) * ar + c] = prob.obs_cov[j, c]
        return sp.csr_matrix(A)
    orig = M.projection
    monkeypatch.setattr(M, "projection", shifted)
    assert projection_gaps(two_response_problem()) > 0.1
