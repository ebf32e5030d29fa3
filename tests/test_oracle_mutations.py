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
