"""Pins for the observation side of the oracle: the Gaussian log-likelihood
log l of Eq. 1 (Section II-A) and the projection A with r = tau A^T y.

Neither is checked by the spectral or selected-inversion pins: those see
only Q_p, and a wrong likelihood normalisation or a wrong fixed-effect
column moves the dense and the block oracle together.  The facts used here
come from outside the oracle:

* log l is the log-density of independent Gaussian observations with mean
  (A x)_j and precision tau of the row's response, so log l - (n/2) log 2 pi
  (log l omits that constant) equals the sum of ``scipy.stats.norm.logpdf``
  terms (a library routine for the textbook density), at any x and for every
  response separately.
* On a one-node, one-step model every matrix of Eq. 1 collapses to a scalar
  (a = 0) or a 2 x 2 matrix (a = 1): Q_p = s (kappa^4 + 4 kappa^3 gamma + 1)
  because C = 1, G = GG = 0, M0 = M2 = 1 and M1 = 2 there.  f is then written
  out by hand, its log-determinants, solve and likelihood included, and its
  gradient is checked by central differences of that hand-written f.
* A design of three observations on two responses with its projection
  matrix typed out entry by entry from the latent ordering (time-major,
  then variable, then grid node; the fixed effects of response v at columns
  n b + v a_r + c), and r and tau A^T A written from it by hand.
"""
import dataclasses

import numpy as np
import pytest
import scipy.stats as st

import workloads
from oracle import bta, dense, model as M

LOG2PI = np.log(2.0 * np.pi)


# ----------------------------------------------------------------------------
# log l against the Gaussian density
# ----------------------------------------------------------------------------
def loglik_density_gap(prob, x):
    """|log l(x) - (n/2) log 2 pi - sum_j log N(y_j; (A x)_j, 1/tau_j)| and the
    largest error of d log l / d log tau_m against central differences of
    the density sum with x held fixed; both relative to the value."""
    mdl = M.build_model(prob)
    val, grad = M.log_lik(mdl, x)
    mean = mdl.A @ x

    def density(log_tau):
        tau_row = np.exp(log_tau)[prob.obs_v]
        return float(np.sum(st.norm.logpdf(prob.y, loc=mean, scale=1.0 / np.sqrt(tau_row))))

    lt = np.log(mdl.par.tau)
    ref = density(lt)
    gap = abs(val - 0.5 * prob.n_obs * LOG2PI - ref) / abs(ref)
    k, d = prob.k, prob.d
    h = 1e-5
    gerr = 0.0
    for m in range(k):
        e = np.zeros(k)
        e[m] = h
        gfd = (density(lt + e) - density(lt - e)) / (2 * h)
        gerr = max(gerr, abs(grad[d - k + m] - gfd) / max(abs(gfd), 1.0))
    return gap, gerr


@pytest.mark.parametrize("name", ["st_tiny", "coreg_tiny", "coreg_k2_small"])
def test_loglik_is_the_gaussian_density(name):
    p = workloads.make_problem(name)
    x_star = dense.evaluate(p, grad=False).x
    x_rand = np.random.default_rng(7).standard_normal(p.N)
    for x in (x_star, x_rand):
        gap, gerr = loglik_density_gap(p, x)
        assert gap < 1e-12
        assert gerr < 1e-7


# ----------------------------------------------------------------------------
# one-node, one-step model written out by hand
# ----------------------------------------------------------------------------
def scalar_problem(a, seed=11):
    return workloads.make_problem("st_tiny", nx=1, ny=1, nt=1, a=a, n_obs=3, seed=seed,
                                  theta=[0.3, -0.2, 0.4, 1.1])


def scalar_closed_form(prob, theta):
    """f, x*, log|Q_p|, log|Q_c| and log l of Eq. 1 for the one-node model,
    from the definitions collapsed by hand (a = 0 or 1)."""
    s, kap, gam, tau = np.exp(theta)
    q = s * (kap ** 4 + 4 * kap ** 3 * gam + 1.0)    # Q_st: s [K0 + 2 k g M1 K1 + C]
    y = prob.y
    n = y.shape[0]
    if prob.a == 0:
        qc = q + tau * n                             # every row hits the node with weight 1
        x = np.array([tau * y.sum() / qc])
        ld_p, ld_c = np.log(q), np.log(qc)
        quad = q * x[0] ** 2
        mean = np.full(n, x[0])
    else:
        c = prob.obs_cov[:, 0]
        q11, q12, q22 = q + tau * n, tau * c.sum(), 1e-3 + tau * (c @ c)
        r1, r2 = tau * y.sum(), tau * (c @ y)
        det = q11 * q22 - q12 ** 2
        x = np.array([(q22 * r1 - q12 * r2) / det, (q11 * r2 - q12 * r1) / det])
        ld_p, ld_c = np.log(q) + np.log(1e-3), np.log(det)
        quad = q * x[0] ** 2 + 1e-3 * x[1] ** 2
        mean = x[0] + c * x[1]
    loglik = float(np.sum(st.norm.logpdf(y, loc=mean, scale=1.0 / np.sqrt(tau)))) + 0.5 * n * LOG2PI
    logp = -float(theta @ theta) / 200.0
    f = 0.5 * ld_p - 0.5 * ld_c - 0.5 * quad + loglik + logp
    return dict(f=f, x=x, ld_p=ld_p, ld_c=ld_c, loglik=loglik)


def closed_form_gaps(prob):
    """Largest relative gaps of the oracle (both paths) from the hand-written
    one-node model: values, and the gradient against central differences
    of the hand-written f."""
    th = prob.theta
    cf = scalar_closed_form(prob, th)
    h = 1e-5
    gfd = np.array([(scalar_closed_form(prob, th + h * e)["f"] -
                     scalar_closed_form(prob, th - h * e)["f"]) / (2 * h) for e in np.eye(4)])
    worst_val, worst_grad = 0.0, 0.0
    for r in (dense.evaluate(prob), bta.evaluate(prob)):
        for got, want in ((r.f, cf["f"]), (r.logdet_p, cf["ld_p"]), (r.logdet_c, cf["ld_c"]),
                          (r.loglik, cf["loglik"])):
            worst_val = max(worst_val, abs(got - want) / max(abs(want), 1.0))
        worst_val = max(worst_val, float(np.max(np.abs(r.x - cf["x"]) /
                                                np.maximum(np.abs(cf["x"]), 1e-3))))
        worst_grad = max(worst_grad, float(np.max(np.abs(r.grad - gfd) /
                                                  np.maximum(np.abs(gfd), 1.0))))
    return worst_val, worst_grad


@pytest.mark.parametrize("a", [0, 1])
def test_one_node_model_matches_hand_written_eq1(a):
    p = scalar_problem(a)
    assert p.b == 1 and p.nt == 1 and p.n_obs == 3
    worst_val, worst_grad = closed_form_gaps(p)
    assert worst_val < 1e-12
    assert worst_grad < 1e-7


# ----------------------------------------------------------------------------
# projection matrix of a two-response design, typed by hand
# ----------------------------------------------------------------------------
def two_response_problem():
    """k = 2 responses on a 2 x 1 grid, 2 time steps, one covariate per
    response (a = 2): b = 4, N = 10.  Rows (t, v, s, covariate, y)."""
    base = workloads.make_problem("coreg_k2_small", nx=2, ny=1, nt=2, a=2, n_obs=3)
    rows = [(1, 0, 1, 0.5, 1.0), (0, 1, 0, -2.0, 0.25), (1, 1, 1, 3.0, -1.5)]
    t, v, s, c, y = (np.array(col) for col in zip(*rows))
    return dataclasses.replace(
        base, obs_t=t.astype(np.int32), obs_v=v.astype(np.int32), obs_s=s.astype(np.int32),
        obs_cov=c.reshape(3, 1).astype(np.float64), y=y.astype(np.float64))


# latent index t*b + v*ns + s: rows hit 4+0+1 = 5, 0+2+0 = 2, 4+2+1 = 7;
# fixed effect of response v: column nt*b + v*a_r + 0 = 8 + v
HAND_A = np.zeros((3, 10))
HAND_A[0, 5], HAND_A[0, 8] = 1.0, 0.5
HAND_A[1, 2], HAND_A[1, 9] = 1.0, -2.0
HAND_A[2, 7], HAND_A[2, 9] = 1.0, 3.0


def projection_gaps(prob):
    """Largest gaps of A, r = sum_m tau_m A_m^T y_m and Q_c - Q_p =
    sum_m tau_m A_m^T A_m from their hand-written values."""
    mdl = M.build_model(prob)
    t0, t1 = mdl.par.tau
    r = np.zeros(10)
    r[5], r[8] = t0 * 1.0, t0 * 0.5 * 1.0
    r[2], r[7] = t1 * 0.25, t1 * -1.5
    r[9] = t1 * (-2.0 * 0.25 + 3.0 * -1.5)
    AtA = np.zeros((10, 10))
    for (i, j, val) in [(5, 5, t0), (8, 8, t0 * 0.25), (5, 8, t0 * 0.5),
                        (2, 2, t1), (7, 7, t1), (9, 9, t1 * (4.0 + 9.0)),
                        (2, 9, t1 * -2.0), (7, 9, t1 * 3.0)]:
        AtA[i, j] = AtA[j, i] = val
    ga = float(np.max(np.abs(mdl.A.toarray() - HAND_A)))
    gr = float(np.max(np.abs(mdl.r - r)))
    gq = float(np.max(np.abs((mdl.Qc - mdl.Qp).toarray() - AtA)))
    return max(ga, gr / max(t0, t1), gq / max(t0, t1))


def test_projection_of_a_two_response_design():
    p = two_response_problem()
    assert p.b == 4 and p.N == 10 and p.a_r == 1
    assert projection_gaps(p) < 1e-14


def test_two_response_design_block_oracle_matches_dense():
    # the hand-checked design also runs through both evaluation paths
    p = two_response_problem()
    d, b = dense.evaluate(p), bta.evaluate(p)
    assert abs(d.f - b.f) <= 1e-12 * abs(d.f)
    np.testing.assert_allclose(b.grad, d.grad, rtol=1e-10, atol=1e-10)
