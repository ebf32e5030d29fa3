"""Posterior Hessian from exact gradients (Eq. 13) and the L-BFGS driver.

* The Hessian's columns are central differences of the library's exact
  gradients; the oracle forms the same differences from its dense gradient,
  so the two agree to the gradients' parity divided by h.  H is symmetric up
  to the O(h^2) error of the differences.
* L-BFGS with batched line-search candidates reaches the same maximiser as
  SciPy's L-BFGS-B run on the oracle's dense objective and gradient.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06392_gb300 import build
    build.build()
    import paper_2605_06392_gb300 as P
    return P


@pytest.mark.parametrize("name", ["st_tiny", "coreg_k2_small"])
def test_hessian_matches_oracle_differences(P, name):
    from oracle import dense
    prob = workloads.make_problem(name)
    m = P.InlaModel(prob)
    h = 5e-3
    H, g0 = m.hessian(prob.theta, h=h, concurrent=4)
    d = prob.d
    Ho = np.zeros((d, d))
    for j in range(d):
        tp = prob.theta.copy(); tp[j] += h
        tm = prob.theta.copy(); tm[j] -= h
        Ho[:, j] = (dense.evaluate(prob, tp).grad - dense.evaluate(prob, tm).grad) / (2 * h)
    scale = np.max(np.abs(Ho))
    assert np.max(np.abs(H - Ho)) <= 1e-7 * scale
    # symmetric up to the O(h^2) truncation of the differences
    assert np.max(np.abs(H - H.T)) <= 1e-3 * scale
    np.testing.assert_allclose(g0, dense.evaluate(prob).grad, rtol=1e-9, atol=1e-7)


def test_lbfgs_reaches_the_oracle_maximiser(P):
    import scipy.optimize as so
    from oracle import dense
    from paper_2605_06392_gb300.optimize import lbfgs
    prob = workloads.make_problem("st_tiny", nx=6, ny=6, nt=3, n_obs=300)
    m = P.InlaModel(prob)
    theta0 = prob.theta + 0.3
    res = lbfgs(m, theta0, gtol=1e-7, max_iter=300)
    assert res.converged, res.history[-3:]

    def negf(t):
        r = dense.evaluate(prob, t)
        return -r.f, -r.grad
    ref = so.minimize(negf, theta0, jac=True, method="L-BFGS-B",
                      options={"gtol": 1e-10, "ftol": 1e-15, "maxiter": 1000})
    np.testing.assert_allclose(res.theta, ref.x, rtol=1e-4, atol=1e-4)
    assert abs(res.f + ref.fun) <= 1e-8 * abs(ref.fun)
