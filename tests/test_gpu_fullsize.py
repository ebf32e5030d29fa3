"""GPU checks at the benchmark's full size, and on the large ragged-block
model, through the same entry point and launch configuration bench.py
times (inla_value_and_grad, CUDA graph, two sweep streams).

* 32x32 grid, b = 1024, 50 time blocks (the benchmark model): f and every
  gradient component against the oracle's block sweep (the oracle finishes
  it in well under a minute), log|Q_p| and all Phase C terms against the
  spectral closed form, and the mode's residual ||Q_c x - r|| / ||r||.
* 45x45 grid, b = 2025 (ld = 2048, a ragged tail), 100 time blocks: the
  closed forms and the residual, and the mixed-precision mode against the
  FP64 path (1e-6 on f, 1e-4 per gradient component).
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


def _spectral(prob):
    from test_oracle_pins import _spectral_univariate
    th = prob.theta
    lam, dk, dg = _spectral_univariate(prob.nx, prob.ny, prob.nt, np.exp(th[0]), np.exp(th[1]),
                                       np.exp(th[2]))
    ld = float(np.sum(np.log(lam))) + prob.a * np.log(1e-3)
    pc = np.array([0.5 * lam.size, 0.5 * np.sum(dk / lam), 0.5 * np.sum(dg / lam), 0.0])
    return ld, pc


def _residual(prob, x):
    from oracle import model as M
    mdl = M.build_model(prob)
    return np.linalg.norm(mdl.Qc @ x - mdl.r) / np.linalg.norm(mdl.r)


def test_benchmark_model_full_size(P):
    from oracle import bta
    prob = workloads.make_problem("st_medium")
    m = P.InlaModel(prob)
    f, g = m.value_and_grad(prob.theta)
    parts = m.last_parts()
    x = m.mode().cpu().numpy()
    ld, pc = _spectral(prob)
    assert abs(parts["logdet_p"] - ld) <= 1e-10 * abs(ld)
    np.testing.assert_allclose(parts["phase_c"], pc, rtol=1e-10, atol=1e-8)
    assert _residual(prob, x) < 1e-10
    o = bta.evaluate(prob)
    scale = np.maximum(np.abs(o.grad), np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
    assert abs(f - o.f) <= 1e-10 * abs(o.f)
    assert np.max(np.abs(g - o.grad) / scale) <= 1e-10
    m.close()


def test_large_ragged_model_fp64_and_mixed(P):
    prob = workloads.make_problem("st_large")
    m = P.InlaModel(prob)
    assert m.ld == 2048 and m.b == 2025
    f, g = m.value_and_grad(prob.theta)
    parts = m.last_parts()
    x = m.mode().cpu().numpy()
    ld, pc = _spectral(prob)
    assert abs(parts["logdet_p"] - ld) <= 1e-10 * abs(ld)
    np.testing.assert_allclose(parts["phase_c"], pc, rtol=1e-10, atol=1e-8)
    assert _residual(prob, x) < 1e-10
    fm, gm = m.value_and_grad(prob.theta, precision=1)
    pm = m.last_parts()
    xm = m.mode().cpu().numpy()
    scale = np.maximum(np.abs(g), np.abs(parts["phase_a"]) + np.abs(parts["phase_b"]) +
                       np.abs(parts["phase_c"]))
    assert abs(fm - f) <= 1e-6 * abs(f)
    assert np.max(np.abs(gm - g) / scale) <= 1e-4
    assert np.max(np.abs(xm - x)) <= 1e-8 * np.max(np.abs(x))
    assert _residual(prob, xm) < 1e-10
    np.testing.assert_allclose(pm["phase_c"], pc, rtol=1e-5, atol=1e-3)
    m.close()
