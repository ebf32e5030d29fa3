"""Mixed-precision mode against the FP64 oracle.

The b x b off-diagonal Schur products and the selected-inversion products
run in split TF32 on the tensor cores (FP32 accumulation); the diagonal
factorisation, log-determinants and tip stay FP64 and x* gets one FP64
refinement step.  Tolerances: relative 1e-6 on f and 1e-4 on every gradient
component (cancellation-aware scale max(|g_k|, |A_k|+|B_k|+|C_k|)), and the
refined x* within 1e-8 of the oracle's (relative to max |x*|).
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


def _check(P, prob):
    from oracle import bta
    m = P.InlaModel(prob)
    f, g = m.value_and_grad(prob.theta, precision=1)
    x = m.mode().cpu().numpy()
    o = bta.evaluate(prob)
    scale = np.maximum(np.abs(o.grad), np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
    ef = abs(f - o.f) / abs(o.f)
    eg = np.max(np.abs(g - o.grad) / scale)
    ex = np.max(np.abs(x - o.x)) / np.max(np.abs(o.x))
    m.close()
    return ef, eg, ex


@pytest.mark.parametrize("name,over", [
    ("st_tiny", {}),
    ("coreg_tiny", {}),
    ("st_tiny", dict(nx=16, ny=12, nt=3, n_obs=700)),
])
def test_mixed_small(P, name, over):
    ef, eg, ex = _check(P, workloads.make_problem(name, **over))
    assert ef <= 1e-6 and eg <= 1e-4 and ex <= 1e-8, (ef, eg, ex)


def test_mixed_block_1024(P):
    ef, eg, ex = _check(P, workloads.make_problem("st_medium_nt6"))
    assert ef <= 1e-6 and eg <= 1e-4 and ex <= 1e-8, (ef, eg, ex)


def test_mixed_backward_split(P):
    import torch
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    f1, g1 = m.value_and_grad(prob.theta, precision=1)
    f0 = m.value(prob.theta)                     # FP64 value-only call
    fm, _ = m.value_and_grad(prob.theta, grad=False, precision=1)
    assert fm == f1
    assert abs(fm - f0) <= 1e-6 * abs(f0)
