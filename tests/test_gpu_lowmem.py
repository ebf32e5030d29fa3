"""Low-memory evaluations (the carry-based variant of Algorithm 1): only the
diagonal factors are kept between the forward and the reverse pass, and each
step that needs an off-diagonal factor re-assembles B_i and recomputes
L_Bi = B_i L_Di^{-T}.  Same bar as the FP64 path against the oracle (relative
1e-10 on f, every gradient component and x*), in FP64 and in emulated FP64;
agreement with the standard model; the mixed mode is refused; less device
memory."""
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


def _errs(P, prob, precision, low_memory=True):
    from oracle import bta
    m = P.InlaModel(prob, low_memory=low_memory)
    f, g = m.value_and_grad(prob.theta, precision=precision)
    x = m.mode().cpu().numpy()
    m.close()
    o = bta.evaluate(prob)
    scale = np.maximum(np.abs(o.grad), np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
    return (abs(f - o.f) / abs(o.f), float(np.max(np.abs(g - o.grad) / scale)),
            float(np.max(np.abs(x - o.x)) / np.max(np.abs(o.x))))


@pytest.mark.parametrize("name,over", [
    ("st_tiny", {}),
    ("coreg_tiny", {}),
    ("coreg_small", {}),
    ("st_tiny", dict(nt=1)),
    ("st_medium_nt6", {}),
])
def test_low_memory_fp64_against_oracle(P, name, over):
    ef, eg, ex = _errs(P, workloads.make_problem(name, **over), 0)
    assert ef <= 1e-10 and eg <= 1e-10 and ex <= 1e-10, (ef, eg, ex)


@pytest.mark.parametrize("name", ["coreg_small", "st_medium_nt6"])
def test_low_memory_emulated_against_oracle(P, name):
    ef, eg, ex = _errs(P, workloads.make_problem(name), 2)
    assert ef <= 1e-10 and eg <= 1e-10 and ex <= 1e-10, (ef, eg, ex)


def test_low_memory_matches_standard_model(P):
    prob = workloads.make_problem("coreg_small")
    out = []
    for low in (False, True):
        m = P.InlaModel(prob, low_memory=low)
        f, g = m.value_and_grad(prob.theta)
        # batched evaluations and the value-only / reverse split use the same sweeps
        fb, gb = m.value_and_grad(np.array([prob.theta, prob.theta * 0.9]), concurrent=2)
        out.append((f, g, fb, gb))
        m.close()
    (f0, g0, fb0, gb0), (f1, g1, fb1, gb1) = out
    assert abs(f1 - f0) <= 1e-12 * abs(f0)
    np.testing.assert_allclose(g1, g0, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(fb1, fb0, rtol=1e-12)
    np.testing.assert_allclose(gb1, gb0, rtol=1e-10, atol=1e-9)


def test_low_memory_refuses_mixed_mode(P):
    from paper_2605_06392_gb300._capi import BtaError
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob, low_memory=True)
    with pytest.raises(BtaError):
        m.value_and_grad(prob.theta, precision=1)
    f, _ = m.value_and_grad(prob.theta)          # the model stays usable
    assert np.isfinite(f)
    m.close()


def test_low_memory_value_then_backward(P):
    import torch
    prob = workloads.make_problem("coreg_tiny")
    m = P.InlaModel(prob, low_memory=True)
    f_ref, g_ref = m.value_and_grad(prob.theta)
    th = torch.tensor(prob.theta, dtype=torch.float64, requires_grad=True)
    y = P.inla_objective(th, m)
    y.backward()
    assert float(y.detach()) == f_ref
    np.testing.assert_array_equal(th.grad.numpy(), g_ref)
    m.close()


def test_low_memory_allocates_less(P):
    import torch
    prob = workloads.make_problem("st_medium_nt6")
    used = []
    for low in (False, True):
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        m = P.InlaModel(prob, low_memory=low)
        m.value_and_grad(prob.theta)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        used.append(free0 - free1)
        m.close()
    # two matrices x 5 B blocks of 1024^2 doubles, less two spare blocks
    saved = used[0] - used[1]
    assert saved >= 0.75 * (2 * 5 - 2) * 1024 * 1024 * 8, used
