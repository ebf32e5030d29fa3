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
* 3 x 40x40 grid, b = 4800, 192 time blocks, d = 15 (the production model),
  emulated FP64, both with the default sweeps (both factors kept) and with
  the low-memory ones: closed forms and identities.
* 31 coregionalised models of uneven block size (b = 768 / 1728 / 3072, 40
  time blocks, d = 15) as one CUDA graph in emulated FP64: every model bit for
  bit against its own single call, and against the same closed forms.
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


def test_large_ragged_model_all_precisions(P):
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
    # emulated FP64 (split diagonal factor: 2048 -> 1024-row task graphs with
    # emulated level products): the FP64 bar against the closed forms and the
    # FP64 path
    fe, ge = m.value_and_grad(prob.theta, precision=2)
    pe = m.last_parts()
    xe = m.mode().cpu().numpy()
    assert abs(pe["logdet_p"] - ld) <= 1e-10 * abs(ld)
    np.testing.assert_allclose(pe["phase_c"], pc, rtol=1e-10, atol=1e-8)
    assert abs(fe - f) <= 1e-10 * abs(f)
    assert np.max(np.abs(ge - g) / scale) <= 1e-10
    assert np.max(np.abs(xe - x)) <= 1e-10 * np.max(np.abs(x))
    m.close()


def test_blocks_above_task_graph_limit(P):
    """b = 5184 (72 x 72 grid, two time blocks): past the task graph's 160
    tile rows the diagonal factor takes the recursive launch sequence, and
    past K = 5120 the emulated products fall back to FP64.  Every mode
    against the oracle at its own bar."""
    from oracle import bta
    prob = workloads.make_problem("st_tiny", nx=72, ny=72, nt=2, n_obs=3000)
    o = bta.evaluate(prob)
    scale = np.maximum(np.abs(o.grad), np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
    m = P.InlaModel(prob)
    assert m.ld == 5184
    for prec, (tf, tg) in ((0, (1e-10, 1e-10)), (1, (1e-6, 1e-4)), (2, (1e-10, 1e-10))):
        f, g = m.value_and_grad(prob.theta, precision=prec)
        assert abs(f - o.f) <= tf * abs(o.f), (prec, f, o.f)
        assert np.max(np.abs(g - o.grad) / scale) <= tg, prec
    m.close()


def _coreg_closed_form_checks(prob, parts, x, tol=1e-10):
    """log|Q_p| and every Phase C term of a coregionalised model against the
    spectral closed form, and the two scaling identities of its prior (see
    test_oracle_pins), which tie the Phase A and Phase B terms of every scale
    and coupling parameter to N and x*'Q_st x*."""
    from test_oracle_pins import _coreg_scaling_sums, _spectral_univariate
    assert parts["fail_c"] < 0 and parts["fail_p"] < 0
    k, th = prob.k, prob.theta
    kap, gam, sig = np.exp(th[:k]), np.exp(th[k:2 * k]), np.exp(th[2 * k:3 * k])
    nst = prob.nt * prob.ns
    ld = -2.0 * nst * float(np.sum(np.log(sig))) + prob.a * np.log(1e-3)
    pc = np.zeros(prob.d)
    for v in range(k):
        lam, dk, dg = _spectral_univariate(prob.nx, prob.ny, prob.nt, 1.0, kap[v], gam[v])
        ld += float(np.sum(np.log(lam)))
        pc[v] = 0.5 * np.sum(dk / lam)
        pc[k + v] = 0.5 * np.sum(dg / lam)
        pc[2 * k + v] = -nst
    assert abs(parts["logdet_p"] - ld) <= tol * abs(ld)
    np.testing.assert_allclose(parts["phase_c"], pc, rtol=tol, atol=1e-6)

    class R:
        phase_a, phase_b = parts["phase_a"], parts["phase_b"]
    sa, sb = _coreg_scaling_sums(prob, R)
    N = prob.N
    # 0 <= 1e-3 tr(Z_T) <= a (the tip's Schur complement is at least 1e-3 I)
    assert N - prob.a - 1e-9 * N <= sa <= N + 1e-9 * N
    beta = x[N - prob.a:]
    xqx = parts["quad"] - 1e-3 * float(beta @ beta)
    assert abs(sb - xqx) <= tol * abs(xqx)


@pytest.mark.parametrize("low_memory", [False, True])
def test_production_model_emulated(P, low_memory):
    """Three coregionalised responses on a 40 x 40 grid, b = 4800, 192 time
    blocks, a = 12, d = 15, 2e6 observations, in the emulated-FP64 mode the
    benchmark times: with both factors kept (the default, ~141 GB of blocks)
    and with the low-memory sweeps (only the diagonal factors kept, ~71 GB).
    log|Q_p| and all 15 Phase C terms against the spectral closed form at the
    FP64 bar (1e-10), and the two scaling identities; the two sweeps agree
    with each other to 1e-10 on f and every gradient component."""
    import time
    import torch
    prob = workloads.make_problem("coreg_production")
    assert prob.b == 4800 and prob.nt == 192 and prob.d == 15
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    m = P.InlaModel(prob, low_memory=low_memory)
    t0 = time.perf_counter()
    f, g = m.value_and_grad(prob.theta, use_graph=False, precision=2)
    elapsed = time.perf_counter() - t0
    free1, _ = torch.cuda.mem_get_info()
    parts = m.last_parts()
    x = m.mode().cpu().numpy()
    m.close()
    used = (free0 - free1) / 2 ** 30
    print(f"production model, emulated FP64, low memory {low_memory}: {elapsed:.1f} s per "
          f"f + gradient, {used:.1f} GiB on the device")
    if low_memory:
        assert used < 90.0   # both factors kept whole would take > 131 GiB
    assert np.isfinite(f) and np.all(np.isfinite(g))
    _coreg_closed_form_checks(prob, parts, x)
    key = "low" if low_memory else "both"
    _PRODUCTION[key] = (f, np.asarray(g), parts)
    if len(_PRODUCTION) == 2:
        fb, gb, pb = _PRODUCTION["both"]
        fl, gl, _ = _PRODUCTION["low"]
        scale = np.maximum(np.abs(gb), np.abs(pb["phase_a"]) + np.abs(pb["phase_b"]) +
                           np.abs(pb["phase_c"]))
        assert abs(fl - fb) <= 1e-10 * abs(fb)
        assert np.max(np.abs(gl - gb) / scale) <= 1e-10


_PRODUCTION = {}


def test_31_coregionalised_models_one_graph(P):
    """The batched evaluation of 31 coregionalised models (3 responses, grid
    side drawn from 16 / 24 / 32, b = 768 / 1728 / 3072, 40 time blocks, a = 9,
    d = 15, 5e4 observations each, theta the FD stencil points around theta0)
    as one CUDA graph in emulated FP64: every f and gradient bit for bit equal
    to the model's own single call, and every model against its closed forms
    and scaling identities at the FP64 bar."""
    import time
    probs = workloads.make_batch(31)
    assert sorted({p.b for p in probs}) == [768, 1728, 3072]
    models = [P.InlaModel(p) for p in probs]
    singles = []
    for m, p in zip(models, probs):
        f, g = m.value_and_grad(p.theta, use_graph=False, precision=2)
        singles.append((f, np.asarray(g), m.last_parts(), m.mode().cpu().numpy()))
    batch = P.InlaBatch(models)
    t0 = time.perf_counter()
    fb, gb = batch.value_and_grad([p.theta for p in probs], precision=2)
    print(f"31 coregionalised models, one graph (capture included): "
          f"{time.perf_counter() - t0:.1f} s")
    for i, (p, (f, g, parts, x)) in enumerate(zip(probs, singles)):
        assert fb[i] == f, i
        np.testing.assert_array_equal(gb[i], g)
        _coreg_closed_form_checks(p, parts, x)
    batch.close()
    for m in models:
        m.close()
