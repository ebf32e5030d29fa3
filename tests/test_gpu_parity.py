"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerance for the FP64 path: relative 1e-10 on f, log-determinants, x*,
selected-inverse blocks and every gradient component (scaled by
max(|g_k|, |Phase A_k| + |Phase B_k| + |Phase C_k|), the cancellation-aware
scale, since a gradient component is a small difference of large phases).
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06392_gb300 import build
    build.build()
    import paper_2605_06392_gb300 as P
    return P


def _oracle(prob, grad=True):
    from oracle import bta
    return bta.evaluate(prob, grad=grad)


def _grad_scale(o):
    return np.maximum(np.abs(o.grad), np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))


CASES = [
    ("st_tiny", {}),                                              # b=64: two leaf tiles
    ("st_tiny", dict(nx=10, ny=9, nt=5, n_obs=900)),              # b=90 -> ld=96, ragged
    ("st_tiny", dict(nx=16, ny=12, nt=3, n_obs=700)),             # b=192: 6 tiles, odd split
    ("st_tiny", dict(nt=1, n_obs=100)),                           # a single time block
    ("st_tiny", dict(a=0)),                                       # no fixed effects: no arrow
    ("st_tiny", dict(n_obs=0)),                                   # no observations: Q_c = Q_p
    ("st_tiny", dict(nx=1, ny=1)),                                # b = 1 padded to 32
    ("st_tiny", dict(nx=3, ny=1, nt=2, n_obs=30)),                # a 1-D grid, b = 3
    ("coreg_tiny", dict(n_obs=0)),
    ("coreg_tiny", {}),                                           # k=3, b=48 -> 64
    ("coreg_k2_small", {}),                                       # k=2, b=60 -> 64
    ("coreg_small", dict(nt=3, n_obs=1200)),                      # k=3, b=192
]


@pytest.mark.parametrize("name,over", CASES)
def test_value_and_grad_matches_oracle(P, name, over):
    prob = workloads.make_problem(name, **over)
    m = P.InlaModel(prob)
    f, g = m.value_and_grad(prob.theta)
    parts = m.last_parts()
    o = _oracle(prob)
    assert abs(f - o.f) <= RTOL * abs(o.f)
    assert abs(parts["logdet_c"] - o.logdet_c) <= RTOL * abs(o.logdet_c)
    assert abs(parts["logdet_p"] - o.logdet_p) <= RTOL * abs(o.logdet_p)
    assert abs(parts["quad"] - o.quad) <= RTOL * abs(o.quad)
    scale = _grad_scale(o)
    assert np.max(np.abs(g - o.grad) / scale) <= RTOL, (g, o.grad)
    for key in ("phase_a", "phase_b", "phase_c", "explicit"):
        np.testing.assert_allclose(parts[key], getattr(o, key), rtol=RTOL,
                                   atol=RTOL * scale.max())
    x = m.mode().cpu().numpy()
    np.testing.assert_allclose(x, o.x, rtol=RTOL, atol=RTOL * np.abs(o.x).max())
    m.close()


def test_value_only_and_backward_split(P):
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    f_full, g_full = m.value_and_grad(prob.theta)
    f_val = m.value(prob.theta)
    assert f_val == f_full
    import torch
    th = torch.tensor(prob.theta, requires_grad=True)
    y = P.inla_objective(th, m)
    y.backward()
    np.testing.assert_array_equal(th.grad.numpy(), g_full)
    assert float(y) == f_full


def test_deterministic_and_graph_equals_eager(P):
    prob = workloads.make_problem("coreg_tiny")
    m = P.InlaModel(prob)
    r1 = m.value_and_grad(prob.theta, use_graph=True)
    r2 = m.value_and_grad(prob.theta, use_graph=True)
    r3 = m.value_and_grad(prob.theta, use_graph=False)
    assert r1[0] == r2[0] == r3[0]
    np.testing.assert_array_equal(r1[1], r2[1])
    np.testing.assert_array_equal(r1[1], r3[1])


def test_batch_of_thetas_equals_single_calls(P):
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    pts = workloads.fd_stencil(prob.theta, 1e-3)
    fb, gb = m.value_and_grad(pts)
    for i in range(pts.shape[0]):
        f, g = m.value_and_grad(pts[i])
        assert f == fb[i]
        np.testing.assert_array_equal(g, gb[i])


@pytest.mark.parametrize("name", ["st_tiny", "coreg_tiny"])
def test_concurrent_batch_equals_single_calls(P, name):
    # A batch evaluated together (all matrices in the same launches) gives the
    # same bits as one theta at a time: each product accumulates over k in
    # the same order whatever the tile shape the batch size selects.
    prob = workloads.make_problem(name)
    m = P.InlaModel(prob)
    pts = workloads.fd_stencil(prob.theta, 1e-3)
    for grad in (True, False):
        fb, gb = m.value_and_grad(pts, grad=grad, concurrent=5)
        for i in range(pts.shape[0]):
            f, g = m.value_and_grad(pts[i], grad=grad)
            assert f == fb[i]
            if grad:
                np.testing.assert_array_equal(g, gb[i])


def test_gradient_matches_gpu_central_fd(P):
    prob = workloads.make_problem("coreg_k2_small")
    m = P.InlaModel(prob)
    f, g = m.value_and_grad(prob.theta)
    h = 1e-5
    pts = workloads.fd_stencil(prob.theta, h)
    fv, _ = m.value_and_grad(pts, grad=False)
    gfd = (fv[1::2] - fv[2::2]) / (2 * h)
    assert np.max(np.abs(g - gfd) / np.maximum(np.abs(g), 1.0)) < 1e-6


def test_autograd_gradcheck(P):
    import torch
    prob = workloads.make_problem("st_tiny", nx=4, ny=4, nt=3, n_obs=80)
    m = P.InlaModel(prob)
    th = torch.tensor(prob.theta, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: P.inla_objective(t, m), (th,), eps=1e-6,
                                    atol=1e-5, rtol=1e-6)


def test_primitives_against_oracle_blocks(P):
    import torch
    from oracle import bta, model as M
    prob = workloads.make_problem("st_tiny", nx=12, ny=10, nt=4, n_obs=1500)   # b=120, ld=128
    m = P.InlaModel(prob)
    n, b, a = prob.nt, prob.b, prob.a
    mdl = M.build_model(prob)
    blk = bta.extract(mdl.Qc, n, b, a)
    Q = m.new_matrix(1)
    rhs = torch.zeros(n * m.ld + a, dtype=torch.float64, device="cuda")
    P.bta_assemble(m, prob.theta, 1, Q, rhs)
    torch.cuda.synchronize()
    for i in range(n):
        np.testing.assert_allclose(Q.block_D(i).cpu().numpy(), blk.D[i], rtol=1e-14, atol=1e-12)
        np.testing.assert_allclose(Q.block_C(i).cpu().numpy(), blk.C[i], rtol=1e-14, atol=1e-12)
        if i < n - 1:
            np.testing.assert_allclose(Q.block_B(i).cpu().numpy(), blk.B[i], rtol=1e-14,
                                       atol=1e-12)
    np.testing.assert_allclose(Q.tip().cpu().numpy(), blk.T, rtol=1e-14, atol=1e-12)
    # padding: identity on D, zero on B and C
    Dp = Q.D[0].T.cpu().numpy()
    np.testing.assert_array_equal(Dp[b:, b:], np.eye(m.ld - b))
    np.testing.assert_array_equal(Dp[:b, b:], 0)
    r_lat = rhs[: n * m.ld].view(n, m.ld)[:, :b].reshape(-1)
    r = torch.cat([r_lat, rhs[n * m.ld:]]).cpu().numpy()
    np.testing.assert_allclose(r, mdl.r, rtol=1e-13, atol=1e-12)
    # factor + fused lower solve
    F = bta.factor(blk, mdl.r)
    logdet, fail = P.bta_factor(Q, rhs)
    torch.cuda.synchronize()
    assert int(fail.item()) == -1
    assert abs(logdet.item() - F.logdet) <= RTOL * abs(F.logdet)
    import scipy.linalg as la
    for i in range(n):
        Linv = la.solve_triangular(F.LD[i], np.eye(b), lower=True)
        got = np.tril(Q.block_D(i).cpu().numpy())
        np.testing.assert_allclose(got, Linv, rtol=1e-9, atol=1e-11 * np.abs(Linv).max())
        np.testing.assert_allclose(Q.block_C(i).cpu().numpy(), F.LC[i], rtol=1e-9,
                                   atol=1e-11 * np.abs(F.LC[i]).max())
        if i < n - 1:
            np.testing.assert_allclose(Q.block_B(i).cpu().numpy(), F.LB[i], rtol=1e-9,
                                       atol=1e-11 * np.abs(F.LB[i]).max())
    z_lat = rhs[: n * m.ld].view(n, m.ld)[:, :b].reshape(-1)
    z = torch.cat([z_lat, rhs[n * m.ld:]]).cpu().numpy()
    np.testing.assert_allclose(z, bta.join_vec(F.z, F.zT), rtol=1e-10, atol=1e-10)
    # upper solve
    P.bta_solve(Q, rhs)
    x_lat = rhs[: n * m.ld].view(n, m.ld)[:, :b].reshape(-1)
    x = torch.cat([x_lat, rhs[n * m.ld:]]).cpu().numpy()
    xo = bta.upper_solve(F)
    np.testing.assert_allclose(x, xo, rtol=RTOL, atol=RTOL * np.abs(xo).max())
    # selected inversion with fused traces
    Z = bta.selinv(F)
    tr = P.bta_selinv(Q, m, prob.theta, 1).cpu().numpy()
    for i in range(n):
        np.testing.assert_allclose(Q.block_D(i).cpu().numpy(), Z.ZD[i], rtol=RTOL,
                                   atol=RTOL * np.abs(Z.ZD[i]).max())
        np.testing.assert_allclose(Q.block_C(i).cpu().numpy(), Z.ZC[i], rtol=RTOL,
                                   atol=RTOL * np.abs(Z.ZC[i]).max())
        if i < n - 1:
            np.testing.assert_allclose(Q.block_B(i).cpu().numpy(), Z.ZB[i], rtol=RTOL,
                                       atol=RTOL * np.abs(Z.ZB[i]).max())
    np.testing.assert_allclose(Q.tip().cpu().numpy(), Z.ZT, rtol=RTOL)
    tro = np.array([bta.trace_eq7(Z, mdl.dQc[j], n, b, a) for j in range(prob.d)])
    np.testing.assert_allclose(tr, tro, rtol=RTOL, atol=RTOL * np.abs(tro).max())
    assert Q.state == 3


def test_prior_factor_and_phase_c_traces(P):
    import torch
    from oracle import bta, model as M
    prob = workloads.make_problem("coreg_tiny")
    m = P.InlaModel(prob)
    mdl = M.build_model(prob)
    n, b = prob.nt, prob.b
    Fp = bta.factor(bta.extract(mdl.Qst, n, b, 0))
    Zp = bta.selinv(Fp)
    Q = m.new_matrix(0)
    P.bta_assemble(m, prob.theta, 0, Q)
    logdet, fail = P.bta_factor(Q)
    tr = P.bta_selinv(Q, m, prob.theta, 0).cpu().numpy()
    torch.cuda.synchronize()
    assert abs(logdet.item() - Fp.logdet) <= RTOL * abs(Fp.logdet)
    tro = np.array([bta.trace_eq7(Zp, mdl.dQp[j][:n * b, :n * b], n, b, 0)
                    for j in range(prob.d)])
    np.testing.assert_allclose(tr, tro, rtol=RTOL, atol=RTOL * np.abs(tro).max())


def test_not_spd_is_reported_without_trapping(P):
    import torch
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    Q = m.new_matrix(1)
    P.bta_assemble(m, prob.theta, 1, Q)
    Q.D[2, 5, 5] = -1.0            # make the third diagonal block indefinite
    logdet, fail = P.bta_factor(Q)
    torch.cuda.synchronize()
    assert int(fail.item()) == 2
    # the model and the context stay usable
    f, g = m.value_and_grad(prob.theta)
    assert np.isfinite(f) and np.all(np.isfinite(g))


def test_argument_and_state_errors(P):
    from paper_2605_06392_gb300._capi import BtaError
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    bad = prob.theta.copy()
    bad[1] = np.nan
    with pytest.raises(BtaError) as e:
        m.value_and_grad(bad)
    assert e.value.code == -1
    Q = m.new_matrix(1)
    with pytest.raises(BtaError) as e:
        P.bta_factor(Q)                 # not assembled
    assert e.value.code == -6
    import torch
    with pytest.raises(BtaError) as e:
        P.bta_solve(Q, torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.code == -6
    import ctypes as C
    from paper_2605_06392_gb300._capi import lib
    g = np.zeros(prob.d)
    m.value_and_grad(prob.theta)        # full evaluation consumes nothing but leaves no factors
    assert lib().inla_backward(m.handle, g.ctypes.data_as(C.POINTER(C.c_double)), 1, None) == -6


@pytest.mark.parametrize("name", ["st_medium_nt6"])
def test_multi_tile_block_1024(P, name):
    # b = 1024: 32 leaf tiles per diagonal block, full-size blocks of the
    # benchmark model on a shortened time axis.
    prob = workloads.make_problem(name)
    m = P.InlaModel(prob)
    f, g = m.value_and_grad(prob.theta)
    o = _oracle(prob)
    assert abs(f - o.f) <= RTOL * abs(o.f)
    assert np.max(np.abs(g - o.grad) / _grad_scale(o)) <= RTOL


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_multi_model_single_graph_batch(P, precision):
    # models of uneven block size (b = 64, 120, 48 -> ld 64, 128, 64) in one graph
    probs = [workloads.make_problem("st_tiny"),
             workloads.make_problem("st_tiny", nx=12, ny=10, nt=3, n_obs=600, seed=9),
             workloads.make_problem("coreg_tiny")]
    models = [P.InlaModel(p) for p in probs]
    singles = [m.value_and_grad(p.theta, precision=precision) for m, p in zip(models, probs)]
    batch = P.InlaBatch(models)
    for _ in range(2):    # captured on the first call, replayed on the second
        f, g = batch.value_and_grad([p.theta for p in probs], precision=precision)
        for i in range(len(probs)):
            assert f[i] == singles[i][0]
            np.testing.assert_array_equal(g[i], singles[i][1])
    fv, _ = batch.value_and_grad([p.theta for p in probs], grad=False, precision=precision)
    np.testing.assert_array_equal(fv, f)
    if precision != 1:   # FP64 and emulated FP64 meet the FP64 bar
        for i, p in enumerate(probs):
            o = _oracle(p)
            assert abs(f[i] - o.f) <= RTOL * abs(o.f)
    batch.close()
