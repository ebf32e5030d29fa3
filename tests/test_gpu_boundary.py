"""The descriptor calls of the C ABI beyond FP64: bta_factor with precision
1 (split TF32) and 2 (emulated FP64), bta_solve with one refinement step
against the assembled matrix, the timeout status of a bounded device wait,
and the pivot reciprocals of the diagonal factor, against the FP64 oracle
and against CUDA's own functions.

Tolerances: FP64 and emulated FP64 relative 1e-10 (the FP64 bar); mixed
precision 1e-6 on the log-determinant (the bar on f) and 1e-4 on the solve
before refinement; after one FP64 refinement step the solve meets 1e-8.
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


def _oracle_factor(prob):
    from oracle import bta, model as M
    mdl = M.build_model(prob)
    blk = bta.extract(mdl.Qc, prob.nt, prob.b, prob.a)
    F = bta.factor(blk, mdl.r)
    return F, bta.upper_solve(F)


def _unpad(v, prob, ld):
    n, b = prob.nt, prob.b
    v = v.cpu().numpy()
    return np.concatenate([v[: n * ld].reshape(n, ld)[:, :b].reshape(-1), v[n * ld:]])


def _assembled(P, m, prob):
    import torch
    Q = m.new_matrix(1)
    r = torch.zeros(prob.nt * m.ld + prob.a, dtype=torch.float64, device="cuda")
    P.bta_assemble(m, prob.theta, 1, Q, r)
    return Q, r


# b = 64 (one task-graph leaf), b = 1024 (a split diagonal block in the
# tensor-core modes, every product on the tensor cores)
FACTOR_CASES = [("st_tiny", {}), ("st_medium_nt6", dict(nt=3, n_obs=4000))]


@pytest.mark.parametrize("name,over", FACTOR_CASES)
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_factor_precision_and_refined_solve(P, name, over, precision):
    import torch
    prob = workloads.make_problem(name, **over)
    m = P.InlaModel(prob)
    F, x_or = _oracle_factor(prob)
    Q, r = _assembled(P, m, prob)
    Qkeep, r0 = _assembled(P, m, prob)        # the assembled matrix for the refinement
    logdet, fail = P.bta_factor(Q, r, precision=precision)
    torch.cuda.synchronize()
    assert int(fail.item()) == -1 and Q.state == 2
    tol_ld = 1e-6 if precision == 1 else 1e-10
    assert abs(logdet.item() - F.logdet) <= tol_ld * abs(F.logdet)
    z_or = np.concatenate(F.z + [F.zT])
    z = _unpad(r, prob, m.ld)
    tol_z = 1e-4 if precision == 1 else 1e-10
    assert np.max(np.abs(z - z_or)) <= tol_z * np.max(np.abs(z_or))
    # plain solve from z, and the refined solve from r
    x = r.clone()
    P.bta_solve(Q, x)
    xr = r0.clone()
    P.bta_solve(Q, xr, lower=True, refine=True, Q=Qkeep)
    torch.cuda.synchronize()
    scale = np.max(np.abs(x_or))
    err_plain = np.max(np.abs(_unpad(x, prob, m.ld) - x_or)) / scale
    err_ref = np.max(np.abs(_unpad(xr, prob, m.ld) - x_or)) / scale
    assert err_plain <= (1e-4 if precision == 1 else 1e-10)
    assert err_ref <= (1e-8 if precision == 1 else 1e-10)
    if precision == 1:
        assert err_ref < 0.1 * err_plain            # the FP64 step reduces the error
    assert Qkeep.state == 1                          # read, not changed
    m.close()


def test_solve_refinement_argument_errors(P):
    import torch
    from paper_2605_06392_gb300._capi import BtaError
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    Q, r = _assembled(P, m, prob)
    Qkeep, _ = _assembled(P, m, prob)
    P.bta_factor(Q, r)
    x = r.clone()
    with pytest.raises(BtaError) as e:            # refinement needs r (lower = 1)
        P.bta_solve(Q, x, lower=False, refine=True, Q=Qkeep)
    assert e.value.code == -1
    with pytest.raises(BtaError) as e:            # ... and the assembled matrix
        P.bta_solve(Q, x, lower=True, refine=True, Q=None)
    assert e.value.code == -1
    with pytest.raises(BtaError) as e:            # the factor is not an assembled matrix
        P.bta_solve(Q, x, lower=True, refine=True, Q=Q)
    assert e.value.code in (-1, -6)
    with pytest.raises(BtaError) as e:            # precision out of range
        P.bta_factor(Qkeep, None, precision=3)
    assert e.value.code == -1
    assert Qkeep.state == 1
    torch.cuda.synchronize()
    m.close()


def test_bounded_wait_expiry_reports_timeout_and_model_stays_usable(P):
    """The task-graph factor's chain waits on a counter nothing sets (test
    switch) with a 20 ms bound: the factor reports BTA_ERR_TIMEOUT through
    bta_factor's failure word and inla_value_and_grad's status, no fault, and
    the same model then evaluates exactly as before.  FP64 model of 64-row
    blocks: the task graph is the only kernel that waits."""
    import torch
    from paper_2605_06392_gb300._capi import BtaError, check, lib
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    f0, g0 = m.value_and_grad(prob.theta, use_graph=False)
    try:
        check(lib().bta_set_wait_limit(20_000_000, 1), "bta_set_wait_limit")
        Q, r = _assembled(P, m, prob)
        _, fail = P.bta_factor(Q, r)
        torch.cuda.synchronize()
        assert int(fail.item()) == -5
        with pytest.raises(BtaError) as e:
            m.value_and_grad(prob.theta, use_graph=False)
        assert e.value.code == -5
    finally:
        check(lib().bta_set_wait_limit(0, 0), "bta_set_wait_limit")
    torch.cuda.synchronize()
    f1, g1 = m.value_and_grad(prob.theta, use_graph=False)
    f2, g2 = m.value_and_grad(prob.theta, use_graph=True)
    assert f1 == f0 and f2 == f0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(g2, g0)
    Q, r = _assembled(P, m, prob)
    _, fail = P.bta_factor(Q, r)
    torch.cuda.synchronize()
    assert int(fail.item()) == -1
    # the switch's limits are checked
    assert lib().bta_set_wait_limit(10, 0) == -1
    assert lib().bta_set_wait_limit(0, 2) == -1
    m.close()


def _edge_values():
    v = [1.0, 2.0, 0.5, 3.0, np.nextafter(2.0, 0.0), np.nextafter(1.0, 2.0), 1e-30, 1e30,
         2.0 ** -100, 2.0 ** -101, 2.0 ** 100, 2.0 ** 101, 2.0 ** -99 * 1.7, 2.0 ** 99 * 1.9,
         np.finfo(np.float64).tiny, 5e-324, 1e-310, 1e300, np.finfo(np.float64).max]
    return np.array(v + [-x for x in v])


def test_pivot_reciprocals_against_cuda(P):
    import ctypes as C
    import torch
    from paper_2605_06392_gb300._capi import check, lib
    rng = np.random.default_rng(3)
    rand = np.exp(rng.uniform(-230.0, 230.0, 200_000)) * rng.choice([-1.0, 1.0], 200_000)
    near = np.exp(rng.uniform(-2.0, 2.0, 50_000))      # the pivots' usual range
    v = torch.tensor(np.concatenate([_edge_values(), rand, near]), dtype=torch.float64,
                     device="cuda")
    rc = torch.empty_like(v)
    rq = torch.empty_like(v)
    check(lib().bta_pivot_reciprocals(C.c_void_p(v.data_ptr()), v.numel(),
                                      C.c_void_p(rc.data_ptr()), C.c_void_p(rq.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream)),
          "bta_pivot_reciprocals")
    torch.cuda.synchronize()
    want_r = 1.0 / v                                     # CUDA's division
    pos = v > 0
    want_q = torch.rsqrt(v[pos])                         # CUDA's rsqrt
    vv = v.abs()
    inside = (vv >= 2.0 ** -100) & (vv < 2.0 ** 101)
    # reciprocal: within 2^-52 relative in the seeded range, identical outside
    rel_r = ((rc - want_r).abs() / want_r.abs())[inside]
    assert float(rel_r.max()) <= 2.0 ** -52
    assert torch.equal(rc[~inside], want_r[~inside])
    # inverse square root: within 2^-51 relative of CUDA's rsqrt in the range
    inq = inside[pos]
    rel_q = ((rq[pos] - want_q).abs() / want_q)[inq]
    assert float(rel_q.max()) <= 2.0 ** -51
    outq = rq[pos][~inq]
    ref_out = 1.0 / torch.sqrt(v[pos][~inq])
    assert torch.equal(outq, ref_out)
    # non-positive arguments take 1 / sqrt: NaN for negatives
    assert bool(torch.isnan(rq[v < 0]).all())
