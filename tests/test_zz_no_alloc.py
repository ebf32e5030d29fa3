"""bta_factor_noalloc against bta_factor, through the C ABI.

bta_factor_noalloc serves callers that cannot allocate device memory during
the call (their device memory belongs to their own allocator or a fixed
budget, or they cannot take the synchronisation a free may bring).  It runs
the same factorisation out of a fixed scratch array the library reserves on
the device.  Here it must reproduce bta_factor's results (factor blocks, the
fused lower solve, the log-determinant, the failure flag) within the 1e-10
relative tolerance of the other GPU parity tests, on two calls in a row, must
refuse sizes beyond its stated limits, and once set up on the device must
leave the device's free memory and the stream-ordered memory pool untouched.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes as C

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


def _close(got, want):
    got = got.cpu().numpy()
    want = want.cpu().numpy()
    scale = max(np.abs(want).max(), 1e-300)
    np.testing.assert_allclose(got, want, rtol=RTOL, atol=RTOL * scale)


def _factor_noalloc(Q, rhs):
    import torch
    from paper_2605_06392_gb300._capi import check, lib
    logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
    fail = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    check(lib().bta_factor_noalloc(C.byref(Q.desc), C.c_void_p(rhs.data_ptr()),
                                   C.c_void_p(logdet.data_ptr()), C.c_void_p(fail.data_ptr()),
                                   stream), "bta_factor_noalloc")
    return logdet, fail


@pytest.mark.parametrize("over", [{}, dict(nx=12, ny=10, nt=4, n_obs=1500)])
def test_noalloc_factor_matches_bta_factor_twice(P, over):
    import torch
    prob = workloads.make_problem("st_tiny", **over)
    m = P.InlaModel(prob)
    n, a = prob.nt, prob.a
    # the existing entry point
    Qref = m.new_matrix(1)
    rref = torch.zeros(n * m.ld + a, dtype=torch.float64, device="cuda")
    P.bta_assemble(m, prob.theta, 1, Qref, rref)
    ld_ref, fail_ref = P.bta_factor(Qref, rref)
    torch.cuda.synchronize()
    assert int(fail_ref.item()) == -1
    for _ in range(2):       # two calls in a row share the fixed scratch
        Q = m.new_matrix(1)
        r = torch.zeros(n * m.ld + a, dtype=torch.float64, device="cuda")
        P.bta_assemble(m, prob.theta, 1, Q, r)
        logdet, fail = _factor_noalloc(Q, r)
        torch.cuda.synchronize()
        assert int(fail.item()) == int(fail_ref.item())
        assert abs(logdet.item() - ld_ref.item()) <= RTOL * abs(ld_ref.item())
        assert Q.state == 2
        _close(Q.D, Qref.D)
        _close(Q.B, Qref.B)
        _close(Q.C, Qref.C)
        _close(Q.T, Qref.T)
        _close(r, rref)
    m.close()


def test_noalloc_refuses_sizes_beyond_its_scratch(P):
    import torch
    from paper_2605_06392_gb300._capi import lib
    prob = workloads.make_problem("st_tiny", nx=17, ny=16, nt=2, n_obs=400)   # b=272 -> ld=288
    m = P.InlaModel(prob)
    Q = m.new_matrix(1)
    r = torch.zeros(prob.nt * m.ld + prob.a, dtype=torch.float64, device="cuda")
    P.bta_assemble(m, prob.theta, 1, Q, r)
    logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
    fail = torch.zeros(1, dtype=torch.int32, device="cuda")
    code = lib().bta_factor_noalloc(C.byref(Q.desc), C.c_void_p(r.data_ptr()),
                                    C.c_void_p(logdet.data_ptr()), C.c_void_p(fail.data_ptr()),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == -1
    assert Q.state == 1          # untouched: still assembled
    m.close()


def _pool_used_high(cu, pool):
    v = C.c_uint64(0)
    assert cu.cuMemPoolGetAttribute(pool, 8, C.byref(v)) == 0   # USED_MEM_HIGH
    return v.value


def _pool_reset_high(cu, pool):
    z = C.c_uint64(0)                                          # resets to the current use
    assert cu.cuMemPoolSetAttribute(pool, 8, C.byref(z)) == 0


def test_noalloc_call_allocates_nothing(P):
    """After a set-up call on the device, a call on a fresh model changes
    neither the device's free memory nor the high-water mark of the default
    memory pool (where cudaMallocAsync allocates).  bta_factor, which takes
    its workspace from that pool, moves the mark: the probe can see a
    stream-ordered allocation."""
    import torch
    cu = C.CDLL("libcuda.so.1")
    dev = C.c_int(0)
    assert cu.cuDeviceGet(C.byref(dev), torch.cuda.current_device()) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0

    def assembled(model, p):
        Q = model.new_matrix(1)
        r = torch.zeros(p.nt * model.ld + p.a, dtype=torch.float64, device="cuda")
        P.bta_assemble(model, p.theta, 1, Q, r)
        return Q, r
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    Q0, r0 = assembled(m, prob)
    _factor_noalloc(Q0, r0)                     # set-up call on this device
    torch.cuda.synchronize()
    prob2 = workloads.make_problem("st_tiny", seed=9)
    m2 = P.InlaModel(prob2)
    Qa, ra = assembled(m2, prob2)
    Q2, r2 = assembled(m2, prob2)
    torch.cuda.synchronize()
    _pool_reset_high(cu, pool)
    base = _pool_used_high(cu, pool)
    ld_ref, _ = P.bta_factor(Qa, ra)            # allocates its workspace from the pool
    torch.cuda.synchronize()
    assert _pool_used_high(cu, pool) > base
    _pool_reset_high(cu, pool)
    high0 = _pool_used_high(cu, pool)
    free0 = torch.cuda.mem_get_info()[0]
    logdet, fail = _factor_noalloc(Q2, r2)      # first call on the fresh model
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert _pool_used_high(cu, pool) == high0
    assert free1 == free0
    assert int(fail.item()) == -1
    assert abs(logdet.item() - ld_ref.item()) <= RTOL * abs(ld_ref.item())
    m2.close()
    m.close()


def test_noalloc_refuses_wide_arrow_and_too_many_slots(P):
    import torch
    from paper_2605_06392_gb300._capi import lib
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
    fail = torch.zeros(1, dtype=torch.int32, device="cuda")
    # a = 33 > 32 (no model allows it: the descriptor is built by hand)
    Q = P.BtaMatrix(1, 64, 33, 64)
    Q.desc.state = 1
    assert lib().bta_factor_noalloc(C.byref(Q.desc), None, C.c_void_p(logdet.data_ptr()),
                                    C.c_void_p(fail.data_ptr()), stream) == -1
    assert Q.state == 1
    # ld = 32: n * 1 + 1 = 16385 log-determinant slots, one beyond the limit
    Q = P.BtaMatrix(16384, 32, 0, 32)
    Q.desc.state = 1
    assert lib().bta_factor_noalloc(C.byref(Q.desc), None, C.c_void_p(logdet.data_ptr()),
                                    C.c_void_p(fail.data_ptr()), stream) == -1
    assert Q.state == 1
    torch.cuda.synchronize()
