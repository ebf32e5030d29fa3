"""Emulated-FP64 mode: the b x b products computed on the BF16 tensor cores
from base-128 digit slices of each operand (Ozaki splitting).

Pins of the GEMM itself: integer operands, whose product FP64 holds
exactly, must come out bit-exact (the slice products and the level sums are
exact by construction); random and wide-range operands must stay within
the splitting's error bound (slices + 4) 2^(-7 slices) K max_k|a_ik|
max_k|b_kn| (the truncated digits of both operands and the dropped pair
levels) plus FP64 rounding of the result and of the host reference.  The whole evaluation in this mode must meet
the FP64 path's bar against the oracle (relative 1e-10).
"""
import json
import os
import subprocess
import sys

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


def _run(P, A, B, C0, alpha, beta, transA, transB, slices):
    """Emulated product through the C ABI, and the operands as numpy
    matrices op(A) (M x K), op(B) (K x N), C0 (M x N)."""
    import torch
    Cd = C0.clone()
    st = P.bta_gemm_emulated(A, B, Cd, alpha=alpha, beta=beta, transA=transA, transB=transB,
                             slices=slices)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    a = A.cpu().numpy()
    b = B.cpu().numpy()
    opA = a if transA else a.T
    opB = b if transB else b.T
    return Cd.cpu().numpy().T, opA, opB, C0.cpu().numpy().T


def test_integer_operands_bit_exact(P):
    import torch
    g = torch.Generator().manual_seed(11)
    M, N, K = 256, 192, 1024
    A = torch.randint(-100, 101, (K, M), generator=g).double().cuda()
    B = torch.randint(-100, 101, (N, K), generator=g).double().cuda()
    C0 = torch.randint(-1000, 1001, (N, M), generator=g).double().cuda()
    C, opA, opB, c0 = _run(P, A, B, C0, -1.0, 1.0, False, False, 8)
    exact = c0 - opA.astype(np.int64) @ opB.astype(np.int64)   # integers, exact
    assert np.array_equal(C, exact.astype(np.float64))


@pytest.mark.parametrize("M,N,K,transA,transB,slices", [
    (1024, 1024, 1024, False, True, 8),
    (300, 200, 700, False, False, 8),
    (130, 70, 33, True, False, 8),
    (512, 256, 2048, True, True, 8),
    (256, 256, 1024, False, True, 7),
    (256, 256, 1024, False, True, 6),
])
def test_random_within_bound(P, M, N, K, transA, transB, slices):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((M, K) if transA else (K, M), generator=g, dtype=torch.float64)
    B = torch.randn((K, N) if transB else (N, K), generator=g, dtype=torch.float64)
    C0 = torch.randn((N, M), generator=g, dtype=torch.float64)
    C, opA, opB, c0 = _run(P, A.cuda(), B.cuda(), C0.cuda(), -1.0, 1.0, transA, transB, slices)
    ref = c0 - opA @ opB
    bound = ((slices + 4) * 2.0 ** (-7 * slices) * K * np.max(np.abs(opA), axis=1)[:, None]
             * np.max(np.abs(opB), axis=0)[None, :]
             + 4.0 * K * 2.0 ** -53 * (np.abs(opA) @ np.abs(opB) + np.abs(c0)))
    err = np.abs(C - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_wide_range_rows_and_columns(P):
    """Rows and columns spread over 12 orders of magnitude, entries inside a
    row over 6: each row/column keeps its own scale."""
    import torch
    rng = np.random.default_rng(5)
    M, N, K = 256, 128, 512
    opA = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-6, 6, (M, 1)) \
        * 10.0 ** rng.uniform(-3, 3, (M, K))
    opB = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-6, 6, (1, N)) \
        * 10.0 ** rng.uniform(-3, 3, (K, N))
    A = torch.from_numpy(np.ascontiguousarray(opA.T)).cuda()   # column-major M x K
    B = torch.from_numpy(np.ascontiguousarray(opB.T)).cuda()
    C0 = torch.zeros((N, M), dtype=torch.float64, device="cuda")
    C, _, _, _ = _run(P, A, B, C0, 1.0, 0.0, False, False, 8)
    ref = opA @ opB
    bound = (12.0 * 2.0 ** -56 * K * np.max(np.abs(opA), axis=1)[:, None]
             * np.max(np.abs(opB), axis=0)[None, :]
             + 4.0 * K * 2.0 ** -53 * (np.abs(opA) @ np.abs(opB)))
    assert np.all(np.abs(C - ref) <= bound)


def _eval(P, prob, precision):
    from oracle import bta
    m = P.InlaModel(prob)
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
    ("st_tiny", dict(nx=16, ny=12, nt=3, n_obs=700)),
    ("st_tiny", dict(a=0)),
    ("st_medium_nt6", {}),
])
def test_emulated_mode_meets_fp64_bar(P, name, over):
    ef, eg, ex = _eval(P, workloads.make_problem(name, **over), 2)
    assert ef <= 1e-10 and eg <= 1e-10 and ex <= 1e-10, (ef, eg, ex)


def test_emulated_mode_value_backward_split(P):
    prob = workloads.make_problem("st_tiny")
    m = P.InlaModel(prob)
    f1, g1 = m.value_and_grad(prob.theta, precision=2)
    fv, _ = m.value_and_grad(prob.theta, grad=False, precision=2)
    assert fv == f1
    m.close()


# ---- every GEMM kernel on every shape --------------------------------------
# The kernel (128 x 64 tiles; 128 x 128 tiles with split K; 256 x 128 tiles on
# CTA pairs with split K) is chosen from the shape; BTA_OZAKI_N128 and
# BTA_OZAKI_PAIR force it, read once per process, so each forced run is a
# child process that reports max(error / bound) per shape.
_SHAPES = [(1024, 1024, 1024, False, True), (300, 200, 700, False, False),
           (130, 70, 33, True, False), (512, 256, 2048, True, True),
           (256, 256, 5120, False, True), (640, 384, 1536, True, False)]


def _child_gemm():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import paper_2605_06392_gb300 as P
    out = []
    for M, N, K, ta, tb in _SHAPES:
        g = torch.Generator().manual_seed(M + 3 * N + 7 * K)
        A = torch.randn((M, K) if ta else (K, M), generator=g, dtype=torch.float64)
        B = torch.randn((K, N) if tb else (N, K), generator=g, dtype=torch.float64)
        C0 = torch.randn((N, M), generator=g, dtype=torch.float64)
        C, opA, opB, c0 = _run(P, A.cuda(), B.cuda(), C0.cuda(), -1.0, 1.0, ta, tb, 8)
        ref = c0 - opA @ opB
        bound = (12.0 * 2.0 ** -56 * K * np.max(np.abs(opA), axis=1)[:, None]
                 * np.max(np.abs(opB), axis=0)[None, :]
                 + 4.0 * K * 2.0 ** -53 * (np.abs(opA) @ np.abs(opB) + np.abs(c0)))
        out.append({"shape": [M, N, K], "ratio": float(np.max(np.abs(C - ref) / bound))})
    gi = torch.Generator().manual_seed(11)
    A = torch.randint(-100, 101, (1024, 384), generator=gi).double().cuda()
    B = torch.randint(-100, 101, (640, 1024), generator=gi).double().cuda()
    C0 = torch.randint(-1000, 1001, (640, 384), generator=gi).double().cuda()
    C, opA, opB, c0 = _run(P, A, B, C0, -1.0, 1.0, False, False, 8)
    exact = c0 - opA.astype(np.int64) @ opB.astype(np.int64)
    # whole evaluations (the sweeps' lower-triangle and triangular-operand products)
    evals = {}
    for name in ("st_tiny", "coreg_small"):
        prob = workloads.make_problem(name)
        m = P.InlaModel(prob)
        f, gr = m.value_and_grad(prob.theta, precision=2)
        evals[name] = {"f": f, "g": np.asarray(gr).tolist(),
                       "x": m.mode().cpu().numpy().tolist()}
        m.close()
    print("RESULT " + json.dumps({"shapes": out, "evals": evals,
                                  "integer_exact": bool(np.array_equal(C, exact.astype(np.float64)))}),
          flush=True)


@pytest.mark.parametrize("force", [
    {"BTA_OZAKI_N128": "0", "BTA_OZAKI_PAIR": "0"},     # 128 x 64 tiles
    {"BTA_OZAKI_N128": "1", "BTA_OZAKI_PAIR": "0"},     # 128 x 128 tiles, one CTA
    {"BTA_OZAKI_N128": "1", "BTA_OZAKI_PAIR": "1"},     # 256 x 128 tiles, CTA pairs
], ids=["n64", "n128", "pair"])
def test_every_kernel_within_bound(P, force):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **force,
               PYTHONPATH=os.pathsep.join([root, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1][7:])
    assert res["integer_exact"]
    for v in res["shapes"]:
        assert v["ratio"] <= 1.0, v
    from oracle import bta
    for name, v in res["evals"].items():
        o = bta.evaluate(workloads.make_problem(name))
        scale = np.maximum(np.abs(o.grad),
                           np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
        assert abs(v["f"] - o.f) <= 1e-10 * abs(o.f), name
        assert np.max(np.abs(np.array(v["g"]) - o.grad) / scale) <= 1e-10, name
        assert np.max(np.abs(np.array(v["x"]) - o.x)) <= 1e-10 * np.max(np.abs(o.x)), name


if __name__ == "__main__":
    _child_gemm()


@pytest.mark.parametrize("precision", [2, 1])
def test_concurrent_thetas_equal_single_calls(P, precision):
    """Three thetas evaluated as one concurrent group (every block step one
    launch over the three matrices, the 1024-row diagonal blocks split over
    512-row task graphs with per-matrix level products) give the bits of
    three single evaluations."""
    prob = workloads.make_problem("st_medium_nt6")
    m = P.InlaModel(prob)
    thetas = np.array([prob.theta, prob.theta + 0.05, prob.theta - 0.05])
    singles = [m.value_and_grad(t, precision=precision) for t in thetas]
    f, g = m.value_and_grad(thetas, concurrent=3, precision=precision)
    for i in range(3):
        assert f[i] == singles[i][0]
        np.testing.assert_array_equal(g[i], singles[i][1])
    m.close()
