"""Diagonal-block factor split 2 x 2 recursively above a leaf size: the
task-graph kernel factors and inverts the leaves and each level's four
products run in FP64 (precision 0) or emulated FP64 (precisions 1 and 2).

The leaf sizes are read once per process from BTA_POTRF_LEAF_FP64 and
BTA_POTRF_LEAF_TC, so each case runs in a child process with small leaves
(32 to 256 rows) that force one to three recursion levels, including ragged
splits (192 rows into 96 + 96 and then 32 + 64).  Bar: the FP64 and
emulated-FP64 evaluations meet the FP64 bar against the oracle (relative
1e-10 on f, every gradient component and x*), the mixed mode its own
(1e-6 on f, 1e-4 per gradient component)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _launches(P, prob):
    """Kernels launched by one evaluation at each precision (default leaves)."""
    m = P.InlaModel(prob)
    out = {}
    for prec in (0, 1, 2):
        k0 = m.kernel_launches()
        m.value_and_grad(prob.theta, precision=prec)
        out[str(prec)] = m.kernel_launches() - k0
    m.close()
    return out


def _child(names):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import paper_2605_06392_gb300 as P
    import workloads
    out = {}
    for name in names:
        prob = workloads.make_problem(name)
        m = P.InlaModel(prob)
        res = {}
        for prec in (0, 1, 2):
            k0 = m.kernel_launches()
            f, g = m.value_and_grad(prob.theta, precision=prec)
            res[str(prec)] = {"f": f, "g": np.asarray(g).tolist(),
                              "x": m.mode().cpu().numpy().tolist(),
                              "launches": m.kernel_launches() - k0}
        m.close()
        out[name] = res
    print("RESULT " + json.dumps(out), flush=True)


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_06392_gb300 import build
    build.build()


@pytest.mark.gpu
@pytest.mark.parametrize("leaf,names", [
    (32, ["st_tiny", "coreg_tiny"]),
    (64, ["coreg_small"]),
    (256, ["st_medium_nt6"]),
])
def test_split_factor_against_oracle(built, leaf, names):
    from oracle import bta
    import workloads
    env = dict(os.environ, BTA_POTRF_LEAF_FP64=str(leaf), BTA_POTRF_LEAF_TC=str(leaf),
               PYTHONPATH=os.pathsep.join([ROOT, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, os.path.abspath(__file__)] + names, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    import paper_2605_06392_gb300 as P
    for name in names:
        prob = workloads.make_problem(name)
        whole = _launches(P, prob)
        o = bta.evaluate(prob)
        scale = np.maximum(np.abs(o.grad),
                           np.abs(o.phase_a) + np.abs(o.phase_b) + np.abs(o.phase_c))
        for prec, (tf, tg) in {"0": (1e-10, 1e-10), "1": (1e-6, 1e-4),
                               "2": (1e-10, 1e-10)}.items():
            v = res[name][prec]
            ef = abs(v["f"] - o.f) / abs(o.f)
            eg = float(np.max(np.abs(np.array(v["g"]) - o.grad) / scale))
            ex = float(np.max(np.abs(np.array(v["x"]) - o.x)) / np.max(np.abs(o.x)))
            assert ef <= tf and eg <= tg, (name, prec, ef, eg)
            assert ex <= (1e-10 if prec != "1" else 1e-8), (name, prec, ex)
            # the split path ran: more launches than the whole-block factor
            assert v["launches"] > whole[prec], (name, prec, v["launches"], whole[prec])


if __name__ == "__main__":
    _child(sys.argv[1:])
