"""The oracle reproduces its stored fixtures (written by
tests/golden/make_golden.py from the oracle alone) through both of its
paths: the dense definition and the block sweep."""
import json
import os

import numpy as np
import pytest

import workloads
from oracle import bta, dense

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", ["st_tiny", "coreg_tiny", "coreg_k2_small"])
def test_golden(name):
    with open(os.path.join(HERE, f"{name}.json")) as fh:
        g = json.load(fh)
    p = workloads.make_problem(name)
    np.testing.assert_array_equal(p.theta, np.array(g["theta"]))
    for r in (dense.evaluate(p), bta.evaluate(p)):
        assert abs(r.f - g["f"]) <= 1e-12 * abs(g["f"])
        np.testing.assert_allclose(r.grad, g["grad"], rtol=1e-11, atol=1e-9)
        np.testing.assert_allclose(r.phase_a, g["phase_a"], rtol=1e-11, atol=1e-9)
