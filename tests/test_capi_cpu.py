"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every function include/bta.h declares; host-only entry points work."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bta.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_06392_gb300 import build
    build.build()
    from paper_2605_06392_gb300 import _capi
    return _capi.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("bta_assemble", "bta_factor", "bta_solve", "bta_selinv", "inla_value_and_grad",
                 "inla_model_create", "inla_model_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2605_06392_gb300 import _capi
    names = _declared()
    assert names
    for n in names:
        assert hasattr(lib, n), n
        assert n in _capi.SIGNATURES, n


def test_status_strings(lib):
    assert lib.bta_status_string(0) == b"ok"
    assert b"positive definite" in lib.bta_status_string(-2)


def test_grid_stencil_host_only():
    import paper_2605_06392_gb300 as P
    row_ptr, col, vC, vG, vGG = P.grid_stencil(4, 3)
    ns = 12
    G = np.zeros((ns, ns))
    GG = np.zeros((ns, ns))
    I = np.zeros((ns, ns))
    for s in range(ns):
        for e in range(row_ptr[s], row_ptr[s + 1]):
            G[s, col[e]] = vG[e]
            GG[s, col[e]] = vGG[e]
            I[s, col[e]] = vC[e]
    np.testing.assert_array_equal(I, np.eye(ns))
    np.testing.assert_array_equal(G.sum(1), np.zeros(ns))       # Laplacian rows sum to 0
    np.testing.assert_array_equal(G, G.T)
    np.testing.assert_array_equal(GG, G @ G)
    assert np.all(np.diff(col[row_ptr[0]:row_ptr[1]]) > 0)       # sorted columns


def test_build_is_sm103a_only():
    from paper_2605_06392_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
