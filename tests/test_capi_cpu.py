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


def _valid_spec_arrays():
    import paper_2605_06392_gb300 as P
    row_ptr, col, vC, vG, vGG = P.grid_stencil(3, 2)
    keep = dict(row_ptr=row_ptr, col=col, vC=vC, vG=vG, vGG=vGG,
                mdiag=np.ones(6), msub=np.zeros(5), t=np.zeros(4, np.int32),
                s=np.arange(4, dtype=np.int32), v=np.zeros(4, np.int32), cov=np.zeros(8),
                y=np.ones(4))
    return keep


def _spec(keep, **over):
    import ctypes as C
    from paper_2605_06392_gb300 import _capi

    def ptr(a):
        return a.ctypes.data_as(C.c_void_p)
    f = dict(k=1, ns=6, nt=2, a=2, nnz=int(keep["col"].shape[0]), row_ptr=ptr(keep["row_ptr"]),
             col=ptr(keep["col"]), val_C=ptr(keep["vC"]), val_G=ptr(keep["vG"]),
             val_GG=ptr(keep["vGG"]), m_diag=ptr(keep["mdiag"]), m_sub=ptr(keep["msub"]),
             n_obs=4, obs_t=ptr(keep["t"]), obs_s=ptr(keep["s"]), obs_v=ptr(keep["v"]),
             obs_cov=ptr(keep["cov"]), y=ptr(keep["y"]), tip_prior=1e-3, theta_prior_var=100.0,
             low_memory=0)
    f.update(over)
    return _capi.inla_model_spec(**f)


@pytest.mark.parametrize("over", [
    dict(k=0), dict(k=5), dict(ns=0), dict(nt=0), dict(a=-1), dict(a=33),
    dict(k=2, ns=3, a=3),               # a must split evenly over the responses
    dict(nnz=0), dict(row_ptr=None), dict(m_sub=None), dict(n_obs=-1),
    dict(obs_cov=None), dict(y=None),
])
def test_model_spec_rejected_before_any_device_work(lib, over):
    """Invalid specs return BTA_ERR_ARG from the host checks, which run before
    the first device allocation (so this needs no GPU)."""
    import ctypes as C
    keep = _valid_spec_arrays()
    h = C.c_void_p()
    assert lib.inla_model_create(C.byref(_spec(keep, **over)), C.byref(h)) == -1
    assert not h.value


def test_model_spec_pattern_checks(lib):
    import ctypes as C
    keep = _valid_spec_arrays()
    h = C.c_void_p()
    bad = keep["col"].copy()
    bad[0] = 99                          # column outside the grid
    keep2 = dict(keep, col=bad)
    assert lib.inla_model_create(C.byref(_spec(keep2)), C.byref(h)) == -1
    nodiag = keep["col"].copy()
    r0, r1 = keep["row_ptr"][0], keep["row_ptr"][1]
    nodiag[r0:r1] = np.where(nodiag[r0:r1] == 0, 1, nodiag[r0:r1])   # row 0 loses its diagonal
    keep3 = dict(keep, col=nodiag)
    assert lib.inla_model_create(C.byref(_spec(keep3)), C.byref(h)) == -1
    assert lib.inla_model_create(None, C.byref(h)) == -1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the compiled library the binding raises; there is no other
    compute path to fall back to."""
    from paper_2605_06392_gb300 import _capi
    monkeypatch.setattr(_capi, "_lib", None)
    monkeypatch.setattr(_capi, "LIB_PATH", str(tmp_path / "absent" / "libbta.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _capi.lib()


def test_package_imports_without_touching_the_gpu():
    import subprocess
    import sys
    code = ("import sys, torch; import paper_2605_06392_gb300 as P; "
            "import paper_2605_06392_gb300.optimize; "
            "assert not torch.cuda.is_initialized(); "
            "assert 'oracle' not in sys.modules; print('ok')")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stderr[-2000:]
