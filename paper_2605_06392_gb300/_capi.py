"""ctypes declarations of the C ABI in ``include/bta.h`` (argument marshalling
only; every computation runs in ``libbta.so``).

The library is built in-tree by ``paper_2605_06392_gb300.build``.  Loading
fails loudly if it is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libbta.so")

BTA_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "matrix not positive definite",
          -3: "CUDA error", -4: "out of device memory", -5: "bounded device wait timed out",
          -6: "descriptor in the wrong state"}


class BtaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS.get(code, code)} ({code})")


class bta_desc(C.Structure):
    _fields_ = [("n", C.c_int32), ("b", C.c_int32), ("a", C.c_int32), ("ld", C.c_int32),
                ("D", C.c_void_p), ("B", C.c_void_p), ("C", C.c_void_p), ("T", C.c_void_p),
                ("state", C.c_int32)]


class inla_model_spec(C.Structure):
    _fields_ = [("k", C.c_int32), ("ns", C.c_int32), ("nt", C.c_int32), ("a", C.c_int32),
                ("nnz", C.c_int32),
                ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val_C", C.c_void_p), ("val_G", C.c_void_p), ("val_GG", C.c_void_p),
                ("m_diag", C.c_void_p), ("m_sub", C.c_void_p),
                ("n_obs", C.c_int64),
                ("obs_t", C.c_void_p), ("obs_s", C.c_void_p), ("obs_v", C.c_void_p),
                ("obs_cov", C.c_void_p), ("y", C.c_void_p),
                ("tip_prior", C.c_double), ("theta_prior_var", C.c_double),
                ("low_memory", C.c_int32)]


class inla_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("use_graph", C.c_int32), ("streams", C.c_int32),
                ("reserved", C.c_int32)]


# name -> (restype, argtypes); every symbol include/bta.h declares
SIGNATURES = {
    "bta_status_string": (C.c_char_p, [C.c_int]),
    "inla_model_create": (C.c_int, [C.POINTER(inla_model_spec), C.POINTER(C.c_void_p)]),
    "inla_model_destroy": (None, [C.c_void_p]),
    "inla_model_dims": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int32)] * 5),
    "bta_assemble": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                               C.POINTER(bta_desc), C.c_void_p, C.c_void_p]),
    "bta_factor": (C.c_int, [C.POINTER(bta_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_int32, C.c_void_p]),
    "bta_factor_noalloc": (C.c_int, [C.POINTER(bta_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "bta_solve": (C.c_int, [C.POINTER(bta_desc), C.c_void_p, C.c_int32, C.c_int32,
                            C.POINTER(bta_desc), C.c_void_p]),
    "bta_selinv": (C.c_int, [C.POINTER(bta_desc), C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                             C.c_void_p, C.c_void_p]),
    "inla_value_and_grad": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(inla_opts), C.c_void_p]),
    "inla_backward": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int32, C.c_void_p]),
    "inla_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "inla_batch_destroy": (None, [C.c_void_p]),
    "inla_batch_value_and_grad": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int32,
                                            C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.POINTER(inla_opts), C.c_void_p]),
    "inla_hessian": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double,
                               C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(inla_opts), C.c_void_p]),
    "inla_last_parts": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "inla_copy_mode": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "inla_kernel_launches": (C.c_int64, [C.c_void_p]),
    "bta_set_wait_limit": (C.c_int, [C.c_int64, C.c_int32]),
    "bta_pivot_reciprocals": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                        C.c_void_p]),
    "bta_gemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_void_p, C.c_int32,
                           C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                           C.c_int32, C.c_void_p]),
    "bta_gemm_mixed": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                 C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                 C.c_double, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "bta_gemm_emulated": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                    C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_int32,
                                    C.c_double, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                    C.c_void_p]),
    "bta_gemm_emulated_timed": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                          C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                          C.c_int32, C.c_int32, C.c_double, C.c_void_p,
                                          C.c_int32, C.c_int32, C.c_void_p,
                                          C.POINTER(C.c_float), C.c_void_p]),
    "inla_grid_stencil": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """Load libbta.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libbta.so not found at {LIB_PATH}; build it with "
                "`python -m paper_2605_06392_gb300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int, what: str):
    if code != BTA_OK:
        raise BtaError(code, what)
