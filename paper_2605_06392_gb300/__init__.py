"""GB300-native INLA objective and exact gradient on BTA precision matrices.

The compute path is the CUDA library ``_lib/libbta.so`` (sources in
``csrc/``, C ABI in ``include/bta.h``); this package is its binding.
Import does not touch the GPU; the library is loaded on first use and a
missing build raises instead of falling back to anything else.
"""
from .api import (BtaMatrix, InlaBatch, InlaModel, bta_assemble, bta_factor, bta_gemm, bta_selinv,  # noqa: F401
                  bta_gemm_emulated,
                  bta_solve, grid_stencil, inla_value_and_grad, theta_dim)
from .autograd import InlaFn, inla_objective  # noqa: F401
