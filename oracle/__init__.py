"""FP64 CPU oracle for the INLA objective f(theta) and its gradient.

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is the independent reference the
GPU library is checked against; it shares no code with the library (no
kernels, headers, helpers or constants) and neither side imports the other.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The only module both sides use is the seeded
input generator ``workloads``, which holds none of the method's arithmetic.

Modules:
  * ``model``  -- sparse Q_p, Q_c, A, r and the exact dQ/dtheta_k
                  (Eq. 1, Section II-A/B, Eqs. 10-12).
  * ``dense``  -- the plain dense definition: Cholesky log-dets and
                  inverse-based Eq. 6 gradient (small N).
  * ``bta``    -- the block sweep: Algorithm 1, Eqs. 3-5, selected
                  inversion, Eq. 7 (Phases A and C) and Eq. 8 (Phase B).
  * ``fd``     -- central finite differences (Eq. 2) of either path.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms (spectral log-determinants of the Kronecker-structured prior),
brute force (dense inverse on tiny inputs), invariants and finite
differences.
"""
from . import model, dense, bta, fd  # noqa: F401
