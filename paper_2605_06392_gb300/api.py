"""Python binding of the C ABI (argument marshalling only).

PyTorch provides device memory and streams; every step of the objective
and gradient runs in ``libbta.so``'s CUDA kernels.  Function names follow
``include/bta.h``: ``bta_assemble``, ``bta_factor``, ``bta_solve``,
``bta_selinv``, ``inla_value_and_grad``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _capi
from ._capi import bta_desc, check, inla_model_spec, inla_opts, lib

__all__ = ["InlaModel", "InlaBatch", "BtaMatrix", "bta_assemble", "bta_factor", "bta_solve", "bta_selinv",
           "inla_value_and_grad", "grid_stencil", "theta_dim", "bta_gemm"]


def theta_dim(k: int) -> int:
    return 4 * k + k * (k - 1) // 2


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def grid_stencil(nx: int, ny: int):
    """CSR (row_ptr, col, val_C, val_G, val_GG) of the grid's base matrices,
    built by the library (inla_grid_stencil)."""
    L = lib()
    nnz = C.c_int32(0)
    check(L.inla_grid_stencil(nx, ny, C.byref(nnz), None, None, None, None, None),
          "inla_grid_stencil")
    ns = nx * ny
    row_ptr = np.zeros(ns + 1, np.int32)
    col = np.zeros(nnz.value, np.int32)
    vals = [np.zeros(nnz.value) for _ in range(3)]
    check(L.inla_grid_stencil(nx, ny, C.byref(nnz), _ptr(row_ptr), _ptr(col), _ptr(vals[0]),
                              _ptr(vals[1]), _ptr(vals[2])), "inla_grid_stencil")
    return row_ptr, col, vals[0], vals[1], vals[2]


def _temporal(nt: int):
    """Tridiagonal M0 = I, M1 = tridiag(-1, 2, -1), M2 = I as (diag, sub)."""
    diag = np.concatenate([np.ones(nt), np.full(nt, 2.0), np.ones(nt)])
    sub = np.concatenate([np.zeros(nt - 1), -np.ones(nt - 1), np.zeros(nt - 1)])
    return np.ascontiguousarray(diag), np.ascontiguousarray(sub if nt > 1 else np.zeros(1))


class InlaModel:
    """A model on the current CUDA device (inla_model_create)."""

    def __init__(self, prob, tip_prior: float = 1e-3, theta_prior_var: float = 100.0,
                 low_memory: bool = False):
        L = lib()
        self.prob = prob
        row_ptr, col, vC, vG, vGG = grid_stencil(prob.nx, prob.ny)
        mdiag, msub = _temporal(prob.nt)
        self._keep = [row_ptr, col, vC, vG, vGG, mdiag, msub]
        obs_t = np.ascontiguousarray(prob.obs_t, dtype=np.int32)
        obs_s = np.ascontiguousarray(prob.obs_s, dtype=np.int32)
        obs_v = np.ascontiguousarray(prob.obs_v, dtype=np.int32)
        cov = np.ascontiguousarray(prob.obs_cov, dtype=np.float64)
        y = np.ascontiguousarray(prob.y, dtype=np.float64)
        self._keep += [obs_t, obs_s, obs_v, cov, y]
        spec = inla_model_spec(
            k=prob.k, ns=prob.ns, nt=prob.nt, a=prob.a, nnz=int(col.shape[0]),
            row_ptr=_ptr(row_ptr), col=_ptr(col), val_C=_ptr(vC), val_G=_ptr(vG),
            val_GG=_ptr(vGG), m_diag=_ptr(mdiag), m_sub=_ptr(msub), n_obs=int(y.shape[0]),
            obs_t=_ptr(obs_t), obs_s=_ptr(obs_s), obs_v=_ptr(obs_v), obs_cov=_ptr(cov),
            y=_ptr(y), tip_prior=tip_prior, theta_prior_var=theta_prior_var,
            low_memory=int(bool(low_memory)))
        h = C.c_void_p()
        torch.cuda.init()
        check(L.inla_model_create(C.byref(spec), C.byref(h)), "inla_model_create")
        self.handle = h
        dims = [C.c_int32() for _ in range(5)]
        check(L.inla_model_dims(h, *[C.byref(x) for x in dims]), "inla_model_dims")
        self.d, self.b, self.ld, self.n, self.a = [x.value for x in dims]

    def close(self):
        if getattr(self, "handle", None):
            lib().inla_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- evaluation ----------------------------------------------------------
    def value_and_grad(self, theta, grad: bool = True, use_graph: bool = True, stream=None,
                       concurrent: int = 1, precision: int = 0):
        return inla_value_and_grad(self, theta, grad=grad, use_graph=use_graph, stream=stream,
                                   concurrent=concurrent, precision=precision)

    def value(self, theta, use_graph: bool = True, stream=None):
        return inla_value_and_grad(self, theta, grad=False, use_graph=use_graph,
                                   stream=stream)[0]

    def hessian(self, theta, h: float = 5e-3, precision: int = 0, concurrent: int = 1,
                stream=None):
        """Eq. 13: central differences of exact gradients (2d + 1 gradient
        evaluations).  Returns (H, grad at theta); H[i, j] = d grad_i / d theta_j."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        H = np.zeros((self.d, self.d))
        g0 = np.zeros(self.d)
        opts = inla_opts(precision=int(precision), use_graph=1, streams=int(concurrent),
                         reserved=0)
        dp = C.POINTER(C.c_double)
        check(lib().inla_hessian(self.handle, th.ctypes.data_as(dp), float(h),
                                 H.ctypes.data_as(dp), g0.ctypes.data_as(dp), C.byref(opts),
                                 _stream(stream)), "inla_hessian")
        return H, g0

    def last_parts(self) -> dict:
        parts = (C.c_double * 8)()
        ph = (C.c_double * (4 * self.d))()
        check(lib().inla_last_parts(self.handle, parts, ph), "inla_last_parts")
        ph = np.array(ph[:]).reshape(4, self.d)
        return dict(logdet_p=parts[0], logdet_c=parts[1], quad=parts[2], loglik=parts[3],
                    logprior=parts[4], f=parts[5], fail_c=int(parts[6]), fail_p=int(parts[7]),
                    phase_a=ph[0], phase_b=ph[1], phase_c=ph[2], explicit=ph[3])

    def mode(self, stream=None) -> torch.Tensor:
        """x* of the last evaluation, unpadded, as a device tensor of N values."""
        buf = torch.empty(self.n * self.ld + self.a, dtype=torch.float64, device="cuda")
        check(lib().inla_copy_mode(self.handle, C.c_void_p(buf.data_ptr()), _stream(stream)),
              "inla_copy_mode")
        lat = buf[: self.n * self.ld].view(self.n, self.ld)[:, : self.b].reshape(-1)
        return torch.cat([lat, buf[self.n * self.ld:]])

    def kernel_launches(self) -> int:
        return int(lib().inla_kernel_launches(self.handle))

    def new_matrix(self, which: int) -> "BtaMatrix":
        return BtaMatrix(self.n, self.b, self.a if which else 0, self.ld)


class BtaMatrix:
    """Caller-owned device storage of one BTA matrix in the bta_desc layout."""

    def __init__(self, n: int, b: int, a: int, ld: int):
        dev = "cuda"
        self.D = torch.zeros(n, ld, ld, dtype=torch.float64, device=dev)
        self.B = torch.zeros(max(n - 1, 1), ld, ld, dtype=torch.float64, device=dev)
        self.C = torch.zeros(n, ld, a, dtype=torch.float64, device=dev) if a else None
        self.T = torch.zeros(a, a, dtype=torch.float64, device=dev) if a else None
        self.desc = bta_desc(n=n, b=b, a=a, ld=ld, D=self.D.data_ptr(), B=self.B.data_ptr(),
                             C=self.C.data_ptr() if a else None,
                             T=self.T.data_ptr() if a else None, state=0)
        self.n, self.b, self.a, self.ld = n, b, a, ld

    # Column-major views: block i of D as a (row, col) matrix is D[i].T
    def block_D(self, i):
        return self.D[i].T[: self.b, : self.b]

    def block_B(self, i):
        return self.B[i].T[: self.b, : self.b]

    def block_C(self, i):
        return self.C[i].T[:, : self.b]

    def tip(self):
        return self.T.T

    @property
    def state(self) -> int:
        return self.desc.state


def bta_assemble(model: InlaModel, theta, which: int, out: BtaMatrix, rhs=None, stream=None):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    check(lib().bta_assemble(model.handle, th.ctypes.data_as(C.POINTER(C.c_double)), which,
                             C.byref(out.desc),
                             C.c_void_p(rhs.data_ptr()) if rhs is not None else None,
                             _stream(stream)), "bta_assemble")


def bta_factor(q: BtaMatrix, rhs=None, precision: int = 0, stream=None):
    """Returns (logdet, fail_block) as device tensors (fail_block: -1, the
    first failing block, or -5 if a bounded device wait expired)."""
    logdet = torch.zeros(1, dtype=torch.float64, device="cuda")
    fail = torch.zeros(1, dtype=torch.int32, device="cuda")
    check(lib().bta_factor(C.byref(q.desc), C.c_void_p(rhs.data_ptr()) if rhs is not None else None,
                           C.c_void_p(logdet.data_ptr()), C.c_void_p(fail.data_ptr()),
                           int(precision), _stream(stream)), "bta_factor")
    return logdet, fail


def bta_solve(L: BtaMatrix, z, lower: bool = False, refine: bool = False,
              Q: BtaMatrix | None = None, stream=None):
    """z <- Q^{-1} z (lower = True: z holds r) with the factor L; refine =
    True adds one FP64 refinement step against the assembled Q (needs lower)."""
    check(lib().bta_solve(C.byref(L.desc), C.c_void_p(z.data_ptr()), int(lower), int(refine),
                          C.byref(Q.desc) if Q is not None else None, _stream(stream)),
          "bta_solve")


def bta_selinv(L: BtaMatrix, model: InlaModel | None = None, theta=None, which: int = 1,
               stream=None):
    """Selected inversion in place; with a model and theta also returns the
    fused traces tr(Q^{-1} dQ/dtheta_k) as a device tensor."""
    if model is None:
        check(lib().bta_selinv(C.byref(L.desc), None, None, which, None, _stream(stream)),
              "bta_selinv")
        return None
    th = np.ascontiguousarray(theta, dtype=np.float64)
    tr = torch.zeros(model.d, dtype=torch.float64, device="cuda")
    check(lib().bta_selinv(C.byref(L.desc), model.handle,
                           th.ctypes.data_as(C.POINTER(C.c_double)), which,
                           C.c_void_p(tr.data_ptr()), _stream(stream)), "bta_selinv")
    return tr


def inla_value_and_grad(model: InlaModel, theta, grad: bool = True, use_graph: bool = True,
                        stream=None, concurrent: int = 1, precision: int = 0):
    """f(theta) (Eq. 1) and its gradient (Eq. 6) for one theta (d,) or a
    batch (B, d).  With concurrent > 1, up to that many thetas are evaluated
    together (their matrices swept in the same launches; each needs its own
    device buffers).  precision 1 selects the mixed-precision mode (tensor-core
    split-TF32 Schur products, FP64 diagonal factors and log-dets, one FP64
    refinement of x*).  Returns numpy arrays (f, grad or None)."""
    th = np.ascontiguousarray(np.atleast_2d(np.asarray(theta, dtype=np.float64)))
    batch = th.shape[0]
    if th.shape[1] != model.d:
        raise ValueError(f"theta must have {model.d} columns")
    f = np.zeros(batch)
    g = np.zeros((batch, model.d)) if grad else None
    opts = inla_opts(precision=int(precision), use_graph=int(use_graph), streams=int(concurrent),
                     reserved=0)
    dp = C.POINTER(C.c_double)
    check(lib().inla_value_and_grad(model.handle, th.ctypes.data_as(dp), batch,
                                    f.ctypes.data_as(dp),
                                    g.ctypes.data_as(dp) if grad else None, C.byref(opts),
                                    _stream(stream)), "inla_value_and_grad")
    if np.ndim(theta) == 1:
        return f[0], (g[0] if grad else None)
    return f, g


def bta_gemm(A: torch.Tensor, B: torch.Tensor, C_out: torch.Tensor, alpha: float = 1.0,
             beta: float = 0.0, transA: bool = False, transB: bool = False, stream=None):
    """C_out = alpha op(A) op(B) + beta C_out with the library's FP64 tile
    kernel.  Tensors hold column-major matrices: a (rows, cols) matrix is
    stored as a torch tensor of shape (cols, rows)."""
    M = A.shape[0] if transA else A.shape[1]
    K = A.shape[1] if transA else A.shape[0]
    N = B.shape[1] if transB else B.shape[0]
    check(lib().bta_gemm(M, N, K, alpha, C.c_void_p(A.data_ptr()), A.shape[1], int(transA),
                         C.c_void_p(B.data_ptr()), B.shape[1], int(transB), beta,
                         C.c_void_p(C_out.data_ptr()), C_out.shape[1], _stream(stream)),
          "bta_gemm")


def bta_gemm_emulated(A: torch.Tensor, B: torch.Tensor, C_out: torch.Tensor, alpha: float = 1.0,
                      beta: float = 0.0, transA: bool = False, transB: bool = False,
                      slices: int = 8, stream=None) -> torch.Tensor:
    """As bta_gemm, computed to FP64 accuracy on the BF16 tensor cores from
    `slices` base-128 digits per operand (bta_gemm_emulated).  Returns the
    device status word (0, or BTA_ERR_TIMEOUT if a bounded wait expired)."""
    M = A.shape[0] if transA else A.shape[1]
    K = A.shape[1] if transA else A.shape[0]
    N = B.shape[1] if transB else B.shape[0]
    st = torch.zeros(1, dtype=torch.int32, device=C_out.device)
    check(lib().bta_gemm_emulated(M, N, K, alpha, C.c_void_p(A.data_ptr()), A.shape[1],
                                  int(transA), C.c_void_p(B.data_ptr()), B.shape[1], int(transB),
                                  beta, C.c_void_p(C_out.data_ptr()), C_out.shape[1], slices,
                                  C.c_void_p(st.data_ptr()), _stream(stream)),
          "bta_gemm_emulated")
    return st


class InlaBatch:
    """Several models evaluated by one CUDA graph launch
    (inla_batch_value_and_grad): each model's whole evaluation is a branch of
    the graph, so models of uneven block size run concurrently."""

    def __init__(self, models):
        self.models = list(models)
        arr = (C.c_void_p * len(self.models))(*[m.handle.value for m in self.models])
        h = C.c_void_p()
        check(lib().inla_batch_create(arr, len(self.models), C.byref(h)), "inla_batch_create")
        self.handle = h
        self.ldt = max(m.d for m in self.models)

    def close(self):
        if getattr(self, "handle", None):
            lib().inla_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def value_and_grad(self, thetas, grad: bool = True, precision: int = 0, stream=None):
        n = len(self.models)
        th = np.zeros((n, self.ldt))
        for i, t in enumerate(thetas):
            th[i, :len(t)] = t
        f = np.zeros(n)
        g = np.zeros((n, self.ldt)) if grad else None
        opts = inla_opts(precision=int(precision), use_graph=1, streams=1, reserved=0)
        dp = C.POINTER(C.c_double)
        check(lib().inla_batch_value_and_grad(self.handle, th.ctypes.data_as(dp), self.ldt,
                                              f.ctypes.data_as(dp),
                                              g.ctypes.data_as(dp) if grad else None,
                                              C.byref(opts), _stream(stream)),
              "inla_batch_value_and_grad")
        grads = [g[i, :m.d].copy() for i, m in enumerate(self.models)] if grad else None
        return f, grads
