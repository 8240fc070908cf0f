"""GB300-native robust LOBPCG (Duersch, Shao, Yang, Gu, 2018; Algorithm 8).

The solver and its kernels live in a CUDA shared library with a C ABI
(include/lobpcg.h).  This package is only its binding:

  _native   one Python function per C entry point, same names (ctypes)
  Solver    convenience wrapper: create / set_operator / solve / adjoint / stats
  autograd  LobpcgEig, a torch.autograd.Function over solve and adjoint

PyTorch is used, when present, only to hand device buffers and streams to the
library.  There is no CPU fallback: if the library is not built, importing the
binding functions raises.
"""
import numpy as np

from . import _native
from ._native import (  # noqa: F401
    LOBPCG_OK, LOBPCG_ERR_ARG, LOBPCG_ERR_NOT_CONVERGED, LOBPCG_ERR_BREAKDOWN,
    LOBPCG_ERR_CUDA, LOBPCG_ERR_OOM, LOBPCG_ERR_TIMEOUT, LOBPCG_ERR_CALLBACK,
    LOBPCG_ERR_DEGENERATE,
    LOBPCG_MEM_HOST, LOBPCG_MEM_DEVICE, LOBPCG_GEMM_F64, LOBPCG_GEMM_OZAKI, LOBPCG_GEMM_OZAKI_TC,
    lobpcg_options_t, lobpcg_stats_t, LobpcgError,
    lobpcg_create, lobpcg_set_operator, lobpcg_set_precond_diag,
    lobpcg_set_precond_callback, lobpcg_solve, lobpcg_get_stats, lobpcg_last_error,
    lobpcg_destroy, lobpcg_spmm, lobpcg_gram, lobpcg_gram_workspace, lobpcg_gram_noalloc,
    lobpcg_update, lobpcg_eig_adjoint, lobpcg_syev,
    lobpcg_residual, lobpcg_philox_normal, load, library_path,
    lobpcg_chebyshev_create, lobpcg_chebyshev_apply, lobpcg_chebyshev_destroy,
    lobpcg_wait_selftest, lobpcg_set_operator_ex, LOBPCG_F64, LOBPCG_F32, LOBPCG_BORROW,
)

__all__ = [n for n in dir() if n.startswith("lobpcg_") or n.startswith("LOBPCG_")] + [
    "Solver", "options", "LobpcgError", "load", "library_path"]


def options(**kw):
    """lobpcg_options_t with the given fields set (zeros select defaults)."""
    o = lobpcg_options_t()
    for k, v in kw.items():
        if k == "gemm_mode" and isinstance(v, str):
            v = {"f64": LOBPCG_GEMM_F64, "ozaki": LOBPCG_GEMM_OZAKI,
                 "ozaki_tc": LOBPCG_GEMM_OZAKI_TC}[v]
        if k == "implicit" and isinstance(v, str):
            v = {"auto": 0, "never": 1, "always": 2}[v]
        if k == "basis" and isinstance(v, str):
            v = {"robust": 0, "chl": 1, "ahl": 2}[v]
        if k == "explicit_rr" and isinstance(v, str):
            v = {"auto": 0, "off": 1, "on": 2}[v]
        setattr(o, k, v)
    return o


class Solver:
    """Owning wrapper of one lobpcg_t handle.

    Host arrays (numpy) or device tensors (torch, cuda) are accepted; the
    memory kind is detected per argument group.
    """

    def __init__(self, stream=None, **opts):
        self.opts = options(**opts)
        self.stream = stream
        self.h = lobpcg_create(self.opts, stream)
        self.n = 0
        self._cb = None
        self._cheb = None

    def close(self):
        if self.h:
            lobpcg_destroy(self.h)
            self.h = None
        if getattr(self, "_cheb", None) is not None:
            lobpcg_chebyshev_destroy(self._cheb)
            self._cheb = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @staticmethod
    def _mem(x):
        if x is not None and hasattr(x, "is_cuda") and x.is_cuda:
            return LOBPCG_MEM_DEVICE
        return LOBPCG_MEM_HOST

    def _check(self, rc, what):
        if rc != LOBPCG_OK:
            raise LobpcgError(rc, f"{what}: {lobpcg_last_error(self.h)}")

    @staticmethod
    def _arg(x, mem, dtype, name):
        """Marshal one array argument: host arrays become contiguous numpy of
        `dtype`; device tensors must already be contiguous CUDA tensors of
        that dtype (the library reads them as raw int32 / float64 memory)."""
        if x is None:
            return None
        if mem == LOBPCG_MEM_HOST:
            if hasattr(x, "is_cuda"):
                if x.is_cuda:
                    raise ValueError(f"{name}: a CUDA tensor among host arguments")
                x = x.detach().numpy()
            return np.ascontiguousarray(x, dtype=dtype)
        if not (hasattr(x, "is_cuda") and x.is_cuda):
            raise ValueError(f"{name}: a host array among device arguments")
        want = {np.int32: "torch.int32", np.float64: "torch.float64",
                np.float32: "torch.float32"}[dtype]
        if str(x.dtype) != want:
            raise TypeError(f"{name}: device tensor must be {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: device tensor must be contiguous")
        return x

    @staticmethod
    def _f32(x):
        """True for FP32 values (numpy float32 or a float32 tensor)."""
        return x is not None and str(getattr(x, "dtype", "")) in ("float32", "torch.float32")

    def set_operator(self, rowptr, col, val, b_diag=None, b_csr=None, borrow=False):
        """Set the pencil (lobpcg_set_operator_ex).  FP32 values (numpy
        float32 or float32 tensors) are passed as FP32 and widened by the
        library; borrow=True (device tensors only) lets the handle use the CSR
        tensors in place, which this object then keeps alive."""
        mem = self._mem(val)
        n = len(rowptr) - 1
        rowptr = self._arg(rowptr, mem, np.int32, "rowptr")
        col = self._arg(col, mem, np.int32, "col")
        a_dt = np.float32 if self._f32(val) else np.float64
        val = self._arg(val, mem, a_dt, "val")
        if len(col) != len(val):
            raise ValueError("col and val differ in length")
        b_src = b_csr[2] if b_csr is not None else b_diag
        b_dt = np.float32 if self._f32(b_src) else np.float64
        args = dict(B_diag=self._arg(b_diag, mem, b_dt, "b_diag"))
        if b_csr is not None:
            brp = self._arg(b_csr[0], mem, np.int32, "b_csr rowptr")
            bcol = self._arg(b_csr[1], mem, np.int32, "b_csr col")
            bval = self._arg(b_csr[2], mem, b_dt, "b_csr val")
            if len(brp) != n + 1 or len(bcol) != len(bval):
                raise ValueError("b_csr does not match the size of A")
            args = dict(B_rowptr=brp, B_col=bcol, B_val=bval, B_nnz=len(bval))
        elif b_diag is not None and len(args["B_diag"]) != n:
            raise ValueError("b_diag must have n entries")
        self._keep = (rowptr, col, val, args)
        self.n = 0
        dt = lambda d: LOBPCG_F32 if d is np.float32 else LOBPCG_F64
        rc = lobpcg_set_operator_ex(self.h, n, rowptr, col, val, len(val), dt(a_dt), mem=mem,
                                    B_dtype=dt(b_dt), flags=LOBPCG_BORROW if borrow else 0,
                                    **args)
        self._check(rc, "set_operator")
        self.n = n

    def set_precond_diag(self, kdiag):
        mem = self._mem(kdiag)
        kdiag = self._arg(kdiag, mem, np.float64, "kdiag")
        if kdiag is not None and len(kdiag) != self.n:
            raise ValueError("kdiag must have n entries")
        self._check(lobpcg_set_precond_diag(self.h, kdiag, mem), "set_precond_diag")

    def set_precond_identity(self):
        self._check(lobpcg_set_precond_diag(self.h, None, -1), "set_precond_diag")

    def set_precond_callback(self, fn):
        """fn(n, ncols, R_ptr, ldr, W_ptr, ldw, stream_ptr) -> int (device pointers)."""
        def tramp(ctx, n, ncols, R, ldr, W, ldw, stream):
            try:
                return int(fn(n, ncols, R, ldr, W, ldw, stream))
            except Exception:
                return 1
        self._cb = _native.PRECOND_FN(tramp)
        self._check(lobpcg_set_precond_callback(self.h, self._cb, None), "set_precond_callback")

    def set_precond_chebyshev(self, rowptr, col, val, degree, lmin, lmax, max_cols,
                              diag=None):
        """K^-1 = `degree` Chebyshev steps for A (device CSR tensors, kept
        alive by this object) over the interval [lmin, lmax] of D^-1 A, applied
        by the library through its callback slot (lobpcg_chebyshev_apply)."""
        if self._cheb is not None:
            lobpcg_chebyshev_destroy(self._cheb)
        self._cheb_refs = (rowptr, col, val, diag)
        self._cheb = lobpcg_chebyshev_create(self.n, rowptr, col, val, diag, degree, lmin, lmax,
                                             max_cols)
        self._cb = _native.chebyshev_callback()
        self._check(lobpcg_set_precond_callback(self.h, self._cb, self._cheb),
                    "set_precond_callback")

    def solve(self, k, tol=1e-8, X0=None, seed=0, device=False, raise_on_error=True):
        """Return (lam, X, iters, backward_errors, status).

        device=True returns torch CUDA tensors (outputs written in place by the
        library); otherwise numpy arrays.
        """
        n = self.n
        mem_in = self._mem(X0)
        ldx0 = 0
        if X0 is not None:
            X0 = self._arg(X0, mem_in, np.float64, "X0")
            if X0.ndim != 2 or X0.shape[0] != n:
                raise ValueError("X0 must be n x n_x")
            ldx0 = X0.shape[1]
        if device:
            import torch
            lam = torch.empty(k, dtype=torch.float64, device="cuda")
            X = torch.empty((n, k), dtype=torch.float64, device="cuda")
            be = torch.empty(k, dtype=torch.float64, device="cuda")
            mem_out = LOBPCG_MEM_DEVICE
        else:
            lam = np.empty(k)
            X = np.empty((n, k))
            be = np.empty(k)
            mem_out = LOBPCG_MEM_HOST
        rc, it = lobpcg_solve(self.h, k, tol, X0, ldx0, seed, mem_in, lam, X, k, mem_out, be)
        if rc not in (LOBPCG_OK, LOBPCG_ERR_NOT_CONVERGED) and raise_on_error:
            self._check(rc, "solve")
        return lam, X, it, be, rc

    def adjoint(self, k, lam, X, glam=None, G=None, cg_tol=0.0, cg_maxit=0,
                raise_on_error=True):
        """Gradients (gA on A's stored entries, gB) of a loss with upstream
        gradients glam = dL/dlambda and G = dL/dX at the eigenpairs (lam, X)
        of the current pencil.  Returns (gA, gB or None, cg_iterations, status).
        Device tensors in give device tensors out; numpy in gives numpy out."""
        mem = self._mem(X)
        n = self.n
        nnz_a = len(self._keep[2])
        b_args = self._keep[3]
        b_len = (len(b_args["B_val"]) if "B_val" in b_args else
                 (n if b_args.get("B_diag") is not None else 0))
        X = self._arg(X, mem, np.float64, "X")
        lam = self._arg(lam, mem, np.float64, "lam")
        glam = self._arg(glam, mem, np.float64, "glam")
        G = self._arg(G, mem, np.float64, "G")
        if X.ndim != 2 or X.shape[0] != n or X.shape[1] < k or len(lam) < k:
            raise ValueError("X must be n x (>= k) and lam hold >= k values")
        if (glam is not None and len(glam) < k) or (
                G is not None and (G.ndim != 2 or G.shape[0] != n or G.shape[1] < k)):
            raise ValueError("glam must hold >= k values and G be n x (>= k)")
        if mem == LOBPCG_MEM_DEVICE:
            import torch
            gA = torch.empty(nnz_a, dtype=torch.float64, device="cuda")
            gB = torch.empty(b_len, dtype=torch.float64, device="cuda") if b_len else None
        else:
            gA = np.empty(nnz_a)
            gB = np.empty(b_len) if b_len else None
        rc, its = lobpcg_eig_adjoint(self.h, k, lam, X, X.shape[1], glam, G,
                                     G.shape[1] if G is not None else 0, mem, gA, gB, mem,
                                     cg_tol, cg_maxit)
        if rc not in (LOBPCG_OK, LOBPCG_ERR_NOT_CONVERGED) and raise_on_error:
            self._check(rc, "adjoint")
        return gA, gB, its, rc

    def stats(self):
        return lobpcg_get_stats(self.h).as_dict()
