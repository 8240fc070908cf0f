"""torch.autograd.Function over the eigensolver and its adjoint.

  lam, X = LobpcgEig.apply(A_vals, B_vals, rowptr, col, k, tol, X0, opts, b_csr)

A_vals: the stored values of a symmetric CSR matrix A (float64, CUDA),
B_vals: None (B = I), the n diagonal entries of a diagonal B, or the stored
values of a CSR B whose (rowptr, col) pattern is given as b_csr.  The forward
pass runs lobpcg_solve on a handle of its own; the backward pass runs
lobpcg_eig_adjoint on the same handle, i.e. on the pencil of the forward
pass.  Gradients flow to A_vals and B_vals only; the eigenvectors are the
sign-fixed, B-orthonormal ones lobpcg_solve returns, so dL/dX is taken with
that normalisation held fixed.  Every step runs in the CUDA library; this
module only passes device pointers.
"""
import torch

from . import Solver, LOBPCG_OK


class LobpcgEig(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A_vals, B_vals, rowptr, col, k, tol, X0=None, opts=None, b_csr=None,
                cg_tol=0.0, cg_maxit=0):
        if not (A_vals.is_cuda and A_vals.dtype == torch.float64):
            raise TypeError("A_vals must be a float64 CUDA tensor")
        s = Solver(stream=torch.cuda.current_stream(), **(opts or {}))
        A = A_vals.detach().contiguous()
        if B_vals is None:
            s.set_operator(rowptr, col, A)
        elif b_csr is None:
            s.set_operator(rowptr, col, A, b_diag=B_vals.detach().contiguous())
        else:
            s.set_operator(rowptr, col, A,
                           b_csr=(b_csr[0], b_csr[1], B_vals.detach().contiguous()))
        lam, X, it, be, rc = s.solve(k, tol, X0=X0, device=True)
        if rc != LOBPCG_OK:
            s.close()
            raise RuntimeError(f"lobpcg_solve returned status {rc}")
        ctx.solver = s
        ctx.k = k
        ctx.has_b = B_vals is not None
        ctx.cg = (cg_tol, cg_maxit)
        ctx.save_for_backward(lam, X)
        return lam, X

    @staticmethod
    def backward(ctx, glam, gX):
        lam, X = ctx.saved_tensors
        s = ctx.solver
        gl = glam.contiguous() if glam is not None else None
        G = gX.contiguous() if gX is not None else None
        gA, gB, its, rc = s.adjoint(ctx.k, lam, X, gl, G, cg_tol=ctx.cg[0], cg_maxit=ctx.cg[1])
        s.close()
        ctx.solver = None
        return (gA, gB if ctx.has_b else None) + (None,) * 9
