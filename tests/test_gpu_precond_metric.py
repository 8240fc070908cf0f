"""General preconditioners and ill-conditioned metrics on the GPU path.

  * The Chebyshev polynomial preconditioner (lobpcg_chebyshev_apply, plugged
    into the callback slot of Algorithm 1 / Eq. 2 by the library itself)
    against the oracle running the same K: same eigenvalues, same closed
    form, fewer iterations than Jacobi.
  * A sparse metric B = I + c (grid adjacency) with cond(B) ~ 1e5, the SIESTA
    regime of Sec. 6 (where Sec. 5.2's safety rule turns the implicit
    products off): eigenvalues against the closed form (4 - mu) / (1 + c mu),
    the oracle, and B-orthonormality of the output.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
import paper_1704_07458_gb300 as gb
from oracle import lobpcg as L
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _x0(p):
    return synth.normal_block(0, synth.STREAM_X0, p.n, synth.block_width(p.k, p.n))


def _om(p):
    return synth.normal_block(0, synth.STREAM_OMEGA, p.n, 16).T


@pytest.mark.parametrize("mode", ["f64", "ozaki_tc"])
@pytest.mark.parametrize("name,kw,lmin,lmax", [
    ("lap2d_32", {}, 0.05, 2.0),
    ("lap3d_64_diagB", dict(N=16, k=16), 0.05, 2.0),
])
def test_chebyshev_callback_matches_oracle_same_k(name, kw, lmin, lmax, mode):
    torch = torch_cuda()
    p = synth.make_problem(name, **kw)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rp, ci, va = dev(p.A.rowptr), dev(p.A.col), dev(p.A.val)
    nx = synth.block_width(p.k, p.n)
    with gb.Solver(gemm_mode=mode) as s:
        s.set_operator(rp, ci, va, b_diag=None if p.b_diag is None else dev(p.b_diag))
        s.set_precond_chebyshev(rp, ci, va, degree=4, lmin=lmin, lmax=lmax, max_cols=nx)
        lam, X, it, be, rc = s.solve(p.k, p.tol, X0=_x0(p))
        st = s.stats()
    assert rc == gb.LOBPCG_OK
    A = sp.csr_matrix((p.A.val, p.A.col, p.A.rowptr), shape=(p.n, p.n))
    K = L.chebyshev_precond(A, 4, lmin, lmax)
    pen = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), p.b_diag, None, k_fn=K)
    r = L.lobpcg(pen, _x0(p), p.k, p.tol, _om(p))
    np.testing.assert_allclose(lam, r.lam, rtol=1e-10)
    if p.closed_form is not None:
        np.testing.assert_allclose(lam, p.closed_form[:p.k], rtol=1e-10)
    # the polynomial preconditioner beats Jacobi on iterations (as in the oracle)
    pj = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), p.b_diag, p.kdiag)
    rj = L.lobpcg(pj, _x0(p), p.k, p.tol, _om(p))
    assert it < rj.iters and r.iters < rj.iters


def test_chebyshev_apply_entry_point_against_oracle():
    """One application through the C ABI equals the oracle's K^-1 R."""
    torch = torch_cuda()
    p = synth.make_problem("lap2d_32")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    R = synth.normal_block(3, 1, p.n, 7)
    # the object borrows the CSR arrays: they must stay alive while it is used
    rp, ci, va = dev(p.A.rowptr), dev(p.A.col), dev(p.A.val)
    c = gb.lobpcg_chebyshev_create(p.n, rp, ci, va, None, 5, 0.05, 2.0, 7)
    Rd = dev(R)
    Wd = torch.empty_like(Rd)
    rc = gb.lobpcg_chebyshev_apply(c, p.n, 7, Rd, 7, Wd, 7, None)
    torch.cuda.synchronize()
    gb.lobpcg_chebyshev_destroy(c)
    assert rc == 0
    A = sp.csr_matrix((p.A.val, p.A.col, p.A.rowptr), shape=(p.n, p.n))
    ref = L.chebyshev_precond(A, 5, 0.05, 2.0)(R)
    np.testing.assert_allclose(Wd.cpu().numpy(), ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mode", ["f64", "ozaki_tc"])
def test_ill_conditioned_sparse_metric(mode):
    """B = I + c Adj on the 32 x 32 grid with c = 0.251133: the extreme
    eigenvalues of B are 1 -/+ 4 c cos(pi/33), cond(B) ~ 1e5."""
    N, c = 32, 0.251133
    A = synth.laplacian_2d_dirichlet(N)
    Bm = synth.mass_matrix_2d(N, c)
    mu = 4 * np.cos(np.pi / (N + 1))
    assert (1 + c * mu) / (1 - c * mu) > 5e4
    k = 8
    ref = synth.closed_form_mass_pencil(N, c, k)
    torch_cuda()
    with gb.Solver(gemm_mode=mode) as s:
        s.set_operator(A.rowptr, A.col, A.val, b_csr=(Bm.rowptr, Bm.col, Bm.val))
        X0 = synth.normal_block(0, synth.STREAM_X0, A.n, synth.block_width(k, A.n))
        lam, X, it, be, rc = s.solve(k, 1e-8, X0=X0)
    assert rc == gb.LOBPCG_OK
    np.testing.assert_allclose(lam, ref, rtol=1e-9)
    Bs = sp.csr_matrix((Bm.val, Bm.col, Bm.rowptr), shape=(A.n, A.n))
    np.testing.assert_allclose(X.T @ (Bs @ X), np.eye(k), atol=1e-9)
    pen = L.Pencil(A.n, (A.rowptr, A.col, A.val), (Bm.rowptr, Bm.col, Bm.val), A.diagonal())
    Om = synth.normal_block(0, synth.STREAM_OMEGA, A.n, 16).T
    r = L.lobpcg(pen, X0, k, 1e-8, Om)
    np.testing.assert_allclose(lam, r.lam, rtol=1e-10)
