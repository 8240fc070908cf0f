"""Parity of the eigenpair adjoint (lobpcg_eig_adjoint, LobpcgEig) with the
gradient oracle, through the C ABI on the GPU.

Tolerances follow from the conditioning: the solve reaches backward error
tol, so the eigenvectors carry errors up to ~tol ||A|| / gap and the
eigenvector part of the gradient up to ~tol ||A|| |g| / gap^2; the tests solve
at tol 1e-12 and allow 1e-6 of the largest gradient entry (the eigenvalue-only
gradient, x_i x_i^T, gets 1e-8).
"""
import numpy as np
import pytest

import synth
from oracle import gradients as og
import paper_1704_07458_gb300 as gb
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

MODES = ["f64", "ozaki_tc"]


def _instance(N, k, seed=0, diagB=False):
    p = synth.make_problem("lap2d_512_V", seed=seed, N=N, k=k)
    G = synth.normal_block(seed, synth.STREAM_GRAD, p.n, k)
    b = synth.uniform_block(seed, synth.STREAM_BDIAG, p.n, 1.0, 2.0) if diagB else None
    return p, G, b


def _solve(p, b, k, tol, mode):
    s = gb.Solver(gemm_mode=mode)
    s.set_operator(p.A.rowptr, p.A.col, p.A.val, b_diag=b)
    nx = synth.block_width(k, p.n)
    X0 = synth.normal_block(0, synth.STREAM_X0, p.n, nx)
    lam, X, it, be, rc = s.solve(k, tol, X0=X0)
    assert rc == gb.LOBPCG_OK
    return s, lam, X


def _oracle(p, b, k, glam, G, use_jacobi=True):
    A = p.A.to_dense()
    B = None if b is None else np.diag(b)
    lam, X, GA, GB = og.grad_full(A, B, k, glam, G, use_jacobi=use_jacobi)
    gA = og.on_pattern(GA, p.A.rowptr, p.A.col)
    gB = None if b is None else np.diag(GB).copy()
    return lam, X, gA, gB


@pytest.mark.parametrize("mode", MODES)
def test_adjoint_c5_12x12(mode):
    """The 12 x 12 instance of the 2D Laplacian + diag(V) (n = 144, k = 32)."""
    torch_cuda()
    k = 32
    p, G, _ = _instance(12, k)
    glam = np.ones(k)
    lam_o, X_o, gA_o, _ = _oracle(p, None, k, glam, G)
    s, lam, X = _solve(p, None, k, 1e-12, mode)
    np.testing.assert_allclose(lam, lam_o, rtol=1e-10)
    gA, gB, its, rc = s.adjoint(k, lam, X, glam, G)
    assert rc == gb.LOBPCG_OK and gB is None and its > 0
    scale = np.abs(gA_o).max()
    assert np.abs(gA - gA_o).max() <= 1e-6 * scale, np.abs(gA - gA_o).max() / scale
    # eigenvalue-only gradient: dlambda_i/dA = x_i x_i^T
    gA1, _, its1, rc1 = s.adjoint(k, lam, X, glam, None)
    _, _, gA1_o, _ = _oracle(p, None, k, glam, np.zeros((p.n, k)))
    assert rc1 == gb.LOBPCG_OK and its1 == 0
    assert np.abs(gA1 - gA1_o).max() <= 1e-8 * np.abs(gA1_o).max()
    s.close()


@pytest.mark.parametrize("mode", MODES)
def test_adjoint_generalised_diagonal_B(mode):
    torch_cuda()
    k = 6
    p, G, b = _instance(8, k, diagB=True)
    glam = np.linspace(1.0, 2.0, k)
    lam_o, X_o, gA_o, gB_o = _oracle(p, b, k, glam, G)
    s, lam, X = _solve(p, b, k, 1e-12, mode)
    np.testing.assert_allclose(lam, lam_o, rtol=1e-10)
    gA, gB, its, rc = s.adjoint(k, lam, X, glam, G)
    assert rc == gb.LOBPCG_OK
    sa, sb = np.abs(gA_o).max(), np.abs(gB_o).max()
    assert np.abs(gA - gA_o).max() <= 1e-6 * sa
    assert np.abs(gB - gB_o).max() <= 1e-6 * sb
    s.close()


def test_adjoint_mid_size_several_tiles():
    """48 x 48 grid (n = 2304, k = 32): CG over many row blocks, LAPACK oracle."""
    torch_cuda()
    k = 32
    p, G, _ = _instance(48, k)
    glam = np.ones(k)
    lam_o, X_o, gA_o, _ = _oracle(p, None, k, glam, G, use_jacobi=False)
    s, lam, X = _solve(p, None, k, 1e-12, "ozaki_tc")
    np.testing.assert_allclose(lam, lam_o, rtol=1e-10)
    gA, _, its, rc = s.adjoint(k, lam, X, glam, G, cg_tol=1e-12)
    assert rc == gb.LOBPCG_OK
    scale = np.abs(gA_o).max()
    assert np.abs(gA - gA_o).max() <= 1e-5 * scale, np.abs(gA - gA_o).max() / scale
    s.close()


def test_autograd_function_potential_gradient():
    """LobpcgEig: dL/dV for A = Lap + diag(V) through torch autograd."""
    torch = torch_cuda()
    from paper_1704_07458_gb300.autograd import LobpcgEig
    k = 32
    p, G, _ = _instance(12, k)
    V = p.extra["V"]
    base = p.A.val.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.A.rowptr))
    diag_pos = np.nonzero(rows == p.A.col)[0]
    base[diag_pos] -= V
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Vt = dev(V).requires_grad_(True)
    vals = dev(base).index_add(0, dev(diag_pos.astype(np.int64)), Vt)
    nx = synth.block_width(k, p.n)
    X0 = dev(synth.normal_block(0, synth.STREAM_X0, p.n, nx))
    lam, X = LobpcgEig.apply(vals, None, dev(p.A.rowptr), dev(p.A.col), k, 1e-12, X0,
                             {"gemm_mode": "f64"})
    loss = lam.sum() + (X * dev(G)).sum()
    loss.backward()
    _, _, GA, _ = og.grad_full(p.A.to_dense(), None, k, np.ones(k), G)
    got = Vt.grad.cpu().numpy()
    want = np.diag(GA)
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()


def test_adjoint_rejects_degenerate_pair():
    torch_cuda()
    # 2D Laplacian without potential: lambda_2 = lambda_3 exactly (symmetry)
    p = synth.make_problem("lap2d_32")
    k = 4
    s = gb.Solver(gemm_mode="f64")
    s.set_operator(p.A.rowptr, p.A.col, p.A.val)
    lam, X, it, be, rc = s.solve(k, 1e-10)
    assert rc == gb.LOBPCG_OK
    G = synth.normal_block(0, synth.STREAM_GRAD, p.n, k)
    _, _, _, rc = s.adjoint(k, lam, X, np.ones(k), G, raise_on_error=False)
    assert rc == gb.LOBPCG_ERR_DEGENERATE
    s.close()
