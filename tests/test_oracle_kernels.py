"""Pins of the single-step definitions in oracle/kernels.py.

Each definition is checked against something other than itself: a dense
product built independently of the CSR arrays (the stencil written out
entry by entry), the library CSR product of scipy, closed-form eigenvectors
for which the residual of Algorithm 8 vanishes, and hand-computed values.
A transposed rowptr/col pair, a wrong row range or a dropped term fails one
of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import kernels as K


def _dense_laplacian_2d(nx, ny):
    """The 5-point Dirichlet Laplacian written out entry by entry (no CSR)."""
    n = nx * ny
    A = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            i = x + nx * y
            A[i, i] = 4.0
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xx, yy = x + dx, y + dy
                if 0 <= xx < nx and 0 <= yy < ny:
                    A[i, xx + nx * yy] = -1.0
    return A


def _csr_with_empty_rows():
    """A non-symmetric 7 x 7 CSR with empty rows 0, 3 and 6 and unsorted row lengths."""
    dense = np.zeros((7, 7))
    dense[1, [0, 4, 6]] = [2.0, -1.5, 0.25]
    dense[2, 2] = 3.0
    dense[4, [1, 2, 3, 5]] = [1.0, -2.0, 0.5, 7.0]
    dense[5, 0] = -4.0
    m = sp.csr_matrix(dense)
    return (m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.copy(), dense)


@pytest.mark.parametrize("m", [1, 3, 8])
def test_spmm_matches_written_out_stencil(m):
    A = synth.laplacian_2d_dirichlet(5, 4)
    D = _dense_laplacian_2d(5, 4)
    X = synth.normal_block(3, 1, A.n, m)
    np.testing.assert_allclose(K.spmm(A.rowptr, A.col, A.val, X), D @ X, rtol=0, atol=1e-13)


def test_spmm_and_sampled_rows_with_empty_rows():
    rp, ci, v, D = _csr_with_empty_rows()
    X = synth.normal_block(1, 1, 7, 5)
    Y = K.spmm(rp, ci, v, X)
    np.testing.assert_allclose(Y, D @ X, rtol=0, atol=1e-14)
    assert np.all(Y[[0, 3, 6]] == 0.0)
    rows = np.array([6, 4, 0, 1])
    np.testing.assert_allclose(K.spmm_rows(rp, ci, v, X, rows), (D @ X)[rows], rtol=0,
                               atol=1e-14)


def test_spmm_matches_scipy_on_diffusion_operator():
    A = synth.diffusion_3d_lognormal(6, 1.0, seed=2)
    X = synth.normal_block(5, 1, A.n, 4)
    ref = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)) @ X
    np.testing.assert_allclose(K.spmm(A.rowptr, A.col, A.val, X), ref, rtol=1e-14, atol=1e-13)
    rows = np.array([0, 17, A.n - 1, 100])
    np.testing.assert_allclose(K.spmm_rows(A.rowptr, A.col, A.val, X, rows), ref[rows],
                               rtol=1e-14, atol=1e-13)


def test_residual_vanishes_on_closed_form_eigenpairs():
    """The 1D Dirichlet Laplacian has eigenvectors sin(pi j i/(N+1)) with
    eigenvalues 4 sin^2(pi j/(2(N+1))): R = A X - X Theta is zero to rounding."""
    N = 40
    A = synth.laplacian_1d(N)
    i = np.arange(1, N + 1)[:, None]
    j = np.arange(1, 6)[None, :]
    X = np.sin(np.pi * i * j / (N + 1))
    theta = 4.0 * np.sin(np.pi * j[0] / (2.0 * (N + 1))) ** 2
    AX = K.spmm(A.rowptr, A.col, A.val, X)
    R = K.residual(AX, X, theta)
    assert np.max(np.abs(R)) < 1e-13
    # a wrong eigenvalue leaves exactly (theta_true - theta_wrong) x_j
    bad = theta.copy()
    bad[2] += 0.5
    R = K.residual(AX, X, bad)
    np.testing.assert_allclose(R[:, 2], -0.5 * X[:, 2], atol=1e-13)


def test_residual_generalised_hand_values():
    AX = np.array([[1.0, 2.0], [3.0, 4.0]])
    BX = np.array([[2.0, 1.0], [0.5, -1.0]])
    theta = np.array([0.5, 3.0])
    np.testing.assert_array_equal(K.residual(AX, BX, theta), [[0.0, -1.0], [2.75, 7.0]])


def test_gram_and_update_hand_values():
    U = np.array([[1.0, 2.0], [0.0, 1.0], [3.0, -1.0]])
    V = np.array([[2.0], [5.0], [1.0]])
    np.testing.assert_array_equal(K.gram(U, V), [[5.0], [8.0]])
    C = np.array([[1.0, 0.0, 2.0], [-1.0, 1.0, 0.5]])
    np.testing.assert_array_equal(K.update(U, C), [[-1.0, 2.0, 3.0], [-1.0, 1.0, 0.5],
                                                   [4.0, -1.0, 5.5]])
