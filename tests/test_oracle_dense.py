"""Pins of the oracle's dense layer against closed forms and identities."""
import numpy as np
import pytest

from oracle import dense


def _householder_orthogonal(n, seed):
    """Q = product of three Householder reflectors, built from the formula."""
    rng = np.random.default_rng(seed)
    Q = np.eye(n)
    for _ in range(3):
        v = rng.standard_normal(n)
        Q = Q @ (np.eye(n) - 2.0 * np.outer(v, v) / (v @ v))
    return Q


@pytest.mark.parametrize("n", [1, 2, 7, 20])
def test_jacobi_1d_laplacian_closed_form(n):
    A = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = dense.jacobi_eigh(A)
    ref = 4 * np.sin(np.pi * np.arange(1, n + 1) / (2 * (n + 1))) ** 2
    np.testing.assert_allclose(w, ref, atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(A @ V, V * w, atol=1e-12)


def test_jacobi_tiny_coupling_small_angle():
    """A coupling of 1e-160 gives tau = 5e159, whose square overflows: the
    rotation must still take the small-angle tangent 1/(2 tau) = 1e-160, so
    the eigenvector of eigenvalue 2 carries 1e-160 in its first entry
    ((A - 2 I) v = 0 with v = (e, 1): e = 1e-160 / (2 - 1))."""
    c = 1e-160
    A = np.array([[1.0, c], [c, 2.0]])
    with np.errstate(over="raise", invalid="raise"):
        # tol = 0: the sweep may not stop before rotating the tiny coupling away
        w, V = dense.jacobi_eigh(A, tol=0.0)
    np.testing.assert_array_equal(w, [1.0, 2.0])
    v = V[:, 1] * np.sign(V[1, 1])
    assert v[1] == 1.0
    np.testing.assert_allclose(v[0], c, rtol=1e-14)


def test_jacobi_prescribed_spectrum():
    n = 30
    Q = _householder_orthogonal(n, 1)
    lam = np.linspace(-3, 5, n) ** 3
    A = Q @ np.diag(lam) @ Q.T
    w, V = dense.jacobi_eigh(A)
    np.testing.assert_allclose(w, np.sort(lam), atol=1e-11)
    np.testing.assert_allclose(np.abs(V.T @ Q).max(axis=0), 1.0, atol=1e-10)


def test_library_eigh_matches_jacobi_and_is_ascending():
    rng = np.random.default_rng(2)
    for n in [3, 17, 60]:
        M = rng.standard_normal((n, n))
        M = M + M.T
        w, V = dense.eigh(M)
        wj, _ = dense.jacobi_eigh(M)
        np.testing.assert_allclose(w, wj, atol=1e-12 * np.abs(wj).max())
        assert np.all(np.diff(w) >= 0)
        np.testing.assert_allclose(M @ V, V * w, atol=1e-12 * np.abs(w).max())


def test_cholesky_wrappers():
    rng = np.random.default_rng(3)
    G = rng.standard_normal((12, 12))
    M = G @ G.T + 12 * np.eye(12)
    R = dense.cholesky_upper(M)
    assert np.allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(R.T @ R, M, atol=1e-12)
    L = dense.cholesky_lower_plain(M)
    np.testing.assert_allclose(L, R.T, atol=1e-12)
    bad = M.copy()
    bad[0, 0] = -1
    with pytest.raises(np.linalg.LinAlgError):
        dense.cholesky_upper(bad)
    with pytest.raises(np.linalg.LinAlgError):
        dense.cholesky_lower_plain(bad)


def test_householder_qr_rank_deficient_still_orthonormal():
    rng = np.random.default_rng(4)
    M = rng.standard_normal((20, 3)) @ rng.standard_normal((3, 8))
    Q, R = dense.qr_householder(M)
    np.testing.assert_allclose(Q.T @ Q, np.eye(8), atol=1e-14)
    np.testing.assert_allclose(Q @ R, M, atol=1e-12)
    assert np.allclose(np.tril(R, -1), 0)


def test_pencil_eigh_definition():
    rng = np.random.default_rng(5)
    n = 15
    A = rng.standard_normal((n, n))
    A = A + A.T
    b = rng.uniform(1, 2, n)
    w, X = dense.pencil_eigh(A, np.diag(b))
    np.testing.assert_allclose(A @ X, (b[:, None] * X) * w, atol=1e-11)
    np.testing.assert_allclose(X.T @ (b[:, None] * X), np.eye(n), atol=1e-12)
    # B = c I scales the spectrum by 1/c
    w2, _ = dense.pencil_eigh(A, 4.0 * np.eye(n))
    wa, _ = dense.jacobi_eigh(A)
    np.testing.assert_allclose(w2, wa / 4.0, atol=1e-12)
