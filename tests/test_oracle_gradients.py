"""Pins of the eigenpair-gradient oracle (oracle/gradients.py), CPU only.

The gradient has no closed form on a random potential, so it is pinned by:
central finite differences of the loss through an independent dense
eigensolver (LAPACK), the special case d lambda_i / d V_r = x_ri^2, Euler's
homogeneity identities of the pencil, and agreement of the full-decomposition
route with the bordered-solve route a large-n solver takes.
"""
import numpy as np
import pytest

import synth
from oracle import dense, gradients as og


def _c5_small(N=12, seed=0, k=32):
    """The 12x12 instance of the 2D Dirichlet Laplacian + diag(V), V ~ U[0,1]."""
    p = synth.make_problem("lap2d_512_V", seed=seed, N=N, k=k)
    A = p.A.to_dense()
    G = synth.normal_block(seed, synth.STREAM_GRAD, p.n, k)
    return p, A, G


def _loss_lapack(A, B, k, glam, G):
    w, X = dense.pencil_eigh(A, B, use_jacobi=False)
    X = og.sign_fix(X)
    return float(np.dot(glam, w[:k]) + np.sum(X[:, :k] * G))


@pytest.fixture(scope="module")
def c5():
    p, A, G = _c5_small()
    k = p.k
    glam = np.ones(k)
    lam, X, GA, GB = og.grad_full(A, None, k, glam, G)
    return dict(p=p, A=A, G=G, k=k, glam=glam, lam=lam, X=X, GA=GA, GB=GB)


def test_small_instance_has_gaps(c5):
    lam = np.linalg.eigvalsh(c5["A"])
    k = c5["k"]
    assert np.diff(lam[:k + 1]).min() > 1e-4


def test_eigenvalue_gradient_special_case(c5):
    # L = lambda_i: dL/dA = x_i x_i^T, so dL/dV_r = x_ri^2 and sum_r = 1 (B = I)
    A, k = c5["A"], c5["k"]
    for i in (0, 5, k - 1):
        glam = np.zeros(k)
        glam[i] = 1.0
        lam, X, GA, GB = og.grad_full(A, None, k, glam, np.zeros((A.shape[0], k)))
        np.testing.assert_allclose(np.diag(GA), X[:, i] ** 2, atol=1e-14)
        assert abs(np.trace(GA) - 1.0) < 1e-12
        np.testing.assert_allclose(np.diag(GB), -lam[i] * X[:, i] ** 2, atol=1e-14)


def test_finite_differences_potential(c5):
    A, G, k, glam, GA = c5["A"], c5["G"], c5["k"], c5["glam"], c5["GA"]
    h = 1e-6
    for r in (0, 17, 77, 143):
        Ap, Am = A.copy(), A.copy()
        Ap[r, r] += h
        Am[r, r] -= h
        fd = (_loss_lapack(Ap, None, k, glam, G) - _loss_lapack(Am, None, k, glam, G)) / (2 * h)
        assert abs(fd - GA[r, r]) <= 1e-6 * max(1.0, abs(GA[r, r])), (r, fd, GA[r, r])


def test_finite_differences_offdiagonal_pair(c5):
    # a symmetric pair is one parameter: dL = (G_rc + G_cr) h
    A, G, k, glam, GA = c5["A"], c5["G"], c5["k"], c5["glam"], c5["GA"]
    p = c5["p"]
    h = 1e-6
    for r in (3, 50, 100):
        c = int(p.A.col[p.A.rowptr[r]:p.A.rowptr[r + 1]][-1])
        assert c != r
        Ap, Am = A.copy(), A.copy()
        for (a, b) in ((r, c), (c, r)):
            Ap[a, b] += h
            Am[a, b] -= h
        fd = (_loss_lapack(Ap, None, k, glam, G) - _loss_lapack(Am, None, k, glam, G)) / (2 * h)
        want = GA[r, c] + GA[c, r]
        assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (r, c, fd, want)


def test_generalised_pencil_finite_differences():
    # diagonal B ~ U[1, 2]: derivatives with respect to A_rr and B_rr
    p, A, G = _c5_small(N=8, k=6)
    n, k = p.n, 6
    b = synth.uniform_block(0, synth.STREAM_BDIAG, n, 1.0, 2.0)
    B = np.diag(b)
    glam = np.linspace(1.0, 2.0, k)
    lam, X, GA, GB = og.grad_full(A, B, k, glam, G)
    h = 1e-6
    for r in (0, 9, 40, 63):
        for which, Gd in (("A", GA), ("B", GB)):
            Ap, Am, Bp, Bm = A.copy(), A.copy(), B.copy(), B.copy()
            if which == "A":
                Ap[r, r] += h
                Am[r, r] -= h
            else:
                Bp[r, r] += h
                Bm[r, r] -= h
            fd = (_loss_lapack(Ap, Bp, k, glam, G) - _loss_lapack(Am, Bm, k, glam, G)) / (2 * h)
            assert abs(fd - Gd[r, r]) <= 1e-6 * max(1.0, abs(Gd[r, r])), (which, r, fd, Gd[r, r])


def test_homogeneity_identities():
    # lambda(aA, B) = a lambda, x(aA, B) = x        =>  <dL/dA, A> = sum gl_i lambda_i
    # lambda(A, bB) = lambda/b, x(A, bB) = x/sqrt(b) =>  <dL/dB, B> = -sum gl_i lambda_i
    #                                                    - 1/2 sum g_i^T x_i
    p, A, G = _c5_small(N=8, k=6)
    k = 6
    B = np.diag(synth.uniform_block(0, synth.STREAM_BDIAG, p.n, 1.0, 2.0))
    glam = np.linspace(-1.0, 3.0, k)
    lam, X, GA, GB = og.grad_full(A, B, k, glam, G)
    assert abs(np.sum(GA * A) - glam @ lam) < 1e-10
    want = -glam @ lam - 0.5 * np.sum(G * X)
    assert abs(np.sum(GB * B) - want) < 1e-10


def test_split_route_matches_full_decomposition(c5):
    A, G, k, glam = c5["A"], c5["G"], c5["k"], c5["glam"]
    lam, X = c5["lam"], c5["X"]
    GA, GB, W = og.grad_split(A, None, lam, X, glam, G)
    np.testing.assert_allclose(GA, c5["GA"], atol=1e-10)
    np.testing.assert_allclose(GB, c5["GB"], atol=1e-10)


def test_split_route_generalised():
    p, A, G = _c5_small(N=8, k=6)
    k = 6
    B = np.diag(synth.uniform_block(0, synth.STREAM_BDIAG, p.n, 1.0, 2.0))
    glam = np.ones(k)
    lam, X, GA, GB = og.grad_full(A, B, k, glam, G)
    GA2, GB2, W = og.grad_split(A, B, lam, X, glam, G)
    np.testing.assert_allclose(GA2, GA, atol=1e-10)
    np.testing.assert_allclose(GB2, GB, atol=1e-10)


def test_complement_solution_properties(c5):
    A, G, lam, X = c5["A"], c5["G"], c5["lam"], c5["X"]
    U, F = og.complement_solve(A, None, X, lam, G)
    R = A @ U - U * lam - F
    assert np.abs(R).max() < 1e-10
    assert np.abs(X.T @ U).max() < 1e-12


def test_degenerate_pair_is_rejected():
    A = np.diag([1.0, 1.0, 2.0, 3.0])
    with pytest.raises(ValueError):
        og.grad_full(A, None, 2, np.ones(2), np.ones((4, 2)))


def test_on_pattern_samples_stored_entries(c5):
    p, GA = c5["p"], c5["GA"]
    vals = og.on_pattern(GA, p.A.rowptr, p.A.col)
    rows = np.repeat(np.arange(p.n), np.diff(p.A.rowptr))
    np.testing.assert_array_equal(vals, GA[rows, p.A.col])
