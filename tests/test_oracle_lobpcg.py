"""Pins of the LOBPCG oracle against the paper's worked example, the algorithms'
output contracts, closed-form spectra, brute force and invariances."""
import os

import numpy as np
import pytest

import synth
from oracle import dense
from oracle import lobpcg as L

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            out[k] = [float(x) for x in v]
    return out


def _pencil(A, b=None, kdiag=None):
    return L.Pencil(A.n, (A.rowptr, A.col, A.val), b, kdiag)


def _run(p, seed=0, opts=None, scaleA=1.0, scaleB=None, nx=None):
    A = synth.CSR(p.A.n, p.A.rowptr, p.A.col, p.A.val * scaleA)
    b = p.b_diag
    if scaleB is not None:
        b = (np.ones(A.n) if b is None else b) * scaleB
    kd = None if p.kdiag is None else p.kdiag * scaleA
    pen = _pencil(A, b, kd)
    nx = nx or synth.block_width(p.k, A.n)
    X0 = synth.normal_block(seed, synth.STREAM_X0, A.n, nx)
    Om = synth.normal_block(seed, synth.STREAM_OMEGA, A.n, 16).T
    return pen, L.lobpcg(pen, X0, p.k, p.tol, Om, opts)


# ---------------------------------------------------------------- Sec. 4.1

def _e1():
    g = _golden("e1_worked_example.txt")
    m = int(g["m"][0])
    A = synth.tridiag(m, 3.0, 1.0)
    X0 = np.zeros((m, 2))
    X0[0] = [1, 1]
    X0[1] = [-1, 1]
    X0 /= np.sqrt(2)
    return g, A, _pencil(A), X0


def test_e1_theta0_and_w0():
    g, A, pen, X0 = _e1()
    AX = pen.A_mul(X0)
    np.testing.assert_allclose(X0.T @ AX, np.diag(g["theta0"]), atol=1e-15)
    C, theta = L.rayleigh_ritz(X0.T @ AX, X0.T @ X0)
    np.testing.assert_allclose(theta, g["theta0"], atol=1e-14)
    W0 = AX - X0 * np.array(g["theta0"])
    expect = np.zeros_like(W0)
    expect[int(g["w0_row"][0]) - 1] = g["w0_values"]
    np.testing.assert_allclose(W0, expect, atol=1e-15)


def test_e1_ortho_drop_keeps_one_column_and_ritz_values():
    g, A, pen, X0 = _e1()
    W0 = pen.A_mul(X0) - X0 * np.array(g["theta0"])
    U, BU = L.ortho_drop(pen.B_mul, W0, X0, X0, 100 * L.EPS)
    assert U.shape[1] == int(g["span_dim"][0]) - 2
    e3 = np.zeros(A.n)
    e3[2] = 1
    np.testing.assert_allclose(np.abs(U[:, 0]), e3, atol=1e-15)
    S = np.hstack([X0, U])
    theta = np.linalg.eigvalsh(S.T @ A.to_dense() @ S)
    np.testing.assert_allclose(theta, g["ritz_next"], atol=1e-14)


def test_e1_plain_svqb_gives_spurious_ritz_value():
    """Negative test: Algorithm 4 alone keeps four columns and a zero Ritz value."""
    g, A, pen, X0 = _e1()
    W0 = pen.A_mul(X0) - X0 * np.array(g["theta0"])
    S = np.hstack([X0, W0])
    U = L.svqb(S, S, 4 * L.EPS)
    assert U.shape[1] == 4
    theta = np.linalg.eigvalsh(U.T @ A.to_dense() @ U)
    assert theta[0] < 1e-10 < 1.0 < theta[1]
    assert np.linalg.norm(U.T @ U - np.eye(4)) > 0.5


# ---------------------------------------------------------- contracts

def _rand_metric(n, rng):
    return rng.uniform(1, 2, n)


def test_rayleigh_ritz_contract():
    rng = np.random.default_rng(1)
    n, m = 200, 9
    A = rng.standard_normal((n, n))
    A = A + A.T
    b = _rand_metric(n, rng)
    X = rng.standard_normal((n, m)) * np.logspace(0, 3, m)
    C, theta = L.rayleigh_ritz(X.T @ A @ X, X.T @ (b[:, None] * X))
    Y = X @ C
    np.testing.assert_allclose(Y.T @ (b[:, None] * Y), np.eye(m), atol=1e-12)
    np.testing.assert_allclose(Y.T @ A @ Y, np.diag(theta), atol=1e-10)
    assert np.all(np.diff(theta) >= 0)


def test_rayleigh_ritz_breakdown_on_dependent_columns():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((50, 3))
    X = np.hstack([X, X[:, :1]])
    with pytest.raises(L.Breakdown):
        L.rayleigh_ritz(X.T @ X, X.T @ X)


@pytest.mark.parametrize("deficient", [False, True])
def test_ortho_drop_contract(deficient):
    rng = np.random.default_rng(2)
    n = 300
    b = _rand_metric(n, rng)
    Bm = lambda Y: b[:, None] * Y
    V0 = rng.standard_normal((n, 6))
    C, _ = L.rayleigh_ritz(V0.T @ V0, V0.T @ Bm(V0))
    V = V0 @ C
    U0 = rng.standard_normal((n, 8))
    if deficient:
        U0 = np.hstack([U0, U0[:, :3] @ rng.standard_normal((3, 4)) + 1e-13 * rng.standard_normal((n, 4)),
                        V[:, :2]])
    U, BU = L.ortho_drop(Bm, U0, V, Bm(V), 100 * L.EPS)
    k = U.shape[1]
    assert k <= U0.shape[1]
    # Algorithm 5's first inner pass (svqb with replacement) may keep roundoff
    # directions as orthonormal columns, so only the contracts are pinned.
    np.testing.assert_allclose(U.T @ Bm(U), np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V.T @ Bm(U), 0, atol=1e-12)
    # span([U, V]) contains span(U0) (up to the dropped roundoff directions)
    Q = np.hstack([V, U])
    proj = Q @ (Q.T @ Bm(U0))
    rel = np.linalg.norm(U0 - proj, axis=0) / np.linalg.norm(U0, axis=0)
    assert rel.max() < 1e-10


def test_svqb_drop_span_equality():
    rng = np.random.default_rng(3)
    n = 100
    U = rng.standard_normal((n, 5))
    U = np.hstack([U, U @ rng.standard_normal((5, 2))])
    out = L.svqb_drop(U, U, 7 * L.EPS)
    assert out.shape[1] == 5
    np.testing.assert_allclose(out.T @ out, np.eye(5), atol=1e-12)
    np.testing.assert_allclose(out @ (out.T @ U), U, atol=1e-11)


def _random_projected(rng, nx, np_, nw, orthonormal):
    n = 400
    A = rng.standard_normal((n, n))
    A = A + A.T
    b = rng.uniform(1, 2, n)
    S = rng.standard_normal((n, nx + np_ + nw))
    if orthonormal:
        C, _ = L.rayleigh_ritz(S.T @ S, S.T @ (b[:, None] * S))
        S = S @ C
    return S.T @ A @ S, S.T @ (b[:, None] * S)


@pytest.mark.parametrize("use_ortho,nc", [(False, 0), (False, 3), (True, 0), (True, 2)])
def test_rayleigh_ritz_modified_contract(use_ortho, nc):
    rng = np.random.default_rng(4)
    nx, np_, nw = 8, 8 - nc, 8 - nc
    SAS, SBS = _random_projected(rng, nx, np_, nw, use_ortho)
    rr = L.rayleigh_ritz_modified(SAS, SBS, nx, nc, use_ortho)
    assert not rr.flip
    C = np.hstack([rr.Cx, rr.Cp])
    assert C.shape == (nx + np_ + nw, 2 * nx - nc)
    np.testing.assert_allclose(C.T @ SBS @ C, np.eye(2 * nx - nc), atol=1e-10)
    G = C.T @ SAS @ C
    np.testing.assert_allclose(G[:nx, :nx], np.diag(rr.theta), atol=1e-9)
    np.testing.assert_allclose(G[:nx, nx:], 0, atol=1e-9)
    np.testing.assert_allclose(G[nx:, nx:], rr.PAP, atol=1e-9)
    # X is the Ritz block: the lowest n_x Ritz values of the pencil
    w, _ = dense.pencil_eigh(SAS, SBS, use_jacobi=True)
    np.testing.assert_allclose(rr.theta, w[:nx], atol=1e-9)


def test_rayleigh_ritz_modified_flips_on_ill_conditioning():
    rng = np.random.default_rng(5)
    SAS, SBS = _random_projected(rng, 4, 0, 4, False)
    # make the W block nearly dependent on X in the B metric
    T = np.eye(8)
    T[:4, 4:] = 1.0
    T[4:, 4:] = 1e-7 * np.eye(4)
    rr = L.rayleigh_ritz_modified(T.T @ SAS @ T, T.T @ SBS @ T, 4, 0, False)
    assert rr.flip and rr.condR > 1e4


def test_cp_reduces_to_lq_form_without_locking():
    """With n_c = 0 the C_p reading spans the rows of Z_1perp (Sec. 4.2, LQ form)."""
    rng = np.random.default_rng(6)
    nx = 5
    SAS, SBS = _random_projected(rng, nx, nx, nx, True)
    rr = L.rayleigh_ritz_modified(SAS, SBS, nx, 0, True)
    _, Z = np.linalg.eigh(SAS)
    Z1p = Z[:nx, nx:]
    Qt, _ = np.linalg.qr(Z1p.T)           # orthonormal basis of the rows of Z_1perp
    Cp_lq = Z[:, nx:] @ Qt
    # same column space
    P1 = rr.Cp @ rr.Cp.T
    P2 = Cp_lq @ Cp_lq.T
    np.testing.assert_allclose(P1, P2, atol=1e-10)


# ---------------------------------------------------------- convergence control

def test_norm_estimate_bounds():
    A = synth.laplacian_2d_dirichlet(20)
    pen = _pencil(A)
    Om = synth.normal_block(0, synth.STREAM_OMEGA, A.n, 16).T
    est = L.norm_estimate(pen.A_mul, Om)
    true = np.linalg.norm(A.to_dense(), 2)
    assert 0.3 * true < est <= true
    I3 = synth.CSR(A.n, np.arange(A.n + 1, dtype=np.int32), np.arange(A.n, dtype=np.int32),
                   np.full(A.n, -3.0))
    assert abs(L.norm_estimate(_pencil(I3).A_mul, Om) - 3.0) < 1e-14


def test_backward_error_scale_invariance_and_contrasts():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((50, 3))
    R = 1e-9 * rng.standard_normal((50, 3))
    th = np.array([1e-14, 0.5, 2.0])
    be = L.backward_error(R, X, th, 10.0, 1.0)
    be2 = L.backward_error(5 * R, X, 5 * th / 0.5, 50.0, 0.5)  # (5A, 0.5B)
    np.testing.assert_allclose(be, be2, rtol=1e-14)
    # criterion (7) cannot be met for a ~1e-14 eigenvalue; (9) can
    c7 = L.criterion7(R, X, th)
    assert c7[0] > 1e-4 and be[0] < 1e-8
    # criterion (8) with B scaled by 1e-10: passes trivially, (9) does not
    Xb = X
    BX = 1e-10 * Xb
    Rb = rng.standard_normal((50, 3))
    thb = np.array([1e10, 2e10, 3e10])
    assert np.all(L.criterion8(Rb, Xb, BX, thb) < 1e-4)
    assert np.all(L.backward_error(Rb, Xb, thb, 1.0, 1e-10) > 1e-4)


# ---------------------------------------------------------- Algorithm 8

@pytest.fixture(scope="module")
def c1_run():
    p = synth.make_problem("lap2d_32")
    pen, r = _run(p)
    return p, pen, r


def test_c1_closed_form(c1_run):
    p, pen, r = c1_run
    assert r.status == L.OK
    np.testing.assert_allclose(r.lam, p.closed_form[:8], rtol=1e-10)
    assert np.all(r.be <= p.tol)
    np.testing.assert_allclose(r.X.T @ r.X, np.eye(8), atol=1e-12)
    np.testing.assert_allclose(r.X.T @ pen.A_mul(r.X), np.diag(r.lam), atol=1e-12)
    # the returned backward errors are the true explicit ones of Eq. (9)
    R = pen.A_mul(r.X) - r.X * r.lam
    np.testing.assert_allclose(L.backward_error(R, r.X, r.lam, r.normA, r.normB), r.be,
                               rtol=1e-6, atol=1e-15)
    # Eq. (9) with the true 2-norm is at least as strict as with the estimate
    assert r.normA <= 7.981887690292338 + 1e-12
    assert 10 < r.iters < 400


def test_c1_sign_normalisation(c1_run):
    _, _, r = c1_run
    idx = np.argmax(np.abs(r.X), axis=0)
    assert np.all(r.X[idx, np.arange(8)] > 0)


def test_brute_force_generalised_small():
    rng_b = synth.uniform_block(3, synth.STREAM_BDIAG, 144, 1.0, 2.0)
    A = synth.add_diagonal(synth.laplacian_2d_dirichlet(12),
                           synth.uniform_block(3, synth.STREAM_POTENTIAL, 144))
    p = synth.Problem("bf", A, 10, 1e-10, b_diag=rng_b, kdiag=A.diagonal())
    pen, r = _run(p, seed=3)
    assert r.status == L.OK
    w, _ = dense.pencil_eigh(A.to_dense(), np.diag(rng_b))
    np.testing.assert_allclose(r.lam, w[:10], rtol=1e-10)
    np.testing.assert_allclose(r.X.T @ (rng_b[:, None] * r.X), np.eye(10), atol=1e-12)


def test_scaling_invariance():
    p = synth.make_problem("lap2d_32")
    p.A = synth.laplacian_2d_dirichlet(16)
    p.kdiag = p.A.diagonal()
    p.k = 6
    _, r1 = _run(p)
    _, r2 = _run(p, scaleA=8.0, scaleB=0.25)
    np.testing.assert_allclose(r2.lam, r1.lam * 32.0, rtol=1e-10)
    assert abs(r1.iters - r2.iters) <= 1


def test_direct_gram_mode_agrees():
    p = synth.make_problem("lap3d_64_diagB", N=8, k=6)
    _, r1 = _run(p)
    _, r2 = _run(p, opts=L.Options(direct_gram=True))
    np.testing.assert_allclose(r1.lam, r2.lam, rtol=1e-10)


def test_generalised_closed_form_b_constant():
    p = synth.make_problem("lap3d_64_diagB", N=8, k=6)
    p.b_diag = np.full(p.A.n, 2.0)
    _, r = _run(p)
    ref = synth.problems.closed_form_laplacian((8, 8, 8), 6) / 2.0
    np.testing.assert_allclose(r.lam, ref, rtol=1e-10)


def test_forced_orthogonalisation_path():
    """tau_skip = 1 forces the orthoDrop branch from the first iteration."""
    p = synth.make_problem("lap3d_64_diagB", N=8, k=6)
    _, r = _run(p, opts=L.Options(tau_skip=1.0))
    assert r.stats["flip_iter"] == 1 and r.stats["ortho_calls"] >= r.iters
    _, r0 = _run(p)
    np.testing.assert_allclose(r.lam, r0.lam, rtol=1e-10)


def test_explicit_products_agree():
    p = synth.make_problem("lap2d_32")
    _, r1 = _run(p, opts=L.Options(implicit="never"))
    np.testing.assert_allclose(r1.lam, p.closed_form[:8], rtol=1e-10)


def test_periodic_hamiltonian_singular_a():
    """V = 0: lambda_1 = 0 exactly; criterion (9) still converges."""
    N = 6
    A = synth.hamiltonian_3d_periodic(N, np.zeros(N ** 3))
    p = synth.Problem("h0", A, 7, 1e-8, kdiag=None)
    _, r = _run(p)
    assert r.status == L.OK and abs(r.lam[0]) < 1e-12
    j = np.arange(N)
    one = 2.0 * np.sin(np.pi * j / N) ** 2
    ref = np.sort((one[:, None, None] + one[None, :, None] + one[None, None, :]).ravel())
    np.testing.assert_allclose(r.lam, ref[:7], atol=1e-10)


def test_breakdown_and_not_converged():
    A = synth.laplacian_2d_dirichlet(10)
    pen = _pencil(A)
    X0 = synth.normal_block(0, 1, A.n, 4)
    X0[:, 3] = X0[:, 1]
    Om = synth.normal_block(0, 5, A.n, 16).T
    assert L.lobpcg(pen, X0, 2, 1e-8, Om).status == L.BREAKDOWN
    X0 = synth.normal_block(0, 1, A.n, 4)
    r = L.lobpcg(pen, X0, 2, 1e-8, Om, L.Options(maxit=3))
    assert r.status == L.NOT_CONVERGED and r.iters == 3


def test_csr_metric_closed_form_and_brute_force():
    """Sparse B (I + c * grid adjacency): the pencil with the 2D Laplacian has
    the closed form (4 - mu) / (1 + c mu); the closed form itself is checked
    against the dense pencil solver on a small grid."""
    N, c = 6, 0.2
    A = synth.laplacian_2d_dirichlet(N)
    B = synth.mass_matrix_2d(N, c)
    w, _ = dense.pencil_eigh(A.to_dense(), B.to_dense(), use_jacobi=True)
    np.testing.assert_allclose(w, synth.closed_form_mass_pencil(N, c, N * N), rtol=1e-12)
    N, k = 20, 6
    A = synth.laplacian_2d_dirichlet(N)
    B = synth.mass_matrix_2d(N, c)
    pen = L.Pencil(A.n, (A.rowptr, A.col, A.val), (B.rowptr, B.col, B.val), A.diagonal())
    nx = synth.block_width(k)
    X0 = synth.normal_block(0, synth.STREAM_X0, A.n, nx)
    Om = synth.normal_block(0, synth.STREAM_OMEGA, A.n, 16).T
    r = L.lobpcg(pen, X0, k, 1e-10, Om)
    assert r.status == L.OK
    np.testing.assert_allclose(r.lam, synth.closed_form_mass_pencil(N, c, k), rtol=1e-9)
    Bd = B.to_dense()
    np.testing.assert_allclose(r.X.T @ Bd @ r.X, np.eye(k), atol=1e-12)


# ---------------------------------------------------- HL comparison variants

def test_ortho_algorithm3_contract():
    """Algorithm 3: the output is B-orthonormal, B-orthogonal to V, and keeps
    every column (svqb replaces small singular values instead of dropping)."""
    rng = np.random.default_rng(4)
    n = 150
    b = _rand_metric(n, rng)
    V = rng.standard_normal((n, 5))
    V, _ = L.ortho(lambda Y: b[:, None] * Y, V, np.zeros((n, 0)), np.zeros((n, 0)), 100 * L.EPS)
    U = rng.standard_normal((n, 7))
    U[:, 6] = U[:, 0] + 1e-9 * U[:, 1]  # nearly dependent column
    Uo, BUo = L.ortho(lambda Y: b[:, None] * Y, U, V, b[:, None] * V, 100 * L.EPS)
    assert Uo.shape[1] == 7
    np.testing.assert_allclose(Uo.T @ BUo, np.eye(7), atol=1e-10)
    np.testing.assert_allclose(V.T @ (b[:, None] * Uo), 0.0, atol=1e-12)


def test_rayleigh_ritz_hl_cp_is_orthonormal_and_orthogonal_to_cx():
    rng = np.random.default_rng(5)
    ns, nx, nc = 24, 8, 2
    M = rng.standard_normal((ns, ns))
    SAS = M @ M.T
    rr = L.rayleigh_ritz_hl(SAS, nx, nc)
    C = np.hstack([rr.Cx, rr.Cp])
    np.testing.assert_allclose(C.T @ C, np.eye(C.shape[1]), atol=1e-12)
    np.testing.assert_allclose(rr.Cx.T @ SAS @ rr.Cx, np.diag(rr.theta), atol=1e-10)
    np.testing.assert_allclose(rr.PAP, rr.Cp.T @ SAS @ rr.Cp, atol=1e-12)
    assert rr.Cp.shape[1] == nx - nc


@pytest.mark.parametrize("basis", ["chl", "ahl"])
def test_hl_variants_reach_the_closed_form_on_c1(basis):
    p = synth.make_problem("lap2d_32")
    _, r = _run(p, opts=L.Options(basis=basis))
    assert r.status == L.OK
    np.testing.assert_allclose(r.lam, p.closed_form[:p.k], rtol=1e-10)
    assert r.stats["ortho_calls"] == r.iters  # HL orthogonalises W on every iteration


@pytest.mark.parametrize("basis", ["chl", "ahl"])
def test_hl_variants_agree_with_algorithm8_generalised(basis):
    p = synth.make_problem("lap3d_64_diagB", N=8, k=6)
    _, r8 = _run(p)
    _, rh = _run(p, opts=L.Options(basis=basis))
    assert rh.status == L.OK
    np.testing.assert_allclose(rh.lam, r8.lam, rtol=1e-10)


# ---------------------------------------------------- Chebyshev preconditioner

def _spd_with_spectrum(n, w, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return Q @ np.diag(w) @ Q.T


def test_chebyshev_precond_degree_one_is_scaled_jacobi():
    import scipy.sparse as sp_
    A = sp_.csr_matrix(_spd_with_spectrum(20, np.linspace(1, 3, 20), 1) + 5 * np.eye(20))
    R = np.random.default_rng(2).standard_normal((20, 3))
    K = L.chebyshev_precond(A, 1, 0.5, 2.5)
    np.testing.assert_allclose(K(R), R / A.diagonal()[:, None] / 1.5, rtol=1e-15)


def test_chebyshev_precond_error_bound_and_symmetry():
    """For D = I (unit diagonal) and the spectrum inside [lmin, lmax], the
    Chebyshev iteration's error after k steps is at most 2 q^k ||A^-1 r||_A
    in the A-norm, q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1) (Saad, Eq.
    12.14), and K^-1 = p(A) is symmetric."""
    import scipy.sparse as sp_
    n = 40
    w = np.linspace(0.2, 1.8, n)
    M = _spd_with_spectrum(n, w, 3)
    d = np.sqrt(np.diag(M))
    A = M / d[:, None] / d[None, :]          # unit diagonal, D^-1 A = A
    lam = np.linalg.eigvalsh(A)
    lmin, lmax = lam[0] * 0.999, lam[-1] * 1.001
    Asp = sp_.csr_matrix(A)
    r = np.random.default_rng(4).standard_normal((n, 1))
    x = np.linalg.solve(A, r)
    kappa = lmax / lmin
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    anorm = lambda v: float(np.sqrt((v.T @ A @ v).item()))
    for k in (2, 5, 10, 20):
        e = L.chebyshev_precond(Asp, k, lmin, lmax)(r) - x
        assert anorm(e) <= 2 * q ** k * anorm(x) * (1 + 1e-10)
    K = L.chebyshev_precond(Asp, 6, lmin, lmax)
    Kmat = K(np.eye(n))
    np.testing.assert_allclose(Kmat, Kmat.T, atol=1e-12)
    assert np.linalg.eigvalsh(Kmat)[0] > 0


def test_lobpcg_with_chebyshev_precond_converges_faster():
    import scipy.sparse as sp_
    p = synth.make_problem("lap2d_32")
    A = sp_.csr_matrix((p.A.val, p.A.col, p.A.rowptr), shape=(p.n, p.n))
    K = L.chebyshev_precond(A, 4, 0.05, 2.0)   # D^-1 A of the Laplacian lies in (0, 2)
    pen = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), None, None, k_fn=K)
    nx = synth.block_width(p.k, p.n)
    X0 = synth.normal_block(0, synth.STREAM_X0, p.n, nx)
    Om = synth.normal_block(0, synth.STREAM_OMEGA, p.n, 16).T
    r = L.lobpcg(pen, X0, p.k, p.tol, Om)
    assert r.status == L.OK
    np.testing.assert_allclose(r.lam, p.closed_form[:p.k], rtol=1e-10)
    _, rj = _run(p)
    assert r.iters < rj.iters


def test_zero_b_norm_column_reading():
    """A column of zero B-norm gets D_jj = 0 (Algorithm 4 leaves D undefined
    there): svqb (Algorithm 4) returns it as a zero column beside B-orthonormal
    ones, svqbDrop (Algorithm 6) drops it through its own threshold, and
    orthoDrop (Algorithm 5) returns a B-orthonormal block without it."""
    rng = np.random.default_rng(7)
    n = 200
    b = _rand_metric(n, rng)
    Bm = lambda Y: b[:, None] * Y
    U = rng.standard_normal((n, 5))
    U[:, 2] = 0.0
    T = L.svqb(U, Bm(U), n * L.EPS)
    # the zero column comes out as rounding (eigenvector mixing of ~eps,
    # divided by the replaced sqrt(theta)): zero up to 1e-8
    norms = np.sqrt(np.einsum("ij,ij->j", T, Bm(T)))
    assert np.sum(norms < 1e-8) == 1 and np.all(np.isfinite(T))
    Tk = T[:, norms >= 1e-8]
    np.testing.assert_allclose(Tk.T @ Bm(Tk), np.eye(4), atol=1e-12)
    Td = L.svqb_drop(U, Bm(U), n * L.EPS)
    assert Td.shape[1] == 4
    np.testing.assert_allclose(Td.T @ Bm(Td), np.eye(4), atol=1e-12)
    V0 = rng.standard_normal((n, 3))
    C, _ = L.rayleigh_ritz(V0.T @ V0, V0.T @ Bm(V0))
    V = V0 @ C
    W, BW = L.ortho_drop(Bm, U, V, Bm(V), 100 * L.EPS)
    assert W.shape[1] == 4
    np.testing.assert_allclose(W.T @ Bm(W), np.eye(4), atol=1e-12)
    np.testing.assert_allclose(V.T @ Bm(W), 0, atol=1e-12)


def _random_sparse_symmetric(n, seed, per_row=4, stream=synth.STREAM_COEF):
    """A random sparse symmetric CSR matrix from the seeded generator: about
    per_row off-diagonal pairs per row with N(0, 1) values and a N(0, 1)
    diagonal (so the spectrum is indefinite)."""
    import scipy.sparse as sp
    m = n * per_row
    u = synth.uniform_block(seed, stream, 2 * m)
    i = np.minimum((u[:m] * n).astype(np.int64), n - 1)
    j = np.minimum((u[m:] * n).astype(np.int64), n - 1)
    v = synth.normal_flat(seed, stream, 2 * m, m)
    d = synth.normal_flat(seed, stream, 3 * m, n)
    S = sp.coo_matrix((v, (i, j)), shape=(n, n)).tocsr()
    S = S + S.T + sp.diags(d)
    S = sp.csr_matrix(S)
    S.sort_indices()
    return S


def _csr(S):
    return synth.CSR(S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32),
                     S.data.astype(np.float64))


@pytest.mark.parametrize("n,k,bkind,seed", [(40, 3, "identity", 11), (90, 6, "diag", 12),
                                            (160, 4, "csr", 13), (200, 8, "diag", 14),
                                            (120, 1, "csr", 15)])
def test_brute_force_random_pencils(n, k, bkind, seed):
    """Algorithm 8 on random sparse symmetric A (indefinite) with B = I, a
    diagonal B ~ U[1, 2] or a sparse SPD B = I + 0.1 (S + S^T) / ||S + S^T||_inf,
    against a dense generalised eigensolver (LAPACK through scipy, independent
    of the oracle): lambda within the first-order bound of Eq. (9)'s residual,
    X^T B X = I, and Eq. (9) recomputed on the returned pairs."""
    import scipy.linalg as sla
    import scipy.sparse as sp
    S = _random_sparse_symmetric(n, seed)
    A = _csr(S)
    Ad = S.toarray()
    if bkind == "identity":
        b, Bd = None, np.eye(n)
    elif bkind == "diag":
        b = synth.uniform_block(seed, synth.STREAM_BDIAG, n, 1.0, 2.0)
        Bd = np.diag(b)
    else:
        T = _random_sparse_symmetric(n, seed + 100, per_row=2, stream=synth.STREAM_POTENTIAL)
        T = T - sp.diags(T.diagonal())
        T = T * (0.1 / abs(T).sum(axis=1).max())
        Bm = sp.csr_matrix(sp.identity(n) + T)
        Bm.sort_indices()
        b = (Bm.indptr.astype(np.int32), Bm.indices.astype(np.int32), Bm.data)
        Bd = Bm.toarray()
    kdiag = np.abs(Ad.diagonal()) + 1.0
    pen = L.Pencil(n, (A.rowptr, A.col, A.val), b, kdiag)
    nx = synth.block_width(k, n)
    X0 = synth.normal_block(seed, synth.STREAM_X0, n, nx)
    Om = synth.normal_block(seed, synth.STREAM_OMEGA, n, 16).T
    tol = 1e-10
    r = L.lobpcg(pen, X0, k, tol, Om)
    assert r.status == L.OK, r.status
    w = sla.eigh(Ad, Bd, eigvals_only=True, subset_by_index=[0, k - 1])
    X = r.X[:, :k]
    BX = Bd @ X
    np.testing.assert_allclose(X.T @ BX, np.eye(k), atol=1e-12)
    R = Ad @ X - BX * r.lam[None, :]
    # Eq. (9) on the returned pairs with the solve's own norm estimates
    be = np.linalg.norm(R, axis=0) / (
        (r.normA + np.abs(r.lam) * r.normB) * np.linalg.norm(X, axis=0))
    assert np.all(be <= tol * (1 + 1e-6)), be.max()
    # a pair with B-residual r has an eigenvalue within ||r||_{B^-1} / ||x||_B;
    # here ||x||_B = 1 and ||r||_{B^-1} <= ||r|| / sqrt(lambda_min(B))
    lmin_b = np.linalg.eigvalsh(Bd)[0]
    bound = np.linalg.norm(R, axis=0) / np.sqrt(lmin_b) + 1e-13 * np.abs(w).max()
    assert np.all(np.abs(r.lam - w) <= bound), (np.abs(r.lam - w) / bound).max()


class _Fp32Products(L.Pencil):
    """The pencil with every product A X rounded as an FP32 sparse product
    (values and block in FP32): a model of an FP32-storage form."""

    def A_mul(self, X):
        return np.asarray(self.A.astype(np.float32) @ X.astype(np.float32), dtype=np.float64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp32_a_products_level_off_above_tol_1e8(seed):
    """With A X rounded to FP32 the residual of Eq. (9) carries errors of
    order 2^-24 ||A|| ||x||: Algorithm 8 on c1 still reaches backward error
    1e-6 in about the FP64 iteration count, but not 1e-8 within 400
    iterations (the FP64 oracle needs about 100).  Why a form with FP32 A
    products needs an FP64-product phase to report tol 1e-8."""
    p = synth.make_problem("lap2d_32")
    A = p.A
    nx = synth.block_width(p.k, A.n)
    X0 = synth.normal_block(seed, synth.STREAM_X0, A.n, nx)
    Om = synth.normal_block(seed, synth.STREAM_OMEGA, A.n, 16).T
    pen64 = L.Pencil(A.n, (A.rowptr, A.col, A.val), None, A.diagonal())
    r64 = L.lobpcg(pen64, X0, p.k, 1e-8, Om)
    assert r64.status == L.OK and r64.iters < 200
    pen32 = _Fp32Products(A.n, (A.rowptr, A.col, A.val), None, A.diagonal())
    r = L.lobpcg(pen32, X0, p.k, 1e-6, Om, L.Options(maxit=400))
    assert r.status == L.OK and r.iters < 200
    r = L.lobpcg(pen32, X0, p.k, 1e-8, Om, L.Options(maxit=400))
    assert r.status == L.NOT_CONVERGED


@pytest.mark.parametrize("name,kw,seed", [("lap2d_32", {}, 0), ("lap2d_32", {}, 1),
                                          ("lap3d_64_diagB", {"N": 16, "k": 16}, 1)])
def test_two_phase_fp32_then_fp64_schedule(name, kw, seed):
    """A model of a two-phase precision schedule: Algorithm 8 with FP32
    A-products to backward error 1e-5, then the FP64 solve restarted from
    its k vectors (padded with the start block's other columns) to 1e-8.  The two phases together take about the FP64 solve's
    iterations (within 15 %), most of them in the FP32 phase, and reach the
    same eigenvalues."""
    p = synth.make_problem(name, **kw)
    A = p.A
    nx = synth.block_width(p.k, A.n)
    X0 = synth.normal_block(seed, synth.STREAM_X0, A.n, nx)
    Om = synth.normal_block(seed, synth.STREAM_OMEGA, A.n, 16).T
    pen64 = L.Pencil(A.n, (A.rowptr, A.col, A.val), p.b_diag, A.diagonal())
    pen32 = _Fp32Products(A.n, (A.rowptr, A.col, A.val), p.b_diag, A.diagonal())
    r64 = L.lobpcg(pen64, X0, p.k, 1e-8, Om)
    r1 = L.lobpcg(pen32, X0, p.k, 1e-5, Om, L.Options(maxit=400))
    assert r64.status == L.OK and r1.status == L.OK
    # phase 2 starts from the k returned vectors and the remaining start columns
    X1 = np.hstack([r1.X[:, :p.k], X0[:, p.k:]])
    r2 = L.lobpcg(pen64, X1, p.k, 1e-8, Om)
    assert r2.status == L.OK
    assert r1.iters + r2.iters <= 1.15 * r64.iters
    assert r1.iters >= r2.iters
    np.testing.assert_allclose(r2.lam, r64.lam, rtol=1e-11)
