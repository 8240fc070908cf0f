"""CPU pins of the closed-form checks that the full-size GPU tests apply
(tests/closed_form.py): the checker accepts pairs that meet the quadratic
residual bound and rejects the mistakes it exists to catch (a dropped or
doubled member of a degenerate cluster, a value off by more than its
bound), and the oracle's Algorithm 8 passes it on a periodic Hamiltonian
with constant potential whose block edges k and n_x cut through clusters of
equal eigenvalues, as on the 96^3 workload."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from closed_form import closed_form_match, periodic_closed_form
from oracle import lobpcg as L


def _cases():
    yield synth.problems.closed_form_laplacian((128, 128, 128), 320), 256
    yield periodic_closed_form(96, 5.0, 1400), 1024


@pytest.mark.parametrize("case", [0, 1])
def test_checker_accepts_bounded_pairs_and_rejects_planted_mistakes(case):
    ref, k = list(_cases())[case]
    rng = np.random.default_rng(case)
    rn = np.full(k, 1e-7)  # residual norms of the returned pairs
    rho = ref[:k] + rng.uniform(-1, 1, k) * 1e-13
    lam = rho + 4e-12      # Ritz values a little off their vectors' quotients
    e_lam, e_rho = closed_form_match(lam, rho, rn, rn + 4e-12, ref)
    assert e_lam < 1e-11 and e_rho < 1e-12
    # a cluster member dropped: every pair is accurate, the multiset is not
    dropped = np.delete(ref, 5)[:k]
    with pytest.raises(AssertionError):
        closed_form_match(dropped, dropped, rn, rn, ref)
    # a member counted twice (the next distinct value missing at the top)
    doubled = np.sort(np.concatenate([ref[:1], ref[:k - 1]]))
    with pytest.raises(AssertionError):
        closed_form_match(doubled, doubled, rn, rn, ref)
    # a vector's quotient off by more than ||r||^2 / delta
    off = ref[:k].copy()
    off[3] += 1e-6
    with pytest.raises(AssertionError):
        closed_form_match(off, off, rn, rn, ref)
    # a Ritz value off by more than its residual allows
    with pytest.raises(AssertionError):
        closed_form_match(lam + 1e-6, rho, rn, rn, ref)


def test_periodic_closed_form_matches_dense_eigenvalues():
    N, c = 6, 0.7
    H = synth.hamiltonian_3d_periodic(N, np.full(N ** 3, c))
    A = sp.csr_matrix((H.val, H.col, H.rowptr), shape=(H.n, H.n)).toarray()
    np.testing.assert_allclose(np.linalg.eigvalsh(A), periodic_closed_form(N, c, N ** 3),
                               atol=1e-12)


def test_oracle_passes_with_block_edges_inside_clusters():
    """8^3 torus, V = 2: the spectrum 2 + sums of 2 sin^2(pi j / 8) has a
    12-fold cluster at indices 7-18; k = 10 and n_x = 12 both fall inside
    it."""
    N, c, k = 8, 2.0, 10
    H = synth.hamiltonian_3d_periodic(N, np.full(N ** 3, c))
    ref = periodic_closed_form(N, c, 64)
    nx = synth.block_width(k)
    u = np.abs(ref - ref[k - 1]) < 1e-12
    assert u[k - 1] and u[k] and u[nx - 1] and u[nx]
    pen = L.Pencil(H.n, (H.rowptr, H.col, H.val), None, H.diagonal())
    X0 = synth.normal_block(0, synth.STREAM_X0, H.n, nx)
    Om = synth.normal_block(0, synth.STREAM_OMEGA, H.n, 16).T
    r = L.lobpcg(pen, X0, k, 1e-8, Om)
    assert r.status == L.OK
    A = sp.csr_matrix((H.val, H.col, H.rowptr), shape=(H.n, H.n))
    X = r.X[:, :k]
    AX = A @ X
    xx = (X * X).sum(0)
    rho = (X * AX).sum(0) / xx
    rn_rho = np.linalg.norm(AX - X * rho, axis=0) / np.sqrt(xx)
    rn_lam = np.linalg.norm(AX - X * r.lam[:k], axis=0) / np.sqrt(xx)
    closed_form_match(r.lam[:k], rho, rn_rho, rn_lam, ref)
    assert np.abs(X.T @ X - np.eye(k)).max() < 1e-12
