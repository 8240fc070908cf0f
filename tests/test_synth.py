"""Seeded generators: Philox known answers, stencil structure and closed forms."""
import os

import numpy as np
import pytest

import synth
from synth.philox import philox4x32_10, uniform52
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniform52_range_and_resolution():
    u = uniform52(np.array([0, 0xFFFFFFFF], dtype=np.uint64),
                  np.array([0, 0xFFFFFFFF], dtype=np.uint64))
    assert u[0] == 0.5 * 2.0 ** -52
    assert u[1] == 1.0 - 0.5 * 2.0 ** -52
    assert np.all((u > 0) & (u < 1))


def test_streams_are_counter_based():
    a = synth.normal_block(7, synth.STREAM_X0, 40, 6)
    b = synth.normal_block(7, synth.STREAM_X0, 10, 6, row0=30)
    np.testing.assert_array_equal(a[30:], b)
    c = synth.normal_block(8, synth.STREAM_X0, 40, 6)
    assert not np.allclose(a, c)
    x = synth.normal_flat(3, synth.STREAM_OMEGA, 0, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    u = synth.uniform_block(3, synth.STREAM_BDIAG, 100000, 1.0, 2.0)
    assert u.min() > 1.0 and u.max() < 2.0 and abs(u.mean() - 1.5) < 0.01


def _sym(A):
    D = A.to_dense()
    return np.array_equal(D, D.T)


def test_stencil_structure():
    A = synth.laplacian_2d_dirichlet(32)
    assert A.n == 1024 and A.nnz == 4992 and _sym(A)
    A = synth.laplacian_3d_dirichlet(5)
    assert A.nnz == 7 * 125 - 6 * 25 and _sym(A)
    for i in range(A.n):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    B = synth.laplacian_3d_dirichlet(64)
    assert B.n == 262144 and B.nnz == 1810432


def test_laplacian_closed_forms_by_jacobi():
    w, _ = dense.jacobi_eigh(synth.laplacian_2d_dirichlet(6, 5).to_dense())
    np.testing.assert_allclose(w, synth.problems.closed_form_laplacian((6, 5), 30),
                               rtol=0, atol=1e-12)
    w, _ = dense.jacobi_eigh(synth.laplacian_3d_dirichlet(4).to_dense())
    np.testing.assert_allclose(w, synth.problems.closed_form_laplacian((4, 4, 4), 64),
                               rtol=0, atol=1e-12)


def test_c1_closed_form_values():
    lam = synth.problems.closed_form_laplacian((32, 32), 10)
    ref = [0.018112309707662, 0.045198760328417, 0.045198760328417,
           0.072285210949173, 0.090070207624836, 0.090070207624836,
           0.117156658245592, 0.117156658245592, 0.152320288821686,
           0.152320288821686]
    np.testing.assert_allclose(lam, ref, rtol=1e-12)


def test_diffusion_sigma0_is_laplacian():
    A = synth.diffusion_3d_lognormal(5, 0.0, 1)
    L = synth.laplacian_3d_dirichlet(5)
    np.testing.assert_allclose(A.to_dense(), L.to_dense(), atol=0)
    D = synth.diffusion_3d_lognormal(6, 1.0, 2)
    assert _sym(D)
    # diagonally dominant with positive diagonal: row sums equal the boundary faces
    M = D.to_dense()
    assert np.all(np.diag(M) > 0) and np.all(M.sum(1) > -1e-12)


def test_periodic_hamiltonian_constant_potential():
    N, c = 6, 0.7
    H = synth.hamiltonian_3d_periodic(N, np.full(N ** 3, c))
    w, _ = dense.jacobi_eigh(H.to_dense())
    j = np.arange(N)
    one = 2.0 * np.sin(np.pi * j / N) ** 2
    ref = np.sort((one[:, None, None] + one[None, :, None] + one[None, None, :]).ravel())
    np.testing.assert_allclose(w, c + ref, atol=1e-12)


def test_block_width():
    assert synth.block_width(8) == 10
    assert synth.block_width(64) == 71
    assert synth.block_width(1024) == 1127
    assert synth.block_width(32) == 36
