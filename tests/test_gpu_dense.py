"""Parity of the projected-pencil eigensolver (lobpcg_syev) with LAPACK.

Cases: random symmetric matrices with prescribed spectra (separated,
clustered to 1e-9, exactly degenerate), and the 18 x 18 and 54 x 54 projected
pencils that the oracle's Algorithm 7 builds on the 16^3 generalised pencil.
The bar is that of an FP64 eigensolver: eigenvalues within 1e-13 ||A||,
orthonormality and residual ||A Z - Z diag(w)|| within 1e-13 ||A||.
Modes: 0 cuSOLVER FP64, 1 FP32 cuSOLVER refined, 2 the device-resident
eigensolver with its fallback, 3 the device-resident eigensolver alone (its
own check must pass on every case).
"""
import numpy as np
import pytest

import synth
import paper_1704_07458_gb300 as gb
from oracle import lobpcg as L, dense
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _spectrum_matrix(n, w, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(w) @ Q.T
    return 0.5 * (A + A.T)


def _cases():
    rng = np.random.default_rng(7)
    out = []
    for n in (3, 7, 18, 54, 213, 224, 240):
        out.append(("separated", _spectrum_matrix(n, np.sort(rng.uniform(0, 10, n)), n)))
    w = np.sort(rng.uniform(0, 10, 71))
    w[10:13] = w[10] + np.array([0.0, 1e-9, 2e-12])
    w[40:46] = w[40]
    out.append(("clusters", _spectrum_matrix(71, np.sort(w), 3)))
    w = np.sort(np.concatenate([rng.uniform(1e-14, 1e-12, 5), rng.uniform(0.1, 50, 45)]))
    out.append(("tiny eigenvalues", _spectrum_matrix(50, w, 4)))
    # the spectrum of a Rayleigh-Ritz matrix of the 64^3 pencil: 71 Ritz
    # values in [0.007, 0.08] (one pair 1e-6 apart, one triple 3e-7 apart,
    # below FP32 resolution at this norm) and 142 values in [0.1, 12]
    low = np.sort(rng.uniform(0.007, 0.08, 71))
    low[20] = low[19] + 1e-6
    low[40:43] = low[40] + np.array([0.0, 3e-7, 9e-7])
    w = np.sort(np.concatenate([low, rng.uniform(0.1, 12, 142)]))
    out.append(("ritz-like", _spectrum_matrix(213, w, 5)))
    return out


def _projected():
    """Projected matrices from the oracle's Algorithm 7 on the 16^3 pencil."""
    mats = []
    orig = dense.eigh

    def cap(M):
        if len(mats) < 40:
            mats.append(np.array(M))
        return orig(M)
    L.dense.eigh = cap
    try:
        p = synth.make_problem("lap3d_64_diagB", N=16, k=16)
        nx = synth.block_width(p.k)
        X0 = synth.normal_block(0, synth.STREAM_X0, p.n, nx)
        Om = synth.normal_block(0, synth.STREAM_OMEGA, p.n, 16).T
        pen = L.Pencil(p.n, (p.A.rowptr, p.A.col, p.A.val), p.b_diag, p.kdiag)
        L.lobpcg(pen, X0, p.k, p.tol, Om, L.Options(maxit=30))
    finally:
        L.dense.eigh = orig
    return [("projected", m) for m in mats[::4]]


def _run(A, mode):
    torch = torch_cuda()
    n = A.shape[0]
    At = torch.from_numpy(np.asfortranarray(A).ravel(order="F").copy()).cuda()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    rc = gb.lobpcg_syev(n, At, n, w, mode)
    assert rc == 0, rc
    Z = At.cpu().numpy().reshape(n, n, order="F")
    return w.cpu().numpy(), Z


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_syev_matches_lapack(mode):
    for name, A in _cases() + _projected():
        A = 0.5 * (A + A.T)
        n = A.shape[0]
        wl = np.linalg.eigvalsh(A)
        nA = np.abs(wl).max()
        w, Z = _run(A, mode)
        assert np.all(np.diff(w) >= -1e-13 * nA), name
        assert np.abs(w - wl).max() <= 1e-13 * nA * max(1, n / 50), (name, n, np.abs(w - wl).max())
        assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-13 * max(1, n / 50), (name, n)
        assert np.abs(A @ Z - Z * w).max() <= 1e-13 * nA * max(1, n / 50), (name, n)
