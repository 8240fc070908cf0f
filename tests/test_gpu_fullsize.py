"""Full-size parity against the stored oracle eigenvalues.

tests/golden/oracle_lambda_<workload>.txt holds the eigenvalues the CPU
oracle (plain FP64 Algorithm 8) reached on the full workload with the same
seeded X0 and sketch Omega, written by tests/golden/make_oracle_lambda.py.
The GPU solve of the same input must match them per eigenvalue: to relative
1e-10 in the FP64 form and with 7-slice contractions, to 1e-9 with the
default 6 slices (each emulated product is exact to 2^-44 relative to its
block maxima, and the iteration stops at the same backward error 1e-8, so the
Ritz values agree to ~1e-10 but not to the FP64 form's margin); and the
returned pairs must satisfy the explicit FP64 Eq. (9) on the host.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
import paper_1704_07458_gb300 as gb
from oracle import lobpcg as L
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(workload):
    lam = {}
    meta = {}
    for line in open(os.path.join(GOLDEN, f"oracle_lambda_{workload}.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "lambda":
            lam[int(f[1])] = float(f[2])
        else:
            meta[f[0]] = float(f[1])
    return np.array([lam[i] for i in range(len(lam))]), meta


def _solve(p, **opts):
    torch = torch_cuda()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = gb.Solver(**opts)
    s.set_operator(dev(p.A.rowptr), dev(p.A.col), dev(p.A.val),
                   b_diag=None if p.b_diag is None else dev(p.b_diag))
    nx = synth.block_width(p.k, p.n)
    X0 = dev(synth.normal_block(0, synth.STREAM_X0, p.n, nx))
    lam, X, it, be, rc = s.solve(p.k, p.tol, X0=X0, device=True, raise_on_error=False)
    st = s.stats()
    s.close()
    return (lam.cpu().numpy(), X.cpu().numpy(), int(it), be.cpu().numpy(), rc, st)


def _solve_dev(p, **opts):
    """As _solve, outputs left on the device (torch tensors)."""
    torch = torch_cuda()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = gb.Solver(**opts)
    s.set_operator(dev(p.A.rowptr), dev(p.A.col), dev(p.A.val),
                   b_diag=None if p.b_diag is None else dev(p.b_diag))
    nx = synth.block_width(p.k, p.n)
    X0 = dev(synth.normal_block(0, synth.STREAM_X0, p.n, nx))
    lam, X, it, be, rc = s.solve(p.k, p.tol, X0=X0, device=True, raise_on_error=False)
    st = s.stats()
    s.close()
    return lam, X, int(it), be, rc, st


def _check_eq9(p, lam, X, normA, normB):
    A = sp.csr_matrix((p.A.val, p.A.col, p.A.rowptr), shape=(p.n, p.n))
    BX = X if p.b_diag is None else p.b_diag[:, None] * X
    R = A @ X - BX * lam[None, :]
    ref = L.backward_error(R, X, lam, normA, normB)
    assert np.all(ref <= p.tol * (1 + 1e-6)), ref.max()
    return np.abs(X.T @ BX - np.eye(p.k)).max()


@pytest.mark.parametrize("form,opts,rtol", [
    ("fp64", dict(gemm_mode="f64"), 1e-10),
    ("bf16x7", dict(gemm_mode="ozaki_tc", ozaki_slices=7), 1e-10),
    ("bf16x6", dict(gemm_mode="ozaki_tc"), 1e-9),
])
def test_c2_full_size_matches_stored_oracle(form, opts, rtol):
    """64^3 Laplacian with diagonal B ~ U[1, 2], k = 64, tol 1e-8."""
    p = synth.make_problem("lap3d_64_diagB")
    ref, meta = _golden("lap3d_64_diagB")
    lam, X, it, be, rc, st = _solve(p, **opts)
    assert rc == gb.LOBPCG_OK, rc
    np.testing.assert_allclose(st["norm_a"], meta["norm_a"], rtol=1e-12)
    np.testing.assert_allclose(st["norm_b"], meta["norm_b"], rtol=1e-12)
    rel = np.abs(lam - ref) / np.abs(ref)
    assert rel.max() <= rtol, (form, rel.max(), int(np.argmax(rel)))
    orth = _check_eq9(p, lam, X, meta["norm_a"], meta["norm_b"])
    assert orth <= 1e-10, orth


def test_c5_full_size_fp64_form_matches_stored_oracle():
    """512^2 Laplacian + V ~ U[0, 1], k = 32, tol 1e-8, FP64 form: the low
    states are localised and nearly degenerate (minimum gap ~1.7e-5), and
    the solve needs more than the paper's 2000 iterations, within the
    library's default cap."""
    p = synth.make_problem("lap2d_512_V")
    ref, meta = _golden("lap2d_512_V")
    lam, X, it, be, rc, st = _solve(p, gemm_mode="f64")  # the default maxit covers it
    assert rc == gb.LOBPCG_OK, rc
    rel = np.abs(lam - ref) / np.abs(ref)
    assert rel.max() <= 1e-10, (rel.max(), int(np.argmax(rel)))
    orth = _check_eq9(p, lam, X, meta["norm_a"], meta["norm_b"])
    assert orth <= 1e-10, orth


def test_c5_full_size_default_form_matches_stored_oracle():
    """The same c5 solve in the default form (6-slice tcgen05 contractions,
    explicit Rayleigh-Ritz after every refresh): eigenvalues within relative
    1e-9 of the oracle's, explicit Eq. (9) on the host, and X^T X = I to
    1e-10 (the explicit Rayleigh-Ritz re-imposes the B-orthonormality that
    the identities (12)-(14) assume)."""
    p = synth.make_problem("lap2d_512_V")
    ref, meta = _golden("lap2d_512_V")
    lam, X, it, be, rc, st = _solve(p, gemm_mode="ozaki_tc")
    assert rc == gb.LOBPCG_OK, rc
    assert st["explicit_rr_calls"] > 0
    rel = np.abs(lam - ref) / np.abs(ref)
    assert rel.max() <= 1e-9, (rel.max(), int(np.argmax(rel)))
    orth = _check_eq9(p, lam, X, meta["norm_a"], meta["norm_b"])
    assert orth <= 1e-10, orth


def _properties_on_device(p, lam, X, st, tol_orth):
    """Explicit FP64 Eq. (9) and X^T X = I for B = I, computed on the device
    with torch's own sparse and dense products (independent of the library)."""
    torch = torch_cuda()
    A = torch.sparse_csr_tensor(torch.from_numpy(p.A.rowptr.astype(np.int64)),
                                torch.from_numpy(p.A.col.astype(np.int64)),
                                torch.from_numpy(p.A.val), size=(p.n, p.n)).cuda()
    R = (A @ X) - X * lam[None, :]
    be = torch.linalg.norm(R, dim=0) / (
        (st["norm_a"] + lam.abs() * st["norm_b"]) * torch.linalg.norm(X, dim=0))
    del R
    assert float(be.max()) <= p.tol * (1 + 1e-6), float(be.max())
    G = X.T @ X
    G -= torch.eye(p.k, dtype=G.dtype, device=G.device)
    orth = float(G.abs().max())
    assert orth <= tol_orth, orth
    assert bool(torch.all(lam[1:] >= lam[:-1] - 1e-14))
    return float(be.max()), orth


def test_c3_full_size_properties():
    """128^3 log-normal diffusion (sigma = 1), B = I, Jacobi K, k = 256,
    tol 1e-8, default form: explicit Eq. (9), X^T X = I, and the spectrum of
    the SPD operator positive.  No closed form: the oracle's eigenvalues are
    compared at 16^3 in test_gpu_solve."""
    p = synth.make_problem("diffusion_128")
    lam, X, it, be, rc, st = _solve_dev(p, gemm_mode="ozaki_tc")
    assert rc == gb.LOBPCG_OK, rc
    bmax, orth = _properties_on_device(p, lam, X, st, 1e-10)
    assert float(lam[0]) > 0
    print(f"c3: {it} iterations, max backward error {bmax:.3e}, |X^T X - I| {orth:.2e}")


def test_c4_full_size_properties():
    """-1/2 Laplacian (periodic 96^3) + V, V ~ U[0, 10], k = 1024 (n_x = 1127,
    projected pencils of order up to 3381), tol 1e-8, default form: explicit
    Eq. (9), X^T X = I, and 0 <= lambda <= 16 (the spectrum of -1/2 Laplacian
    lies in [0, 6], V in [0, 10])."""
    p = synth.make_problem("hamiltonian_96")
    lam, X, it, be, rc, st = _solve_dev(p, gemm_mode="ozaki_tc")
    assert rc == gb.LOBPCG_OK, rc
    bmax, orth = _properties_on_device(p, lam, X, st, 1e-10)
    assert float(lam[0]) >= 0 and float(lam[-1]) <= 16
    print(f"c4: {it} iterations, max backward error {bmax:.3e}, |X^T X - I| {orth:.2e}, "
          f"dropped columns {st['dropped_columns']}, switch at {st['flip_iteration']}")
