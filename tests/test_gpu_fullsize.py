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
    lam, X, it, be, rc, st = _solve(p)
    assert rc == gb.LOBPCG_OK, rc
    assert st["explicit_rr_calls"] > 0
    rel = np.abs(lam - ref) / np.abs(ref)
    assert rel.max() <= 1e-9, (rel.max(), int(np.argmax(rel)))
    orth = _check_eq9(p, lam, X, meta["norm_a"], meta["norm_b"])
    assert orth <= 1e-10, orth
