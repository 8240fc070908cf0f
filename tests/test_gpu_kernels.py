"""Element-by-element parity of single kernels (through the C ABI) with the oracle.

Tolerances: FP64 kernels reorder sums, so each output is compared with the
classical forward bound |fl(x^T y) - x^T y| <= gamma_n |x|^T |y| (both the
kernel and the reference carry at most that error, hence the factor 2).
"""
import numpy as np
import pytest

import synth
from oracle import kernels as ok
import paper_1704_07458_gb300 as gb
from gpu_util import torch_cuda, dev, host, dev_i32, gamma

pytestmark = pytest.mark.gpu

MODES = [(gb.LOBPCG_GEMM_F64, 0), (gb.LOBPCG_GEMM_OZAKI, 6), (gb.LOBPCG_GEMM_OZAKI, 4),
         (gb.LOBPCG_GEMM_OZAKI, 7), (gb.LOBPCG_GEMM_OZAKI_TC, 6), (gb.LOBPCG_GEMM_OZAKI_TC, 4),
         (gb.LOBPCG_GEMM_OZAKI_TC, 7)]


def ozaki_unit(slices):
    """Per-term error unit of the S-slice split: truncation of the fixed-point
    digits (2^(1-8S) of the chunk maximum, both operands) plus the dropped
    digit pairs of levels above S + 1 (< 4 S 2^(-8S) of the product of maxima),
    with a factor 4 of slack."""
    return 4 * (4 + 4 * slices) * 2.0 ** (-8 * slices)


def _csr_with_empty_rows():
    A = synth.laplacian_2d_dirichlet(9, 7)
    # zero out rows 0, 5 and the last one by rebuilding the CSR without them
    keep = np.ones(A.n, bool)
    keep[[0, 5, A.n - 1]] = False
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    m = keep[rows]
    rp = np.zeros(A.n + 1, np.int64)
    np.add.at(rp, rows[m] + 1, 1)
    return synth.CSR(A.n, np.cumsum(rp).astype(np.int32), A.col[m], A.val[m])


@pytest.mark.parametrize("m", [1, 3, 8, 10, 17, 33, 71, 130])
@pytest.mark.parametrize("which", ["lap2d", "empty_rows", "diffusion"])
def test_spmm_parity(m, which):
    torch = torch_cuda()
    A = {"lap2d": lambda: synth.laplacian_2d_dirichlet(32),
         "empty_rows": _csr_with_empty_rows,
         "diffusion": lambda: synth.diffusion_3d_lognormal(9, 1.0, 4)}[which]()
    X = synth.normal_block(2, synth.STREAM_X0, A.n, m)
    b = synth.uniform_block(2, synth.STREAM_BDIAG, A.n, 1.0, 2.0)
    ld = m + 5
    Xd, Yd, BYd = dev(X, ld), dev(np.zeros((A.n, m)), ld + 3), dev(np.zeros((A.n, m)), ld)
    rc = gb.lobpcg_spmm(A.n, dev_i32(A.rowptr), dev_i32(A.col), dev(A.val), Xd, ld, m, Yd,
                        ld + 3, dev(b), BYd, ld)
    torch.cuda.synchronize()
    assert rc == 0
    ref = ok.spmm(A.rowptr, A.col, A.val, X)
    absref = ok.spmm(A.rowptr, A.col, np.abs(A.val), np.abs(X))
    err = np.abs(host(Yd, m) - ref)
    assert np.all(err <= 2 * gamma(8) * absref + 1e-300)
    np.testing.assert_array_equal(host(BYd, m), b[:, None] * X)
    # padding columns untouched
    assert np.all(host(Yd)[:, m:] == 0)


def test_spmm_full_size_sampled_rows():
    torch = torch_cuda()
    A = synth.laplacian_3d_dirichlet(64)
    m = 71
    Xd = torch.empty((A.n, 72), dtype=torch.float64, device="cuda")
    assert gb.lobpcg_philox_normal(A.n, m, 9, 1, Xd, 72) == 0
    Yd = torch.empty_like(Xd)
    rc = gb.lobpcg_spmm(A.n, dev_i32(A.rowptr), dev_i32(A.col), dev(A.val), Xd, 72, m, Yd, 72)
    torch.cuda.synchronize()
    assert rc == 0
    rows = np.unique(np.concatenate([np.arange(0, A.n, 4099), [A.n - 1, 4095, 4096]]))
    X = synth.normal_block(9, 1, A.n, m)  # same stream, regenerated on the host
    ref = ok.spmm_rows(A.rowptr, A.col, A.val, X, rows)
    got = host(Yd, m)[rows]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,p,q", [(1, 3, 2), (37, 5, 7), (1000, 30, 20), (4099, 71, 142),
                                   (20000, 213, 142)])
@pytest.mark.parametrize("mode,slices", MODES)
def test_gram_parity(n, p, q, mode, slices):
    torch = torch_cuda()
    U = synth.normal_block(3, 1, n, p) * np.logspace(-6, 2, p)[None, :]
    V = synth.normal_block(4, 1, n, q) * np.logspace(3, -5, q)[None, :]
    G = dev(np.full((p + 3) * q, np.nan))  # column-major p x q, leading dimension p + 3
    rc = gb.lobpcg_gram(n, dev(U, p + 1), p + 1, p, dev(V, q + 2), q + 2, q, G, p + 3, mode,
                        slices)
    torch.cuda.synchronize()
    assert rc == 0
    got = host(G).reshape(q, p + 3).T[:p, :]
    ref = ok.gram(U, V)
    bound = 2 * gamma(n) * (np.abs(U).T @ np.abs(V))
    if mode != gb.LOBPCG_GEMM_F64:
        # rows sharing one exponent per column: 64 (mma.sync kernel) or 256
        # (tcgen05 kernel).  Per block c: unit * len * max_c|u_i| * max_c|v_j|
        # (2x for the exponent bound)
        L = 256 if mode == gb.LOBPCG_GEMM_OZAKI_TC else 64
        nck = (n + L - 1) // L
        mu = np.zeros((nck, p)); mv = np.zeros((nck, q))
        for c in range(nck):
            mu[c] = np.abs(U[L * c:L * c + L]).max(0)
            mv[c] = np.abs(V[L * c:L * c + L]).max(0)
        bound = bound + ozaki_unit(slices) * L * 4 * (mu.T @ mv) + 2.0 ** -44 * (np.abs(U).T @ np.abs(V))
        if mode == gb.LOBPCG_GEMM_OZAKI_TC:
            # the tcgen05 kernel sums the blocks of a row slab (<= 64 blocks) in
            # int64 fixed point at the slab's largest exponents: <= 1 unit, i.e.
            # 2^-44 * 2^(E_i + E_j) <= 2^-42 max|u_i| max|v_j|, lost per block
            bound = bound + 64 * 2.0 ** -42 * np.outer(np.abs(U).max(0), np.abs(V).max(0))
    assert np.all(np.abs(got - ref) <= bound + 1e-300)


@pytest.mark.parametrize("n,s,m", [(1, 4, 3), (65, 17, 9), (4099, 213, 142), (3000, 71, 71),
                                   (1500, 530, 97), (700, 300, 96), (2100, 213, 128),
                                   (1300, 150, 113)])
@pytest.mark.parametrize("beta", [0.0, 1.0])
@pytest.mark.parametrize("mode,slices", MODES)
def test_update_parity(n, s, m, beta, mode, slices):
    torch = torch_cuda()
    S = synth.normal_block(5, 1, n, s) * np.logspace(-8, 1, s)[None, :]
    C = synth.normal_block(6, 1, s, m) * np.logspace(8, -1, s)[:, None]
    Y0 = synth.normal_block(7, 1, n, m)
    Cd = dev(np.asfortranarray(C).T.copy().reshape(-1))  # column-major s x m
    Yd = dev(np.zeros((n, m)), m + 1)
    rc = gb.lobpcg_update(n, dev(S, s + 2), s + 2, s, Cd, s, m, -1.0, beta, dev(Y0, m), m, Yd,
                          m + 1, mode, slices)
    torch.cuda.synchronize()
    assert rc == 0
    ref = beta * Y0 - ok.update(S, C)
    bound = 2 * gamma(s + 1) * (np.abs(S) @ np.abs(C) + abs(beta) * np.abs(Y0))
    if mode != gb.LOBPCG_GEMM_F64:
        # columns of S balanced by 2^E_k (E_k its exponent bound), rows of C by 2^-E_k:
        # the balanced S has entries below 1, the balanced C entries below 2 max|S_k| |C_kj|
        Ct = np.abs(C) * (2 * np.abs(S).max(0))[:, None]
        bound = bound + ozaki_unit(slices) * 4 * s * Ct.max(0)[None, :] + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(host(Yd, m) - ref) <= bound + 1e-300)


@pytest.mark.parametrize("s,m", [(213, 142), (71, 40), (300, 96)])
@pytest.mark.parametrize("slices", [6, 7])
def test_update_parity_aligned_rows(s, m, slices):
    """The tcgen05 update with the solver's padded layout: Y rows of
    round_up(m, 8) doubles, so the epilogue's 32-byte stores run; checked
    element by element against U C within the derived bound."""
    torch = torch_cuda()
    n = 3001
    S = synth.normal_block(5, 1, n, s) * np.logspace(-8, 1, s)[None, :]
    C = synth.normal_block(6, 1, s, m) * np.logspace(8, -1, s)[:, None]
    ldy = (m + 7) // 8 * 8
    Cd = dev(np.asfortranarray(C).T.copy().reshape(-1))
    Yd = dev(np.zeros((n, m)), ldy)
    assert Yd.data_ptr() % 32 == 0
    rc = gb.lobpcg_update(n, dev(S, s), s, s, Cd, s, m, 1.0, 0.0, None, 0, Yd, ldy,
                          gb.LOBPCG_GEMM_OZAKI_TC, slices)
    torch.cuda.synchronize()
    assert rc == 0
    ref = ok.update(S, C)
    Ct = np.abs(C) * (2 * np.abs(S).max(0))[:, None]
    bound = (2 * gamma(s + 1) * (np.abs(S) @ np.abs(C)) + ozaki_unit(slices) * 4 * s *
             Ct.max(0)[None, :] + 2.0 ** -52 * np.abs(ref))
    got = host(Yd, m)
    assert np.all(np.abs(got - ref) <= bound + 1e-300)
    assert np.all(host(Yd)[:, m:] == 0)  # the padding columns are not written


@pytest.mark.parametrize("n,m,c0", [(1, 1, 0), (300, 10, 0), (1024, 10, 4), (5000, 71, 70),
                                    (20000, 71, 3)])
@pytest.mark.parametrize("bdiag", [False, True])
def test_residual_parity(n, m, c0, bdiag):
    torch = torch_cuda()
    X = synth.normal_block(8, 1, n, m)
    AX = synth.normal_block(9, 1, n, m)
    b = synth.uniform_block(8, 2, n, 1.0, 2.0)
    BX = b[:, None] * X if bdiag else None
    th = np.linspace(-1, 3, m)
    kd = synth.uniform_block(9, 2, n, 2.0, 6.0)
    W = dev(np.full((n, m - c0), np.nan), m)
    be = dev(np.zeros(m - c0))
    rc = gb.lobpcg_residual(n, dev(X, m + 1), dev(AX, m + 1), None if BX is None else dev(BX, m + 1),
                            m + 1, m, c0, dev(th), dev(kd), W, m, 7.5, 1.25, be)
    torch.cuda.synchronize()
    assert rc == 0
    BXr = X if BX is None else BX
    R = ok.residual(AX, BXr, th)[:, c0:]
    scale = (np.abs(AX) + np.abs(BXr * th[None, :]))[:, c0:] / kd[:, None]
    assert np.all(np.abs(host(W, m - c0) - R / kd[:, None]) <= 4 * 2.0 ** -53 * scale)
    ref_be = np.linalg.norm(R, axis=0) / ((7.5 + np.abs(th[c0:]) * 1.25) * np.linalg.norm(X[:, c0:], axis=0))
    np.testing.assert_allclose(host(be), ref_be, rtol=1e-13)


def test_philox_normals_match_host_stream():
    torch = torch_cuda()
    n, m = 1001, 7
    Y = dev(np.zeros((n, m)), 8)
    assert gb.lobpcg_philox_normal(n, m, 0x123456789ABCDEF, 5, Y, 8) == 0
    torch.cuda.synchronize()
    ref = synth.normal_block(0x123456789ABCDEF, 5, n, m)
    # the uniforms are bit-identical; log/sincos may differ in the last ulps
    np.testing.assert_allclose(host(Y, m), ref, rtol=0, atol=4e-15 * np.abs(ref).max())
