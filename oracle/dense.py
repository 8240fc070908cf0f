"""Dense FP64 building blocks of the oracle (test infrastructure only).

This module is part of the CPU oracle that the tests, the smoke check and the
benchmark's CPU baseline use to check the CUDA library.  The product path never
imports it.

  jacobi_eigh      cyclic Jacobi eigensolver (Golub & Van Loan, Matrix
                   Computations, Alg. 8.5.3 "cyclic Jacobi"), written out;
                   the definition-level dense oracle for small matrices.
  pencil_eigh      all eigenpairs of a symmetric-definite pencil (A, B) by
                   B = L L^T, eig(L^-1 A L^-T) -- the textbook reduction the
                   paper's Eq. (4) uses for the projected problem.
  eigh / cholesky_upper / qr_householder
                   thin wrappers on LAPACK through numpy, used as library
                   primitives by the iterative oracle; each wrapper is pinned
                   in the tests against jacobi_eigh, closed forms or
                   reconstruction identities.
"""
import numpy as np


def jacobi_eigh(A, tol=1e-15, max_sweeps=60):
    """All eigenpairs of a real symmetric matrix by cyclic Jacobi rotations.

    Each (p, q) rotation zeroes A[p, q] with the stable choice of tangent
    t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq),
    the square root taken as hypot(1, tau) so that a huge tau gives the
    small-angle tangent 1 / (2 tau) rather than an overflow.
    Sweeps repeat until the off-diagonal Frobenius norm is below
    tol * ||A||_F.  Returns (w ascending, V) with A V = V diag(w).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    V = np.eye(n)
    if n == 0:
        return np.zeros(0), V
    fro = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * fro or fro == 0.0:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                # sqrt(1 + tau^2) as hypot(1, tau): for |tau| beyond 1e154 the
                # square overflows, and the tangent must tend to the small-angle
                # value 1 / (2 tau) instead of 0 (Golub & Van Loan, Sec. 8.5.2)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + np.hypot(1.0, tau))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = A[q, p] = 0.0
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def cholesky_lower_plain(M):
    """Textbook Cholesky M = L L^T (outer-product form); raises on a non-positive pivot."""
    M = np.array(M, dtype=np.float64, copy=True)
    n = M.shape[0]
    L = np.zeros_like(M)
    for j in range(n):
        d = M[j, j] - np.dot(L[j, :j], L[j, :j])
        if not d > 0.0:
            raise np.linalg.LinAlgError("non-positive pivot")
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] = (M[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def pencil_eigh(A, B=None, use_jacobi=True):
    """All eigenpairs of the pencil (A, B), B symmetric positive definite.

    Reduction: B = L L^T, H = L^-1 A L^-T, H Y = Y Lambda, X = L^-T Y, so that
    A X = B X Lambda and X^T B X = I.  Eigenvalues ascending.
    """
    A = np.asarray(A, dtype=np.float64)
    if B is None:
        w, X = jacobi_eigh(A) if use_jacobi else eigh(A)
        return w, X
    L = cholesky_lower_plain(B)
    Li = np.linalg.solve(L, np.eye(len(L)))
    H = Li @ A @ Li.T
    H = 0.5 * (H + H.T)
    w, Y = jacobi_eigh(H) if use_jacobi else eigh(H)
    return w, Li.T @ Y


# ---- library primitives (LAPACK through numpy), pinned in the tests ----------

def eigh(M):
    """Symmetric eigendecomposition, eigenvalues ascending (LAPACK syevd)."""
    M = np.asarray(M, dtype=np.float64)
    if M.shape[0] == 0:
        return np.zeros(0), np.zeros((0, 0))
    return np.linalg.eigh(0.5 * (M + M.T))


def cholesky_upper(M):
    """Upper-triangular R with R^T R = M; raises LinAlgError if M is not PD."""
    return np.linalg.cholesky(np.asarray(M, dtype=np.float64)).T


def qr_householder(M):
    """Thin Householder QR (LAPACK geqrf/orgqr): M = Q R, Q^T Q = I."""
    return np.linalg.qr(np.asarray(M, dtype=np.float64), mode="reduced")
