"""FP64 CPU oracle of the eigenpair gradients (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the CUDA library never imports, links or calls it.

The paper computes eigenpairs only; the derivative form here is first-order
perturbation theory of the symmetric-definite pencil A x = lambda B x with
B-orthonormal eigenvectors (x_i^T B x_j = delta_ij).  For a simple eigenvalue

  d lambda_i = x_i^T (dA - lambda_i dB) x_i
  d x_i      = sum_{j != i} x_j [x_j^T (dA - lambda_i dB) x_i] / (lambda_i - lambda_j)
               - 1/2 x_i (x_i^T dB x_i)

so that for a scalar loss L with upstream gradients gl_i = dL/dlambda_i and
g_i = dL/dx_i, writing w_i = sum_{j != i} x_j (x_j^T g_i) / (lambda_i - lambda_j),

  dL/dA = sum_i gl_i x_i x_i^T + sym(w_i x_i^T)
  dL/dB = sum_i -lambda_i gl_i x_i x_i^T - lambda_i sym(w_i x_i^T)
                - 1/2 (g_i^T x_i) x_i x_i^T

with sym(M) = (M + M^T) / 2 (A and B are symmetric parameters).

  grad_full      w_i from the complete eigendecomposition (all j != i): the
                 definition, for small dense pencils.
  grad_split     the same gradient by the route a large-n solver takes:
                 w_i = w_i^in - u_i, where w_i^in sums j <= k and u_i solves
                 (A - lambda_i B) u_i = (I - B X X^T) g_i with X^T B u_i = 0
                 (solved here densely through the bordered system).
  on_pattern     samples a dense symmetric gradient on a CSR pattern: the
                 stored entry (r, c) gets G[r, c]; a symmetric pair (r, c),
                 (c, r) is one parameter whose derivative is G[r,c] + G[c,r].
  loss           L = sum_i gl_i lambda_i + sum_i <x_i, g_i> with sign-fixed
                 eigenvectors, for central finite differences.
"""
import numpy as np

from . import dense


def sign_fix(X):
    """Flip each column so its largest-magnitude entry (lowest index on ties) is positive."""
    X = np.array(X, dtype=np.float64, copy=True)
    for i in range(X.shape[1]):
        r = int(np.argmax(np.abs(X[:, i])))
        if X[r, i] < 0:
            X[:, i] = -X[:, i]
    return X


def eigenpairs(A, B, k):
    """The k smallest eigenpairs of the dense pencil (A, B), sign-fixed."""
    lam, X = dense.pencil_eigh(np.asarray(A, float), None if B is None else np.asarray(B, float),
                               use_jacobi=True)
    return lam, sign_fix(X)


def _gradients(lam, X, W, glam, G):
    """dL/dA and dL/dB from the eigenpairs, the w_i columns and the upstream gradients."""
    k = len(glam)
    Xk = X[:, :k]
    GA = (Xk * glam) @ Xk.T
    SW = W @ Xk.T
    GA = GA + 0.5 * (SW + SW.T)
    c = np.einsum("ri,ri->i", G, Xk)  # g_i^T x_i
    GB = -(Xk * (lam[:k] * glam)) @ Xk.T
    SWl = (W * lam[:k]) @ Xk.T
    GB = GB - 0.5 * (SWl + SWl.T) - 0.5 * (Xk * c) @ Xk.T
    return GA, GB


def grad_full(A, B, k, glam, G, gap_tol=1e-10, use_jacobi=True):
    """(lambda_k, X_k, dL/dA, dL/dB) with w_i from the full decomposition.

    use_jacobi=False takes the decomposition from LAPACK (the pinned library
    primitive) for pencils too large for the written-out Jacobi sweeps.

    Raises ValueError when two of the k wanted eigenvalues, or lambda_k and
    lambda_{k+1}, are closer than gap_tol * max|lambda| (the eigenvector
    derivative is not defined for a degenerate pair).
    """
    n = A.shape[0]
    lam, X = dense.pencil_eigh(np.asarray(A, float), None if B is None else np.asarray(B, float),
                               use_jacobi=use_jacobi)
    X = sign_fix(X)
    scale = np.abs(lam).max()
    gaps = np.diff(lam[:min(k + 1, n)])
    if gaps.size and gaps.min() < gap_tol * scale:
        raise ValueError("degenerate eigenvalues among the wanted pairs")
    W = np.zeros((n, k))
    XG = X.T @ G  # x_j^T g_i
    for i in range(k):
        for j in range(n):
            if j != i:
                W[:, i] += X[:, j] * (XG[j, i] / (lam[i] - lam[j]))
    GA, GB = _gradients(lam, X, W, np.asarray(glam, float), G)
    return lam[:k], X[:, :k], GA, GB


def complement_solve(A, B, X, lam, G):
    """u_i with (A - lambda_i B) u_i = (I - B X X^T) g_i and X^T B u_i = 0.

    Dense bordered system [[A - lambda_i B, B X], [X^T B, 0]] [u; mu] = [f; 0];
    it is nonsingular when lambda_i is simple and separated from the
    eigenvalues outside X.
    """
    n, k = X.shape
    Bm = np.eye(n) if B is None else np.asarray(B, float)
    BX = Bm @ X
    F = G - BX @ (X.T @ G)
    U = np.zeros((n, k))
    for i in range(k):
        K = np.zeros((n + k, n + k))
        K[:n, :n] = A - lam[i] * Bm
        K[:n, n:] = BX
        K[n:, :n] = BX.T
        rhs = np.concatenate([F[:, i], np.zeros(k)])
        U[:, i] = np.linalg.solve(K, rhs)[:n]
    return U, F


def grad_split(A, B, lam, X, glam, G):
    """dL/dA, dL/dB with w_i = w_i^in - u_i (k wanted pairs only)."""
    k = X.shape[1]
    W_in = np.zeros_like(X)
    for i in range(k):
        for j in range(k):
            if j != i:
                W_in[:, i] += X[:, j] * (X[:, j] @ G[:, i]) / (lam[i] - lam[j])
    U, _ = complement_solve(A, B, X, lam, G)
    W = W_in - U
    GA, GB = _gradients(np.asarray(lam, float), X, W, np.asarray(glam, float), G)
    return GA, GB, W


def on_pattern(Gd, rowptr, col):
    """Values of a dense gradient at the stored entries of a CSR pattern."""
    n = len(rowptr) - 1
    out = np.zeros(rowptr[-1])
    for r in range(n):
        for e in range(rowptr[r], rowptr[r + 1]):
            out[e] = Gd[r, col[e]]
    return out


def loss(A, B, k, glam, G):
    """L = sum_i gl_i lambda_i + sum_i <x_i, g_i> over sign-fixed eigenvectors."""
    lam, X = eigenpairs(A, B, k)
    return float(np.dot(glam, lam[:k]) + np.sum(X[:, :k] * G))
