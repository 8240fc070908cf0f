"""Definition-level FP64 references of the single steps of one iteration.

Test infrastructure only (see the package docstring).  Each function is the
plain mathematical definition of one operation of Algorithm 8's hot path, so a
kernel's output can be compared element by element.
"""
import numpy as np


def spmm_rows(rowptr, col, val, X, rows):
    """(A X)[rows, :] by the CSR definition y_i = sum_j a_ij x_j (sampled rows)."""
    out = np.zeros((len(rows), X.shape[1]))
    for t, i in enumerate(rows):
        lo, hi = int(rowptr[i]), int(rowptr[i + 1])
        out[t] = val[lo:hi] @ X[col[lo:hi]]
    return out


def spmm(rowptr, col, val, X):
    """A X for CSR A, by rows (vectorised per nonzero)."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    out = np.zeros((n, X.shape[1]))
    np.add.at(out, rows, val[:, None] * X[col])
    return out


def gram(U, V):
    """U^T V (the tall-skinny block inner product of Sec. 5.2)."""
    return U.T @ V


def update(S, C):
    """S C (the basis update of Eq. 10)."""
    return S @ C


def residual(AX, BX, theta):
    """R = AX - BX Theta (the residual of Algorithm 8)."""
    return AX - BX * theta[None, :]
