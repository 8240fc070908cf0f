"""Synthetic sparse symmetric pencils (A, B) used by tests and the benchmark.

Conventions: grid spacing 1 (unscaled stencils), lexicographic ordering with x
fastest (index = x + Nx*y + Nx*Ny*z), CSR rows sorted by column, int32 indices,
float64 values.  Nothing here performs any step of the eigensolver.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .philox import (normal_flat, uniform_block, STREAM_BDIAG, STREAM_COEF,
                     STREAM_POTENTIAL)


@dataclass
class CSR:
    n: int
    rowptr: np.ndarray   # int32 (or int64 when nnz >= 2**31), n + 1
    col: np.ndarray      # int32, nnz
    val: np.ndarray      # float64, nnz

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def diagonal(self):
        d = np.zeros(self.n)
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        m = rows == self.col
        d[rows[m]] = self.val[m]
        return d

    def to_dense(self):
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(a, (rows, self.col), self.val)
        return a


def _from_coo(n, rows, cols, vals):
    """Sort COO triplets by (row, col), sum duplicates, return CSR."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = uniq // n
    c = uniq % n
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    idx = np.int64 if rowptr[-1] >= 2 ** 31 else np.int32
    return CSR(n, rowptr.astype(idx), c.astype(np.int32), summed.astype(np.float64))


def tridiag(n, diag, off):
    """Symmetric tridiagonal matrix tridiag(off, diag, off)."""
    i = np.arange(n)
    rows = np.concatenate([i, i[:-1], i[1:]])
    cols = np.concatenate([i, i[1:], i[:-1]])
    vals = np.concatenate([np.full(n, diag, float), np.full(n - 1, off, float),
                           np.full(n - 1, off, float)])
    return _from_coo(n, rows, cols, vals)


def laplacian_1d(n):
    """1D Dirichlet Laplacian tridiag(-1, 2, -1)."""
    return tridiag(n, 2.0, -1.0)


def _grid_stencil(dims, periodic, diag_fn, off_fn):
    """Generic nearest-neighbour stencil on a box grid.

    diag_fn(idx) gives the diagonal values, off_fn(idx, nbr, axis) the value
    of the coupling between idx and its + neighbour along axis.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    strides = [int(np.prod(dims[:a])) for a in range(len(dims))]
    rows = [idx]
    cols = [idx]
    vals = [diag_fn(idx)]
    for a, d in enumerate(dims):
        if periodic:
            if d < 2:
                continue
            src = idx
            nb = idx + np.where(coords[a] == d - 1, -(d - 1), 1) * strides[a]
        else:
            m = coords[a] < d - 1
            src = idx[m]
            nb = src + strides[a]
        v = off_fn(src, nb, a)
        rows += [src, nb]
        cols += [nb, src]
        vals += [v, v]
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols),
                     np.concatenate(vals))


def laplacian_2d_dirichlet(nx, ny=None):
    """2D 5-point Dirichlet Laplacian, diagonal 4, couplings -1."""
    ny = nx if ny is None else ny
    return _grid_stencil((nx, ny), False, lambda i: np.full(len(i), 4.0),
                         lambda s, t, a: np.full(len(s), -1.0))


def laplacian_3d_dirichlet(nx, ny=None, nz=None):
    """3D 7-point Dirichlet Laplacian, diagonal 6, couplings -1."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _grid_stencil((nx, ny, nz), False, lambda i: np.full(len(i), 6.0),
                         lambda s, t, a: np.full(len(s), -1.0))


def diffusion_3d_lognormal(nx, sigma, seed):
    """Variable-coefficient 7-point diffusion on an nx^3 grid, Dirichlet walls.

    Every face f of the grid (interior and boundary) carries a coefficient
    a_f = exp(sigma * xi_f) with xi_f ~ N(0, 1) i.i.d. (unit-median log-normal).
    A_ii is the sum of the coefficients of the six faces of cell i; an interior
    face between i and j contributes A_ij = -a_f.  Face f along axis a between
    cells with coordinate c and c+1 (c = -1 .. nx-1) has flat id
    a*(nx+1)*nx*nx + ((c+1) + (nx+1)*(p + nx*q)) with (p, q) the other two
    coordinates in increasing axis order; its xi is normal number f of stream 3.
    """
    n = nx ** 3
    nf = (nx + 1) * nx * nx
    xi = normal_flat(seed, STREAM_COEF, 0, 3 * nf)
    coef = np.exp(sigma * xi)
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    xyz = (x, y, z)

    def face(axis, c_lo, i):
        # c_lo: coordinate of the lower cell along axis (-1 .. nx-1)
        others = [xyz[b][i] for b in range(3) if b != axis]
        return axis * nf + (c_lo + 1) + (nx + 1) * (others[0] + nx * others[1])

    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for a in range(3):
        c = xyz[a]
        diag += coef[face(a, c - 1, idx)] + coef[face(a, c, idx)]
        m = c < nx - 1
        src = idx[m]
        nb = src + nx ** a
        v = -coef[face(a, c[m], src)]
        rows += [src, nb]
        cols += [nb, src]
        vals += [v, v]
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols),
                     np.concatenate(vals))


def hamiltonian_3d_periodic(nx, potential):
    """H = -1/2 * (periodic 7-point Laplacian) + diag(V) on an nx^3 torus.

    H_ii = 3 + V_i and H_ij = -1/2 for the six periodic neighbours.
    """
    V = np.asarray(potential, dtype=np.float64)
    return _grid_stencil((nx, nx, nx), True, lambda i: 3.0 + V[i],
                         lambda s, t, a: np.full(len(s), -0.5))


def mass_matrix_2d(nx, c, ny=None):
    """B = I + c * (adjacency of the 5-point grid), the pattern of the 2D
    Dirichlet Laplacian: SPD for |c| < 1/4, and it shares the Laplacian's
    sine eigenvectors (both are polynomials in the grid adjacency)."""
    L = laplacian_2d_dirichlet(nx, ny)
    rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
    val = np.where(rows == L.col, 1.0, -c * L.val)
    return CSR(L.n, L.rowptr, L.col, val)


def closed_form_mass_pencil(nx, c, count, ny=None):
    """Lowest eigenvalues of (Laplacian, I + c Adj) on the nx x ny Dirichlet
    grid: (4 - mu) / (1 + c mu), mu = 2 cos(pi i/(nx+1)) + 2 cos(pi j/(ny+1))."""
    ny = ny or nx
    i = np.arange(1, nx + 1)[:, None]
    j = np.arange(1, ny + 1)[None, :]
    mu = 2 * np.cos(np.pi * i / (nx + 1)) + 2 * np.cos(np.pi * j / (ny + 1))
    return np.sort(((4 - mu) / (1 + c * mu)).ravel())[:count]


def add_diagonal(a, d):
    """A + diag(d) for a CSR A whose diagonal entries are all stored."""
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    m = rows == a.col
    val = a.val.copy()
    val[m] += np.asarray(d)[rows[m]]
    return CSR(a.n, a.rowptr, a.col, val)


def block_width(k, n=None):
    """Default block width: k padded by about 10 %, at least two extra columns."""
    nx = k + max(int(math.ceil(k / 10.0)), 2)
    if n is not None:
        nx = min(nx, n)
    return nx


@dataclass
class Problem:
    name: str
    A: CSR
    k: int
    tol: float
    b_diag: np.ndarray = None      # None: B = I
    kdiag: np.ndarray = None       # Jacobi preconditioner K = diag(kdiag)
    closed_form: np.ndarray = None  # exact lowest eigenvalues when known
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.A.n


def _dirichlet_1d_eigs(N):
    j = np.arange(1, N + 1)
    return 4.0 * np.sin(np.pi * j / (2.0 * (N + 1))) ** 2


def closed_form_laplacian(dims, count):
    """Lowest eigenvalues of the Dirichlet grid Laplacian, sum of 1D spectra."""
    lam = np.zeros(1)
    for N in dims:
        lam = (lam[:, None] + _dirichlet_1d_eigs(N)[None, :]).ravel()
        lam.sort()
        lam = lam[: max(count, 1) * 4 + 64]
    return np.sort(lam)[:count]


def make_problem(name, seed=0, **kw):
    """Build one of the named workloads (see WORKLOADS) with a seed."""
    if name == "lap2d_32":
        A = laplacian_2d_dirichlet(32)
        return Problem(name, A, 8, 1e-8, kdiag=A.diagonal(),
                       closed_form=closed_form_laplacian((32, 32), 12),
                       note="2D 5-point Dirichlet 32x32, B=I, Jacobi K")
    if name == "lap3d_64_diagB":
        N = kw.get("N", 64)
        A = laplacian_3d_dirichlet(N)
        b = uniform_block(seed, STREAM_BDIAG, A.n, 1.0, 2.0)
        return Problem(name, A, kw.get("k", 64), 1e-8, b_diag=b, kdiag=A.diagonal(),
                       note=f"3D 7-point Dirichlet {N}^3, diagonal B ~ U[1,2], Jacobi K")
    if name == "lap3d_64_B=I":
        N = kw.get("N", 64)
        A = laplacian_3d_dirichlet(N)
        k = kw.get("k", 64)
        return Problem(name, A, k, 1e-8, kdiag=A.diagonal(),
                       closed_form=closed_form_laplacian((N, N, N), k + 8),
                       note=f"3D 7-point Dirichlet {N}^3, B=I, Jacobi K")
    if name == "diffusion_128":
        N = kw.get("N", 128)
        A = diffusion_3d_lognormal(N, kw.get("sigma", 1.0), seed)
        return Problem(name, A, kw.get("k", 256), kw.get("tol", 1e-8), kdiag=A.diagonal(),
                       note=f"3D log-normal diffusion {N}^3, sigma=1, B=I, Jacobi K")
    if name == "hamiltonian_96":
        N = kw.get("N", 96)
        V = uniform_block(seed, STREAM_POTENTIAL, N ** 3, 0.0, 10.0)
        A = hamiltonian_3d_periodic(N, V)
        return Problem(name, A, kw.get("k", 1024), 1e-8, kdiag=A.diagonal(),
                       note=f"-0.5*Laplacian(periodic {N}^3) + V, V ~ U[0,10]")
    if name == "lap2d_512_V":
        N = kw.get("N", 512)
        V = uniform_block(seed, STREAM_POTENTIAL, N * N, 0.0, 1.0)
        A = add_diagonal(laplacian_2d_dirichlet(N), V)
        return Problem(name, A, kw.get("k", 32), 1e-8, kdiag=A.diagonal(),
                       extra={"V": V},
                       note=f"2D 5-point Dirichlet {N}^2 + diag(V), V ~ U[0,1]")
    raise KeyError(name)


WORKLOADS = {
    "lap2d_32": "2D 5-point Dirichlet Laplacian 32x32 (n=1024), B=I, Jacobi K, k=8, tol 1e-8",
    "lap3d_64_diagB": "3D 7-point Dirichlet Laplacian 64^3 (n=262144), diagonal B ~ U[1,2], Jacobi K, k=64, tol 1e-8",
    "lap3d_64_B=I": "3D 7-point Dirichlet Laplacian 64^3 with B=I (closed-form special case), k=64",
    "diffusion_128": "128^3 log-normal (sigma=1) 7-point diffusion (n=2097152), B=I, Jacobi K, k=256",
    "hamiltonian_96": "-0.5*Laplacian(periodic 96^3) + V, V~U[0,10] (n=884736), B=I, Jacobi K, k=1024",
    "lap2d_512_V": "2D 5-point Dirichlet 512^2 + diag(V), V~U[0,1] (n=262144), k=32",
}
