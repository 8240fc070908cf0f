"""Plain FP64 CPU oracle of the robust LOBPCG (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module; the CUDA library never imports, links or calls it, and it shares no
code with the library.  Every routine follows the paper's algorithms in their
order and notation (Duersch, Shao, Yang, Gu, "A robust and efficient
implementation of LOBPCG", 2018):

  norm_estimate            Sec. 4.3, the Gaussian-sketch bound below Eq. (9)
  backward_error           Eq. (9); criteria (7) and (8) for contrast tests
  rayleigh_ritz            Algorithm 2
  svqb                     Algorithm 4
  svqb_drop                Algorithm 6 (basis truncation of Sec. 4.1)
  ortho_drop               Algorithm 5
  rayleigh_ritz_modified   Algorithm 7 with the LQ-based C_p of Sec. 4.2
  lobpcg                   Algorithm 8 with soft locking (Sec. 3), the Gram
                           identities (12)-(14) and implicit product updates
                           (Sec. 5.2, Eq. 10-11)
  ortho                    Algorithm 3 (Stathopoulos-Wu block orthogonalisation)
  rayleigh_ritz_hl         the Rayleigh-Ritz step of the Hetmaniuk-Lehoucq
                           basis selection with C_p of Eq. (6)
  lobpcg(basis="chl"/"ahl") the comparison variants of Sec. 6: HL basis
                           selection every iteration, conservative (CHL: no
                           implicit updates, every Gram block computed) or
                           aggressive (AHL: implicit updates, only (12) assumed)

Readings where the paper is silent or inconsistent (each is a documented
choice, identical in the CUDA library):
  * block width n_x = k + max(ceil(k/10), 2)  (Sec. 6: "padded by about 10%").
  * K^-1 is applied to R in both branches of Algorithm 8 (its W step writes
    R, Algorithm 1 and Eq. (2) apply K^-1).
  * tau_replace = tau_drop = n_u * eps, tau_ortho = 100 eps, tau_skip = 100 eps,
    eps = 2^-52; all norms in the orthogonality tests are Frobenius norms.
  * the skip test flips to orthogonalisation when cond(R)^-3 < tau_skip
    (Sec. 5.3 text), cond(R) in the 2-norm, i.e. sqrt(cond(D S^T B S D)).
  * under soft locking C_p spans Z_perp * (Z_1perp^T Z_1(:, n_c+1:n_x)),
    orthonormalised by Householder QR (equivalently the LQ of its transpose);
    with n_c = 0 and Z_1 nonsingular this is the paper's Z_perp Q_1perp^T.
  * a column whose B-norm squared is below the smallest normal double gets
    D_jj = 0 in svqb / svqbDrop (the paper's D is undefined there): it then
    spans a zero eigenvalue of D U^T B U D, which Algorithm 4 replaces (giving
    a zero output column) and Algorithm 6 drops.
  * n_c is monotone: a locked column stays locked; locking is in order.
  * implicit updates of AX, AP are used when B = I or B is diagonal with
    cond(B) <= 1e4 (Sec. 5.2 safety rule), refreshed explicitly every 50
    iterations and after each locking event; diagonal B products are formed
    explicitly (they are elementwise).
  * on termination AX, BX are recomputed explicitly and Eq. (9) is re-checked;
    columns that fail re-enter the iteration.
  * the initial Rayleigh-Ritz reports breakdown when Cholesky fails or the
    scaled Gram D X0^T B X0 D is numerically singular (smallest eigenvalue
    <= n_x * eps * largest).
  * output vectors are sign-normalised so the largest-magnitude entry (lowest
    index on ties) is positive.
"""
from dataclasses import dataclass, field
import math
import numpy as np
import scipy.sparse as sp

from . import dense

EPS = 2.0 ** -52

OK, NOT_CONVERGED, BREAKDOWN = 0, 2, 3


class Breakdown(Exception):
    pass


# --------------------------------------------------------------------------
# operators

class Pencil:
    """The pencil (A, B) with a preconditioner K, applied to row-major blocks.

    A: CSR given as (rowptr, col, val); B: None (identity), a 1-D array
    (diagonal B) or a CSR triple; kdiag: diagonal of K (Jacobi) or None (K = I).
    Sparse products use scipy.sparse as a library primitive.
    """

    def __init__(self, n, A, B=None, kdiag=None, k_fn=None):
        self.n = n
        self.k_fn = k_fn  # a general K^-1 (callable on a block), e.g. chebyshev_precond
        self.A = sp.csr_matrix((A[2], A[1], A[0]), shape=(n, n))
        if B is None:
            self.b_kind = "identity"
        elif isinstance(B, np.ndarray) and B.ndim == 1:
            self.b_kind = "diag"
            self.b = np.asarray(B, dtype=np.float64)
        else:
            self.b_kind = "csr"
            self.B = sp.csr_matrix((B[2], B[1], B[0]), shape=(n, n))
        self.kdiag = None if kdiag is None else np.asarray(kdiag, dtype=np.float64)

    def A_mul(self, X):
        return np.asarray(self.A @ X)

    def B_mul(self, X):
        if self.b_kind == "identity":
            return X.copy()
        if self.b_kind == "diag":
            return self.b[:, None] * X
        return np.asarray(self.B @ X)

    def K_inv(self, R):
        if self.k_fn is not None:
            return self.k_fn(R)
        if self.kdiag is None:
            return R.copy()
        return R / self.kdiag[:, None]

    def implicit_allowed(self):
        """Sec. 5.2: implicit product updates are safe when ||C|| stays O(1)."""
        if self.b_kind == "identity":
            return True
        if self.b_kind == "diag":
            b = np.abs(self.b)
            return b.min() > 0 and b.max() / b.min() <= 1e4
        return False


def chebyshev_precond(A, degree, lmin, lmax):
    """K^-1 R = `degree` steps of the Chebyshev iteration for A W = R from
    W = 0 with the Jacobi splitting D = diag(A) and the spectral interval
    [lmin, lmax] of D^-1 A (Saad, Iterative Methods for Sparse Linear Systems,
    Algorithm 12.1).  A: scipy CSR.  Returns the callable R -> W."""
    dinv = 1.0 / A.diagonal()
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta

    def apply(R):
        rho = 1.0 / sigma
        d = dinv[:, None] * R / theta
        w = d.copy()
        for _ in range(1, degree):
            z = dinv[:, None] * (R - A @ w)
            rho1 = 1.0 / (2.0 * sigma - rho)
            d = rho1 * rho * d + (2.0 * rho1 / delta) * z
            w = w + d
            rho = rho1
        return w
    return apply


# --------------------------------------------------------------------------
# convergence control (Sec. 4.3)

def norm_estimate(apply, Omega):
    """||M||_2^(Omega) = ||Omega M||_F / ||Omega||_F <= ||M||_2 (M symmetric).

    Omega is the s x n Gaussian sketch; Omega M = (M Omega^T)^T.
    """
    Y = apply(np.ascontiguousarray(Omega.T))
    return float(np.linalg.norm(Y) / np.linalg.norm(Omega))


def backward_error(R, X, theta, normA, normB):
    """Eq. (9): ||r_i||_2 / ((||A|| + |theta_i| ||B||) ||x_i||_2) per column."""
    rn = np.linalg.norm(R, axis=0)
    xn = np.linalg.norm(X, axis=0)
    return rn / ((normA + np.abs(theta) * normB) * xn)


def criterion7(R, X, theta):
    """Eq. (7): ||r_i|| / (|theta_i| ||x_i||) (contrast tests only)."""
    return np.linalg.norm(R, axis=0) / (np.abs(theta) * np.linalg.norm(X, axis=0))


def criterion8(R, X, BX, theta):
    """Eq. (8): ||r_i|| / (|theta_i| ||x_i||_B) (contrast tests only)."""
    xb = np.sqrt(np.abs(np.sum(X * BX, axis=0)))
    return np.linalg.norm(R, axis=0) / (np.abs(theta) * xb)


def leading_converged(be, tol):
    """Length of the leading run of columns with backward error <= tol (in-order locking)."""
    bad = np.nonzero(~(be <= tol))[0]
    return int(bad[0]) if len(bad) else len(be)


# --------------------------------------------------------------------------
# Rayleigh-Ritz (Algorithm 2)

def rayleigh_ritz(GA, GB):
    """Algorithm 2: C, Theta with C^T GB C = I and C^T GA C = Theta (ascending)."""
    d = 1.0 / np.sqrt(np.diag(GB))
    MB = d[:, None] * GB * d[None, :]
    try:
        R = dense.cholesky_upper(MB)
    except np.linalg.LinAlgError as e:
        raise Breakdown("Cholesky of the initial Gram failed") from e
    ev = np.linalg.eigvalsh(MB)
    if not ev[0] > len(ev) * EPS * ev[-1]:
        raise Breakdown("initial block is numerically rank deficient")
    Rinv = np.linalg.solve(R, np.eye(len(R)))
    H = Rinv.T @ (d[:, None] * GA * d[None, :]) @ Rinv
    theta, Z = dense.eigh(H)
    C = d[:, None] * (Rinv @ Z)
    return C, theta


# --------------------------------------------------------------------------
# orthogonalisation (Algorithms 4, 5, 6)

def _scaling(G):
    """D = diag(G)^-1/2, with D_jj = 0 for a column of zero B-norm."""
    g = np.diag(G)
    ok = g > np.finfo(np.float64).tiny
    return np.where(ok, 1.0 / np.sqrt(np.where(ok, g, 1.0)), 0.0)


def svqb(U, BU, tau_replace):
    """Algorithm 4: U D Z Theta^-1/2 with small theta replaced by tau*max|theta|."""
    G = U.T @ BU
    G = 0.5 * (G + G.T)
    if U.shape[1] == 0:
        return U
    d = _scaling(G)
    theta, Z = dense.eigh(d[:, None] * G * d[None, :])
    if not np.max(np.abs(theta)) > 0:
        return U[:, :0]
    floor = tau_replace * np.max(np.abs(theta))
    theta = np.where(theta < floor, floor, theta)
    return U @ ((d[:, None] * Z) / np.sqrt(theta)[None, :])


def svqb_drop(U, BU, tau_drop):
    """Algorithm 6: keep J = {j : theta_j > tau_drop * max|theta|}."""
    G = U.T @ BU
    G = 0.5 * (G + G.T)
    if U.shape[1] == 0:
        return U
    d = _scaling(G)
    theta, Z = dense.eigh(d[:, None] * G * d[None, :])
    J = theta > tau_drop * np.max(np.abs(theta))
    return U @ ((d[:, None] * Z[:, J]) / np.sqrt(theta[J])[None, :])


def ortho_drop(B_mul, U, V, BV, tau_ortho, stats=None, itmax1=3, itmax2=3):
    """Algorithm 5: B-orthonormalise U against the B-orthonormal V, dropping.

    V^T B U is formed as (BV)^T U.  Returns (U, BU).
    """
    BU = B_mul(U)
    for i in range(itmax1):
        if V.shape[1] > 0:
            U = U - V @ (BV.T @ U)
        for j in range(itmax2):
            BU = B_mul(U)
            nu = U.shape[1]
            if j == 0:
                U = svqb(U, BU, nu * EPS)
            else:
                U = svqb_drop(U, BU, nu * EPS)
            if stats is not None:
                stats["svqb_passes"] += 1
            BU = B_mul(U)
            if U.shape[1] == 0:
                return U, BU
            G = U.T @ BU
            err = np.linalg.norm(G - np.eye(U.shape[1])) / (
                np.linalg.norm(BU) * np.linalg.norm(U))
            if err <= tau_ortho:
                break
        if V.shape[1] == 0:
            break
        err = np.linalg.norm(BV.T @ U) / (np.linalg.norm(BV) * np.linalg.norm(U))
        if err <= tau_ortho:
            break
    return U, BU


def ortho(B_mul, U, V, BV, tau_ortho, stats=None, itmax1=3, itmax2=3):
    """Algorithm 3 (Stathopoulos-Wu): B-orthonormalise U against V with block
    classical Gram-Schmidt and inner svqb passes (Algorithm 4, no dropping:
    the column count never changes).  Returns (U, BU)."""
    BU = B_mul(U)
    nu = U.shape[1]
    for i in range(itmax1):
        if V.shape[1] > 0:
            U = U - V @ (BV.T @ U)
        for j in range(itmax2):
            BU = B_mul(U)
            U = svqb(U, BU, nu * EPS)
            if stats is not None:
                stats["svqb_passes"] += 1
            BU = B_mul(U)
            if U.shape[1] == 0:
                return U, BU
            G = U.T @ BU
            err = np.linalg.norm(G - np.eye(U.shape[1])) / (
                np.linalg.norm(BU) * np.linalg.norm(U))
            if err <= tau_ortho:
                break
        if V.shape[1] == 0:
            break
        err = np.linalg.norm(BV.T @ U) / (np.linalg.norm(BV) * np.linalg.norm(U))
        if err <= tau_ortho:
            break
    return U, BU


def rayleigh_ritz_hl(SAS, nx, nc):
    """Rayleigh-Ritz of the Hetmaniuk-Lehoucq basis selection: S is
    B-orthonormal, so eig(S^T A S) = Z Theta Z^T gives C_x = Z(:, :n_x); C_p
    orthonormalises [0; Z_2] - Z_x Z_x^T [0; Z_2] (Eq. 6, restricted to the
    unlocked columns n_c:n_x) with svqb in the Euclidean metric; P^T A P is
    then C_p^T S^T A S C_p (the P block no longer lies in the Ritz basis)."""
    ns = SAS.shape[0]
    theta, Z = dense.eigh(SAS)
    Zx = Z[:, :nx]
    Y = np.zeros((ns, nx - nc))
    Y[nx:, :] = Zx[nx:, nc:nx]
    Y = Y - Zx @ (Zx.T @ Y)
    Cp = svqb(Y, Y, max(Y.shape[1], 1) * EPS) if Y.shape[1] else Y
    PAP = Cp.T @ SAS @ Cp
    return RRResult(Zx, Cp, theta[:nx].copy(), 0.5 * (PAP + PAP.T), False, 1.0)


# --------------------------------------------------------------------------
# Algorithm 7

@dataclass
class RRResult:
    Cx: np.ndarray
    Cp: np.ndarray
    theta: np.ndarray      # Ritz values of the n_x columns of X (ascending)
    PAP: np.ndarray        # Q_p^T Theta_perp Q_p, the next P^T A P (Eq. 14)
    flip: bool = False
    condR: float = 1.0


def rayleigh_ritz_modified(SAS, SBS, nx, nc, use_ortho, tau_skip=100 * EPS):
    """Algorithm 7.  SAS, SBS: the projected pencil on S = [X, P, W]."""
    ns = SAS.shape[0]
    condR = 1.0
    if use_ortho:
        theta, Z = dense.eigh(SAS)
        T = np.eye(ns)
    else:
        d = 1.0 / np.sqrt(np.diag(SBS))
        MB = d[:, None] * SBS * d[None, :]
        try:
            R = dense.cholesky_upper(MB)
        except np.linalg.LinAlgError:
            return RRResult(None, None, None, None, flip=True, condR=math.inf)
        ev = np.linalg.eigvalsh(0.5 * (MB + MB.T))
        condR = math.sqrt(ev[-1] / ev[0]) if ev[0] > 0 else math.inf
        if not (condR ** -3 >= tau_skip):
            return RRResult(None, None, None, None, flip=True, condR=condR)
        Rinv = np.linalg.solve(R, np.eye(ns))
        H = Rinv.T @ (d[:, None] * SAS * d[None, :]) @ Rinv
        theta, Z = dense.eigh(H)
        T = d[:, None] * Rinv
    Z1 = Z[:nx, :nx]
    Z1perp = Z[:nx, nx:]
    M = Z1perp.T @ Z1[:, nc:nx]
    npn = min(ns - nx, nx - nc)
    if npn > 0:
        Q, _ = dense.qr_householder(M)
        Q = Q[:, :npn]
    else:
        Q = np.zeros((ns - nx, 0))
    Cx = T @ Z[:, :nx]
    Cp = T @ (Z[:, nx:] @ Q)
    PAP = Q.T @ (theta[nx:, None] * Q)
    return RRResult(Cx, Cp, theta[:nx].copy(), 0.5 * (PAP + PAP.T), False, condR)


# --------------------------------------------------------------------------
# Algorithm 8

@dataclass
class Options:
    nx: int = None
    maxit: int = 2000
    tau_ortho: float = 100 * EPS
    tau_skip: float = 100 * EPS
    implicit: str = "auto"        # auto | always | never
    refresh_every: int = 50
    direct_gram: bool = False     # compute every block of S^T A S, S^T B S
    certify: bool = True
    basis: str = "robust"         # robust (Algorithm 8) | chl | ahl (Sec. 6 comparisons)


@dataclass
class Result:
    lam: np.ndarray
    X: np.ndarray
    iters: int
    be: np.ndarray
    status: int
    normA: float
    normB: float
    stats: dict = field(default_factory=dict)


def _assemble(theta, PAP, GAw, GBw, nx, np_, nw, SBS_identity):
    """Projected pencil from the identities (12)-(14) and the W columns."""
    ns = nx + np_ + nw
    SAS = np.zeros((ns, ns))
    SBS = np.eye(ns)
    SAS[:nx, :nx] = np.diag(theta)
    SAS[nx:nx + np_, nx:nx + np_] = PAP
    o = nx + np_
    SAS[:, o:] = GAw
    SAS[o:, :] = GAw.T
    if not SBS_identity:
        SBS[:, o:] = GBw
        SBS[o:, :] = GBw.T
    return SAS, SBS


def sign_normalise(X):
    X = X.copy()
    idx = np.argmax(np.abs(X), axis=0)
    s = np.sign(X[idx, np.arange(X.shape[1])])
    s[s == 0] = 1.0
    return X * s[None, :]


def lobpcg(pencil, X0, k, tol, Omega, opts=None):
    """Algorithm 8 on the pencil; X0 is n x n_x.  Returns a Result."""
    opts = opts or Options()
    hl = opts.basis in ("chl", "ahl")
    n, nx = X0.shape
    stats = {"flip_iter": None, "ortho_calls": 0, "svqb_passes": 0,
             "dropped": 0, "nc_history": [], "condR": []}
    normA = norm_estimate(pencil.A_mul, Omega)
    normB = 1.0 if pencil.b_kind == "identity" else norm_estimate(pencil.B_mul, Omega)
    implicit = {"auto": pencil.implicit_allowed(), "always": True,
                "never": False}[opts.implicit]
    if opts.basis == "chl":
        implicit = False  # conservative: every product explicit

    # Algorithm 8, initial step: Rayleigh-Ritz on X0 (Algorithm 2)
    AX0, BX0 = pencil.A_mul(X0), pencil.B_mul(X0)
    try:
        C, theta = rayleigh_ritz(X0.T @ AX0, X0.T @ BX0)
    except Breakdown:
        return Result(None, None, 0, None, BREAKDOWN, normA, normB, stats)
    X = X0 @ C
    AX, BX = pencil.A_mul(X), pencil.B_mul(X)
    theta = theta[:nx]
    P = np.zeros((n, 0)); AP = np.zeros((n, 0)); BP = np.zeros((n, 0))
    PAP = np.zeros((0, 0))
    use_ortho = hl  # the HL variants orthogonalise W on every iteration
    R = AX - BX * theta[None, :]
    be = backward_error(R, X, theta, normA, normB)
    nc = min(leading_converged(be, tol), nx)
    it = 0
    refresh_next = False
    status = OK

    while True:
        while nc < k:
            if it >= opts.maxit:
                status = NOT_CONVERGED
                break
            it += 1
            V = np.hstack([X, P])
            BV = np.hstack([BX, BP])

            def make_w(do_ortho):
                W0 = pencil.K_inv(R[:, nc:])
                if do_ortho and hl:
                    stats["ortho_calls"] += 1
                    W, BW = ortho(pencil.B_mul, W0, V, BV, opts.tau_ortho, stats)
                elif do_ortho:
                    stats["ortho_calls"] += 1
                    W, BW = ortho_drop(pencil.B_mul, W0, V, BV, opts.tau_ortho, stats)
                    stats["dropped"] += W0.shape[1] - W.shape[1]
                else:
                    W, BW = W0, pencil.B_mul(W0)
                return W, BW, pencil.A_mul(W)

            def project(W, AW, BW):
                S = np.hstack([X, P, W])
                if opts.basis == "ahl":
                    # (12) holds: X^T A X = Theta, X^T B X = I; every block
                    # with P or W is computed from the (implicit) products
                    ns_ = S.shape[1]
                    PW = np.hstack([P, W])
                    APW = np.hstack([AP, AW])
                    BPW = np.hstack([BP, BW])
                    SAS = np.zeros((ns_, ns_))
                    SBS = np.zeros((ns_, ns_))
                    SAS[:nx, :nx] = np.diag(theta)
                    SBS[:nx, :nx] = np.eye(nx)
                    SAS[:, nx:] = S.T @ APW
                    SBS[:, nx:] = S.T @ BPW
                    SAS[nx:, :nx] = SAS[:nx, nx:].T
                    SBS[nx:, :nx] = SBS[:nx, nx:].T
                    return 0.5 * (SAS + SAS.T), 0.5 * (SBS + SBS.T)
                if opts.direct_gram or opts.basis == "chl":
                    AS = np.hstack([AX, AP, AW]) if not implicit else np.hstack(
                        [pencil.A_mul(X), pencil.A_mul(P), AW])
                    BS = pencil.B_mul(S)
                    return S.T @ AS, S.T @ BS
                return _assemble(theta, PAP, S.T @ AW, S.T @ BW, nx, P.shape[1],
                                 W.shape[1], use_ortho)

            W, BW, AW = make_w(use_ortho)
            SAS, SBS = project(W, AW, BW)
            if hl:
                rr = rayleigh_ritz_hl(SAS, nx, nc)
            else:
                rr = rayleigh_ritz_modified(SAS, SBS, nx, nc, use_ortho, opts.tau_skip)
            stats["condR"].append(rr.condR)
            if rr.flip:
                # Algorithm 8: switch to orthogonalisation and project again
                use_ortho = True
                stats["flip_iter"] = it
                W, BW, AW = make_w(True)
                SAS, SBS = project(W, AW, BW)
                rr = rayleigh_ritz_modified(SAS, SBS, nx, nc, True, opts.tau_skip)
            # Algorithm 8 update and Sec. 5.2
            S = np.hstack([X, P, W])
            Xn, Pn = S @ rr.Cx, S @ rr.Cp
            if implicit and not refresh_next and it % opts.refresh_every != 0:
                AS = np.hstack([AX, AP, AW])
                AXn, APn = AS @ rr.Cx, AS @ rr.Cp
            else:
                AXn, APn = pencil.A_mul(Xn), pencil.A_mul(Pn)
            if pencil.b_kind == "csr" and implicit and not refresh_next:
                BS = np.hstack([BX, BP, BW])
                BXn, BPn = BS @ rr.Cx, BS @ rr.Cp
            else:
                BXn, BPn = pencil.B_mul(Xn), pencil.B_mul(Pn)
            X, P, AX, AP, BX, BP = Xn, Pn, AXn, APn, BXn, BPn
            theta, PAP = rr.theta, rr.PAP
            # Algorithm 8: residual and convergence test
            R = AX - BX * theta[None, :]
            be = backward_error(R, X, theta, normA, normB)
            nc_new = max(nc, min(leading_converged(be, tol), nx))
            refresh_next = nc_new > nc
            nc = nc_new
            stats["nc_history"].append(nc)
        if status != OK or not opts.certify:
            break
        # certification with explicit products
        AX, BX = pencil.A_mul(X), pencil.B_mul(X)
        R = AX - BX * theta[None, :]
        be = backward_error(R, X, theta, normA, normB)
        good = leading_converged(be, tol)
        if good >= k:
            break
        nc = good
        refresh_next = True

    Xk = sign_normalise(X[:, :k])
    return Result(theta[:k].copy(), Xk, it, be[:k].copy(), status, normA, normB, stats)
