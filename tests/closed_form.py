"""Checks of computed eigenpairs against closed-form spectra with
degenerate clusters (shared by the GPU full-size tests and their CPU pins;
numpy only)."""
import numpy as np


def clusters(ref):
    """Distinct values of a sorted closed-form spectrum (sums of 1-D
    eigenvalues taken in different orders differ by a few ulps)."""
    u = [ref[0]]
    for v in ref[1:]:
        if v - u[-1] > 1e-12 * max(1.0, abs(v)):
            u.append(v)
    return np.array(u)


def periodic_closed_form(N, c, count):
    """c + eigenvalues of -1/2 (periodic 7-point Laplacian) on N^3: sums of
    three 1-D values 2 sin^2(pi j / N), j = 0 .. N-1."""
    one = np.sort(2.0 * np.sin(np.pi * np.arange(N) / N) ** 2)
    lam = np.zeros(1)
    for _ in range(3):
        lam = np.sort((lam[:, None] + one[None, :]).ravel())[: count * 4 + 64]
    return c + lam[:count]


def closed_form_match(lam, rho, rn_rho, rn_lam, ref):
    """Returned pairs against a closed-form spectrum with multiplicities.

    Vectors: for a unit vector x with Rayleigh quotient rho and residual
    r = A x - rho x, the eigenvalue mu nearest rho satisfies |rho - mu| <=
    ||r||^2 / delta, delta the distance from rho to the rest of the spectrum
    (the quadratic residual bound, Parlett 1980, Thm 11.7.1; it holds per
    cluster of equal eigenvalues).  Values: the returned lambda_i comes from
    the projected pencil, not from x_i, and ||A x - lambda x||^2 = ||r||^2 +
    (lambda - rho)^2 ||x||^2, so |lambda_i - mu_i| <= ||A x_i - lambda_i x_i||
    + |rho_i - mu_i|.  The matched mu, sorted, must equal the lowest k of the
    closed form element by element, so a missed or doubled member of a
    cluster fails even where every single pair is accurate.  rn_rho and
    rn_lam are the residual norms divided by ||x_i||.  Returns the largest
    |lambda_i - mu_i| and |rho_i - mu_i|."""
    lam, rho = np.asarray(lam, float), np.asarray(rho, float)
    u = clusters(ref)
    floor = 1e-13 * max(1.0, float(np.abs(ref).max()))
    j = np.clip(np.searchsorted(u, rho), 1, len(u) - 1)
    j = np.where(np.abs(u[j - 1] - rho) <= np.abs(u[j] - rho), j - 1, j)
    mu = u[j]
    lo = np.where(j > 0, rho - u[np.maximum(j - 1, 0)], np.inf)
    hi = np.where(j < len(u) - 1, u[np.minimum(j + 1, len(u) - 1)] - rho, np.inf)
    delta = np.minimum(lo, hi)
    assert np.all(delta > rn_rho), "residuals too large for the quadratic bound"
    err_rho = np.abs(rho - mu)
    bound = rn_rho ** 2 / (delta - rn_rho) + floor
    assert np.all(err_rho <= bound), (float((err_rho / bound).max()),
                                      int(np.argmax(err_rho / bound)))
    err_lam = np.abs(lam - mu)
    assert np.all(err_lam <= rn_lam + bound), int(np.argmax(err_lam - rn_lam - bound))
    k = len(lam)
    ref_k = u[np.searchsorted(u, ref[:k] - 1e-12 * np.maximum(1.0, np.abs(ref[:k])))]
    np.testing.assert_array_equal(np.sort(mu), ref_k)
    return float(err_lam.max()), float(err_rho.max())
