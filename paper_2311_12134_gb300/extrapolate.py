"""LIZ-radius extrapolation of the resistivity (Sec. II.C and Sec. IV).

The conductivity of a finite LIZ depends on its radius; the paper models the
dependence heuristically and extrapolates to an infinite LIZ:

* pure crystal / weak scattering (Eq. linear-fit): rho ~ k_LIZ / (2 alpha a1) + 1/a1
  with k_LIZ = 1 / (r_LIZ - r_c); the intercept 1/a1 is the converged value;
* decaying tau (Eq. sigma-alpha): sigma ~ a0 exp(-2 alpha r_LIZ) + a1;
* alloys (Sec. IV): a lower bound rho = c0 / r + c1 (alpha -> 0, r_c -> 0) and an
  upper bound rho = b0 / (1 + b1 exp(-2 alpha_max r)) with 2 alpha_max = 0.15 in the
  paper's inverse length unit; the extrapolated residual resistivities are c1 and b0.

These fits act on a handful of scalars (rho_xx per radius) on the host; they are
post-processing of the conductivity path, not part of it.  All fits are linear
least squares after the substitution stated in each function.
"""
import numpy as np

# The paper quotes LIZ radii and 2 alpha_max = 0.15 in angstrom; the library works in bohr.
BOHR_IN_ANGSTROM = 0.529177210903


def fit_lower_bound(r, rho):
    """rho = c0 / r + c1 (linear in 1/r).  Returns (c0, c1); c1 is rho at r -> inf."""
    r = np.asarray(r, dtype=np.float64)
    A = np.stack([1.0 / r, np.ones_like(r)], axis=1)
    (c0, c1), *_ = np.linalg.lstsq(A, np.asarray(rho, dtype=np.float64), rcond=None)
    return float(c0), float(c1)


def fit_upper_bound(r, rho, two_alpha=0.15):
    """rho = b0 / (1 + b1 exp(-two_alpha r)), i.e. 1/rho = 1/b0 + (b1/b0) exp(-two_alpha r),
    linear in exp(-two_alpha r).  Returns (b0, b1); b0 is rho at r -> inf.  The default
    two_alpha = 0.15 is the paper's 2 alpha_max in inverse angstrom, so r must be in angstrom
    (radii in bohr times BOHR_IN_ANGSTROM)."""
    r = np.asarray(r, dtype=np.float64)
    x = np.exp(-two_alpha * r)
    A = np.stack([np.ones_like(r), x], axis=1)
    (p, q), *_ = np.linalg.lstsq(A, 1.0 / np.asarray(rho, dtype=np.float64), rcond=None)
    return float(1.0 / p), float(q / p)


def fit_linear_law(r, rho, r_c):
    """Eq. linear-fit: rho = k / (2 alpha a1) + 1 / a1 with k = 1 / (r - r_c).
    Returns (a1, alpha)."""
    r = np.asarray(r, dtype=np.float64)
    k = 1.0 / (r - r_c)
    A = np.stack([k, np.ones_like(k)], axis=1)
    (s, b), *_ = np.linalg.lstsq(A, np.asarray(rho, dtype=np.float64), rcond=None)
    a1 = 1.0 / b
    return float(a1), float(b / (2.0 * s))


def fit_sigma_alpha(r, sigma, alphas):
    """Eq. sigma-alpha: sigma = a0 exp(-2 alpha r) + a1.  For each trial alpha the
    model is linear in (a0, a1); returns (a0, a1, alpha) of the smallest residual."""
    r = np.asarray(r, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    best = None
    for al in np.asarray(alphas, dtype=np.float64):
        A = np.stack([np.exp(-2.0 * al * r), np.ones_like(r)], axis=1)
        coef, *_ = np.linalg.lstsq(A, sigma, rcond=None)
        res = float(np.sum((A @ coef - sigma) ** 2))
        if best is None or res < best[0]:
            best = (res, float(coef[0]), float(coef[1]), float(al))
    return best[1], best[2], best[3]


def spin_sum(sigma_up, sigma_down):
    """Collinear spin-polarised conductivity (Sec. IV, Fe-Si): the two spin channels are
    computed separately and summed."""
    return np.asarray(sigma_up) + np.asarray(sigma_down)


def resistivity_xx(sigma):
    """rho_xx = [(Re sigma)^{-1}]_xx for sigma [..., 3, 3]."""
    return np.linalg.inv(np.real(np.asarray(sigma)))[..., 0, 0]
