"""LIZ-radius extrapolation (Sec. II.C, Sec. IV) pinned by the fitted forms the
paper prints for the bcc Al_x V_{1-x} alloys and Fe-9 wt% Si: points generated
from each printed form are fitted back and must return its coefficients, and
the two bounds must bracket each other as the paper states."""
import os

import numpy as np
import pytest

from paper_2311_12134_gb300 import extrapolate as ex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "liz_fits.txt")


def _rows():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, c0, c1, b0, b1 = line.split()
                out.append((name, float(c0), float(c1), float(b0), float(b1)))
    return out


R = np.linspace(8.0, 24.0, 9)


@pytest.mark.parametrize("name,c0,c1,b0,b1", _rows())
def test_fits_recover_printed_coefficients(name, c0, c1, b0, b1):
    lower = c0 / R + c1
    g0, g1 = ex.fit_lower_bound(R, lower)
    assert abs(g0 - c0) < 1e-9 * c0 and abs(g1 - c1) < 1e-9 * c1
    upper = b0 / (1.0 + b1 * np.exp(-0.15 * R))
    h0, h1 = ex.fit_upper_bound(R, upper)
    assert abs(h0 - b0) < 1e-9 * b0 and abs(h1 - b1) < 1e-9 * abs(b1)
    # extrapolated residual resistivities: lower bound below upper bound
    assert g1 < h0


@pytest.mark.parametrize("name,c0,c1,b0,b1", _rows())
def test_bounds_bracket_over_the_printed_range(name, c0, c1, b0, b1):
    """The paper bounds rho between the two forms; at large radii the lower form lies
    below the upper one (their asymptotes are c1 < b0 in every caption)."""
    r = np.linspace(40.0, 200.0, 50)
    assert np.all(c0 / r + c1 <= b0 / (1.0 + b1 * np.exp(-0.15 * r)) + 1e-9)


def test_linear_law_and_sigma_alpha_roundtrip():
    a1, alpha, r_c = 0.02, 0.01, 2.5
    r = np.linspace(6.0, 14.0, 7)
    rho = (1.0 + 2 * alpha * (r - r_c)) / (2 * alpha * a1 * (r - r_c))
    # the exact small-alpha form of Eq. linear-fit is linear in k = 1/(r - r_c)
    g_a1, g_alpha = ex.fit_linear_law(r, rho, r_c)
    assert abs(g_a1 - a1) < 1e-12 and abs(g_alpha - alpha) < 1e-12
    a0, a1s, al = 3.0, 1.5, 0.07
    sig = a0 * np.exp(-2 * al * r) + a1s
    f0, f1, fal = ex.fit_sigma_alpha(r, sig, np.linspace(0.01, 0.2, 191))
    assert abs(fal - al) < 1e-12 and abs(f0 - a0) < 1e-9 and abs(f1 - a1s) < 1e-12


def test_spin_sum_and_rho():
    up = np.diag([2.0, 2.0, 2.0]).astype(complex)
    dn = np.diag([1.0, 1.0, 1.0]).astype(complex)
    s = ex.spin_sum(up, dn)
    assert np.allclose(ex.resistivity_xx(s), 1.0 / 3.0)
