"""Real spherical harmonics and real Gaunt coefficients (oracle, test infrastructure).

The paper expands the site Green function over angular-momentum channels
L = (l, m) (Sec. II.A, the expression for G(r_n, r_n, e) and the text after it)
but does not fix the harmonic convention.  Reading used throughout: real
harmonics without the Condon-Shortley phase, so that Y_{1,+1}, Y_{1,-1}, Y_{1,0}
are proportional to x, y, z; channel index L = l*l + l + m.

Y_lm(r^) = sqrt(2) N_l^m P_l^m(cos t) cos(m p)      m > 0
         = N_l^0 P_l(cos t)                        m = 0
         = sqrt(2) N_l^|m| P_l^|m|(cos t) sin(|m| p) m < 0
N_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),  P_l^m(x) = (1-x^2)^{m/2} d^m P_l/dx^m.

Here P_l is written out from its explicit coefficient sum, differentiated m times
with exact integer arithmetic, and (1-x^2)^{m/2} e^{i m p} is evaluated as
(x + i y)^m for a unit vector -- a direct evaluation of the definition, not a
recurrence.

Gaunt coefficients C_{L1 L2 L3} = integral of Y_L1 Y_L2 Y_L3 over the unit sphere,
by Gauss-Legendre quadrature in cos(t) times a uniform grid in p, both exact
for the polynomial degree involved.
"""
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial, pi, sqrt

import numpy as np


def lm_index(l, m):
    return l * l + l + m


def lm_of(L):
    l = int(np.floor(np.sqrt(L) + 1e-12))
    while (l + 1) * (l + 1) <= L:
        l += 1
    while l * l > L:
        l -= 1
    return l, L - l * l - l


@lru_cache(maxsize=None)
def _legendre_deriv_coeffs(l, m):
    """Coefficients c_p of d^m P_l / dx^m = sum_p c_p x^p, exact rationals."""
    coeff = [Fraction(0)] * (l + 1)
    for k in range(l // 2 + 1):
        coeff[l - 2 * k] += Fraction((-1) ** k * comb(l, k) * comb(2 * l - 2 * k, l), 2 ** l)
    for _ in range(m):
        coeff = [coeff[p + 1] * (p + 1) for p in range(len(coeff) - 1)] or [Fraction(0)]
    return tuple(float(c) for c in coeff)


def real_ylm(lmax, vec):
    """Y_L(r^) for L < (lmax+1)^2 at directions ``vec`` [..., 3] (need not be unit).

    Returns float64 [..., (lmax+1)^2].
    """
    vec = np.asarray(vec, dtype=np.float64)
    r = np.linalg.norm(vec, axis=-1)
    if np.any(r == 0):
        raise ValueError("Y_L is undefined for a zero vector")
    x, y, z = (vec[..., i] / r for i in range(3))
    xy = x + 1j * y
    out = np.zeros(vec.shape[:-1] + ((lmax + 1) ** 2,), dtype=np.float64)
    for l in range(lmax + 1):
        for m in range(l + 1):
            c = _legendre_deriv_coeffs(l, m)
            poly = np.zeros_like(z)
            for p, cp in enumerate(c):
                poly = poly + cp * z ** p
            norm = sqrt((2 * l + 1) / (4 * pi) * factorial(l - m) / factorial(l + m))
            if m == 0:
                out[..., lm_index(l, 0)] = norm * poly
            else:
                trig = xy ** m  # sin^m(t) e^{i m p}
                out[..., lm_index(l, m)] = sqrt(2.0) * norm * poly * trig.real
                out[..., lm_index(l, -m)] = sqrt(2.0) * norm * poly * trig.imag
    return out


def sphere_quadrature(degree):
    """Nodes and weights integrating every polynomial of total degree <= ``degree``
    on the unit sphere exactly: Gauss-Legendre in cos(t) x uniform in p."""
    n_t = degree // 2 + 2
    n_p = degree + 2
    ct, wt = np.polynomial.legendre.leggauss(n_t)
    ph = 2 * pi * np.arange(n_p) / n_p
    st = np.sqrt(1 - ct ** 2)
    nodes = np.stack(np.broadcast_arrays(st[:, None] * np.cos(ph)[None, :],
                                         st[:, None] * np.sin(ph)[None, :],
                                         ct[:, None] * np.ones(n_p)[None, :]), axis=-1).reshape(-1, 3)
    w = (wt[:, None] * np.full(n_p, 2 * pi / n_p)[None, :]).reshape(-1)
    return nodes, w


@lru_cache(maxsize=None)
def gaunt_real(l1max, l2max, l3max):
    """C[L1, L2, L3] = int Y_L1 Y_L2 Y_L3 dOmega, L_i < (l_imax+1)^2 (float64)."""
    nodes, w = sphere_quadrature(l1max + l2max + l3max)
    lm = max(l1max, l2max, l3max)
    Y = real_ylm(lm, nodes)
    n1, n2, n3 = (l1max + 1) ** 2, (l2max + 1) ** 2, (l3max + 1) ** 2
    C = np.einsum('q,qa,qb,qc->abc', w, Y[:, :n1], Y[:, :n2], Y[:, :n3], optimize=True)
    # The integral vanishes unless l1 + l2 + l3 is even and (l1, l2, l3) obey
    # the triangle rule; zero those entries exactly instead of keeping the
    # quadrature's rounding noise (which h_l of high order would amplify).
    l1 = np.array([lm_of(L)[0] for L in range(n1)])[:, None, None]
    l2 = np.array([lm_of(L)[0] for L in range(n2)])[None, :, None]
    l3 = np.array([lm_of(L)[0] for L in range(n3)])[None, None, :]
    allowed = ((l1 + l2 + l3) % 2 == 0) & (l3 <= l1 + l2) & (l3 >= np.abs(l1 - l2))
    C = np.where(allowed, C, 0.0)
    C[np.abs(C) < 1e-14] = 0.0
    return C
