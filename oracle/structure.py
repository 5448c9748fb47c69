"""Free-electron propagator g^{nm}_{LL'}(z) (oracle, test infrastructure).

Eq. (tau-inverse) defines tau = [T^{-1} - g]^{-1} with g the free-electron
propagator between sites, in the same (l, m) basis; the paper names g but does
not print it.  Reading (Rydberg units, hbar = 2m = 1, so kappa = sqrt(z) as in
the kappa of the LIZ-radius section):

  g^{nm}_{LL'}(z) = -4 pi i kappa  sum_{L''} i^{l-l'-l''} C_{L L' L''} h^(1)_{l''}(kappa R) Y_{L''}(R^),
  R = R_m - R_n  (row site n, column site m),  kappa = principal sqrt(z),  Im z >= 0;

  for Im z < 0 (the advanced side z = E_F - i delta) the propagator is the one
  that decays, -e^{-i kappa |r|}/(4 pi |r|), whose expansion is
  g = +4 pi i kappa sum i^{l-l'-l''} C h^(2)_{l''}(kappa R) Y_{L''}(R^),
  so that g(z*) = conj g(z).

g^{nm} is defined by the two-centre expansion of the free Green function
-e^{i kappa |r - r'|}/(4 pi |r - r'|), r = R_n + r_n, r' = R_m + r_m:
  sum_{LL'} j_l(kappa r_n) Y_L(r_n^) g^{nm}_{LL'} j_l'(kappa r_m) Y_L'(r_m^).
The sign of R and the power of i are pinned against that expansion in the
tests (and g_{00,00} = -e^{i kappa R}/R).  On-site blocks (n = m) are zero.
"""
from functools import lru_cache

import numpy as np

from .hankel import h1, h2
from .sph import gaunt_real, lm_of, real_ylm


def kappa_of(z):
    """Principal square root of the complex energy (Rydberg units)."""
    return np.sqrt(np.complex128(z))


@lru_cache(maxsize=None)
def _coupling(lmax):
    """P[L, L', L''] = i^{l - l' - l''} C_{L L' L''} (complex128), l'' <= 2 lmax."""
    l3 = 2 * lmax
    K, K3 = (lmax + 1) ** 2, (l3 + 1) ** 2
    C = gaunt_real(lmax, lmax, l3)
    l = np.array([lm_of(L)[0] for L in range(K3)])
    phase = (1j) ** ((l[:K, None, None] - l[None, :K, None] - l[None, None, :]) % 4)
    return phase * C


def g_blocks(lmax, R, z):
    """g^{nm}_{LL'} for a batch of separations R = R_m - R_n, shape [..., 3].

    Returns complex128 [..., K, K]."""
    R = np.asarray(R, dtype=np.float64)
    d = np.linalg.norm(R, axis=-1)
    if np.any(d == 0.0):
        raise ValueError("g is not defined for coincident sites")
    l3 = 2 * lmax
    kap = kappa_of(z)
    Y = real_ylm(l3, R)                                      # [..., K3]
    hank = h1 if np.imag(z) >= 0 else h2
    pref = (-4j if np.imag(z) >= 0 else 4j) * np.pi * kap
    lpp = np.array([lm_of(L)[0] for L in range((l3 + 1) ** 2)])
    hl = np.stack([hank(l, kap * d) for l in range(l3 + 1)], axis=-1)  # [..., l3+1]
    v = hl[..., lpp] * Y                                      # h_{l''}(kR) Y_{L''}(R^)
    return pref * np.einsum('abc,...c->...ab', _coupling(lmax), v)


def g_block(lmax, R, z):
    """g^{nm}_{LL'} for one separation R = R_m - R_n (3-vector), energy z.

    Returns complex128 [(lmax+1)^2, (lmax+1)^2]."""
    return g_blocks(lmax, np.asarray(R, dtype=np.float64)[None, :], z)[0]
