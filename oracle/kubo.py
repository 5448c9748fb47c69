"""Kubo-Greenwood conductivity in the LSMS restriction (oracle, test infrastructure).

Eq. (lsms-conductivity-formula):
  sigma~_{mu nu}(z1, z2) = -(4 m_e^2 / (pi N Omega hbar^3))
      sum_m sum_{n in LIZ_m} Tr[ J^{m mu}(z2, z1) tau^{mn}(z1) J^{n nu}(z1, z2) tau^{nm}(z2) ]
with the index order L4 L1, L1 L2, L2 L3, L3 L4 of that equation, i.e. a matrix
trace.  Eq. (sigma-tilde-consolidation) at finite delta (the limit is not taken):
  sigma = 1/4 [ s~(++) - s~(+-) - s~(-+) + s~(--) ],  z+- = E_F +- i delta.
The resistivity is the inverse of the conductivity tensor (end of Sec. II.B);
reading: rho = (Re sigma)^{-1}.

Readings: Rydberg units (hbar = 1, m_e = 1/2) make 4 m_e^2 / hbar^3 = 1; N Omega is
the supercell volume V; no spin factor.  tau^{mn} with m the centre is the row
block tau^{0n} of LIZ_m, tau^{nm} the column block tau^{n0}.

Current matrices are indexed by the energy pair (z_a, z_b) in the order
c = 0: (+,+), 1: (+,-), 2: (-,+), 3: (-,-); the site-m factor of combination
c = (z1, z2) uses the swapped pair (z2, z1).
"""
import numpy as np

from .sph import gaunt_real, lm_index

COMBOS = ((0, 0), (0, 1), (1, 0), (1, 1))  # (z1, z2) as 0 = +, 1 = -
SWAP = (0, 2, 1, 3)
SIGNS = (1.0, -1.0, -1.0, 1.0)
MU_M = (1, -1, 0)  # Cartesian x, y, z <-> real-harmonic m of l = 1


def sigma_tilde(liz, J_atom, tau_col, tau_row, n_delta, volume, atoms=None):
    """sigma~ [n_delta, 4, 3, 3] complex128.

    J_atom [n_atoms, 4, 3, K, K] or [n_delta, n_atoms, 4, 3, K, K];
    tau_col / tau_row [2 n_delta, S_total, K, K] with energies ordered
    (delta_0 +, delta_0 -, delta_1 +, ...).  ``atoms`` restricts the sum over
    centres m (a partial sum, for sampled checks)."""
    off, sa = liz['offsets'], liz['site_atom']
    N = len(off) - 1
    out = np.zeros((n_delta, 4, 3, 3), dtype=np.complex128)
    for d in range(n_delta):
        Jd = J_atom[d] if J_atom.ndim == 6 else J_atom
        for c, (a, b) in enumerate(COMBOS):
            e1, e2 = 2 * d + a, 2 * d + b
            for m in (range(N) if atoms is None else atoms):
                for s in range(off[m], off[m + 1]):
                    n_atom = sa[s]
                    for mu in range(3):
                        for nu in range(3):
                            prod = (Jd[m, SWAP[c], mu] @ tau_row[e1, s]
                                    @ Jd[n_atom, c, nu] @ tau_col[e2, s])
                            out[d, c, mu, nu] += np.trace(prod)
    return -out / (np.pi * volume)


def consolidate(sig_tilde):
    """sigma [n_delta, 3, 3] from sigma~ [n_delta, 4, 3, 3]."""
    return 0.25 * sum(SIGNS[c] * sig_tilde[:, c] for c in range(4))


def resistivity(sigma):
    """rho = (Re sigma)^{-1} per delta, [n_delta, 3, 3] float64."""
    return np.linalg.inv(np.real(sigma))


def dipole_current(lmax, r_ll):
    """Dipole current-matrix model: J^{mu}_{LL'} = r_{l l'} C_{L L' (1, m_mu)}
    for |l - l'| = 1, zero otherwise.

    r_ll [n_species, 4, lmax+1, lmax+1] complex (one radial factor per energy
    pair) -> J [n_species, 4, 3, K, K] complex128."""
    r_ll = np.asarray(r_ll, dtype=np.complex128)
    K = (lmax + 1) ** 2
    C = gaunt_real(lmax, lmax, 1)
    lof = np.array([int(np.floor(np.sqrt(L) + 1e-12)) for L in range(K)])
    J = np.zeros(r_ll.shape[:2] + (3, K, K), dtype=np.complex128)
    for mu in range(3):
        L3 = lm_index(1, MU_M[mu])
        for L in range(K):
            for Lp in range(K):
                if abs(lof[L] - lof[Lp]) == 1:
                    J[:, :, mu, L, Lp] = r_ll[:, :, lof[L], lof[Lp]] * C[L, Lp, L3]
    return J
