"""Gradient of the conductivity with respect to per-site inverse t-matrices
(oracle, test infrastructure).

f = sum_{d, mu, nu} conj(w_{d mu nu}) sigma_{d mu nu}, sigma from
Eq. (lsms-conductivity-formula) and Eq. (sigma-tilde-consolidation).  Each
sigma~ term depends on t^{-1}_i(z_e) through the blocks of the LIZ inverses.
From Eq. (tau-inverse), tau = M^{-1}, a change dX of the diagonal block of
site p gives d tau = -tau dM tau, i.e.

  d tau^{0n} = -tau^{0p} dX tau^{pn},   d tau^{n0} = -tau^{np} dX tau^{p0}.

This module forms the explicit FULL inverse of every LIZ matrix and applies
these two relations term by term (no adjoint solves).  It returns the
holomorphic derivative D[e, i] = df / d t^{-1}_i(z_e) (a K x K matrix with
df = sum_ab D_ab dX_ab) summed over every site that is an image of atom i;
``torch_grad`` turns it into PyTorch's convention for a real loss
L = Re f: dL/dRe X + i dL/dIm X = conj(D).
"""
import numpy as np

from .kkr import kkr_matrix
from .kubo import COMBOS, SIGNS, SWAP


def dense_gradient(lmax, liz, tinv_atom, z, J_atom, n_delta, volume, w, atoms=None):
    """D [2 n_delta, n_atoms, K, K].  w [n_delta, 3, 3] complex weights.

    ``atoms`` restricts the centres m whose LIZ terms are differentiated
    (the derivative of the partial sum over those centres)."""
    K = (lmax + 1) ** 2
    off, sa, disp = liz['offsets'], liz['site_atom'], liz['disp']
    N = len(off) - 1
    nE = 2 * n_delta
    D = np.zeros((nE, N, K, K), dtype=np.complex128)
    for m in (range(N) if atoms is None else atoms):
        s0, s1 = off[m], off[m + 1]
        S = s1 - s0
        sites = sa[s0:s1]
        T = []
        for e in range(nE):
            M = kkr_matrix(lmax, disp[s0:s1], tinv_atom[sites, e], z[e])
            # full inverse as blocks T[p, q] = tau^{pq}
            T.append(np.linalg.inv(M).reshape(S, K, S, K).transpose(0, 2, 1, 3))
        for d in range(n_delta):
            Jd = J_atom[d] if J_atom.ndim == 6 else J_atom
            for c, (a, b) in enumerate(COMBOS):
                e1, e2 = 2 * d + a, 2 * d + b
                T1, T2 = T[e1], T[e2]
                for nu in range(3):
                    # sum over mu folded into the site-m factor
                    coef = -SIGNS[c] / (4.0 * np.pi * volume) * np.conj(w[d, :, nu])
                    A = np.einsum('u,uab->ab', coef, Jd[m, SWAP[c], :])
                    B = Jd[sites, c, nu]                              # [S, K, K]
                    # via tau^{0n}(z1):  -sum_n tau^{0p} dX tau^{pn} B_n tau^{n0}(z2)
                    Q = np.einsum('qab,qbc->qac', B, T2[:, 0])         # B_n tau^{n0}(z2)
                    W = np.einsum('pqab,qbc->pac', T1, Q)              # sum_n tau^{pn}(z1) Q_n
                    acc1 = np.einsum('pab,bc,pcd->pad', W, A, T1[0])  # ... A tau^{0p}(z1)
                    # via tau^{n0}(z2):  -sum_n tau^{0n}(z1) B_n tau^{np} dX tau^{p0}
                    R = np.einsum('qab,qbc->qac', T1[0], B)             # tau^{0n}(z1) B_n
                    V = np.einsum('qab,qpbc->pac', R, T2)              # sum_n R_n tau^{np}(z2)
                    acc2 = np.einsum('pab,bc,pcd->pad', T2[:, 0], A, V)  # tau^{p0}(z2) A V_p
                    np.add.at(D[e1], sites, -np.transpose(acc1, (0, 2, 1)))
                    np.add.at(D[e2], sites, -np.transpose(acc2, (0, 2, 1)))
    return D


def torch_grad(D):
    """PyTorch convention for a real loss L = Re f: conj of the holomorphic derivative."""
    return np.conj(D)
