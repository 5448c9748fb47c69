"""KKR matrix and scattering-path blocks of one LIZ (oracle, test infrastructure).

Eq. (tau-inverse): tau = [T^{-1} - g]^{-1}, T^{mn} = t^m delta^{mn}.  Within the
LIZ of centre atom m (sites p = 0..S-1, site 0 the centre) the oracle builds the
dense matrix M (n = K S) with diagonal blocks t^{-1} of the site's species and
off-diagonal blocks -g^{pq}(z), and takes

  tau^{p0} = block rows of  M^{-1} E0   (column block, numpy.linalg.solve),
  tau^{0p} = block columns of (M^{-T} E0)^T   (row block, its own solve),

E0 = the first K columns of the identity.  No symmetry of M is assumed.
"""
import numpy as np

from .structure import g_blocks


def kkr_matrix(lmax, disp, site_tinv, z):
    """M for one LIZ.  disp [S,3] site positions relative to the centre,
    site_tinv [S, K, K] the t^{-1} block of each site at energy z."""
    K = (lmax + 1) ** 2
    S = disp.shape[0]
    blocks = np.zeros((S, S, K, K), dtype=np.complex128)
    p, q = np.nonzero(~np.eye(S, dtype=bool))
    # row site p, column site q: R = R_q - R_p
    blocks[p, q] = -g_blocks(lmax, disp[q] - disp[p], z)
    blocks[np.arange(S), np.arange(S)] = site_tinv
    return blocks.transpose(0, 2, 1, 3).reshape(S * K, S * K)


def tau_col_row(M, K):
    """(column block [S,K,K] with [p] = tau^{p0}, row block [S,K,K] with [p] = tau^{0p})."""
    n = M.shape[0]
    E0 = np.zeros((n, K), dtype=np.complex128)
    E0[:K, :K] = np.eye(K)
    X = np.linalg.solve(M, E0)
    Y = np.linalg.solve(M.T, E0)
    S = n // K
    col = X.reshape(S, K, K)
    row = np.transpose(Y.reshape(S, K, K), (0, 2, 1))
    return col, row


def tau_blocks(lmax, liz, tinv_atom, z, atoms=None, return_rows=False):
    """tau^{p0} for every site of every LIZ (or of ``atoms`` only).

    tinv_atom [n_atoms, n_energy, K, K] (t^{-1} of each atom; a species table
    indexed by atom), z [n_energy].  Returns complex128
    [n_energy, S_total, K, K] (rows of atoms not requested are left zero) and,
    if asked, the row blocks tau^{0p} in the same layout.
    """
    K = (lmax + 1) ** 2
    off, sa, disp = liz['offsets'], liz['site_atom'], liz['disp']
    N = len(off) - 1
    nE = len(z)
    col = np.zeros((nE, off[-1], K, K), dtype=np.complex128)
    row = np.zeros_like(col)
    for m in (range(N) if atoms is None else atoms):
        s0, s1 = off[m], off[m + 1]
        for e in range(nE):
            M = kkr_matrix(lmax, disp[s0:s1], tinv_atom[sa[s0:s1], e], z[e])
            c, r = tau_col_row(M, K)
            col[e, s0:s1] = c
            row[e, s0:s1] = r
    return (col, row) if return_rows else col
