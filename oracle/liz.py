"""Local interaction zone (oracle, test infrastructure).

Sec. II.A (Fig. 1): each atom m sees only the sites within the LIZ radius;
scattering to sites beyond it is dropped (tau^{mn} = 0).  The conductivity sum
of Eq. (lsms-conductivity-formula) runs over n in LIZ_m.

Readings: a site is included iff |d| <= r_LIZ + 1e-8 bohr; periodic images are
distinct sites (an atom may recur); the centre (d = 0) is included and comes
first; the remaining sites are ordered by (atom index, image i, j, k), where the
site is pos[j] + i a1 + j a2 + k a3.  With lattice None the cluster is finite
(no images).

Brute force: every atom and every lattice translation in a box large enough to
contain the sphere is tested.
"""
import itertools

import numpy as np

LIZ_TOL = 1e-8


def build_liz(pos, lattice, r_liz, atoms=None):
    """Returns dict(offsets [N+1], site_atom [S], disp [S,3], image [S,3]).

    ``atoms``: build only the LIZ of these centre atoms, in the order given
    (offsets then has len(atoms) + 1 entries; site_atom keeps global atom
    indices).  The same test is applied to each centre either way."""
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    if lattice is None:
        shifts = [(0, 0, 0)]
        lat = np.zeros((3, 3))
    else:
        lat = np.asarray(lattice, dtype=np.float64)
        vol = abs(np.linalg.det(lat))
        spacing = [vol / np.linalg.norm(np.cross(lat[(i + 1) % 3], lat[(i + 2) % 3])) for i in range(3)]
        span = np.ptp(pos, axis=0).max() * np.sqrt(3) if N > 1 else 0.0
        nmax = [int(np.ceil((r_liz + span) / s)) + 1 for s in spacing]
        shifts = list(itertools.product(*[range(-n, n + 1) for n in nmax]))
    shift_arr = np.asarray(shifts, dtype=np.int64)
    tvec = shift_arr.astype(np.float64) @ lat                       # [n_shift, 3]
    offsets = [0]
    site_atom, disp, image = [], [], []
    for m in (range(N) if atoms is None else atoms):
        d = pos[None, :, :] + tvec[:, None, :] - pos[m][None, None, :]   # [n_shift, N, 3]
        inside = np.linalg.norm(d, axis=-1) <= r_liz + LIZ_TOL
        found = []
        for si, j in zip(*np.nonzero(inside)):
            sh = tuple(int(v) for v in shift_arr[si])
            centre = (j == m and sh == (0, 0, 0))
            found.append((0 if centre else 1, int(j), sh[0], sh[1], sh[2], d[si, j]))
        found.sort(key=lambda t: t[:5])
        for t in found:
            site_atom.append(t[1])
            image.append(t[2:5])
            disp.append(t[5])
        offsets.append(len(site_atom))
    return dict(offsets=np.asarray(offsets, dtype=np.int64),
                site_atom=np.asarray(site_atom, dtype=np.int64),
                disp=np.asarray(disp, dtype=np.float64).reshape(-1, 3),
                image=np.asarray(image, dtype=np.int64).reshape(-1, 3))
