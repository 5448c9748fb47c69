"""Seeded synthetic workloads shaped like the paper's supercells (Sec. III, Sec. IV).

This module only draws and lays out inputs; it holds none of the conductivity
method's arithmetic (no structure constants, harmonics, Gaunt coefficients,
solves or traces), so the CUDA library and the CPU oracle can both be fed from
it.

The paper runs self-consistent potentials on 16,000-atom bcc and 16,384-atom fcc
supercells of pure metals and random alloys (Sec. III); those potentials are not
available, so every input here is synthetic:

* structure: fcc or bcc supercells of n^3 conventional cells (lattice constant
  a, cubic box of side L = n a), random species assignment with exact counts,
  random vacancies (sites removed), Gaussian displacements per Cartesian
  component;
* single-site scattering (stand-in for the radial solver of Sec. II.A): a
  t-matrix diagonal in L from per-species phase shifts,
  t_l(z) = -sin(d_l) e^{+i d_l} / sqrt(z) for Im z >= 0 and
  t_l(z) = -sin(d_l) e^{-i d_l} / sqrt(z) for Im z < 0 (principal root), so that
  t(z*) = conj t(z) and Im t^{-1} = sqrt(E) on the real axis;
  the library takes t^{-1} as input;
* current matrices (stand-in for the matrix elements J of the Kubo-Greenwood
  formula): radial factors r_{l l'} per species and energy pair,
  r(+,+) = u (1 + 0.2 i), r(-,-) = conj r(+,+), r(+,-) = r(-,+) = |1 + 0.2 i| u,
  u ~ U(0.1, 1) for |l - l'| = 1 and zero otherwise; the dipole model turns them
  into J^mu_{LL'} = r_{l l'} C_{L L' (1 mu)} on each side separately.

Random streams are drawn in a fixed order from numpy's default_rng(seed):
species permutation, vacancies, displacements, current-matrix factors.
"""
from dataclasses import dataclass, field

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
BCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])

# Phase shifts (rad) for l = 0..3 used by the workloads below.
PHASE_PURE = (0.45, 0.12, 0.30, 0.01)
PHASE_A = (0.40, 0.10, 0.05, 0.005)
PHASE_B = (0.55, 0.35, 1.20, 0.02)


@dataclass
class Workload:
    name: str
    lmax: int
    pos: np.ndarray            # [N, 3] bohr
    lattice: np.ndarray        # [3, 3] rows a1, a2, a3 (bohr); None for a finite cluster
    species: np.ndarray        # [N] int32
    r_liz: float               # bohr
    z: np.ndarray              # [2 n_delta] complex128, (E_F + i d, E_F - i d) per delta
    tinv: np.ndarray           # [n_species, 2 n_delta, K, K] complex128
    r_ll: np.ndarray           # [n_species, 4, lmax+1, lmax+1] complex128
    volume: float              # bohr^3
    n_delta: int
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self):
        return self.pos.shape[0]

    @property
    def n_species(self):
        return self.tinv.shape[0]

    @property
    def K(self):
        return (self.lmax + 1) ** 2


def lattice_sites(kind, n_cells, a):
    basis = {"fcc": FCC_BASIS, "bcc": BCC_BASIS}[kind]
    g = np.arange(n_cells)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    pos = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos, np.eye(3) * (n_cells * a)


def energies(e_fermi, deltas):
    z = []
    for d in deltas:
        z += [complex(e_fermi, d), complex(e_fermi, -d)]
    return np.asarray(z, dtype=np.complex128)


def tinv_from_phase_shifts(phases, z, lmax):
    """[n_species, n_energy, K, K]: diagonal t^{-1}_l(z) of the phase-shift model."""
    K = (lmax + 1) ** 2
    out = np.zeros((len(phases), len(z), K, K), dtype=np.complex128)
    for s, ph in enumerate(phases):
        for e, ze in enumerate(z):
            k = np.sqrt(np.complex128(ze))
            sign = 1.0 if ze.imag >= 0 else -1.0
            for L in range(K):
                l = int(np.floor(np.sqrt(L) + 1e-12))
                d = ph[l]
                t = -np.sin(d) * np.exp(sign * 1j * d) / k
                out[s, e, L, L] = 1.0 / t
    return out


def draw_r_ll(rng, n_species, lmax):
    """Radial factors of the dipole current model, [n_species, 4, lmax+1, lmax+1]."""
    r = np.zeros((n_species, 4, lmax + 1, lmax + 1), dtype=np.complex128)
    c = 1.0 + 0.2j
    for s in range(n_species):
        u = rng.uniform(0.1, 1.0, size=(lmax + 1, lmax + 1))
        for l in range(lmax + 1):
            for lp in range(lmax + 1):
                if abs(l - lp) != 1:
                    continue
                r[s, 0, l, lp] = u[l, lp] * c
                r[s, 1, l, lp] = u[l, lp] * abs(c)
                r[s, 2, l, lp] = u[l, lp] * abs(c)
                r[s, 3, l, lp] = u[l, lp] * np.conj(c)
    return r


def make_supercell(*, name, kind, n_cells, a, counts, n_vacancies=0, sigma_disp=0.0,
                   r_liz, phases, e_fermi, deltas, lmax=3, seed):
    """Generic seeded supercell workload.  ``counts`` = sites per species (sum = all
    lattice sites); vacancies are then removed at random."""
    rng = np.random.default_rng(seed)
    pos, lattice = lattice_sites(kind, n_cells, a)
    n_sites = pos.shape[0]
    if sum(counts) != n_sites:
        raise ValueError("species counts must cover every lattice site")
    species = np.concatenate([np.full(c, s, dtype=np.int32) for s, c in enumerate(counts)])
    species = species[rng.permutation(n_sites)]
    keep = np.ones(n_sites, dtype=bool)
    if n_vacancies:
        keep[rng.choice(n_sites, size=n_vacancies, replace=False)] = False
    pos, species = pos[keep], species[keep]
    if sigma_disp > 0:
        pos = pos + rng.normal(0.0, sigma_disp, size=pos.shape)
    r_ll = draw_r_ll(rng, len(counts), lmax)
    z = energies(e_fermi, deltas)
    return Workload(name=name, lmax=lmax, pos=np.ascontiguousarray(pos), lattice=lattice,
                    species=np.ascontiguousarray(species.astype(np.int32)), r_liz=float(r_liz), z=z,
                    tinv=tinv_from_phase_shifts(phases, z, lmax), r_ll=r_ll,
                    volume=float(abs(np.linalg.det(lattice))), n_delta=len(deltas),
                    meta=dict(kind=kind, n_cells=n_cells, a=a, counts=list(counts),
                              n_vacancies=n_vacancies, sigma_disp=sigma_disp, seed=seed,
                              e_fermi=e_fermi, deltas=list(deltas)))


def fcc_pure_32():
    """fcc 2x2x2 conventional cells (32 atoms), a = 7.72 bohr, one species, LIZ = first
    shell (13 sites, n = 208); E_F = 0.55 Ry, delta = 0.002 Ry."""
    a = 7.72
    return make_supercell(name="fcc32_pure_liz13", kind="fcc", n_cells=2, a=a, counts=[32],
                          r_liz=0.85 * a, phases=[PHASE_PURE], e_fermi=0.55, deltas=[0.002],
                          seed=2311 + 0)


def fcc_alloy_256():
    """fcc 4x4x4 (256 atoms) random A/B at x = 0.5 (128/128), a = 7.65 bohr, LIZ of 3
    shells (43 sites, n = 688); E_F = 0.60 Ry, delta = 0.002 Ry."""
    a = 7.65
    return make_supercell(name="fcc256_AB50_liz43", kind="fcc", n_cells=4, a=a, counts=[128, 128],
                          r_liz=1.30 * a, phases=[PHASE_A, PHASE_B], e_fermi=0.60, deltas=[0.002],
                          seed=2311 + 1)


def bcc_disordered_2000(n_cells=10):
    """bcc 10^3 (2000 sites) A/B 1670/330, 20 vacancies, Gaussian displacements of
    0.05 a per component, a = 5.42 bohr, LIZ radius 1.75 a (uneven LIZ sizes);
    E_F = 0.62 Ry, delta in {0.001, 0.002, 0.004} Ry."""
    a = 5.42
    n_sites = 2 * n_cells ** 3
    n_b = int(round(0.165 * n_sites))
    return make_supercell(name=f"bcc{n_sites}_AB_vac_disp_liz175", kind="bcc", n_cells=n_cells, a=a,
                          counts=[n_sites - n_b, n_b], n_vacancies=int(round(0.01 * n_sites)),
                          sigma_disp=0.05 * a, r_liz=1.75 * a, phases=[PHASE_A, PHASE_B],
                          e_fermi=0.62, deltas=[0.001, 0.002, 0.004], seed=2311 + 2)


def fcc_alloy_500():
    """fcc 5^3 (500 atoms) random A/B at x = 0.3 (350/150), a = 7.65 bohr, LIZ of 4
    shells (55 sites, n = 880); E_F = 0.60 Ry, delta = 0.002 Ry."""
    a = 7.65
    return make_supercell(name="fcc500_AB30_liz55", kind="fcc", n_cells=5, a=a, counts=[350, 150],
                          r_liz=1.50 * a, phases=[PHASE_A, PHASE_B], e_fermi=0.60, deltas=[0.002],
                          seed=2311 + 3)


def bcc_large_16000(r_over_a=2.2, n_cells=20):
    """bcc 20^3 (16,000 sites), 2 % B, 0.5 % vacancies, a = 5.42 bohr; LIZ radius
    1.85 a / 2.2 a / 2.5 a (59 / 89 / 137 sites); E_F = 0.62 Ry, delta = 0.002 Ry."""
    a = 5.42
    n_sites = 2 * n_cells ** 3
    n_b = int(round(0.02 * n_sites))
    return make_supercell(name=f"bcc{n_sites}_B2_vac_liz{r_over_a}a", kind="bcc", n_cells=n_cells, a=a,
                          counts=[n_sites - n_b, n_b], n_vacancies=int(round(0.005 * n_sites)),
                          r_liz=r_over_a * a, phases=[PHASE_A, PHASE_B], e_fermi=0.62,
                          deltas=[0.002], seed=2311 + 4)


def cluster(n_atoms=10, lmax=3, seed=7, spread=9.0, r_liz=100.0, e_fermi=0.55, delta=0.002):
    """Finite random cluster (no lattice), two species; with a LIZ radius larger than
    the cluster every LIZ covers the whole cluster."""
    rng = np.random.default_rng(seed)
    pos = [rng.uniform(-spread, spread, size=3)]
    while len(pos) < n_atoms:
        p = rng.uniform(-spread, spread, size=3)
        if min(np.linalg.norm(p - q) for q in pos) > 3.5:
            pos.append(p)
    pos = np.asarray(pos)
    species = (np.arange(n_atoms) % 2).astype(np.int32)
    r_ll = draw_r_ll(rng, 2, lmax)
    z = energies(e_fermi, [delta])
    phases = [PHASE_A[:lmax + 1], PHASE_B[:lmax + 1]]
    return Workload(name=f"cluster{n_atoms}", lmax=lmax, pos=pos, lattice=None, species=species,
                    r_liz=r_liz, z=z, tinv=tinv_from_phase_shifts(phases, z, lmax), r_ll=r_ll,
                    volume=1000.0, n_delta=1, meta=dict(kind="cluster", seed=seed))


WORKLOADS = {
    "fcc32": fcc_pure_32,
    "fcc256": fcc_alloy_256,
    "bcc2000": bcc_disordered_2000,
    "fcc500": fcc_alloy_500,
    "bcc16000": bcc_large_16000,
}
