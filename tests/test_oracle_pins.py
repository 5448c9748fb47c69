"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
closed forms, library routines (scipy, sympy), textbook values, invariants,
special cases of Eq. (tau-inverse) and brute force.  CPU only.
"""
import os

import numpy as np
import pytest

from oracle import grad, hankel, kkr, kubo, liz, sph, structure
from paper_2311_12134_gb300 import workload as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- harmonics
def test_ylm_orthonormal_and_low_order():
    nodes, w = sph.sphere_quadrature(16)
    Y = sph.real_ylm(8, nodes)
    G = np.einsum("q,qa,qb->ab", w, Y, Y)
    assert np.abs(G - np.eye(81)).max() < 1e-13
    v = np.array([[0.3, -0.4, 0.5], [-1.0, 2.0, 0.25]])
    Y1 = sph.real_ylm(1, v)
    r = np.linalg.norm(v, axis=1)
    assert np.allclose(Y1[:, 0], 1 / np.sqrt(4 * np.pi), atol=1e-15)
    c = np.sqrt(3 / (4 * np.pi))
    # L = 1, 2, 3 <-> m = -1, 0, +1 <-> y, z, x
    assert np.allclose(Y1[:, 1], c * v[:, 1] / r, atol=1e-15)
    assert np.allclose(Y1[:, 2], c * v[:, 2] / r, atol=1e-15)
    assert np.allclose(Y1[:, 3], c * v[:, 0] / r, atol=1e-15)


def test_ylm_matches_scipy_complex_harmonics():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(3)
    v = rng.normal(size=(20, 3))
    r = np.linalg.norm(v, axis=1)
    theta = np.arccos(v[:, 2] / r)
    phi = np.arctan2(v[:, 1], v[:, 0])
    Y = sph.real_ylm(6, v)
    for l in range(7):
        for m in range(-l, l + 1):
            yc = sp.sph_harm_y(l, abs(m), theta, phi)  # Condon-Shortley phase included
            if m > 0:
                ref = np.sqrt(2) * (-1) ** m * yc.real
            elif m < 0:
                ref = np.sqrt(2) * (-1) ** abs(m) * yc.imag
            else:
                ref = yc.real
            assert np.allclose(Y[:, sph.lm_index(l, m)], ref, atol=1e-13), (l, m)


def _complex_to_real(l):
    """U[mu, m]: real harmonic (no Condon-Shortley phase) from complex ones (with it)."""
    U = np.zeros((2 * l + 1, 2 * l + 1), dtype=np.complex128)
    for mu in range(-l, l + 1):
        if mu > 0:
            U[mu + l, mu + l] = (-1) ** mu / np.sqrt(2)
            U[mu + l, -mu + l] = 1 / np.sqrt(2)
        elif mu < 0:
            a = -mu
            U[mu + l, a + l] = (-1) ** a / (np.sqrt(2) * 1j)
            U[mu + l, -a + l] = -1 / (np.sqrt(2) * 1j)
        else:
            U[l, l] = 1.0
    return U


def test_gaunt_matches_wigner_3j_closed_form():
    wig = pytest.importorskip("sympy.physics.wigner")
    lmax, l3max = 3, 6
    C = sph.gaunt_real(lmax, lmax, l3max)
    for l1 in range(lmax + 1):
        for l2 in range(lmax + 1):
            for l3 in range(l3max + 1):
                Gc = np.zeros((2 * l1 + 1, 2 * l2 + 1, 2 * l3 + 1))
                for m1 in range(-l1, l1 + 1):
                    for m2 in range(-l2, l2 + 1):
                        for m3 in range(-l3, l3 + 1):
                            if m1 + m2 + m3 == 0:
                                Gc[m1 + l1, m2 + l2, m3 + l3] = float(wig.gaunt(l1, l2, l3, m1, m2, m3))
                U1, U2, U3 = _complex_to_real(l1), _complex_to_real(l2), _complex_to_real(l3)
                Gr = np.einsum("ai,bj,ck,ijk->abc", U1, U2, U3, Gc)
                assert np.abs(Gr.imag).max() < 1e-14
                sl = C[l1 * l1:(l1 + 1) ** 2, l2 * l2:(l2 + 1) ** 2, l3 * l3:(l3 + 1) ** 2]
                assert np.abs(sl - Gr.real).max() < 1e-13, (l1, l2, l3)


def test_gaunt_identities():
    C = sph.gaunt_real(3, 3, 3)
    assert np.allclose(C[:, :, 0], np.eye(16) / np.sqrt(4 * np.pi), atol=1e-15)
    assert np.allclose(C, C.transpose(1, 0, 2), atol=1e-15)
    assert np.allclose(C, C.transpose(2, 1, 0), atol=1e-15)
    l = np.array([sph.lm_of(L)[0] for L in range(16)])
    odd = (l[:, None, None] + l[None, :, None] + l[None, None, :]) % 2 == 1
    assert np.all(C[odd] == 0)


# ---------------------------------------------------------------- Hankel
@pytest.mark.parametrize("x", [0.7 + 0.001j, 2.3 + 0.01j, 5.5 - 0.004j, 9.1 + 0.02j])
def test_hankel_against_scipy(x):
    sp = pytest.importorskip("scipy.special")
    for l in range(7):
        j, y = sp.spherical_jn(l, x), sp.spherical_yn(l, x)
        ref1, ref2 = j + 1j * y, j - 1j * y
        assert abs(hankel.h1(l, x) - ref1) <= 1e-12 * abs(ref1)
        assert abs(hankel.h2(l, x) - ref2) <= 1e-12 * abs(ref2)
    assert abs(hankel.h1(0, x) - (-1j * np.exp(1j * x) / x)) < 1e-15 * abs(x) ** -1 * 10


# ---------------------------------------------------------------- g
def test_g00_closed_form():
    for z in (0.55 + 0.002j, 0.62 - 0.001j):
        R = np.array([1.3, -2.0, 3.7])
        d = np.linalg.norm(R)
        g = structure.g_block(0, R, z)
        k = np.sqrt(z)
        ref = -np.exp(1j * k * d) / d if z.imag >= 0 else -np.exp(-1j * k * d) / d
        assert abs(g[0, 0] - ref) < 1e-14 * abs(ref)


def test_g_two_centre_expansion():
    """Free Green function -e^{ik|r-r'|}/(4 pi |r-r'|) between displaced points equals
    sum_{LL'} j_l(k r_n) Y_L g^{nm}_{LL'} j_l'(k r_m) Y_L' (pins sign of R, i-powers)."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(11)
    lmax = 8
    K = (lmax + 1) ** 2
    ls = np.array([sph.lm_of(L)[0] for L in range(K)])
    Rn, Rm = np.array([0.2, 0.1, -0.3]), np.array([3.1, -2.2, 4.0])
    for z in (0.55 + 0.002j, 0.55 - 0.002j, 0.9 + 0.05j):
        k = np.sqrt(z)
        g = structure.g_block(lmax, Rm - Rn, z)
        for _ in range(3):
            rn = rng.normal(size=3); rn *= 0.3 / np.linalg.norm(rn)
            rm = rng.normal(size=3); rm *= 0.25 / np.linalg.norm(rm)
            dist = np.linalg.norm(Rn + rn - Rm - rm)
            ex = -np.exp(1j * k * dist) / (4 * np.pi * dist) if z.imag >= 0 else \
                -np.exp(-1j * k * dist) / (4 * np.pi * dist)
            an = sp.spherical_jn(ls, k * np.linalg.norm(rn)) * sph.real_ylm(lmax, rn[None])[0]
            am = sp.spherical_jn(ls, k * np.linalg.norm(rm)) * sph.real_ylm(lmax, rm[None])[0]
            assert abs(an @ g @ am - ex) < 1e-10 * abs(ex)


def test_g_symmetries():
    R = np.array([2.0, 1.0, -3.0])
    z = 0.6 + 0.003j
    g = structure.g_block(3, R, z)
    gT = structure.g_block(3, -R, z)
    assert np.abs(g.T - gT).max() < 1e-13 * np.abs(g).max()      # g^{nm}_{L'L} = g^{mn}_{LL'}
    gm = structure.g_block(3, R, np.conj(z))
    assert np.abs(gm - np.conj(g)).max() < 1e-13 * np.abs(g).max()  # g(z*) = conj g(z)


# ---------------------------------------------------------------- LIZ
def _golden_shells():
    rows = []
    with open(os.path.join(GOLDEN, "shell_counts.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, r, c = line.split()
                rows.append((k, float(r), int(c)))
    return rows


@pytest.mark.parametrize("kind,r_over_a,count", _golden_shells())
def test_liz_shell_counts(kind, r_over_a, count):
    a = 5.0
    pos, lat = wl.lattice_sites(kind, 2, a)
    L = liz.build_liz(pos, lat, r_over_a * a)
    sizes = np.diff(L["offsets"])
    assert np.all(sizes == count)
    assert np.all(L["site_atom"][L["offsets"][:-1]] == np.arange(pos.shape[0]))
    assert np.allclose(L["disp"][L["offsets"][:-1]], 0.0)


# ---------------------------------------------------------------- tau
def _single_species_tinv(phases, z, lmax):
    return wl.tinv_from_phase_shifts([phases], np.atleast_1d(z), lmax)[0]


def test_tau_equals_t_single_site():
    """A LIZ with only the centre has g = 0, so tau = t (Eq. tau-inverse with g = 0)."""
    z = np.array([0.55 + 0.002j])
    tinv = _single_species_tinv(wl.PHASE_B, z, 3)          # [nE, K, K]
    pos = np.zeros((1, 3))
    L = liz.build_liz(pos, None, 1.0)
    col = kkr.tau_blocks(3, L, tinv[None], z)
    assert np.abs(col[0, 0] - np.linalg.inv(tinv[0])).max() < 1e-14


def test_tau_two_site_closed_form():
    z = 0.55 + 0.002j
    k = np.sqrt(z)
    R = 4.3
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    tinv = _single_species_tinv((0.7,), np.array([z]), 0)  # [1, 1, 1]
    L = liz.build_liz(pos, None, 10.0)
    col = kkr.tau_blocks(0, L, np.stack([tinv, tinv]), np.array([z]))
    a = tinv[0, 0, 0]
    b = np.exp(1j * k * R) / R
    det = a * a - b * b
    assert abs(col[0, 0, 0, 0] - a / det) < 1e-13 * abs(a / det)
    assert abs(col[0, 1, 0, 0] - (-b / det)) < 1e-13 * abs(b / det)


def test_dyson_first_order():
    """tau^{10} - t g^{10} t = O(t^3) (Eq. Dyson truncated after the first order): relative
    to t g t the rest is O(t^2), so halving the phase shifts shrinks it 4x."""
    z = 0.55 + 0.002j
    pos = np.array([[0.0, 0.0, 0.0], [2.0, 1.5, 3.0]])
    L = liz.build_liz(pos, None, 10.0)
    rest = []
    for s in (1e-3, 5e-4):
        tinv = _single_species_tinv((s, s, s, s), np.array([z]), 3)
        col = kkr.tau_blocks(3, L, np.stack([tinv, tinv]), np.array([z]))
        t = np.linalg.inv(tinv[0])
        g10 = structure.g_block(3, pos[0] - pos[1], z)   # row site 1, column site 0
        rest.append(np.abs(col[0, 1] - t @ g10 @ t).max() / np.abs(t @ g10 @ t).max())
    assert rest[0] < 1e-2
    assert 3.9 < rest[0] / rest[1] < 4.1


def test_finite_cluster_equals_full_inverse():
    """LIZ covering a whole finite cluster: every LSMS column block equals the block of
    the brute-force inverse of the full cluster KKR matrix (Eq. tau-inverse)."""
    w = wl.cluster(n_atoms=10, lmax=3)
    L = liz.build_liz(w.pos, None, w.r_liz)
    tin = w.tinv[w.species]
    col = kkr.tau_blocks(3, L, tin, w.z)
    K = 16
    for e, z in enumerate(w.z):
        Mfull = kkr.kkr_matrix(3, w.pos - w.pos[0], tin[:, e], z)
        T = np.linalg.inv(Mfull)
        for m in range(w.n_atoms):
            for s in range(L["offsets"][m], L["offsets"][m + 1]):
                n = L["site_atom"][s]
                ref = T[n * K:(n + 1) * K, m * K:(m + 1) * K]
                assert np.abs(col[e, s] - ref).max() <= 1e-12 * np.abs(ref).max() + 1e-15


def test_time_reversal_and_complex_symmetry():
    w = wl.fcc_pure_32()
    L = liz.build_liz(w.pos, w.lattice, w.r_liz)
    tin = w.tinv[w.species]
    col, row = kkr.tau_blocks(3, L, tin, w.z, atoms=[0, 5], return_rows=True)
    s = slice(L["offsets"][5], L["offsets"][6])
    # tau(z-) = tau(z+)^{T*}, blockwise tau^{p0}(z-) = conj(tau^{0p}(z+))^T
    assert np.abs(col[1, s] - np.conj(np.transpose(row[0, s], (0, 2, 1)))).max() < 1e-12 * np.abs(col[0, s]).max()
    # complex symmetry tau^T = tau: tau^{0p} = (tau^{p0})^T
    assert np.abs(row[0, s] - np.transpose(col[0, s], (0, 2, 1))).max() < 1e-12 * np.abs(col[0, s]).max()
    M = kkr.kkr_matrix(3, L["disp"][s], tin[L["site_atom"][s], 0], w.z[0])
    assert np.abs(M - M.T).max() < 1e-13 * np.abs(M).max()


# ---------------------------------------------------------------- sigma
def _sigma_full(w, Lz=None, atoms=None):
    Lz = Lz or liz.build_liz(w.pos, w.lattice, w.r_liz)
    tin = w.tinv[w.species]
    col, row = kkr.tau_blocks(w.lmax, Lz, tin, w.z, atoms=atoms, return_rows=True)
    J = kubo.dipole_current(w.lmax, w.r_ll)[w.species]
    st = kubo.sigma_tilde(Lz, J, col, row, w.n_delta, w.volume, atoms=atoms)
    return kubo.consolidate(st), st, Lz


@pytest.fixture(scope="module")
def fcc32():
    w = wl.fcc_pure_32()
    return w, _sigma_full(w)


def test_pure_crystal_isotropy(fcc32):
    w, (sig, st, Lz) = fcc32
    s = sig[0]
    sxx = s[0, 0].real
    assert sxx > 0
    assert abs(s[1, 1] - sxx) < 1e-12 * abs(sxx) and abs(s[2, 2] - sxx) < 1e-12 * abs(sxx)
    off = s - np.diag(np.diag(s))
    assert np.abs(off).max() < 1e-12 * abs(sxx)
    assert np.abs(s.imag).max() < 1e-12 * abs(sxx)


def test_pure_crystal_equal_atom_contributions(fcc32):
    w, (sig, st, Lz) = fcc32
    tin = w.tinv[w.species]
    J = kubo.dipole_current(w.lmax, w.r_ll)[w.species]
    per = []
    for m in (0, 7, 19, 31):
        col, row = kkr.tau_blocks(w.lmax, Lz, tin, w.z, atoms=[m], return_rows=True)
        per.append(kubo.sigma_tilde(Lz, J, col, row, 1, w.volume, atoms=[m]))
    for p in per[1:]:
        assert np.abs(p - per[0]).max() < 1e-12 * np.abs(per[0]).max()
    assert np.abs(per[0] * w.n_atoms - st).max() < 1e-11 * np.abs(st).max()


def _alloy32(seed=99):
    a = 7.65
    return wl.make_supercell(name="t", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                             r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6,
                             deltas=[0.002], seed=seed)


def test_sigma_covariance_translation_permutation_rotation():
    w = _alloy32()
    s0, _, _ = _sigma_full(w)
    # translation
    w2 = _alloy32(); w2.pos = w2.pos + np.array([1.7, -0.4, 2.2])
    s1, _, _ = _sigma_full(w2)
    assert np.abs(s1 - s0).max() < 1e-11 * np.abs(s0).max()
    # permutation of atoms
    perm = np.random.default_rng(5).permutation(w.n_atoms)
    w3 = _alloy32(); w3.pos = w3.pos[perm]; w3.species = w3.species[perm]
    s2, _, _ = _sigma_full(w3)
    assert np.abs(s2 - s0).max() < 1e-11 * np.abs(s0).max()
    # 90 degree rotation about z: sigma -> R sigma R^T (t isotropic, J a vector operator)
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    w4 = _alloy32(); w4.pos = w4.pos @ Rz.T; w4.lattice = w4.lattice @ Rz.T
    s3, _, _ = _sigma_full(w4)
    assert np.abs(s3[0] - Rz @ s0[0] @ Rz.T).max() < 1e-11 * np.abs(s0).max()
    # the alloy is not isotropic, so the rotation test is not empty
    assert np.abs(s0[0, 0, 0] - s0[0, 1, 1]) > 1e-6 * np.abs(s0).max()
    assert np.abs(s0.imag).max() < 1e-12 * np.abs(s0).max()


def test_lmax0_sigma_vanishes():
    w = wl.make_supercell(name="t", kind="fcc", n_cells=2, a=7.72, counts=[32], r_liz=0.85 * 7.72,
                          phases=[wl.PHASE_PURE], e_fermi=0.55, deltas=[0.002], lmax=0, seed=1)
    sig, st, _ = _sigma_full(w)
    assert np.all(st == 0)


def test_tinv_optical_theorem():
    E = 0.6
    tinv = wl.tinv_from_phase_shifts([wl.PHASE_B], np.array([E + 0j]), 3)[0, 0]
    assert np.allclose(np.diag(tinv).imag, np.sqrt(E), atol=1e-14)


# ---------------------------------------------------------------- gradient
def test_dense_gradient_matches_finite_differences():
    lmax = 1
    w = wl.cluster(n_atoms=3, lmax=lmax, seed=3, spread=4.0, r_liz=6.5)
    L = liz.build_liz(w.pos, None, w.r_liz)
    tin = w.tinv[w.species].copy()
    J = kubo.dipole_current(lmax, w.r_ll)[w.species]
    rng = np.random.default_rng(0)
    wgt = rng.normal(size=(1, 3, 3)) + 1j * rng.normal(size=(1, 3, 3))

    def f(tinv_atom):
        col, row = kkr.tau_blocks(lmax, L, tinv_atom, w.z, return_rows=True)
        s = kubo.consolidate(kubo.sigma_tilde(L, J, col, row, 1, w.volume))
        return np.sum(np.conj(wgt) * s)

    D = grad.dense_gradient(lmax, L, tin, w.z, J, 1, w.volume, wgt)
    h = 1e-6
    for (e, i, a, b) in [(0, 0, 0, 0), (1, 1, 2, 3), (0, 2, 3, 1), (1, 0, 1, 1)]:
        for step in (h, 1j * h):
            tp, tm = tin.copy(), tin.copy()
            tp[i, e, a, b] += step
            tm[i, e, a, b] -= step
            fd = (f(tp) - f(tm)) / (2 * h)
            ref = D[e, i, a, b] * (1 if step == h else 1j)
            assert abs(fd - ref) < 1e-6 * np.abs(D).max(), (e, i, a, b, step, fd, ref)


def test_cluster_sigma_equals_global_kubo_sum():
    """With a LIZ covering a finite cluster, the LSMS sum (Eq. lsms-conductivity-formula)
    equals the unrestricted multiple-scattering sum over all pairs (m, n) of the
    Kubo-Greenwood formula written with the full cluster inverse.  A non-symmetric
    t^{-1} and current matrices unrelated across energy pairs make tau^{mn} differ
    from (tau^{nm})^T and every (z_a, z_b) slot distinct, so a swapped row/column
    block or energy pair fails here."""
    w = wl.cluster(n_atoms=4, lmax=2, seed=5, spread=5.0, r_liz=100.0)
    K = 9
    rng = np.random.default_rng(8)
    L = liz.build_liz(w.pos, None, w.r_liz)
    tin = w.tinv[w.species].copy()
    tin = tin + 0.05 * (rng.normal(size=tin.shape) + 1j * rng.normal(size=tin.shape))
    J = rng.normal(size=(w.n_atoms, 4, 3, K, K)) + 1j * rng.normal(size=(w.n_atoms, 4, 3, K, K))
    col, row = kkr.tau_blocks(2, L, tin, w.z, return_rows=True)
    st = kubo.sigma_tilde(L, J, col, row, 1, w.volume)
    T = [np.linalg.inv(kkr.kkr_matrix(2, w.pos - w.pos[0], tin[:, e], w.z[e])) for e in range(2)]
    ref = np.zeros((4, 3, 3), dtype=np.complex128)
    for c, (a, b) in enumerate(kubo.COMBOS):
        for m in range(w.n_atoms):
            for n in range(w.n_atoms):
                t_mn = T[a][m * K:(m + 1) * K, n * K:(n + 1) * K]
                t_nm = T[b][n * K:(n + 1) * K, m * K:(m + 1) * K]
                for mu in range(3):
                    for nu in range(3):
                        # the energy pair of site m's current matrix is (z2, z1)
                        Jm = J[m, [0, 2, 1, 3][c], mu]
                        ref[c, mu, nu] += np.trace(Jm @ t_mn @ J[n, c, nu] @ t_nm)
    ref = -ref / (np.pi * w.volume)
    assert np.abs(st[0] - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(row[0] - np.transpose(col[0], (0, 2, 1))).max() > 1e-3 * np.abs(col[0]).max()
