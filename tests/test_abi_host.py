"""C ABI checks that need no GPU: the library loads, exports every declared
symbol, and its host-side parts (LIZ builder, Gaunt table, dipole current model)
agree with the oracle bit-for-bit on integers and to rounding on floats."""
import numpy as np
import pytest

from oracle import kubo as okubo
from oracle import liz as oliz
from oracle import sph
from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built, header_functions


@pytest.fixture(scope="module")
def L():
    return ensure_built()


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_version_and_errors(L):
    from paper_2311_12134_gb300 import binding as B
    assert B.version() >= 10000
    with pytest.raises(B.LsmsError):
        B.build_liz(np.zeros((0, 3)), None, 1.0)
    assert "atom" in B.lib().lsms_last_error().decode()
    with pytest.raises(B.LsmsError):
        B.build_liz(np.zeros((2, 3)), np.zeros((3, 3)), 1.0)   # singular lattice


def _compare_liz(lz, ref):
    ex = lz.export()
    assert np.array_equal(ex["offsets"], ref["offsets"])
    assert np.array_equal(ex["site_atom"], ref["site_atom"])
    assert np.array_equal(ex["image"], ref["image"])
    assert np.abs(ex["disp"] - ref["disp"]).max() < 1e-12


@pytest.mark.parametrize("maker", [wl.fcc_pure_32, lambda: wl.cluster(n_atoms=12, r_liz=7.0),
                                   lambda: wl.bcc_disordered_2000(n_cells=3)])
def test_liz_matches_oracle_bruteforce(L, maker):
    from paper_2311_12134_gb300 import binding as B
    w = maker()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    ref = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    _compare_liz(lz, ref)


def test_liz_small_cell_many_images(L):
    """A 1-atom cell with a radius of several lattice constants: every site is an image."""
    from paper_2311_12134_gb300 import binding as B
    a = 3.0
    pos = np.array([[0.3, 0.1, -0.2]])
    lat = np.array([[a, 0, 0], [0.5 * a, a, 0], [0, 0.3 * a, a]])
    lz = B.build_liz(pos, lat, 2.2 * a)
    ref = oliz.build_liz(pos, lat, 2.2 * a)
    _compare_liz(lz, ref)
    assert lz.total_sites > 30


def test_liz_unwrapped_positions(L):
    """Positions outside the cell keep their own image labels."""
    from paper_2311_12134_gb300 import binding as B
    w = wl.fcc_pure_32()
    pos = w.pos.copy()
    pos[3] += w.lattice[0] * 2 - w.lattice[2]
    pos[7] -= w.lattice[1]
    lz = B.build_liz(pos, w.lattice, w.r_liz)
    ref = oliz.build_liz(pos, w.lattice, w.r_liz)
    _compare_liz(lz, ref)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_liz_skewed_cells_and_radii_near_cell_sizes(L, seed):
    """Skewed random cells, radii from a fraction of a cell to about two cells
    (the builder skips neighbour cells by a distance bound, so radii close to
    the cell widths are where a wrong bound would drop sites)."""
    from paper_2311_12134_gb300 import binding as B
    rng = np.random.default_rng(seed)
    lat = np.diag(rng.uniform(5.0, 8.0, 3)) + rng.uniform(-1.5, 1.5, (3, 3)) * (1 - np.eye(3))
    pos = rng.random((9, 3)) @ lat + rng.normal(0, 0.05, (9, 3))
    h = 1.0 / np.linalg.norm(np.linalg.inv(lat), axis=0)  # plane spacings
    for r in sorted({0.4 * h.min(), 0.999 * h.min(), h.min(), 1.001 * h.min(), h.max(), 1.7 * h.max()}):
        lz = B.build_liz(pos, lat, r)
        _compare_liz(lz, oliz.build_liz(pos, lat, r))


def test_gaunt_table_matches_oracle(L):
    from paper_2311_12134_gb300 import binding as B
    for lmax in range(4):
        C = B.gaunt_table(lmax)
        ref = sph.gaunt_real(lmax, lmax, 2 * lmax)
        assert np.abs(C - ref).max() < 1e-14


def test_dipole_current_matches_oracle(L):
    from paper_2311_12134_gb300 import binding as B
    w = wl.fcc_alloy_256()
    for lmax in (1, 3):
        r = w.r_ll[:, :, :lmax + 1, :lmax + 1]
        J = B.dipole_current(lmax, r)
        ref = okubo.dipole_current(lmax, r)
        assert np.abs(J - ref).max() < 1e-15


def test_argument_errors_are_reported_before_any_device_work(L):
    """Bad arguments come back as LSMS_ERR_ARG with a message, checked on the host
    before the library touches a device (so this runs without a GPU)."""
    import ctypes
    from paper_2311_12134_gb300 import binding as B
    lib = B.lib()
    w = wl.fcc_pure_32()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    z = np.ascontiguousarray(w.z, dtype=np.complex128)
    zp = z.ctypes.data_as(ctypes.c_void_p)
    dummy = ctypes.c_void_p(16)  # never dereferenced: every call below fails its checks first
    sz_a, sz_b = ctypes.c_size_t(), ctypes.c_size_t()

    def tau(lmax=3, n_species=1, n_energy=2, precision=0, z_ptr=zp, tinv=dummy):
        return lib.lsms_tau_blocks(lz.handle, lmax, dummy, n_species, tinv, z_ptr, n_energy, precision, dummy,
                                   None, None, 0, None, 0, None)

    cases = {
        "lmax": tau(lmax=4),
        "species": tau(n_species=0),
        "n_energy": tau(n_energy=0),
        "too many energies": tau(n_energy=65),
        "precision": tau(precision=7),
        "tinv": tau(tinv=None),
        "conj odd": tau(n_energy=1, precision=B._prec("mixed", True)),
        "sizes lmax": lib.lsms_tau_workspace_bytes(lz.handle, 5, 2, 0, ctypes.byref(sz_a), ctypes.byref(sz_b)),
        "sizes conj odd": lib.lsms_tau_workspace_bytes(lz.handle, 3, 3, B._prec("fp64", True), ctypes.byref(sz_a),
                                                       ctypes.byref(sz_b)),
        "store precision": lib.lsms_lu_store_bytes(lz.handle, 3, 2, 9, ctypes.byref(sz_a)),
        "backward odd n_energy": lib.lsms_backward_workspace_bytes(lz.handle, 3, 3, 0, ctypes.byref(sz_a),
                                                                   ctypes.byref(sz_b)),
        "sigma volume": lib.lsms_kubo_sigma(lz.handle, 3, dummy, 1, dummy, 0, dummy, 1, -1.0, 0, None, dummy, None,
                                            None),
        "sigma precision": lib.lsms_kubo_sigma(lz.handle, 3, dummy, 1, dummy, 0, dummy, 1, 1.0, 5, None, dummy, None,
                                               None),
        "sigma stride": lib.lsms_kubo_sigma(lz.handle, 3, dummy, 1, dummy, -1, dummy, 1, 1.0, 0, None, dummy, None,
                                            None),
    }
    for what, rc in cases.items():
        assert rc == B.LSMS_ERR_ARG, (what, rc)
        assert lib.lsms_last_error().decode(), what
    # conjugate pairs need z[2d+1] = conj z[2d] exactly
    zb = z.copy()
    zb[1] += 1e-12
    assert tau(precision=B._prec("mixed", True), z_ptr=zb.ctypes.data_as(ctypes.c_void_p)) == B.LSMS_ERR_ARG
    assert "conjugate" in lib.lsms_last_error().decode()
    # the sizing calls succeed and are consistent: the store halves with conjugate pairs
    full, half = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.lsms_lu_store_bytes(lz.handle, 3, 2, 1, ctypes.byref(full)) == 0
    assert lib.lsms_lu_store_bytes(lz.handle, 3, 2, B._prec("mixed", True), ctypes.byref(half)) == 0
    assert full.value == 2 * half.value > 0


def test_options_roundtrip_and_range_checks(L):
    """lsms_set_option / lsms_get_option: defaults, round trip, and LSMS_ERR_ARG for unknown names and
    out-of-range values (host only)."""
    from paper_2311_12134_gb300 import binding as B
    saved = {k: B.get_option(k) for k in ("growth_limit", "fallback_slots", "ir_max_sweeps")}
    try:
        assert saved["growth_limit"] > 1.0 and saved["fallback_slots"] >= 1 and saved["ir_max_sweeps"] >= 1
        B.set_option("growth_limit", 123.5)
        assert B.get_option("growth_limit") == 123.5
        B.set_option("fallback_slots", 3)
        assert B.get_option("fallback_slots") == 3
        for name, bad in (("growth_limit", 0.0), ("growth_limit", float("inf")), ("fallback_slots", -1),
                          ("fallback_slots", 1.5), ("ir_max_sweeps", 65), ("streams", 5), ("solve_steps", 4), ("solve_regs", 3),
                          ("nvtx", 2), ("no_such_option", 1)):
            with pytest.raises(B.LsmsError) as ei:
                B.set_option(name, bad)
            assert ei.value.code == B.LSMS_ERR_ARG
        with pytest.raises(B.LsmsError):
            B.get_option("no_such_option")
    finally:
        for k, v in saved.items():
            B.set_option(k, v)


def test_workspace_sizes_with_store_and_fallback_slots(L):
    """With LSMS_WS_STORE the factors leave the workspace; the mixed form's sizes grow with the FP64
    fallback slots (each sized for the largest LIZ matrix) and the FP64 form's do not."""
    from paper_2311_12134_gb300 import binding as B
    w = wl.bcc_disordered_2000(n_cells=3)
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    nE = len(w.z)
    n_max = 16 * lz.max_sites
    saved = B.get_option("fallback_slots")
    try:
        for prec in (B.LSMS_FP64, B.LSMS_MIXED):
            mn, al = B.tau_workspace_bytes(lz, 3, nE, prec)
            mn_s, al_s = B.tau_workspace_bytes(lz, 3, nE, prec | B.LSMS_WS_STORE)
            store = B.lu_store_bytes(lz, 3, nE, prec)
            assert al - al_s == store and mn_s < mn
            bmn, bal = B.backward_workspace_bytes(lz, 3, nE, prec)
            bmn_s, bal_s = B.backward_workspace_bytes(lz, 3, nE, prec | B.LSMS_WS_STORE)
            assert bal - bal_s == store
        B.set_option("fallback_slots", 0)
        a0 = B.tau_workspace_bytes(lz, 3, nE, B.LSMS_MIXED)[1]
        f0 = B.tau_workspace_bytes(lz, 3, nE, B.LSMS_FP64)[1]
        B.set_option("fallback_slots", 4)
        a4 = B.tau_workspace_bytes(lz, 3, nE, B.LSMS_MIXED)[1]
        assert B.tau_workspace_bytes(lz, 3, nE, B.LSMS_FP64)[1] == f0
        assert a4 - a0 >= 4 * n_max * n_max * 16
    finally:
        B.set_option("fallback_slots", saved)


def test_sigma_atoms_argument_errors(L):
    import ctypes
    from paper_2311_12134_gb300 import binding as B
    lib = B.lib()
    w = wl.fcc_pure_32()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    dummy = ctypes.c_void_p(16)
    assert lib.lsms_kubo_sigma_atoms(lz.handle, 3, dummy, 1, dummy, 0, dummy, 1, -1.0, 0, dummy, None) == B.LSMS_ERR_ARG
    assert lib.lsms_kubo_sigma_atoms(lz.handle, 3, dummy, 1, dummy, 0, dummy, 1, 1.0, 0, None, None) == B.LSMS_ERR_ARG
    assert lib.lsms_kubo_sigma_atoms(lz.handle, 3, dummy, 1, dummy, 0, dummy, 0, 1.0, 0, dummy, None) == B.LSMS_ERR_ARG


def test_unit_stats_argument_errors(L):
    """lsms_unit_stats rejects NULL pointers, a negative count and a misaligned record before any launch."""
    import ctypes
    from paper_2311_12134_gb300 import binding as B
    lib = B.lib()
    words = ctypes.c_void_p(256)
    assert lib.lsms_unit_stats(None, 4, ctypes.c_void_p(512), None) == B.LSMS_ERR_ARG
    assert lib.lsms_unit_stats(words, 4, None, None) == B.LSMS_ERR_ARG
    assert lib.lsms_unit_stats(words, -1, ctypes.c_void_p(512), None) == B.LSMS_ERR_ARG
    assert lib.lsms_unit_stats(words, 4, ctypes.c_void_p(516), None) == B.LSMS_ERR_ARG
    assert "lsms_unit_stats" in lib.lsms_last_error().decode()
    for name in ("nvtx", "solve_steps"):
        v = B.get_option(name)
        assert v == 0
