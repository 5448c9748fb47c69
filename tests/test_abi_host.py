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
