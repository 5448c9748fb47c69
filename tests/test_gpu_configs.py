"""Full-size parity on the other workloads of the method, in the launch
configuration of the library (all units batched, chunked to the workspace):

* bcc2000: 2000-site bcc A/B alloy with vacancies and displacements (uneven LIZ
  sizes, n = 688..944), three broadenings delta, both forms; sampled tau blocks
  against the oracle, sigma per delta mixed vs FP64;
* fcc500: 500-atom fcc alloy, n = 880: the adjoint against central finite
  differences of the forward at seeded sites;
* the larger LIZ radii of the 16,000-site bcc recipe (89 and 137 sites, n = 1424
  and 2192) on smaller supercells of the same recipe; sampled tau blocks.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import kkr as okkr
from oracle import liz as oliz
from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built, rel_err_blocks

TOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


def _run(B, w, precision, ws_gib=16, J=None):
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    mn, al = B.tau_workspace_bytes(lz, w.lmax, len(w.z), B._prec(precision))
    ws = torch.empty(min(al, max(mn, ws_gib << 30)), dtype=torch.uint8, device="cuda")
    sp = torch.as_tensor(w.species).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, precision, workspace=ws)
    Jd = torch.as_tensor(B.dipole_current(w.lmax, w.r_ll) if J is None else J).cuda()
    sig, _, rho = B.kubo_sigma(lz, w.lmax, sp, Jd, tau, w.n_delta, w.volume, precision=precision)
    torch.cuda.synchronize()
    del ws
    return lz, tau, st.cpu().numpy(), sig.cpu().numpy()


def _check_sampled(w, lz, tau, atoms, tol):
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    assert np.array_equal(lz.export()["offsets"], L["offsets"])
    col = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms)
    off = L["offsets"]
    worst = 0.0
    for m in atoms:
        s = slice(off[m], off[m + 1])
        t = tau[:, s].cpu().numpy()
        for e in range(len(w.z)):
            worst = max(worst, rel_err_blocks(t[e][None], col[e, s][None]))
    assert worst < tol, worst
    return worst


def test_bcc2000_uneven_three_deltas(B):
    w = wl.bcc_disordered_2000()
    assert w.n_delta == 3 and w.n_atoms == 1980
    lz, tau_m, st_m, sig_m = _run(B, w, "mixed")
    sizes = lz.sizes
    assert sizes.min() < sizes.max()                       # uneven LIZ sizes
    assert np.all((st_m & 0xff) == 0), np.unique(st_m & 0xff, return_counts=True)
    assert ((st_m >> 8) & 0xff).max() <= 6
    assert ((st_m >> 16) & 0xff).max() <= 6
    atoms = [int(np.argmax(sizes)), int(np.argmin(sizes)), 1234]
    _check_sampled(w, lz, tau_m, atoms, TOL["mixed"])
    del tau_m
    torch.cuda.empty_cache()
    lz64, tau_d, st_d, sig_d = _run(B, w, "fp64")
    assert np.all((st_d & 0xff) == 0), np.unique(st_d & 0xff, return_counts=True)
    _check_sampled(w, lz64, tau_d, atoms[:2], TOL["fp64"])
    for d in range(3):                                     # per broadening
        err = np.abs(sig_m[d] - sig_d[d]).max() / np.abs(sig_d[d]).max()
        assert err < TOL["mixed"], (d, err)
        assert np.abs(sig_d[d].imag).max() < 1e-10 * np.abs(sig_d[d]).max()


@pytest.mark.parametrize("r_over_a,n_cells,precisions", [(2.2, 5, ("mixed", "fp64")), (2.5, 6, ("mixed",))])
def test_large_liz_radii(B, r_over_a, n_cells, precisions):
    w = wl.bcc_large_16000(r_over_a=r_over_a, n_cells=n_cells)
    for precision in precisions:
        lz, tau, st, _ = _run(B, w, precision)
        assert lz.max_sites == (89 if r_over_a == 2.2 else 137)
        assert np.all((st & 0xff) == 0)
        _check_sampled(w, lz, tau, [0, w.n_atoms - 1], TOL[precision])
        del tau
        torch.cuda.empty_cache()


def test_fcc500_adjoint_central_differences(B):
    """d Re sigma_xx / d t^{-1}_i on the 500-atom alloy at 10 seeded sites, against
    central differences (h = 1e-6 on Re and Im) of the mixed-form forward.  Every atom
    carries its own t^{-1} (n_species = N), so the per-species gradient is per site;
    (a, b) and (b, a) move together so t^{-1} stays symmetric."""
    base = wl.fcc_alloy_500()
    N = base.n_atoms
    Jsp = B.dipole_current(base.lmax, base.r_ll)
    J_atoms = torch.as_tensor(Jsp[base.species]).cuda()
    tinv = base.tinv[base.species].copy()
    sp = torch.arange(N, dtype=torch.int32, device="cuda")
    lz = B.build_liz(base.pos, base.lattice, base.r_liz)
    assert lz.max_sites == 55
    mn, al = B.tau_workspace_bytes(lz, base.lmax, 2, B.LSMS_MIXED)
    ws = torch.empty(al, dtype=torch.uint8, device="cuda")
    store = torch.empty(B.lu_store_bytes(lz, base.lmax, 2, B.LSMS_MIXED), dtype=torch.uint8, device="cuda")

    def sigma_xx(t):
        tau, _ = B.tau_blocks(lz, base.lmax, sp, torch.as_tensor(t).cuda(), base.z, "mixed", workspace=ws)
        s, _, _ = B.kubo_sigma(lz, base.lmax, sp, J_atoms, tau, 1, base.volume)
        return s.cpu().numpy()[0, 0, 0].real

    td = torch.as_tensor(tinv).cuda()
    tau, st = B.tau_blocks(lz, base.lmax, sp, td, base.z, "mixed", workspace=ws, lu_store=store)
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt[0, 0, 0] = 1.0
    _, g = B.kubo_sigma_backward(lz, base.lmax, sp, td, base.z, J_atoms, tau, base.volume,
                                 torch.as_tensor(wgt).cuda(), "mixed", lu_store=store)
    g = g.cpu().numpy()
    gmax = np.abs(g).max()
    rng = np.random.default_rng(2311 + 3)
    h = 1e-6
    for _ in range(10):
        i, e = int(rng.integers(N)), int(rng.integers(2))
        a = int(rng.integers(16))
        b = a if rng.random() < 0.5 else int(rng.integers(16))
        G = g[i, e, a, b] + (g[i, e, b, a] if a != b else 0)
        for step, part in ((h, "re"), (1j * h, "im")):
            tp, tm = tinv.copy(), tinv.copy()
            for (x, y) in {(a, b), (b, a)}:
                tp[i, e, x, y] += step
                tm[i, e, x, y] -= step
            fd = (sigma_xx(tp) - sigma_xx(tm)) / (2 * h)
            ref = G.real if part == "re" else G.imag
            assert abs(fd - ref) < 1e-5 * gmax, (i, e, a, b, part, fd, ref, gmax)


def test_liz_radius_sweep_and_extrapolation(B):
    """The LIZ-radius sweep of the 16,000-site bcc recipe (1.85a, 2.2a, 2.5a: 59, 89
    and 137 sites) on a 6x6x6-cell supercell of the same recipe, mixed form, then the
    lower/upper-bound extrapolations of Sec. IV on rho_xx(r)."""
    from paper_2311_12134_gb300 import extrapolate as ex
    radii, rho = [], []
    for roa in (1.85, 2.2, 2.5):
        w = wl.bcc_large_16000(r_over_a=roa, n_cells=6)
        lz, tau, st, sig = _run(B, w, "mixed")
        assert np.all((st & 0xff) == 0)
        assert lz.max_sites == {1.85: 59, 2.2: 89, 2.5: 137}[roa]
        radii.append(w.r_liz)
        rho.append(float(ex.resistivity_xx(sig[0])))
        del tau
        torch.cuda.empty_cache()
    c0, c1 = ex.fit_lower_bound(radii, rho)
    b0, b1 = ex.fit_upper_bound(radii, rho, two_alpha=0.15)
    assert np.all(np.isfinite([c0, c1, b0, b1]))
