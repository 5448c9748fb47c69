"""Full-size parity on the other workloads of the method, in the launch
configuration of the library (all units batched, chunked to the workspace):

* bcc2000: 2000-site bcc A/B alloy with vacancies and displacements (uneven LIZ
  sizes, n = 688..944), three broadenings delta, both forms; sampled tau blocks
  and, per delta, sigma summed over the sampled centres against the oracle;
  sigma per delta mixed vs FP64 over all atoms;
* fcc500: the 500-atom fcc alloy recipe (x = 0.3, LIZ 55 sites, n = 880): the
  adjoint against the oracle's dense gradient on a 32-atom cell of the recipe,
  and against central finite differences of the forward at 20 seeded sites of
  the full 500-atom alloy;
* bcc16000: the 16,000-site recipe at full size (LIZ 59, n = 944) with sampled
  tau blocks; the gradient at the 89-site LIZ (n = 1424) against finite
  differences; the LIZ-radius sweep (59, 89, 137 sites) at full size with the
  two extrapolations of Sec. IV;
* a spin-polarised alloy: the two channels through the GPU path, summed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import grad as ograd
from oracle import kkr as okkr
from oracle import kubo as okubo
from oracle import liz as oliz
from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built, rel_err_blocks, unit_rel_errors

TOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


def _run(B, w, precision, ws_gib=16, J=None, tinv=None, atoms_sigma=False):
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    mn, al = B.tau_workspace_bytes(lz, w.lmax, len(w.z), B._prec(precision))
    ws = torch.empty(min(al, max(mn, ws_gib << 30)), dtype=torch.uint8, device="cuda")
    sp = torch.as_tensor(w.species).cuda()
    t = torch.as_tensor(w.tinv if tinv is None else tinv).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, precision, workspace=ws)
    Jd = torch.as_tensor(B.dipole_current(w.lmax, w.r_ll) if J is None else J).cuda()
    sig, _, rho = B.kubo_sigma(lz, w.lmax, sp, Jd, tau, w.n_delta, w.volume, precision=precision)
    per = None
    if atoms_sigma:
        per = B.kubo_sigma_atoms(lz, w.lmax, sp, Jd, tau, w.n_delta, w.volume, precision=precision).cpu().numpy()
    torch.cuda.synchronize()
    del ws
    return lz, tau, st.cpu().numpy(), sig.cpu().numpy(), per


def _check_sampled(w, lz, tau, atoms, tol, rows=False):
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    assert np.array_equal(lz.export()["offsets"], L["offsets"])
    col, row = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms, return_rows=True)
    off = L["offsets"]
    worst = 0.0
    for m in atoms:
        s = slice(off[m], off[m + 1])
        t = tau[:, s].cpu().numpy()
        for e in range(len(w.z)):
            worst = max(worst, rel_err_blocks(t[e][None], col[e, s][None]))
    assert worst < tol, worst
    return (worst, L, col, row) if rows else worst


def _consolidate(st):
    return 0.25 * (st[:, 0] - st[:, 1] - st[:, 2] + st[:, 3])


def test_bcc2000_uneven_three_deltas(B):
    """Config bcc2000: tau of sampled atoms and, per delta, sigma summed over those centres against the
    oracle, in both forms; sigma over all atoms, mixed vs FP64, per delta."""
    w = wl.bcc_disordered_2000()
    assert w.n_delta == 3 and w.n_atoms == 1980
    Jsp = okubo.dipole_current(w.lmax, w.r_ll)
    lz, tau_m, st_m, sig_m, per_m = _run(B, w, "mixed", atoms_sigma=True)
    sizes = lz.sizes
    assert sizes.min() < sizes.max()                       # uneven LIZ sizes
    assert np.all((st_m & 0xff) == 0), np.unique(st_m & 0xff, return_counts=True)
    assert ((st_m >> 8) & 0xff).max() <= 6
    assert ((st_m >> 16) & 0xff).max() <= 6
    atoms = [int(np.argmax(sizes)), int(np.argmin(sizes)), 1234]
    _, L, col, row = _check_sampled(w, lz, tau_m, atoms, TOL["mixed"], rows=True)
    ref = _consolidate(okubo.sigma_tilde(L, Jsp[w.species], col, row, w.n_delta, w.volume, atoms=atoms))
    got_m = _consolidate(per_m[:, :, atoms].sum(axis=2))
    for d in range(3):
        assert np.abs(got_m[d] - ref[d]).max() < TOL["mixed"] * np.abs(ref[d]).max(), d
    del tau_m
    torch.cuda.empty_cache()
    lz64, tau_d, st_d, sig_d, per_d = _run(B, w, "fp64", atoms_sigma=True)
    assert np.all((st_d & 0xff) == 0), np.unique(st_d & 0xff, return_counts=True)
    _check_sampled(w, lz64, tau_d, atoms[:2], TOL["fp64"])
    got_d = _consolidate(per_d[:, :, atoms].sum(axis=2))
    for d in range(3):                                     # per broadening
        assert np.abs(got_d[d] - ref[d]).max() < TOL["fp64"] * np.abs(ref[d]).max(), d
        err = np.abs(sig_m[d] - sig_d[d]).max() / np.abs(sig_d[d]).max()
        assert err < TOL["mixed"], (d, err)
        assert np.abs(sig_d[d].imag).max() < 1e-10 * np.abs(sig_d[d]).max()


@pytest.mark.parametrize("r_over_a,n_cells,precisions", [(2.2, 5, ("mixed", "fp64")), (2.5, 6, ("mixed",))])
def test_large_liz_radii(B, r_over_a, n_cells, precisions):
    w = wl.bcc_large_16000(r_over_a=r_over_a, n_cells=n_cells)
    for precision in precisions:
        lz, tau, st, _, _ = _run(B, w, precision)
        assert lz.max_sites == (89 if r_over_a == 2.2 else 137)
        assert np.all((st & 0xff) == 0)
        _check_sampled(w, lz, tau, [0, w.n_atoms - 1], TOL[precision])
        del tau
        torch.cuda.empty_cache()


def _check_sampled_subset(w, lz, tau, atoms, tol):
    """As _check_sampled for structures too large for the oracle's all-atom LIZ: the oracle builds the
    LIZ of the sampled centres only and is compared site by site with the library's."""
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz, atoms=atoms)
    ex = lz.export()
    off = ex["offsets"]
    col = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z)
    worst = 0.0
    for i, m in enumerate(atoms):
        s = slice(off[m], off[m + 1])
        so = slice(L["offsets"][i], L["offsets"][i + 1])
        assert np.array_equal(ex["site_atom"][s], L["site_atom"][so])
        assert np.abs(ex["disp"][s] - L["disp"][so]).max() < 1e-12
        t = tau[:, s].cpu().numpy()
        for e in range(len(w.z)):
            worst = max(worst, rel_err_blocks(t[e][None], col[e, so][None]))
    assert worst < tol, worst
    return worst


def test_bcc16000_full_size_forward(B):
    """The 16,000-site recipe at full size (15,920 atoms after vacancies, LIZ 59 sites, n = 944,
    31,840 units), mixed form, chunked to a 16 GiB workspace: clean status, sampled tau against the
    oracle, finite sigma with positive diagonal."""
    w = wl.bcc_large_16000(r_over_a=1.85)
    assert w.n_atoms == 15920
    lz, tau, st, sig, _ = _run(B, w, "mixed")
    assert lz.max_sites == 59
    assert np.all((st & 0xff) == 0), np.unique(st & 0xff, return_counts=True)
    _check_sampled_subset(w, lz, tau, [0, 7777, w.n_atoms - 1], TOL["mixed"])
    assert np.all(np.isfinite(sig))
    d = np.real(np.diag(sig[0]))
    assert d.min() > 0


def _per_atom_problem(B, w):
    """Every atom its own species (n_species = N), so the per-species gradient is per site."""
    Jsp = B.dipole_current(w.lmax, w.r_ll)
    return torch.as_tensor(Jsp[w.species]).cuda(), w.tinv[w.species].copy(), \
        torch.arange(w.n_atoms, dtype=torch.int32, device="cuda")


# Relative accuracy of the mixed form's sigma (measured against the FP64 form: ~2e-12 on every
# workload); a central difference at step h inherits |sigma| * this / h of absolute error.
SIGMA_MIXED_REL = 1e-11


def _fd_check(B, w, n_sites, seed, ws_gib=16):
    """d Re sigma_xx / d t^{-1}_i at seeded sites against central differences (h = 1e-6 on Re and
    Im) of the mixed-form forward; (a, b) and (b, a) move together so t^{-1} stays symmetric.
    Tolerance: 1e-5 of the largest gradient entry plus the difference quotient's own rounding
    error, SIGMA_MIXED_REL |sigma_xx| / h."""
    N = w.n_atoms
    J_atoms, tinv, sp = _per_atom_problem(B, w)
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    mn, al = B.tau_workspace_bytes(lz, w.lmax, 2, B.LSMS_MIXED)
    ws = torch.empty(min(al, max(mn, ws_gib << 30)), dtype=torch.uint8, device="cuda")
    store = torch.empty(B.lu_store_bytes(lz, w.lmax, 2, B.LSMS_MIXED), dtype=torch.uint8, device="cuda")

    def sigma_xx(t):
        tau, _ = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(t).cuda(), w.z, "mixed", workspace=ws)
        s, _, _ = B.kubo_sigma(lz, w.lmax, sp, J_atoms, tau, 1, w.volume)
        return s.cpu().numpy()[0, 0, 0].real

    td = torch.as_tensor(tinv).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, td, w.z, "mixed", workspace=ws, lu_store=store)
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt[0, 0, 0] = 1.0
    _, g = B.kubo_sigma_backward(lz, w.lmax, sp, td, w.z, J_atoms, tau, w.volume,
                                 torch.as_tensor(wgt).cuda(), "mixed", lu_store=store)
    g = g.cpu().numpy()
    gmax = np.abs(g).max()
    rng = np.random.default_rng(seed)
    h = 1e-6
    tol = 1e-5 * gmax + SIGMA_MIXED_REL * abs(sigma_xx(tinv)) / h
    for _ in range(n_sites):
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
            assert abs(fd - ref) < tol, (i, e, a, b, part, fd, ref, gmax, tol)
    return lz


def test_fcc500_adjoint_central_differences(B):
    """The 500-atom alloy (LIZ 55, n = 880): the adjoint at 20 seeded sites against central
    differences of the forward."""
    w = wl.fcc_alloy_500()
    lz = _fd_check(B, w, 20, 2311 + 3)
    assert lz.max_sites == 55


@pytest.mark.parametrize("precision,store", [("mixed", True), ("mixed", False), ("fp64", True)])
def test_fcc500_recipe_dense_gradient_32_atoms(B, precision, store):
    """The fcc500 recipe (x = 0.3, a = 7.65, LIZ 1.5a = 55 sites with periodic images, n = 880) on a
    32-atom cell: the adjoint's per-site gradient against the oracle's explicit-inverse gradient."""
    a = 7.65
    w = wl.make_supercell(name="fcc32_AB30_liz55", kind="fcc", n_cells=2, a=a, counts=[22, 10], r_liz=1.50 * a,
                          phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.60, deltas=[0.002], seed=2311 + 3)
    Jsp = okubo.dipole_current(w.lmax, w.r_ll)
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt[0, 0, 0] = 1.0
    wgt[0, 2, 1] = 0.25 + 0.5j
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    ref = ograd.torch_grad(ograd.dense_gradient(w.lmax, L, w.tinv[w.species], w.z, Jsp[w.species], 1, w.volume,
                                                wgt))
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    assert lz.max_sites == 55
    sp = torch.as_tensor(w.species).cuda()
    t = torch.as_tensor(w.tinv).cuda()
    st_buf = None
    if store:
        st_buf = torch.empty(B.lu_store_bytes(lz, w.lmax, 2, B._prec(precision)), dtype=torch.uint8, device="cuda")
    tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, precision, lu_store=st_buf)
    bst = torch.empty_like(st)
    g, _ = B.kubo_sigma_backward(lz, w.lmax, sp, t, w.z, torch.as_tensor(Jsp).cuda(), tau, w.volume,
                                 torch.as_tensor(wgt).cuda(), precision, lu_store=st_buf, unit_status=bst)
    torch.cuda.synchronize()
    assert not np.any(st.cpu().numpy() & 0xff) and not np.any(bst.cpu().numpy() & 0xff)
    g = g.cpu().numpy()
    for e in range(2):
        assert np.linalg.norm(g[e] - ref[e]) < TOL[precision] * np.linalg.norm(ref[e]), e


def test_bcc16000_recipe_gradient_at_89_site_liz(B):
    """The 16,000-site recipe at LIZ 2.2a (89 sites, n = 1424) on a 5x5x5-cell supercell: the
    adjoint against central differences at 6 seeded sites."""
    w = wl.bcc_large_16000(r_over_a=2.2, n_cells=5)
    lz = _fd_check(B, w, 6, 2311 + 4)
    assert lz.max_sites == 89


def test_liz_radius_sweep_and_extrapolation(B):
    """The LIZ-radius sweep of the 16,000-site bcc recipe at full size (1.85a, 2.2a, 2.5a: 59, 89 and
    137 sites, n up to 2192), mixed form, then the lower- and upper-bound extrapolations of Sec. IV on
    rho_xx(r) with r in angstrom (the upper bound's 2 alpha_max = 0.15 is in inverse angstrom).  The
    synthetic alloy's rho(r) need not be monotone over three radii (it is not here), so no ordering
    of the two extrapolations is implied; each fit is checked as the least-squares solution of its
    linearised form, and the two extrapolated values must agree with the samples' scale."""
    from paper_2311_12134_gb300 import extrapolate as ex
    radii, rho = [], []
    for roa in (1.85, 2.2, 2.5):
        w = wl.bcc_large_16000(r_over_a=roa)
        lz, tau, st, sig, _ = _run(B, w, "mixed", ws_gib=24)
        assert np.all((st & 0xff) == 0)
        assert lz.max_sites == {1.85: 59, 2.2: 89, 2.5: 137}[roa]
        radii.append(w.r_liz * ex.BOHR_IN_ANGSTROM)
        rho.append(float(ex.resistivity_xx(sig[0])))
        del tau
        torch.cuda.empty_cache()
    c0, c1 = ex.fit_lower_bound(radii, rho)
    b0, b1 = ex.fit_upper_bound(radii, rho, two_alpha=0.15)
    r, y = np.asarray(radii), np.asarray(rho)
    assert np.all(np.isfinite([c0, c1, b0, b1])) and y.min() > 0
    # normal equations of the two linearised fits: residuals orthogonal to the design columns
    res_lo = c0 / r + c1 - y
    assert abs(res_lo @ (1 / r)) < 1e-9 * np.abs(y).sum() / r.min() and abs(res_lo.sum()) < 1e-9 * np.abs(y).sum()
    x = np.exp(-0.15 * r)
    res_up = (1 + b1 * x) / b0 - 1 / y
    assert abs(res_up @ x) < 1e-9 * np.abs(1 / y).sum() and abs(res_up.sum()) < 1e-9 * np.abs(1 / y).sum()
    for v in (c1, b0):
        assert 0.5 * y.min() < v < 2 * y.max(), (c1, b0, rho)


def test_spin_polarised_sum_through_the_gpu(B):
    """Collinear spin polarisation (Sec. IV, Fe-Si): the two spin channels are separate runs of the
    path with their own t^{-1}; sigma = sigma_up + sigma_down, compared with the oracle's two
    channels summed, and rho_xx from the sum."""
    from paper_2311_12134_gb300 import extrapolate as ex
    a = 7.65
    base = dict(name="spin32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1, r_liz=0.85 * a,
                e_fermi=0.6, deltas=[0.002], seed=321)
    up = wl.make_supercell(phases=[wl.PHASE_A, wl.PHASE_B], **base)
    dn = wl.make_supercell(phases=[(0.30, 0.15, 0.10, 0.004), (0.45, 0.25, 0.60, 0.015)], **base)
    J = okubo.dipole_current(up.lmax, up.r_ll)
    sig = {}
    ref = {}
    L = oliz.build_liz(up.pos, up.lattice, up.r_liz)
    for name, w in (("up", up), ("down", dn)):
        _, _, st, s, _ = _run(B, w, "mixed", J=J)
        assert not np.any(st & 0xff)
        sig[name] = s
        col, row = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, return_rows=True)
        ref[name] = okubo.consolidate(okubo.sigma_tilde(L, J[w.species], col, row, 1, w.volume))
    tot = ex.spin_sum(sig["up"], sig["down"])
    rtot = ref["up"] + ref["down"]
    assert np.abs(tot - rtot).max() < TOL["mixed"] * np.abs(rtot).max()
    assert abs(ex.resistivity_xx(tot[0]) - ex.resistivity_xx(rtot[0])) < 1e-7 * abs(ex.resistivity_xx(rtot[0]))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_liz_of_about_260_sites_n_4000(B, precision):
    """Toward the paper's ~1000-atom LIZ (Sec. III, Sec. V): a bcc cell of 16 atoms (12/4 A/B,
    displacements 0.05 a) with LIZ radius 3.1 a holds 256..264 sites through periodic images, n up to 4224:
    the batched LU (tall panels in global memory, chunked workspace) against the oracle on one atom."""
    a = 5.42
    w = wl.make_supercell(name="bcc16_liz3a", kind="bcc", n_cells=2, a=a, counts=[12, 4], sigma_disp=0.05 * a,
                          r_liz=3.1 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.62, deltas=[0.002],
                          seed=2311 + 4)
    lz, tau, st, sig, _ = _run(B, w, precision, ws_gib=8)
    assert lz.max_sites >= 256 and 16 * lz.max_sites >= 4096
    assert np.all((st & 0xff) == 0), np.unique(st & 0xff)
    _check_sampled_subset(w, lz, tau, [0], TOL[precision])
    assert np.all(np.isfinite(sig))


def test_liz_of_965_sites_n_15440_mixed_against_fp64(B):
    """The paper's ~1000-atom LIZ (Sec. III, Sec. V): a 2-atom bcc cell with LIZ radius 4.9 a holds
    965 sites through periodic images, n = 15,440.  The batched path runs unchanged (global-memory
    panels, tensor-core trailing update over 121 row tiles per matrix, row-order pass, chain
    solves): the mixed form's tau matches the FP64 form's (the FP64 form is pinned to the oracle
    at the smaller sizes above) to the mixed-form tolerance, with clean status words."""
    a = 5.42
    w = wl.make_supercell(name="bcc2_liz965", kind="bcc", n_cells=1, a=a, counts=[1, 1], sigma_disp=0.0,
                          r_liz=4.9 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.62, deltas=[0.002], seed=7)
    out = {}
    for precision in ("mixed", "fp64"):
        lz = B.build_liz(w.pos, w.lattice, w.r_liz)
        assert lz.min_sites == lz.max_sites == 965
        tau, st = B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(),
                               w.z, precision)
        torch.cuda.synchronize()
        assert np.all((st.cpu().numpy() & 0xff) == 0), (precision, np.unique(st.cpu().numpy() & 0xff))
        out[precision] = tau.cpu().numpy()
        del tau
        torch.cuda.empty_cache()
    off = lz.export()["offsets"]
    err = unit_rel_errors(out["mixed"], out["fp64"], off)
    assert err.max() < TOL["mixed"], err.max()
