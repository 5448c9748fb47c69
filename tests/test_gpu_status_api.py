"""Unit status, FP64 fallback and the Python API on the GPU.

* t^{-1} symmetry check: a non-symmetric block flags exactly the units whose LIZ
  holds a site of that species at that energy (LSMS_UNIT_TINV_ASYM).
* FP64 fallback of the mixed form, forced on the host through the options (a
  growth limit below any growth, or no refinement sweeps): the re-solved units
  run the FP64 form's kernels, so their tau blocks (and the gradient) equal the
  FP64 form's bit for bit; units beyond the fallback slots keep their flags.
* lsms_kubo_sigma_atoms: per-atom terms that sum to sigma~ and match the
  oracle's per-centre sums.
* SigmaFn / sigma_autograd (torch.autograd.Function) against the oracle's dense
  gradient, also after a second forward overwrote the first one's factors; the
  host-to-host conductivity() against the oracle; Problem raises on invalid
  units.
"""
import contextlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import grad as ograd
from oracle import kkr as okkr
from oracle import kubo as okubo
from oracle import liz as oliz
from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built, unit_rel_errors

TOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


@contextlib.contextmanager
def options(B, **kw):
    saved = {k: B.get_option(k) for k in kw}
    try:
        for k, v in kw.items():
            B.set_option(k, v)
        yield
    finally:
        for k, v in saved.items():
            B.set_option(k, v)


def _alloy32(seed=99):
    a = 7.65
    return wl.make_supercell(name="alloy32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                             r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002],
                             seed=seed)


@pytest.fixture(scope="module")
def alloy():
    w = _alloy32()
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    col, row = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, return_rows=True)
    J = okubo.dipole_current(w.lmax, w.r_ll)
    return w, L, col, row, J


def _run(B, w, precision, tinv=None, store=None, conj=False):
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    t = torch.as_tensor(w.tinv if tinv is None else tinv).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, precision, lu_store=store, conj_pairs=conj)
    torch.cuda.synchronize()
    return lz, sp, t, tau, st.cpu().numpy()


# ------------------------------------------------------------------ symmetry check
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonsymmetric_tinv_is_flagged(B, alloy, precision):
    w, L, _, _, _ = alloy
    tinv = w.tinv.copy()
    tinv[1, 0, 2, 5] += 1e-3          # species B, energy 0: no longer complex-symmetric
    _, _, _, _, st = _run(B, w, precision, tinv=tinv)
    off, sa = L["offsets"], L["site_atom"]
    has_b = np.array([np.any(w.species[sa[off[m]:off[m + 1]]] == 1) for m in range(w.n_atoms)])
    assert has_b.any()
    flagged = (st & B.UNIT_TINV_ASYM) != 0
    assert np.array_equal(flagged[0], has_b)
    assert not flagged[1].any()
    # a symmetric change of the same size is accepted
    tinv2 = w.tinv.copy()
    tinv2[1, 0, 2, 5] += 1e-3
    tinv2[1, 0, 5, 2] += 1e-3
    _, _, _, _, st2 = _run(B, w, precision, tinv=tinv2)
    assert not np.any(st2 & B.UNIT_INVALID)


def test_problem_raises_on_invalid_units(B, alloy):
    from paper_2311_12134_gb300.conductivity import Problem, UnitStatusError
    w, _, _, _, J = alloy
    tinv = w.tinv.copy()
    tinv[0, 1, 0, 1] += 1e-2
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, tinv, w.z, J, w.volume, precision="mixed")
    with pytest.raises(UnitStatusError):
        p.forward()
    p.check_status = False
    p.forward()                        # no check: returns, the status words still say why
    with pytest.raises(UnitStatusError):
        p.check()


# ------------------------------------------------------------------ FP64 fallback
@pytest.mark.parametrize("conj", [False, True])
@pytest.mark.parametrize("how", ["growth", "no_refinement"])
def test_forced_fallback_equals_fp64_form(B, alloy, how, conj):
    """Every mixed-form unit is flagged (growth limit below any growth, or no refinement sweep so
    every unit ends NOCONV) and re-solved in the FP64 form inside the call: tau equals the FP64
    form's bit for bit, the flags are cleared and LSMS_UNIT_FP64_FALLBACK is set."""
    w, L, col, _, _ = alloy
    nu = w.n_atoms * len(w.z)
    force = {"growth_limit": 1e-30} if how == "growth" else {"ir_max_sweeps": 0}
    with options(B, fallback_slots=nu, **force):
        _, _, _, tau_m, st_m = _run(B, w, "mixed", conj=conj)
    _, _, _, tau_d, st_d = _run(B, w, "fp64", conj=conj)
    assert not np.any(st_m & B.UNIT_INVALID), np.unique(st_m & 0xff)
    assert np.all(st_m & B.UNIT_FP64_FALLBACK)
    assert torch.equal(tau_m, tau_d)
    assert unit_rel_errors(tau_m.cpu().numpy(), col, L["offsets"]).max() < TOL["fp64"]


def test_fallback_slots_limit(B, alloy):
    """With fewer slots than flagged units, the first units in the library's order (atoms by LIZ
    size, energies within an atom) are re-solved and the rest keep LSMS_UNIT_NOCONV."""
    w, _, _, _, _ = alloy
    nu = w.n_atoms * len(w.z)
    with options(B, fallback_slots=5, ir_max_sweeps=0):
        _, _, _, tau_m, st_m = _run(B, w, "mixed")
    _, _, _, tau_d, _ = _run(B, w, "fp64")
    fb = (st_m & B.UNIT_FP64_FALLBACK) != 0
    nc = (st_m & B.UNIT_NOCONV) != 0
    assert fb.sum() == 5 and nc.sum() == nu - 5 and not np.any(fb & nc)
    # alloy32's LIZ are all the same size: atoms 0, 1, 2 in order, both energies per atom
    assert fb[:, :2].all() and fb[0, 2] and not fb[1, 2]
    off = B.build_liz(w.pos, w.lattice, w.r_liz).export()["offsets"]
    for e in range(2):
        for m in range(3):
            s = slice(off[m], off[m + 1])
            same = torch.equal(tau_m[e, s], tau_d[e, s])
            assert same == bool(fb[e, m])


def test_forced_fallback_in_the_adjoint(B, alloy):
    """No refinement sweeps in either call: forward and adjoint both fall back for every unit, so the
    gradient equals the FP64 form's bit for bit (stored factors are complex64; the fallback factors
    again in FP64)."""
    w, _, _, _, J = alloy
    nu = w.n_atoms * len(w.z)
    Jd = torch.as_tensor(J).cuda()
    wgt = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    wgt[0, 0, 0] = 1.0
    wgt[0, 1, 2] = 0.3 - 0.2j
    grads = {}
    for precision in ("mixed", "fp64"):
        lz = B.build_liz(w.pos, w.lattice, w.r_liz)
        store = torch.empty(B.lu_store_bytes(lz, w.lmax, 2, B._prec(precision)), dtype=torch.uint8, device="cuda")
        ctx = options(B, fallback_slots=nu, ir_max_sweeps=0) if precision == "mixed" else contextlib.nullcontext()
        with ctx:
            sp = torch.as_tensor(w.species).cuda()
            t = torch.as_tensor(w.tinv).cuda()
            tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, precision, lu_store=store)
            bst = torch.empty_like(st)
            g, gs = B.kubo_sigma_backward(lz, w.lmax, sp, t, w.z, Jd, tau, w.volume, wgt, precision, lu_store=store,
                                          unit_status=bst)
        torch.cuda.synchronize()
        b = bst.cpu().numpy()
        assert not np.any(b & B.UNIT_INVALID)
        if precision == "mixed":
            assert np.all(b & B.UNIT_FP64_FALLBACK)
        grads[precision] = (g, gs)
    assert torch.equal(grads["mixed"][0], grads["fp64"][0])
    assert torch.equal(grads["mixed"][1], grads["fp64"][1])


def test_default_runs_need_no_fallback(B, alloy):
    w, _, _, _, _ = alloy
    _, _, _, _, st = _run(B, w, "mixed")
    assert not np.any(st & 0xff), np.unique(st & 0xff)


# ------------------------------------------------------------------ per-atom sigma
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_atoms_sum_and_oracle(B, alloy, precision):
    w, L, col, row, J = alloy
    lz, sp, _, tau, st = _run(B, w, precision)
    Jd = torch.as_tensor(J).cuda()
    sig, st_tot, _ = B.kubo_sigma(lz, w.lmax, sp, Jd, tau, 1, w.volume, precision=precision)
    per = B.kubo_sigma_atoms(lz, w.lmax, sp, Jd, tau, 1, w.volume, precision=precision).cpu().numpy()
    tot = st_tot.cpu().numpy()
    assert per.shape == (1, 4, w.n_atoms, 3, 3)
    assert np.abs(per.sum(axis=2) - tot).max() < 1e-13 * np.abs(tot).max()
    Ja = J[w.species]
    scale = np.abs(tot).max()
    for m in (0, 7, 31):
        ref = okubo.sigma_tilde(L, Ja, col, row, 1, w.volume, atoms=[m])
        assert np.abs(per[:, :, m] - ref).max() < TOL[precision] * scale, m


# ------------------------------------------------------------------ autograd and host call
def _species_grad(w, L, J, wgt, tinv):
    D = ograd.dense_gradient(w.lmax, L, tinv[w.species], w.z, J[w.species], w.n_delta, w.volume, wgt)
    out = np.zeros_like(tinv)
    for s in range(tinv.shape[0]):
        out[s] = D[:, w.species == s].sum(axis=1)
    return ograd.torch_grad(out)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_autograd_matches_dense_oracle(B, alloy, precision):
    from paper_2311_12134_gb300.conductivity import Problem, sigma_autograd
    w, L, _, _, J = alloy
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume, precision=precision)
    t1 = torch.as_tensor(w.tinv).cuda().requires_grad_(True)
    t2 = (torch.as_tensor(w.tinv).cuda() * 1.02).requires_grad_(True)
    s1 = sigma_autograd(t1, p)
    s2 = sigma_autograd(t2, p)          # overwrites the first forward's tau and factors
    loss1 = s1[0, 0, 0].real + 0.5 * s1[0, 1, 1].real
    loss1.backward()                    # solved again for t1 (generation changed)
    s2[0, 0, 0].real.backward()         # the latest forward: reuses the stored factors
    wgt1 = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt1[0, 0, 0], wgt1[0, 1, 1] = 1.0, 0.5
    wgt2 = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt2[0, 0, 0] = 1.0
    for t, tin, wgt in ((t1, w.tinv, wgt1), (t2, w.tinv * 1.02, wgt2)):
        ref = _species_grad(w, L, J, wgt, tin)
        got = t.grad.cpu().numpy()
        assert np.linalg.norm(got - ref) < TOL[precision] * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_conductivity_host_call_matches_oracle(B, alloy, precision):
    from paper_2311_12134_gb300.conductivity import conductivity
    w, L, col, row, J = alloy
    sig, rho = conductivity(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume,
                            precision=precision)
    ref = okubo.consolidate(okubo.sigma_tilde(L, J[w.species], col, row, 1, w.volume))
    assert np.abs(sig - ref).max() < TOL[precision] * np.abs(ref).max()
    rref = okubo.resistivity(ref)
    assert np.abs(rho - rref).max() < 10 * TOL[precision] * np.abs(rref).max()


@pytest.mark.parametrize("cols,regs,streams,steps",
                         [(8, 1, 4, 1), (16, 0, 2, 1), (16, 1, 4, 0), (32, 0, 1, 1), (16, 1, 2, 2), (0, 0, 4, 2), (0, 0, 2, 3)])
def test_tuning_options_keep_results(B, alloy, cols, regs, streams, steps):
    """The autotuner's shapes (solve path, solve columns per CTA, register bound, concurrent parts)
    change the launch layout and, between the solve paths, the complex64 rounding of the corrections
    (FP32 pipes or 3xTF32 on the tensor cores): tau and the gradient match the default layout to the
    refinement's tolerance (corrections below 1e-10 of the solution)."""
    w, _, _, _, J = alloy
    Jd = torch.as_tensor(J).cuda()
    wgt = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    wgt[0, 0, 0] = 1.0
    out = []
    for opts in ({}, {"solve_cols": cols, "solve_regs": regs, "streams": streams, "solve_steps": steps}):
        with options(B, **opts) if opts else contextlib.nullcontext():
            lz = B.build_liz(w.pos, w.lattice, w.r_liz)
            sp = torch.as_tensor(w.species).cuda()
            t = torch.as_tensor(w.tinv).cuda()
            store = torch.empty(B.lu_store_bytes(lz, w.lmax, 2, B.LSMS_MIXED), dtype=torch.uint8, device="cuda")
            tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, "mixed", lu_store=store)
            g, _ = B.kubo_sigma_backward(lz, w.lmax, sp, t, w.z, Jd, tau, w.volume, wgt, "mixed", lu_store=store)
            torch.cuda.synchronize()
        assert not np.any(st.cpu().numpy() & 0xff)
        out.append((tau.cpu().numpy(), g.cpu().numpy()))
    (t0, g0), (t1, g1) = out
    assert np.abs(t1 - t0).max() <= 1e-10 * np.abs(t0).max()
    assert np.abs(g1 - g0).max() <= 1e-9 * np.abs(g0).max()
