"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same
seeded inputs.  Tolerances (norm-wise, as defined for the tau blocks, sigma and
the gradient): 1e-10 for the FP64 form; 1e-8 for the mixed form (complex64 LU
with FP64 refinement, which in practice reaches ~1e-12)."""
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _B():
    from paper_2311_12134_gb300 import binding
    return binding


def gpu_tau(w, precision, workspace_bytes=None, lu_store=False, liz=None):
    B = _B()
    lz = liz or B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    tinv = torch.as_tensor(w.tinv).cuda()
    ws = None
    if workspace_bytes is not None:
        ws = torch.empty(workspace_bytes, dtype=torch.uint8, device="cuda")
    store = None
    if lu_store:
        store = torch.empty(B.lu_store_bytes(lz, w.lmax, len(w.z), B._prec(precision)), dtype=torch.uint8,
                            device="cuda")
    tau, st = B.tau_blocks(lz, w.lmax, sp, tinv, w.z, precision, workspace=ws, lu_store=store)
    torch.cuda.synchronize()
    return lz, tau, st, store


def oracle_tau(w, atoms=None):
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    col, row = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms, return_rows=True)
    return L, col, row


@pytest.fixture(scope="module")
def fcc32():
    w = wl.fcc_pure_32()
    L, col, row = oracle_tau(w)
    J = okubo.dipole_current(w.lmax, w.r_ll)
    st = okubo.sigma_tilde(L, J[w.species], col, row, w.n_delta, w.volume)
    return w, L, col, st


def _alloy32(seed=99, lmax=3):
    a = 7.65
    return wl.make_supercell(name="alloy32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                             r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002],
                             lmax=lmax, seed=seed)


@pytest.fixture(scope="module")
def alloy32():
    w = _alloy32()
    L, col, row = oracle_tau(w)
    J = okubo.dipole_current(w.lmax, w.r_ll)
    st = okubo.sigma_tilde(L, J[w.species], col, row, w.n_delta, w.volume)
    return w, L, col, st, J


# ------------------------------------------------------------------ tau
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_fcc32(fcc32, precision):
    w, L, col, _ = fcc32
    lz, tau, st, _ = gpu_tau(w, precision)
    assert int((st & 0xff).abs().sum()) == 0
    err = unit_rel_errors(tau.cpu().numpy(), col, L["offsets"])
    assert err.max() < TOL[precision], err.max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_alloy32_elementwise(alloy32, precision):
    w, L, col, _, _ = alloy32
    lz, tau, st, _ = gpu_tau(w, precision)
    t = tau.cpu().numpy()
    assert int((st & 0xff).abs().sum()) == 0
    scale = np.abs(col).max()
    assert np.abs(t - col).max() < TOL[precision] * scale
    assert unit_rel_errors(t, col, L["offsets"]).max() < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_uneven_bcc_sampled(precision):
    """Displaced bcc alloy with a vacancy: uneven LIZ sizes, several tiles and a ragged
    tail per matrix; three delta values.  Sampled atoms against the oracle."""
    w = wl.bcc_disordered_2000(n_cells=3)
    lz, tau, st, _ = gpu_tau(w, precision)
    sizes = np.diff(lz.export()["offsets"])
    assert sizes.min() < sizes.max()
    atoms = [int(np.argmax(sizes)), int(np.argmin(sizes)), 7]
    L, col, _ = oracle_tau(w, atoms=atoms)
    t = tau.cpu().numpy()
    assert int((st & 0xff).abs().sum()) == 0
    for m in atoms:
        s = slice(L["offsets"][m], L["offsets"][m + 1])
        for e in range(len(w.z)):
            assert rel_err_blocks(t[e, s][None], col[e, s][None]) < TOL[precision]


@pytest.mark.parametrize("lmax", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_cluster_all_lmax(lmax, precision):
    w = wl.cluster(n_atoms=9, lmax=lmax, r_liz=8.5, seed=4)
    lz, tau, st, _ = gpu_tau(w, precision)
    L, col, _ = oracle_tau(w)
    assert np.array_equal(lz.export()["offsets"], L["offsets"])
    assert unit_rel_errors(tau.cpu().numpy(), col, L["offsets"]).max() < TOL[precision]


def test_single_site_liz_is_t():
    """r_liz below the nearest-neighbour distance: S = 1, n = 16 < panel width, tau = t."""
    w = wl.fcc_pure_32()
    w.r_liz = 1.0
    lz, tau, st, _ = gpu_tau(w, "fp64")
    t = np.linalg.inv(w.tinv[0])
    got = tau.cpu().numpy()
    for e in range(2):
        assert np.abs(got[e] - t[e][None]).max() < 1e-13 * np.abs(t[e]).max()


def test_chunking_is_invisible(alloy32):
    """A workspace that holds only a few units at a time gives identical results."""
    w = alloy32[0]
    B = _B()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    mn, al = B.tau_workspace_bytes(lz, w.lmax, len(w.z), B.LSMS_MIXED)
    _, t_all, _, _ = gpu_tau(w, "mixed", workspace_bytes=al, liz=lz)
    _, t_few, _, _ = gpu_tau(w, "mixed", workspace_bytes=mn + (al - mn) // 7, liz=lz)
    assert torch.equal(t_all, t_few)


def test_misaligned_buffers_are_rejected(alloy32):
    """Caller-provided workspace and lu_store must be 256-byte aligned (the
    kernels read them with 16-byte vector loads); otherwise LSMS_ERR_ARG."""
    w = alloy32[0]
    B = _B()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    mn, _ = B.tau_workspace_bytes(lz, w.lmax, len(w.z), B.LSMS_MIXED)
    ws = torch.empty(mn + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.LsmsError) as e:
        B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(), w.z, "mixed",
                     workspace=ws[16:16 + mn])
    assert e.value.code == B.LSMS_ERR_ARG and "aligned" in str(e.value)
    need = B.lu_store_bytes(lz, w.lmax, len(w.z), B.LSMS_MIXED)
    store = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.LsmsError) as e:
        B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(), w.z, "mixed",
                     lu_store=store[16:16 + need])
    assert e.value.code == B.LSMS_ERR_ARG and "aligned" in str(e.value)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_stream_split_is_invisible(precision):
    """Each chunk runs as two halves on two streams; with the kernel timers on it
    runs on one stream.  Both give bit-identical tau, sigma and gradient."""
    from paper_2311_12134_gb300 import binding as B
    from paper_2311_12134_gb300.conductivity import Problem
    w = _alloy32(seed=23)
    J = B.dipole_current(w.lmax, w.r_ll)
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume, precision=precision)
    gs = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    gs[0, 1, 1] = 1.0

    def step():
        p.forward()
        g = [t.clone() for t in p.backward(gs)]
        torch.cuda.synchronize()
        return p.tau.clone(), p.sigma_out.clone(), g

    tau2, sig2, g2 = step()
    B.kernel_timer_start()
    try:
        tau1, sig1, g1 = step()
    finally:
        B.kernel_timer_stop()
    assert torch.equal(tau1, tau2)
    assert torch.equal(sig1, sig2)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])


def test_nonfinite_input_flags_units():
    w = _alloy32()
    w.tinv = w.tinv.copy()
    w.tinv[1, 0, 3, 3] = np.nan
    lz, tau, st, _ = gpu_tau(w, "fp64")
    st = st.cpu().numpy()
    b_atoms = np.nonzero(w.species == 1)[0]
    assert np.all(st[0, b_atoms] & 4)       # an atom of species 1 is its own centre
    assert np.all(st[1] == 0)                # the other energy is untouched


# ------------------------------------------------------------------ sigma
def gpu_sigma(w, precision, J=None):
    B = _B()
    lz, tau, st, _ = gpu_tau(w, precision)
    Jh = B.dipole_current(w.lmax, w.r_ll) if J is None else J
    sp = torch.as_tensor(w.species).cuda()
    sig, sigt, rho = B.kubo_sigma(lz, w.lmax, sp, torch.as_tensor(Jh).cuda(), tau, w.n_delta, w.volume,
                                  precision=precision)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), sigt.cpu().numpy(), rho.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_fcc32(fcc32, precision):
    w, L, col, st = fcc32
    sig, sigt, rho = gpu_sigma(w, precision)
    ref = okubo.consolidate(st)
    assert np.abs(sigt - st).max() < TOL[precision] * np.abs(st).max()
    assert np.abs(sig - ref).max() < TOL[precision] * np.abs(ref).max()
    assert np.abs(rho - okubo.resistivity(ref)).max() < TOL[precision] * np.abs(okubo.resistivity(ref)).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sigma_alloy32(alloy32, precision):
    w, L, col, st, J = alloy32
    sig, sigt, rho = gpu_sigma(w, precision)
    ref = okubo.consolidate(st)
    assert np.abs(sigt - st).max() < TOL[precision] * np.abs(st).max()
    assert np.abs(sig - ref).max() < TOL[precision] * np.abs(ref).max()


def test_sigma_general_current_matrices(alloy32):
    """Random dense J (every energy pair distinct) exercises the J(z2,z1)/J(z1,z2) slots."""
    w, L, col, _, _ = alloy32
    rng = np.random.default_rng(12)
    J = rng.normal(size=(2, 4, 3, 16, 16)) + 1j * rng.normal(size=(2, 4, 3, 16, 16))
    col2, row2 = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, return_rows=True)
    ref = okubo.sigma_tilde(L, J[w.species], col2, row2, 1, w.volume)
    _, sigt, _ = gpu_sigma(w, "fp64", J=J)
    assert np.abs(sigt - ref).max() < 1e-10 * np.abs(ref).max()


def test_sigma_lmax0_is_zero():
    w = wl.make_supercell(name="t", kind="fcc", n_cells=2, a=7.72, counts=[32], r_liz=0.85 * 7.72,
                          phases=[wl.PHASE_PURE], e_fermi=0.55, deltas=[0.002], lmax=0, seed=1)
    sig, sigt, _ = gpu_sigma(w, "fp64")
    assert np.all(sigt == 0)


# ------------------------------------------------------------------ gradient
def _grad_case(precision, lu_store):
    w = _alloy32(seed=5)
    B = _B()
    lz, tau, st, store = gpu_tau(w, precision, lu_store=lu_store)
    Jh = B.dipole_current(w.lmax, w.r_ll)
    sp = torch.as_tensor(w.species).cuda()
    rng = np.random.default_rng(3)
    wgt = rng.normal(size=(1, 3, 3)) + 1j * rng.normal(size=(1, 3, 3))
    g, gs = B.kubo_sigma_backward(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, torch.as_tensor(Jh).cuda(),
                                  tau, w.volume, torch.as_tensor(wgt).cuda(), precision, lu_store=store)
    torch.cuda.synchronize()
    return w, Jh, wgt, g.cpu().numpy(), gs.cpu().numpy()


@pytest.fixture(scope="module")
def dense_grad_alloy():
    w = _alloy32(seed=5)
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    J = okubo.dipole_current(w.lmax, w.r_ll)
    rng = np.random.default_rng(3)
    wgt = rng.normal(size=(1, 3, 3)) + 1j * rng.normal(size=(1, 3, 3))
    D = ograd.dense_gradient(w.lmax, L, w.tinv[w.species], w.z, J[w.species], 1, w.volume, wgt)
    return ograd.torch_grad(D)


@pytest.mark.parametrize("precision,lu_store", [("fp64", False), ("fp64", True), ("mixed", False), ("mixed", True)])
def test_gradient_matches_dense_oracle(dense_grad_alloy, precision, lu_store):
    w, Jh, wgt, g, gs = _grad_case(precision, lu_store)
    ref = dense_grad_alloy
    for e in range(2):
        assert rel_err_blocks(g[e][None], ref[e][None]) < TOL[precision]
    for s in range(2):
        ref_s = ref[:, w.species == s].sum(axis=1)
        assert np.abs(gs[s] - ref_s).max() < TOL[precision] * np.abs(ref_s).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("weights", ["xx", "column_z", "dense"])
def test_gradient_general_current_and_sparse_weights(precision, weights):
    """The adjoint's right-hand sides run over the nonzero entries of J and Abar and skip a zero
    Abar^nu: random dense J (no zero entries) and weights with zero columns nu (only d Re sigma_xx;
    only the nu = z column) against the oracle's dense gradient."""
    w = _alloy32(seed=5)
    B = _B()
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    rng = np.random.default_rng(17)
    J = rng.normal(size=(2, 4, 3, 16, 16)) + 1j * rng.normal(size=(2, 4, 3, 16, 16))
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    if weights == "xx":
        wgt[0, 0, 0] = 1.0
    elif weights == "column_z":
        wgt[0, :, 2] = rng.normal(size=3) + 1j * rng.normal(size=3)
    else:
        wgt[0] = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
    ref = ograd.torch_grad(ograd.dense_gradient(w.lmax, L, w.tinv[w.species], w.z, J[w.species], 1, w.volume, wgt))
    lz, tau, st, _ = gpu_tau(w, precision)
    sp = torch.as_tensor(w.species).cuda()
    g, _ = B.kubo_sigma_backward(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, torch.as_tensor(J).cuda(), tau,
                                 w.volume, torch.as_tensor(wgt).cuda(), precision)
    g = g.cpu().numpy()
    for e in range(2):
        assert rel_err_blocks(g[e][None], ref[e][None]) < TOL[precision]


def test_gradient_store_equals_recompute():
    a = _grad_case("fp64", False)
    b = _grad_case("fp64", True)
    assert np.array_equal(a[3], b[3])


def test_gradient_central_differences():
    """FD of the GPU forward (FP64): every atom is its own species, so the per-species
    gradient is the per-site map; perturb (a,b) and (b,a) together (t^{-1} stays symmetric)."""
    B = _B()
    base = _alloy32(seed=21)
    N = base.n_atoms
    w = base
    w.tinv = base.tinv[base.species].copy()          # [N, nE, K, K]
    J_species = B.dipole_current(w.lmax, base.r_ll)
    J_atoms = J_species[base.species].copy()
    w.species = np.arange(N, dtype=np.int32)
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    Jd = torch.as_tensor(J_atoms).cuda()
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt[0, 0, 0] = 1.0                                # d Re sigma_xx

    def f(tinv):
        tau, _ = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(tinv).cuda(), w.z, "fp64")
        s, _, _ = B.kubo_sigma(lz, w.lmax, sp, Jd, tau, 1, w.volume)
        return s.cpu().numpy()[0, 0, 0].real

    tau, _ = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, "fp64")
    _, gs = B.kubo_sigma_backward(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, Jd, tau, w.volume,
                                  torch.as_tensor(wgt).cuda(), "fp64")
    gs = gs.cpu().numpy()                              # [N, nE, K, K], PyTorch convention
    h = 1e-6
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(6):
        i, e = int(rng.integers(N)), int(rng.integers(2))
        a, b = int(rng.integers(16)), int(rng.integers(16))
        for step, part in ((h, "re"), (1j * h, "im")):
            tp, tm = w.tinv.copy(), w.tinv.copy()
            for (x, y) in {(a, b), (b, a)}:
                tp[i, e, x, y] += step
                tm[i, e, x, y] -= step
            fd = (f(tp) - f(tm)) / (2 * h)
            G = gs[i, e, a, b] + (gs[i, e, b, a] if a != b else 0)
            ref = G.real if part == "re" else G.imag
            assert abs(fd - ref) < 1e-5 * np.abs(gs).max() + 1e-7 * abs(ref), (i, e, a, b, part, fd, ref)
            checked += 1
    assert checked == 12


# ------------------------------------------------------------------ full size
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_fcc256_sampled(precision):
    """The 256-atom fcc alloy (n = 688, 512 units) in the launch configuration the
    benchmark times: sampled atoms against the oracle, all unit statuses clean."""
    w = wl.fcc_alloy_256()
    B = _B()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    _, al = B.tau_workspace_bytes(lz, w.lmax, len(w.z), B._prec(precision))
    _, tau, st, _ = gpu_tau(w, precision, workspace_bytes=al, liz=lz)
    assert int((st & 0xff).abs().sum()) == 0
    atoms = [0, 101, 255]
    L, col, _ = oracle_tau(w, atoms=atoms)
    t = tau.cpu().numpy()
    for m in atoms:
        s = slice(L["offsets"][m], L["offsets"][m + 1])
        for e in range(2):
            assert rel_err_blocks(t[e, s][None], col[e, s][None]) < TOL[precision]


@pytest.mark.parametrize("lmax", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_odd_sizes_several_panels(lmax, precision):
    """45-atom cluster covered by every LIZ: n = 45 (odd, lmax = 0) or 180, so the
    factorization runs several panels with a ragged last one and odd strides."""
    w = wl.cluster(n_atoms=45, lmax=lmax, r_liz=200.0, seed=9, spread=13.0)
    lz, tau, st, _ = gpu_tau(w, precision)
    assert int((st & 0xff).abs().sum()) == 0
    atoms = [0, 17, 44]
    L, col, _ = oracle_tau(w, atoms=atoms)
    t = tau.cpu().numpy()
    for m in atoms:
        s = slice(L["offsets"][m], L["offsets"][m + 1])
        for e in range(2):
            assert rel_err_blocks(t[e, s][None], col[e, s][None]) < TOL[precision]


@pytest.mark.parametrize("lmax,n_atoms", [(3, 2), (1, 8), (3, 24), (3, 26), (3, 28), (3, 29)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_sizes_multiple_of_the_panel_width(lmax, n_atoms, precision):
    """Clusters covered by every LIZ with n = 32, 32, 384, 416, 448 and 464: full last
    panels (n a multiple of 32), a single-panel matrix, and the first panel at and just
    above the complex128 shared-memory panel limit (448 rows)."""
    w = wl.cluster(n_atoms=n_atoms, lmax=lmax, r_liz=400.0, seed=11, spread=4.0 * n_atoms ** (1 / 3) + 3.0)
    lz, tau, st, _ = gpu_tau(w, precision)
    assert int((st & 0xff).abs().sum()) == 0
    atoms = sorted({0, n_atoms - 1})
    L, col, _ = oracle_tau(w, atoms=atoms)
    t = tau.cpu().numpy()
    for m in atoms:
        s = slice(L["offsets"][m], L["offsets"][m + 1])
        for e in range(2):
            assert rel_err_blocks(t[e, s][None], col[e, s][None]) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_step_overlap_matches_forward_then_backward(precision):
    """Problem.step runs sigma's traces on a side stream beside the adjoint; the
    results are bit-identical to forward() followed by backward()."""
    from paper_2311_12134_gb300 import binding as B
    from paper_2311_12134_gb300.conductivity import Problem
    w = _alloy32(seed=29)
    J = B.dipole_current(w.lmax, w.r_ll)
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume, precision=precision)
    gs = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    gs[0, 2, 0] = 1.0
    p.forward()
    g_seq = [t.clone() for t in p.backward(gs)]
    torch.cuda.synchronize()
    sig_seq, tau_seq = p.sigma_out.clone(), p.tau.clone()
    p.sigma_out.zero_()
    sig, g = p.step(gs)
    torch.cuda.synchronize()
    assert torch.equal(sig, sig_seq) and torch.equal(p.tau, tau_seq)
    assert torch.equal(g[0], g_seq[0]) and torch.equal(g[1], g_seq[1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cuda_graph_replay_matches_eager(precision):
    """The whole forward + adjoint step captured in one CUDA graph and replayed gives
    bit-identical tau, sigma and gradient to the eager calls."""
    from paper_2311_12134_gb300 import binding as B
    from paper_2311_12134_gb300.conductivity import Problem, StepGraph
    w = _alloy32(seed=17)
    J = B.dipole_current(w.lmax, w.r_ll)
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume, precision=precision)
    gs = torch.zeros((1, 3, 3), dtype=torch.complex128, device="cuda")
    gs[0, 0, 0] = 1.0
    p.forward()
    g_eager, gs_eager = [t.clone() for t in p.backward(gs)]
    torch.cuda.synchronize()
    tau_e, sig_e = p.tau.clone(), p.sigma_out.clone()
    sg = StepGraph(p, gs)
    p.tau.zero_()
    p.sigma_out.zero_()
    sg.grads[0].zero_()
    sg.replay()
    sg.replay()
    torch.cuda.synchronize()
    assert torch.equal(p.tau, tau_e)
    assert torch.equal(p.sigma_out, sig_e)
    assert torch.equal(sg.grads[0], g_eager)
    assert torch.equal(sg.grads[1], gs_eager)
