"""The conjugate-pair mode (LSMS_CONJ_PAIRS): with z[2d+1] = conj z[2d] and
conjugate t^-1, M(conj z) = conj M(z) in the real-harmonic basis (g(z*) =
conj g(z)), so only z is factored and tau(conj z) = conj tau(z); the adjoint of
the conj z systems reuses the z factors on conjugated right-hand sides.  Checked
against the plain mode (every energy factored) and, for tau, against the oracle."""
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


def _alloy(seed=5):
    a = 7.65
    return wl.make_supercell(name="conj", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                             r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002, 0.004],
                             lmax=3, seed=seed)


def _step(B, w, precision, conj, lu_store):
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    tinv = torch.as_tensor(w.tinv).cuda()
    store = None
    if lu_store:
        store = torch.empty(B.lu_store_bytes(lz, w.lmax, len(w.z), B._prec(precision, conj)), dtype=torch.uint8,
                            device="cuda")
    tau, st = B.tau_blocks(lz, w.lmax, sp, tinv, w.z, precision, lu_store=store, conj_pairs=conj)
    J = torch.as_tensor(B.dipole_current(w.lmax, w.r_ll)).cuda()
    sig, _, _ = B.kubo_sigma(lz, w.lmax, sp, J, tau, w.n_delta, w.volume, precision=precision)
    wgt = torch.zeros((w.n_delta, 3, 3), dtype=torch.complex128, device="cuda")
    wgt[:, 0, 0] = 1.0
    wgt[1, 1, 2] = 0.5 - 0.25j
    bst = torch.empty((len(w.z), w.n_atoms), dtype=torch.int32, device="cuda")
    g, gs = B.kubo_sigma_backward(lz, w.lmax, sp, tinv, w.z, J, tau, w.volume, wgt, precision, lu_store=store,
                                  unit_status=bst, conj_pairs=conj)
    torch.cuda.synchronize()
    return (lz, tau.cpu().numpy(), st.cpu().numpy(), sig.cpu().numpy(), g.cpu().numpy(), gs.cpu().numpy(),
            bst.cpu().numpy())


@pytest.mark.parametrize("lu_store", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_conj_pairs_match_plain_mode(B, precision, lu_store):
    w = _alloy()
    lz, t0, st0, s0, g0, gs0, b0 = _step(B, w, precision, False, lu_store)
    lz, t1, st1, s1, g1, gs1, b1 = _step(B, w, precision, True, lu_store)
    assert np.all((st1 & 0xff) == 0) and np.all((b1 & 0xff) == 0)
    # the second energy of each pair copies its partner's status (no solves of its own)
    assert np.array_equal(st1[1::2], st1[0::2])
    off = lz.export()["offsets"]
    worst = 0.0
    for e in range(len(w.z)):
        for m in range(w.n_atoms):
            s = slice(off[m], off[m + 1])
            worst = max(worst, rel_err_blocks(t1[e, s][None], t0[e, s][None]))
    assert worst < TOL[precision], worst
    assert np.abs(s1 - s0).max() < TOL[precision] * np.abs(s0).max()
    assert np.linalg.norm(g1 - g0) < TOL[precision] * np.linalg.norm(g0)
    assert np.linalg.norm(gs1 - gs0) < TOL[precision] * np.linalg.norm(gs0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_conj_pairs_tau_against_oracle(B, precision):
    w = _alloy(seed=6)
    lz, t, st, _, _, _, _ = _step(B, w, precision, True, True)
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    atoms = [0, 17, w.n_atoms - 1]
    col = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms)
    off = L["offsets"]
    for m in atoms:
        s = slice(off[m], off[m + 1])
        for e in range(len(w.z)):
            assert rel_err_blocks(t[e, s][None], col[e, s][None]) < TOL[precision]


def test_conj_pairs_store_is_half(B):
    w = _alloy()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    for precision in ("fp64", "mixed"):
        full = B.lu_store_bytes(lz, w.lmax, len(w.z), B._prec(precision))
        half = B.lu_store_bytes(lz, w.lmax, len(w.z), B._prec(precision, True))
        assert 2 * half == full


def test_conj_pairs_flags_nonconjugate_tinv(B):
    """A t^-1 pair that is not conjugate: the second energies of that pair are
    flagged LSMS_UNIT_BAD_INPUT (their tau would be wrong), the rest stay clean."""
    w = _alloy()
    tinv = w.tinv.copy()
    tinv[:, 3] += 1e-6  # pair d = 1
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    _, st = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(tinv).cuda(), w.z, "mixed", conj_pairs=True)
    st = st.cpu().numpy()
    assert np.all(st[3] & 8) and np.all((st[[0, 1, 2]] & 0xff) == 0)


def test_conj_pairs_rejects_nonconjugate_energies(B):
    w = _alloy()
    z = w.z.copy()
    z[1] = z[1] + 1e-9
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    with pytest.raises(B.LsmsError):
        B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), z, "fp64", conj_pairs=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_conj_pairs_trace_halving(B, precision):
    """With conjugate-pair tau and J(-,-) = conj J(+,+), J(-,+) = conj J(+,-) (the dipole model), the
    halved traces (only (+,+) and (+,-) computed) give the sigma~ and sigma of all four; with current
    matrices that break the relation all four are computed, as without the flag."""
    w = _alloy()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, precision, conj_pairs=True)
    J = torch.as_tensor(B.dipole_current(w.lmax, w.r_ll)).cuda()
    rng = np.random.default_rng(17)
    Jr = J.clone()
    Jr[:, 3] += torch.as_tensor(1e-3 * rng.standard_normal(Jr[:, 3].shape)).cuda()   # breaks J(-,-) = conj J(+,+)
    for Jx, halves in ((J, True), (Jr, False)):
        s_full, st_full, _ = B.kubo_sigma(lz, w.lmax, sp, Jx, tau, w.n_delta, w.volume, precision=precision)
        s_half, st_half, _ = B.kubo_sigma(lz, w.lmax, sp, Jx, tau, w.n_delta, w.volume, precision=precision,
                                          conj_pairs=True)
        torch.cuda.synchronize()
        a, b = st_half.cpu().numpy(), st_full.cpu().numpy()
        if halves:
            assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
            assert np.array_equal(a[:, 3], np.conj(a[:, 0])) and np.array_equal(a[:, 2], np.conj(a[:, 1]))
        else:
            assert np.array_equal(a, b)
        sa, sb = s_half.cpu().numpy(), s_full.cpu().numpy()
        assert np.abs(sa - sb).max() <= 1e-12 * np.abs(sb).max()
