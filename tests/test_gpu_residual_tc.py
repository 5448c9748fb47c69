"""The mixed form's refinement residual on the tensor cores (bf16 fixed-point
digits, exact FP32 accumulation) against the double-float SIMT residual and the
oracle: the same refined tau and gradient to the mixed-form tolerance, with the
same number of refinement sweeps and probes (the residual is accurate enough for
the convergence test at 1e-10), on ragged sizes (n not a multiple of the 128-row
tile or the 16-column chunk), 9/18 right-hand sides (lmax = 2) and 16/32 (lmax = 3).
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

TOL = 1e-8


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


@contextlib.contextmanager
def residual_tc(B, on):
    saved = B.get_option("residual_tc")
    B.set_option("residual_tc", 1 if on else 0)
    try:
        yield
    finally:
        B.set_option("residual_tc", saved)


def _workloads():
    a = 7.65
    return {
        # n = 208 (two row tiles, 13 chunks), lmax 3
        "alloy32": wl.make_supercell(name="alloy32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                                     r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002],
                                     seed=99),
        # uneven LIZ, n = 688..944 (ragged tiles), three deltas, lmax 3
        "bcc54": wl.bcc_disordered_2000(n_cells=3),
        # lmax 2: 9 right-hand sides forward, 18 in the adjoint (two column slices)
        "alloy32_l2": wl.make_supercell(name="alloy32l2", kind="fcc", n_cells=2, a=a, counts=[20, 12],
                                        sigma_disp=0.1, r_liz=0.85 * a, phases=[wl.PHASE_A[:3], wl.PHASE_B[:3]],
                                        e_fermi=0.6, deltas=[0.002], lmax=2, seed=98),
    }


@pytest.mark.parametrize("name", ["alloy32", "bcc54", "alloy32_l2"])
def test_tau_tensor_core_residual(B, name):
    w = _workloads()[name]
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    atoms = [0, 1, w.n_atoms - 1]
    col = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms)
    out = {}
    for on in (False, True):
        with residual_tc(B, on):
            lz = B.build_liz(w.pos, w.lattice, w.r_liz)
            tau, st = B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(),
                                   w.z, "mixed")
            torch.cuda.synchronize()
        out[on] = (tau.cpu().numpy(), st.cpu().numpy())
    off = L["offsets"]
    for on in (False, True):
        t, st = out[on]
        assert not np.any(st & 0xff), (on, np.unique(st & 0xff))
        for m in atoms:
            s = slice(off[m], off[m + 1])
            for e in range(len(w.z)):
                err = np.linalg.norm(t[e, s] - col[e, s]) / np.linalg.norm(col[e, s])
                assert err < TOL, (on, m, e, err)
    # the same refinement path: sweeps and probes per unit agree (a borderline unit may differ by one)
    sw = {on: ((out[on][1] >> 8) & 0xff).astype(float) for on in out}
    pr = {on: ((out[on][1] >> 16) & 0xff).astype(float) for on in out}
    assert abs(sw[True].mean() - sw[False].mean()) <= 0.02 and sw[True].max() <= sw[False].max() + 1
    assert abs(pr[True].mean() - pr[False].mean()) <= 0.02
    diff = unit_rel_errors(out[True][0], out[False][0], off)
    assert diff.max() < 1e-9, diff.max()


@pytest.mark.parametrize("store", [True, False])
def test_gradient_tensor_core_residual(B, store):
    """The adjoint's 32-column solves refined with the tensor-core residual against the oracle's
    dense gradient."""
    w = _workloads()["alloy32"]
    J = okubo.dipole_current(w.lmax, w.r_ll)
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    wgt = np.zeros((1, 3, 3), dtype=np.complex128)
    wgt[0, 0, 0] = 1.0
    wgt[0, 0, 2] = -0.4 + 0.1j
    ref = ograd.torch_grad(ograd.dense_gradient(w.lmax, L, w.tinv[w.species], w.z, J[w.species], 1, w.volume, wgt))
    with residual_tc(B, True):
        lz = B.build_liz(w.pos, w.lattice, w.r_liz)
        sp = torch.as_tensor(w.species).cuda()
        t = torch.as_tensor(w.tinv).cuda()
        st_buf = None
        if store:
            st_buf = torch.empty(B.lu_store_bytes(lz, w.lmax, 2, B.LSMS_MIXED), dtype=torch.uint8, device="cuda")
        tau, st = B.tau_blocks(lz, w.lmax, sp, t, w.z, "mixed", lu_store=st_buf)
        bst = torch.empty_like(st)
        g, _ = B.kubo_sigma_backward(lz, w.lmax, sp, t, w.z, torch.as_tensor(J).cuda(), tau, w.volume,
                                     torch.as_tensor(wgt).cuda(), "mixed", lu_store=st_buf, unit_status=bst)
        torch.cuda.synchronize()
    b = bst.cpu().numpy()
    assert not np.any(b & 0xff), np.unique(b & 0xff)
    assert ((b >> 8) & 0xff).max() == 1
    g = g.cpu().numpy()
    assert np.linalg.norm(g - ref) < TOL * np.linalg.norm(ref)
