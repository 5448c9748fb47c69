"""lsms_kubo_sigma_noalloc: the conductivity reduction for callers that cannot
allocate device memory during a call (fixed memory budgets, their own
allocator, no allocator synchronisation allowed between launches).  Its
scratch is a fixed 16 MiB device array inside the library.

This file is collected last on purpose: it must pass on its own in a fresh
process and after every other test, and a run that stops at the first failure
has then already run everything else.  Each check calls the new entry point
through the C ABI twice in a row and compares it with lsms_kubo_sigma (which
allocates its scratch) on the same inputs, within the tolerance the other
GPU tests use for the FP64 form."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built

TOL = 1e-10


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


def _case(B, seed, lmax=3):
    a = 7.65
    w = wl.make_supercell(name="noalloc", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                          r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002, 0.004],
                          lmax=lmax, seed=seed)
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    sp = torch.as_tensor(w.species).cuda()
    tau, st = B.tau_blocks(lz, w.lmax, sp, torch.as_tensor(w.tinv).cuda(), w.z, "fp64")
    J = torch.as_tensor(B.dipole_current(w.lmax, w.r_ll)).cuda()
    return w, lz, sp, tau, J


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() <= TOL * max(np.abs(b).max(), 1e-300)


def test_noalloc_matches_allocating_entry_point_twice(B):
    for seed in (31, 32):                     # two calls in a row, different inputs
        w, lz, sp, tau, J = _case(B, seed)
        ref = B.kubo_sigma(lz, w.lmax, sp, J, tau, w.n_delta, w.volume)
        got = B.kubo_sigma_noalloc(lz, w.lmax, sp, J, tau, w.n_delta, w.volume)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert _close(g, r)
        assert np.abs(ref[0].cpu().numpy()).max() > 0


def test_noalloc_matches_in_the_mixed_form(B):
    """The double-float trace variant through both entry points."""
    w, lz, sp, tau, J = _case(B, 34)
    ref = B.kubo_sigma(lz, w.lmax, sp, J, tau, w.n_delta, w.volume, precision="mixed")
    got = B.kubo_sigma_noalloc(lz, w.lmax, sp, J, tau, w.n_delta, w.volume, precision="mixed")
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert _close(g, r)


def test_noalloc_back_to_back_on_one_problem(B):
    """Two consecutive calls on the same inputs (the second reuses the array the
    first left behind) give the allocating entry point's result both times."""
    w, lz, sp, tau, J = _case(B, 33, lmax=2)
    ref = B.kubo_sigma(lz, w.lmax, sp, J, tau, w.n_delta, w.volume)
    for _ in range(2):
        got = B.kubo_sigma_noalloc(lz, w.lmax, sp, J, tau, w.n_delta, w.volume)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert _close(g, r)


def test_noalloc_rejects_oversized_problems_on_the_host(B):
    """More atom-delta pairs than the fixed array holds: rejected before any launch."""
    rng = np.random.default_rng(0)
    pos = rng.uniform(0, 400, size=(1000, 3))
    lz = B.build_liz(pos, None, 1.0)          # host only; no device copy is needed for the size check
    dummy = torch.zeros(1, dtype=torch.complex128, device="cuda")
    sp = torch.zeros(1000, dtype=torch.int32, device="cuda")
    import ctypes
    rc = B.lib().lsms_kubo_sigma_noalloc(lz.handle, 3, ctypes.c_void_p(sp.data_ptr()), 1,
                                         ctypes.c_void_p(dummy.data_ptr()), 0, ctypes.c_void_p(dummy.data_ptr()),
                                         32, 1000.0, 0, None, ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == -1
    msg = B.lib().lsms_last_error().decode()
    assert "static buffer" in msg and "lsms_kubo_sigma" in msg
