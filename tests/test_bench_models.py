"""The bench's count of the sparse trace and adjoint products (the work its
per-kernel rooflines divide by) against a loop-by-loop count of what the
kernels do: per site, the J rows (columns) with their nonzero entries, the Abar
columns (rows) with theirs, a zero Abar^nu skipped, and the Y entries the trace
reads (the transposed union of the centre's J patterns)."""
import os
import sys

import numpy as np
import pytest

from oracle import kubo as okubo
from oracle import liz as oliz
from paper_2311_12134_gb300 import workload as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _loop_count(J, species, L, gs, K, n_delta):
    off, sa, sp = L["offsets"], L["site_atom"], species
    swap = [0, 2, 1, 3]
    adj = tr = 0
    for m in range(len(off) - 1):
        spm = sp[m]
        for e in range(2 * n_delta):
            d, sgn = e >> 1, e & 1
            for n in range(off[m], off[m + 1]):
                s = sp[sa[n]]
                for part in range(2):
                    for cc in range(2):
                        c = (sgn << 1) | cc if part == 0 else (cc << 1) | sgn
                        for v in range(3):
                            A = sum(np.conj(gs[d, u, v]) * J[spm, swap[c], u] for u in range(3))
                            if not np.any(A != 0):
                                continue
                            Jm = J[s, c, v]
                            for i in range(K):
                                adj += K * (np.count_nonzero(Jm[i]) if part == 0 else np.count_nonzero(Jm[:, i]))
                                adj += K * (np.count_nonzero(A[:, i]) if part == 0 else np.count_nonzero(A[i]))
        for d in range(n_delta):
            for c in range(4):
                need = np.zeros((K, K), bool)
                for u in range(3):
                    need |= (J[spm, swap[c], u] != 0).T
                for n in range(off[m], off[m + 1]):
                    s = sp[sa[n]]
                    for v in range(3):
                        tr += K * np.count_nonzero(J[s, c, v])
                    tr += int(need.sum()) * 3 * K
    return adj, tr


@pytest.mark.parametrize("weights", ["xx", "xx_yz"])
def test_sparse_product_count_matches_the_kernels_loops(weights):
    w = wl.make_supercell(name="t", kind="bcc", n_cells=1, a=5.42, counts=[1, 1], sigma_disp=0.0, r_liz=1.2 * 5.42,
                          phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.62, deltas=[0.002, 0.004], seed=3)
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    J = okubo.dipole_current(w.lmax, w.r_ll)
    gs = np.zeros((w.n_delta, 3, 3), dtype=np.complex128)
    gs[:, 0, 0] = 1.0
    if weights == "xx_yz":
        gs[:, 1, 2] = 0.3 - 0.1j
    got = bench.sparse_product_cmacs(J, np.asarray(w.species), L["offsets"], L["site_atom"], gs, w.K)
    want = _loop_count(J, np.asarray(w.species), L, gs, w.K, w.n_delta)
    assert got == pytest.approx(want, rel=0, abs=0)
