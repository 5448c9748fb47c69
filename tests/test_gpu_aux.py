"""Auxiliary subsystems on the GPU: the per-call statistics record
(lsms_unit_stats) against a host decoding of the same status words, the pivot-
growth code in the status words, NVTX ranges leaving results unchanged, and the
LSMS_DEBUG_BOUNDS build (device-side index checks) matching the oracle with no
check firing, in a child process that loads that build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2311_12134_gb300 import workload as wl

from ._util import ensure_built

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2311_12134_gb300 import binding
    return binding


def _alloy():
    a = 7.65
    return wl.make_supercell(name="alloy32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                             r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002, 0.004],
                             seed=99)


def _host_stats(st):
    st = st.astype(np.int64)
    flags = st & 0xff
    return {
        "units": st.size,
        "zero_pivot": int(np.sum(flags & 1 != 0)), "noconv": int(np.sum(flags & 2 != 0)),
        "nonfinite": int(np.sum(flags & 4 != 0)), "bad_input": int(np.sum(flags & 8 != 0)),
        "tinv_asym": int(np.sum(flags & 16 != 0)), "growth": int(np.sum(flags & 32 != 0)),
        "fp64_fallback": int(np.sum(flags & 64 != 0)), "timeout": int(np.sum(flags & 128 != 0)),
        "invalid": int(np.sum((flags & ~64) != 0)),
        "sweeps_sum": int(((st >> 8) & 0xff).sum()), "sweeps_max": int(((st >> 8) & 0xff).max()),
        "probes_sum": int(((st >> 16) & 0xff).sum()), "probes_max": int(((st >> 16) & 0xff).max()),
        "growth_code_max": int(((st >> 24) & 0x7f).max()),
    }


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_unit_stats_match_host_decoding(B, precision):
    w = _alloy()
    lz = B.build_liz(w.pos, w.lattice, w.r_liz)
    tau, st = B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(), w.z,
                           precision)
    d = B.unit_stats(st)
    h = _host_stats(st.cpu().numpy())
    for k, v in h.items():
        assert d[k] == v, (k, d[k], v)
    if precision == "mixed":
        # growth recorded for every unit; max|U| / max|M| of a pivoted LU of these matrices is O(1)
        codes = (st.cpu().numpy() >> 24) & 0x7f
        assert np.all(codes > 0)
        assert 2.0 ** -8 <= d["growth_max"] <= 2.0 ** 8
        assert d["sweeps_max"] >= 1 and d["invalid"] == 0
    else:
        assert d["growth_code_max"] == 0 and d["growth_max"] is None and d["sweeps_sum"] == 0


def test_unit_stats_counts_planted_flags(B):
    """Words with flags planted on the host: counts, sums and maxima per field."""
    rng = np.random.default_rng(7)
    st = rng.integers(0, 1 << 31, size=5000, dtype=np.int64).astype(np.int32)
    d = B.unit_stats(torch.as_tensor(st).cuda())
    h = _host_stats(st)
    for k, v in h.items():
        assert d[k] == v, (k, d[k], v)
    assert B.unit_stats(torch.zeros(0, dtype=torch.int32, device="cuda"))["units"] == 0


def test_problem_stats_json(B, tmp_path):
    from oracle import kubo as okubo
    from paper_2311_12134_gb300.conductivity import Problem
    w = _alloy()
    J = okubo.dipole_current(w.lmax, w.r_ll)
    p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume, precision="mixed")
    gs = torch.zeros((w.n_delta, 3, 3), dtype=torch.complex128, device="cuda")
    gs[:, 0, 0] = 1.0
    p.step(gs)
    torch.cuda.synchronize()
    path = tmp_path / "stats.jsonl"
    with open(path, "w") as f:
        s = p.stats(log=f)
    rec = json.loads(path.read_text().splitlines()[0])
    assert rec == json.loads(json.dumps(s))
    assert s["forward"]["units"] == s["backward"]["units"] == p.n_units
    assert s["forward"]["invalid"] == 0 and s["backward"]["invalid"] == 0


def test_nvtx_ranges_keep_results(B):
    w = _alloy()
    out = []
    saved = B.get_option("nvtx")
    try:
        for on in (0, 1):
            B.set_option("nvtx", on)
            lz = B.build_liz(w.pos, w.lattice, w.r_liz)
            tau, st = B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(),
                                   w.z, "mixed")
            torch.cuda.synchronize()
            out.append((tau.cpu(), st.cpu()))
    finally:
        B.set_option("nvtx", saved)
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


_CHILD = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2311_12134_gb300 import binding as B
from paper_2311_12134_gb300 import workload as wl
from oracle import kkr as okkr, liz as oliz
res = {"lib": B.lib_path()}
a = 7.65
cases = {
    "alloy32": wl.make_supercell(name="alloy32", kind="fcc", n_cells=2, a=a, counts=[20, 12], sigma_disp=0.1,
                                 r_liz=0.85 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.6, deltas=[0.002],
                                 seed=99),
    "cluster24": wl.cluster(n_atoms=24, lmax=3, r_liz=400.0, seed=11, spread=4.0 * 24 ** (1 / 3) + 3.0),
}
for name, w in cases.items():
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    atoms = [0, w.n_atoms - 1]
    col = okkr.tau_blocks(w.lmax, L, w.tinv[w.species], w.z, atoms=atoms)
    for prec in ("fp64", "mixed"):
        lz = B.build_liz(w.pos, w.lattice, w.r_liz)
        tau, st = B.tau_blocks(lz, w.lmax, torch.as_tensor(w.species).cuda(), torch.as_tensor(w.tinv).cuda(),
                               w.z, prec)
        t = tau.cpu().numpy()
        err = 0.0
        for m in atoms:
            s = slice(L["offsets"][m], L["offsets"][m + 1])
            for e in range(len(w.z)):
                err = max(err, float(np.linalg.norm(t[e, s] - col[e, s]) / np.linalg.norm(col[e, s])))
        res[name + "/" + prec] = {"err": err, "flags": int(np.bitwise_or.reduce((st.cpu().numpy() & 0xff).ravel())),
                                  "n": int(16 * lz.max_sites)}
print("RESULT " + json.dumps(res))
"""


def test_debug_bounds_build_matches_oracle(B):
    """The LSMS_DEBUG_BOUNDS build (index checks on pivots and the row permutation) gives the oracle's
    tau, with no check firing, on a ragged size and on n = 384 (full last panels)."""
    from paper_2311_12134_gb300 import build as bld
    if not os.path.exists(bld.LIB_DEBUG):
        bld.build(debug_bounds=True)
    env = dict(os.environ, LSMS_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert res.pop("lib").endswith("liblsmskubo_debug.so")
    assert res["cluster24/fp64"]["n"] == 384
    for k, v in res.items():
        assert v["flags"] == 0, (k, v)
        assert v["err"] < (1e-10 if k.endswith("fp64") else 1e-8), (k, v)
