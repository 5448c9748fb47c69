"""Benchmark of the LSMS Kubo-Greenwood hot path on GB300.

Default workload (bcc2000): the 1980-site bcc A/B alloy of 10x10x10 cells
(a = 5.42 bohr, 1670/330 A/B minus 20 random vacancies, Gaussian displacements
of 0.05 a per component), lmax = 3, LIZ radius 1.75 a (43..59 sites, uneven
LIZ matrices of n = 688..944), E_F = 0.62 Ry and three broadenings
delta = 0.001, 0.002, 0.004 Ry, energies E_F +- i delta: 11,880 (atom, energy)
units per step.  Synthetic, seeded inputs (no self-consistent potentials).

One step = the whole path: KKR matrix assembly, LU, tau column blocks (+ FP64
refinement and the FP64 fallback in the mixed form), Kubo-Greenwood traces,
sigma and rho per delta, and the adjoint d sigma_xx / d t^{-1} reusing the
stored LU factors.  Metric: (atom, energy) LIZ tau-solves per second;
value = units / step time, mixed form (complex64 tensor-core LU + FP64-class
refinement); the FP64 form runs on the same GPU for comparison, and both are
checked against the CPU FP64 oracle per delta.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--workload bcc2000|fcc256|fcc108|bcc432] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) each rank runs an independent replica of
the workload (the path has no exchange step on one structure of this size).
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom·energy LIZ τ-solves/s and σ time: mixed-prec vs FP64, rel err ≤1e-8"
UNIT = "units/s"

WORKLOADS = {
    "bcc2000": "bcc2000_AB_vac_disp_liz175: 1980-site bcc A/B alloy (10^3 cells, a=5.42 bohr, 1670/330 A/B, "
               "20 vacancies, displacements 0.05a), lmax=3, LIZ 1.75a = 43..59 sites (n=688..944), E_F=0.62 Ry, "
               "delta=0.001/0.002/0.004 Ry, 11880 units",
    "bcc432": "bcc432_AB_vac_disp_liz175: the bcc2000 recipe on 6^3 cells (432 sites, 4 vacancies), "
              "LIZ 1.75a, three deltas",
    "fcc256": "fcc256_AB50_liz43: 256-atom fcc A/B alloy, lmax=3, LIZ 43 sites (n=688), E_F=0.60 Ry, "
              "delta=0.002 Ry, 512 units",
    "fcc108": "fcc108_AB50_liz43: the fcc256 recipe on 3^3 cells (108 atoms), 216 units",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="bcc2000", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64-form comparison leg")
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the FP64-form leg")
    ap.add_argument("--no-conj-leg", action="store_true", help="skip the conjugate-pair leg")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kernel-timers", action="store_true")
    ap.add_argument("--oracle-s", type=float, default=20.0, help="CPU budget of the oracle sample (s)")
    ap.add_argument("--chunk-mb", type=int, default=8192,
                    help="workspace size in MiB (units are processed in chunks that fit); 0 = all units at once")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return world > 1


def barrier(active):
    if active:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, active, device="cpu"):
    if not active:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # samples go to LSMS_CLOCKS_DIR (default: the system temporary directory)
        out_dir = os.environ.get("LSMS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"lsms_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- workload / algorithmic work
def workload(name):
    from paper_2311_12134_gb300 import workload as wl
    if name == "bcc2000":
        return wl.bcc_disordered_2000()
    if name == "bcc432":
        return wl.bcc_disordered_2000(n_cells=6)
    if name == "fcc108":
        a = 7.65
        return wl.make_supercell(name="fcc108_AB50_liz43", kind="fcc", n_cells=3, a=a, counts=[54, 54],
                                 r_liz=1.30 * a, phases=[wl.PHASE_A, wl.PHASE_B], e_fermi=0.60, deltas=[0.002],
                                 seed=2311 + 1)
    return wl.fcc_alloy_256()


def path_flops(n_list):
    """The method's algorithmic work per (atom, energy) unit, summed: F(n) = (8/3) n^3 + 128 n^2 real
    flops (LU of the n x n complex LIZ matrix + the 16-column solve for tau^{n0}).  Refinement, split
    products and the adjoint are not counted."""
    n = np.asarray(n_list, dtype=np.float64)
    return float(np.sum(8.0 / 3.0 * n ** 3 + 128.0 * n ** 2))


def gemm_bytes(n_list, nb):
    """Algorithmic DRAM bytes of the complex64 trailing updates: A22 read + written,
    L21 and U12 read once per panel step."""
    tot = 0.0
    for n in n_list:
        for k in range(0, n, nb):
            t = n - k - nb
            if t > 0:
                tot += 16.0 * t * t + 2 * 8.0 * nb * t
    return tot


def gemm_flops(n_list, nb):
    """Algorithmic flops of the trailing-update GEMMs of a blocked LU with panel width nb."""
    tot = 0.0
    for n in n_list:
        for k in range(0, n, nb):
            t = n - k - nb
            if t > 0:
                tot += 8.0 * nb * t * t
    return tot


def file_peaks():
    """Measured peaks of this GPU pool (MEASURED_PEAKS.json), else the fallback figures."""
    p = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
         "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p.update({k: m[k] for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained", "sm_max_mhz") if k in m})
        p["source"] = "measured (MEASURED_PEAKS.json)"
    return p


def measure_gemm_peaks(dev):
    """cuBLAS dense GEMM throughput measured here, for the rooflines the pool file lacks:
    TF32 (FP32 inputs on the tensor cores, 8192^3) and FP64 (4096^3); best of several runs,
    CUDA events.  The 3xTF32 complex product of the mixed form peaks at TF32 / 3."""
    import torch
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dtype, n, reps, tf32 in (("tf32_tflops", torch.float32, 8192, 6, True),
                                           ("fp64_tflops", torch.float64, 4096, 3, False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            a = torch.randn(n, n, device=dev, dtype=dtype)
            b = torch.randn(n, n, device=dev, dtype=dtype)
            torch.matmul(a, b)
            torch.cuda.synchronize(dev)
            best = 0.0
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize(dev)
                best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
            out[name] = best
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    out["how"] = ("torch.matmul (cuBLAS) best of 6 at 8192^3 with TF32 allowed (FP32 inputs), best of 3 at "
                  "4096^3 in float64, CUDA events, in this run")
    return out


# ---------------------------------------------------------------- CPU oracle
def sample_atoms(w, liz_offsets, count, seed=2311):
    """Seeded atoms for the oracle checks: the largest and the smallest LIZ, then random ones."""
    sizes = np.diff(liz_offsets)
    first = [int(np.argmax(sizes)), int(np.argmin(sizes))]
    rng = np.random.default_rng(seed)
    rest = [int(a) for a in rng.permutation(w.n_atoms) if int(a) not in first]
    return (first + rest)[:count]


def time_oracle(w, atoms, budget_s):
    """Oracle (NumPy FP64, LAPACK) on a bounded sample: for each atom in turn, the tau blocks of every
    energy (column and row blocks, dense solves) and the atom's trace terms, until the budget is spent.
    Returns (units/s, units, seconds, cores, results)."""
    from oracle import kkr as okkr
    from oracle import kubo as okubo
    from oracle import liz as oliz
    L = oliz.build_liz(w.pos, w.lattice, w.r_liz)
    J = okubo.dipole_current(w.lmax, w.r_ll)[w.species]
    tin = w.tinv[w.species]
    off, sa = L["offsets"], L["site_atom"]
    nE = len(w.z)
    col, row, st_atoms = {}, {}, {}
    t0 = time.perf_counter()
    done = []
    for m in atoms:
        s0, s1 = off[m], off[m + 1]
        c = np.zeros((nE, off[-1], w.K, w.K), dtype=np.complex128)
        r = np.zeros_like(c)
        for e in range(nE):
            M = okkr.kkr_matrix(w.lmax, L["disp"][s0:s1], tin[sa[s0:s1], e], w.z[e])
            c[e, s0:s1], r[e, s0:s1] = okkr.tau_col_row(M, w.K)
        st_atoms[m] = okubo.sigma_tilde(L, J, c, r, w.n_delta, w.volume, atoms=[m])
        col[m] = c[:, s0:s1].copy()
        done.append(m)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    units = len(done) * nE
    return units / dt, units, dt, os.cpu_count(), dict(col=col, sigma_tilde_atoms=st_atoms, atoms=done,
                                                         offsets=off)


def rel_sigma(a, b):
    """Norm-wise relative difference of sigma-like arrays per delta: max|a - b| / max|b|."""
    return [float(np.abs(a[d] - b[d]).max() / np.abs(b[d]).max()) for d in range(b.shape[0])]


def consolidate(st):
    """sigma = 1/4 (st++ - st+- - st-+ + st--) per delta (Eq. sigma-tilde-consolidation); st [n_delta, 4, 3, 3]."""
    return 0.25 * (st[:, 0] - st[:, 1] - st[:, 2] + st[:, 3])


def accuracy(res, tau_rows, st_atoms_gpu):
    """Errors of one GPU form against the oracle sample: worst-unit tau (norm-wise per unit) and, per
    delta, sigma summed over the sampled atoms."""
    if res is None:
        return None
    off = res["offsets"]
    errs = []
    for m in res["atoms"]:
        ref = res["col"][m]
        got = tau_rows[m]
        for e in range(ref.shape[0]):
            errs.append(np.linalg.norm(got[e] - ref[e]) / np.linalg.norm(ref[e]))
    atoms = res["atoms"]
    ref_st = sum(res["sigma_tilde_atoms"][m] for m in atoms)
    got_st = st_atoms_gpu[:, :, atoms].sum(axis=2)
    return {"tau_rel_err_max": float(max(errs)), "oracle_atoms": [int(a) for a in atoms],
            "sigma_sampled_rel_err_per_delta": rel_sigma(consolidate(got_st), consolidate(ref_st)),
            "offsets_checked": int(len(atoms))}


def run_reference(args):
    """The oracle itself on the host cores, one bounded sample of the workload per step:
    two atoms (largest and smallest LIZ) x every energy, tau blocks + their trace terms."""
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    from oracle import liz as oliz
    w = workload(args.workload)
    off = oliz.build_liz(w.pos, w.lattice, w.r_liz)["offsets"]
    atoms = sample_atoms(w, off, 2)
    vals = []
    for i in range(args.warmup + args.steps):
        v, units, dt, cores, _ = time_oracle(w, atoms, budget_s=1e9)
        if i >= args.warmup:
            vals.append((v, units, dt))
    units = vals[0][1]
    ms = float(np.mean([x[2] for x in vals])) * 1e3
    v = units / (ms * 1e-3)
    sample = (f"{len(atoms)} atoms (largest and smallest LIZ) x {len(w.z)} energies = {units} units per step: "
              "tau column and row blocks by LAPACK solves + their Kubo-Greenwood trace terms")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "global_batch": units, "parallelism": "host cores",
                       "step": "a bounded sample of the workload (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- per-kernel models
# Double-float complex multiply-accumulate: 4 real products x 11 FP32 ops
# (FMA two-product 2, cross terms 2, two-sum 6, carry 1).
DF_OPS_PER_CMAC = 44.0
PROBES = 2  # columns of the convergence probe after each refinement sweep (mixed form)


def sparse_product_cmacs(J, species, offsets, site_atom, weights, K):
    """Complex multiply-adds per step of the adjoint right-hand sides and of the
    traces as the kernels run them: products over the nonzero entries of J (and
    of Abar, the weighted sum of the centre's J), Abar^nu_c that are zero skipped,
    and only the entries of Y^nu that the trace reads (the union of the centre
    J^{m mu} patterns) accumulated.  J: [n_species, 4, 3, K, K] (or with a
    leading delta axis); weights: [n_delta, 3, 3]."""
    n_delta = weights.shape[0]
    Jd = [J[d] if J.ndim == 6 else J for d in range(n_delta)]
    n_sp = Jd[0].shape[0]
    sizes = np.diff(offsets)
    site_sp = species[site_atom]
    # LIZ sites of each atom per species
    cnt_sp = np.zeros((len(sizes), n_sp), dtype=np.int64)
    np.add.at(cnt_sp, (np.repeat(np.arange(len(sizes)), sizes), site_sp), 1)
    swap = [0, 2, 1, 3]
    adj = trace = 0.0
    for d in range(n_delta):
        nzJ = (Jd[d] != 0).sum(axis=(-1, -2))  # [sp, c, v]
        for spm in range(n_sp):
            atoms = np.nonzero(species == spm)[0]
            if len(atoms) == 0:
                continue
            S_m = sizes[atoms].astype(np.float64)
            sumJ = cnt_sp[atoms].astype(np.float64) @ nzJ.reshape(n_sp, 12)  # [atoms, (c, v)]
            for c in range(4):
                cb = swap[c]
                pat = [Jd[d][spm, cb, u] != 0 for u in range(3)]
                union = pat[0] | pat[1] | pat[2]
                trace += float(np.sum(K * sumJ[:, 3 * c:3 * c + 3].sum(axis=1) + S_m * union.sum() * 3 * K))
                for v in range(3):
                    a_pat = np.zeros((K, K), dtype=bool)
                    for u in range(3):
                        if weights[d, u, v] != 0:
                            a_pat |= pat[u]
                    nA = int(a_pat.sum())
                    if nA == 0:
                        continue
                    # unit (m, e) uses combination c in part 0 when e's sign is c's first
                    # index and in part 1 when it is c's second: each c once per part
                    adj += 2.0 * float(np.sum(K * sumJ[:, 3 * c + v] + S_m * K * nA))
    return adj, trace


def kernel_models(K, n_fwd, sweeps, n_delta, n_energy, fp32_ops, fp64_peak, tc_peak, hbm_gbs, precision, nb=32,
                  sparse=None, solve_cols=0):
    """Algorithmic real flops per step and the matching peak (TFLOP/s) for each library kernel;
    1 complex multiply-add = 8 real flops.  n_fwd: n of every forward unit; sweeps: per-unit
    refinement sweeps and probes of the forward and of the adjoint."""
    n = np.asarray(n_fwd, dtype=np.float64)
    S = n / K
    mixed = precision == "mixed"
    simt_peak = 2.0 * fp32_ops / 1e12 if mixed else fp64_peak
    df_peak = 8.0 * fp32_ops / DF_OPS_PER_CMAC / 1e12
    m = {}
    ni = [int(x) for x in n_fwd]
    if mixed:
        m["k_gemm_tc"] = (gemm_flops(ni, nb), tc_peak, "complex trailing update on tcgen05 (3xTF32); peak = "
                          "measured TF32 / 3", gemm_bytes(ni, nb))
    else:
        m["k_gemm"] = (gemm_flops(ni, nb), simt_peak, "complex trailing update, FP64 DFMA pipe")
    fs, fp, bs, bp = sweeps
    if mixed:
        rhs = K * (1 + fs) + 2 * K * (1 + bs) + PROBES * (fp + bp)
        def slices(ncols):  # column slices of a chain solve (the library's rule for solve_cols)
            if ncols <= 8:
                return 1
            sl = solve_cols if solve_cols > 0 else (8 if ncols <= 16 else 16)
            if sl == 32 and ncols <= 16:
                sl = 16
            return -(-ncols // sl)
        # bytes: one read of the complex64 factors (8 n^2) per unit, column slice and solve
        reads = slices(K) * (1 + fs) + slices(2 * K) * (1 + bs) + (fp + bp)
        m["k_solve_c64"] = (float(np.sum(8.0 * n * n * rhs)), simt_peak, "triangular solves (complex64, FP32 pipe)",
                            float(np.sum(8.0 * n * n * reads)))
        m["k_residual"] = (float(np.sum(8.0 * n * n * (K * fs + 2 * K * bs))), df_peak,
                           "FP64-accurate residual in double-float FP32 arithmetic (44 FP32 ops per complex MAC)")
        m["k_probe_residual"] = (float(np.sum(8.0 * n * n * PROBES * (fp + bp))), df_peak,
                                 "convergence-probe residual, double-float (2 columns)",
                                 float(np.sum(16.0 * n * n * (fp + bp))))
    else:
        m["k_solve"] = (float(np.sum(8.0 * n * n * 3.0 * K)), simt_peak, "triangular solves (FP64)")
    # assembly: 708 nonzero Gaunt couplings x (complex x real) per off-diagonal block pair (p < q; the
    # block (q, p) is its transpose), once per forward unit
    m["k_assemble"] = (float(np.sum(S * (S - 1) / 2)) * 708 * 4.0, df_peak if mixed else fp64_peak,
                       "Gaunt sums, %s" % ("double-float FP32" if mixed else "FP64"))
    if sparse is not None:
        adj, trace = sparse
        what = "complex products over the nonzero entries of J and Abar (%s)" % ("double-float" if mixed else "FP64")
        m["k_adj_rhs"] = (adj * 8.0, df_peak if mixed else fp64_peak, what)
        m["k_kubo_partial"] = (trace * 8.0, df_peak if mixed else fp64_peak, what)
    return m


def kernel_rows(kt, models, hbm_gbs):
    """Per-kernel rows {kernel: achieved, peak, frac, ms}; template instances summed."""
    if not kt:
        return {}
    merged = {}
    for name, (ms, launches) in kt.items():
        base = name.split("<")[0]
        tot = merged.setdefault(base, [0.0, 0.0, {}])
        tot[0] += ms
        tot[1] += launches
        tot[2][name] = round(ms, 4)
    rows = {}
    for base, (ms, launches, inst) in merged.items():
        row = {"kernel": base, "ms_per_step": ms, "launches_per_step": launches, "instances": inst}
        if base in models:
            flops, peak, what = models[base][:3]
            ach = flops / (ms * 1e-3) / 1e12
            row.update({"bound": "tensor" if base == "k_gemm_tc" else "alu", "achieved": ach, "peak": peak,
                        "unit": "TFLOP/s", "frac": ach / peak, "work": what})
            if len(models[base]) > 3:  # also HBM-limited: keep whichever roof is closer
                gbs = models[base][3] / (ms * 1e-3) / 1e9
                row["flop_frac"] = ach / peak
                row["hbm_frac"] = gbs / hbm_gbs
                if gbs / hbm_gbs > row["frac"]:
                    row.update({"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s",
                                "frac": gbs / hbm_gbs})
        rows[base] = row
    return rows


def load_traffic():
    """DRAM bytes per launch from the committed ncu summary, valid only while the
    kernel sources it was taken from are unchanged (content hash)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        rec = json.load(f)
    h = hashlib.sha256()
    for src in sorted(rec.get("sources", [])):
        p = os.path.join(ROOT, src)
        if not os.path.exists(p):
            return {}
        with open(p, "rb") as g:
            h.update(g.read())
    if h.hexdigest() != rec.get("sha256"):
        return {}
    return rec.get("bytes_per_launch", {})


def kernel_times(B, fn, dev, steps):
    """Per-kernel device time over `steps` steps via the library's event timers (one launch stream)."""
    import torch
    B.kernel_timer_start()
    for _ in range(steps):
        fn()
    torch.cuda.synchronize(dev)
    return B.kernel_timer_stop(steps)


# ---------------------------------------------------------------- our path
def run_ours(args):
    import torch

    from paper_2311_12134_gb300 import binding as B
    from paper_2311_12134_gb300.conductivity import Problem, StepGraph, check_unit_status

    rank, world, local = dist_env()
    active = init_dist(world, "nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(B.LIB_PATH):
        if rank == 0:
            from paper_2311_12134_gb300 import build
            build.build()
        barrier(active)
    w = workload(args.workload)
    J = B.dipole_current(w.lmax, w.r_ll)
    grad_sigma = np.zeros((w.n_delta, 3, 3), dtype=np.complex128)
    grad_sigma[:, 0, 0] = 1.0  # d Re sigma_xx per delta
    gs_d = torch.as_tensor(grad_sigma).to(dev)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    fpk = file_peaks()
    gemm_pk = measure_gemm_peaks(dev)
    ws_bytes = (args.chunk_mb << 20) if args.chunk_mb else None

    def make(precision, conj_pairs=False):
        return Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume,
                       precision=precision, device=dev, keep_factors=True, workspace_bytes=ws_bytes,
                       conj_pairs=conj_pairs, check_status=False)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier(active)
        torch.cuda.synchronize(dev)
        l0 = B.launch_count()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(active)
        ms = ev0.elapsed_time(ev1) / steps
        return max_over_ranks(ms, active, device=dev), (B.launch_count() - l0) / steps

    main = make(args.precision)
    tuning, tuning_source = main.tuning, main.tuning_source  # autotuned shapes of this size class
    units = main.n_units
    main_export = main.liz.export()
    offsets = main_export["offsets"]
    sizes = np.diff(offsets)
    n_fwd = np.tile(w.K * sizes, len(w.z))  # one n per forward unit
    oracle_atoms = sample_atoms(w, offsets, 64)

    # eager launches (also the warm-up that builds plans and workspaces): Problem.step as users run it
    ms_eager, _ = timed(lambda: main.step(gs_d), args.steps, args.warmup)
    main.check()
    # the same step captured in one CUDA graph and replayed: the timed value
    sg = StepGraph(main, gs_d)
    sampler = ClockSampler(local)
    sampler.start()
    l0 = B.launch_count()
    ms, _ = timed(sg.replay, args.steps, args.warmup)
    clocks = sampler.stop()
    # graph replays do not pass through the library's launch counter: one eager step counts them
    l0 = B.launch_count()
    main.step(gs_d)
    torch.cuda.synchronize(dev)
    launches = B.launch_count() - l0
    status = main.unit_status.cpu().numpy()
    bw_status = main.bw_status.cpu().numpy()
    check_unit_status(status)
    check_unit_status(bw_status)
    value = world * units / (ms * 1e-3)
    # sigma time: the forward alone (a2..a8)
    sigma_ms, _ = timed(main.forward, args.steps, 1)
    main.check()
    sig_main = main.sigma_out.cpu().numpy()
    rho_main = main.rho.cpu().numpy()
    st_atoms_main = B.kubo_sigma_atoms(main.liz, w.lmax, main.species, main.J, main.tau, w.n_delta, w.volume,
                                       precision=args.precision).cpu().numpy()
    tau_rows_main = {m: main.tau[:, offsets[m]:offsets[m + 1]].cpu().numpy() for m in oracle_atoms}

    # per-kernel CUDA-event times, everything on one launch stream (library timers)
    kt = None
    if not args.no_kernel_timers:
        def one_stream_step():
            main.forward()
            main.backward(gs_d)
        kt = kernel_times(B, one_stream_step, dev, max(1, min(args.steps, 2)))

    # end to end through the public API: LIZ built from the positions, pinned H2D of the inputs,
    # forward + adjoint, D2H of sigma, rho, the gradient and the unit status words
    e2e = None if args.no_e2e else measure_e2e(w, J, main, args, dev, active, world)
    del sg
    del main
    torch.cuda.empty_cache()

    # conjugate-pair mode (tau(conj z) = conj tau(z): only the z systems are factored);
    # reported on its own, never counted as solves
    conj = None
    if not args.no_conj_leg:
        pc = make(args.precision, conj_pairs=True)
        sgc = StepGraph(pc, gs_d)
        msc, _ = timed(sgc.replay, args.steps, 1)
        pc.check()
        sc, _ = timed(pc.forward, args.steps, 1)
        conj = {"ms_per_step": msc, "sigma_ms": sc, "factored_units": units // 2, "tau_results": units,
                "sigma_rel_diff_vs_main_per_delta": rel_sigma(pc.sigma_out.cpu().numpy(), sig_main),
                "note": "LSMS_CONJ_PAIRS: z_- = conj z_+ and t^-1(z_-) = conj t^-1(z_+), so only the z_+ LIZ "
                        "matrices are factored; not counted in value"}
        del sgc, pc
        torch.cuda.empty_cache()

    fp64 = None
    st_atoms_64 = tau_rows_64 = None
    if not args.no_fp64_leg and args.precision != "fp64":
        p64 = make("fp64")
        ms64, _ = timed(lambda: p64.step(gs_d), max(1, args.fp64_steps), 1)
        p64.check()
        sig64 = p64.sigma_out.cpu().numpy()
        st_atoms_64 = B.kubo_sigma_atoms(p64.liz, w.lmax, p64.species, p64.J, p64.tau, w.n_delta, w.volume,
                                         precision="fp64").cpu().numpy()
        tau_rows_64 = {m: p64.tau[:, offsets[m]:offsets[m + 1]].cpu().numpy() for m in oracle_atoms}
        fp64 = {"value": world * units / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                "steps": max(1, args.fp64_steps), "warmup": 1, "timing": "eager Problem.step, CUDA events",
                "sigma_mixed_vs_fp64_rel_err_per_delta": rel_sigma(sig_main, sig64)}
        del p64
        torch.cuda.empty_cache()

    if rank != 0:
        return 0
    # refinement statistics of the mixed form: bits 8-15 sweeps, 16-23 probes
    fs = ((status >> 8) & 0xff).reshape(-1).astype(np.float64)
    fp = ((status >> 16) & 0xff).reshape(-1).astype(np.float64)
    bs = ((bw_status >> 8) & 0xff).reshape(-1).astype(np.float64)
    bp = ((bw_status >> 16) & 0xff).reshape(-1).astype(np.float64)

    # rooflines
    sm_mhz_max = (clocks or {}).get("sm_max_mhz") or fpk["sm_max_mhz"]
    fp32_ops = props.multi_processor_count * 128 * sm_mhz_max * 1e6
    tc_peak = gemm_pk["tf32_tflops"] / 3.0
    fp64_peak = gemm_pk["fp64_tflops"]
    F = path_flops(n_fwd)
    path = {"work": "sum over forward units of F(n) = (8/3) n^3 + 128 n^2 real flops (LU + 16-column solve); "
                    "refinement, split products and the adjoint not counted",
            "flops_per_step": F,
            args.precision: {"achieved": F / (ms * 1e-3) / 1e12,
                             "peak": tc_peak if args.precision == "mixed" else fp64_peak,
                             "peak_source": ("3xTF32: measured cuBLAS TF32 / 3" if args.precision == "mixed"
                                             else "measured cuBLAS FP64"), "unit": "TFLOP/s"}}
    path[args.precision]["frac"] = path[args.precision]["achieved"] / path[args.precision]["peak"]
    if fp64:
        path["fp64"] = {"achieved": F / (fp64["ms_per_step"] * 1e-3) / 1e12, "peak": fp64_peak,
                        "peak_source": "measured cuBLAS FP64", "unit": "TFLOP/s"}
        path["fp64"]["frac"] = path["fp64"]["achieved"] / fp64_peak
    ex = main_export
    sparse = sparse_product_cmacs(np.asarray(J), np.asarray(w.species), ex["offsets"], ex["site_atom"], grad_sigma,
                                  w.K)
    models = kernel_models(w.K, n_fwd, (fs, fp, bs, bp), w.n_delta, len(w.z), fp32_ops, fp64_peak, tc_peak,
                           fpk["hbm_gbs"], args.precision, sparse=sparse,
                           solve_cols=int((tuning or {}).get("solve_cols", 0)))
    rows = kernel_rows(kt, models, fpk["hbm_gbs"])
    roof = None
    modelled = [r for r in rows.values() if "frac" in r]
    if modelled:
        top = dict(max(modelled, key=lambda r: r["ms_per_step"]))
        top["traffic"] = load_traffic().get(top["kernel"])
        if top["bound"] == "alu":
            top["peak_source"] = (f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x {sm_mhz_max:.0f} "
                                  "MHz; double-float kernels at 44 lane ops per complex multiply-add")
        elif top["bound"] == "hbm":
            top["peak_source"] = fpk["source"]
        else:
            top["peak_source"] = "3xTF32 = measured cuBLAS TF32 / 3 (this run)"
        roof = {k: top[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic", "ms_per_step",
                                    "launches_per_step", "peak_source", "work") if k in top}

    cpu = acc = None
    if not args.no_cpu_baseline:
        v, u, dt, cores, res = time_oracle(w, oracle_atoms, budget_s=args.oracle_s)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{u} units ({u // len(w.z)} atoms: largest and smallest LIZ, then seeded random; x "
                         f"{len(w.z)} energies): tau column and row blocks by LAPACK + trace terms, {dt:.1f} s"}
        acc = {args.precision: accuracy(res, tau_rows_main, st_atoms_main)}
        if fp64:
            acc["fp64"] = accuracy(res, tau_rows_64, st_atoms_64)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "global_batch": units * world, "units_per_gpu": units,
                   "liz_sizes": {"min": int(sizes.min()), "max": int(sizes.max()), "mean": float(sizes.mean())},
                   "workspace_mib": args.chunk_mb or "all units", "precision": args.precision,
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (working set > 100 GB)",
                   "step": "Problem.step: forward (assembly, LU, tau, refinement, traces, sigma, rho) + adjoint "
                           "d Re sigma_xx / d t^-1 per delta, one CUDA graph",
                   "tuning": tuning, "tuning_source": tuning_source},
        "sigma_ms": sigma_ms, "ms_per_step_eager": ms_eager,
        "timing": "CUDA-graph replay of the whole step, CUDA events on the launch stream",
        "unit_status_clean": True,
        "fp64_fallback_units": int(np.sum((status & B.UNIT_FP64_FALLBACK) != 0)
                                   + np.sum((bw_status & B.UNIT_FP64_FALLBACK) != 0)),
        "ir_sweeps_mean": float(fs.mean()), "ir_sweeps_max": int(fs.max()),
        "ir_sweeps_adjoint_mean": float(bs.mean()),
        "ir_probes_mean": float(fp.mean()), "ir_probes_adjoint_mean": float(bp.mean()),
        "sigma_per_delta": {"sigma_xx": [complex(x).real for x in sig_main[:, 0, 0]],
                            "rho_xx": [float(x) for x in rho_main[:, 0, 0]]},
        "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
        "roofline_path": path, "kernels": rows, "peaks": {"file": fpk, "measured_here": gemm_pk,
                                                          "sms": props.multi_processor_count},
        "cpu_baseline": cpu, "fp64_form": fp64, "conj_pairs": conj, "accuracy_vs_oracle": acc,
    }
    if fp64:
        line["speedup_vs_fp64_form"] = value / fp64["value"]
    print(json.dumps(line), flush=True)
    return 0


def measure_e2e(w, J, p, args, dev, active, world):
    """Host-to-host through the public API on the bench's Problem: every step builds the LIZ from the
    positions, copies the inputs from pinned host memory, runs Problem.step (forward + adjoint) and
    reads back sigma, rho, the gradient and the unit status words."""
    import torch

    from paper_2311_12134_gb300 import binding as B
    from paper_2311_12134_gb300.conductivity import check_unit_status
    h_species = torch.as_tensor(w.species).pin_memory()
    h_tinv = torch.as_tensor(w.tinv).pin_memory()
    h_J = torch.as_tensor(J).pin_memory()
    gs = np.zeros((w.n_delta, 3, 3), dtype=np.complex128)
    gs[:, 0, 0] = 1.0
    h_gs = torch.as_tensor(gs).pin_memory()
    out_sig = torch.empty((w.n_delta, 3, 3), dtype=torch.complex128).pin_memory()
    out_rho = torch.empty((w.n_delta, 3, 3), dtype=torch.float64).pin_memory()
    out_g = torch.empty((len(w.z), w.n_atoms, w.K, w.K), dtype=torch.complex128).pin_memory()
    out_st = torch.empty((2, len(w.z), w.n_atoms), dtype=torch.int32).pin_memory()
    h2d = h_species.numel() * 4 + h_tinv.numel() * 16 + h_J.numel() * 16 + h_gs.numel() * 16 + w.pos.nbytes
    d2h = out_sig.numel() * 16 + out_rho.numel() * 8 + out_g.numel() * 16 + out_st.numel() * 4
    d_gs = torch.empty_like(h_gs, device=dev)

    def one():
        p.liz = B.build_liz(w.pos, w.lattice, w.r_liz)
        p.species.copy_(h_species, non_blocking=True)
        p.tinv.copy_(h_tinv, non_blocking=True)
        p.J.copy_(h_J, non_blocking=True)
        d_gs.copy_(h_gs, non_blocking=True)
        _, (g, _) = p.step(d_gs)
        out_sig.copy_(p.sigma_out, non_blocking=True)
        out_rho.copy_(p.rho, non_blocking=True)
        out_g.copy_(g, non_blocking=True)
        out_st[0].copy_(p.unit_status, non_blocking=True)
        out_st[1].copy_(p.bw_status, non_blocking=True)
        torch.cuda.synchronize(dev)
        check_unit_status(out_st.numpy())

    steps = max(1, min(args.steps, 3))
    for _ in range(max(1, min(args.warmup, 2))):
        one()
    barrier(active)
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    dt = (time.perf_counter() - t0) / steps
    dt = max_over_ranks(dt, active, device=dev)
    return {"value": world * p.n_units / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "steps": steps,
            "note": "public API per step: lsms_build_liz + pinned H2D of inputs + Problem.step (forward + adjoint) "
                    "+ D2H of sigma, rho, gradient and unit status, host clock"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
