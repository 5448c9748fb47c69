"""Autotuner of the library's tile and launch shapes.

The batched path has a few shapes whose best value depends on the LIZ matrix
size n and on how many (atom, energy) units a step holds (how much parallelism
the batched launches have):

* ``solve_cols``  right-hand-side columns per CTA of the mixed form's triangular
                  solves (8, 16 or 32): wider slices read the factors fewer
                  times, narrower slices run more independent block-step chains;
* ``solve_regs``  8 solve CTAs per SM with 64 registers (0), 4 with 128 (1) or
                  6 with 85 (2);
* ``solve_steps`` the solves by the library's choice (0), as one CTA chain per
                  unit and slice (1) or as one launch per block step over all
                  units, row updates on the FP32 pipes (2) or the tensor cores (3);
* ``streams``     concurrent parts of each chunk of units (2 or 4).

``tune`` times ``Problem.step`` (forward + adjoint) under every candidate with
CUDA events and keeps the fastest; the results live in a JSON table keyed by
GPU, precision, lmax and size class (largest n rounded up to a bucket, and the
unit count bucket).  ``Problem(..., tuning="auto")`` looks its class up in the
committed table (``tuning_gb300.json`` next to this file) and applies it
through ``lsms_set_option`` before each library call.

    python -m paper_2311_12134_gb300.autotune --workload bcc2000 [--workload fcc256 ...]

writes or updates the table (a GPU is needed).
"""
import argparse
import json
import os

import numpy as np

from . import binding as B

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning_gb300.json")

N_BUCKETS = (256, 512, 768, 1024, 1536, 2048, 3072, 4096, 8192, 16384)
U_BUCKETS = (1024, 8192, 65536, 1 << 30)

DEFAULTS = {"solve_cols": 0, "solve_regs": 0, "solve_steps": 0, "streams": 4}


def candidates():
    out = []
    for streams in (2, 4):
        out.append({"solve_cols": 0, "solve_regs": 0, "solve_steps": 0, "streams": streams})
        out.append({"solve_cols": 0, "solve_regs": 0, "solve_steps": 2, "streams": streams})
        out.append({"solve_cols": 0, "solve_regs": 0, "solve_steps": 3, "streams": streams})
        for cols, regs in ((0, 0), (0, 1), (0, 2), (8, 0), (8, 1), (8, 2), (16, 0), (16, 1), (16, 2), (32, 0)):
            out.append({"solve_cols": cols, "solve_regs": regs, "solve_steps": 1, "streams": streams})
    return out


def size_class(gpu_name, precision, lmax, n_max, n_units):
    nb = next((b for b in N_BUCKETS if n_max <= b), N_BUCKETS[-1])
    ub = next((b for b in U_BUCKETS if n_units <= b), U_BUCKETS[-1])
    return f"{gpu_name}|{precision}|lmax{lmax}|n<={nb}|units<={ub}"


def problem_class(problem):
    import torch
    name = torch.cuda.get_device_properties(problem.device).name
    K = problem.K
    return size_class(name, problem.precision, problem.lmax, K * problem.liz.max_sites, problem.n_units)


def load_table(path=TABLE):
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def lookup(problem, path=TABLE):
    """The tuned settings of the problem's size class, or None."""
    entry = load_table(path).get(problem_class(problem))
    return None if entry is None else dict(entry["settings"])


def apply(settings):
    """Set the library options of a settings dict (process-wide)."""
    for k, v in (settings or {}).items():
        B.set_option(k, v)


def tune(problem, grad_sigma, steps=2, warmup=1, cands=None):
    """Time Problem.step under each candidate; returns (best settings, {label: ms})."""
    import torch
    saved = {k: B.get_option(k) for k in DEFAULTS}
    saved_tuning = problem.tuning
    problem.tuning = None
    times = {}
    try:
        for c in cands or candidates():
            apply(c)
            for _ in range(warmup):
                problem.step(grad_sigma)
            torch.cuda.synchronize(problem.device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                problem.step(grad_sigma)
            e1.record()
            torch.cuda.synchronize(problem.device)
            problem.check()
            times[json.dumps(c, sort_keys=True)] = e0.elapsed_time(e1) / steps
    finally:
        apply(saved)
        problem.tuning = saved_tuning
    best = min(times, key=times.get)
    return json.loads(best), times


def main():
    import torch

    from . import workload as wl
    from .conductivity import Problem
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", action="append", required=True, choices=sorted(wl.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--workspace-mib", type=int, default=8192)
    args = ap.parse_args()
    table = load_table(args.out)
    for name in args.workload:
        w = wl.WORKLOADS[name]()
        J = B.dipole_current(w.lmax, w.r_ll)
        lz = B.build_liz(w.pos, w.lattice, w.r_liz)
        keep = B.lu_store_bytes(lz, w.lmax, len(w.z), B._prec(args.precision)) < (160 << 30)  # else recompute
        del lz
        p = Problem(w.pos, w.lattice, w.r_liz, w.lmax, w.species, w.tinv, w.z, J, w.volume,
                    precision=args.precision, keep_factors=keep, workspace_bytes=args.workspace_mib << 20,
                    check_status=False, tuning=None)
        gs = np.zeros((w.n_delta, 3, 3), dtype=np.complex128)
        gs[:, 0, 0] = 1.0
        gs = torch.as_tensor(gs).cuda()
        best, times = tune(p, gs, steps=args.steps)
        key = problem_class(p)
        table[key] = {"settings": best, "ms_per_step": times, "workload": name,
                      "n_max": p.K * p.liz.max_sites, "units": p.n_units,
                      "default_ms": times.get(json.dumps(DEFAULTS, sort_keys=True))}
        print(json.dumps({"class": key, "best": best, "ms": times[json.dumps(best, sort_keys=True)]}), flush=True)
        del p
        torch.cuda.empty_cache()
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
