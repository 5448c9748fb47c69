"""User-level API: the LSMS Kubo-Greenwood conductivity of one structure.

``Problem`` holds one structure's LIZ sets and device inputs and calls the C
ABI (through ``binding``) for tau blocks, sigma and the gradient.
``SigmaFn`` wraps forward and backward as a ``torch.autograd.Function`` of the
per-species inverse t-matrices.  ``conductivity`` is the host-to-host call:
NumPy inputs in, sigma and rho out.
"""
import numpy as np

from . import autotune
from . import binding as B


class UnitStatusError(RuntimeError):
    """Some (energy, atom) units carry a flag that makes their result invalid."""

    def __init__(self, status):
        self.status = status
        bad = (status & B.UNIT_INVALID) != 0
        flags = np.bitwise_or.reduce((status & B.UNIT_INVALID)[bad]) if bad.any() else 0
        super().__init__(f"{int(bad.sum())} of {status.size} units flagged invalid (flags 0x{int(flags):02x}); "
                         "see LSMS_UNIT_* in include/lsmskubo.h")


def check_unit_status(status):
    """Raise UnitStatusError if any unit status word (device or host array) has an invalid flag.
    LSMS_UNIT_FP64_FALLBACK alone is fine: that unit was re-solved in the FP64 form."""
    st = status.cpu().numpy() if hasattr(status, "cpu") else np.asarray(status)
    if np.any(st & B.UNIT_INVALID):
        raise UnitStatusError(st)
    return st


class Problem:
    """One structure on one CUDA device.

    pos [N,3], lattice [3,3] or None, r_liz, lmax, species [N] (host), tinv
    [n_species, 2 n_delta, K, K] (host or device complex128), z [2 n_delta]
    complex (E_F + i d, E_F - i d per delta), J [n_species, 4, 3, K, K] (host or
    device complex128), volume (bohr^3).  conj_pairs: the (z, conj z) pairs have
    conjugate t^-1, so only z is factored (tau(conj z) = conj tau(z)).
    check_status: forward() and backward() read the unit status words back and
    raise UnitStatusError if a unit's result is invalid (a host synchronisation;
    skipped while a CUDA graph is being captured).  Set it False for timing
    loops and check with check() afterwards.
    tuning: "auto" applies the autotuned tile and launch shapes of the problem's
    size class (autotune.lookup; the defaults when the class is not in the
    table), a dict applies those options, None leaves the options alone.  They
    are set through lsms_set_option before each library call.
    """

    def __init__(self, pos, lattice, r_liz, lmax, species, tinv, z, J, volume, precision="fp64", device="cuda",
                 keep_factors=True, workspace_bytes=None, conj_pairs=False, check_status=True, tuning="auto"):
        import torch
        self.check_status = bool(check_status)
        self.generation = 0  # number of tau solves so far (the factors in lu_store belong to the latest)
        self.lmax = int(lmax)
        self.K = (self.lmax + 1) ** 2
        self.liz = B.build_liz(pos, lattice, r_liz)
        self.z = np.ascontiguousarray(z, dtype=np.complex128)
        if self.z.shape[0] % 2:
            raise ValueError("energies must come in (+, -) pairs")
        self.n_delta = self.z.shape[0] // 2
        self.volume = float(volume)
        self.precision = precision
        self.conj_pairs = bool(conj_pairs)  # energies in (z, conj z) pairs: factor z only
        self.device = torch.device(device)
        self.species = torch.as_tensor(np.ascontiguousarray(species, dtype=np.int32)).to(self.device)
        self.tinv = torch.as_tensor(tinv).to(device=self.device, dtype=torch.complex128).contiguous()
        self.J = torch.as_tensor(J).to(device=self.device, dtype=torch.complex128).contiguous()
        nE = self.z.shape[0]
        self._ws_flags = B.LSMS_WS_STORE if keep_factors else 0
        prec = B._prec(precision, self.conj_pairs)
        mn, al = B.tau_workspace_bytes(self.liz, self.lmax, nE, prec | self._ws_flags)
        ws = al if workspace_bytes is None else min(al, max(mn, int(workspace_bytes)))
        self.workspace = torch.empty(ws, dtype=torch.uint8, device=self.device)
        self.lu_store = None
        if keep_factors:
            self.lu_store = torch.empty(B.lu_store_bytes(self.liz, self.lmax, nE, prec), dtype=torch.uint8,
                                        device=self.device)
        self.tau = torch.empty((nE, self.liz.total_sites, self.K, self.K), dtype=torch.complex128,
                               device=self.device)
        self.unit_status = torch.empty((nE, self.liz.n_atoms), dtype=torch.int32, device=self.device)
        self.sigma_out = torch.empty((self.n_delta, 3, 3), dtype=torch.complex128, device=self.device)
        self.sigma_tilde = torch.empty((self.n_delta, 4, 3, 3), dtype=torch.complex128, device=self.device)
        self.rho = torch.empty((self.n_delta, 3, 3), dtype=torch.float64, device=self.device)
        self.bw_status = torch.empty((nE, self.liz.n_atoms), dtype=torch.int32, device=self.device)
        self._bw_ws = None
        self._side = None  # side stream of step()
        if tuning == "auto":
            found = autotune.lookup(self)
            self.tuning = dict(autotune.DEFAULTS) if found is None else found
            self.tuning_source = "default" if found is None else "table"
        else:
            self.tuning = None if tuning is None else dict(tuning)
            self.tuning_source = "given" if tuning is not None else "none"

    @property
    def n_units(self):
        return self.liz.n_atoms * self.z.shape[0]

    def solve_tau(self, tinv=None, stream=None):
        autotune.apply(self.tuning)
        t = self.tinv if tinv is None else tinv
        B.tau_blocks(self.liz, self.lmax, self.species, t, self.z, self.precision, tau=self.tau,
                     unit_status=self.unit_status, workspace=self.workspace, lu_store=self.lu_store, stream=stream,
                     conj_pairs=self.conj_pairs)
        self.generation += 1
        self._maybe_check(self.unit_status)
        return self.tau

    def _maybe_check(self, status):
        import torch
        if self.check_status and not torch.cuda.is_current_stream_capturing():
            check_unit_status(status)

    def check(self):
        """Raise UnitStatusError if the last forward or backward left an invalid unit."""
        check_unit_status(self.unit_status)
        if self._bw_ws is not None:
            check_unit_status(self.bw_status)

    def stats(self, log=None):
        """Per-call statistics of the last forward (and backward) on the device
        (lsms_unit_stats): flag counts, FP64 re-solves, refinement sweeps and
        probes, the largest pivot growth.  With ``log`` (a file object) also
        written there as one JSON line."""
        import json
        out = {"forward": B.unit_stats(self.unit_status)}
        if self._bw_ws is not None:
            out["backward"] = B.unit_stats(self.bw_status)
        out["units"] = self.n_units
        if log is not None:
            log.write(json.dumps(out) + "\n")
        return out

    def sigma(self, stream=None):
        B.kubo_sigma(self.liz, self.lmax, self.species, self.J, self.tau, self.n_delta, self.volume,
                     sigma=self.sigma_out, sigma_tilde=self.sigma_tilde, rho=self.rho, stream=stream,
                     precision=self.precision, conj_pairs=self.conj_pairs)
        return self.sigma_out

    def forward(self, tinv=None, stream=None):
        self.solve_tau(tinv, stream)
        return self.sigma(stream)

    def step(self, grad_sigma, tinv=None):
        """forward() and backward() in one call on the current stream, with sigma's
        traces overlapping the adjoint solves.  Returns (sigma, (grad_tinv,
        grad_tinv_species))."""
        return _step(self, grad_sigma, tinv)

    def backward(self, grad_sigma, tinv=None, stream=None):
        """PyTorch gradients of Re sum(conj(grad_sigma) sigma): per site [nE, N, K, K] and per species."""
        import torch
        if self._bw_ws is None:
            mn, al = B.backward_workspace_bytes(self.liz, self.lmax, self.z.shape[0],
                                                B._prec(self.precision, self.conj_pairs) | self._ws_flags)
            self._bw_ws = torch.empty(min(al, max(mn, self.workspace.numel())), dtype=torch.uint8,
                                      device=self.device)
        autotune.apply(self.tuning)
        t = self.tinv if tinv is None else tinv
        out = B.kubo_sigma_backward(self.liz, self.lmax, self.species, t, self.z, self.J, self.tau, self.volume,
                                    grad_sigma.contiguous(), self.precision, lu_store=self.lu_store,
                                    unit_status=self.bw_status, workspace=self._bw_ws, stream=stream,
                                    conj_pairs=self.conj_pairs)
        self._maybe_check(self.bw_status)
        return out

    def backward_detached(self, grad_sigma, tinv):
        """The gradient for an earlier forward whose tau and factors have since been overwritten:
        tau is solved again for `tinv` into private buffers and the factors are recomputed (no store)."""
        import torch
        autotune.apply(self.tuning)
        nE = self.z.shape[0]
        prec = B._prec(self.precision, self.conj_pairs)
        mn, al = B.tau_workspace_bytes(self.liz, self.lmax, nE, prec)
        ws = torch.empty(min(al, max(mn, self.workspace.numel())), dtype=torch.uint8, device=self.device)
        tau, st = B.tau_blocks(self.liz, self.lmax, self.species, tinv, self.z, self.precision, workspace=ws,
                               conj_pairs=self.conj_pairs)
        self._maybe_check(st)
        del ws
        mn, al = B.backward_workspace_bytes(self.liz, self.lmax, nE, prec)
        bws = torch.empty(min(al, max(mn, self.workspace.numel())), dtype=torch.uint8, device=self.device)
        bst = torch.empty_like(self.bw_status)
        out = B.kubo_sigma_backward(self.liz, self.lmax, self.species, tinv, self.z, self.J, tau, self.volume,
                                    grad_sigma.contiguous(), self.precision, lu_store=None, unit_status=bst,
                                    workspace=bws, conj_pairs=self.conj_pairs)
        self._maybe_check(bst)
        return out


def _step(problem, grad_sigma, tinv=None):
    """Forward (tau, sigma) and adjoint in one call: sigma's traces run on a side
    stream while the adjoint solves run on the current one (the adjoint reads tau
    and grad_sigma, not sigma), joined before returning.  Same results as
    forward() then backward()."""
    import torch
    cur = torch.cuda.current_stream(problem.device)
    problem.solve_tau(tinv)
    if problem._side is None:
        problem._side = torch.cuda.Stream(device=problem.device)
    side = problem._side
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        problem.sigma()
    grads = problem.backward(grad_sigma, tinv)
    cur.wait_stream(side)
    return problem.sigma_out, grads


def _sigma_fn():
    import torch

    class SigmaFn(torch.autograd.Function):
        """sigma [n_delta, 3, 3] as a differentiable function of the per-species tinv."""

        @staticmethod
        def forward(ctx, tinv, problem):
            t = tinv.detach().contiguous()
            s = problem.forward(t)
            ctx.problem = problem
            ctx.generation = problem.generation  # the factors and tau of this forward
            ctx.save_for_backward(t)
            return s.clone()

        @staticmethod
        def backward(ctx, grad_sigma):
            (tinv,) = ctx.saved_tensors
            p = ctx.problem
            gs = grad_sigma.to(torch.complex128).contiguous()
            if p.generation == ctx.generation:
                _, g_species = p.backward(gs, tinv)
            else:  # a later forward overwrote this one's tau and factors: solve again for the saved tinv
                _, g_species = p.backward_detached(gs, tinv)
            return g_species.clone(), None

    return SigmaFn


SigmaFn = None


def sigma_autograd(tinv, problem):
    global SigmaFn
    if SigmaFn is None:
        SigmaFn = _sigma_fn()
    return SigmaFn.apply(tinv, problem)


def conductivity(pos, lattice, r_liz, lmax, species, tinv, z, J, volume, precision="fp64"):
    """Host-to-host conductivity: returns (sigma [n_delta,3,3] complex128, rho [n_delta,3,3]) as NumPy."""
    p = Problem(pos, lattice, r_liz, lmax, species, tinv, z, J, volume, precision=precision, keep_factors=False)
    p.forward()  # raises UnitStatusError if a unit's result is invalid
    return p.sigma_out.cpu().numpy(), p.rho.cpu().numpy()


class StepGraph:
    """The whole step (tau blocks, sigma, adjoint) of a Problem captured in one
    CUDA graph.  The library's first calls on the problem (device tables, work
    plans, workspaces) happen in a warm-up step before capture; every later call
    enqueues kernels, memsets and stream-ordered scratch only, so the captured
    graph replays the same work on the same buffers.  Inputs are read from the
    problem's tensors at replay time (update them in place to change them)."""

    def __init__(self, problem, grad_sigma, with_backward=True):
        import torch
        self.problem = problem
        self.grad_sigma = grad_sigma.contiguous()
        self.with_backward = with_backward
        if with_backward:
            problem.step(self.grad_sigma)
        else:
            problem.forward()
        torch.cuda.synchronize(problem.device)
        self.graph = torch.cuda.CUDAGraph()
        stream = torch.cuda.Stream(device=problem.device)
        stream.wait_stream(torch.cuda.current_stream(problem.device))
        with torch.cuda.graph(self.graph, stream=stream):
            if with_backward:
                _, self.grads = problem.step(self.grad_sigma)
            else:
                problem.forward()
        torch.cuda.synchronize(problem.device)

    def replay(self):
        self.graph.replay()
