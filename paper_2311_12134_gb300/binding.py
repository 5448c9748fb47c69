"""ctypes binding of liblsmskubo (argument marshalling only).

Every function here checks and converts arguments and calls the C ABI of
``include/lsmskubo.h`` with raw pointers: device buffers are torch CUDA
tensors (PyTorch supplies memory and streams), host buffers are NumPy arrays.
No arithmetic of the method happens in Python.  The library is loaded on
first use; a missing library raises at once (there is no fallback path).
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblsmskubo.so")
# LSMS_DEBUG_BOUNDS=1 in the environment: the build with device-side index checks
LIB_DEBUG_PATH = os.path.join(_HERE, "_lib", "liblsmskubo_debug.so")


def lib_path():
    """The library file this process loads (the debug-bounds build if LSMS_DEBUG_BOUNDS=1)."""
    return LIB_DEBUG_PATH if os.environ.get("LSMS_DEBUG_BOUNDS") == "1" else LIB_PATH

LSMS_FP64 = 0
LSMS_MIXED = 1
LSMS_OK = 0
LSMS_ERR_ARG = -1  # status codes of the C ABI (include/lsmskubo.h)
PRECISIONS = {"fp64": LSMS_FP64, "mixed": LSMS_MIXED}

UNIT_ZERO_PIVOT = 1
UNIT_NOCONV = 2
UNIT_NONFINITE = 4
UNIT_BAD_INPUT = 8
UNIT_TINV_ASYM = 16
UNIT_GROWTH = 32
UNIT_FP64_FALLBACK = 64
UNIT_TIMEOUT = 128
# every flag but the fallback marker means the unit's result is not valid
UNIT_INVALID = 0xff & ~UNIT_FP64_FALLBACK

_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double

# name -> (restype, argtypes)
SIGNATURES = {
    "lsms_build_liz": (_I, [_P, _I, _P, _D, ctypes.POINTER(_P)]),
    "lsms_liz_sizes": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I64), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "lsms_liz_export": (_I, [_P, _P, _P, _P, _P]),
    "lsms_liz_destroy": (None, [_P]),
    "lsms_dipole_current": (_I, [_I, _P, _I, _P]),
    "lsms_gaunt_table": (_I, [_I, _P]),
    "lsms_tau_workspace_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "lsms_backward_workspace_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    "lsms_lu_store_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(_SZ)]),
    "lsms_tau_blocks": (_I, [_P, _I, _P, _I, _P, _P, _I, _I, _P, _P, _P, _SZ, _P, _SZ, _P]),
    "lsms_kubo_sigma": (_I, [_P, _I, _P, _I, _P, _I64, _P, _I, _D, _I, _P, _P, _P, _P]),
    "lsms_kubo_sigma_noalloc": (_I, [_P, _I, _P, _I, _P, _I64, _P, _I, _D, _I, _P, _P, _P, _P]),
    "lsms_kubo_sigma_atoms": (_I, [_P, _I, _P, _I, _P, _I64, _P, _I, _D, _I, _P, _P]),
    "lsms_set_option": (_I, [ctypes.c_char_p, _D]),
    "lsms_get_option": (_I, [ctypes.c_char_p, ctypes.POINTER(_D)]),
    "lsms_kubo_sigma_backward": (_I, [_P, _I, _P, _I, _P, _P, _I, _I, _P, _I64, _P, _D, _P, _P, _SZ, _P, _P,
                                      _P, _P, _SZ, _P]),
    "lsms_unit_stats": (_I, [_P, _I64, _P, _P]),
    "lsms_last_error": (ctypes.c_char_p, []),
    "lsms_version": (_I, []),
    "lsms_launch_count": (ctypes.c_longlong, []),
    "lsms_kernel_timer_enable": (_I, [_I]),
    "lsms_kernel_timer_report": (_I, [ctypes.c_char_p, _SZ]),
}


class LsmsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblsmskubo error {code}: {msg}")
        self.code = code


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run python -m paper_2311_12134_gb300.build"
                               + (" --debug-bounds" if path == LIB_DEBUG_PATH else ""))
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise LsmsError(rc, lib().lsms_last_error().decode())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_P)


def _dev(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return _P(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


def _opt(t, dtype, shape, name):
    return _P(0) if t is None else _dev(t, dtype, shape, name)


class Liz:
    """LIZ neighbour sets (lsms_build_liz).  Host arrays exported on demand."""

    def __init__(self, pos, lattice, r_liz):
        pos_h, pos_p = _host(pos, np.float64)
        if pos_h.ndim != 2 or pos_h.shape[1] != 3:
            raise ValueError("pos must be [n_atoms, 3]")
        lat_p = _P(0)
        self._lat = None
        if lattice is not None:
            self._lat, lat_p = _host(lattice, np.float64)
            if self._lat.shape != (3, 3):
                raise ValueError("lattice must be 3x3")
        h = _P()
        _check(lib().lsms_build_liz(pos_p, pos_h.shape[0], lat_p, float(r_liz), ctypes.byref(h)))
        self._h = h
        n, S, smax, smin = _I(), _I64(), _I(), _I()
        _check(lib().lsms_liz_sizes(h, ctypes.byref(n), ctypes.byref(S), ctypes.byref(smax), ctypes.byref(smin)))
        self.n_atoms, self.total_sites, self.max_sites, self.min_sites = n.value, S.value, smax.value, smin.value
        self._export = None

    @property
    def handle(self):
        return self._h

    def export(self):
        if self._export is None:
            off = np.zeros(self.n_atoms + 1, dtype=np.int64)
            sa = np.zeros(self.total_sites, dtype=np.int32)
            im = np.zeros((self.total_sites, 3), dtype=np.int32)
            dp = np.zeros((self.total_sites, 3), dtype=np.float64)
            _check(lib().lsms_liz_export(self._h, off.ctypes.data_as(_P), sa.ctypes.data_as(_P),
                                         im.ctypes.data_as(_P), dp.ctypes.data_as(_P)))
            self._export = dict(offsets=off, site_atom=sa, image=im, disp=dp)
        return self._export

    @property
    def sizes(self):
        return np.diff(self.export()["offsets"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.lsms_liz_destroy(h)
            self._h = None


def build_liz(pos, lattice, r_liz):
    return Liz(pos, lattice, r_liz)


def gaunt_table(lmax):
    K, K3 = (lmax + 1) ** 2, (2 * lmax + 1) ** 2
    out = np.zeros((K, K, K3), dtype=np.float64)
    _check(lib().lsms_gaunt_table(lmax, out.ctypes.data_as(_P)))
    return out


def dipole_current(lmax, r_ll):
    """Host J [n_species, 4, 3, K, K] complex128 from r_ll [n_species, 4, lmax+1, lmax+1]."""
    r, rp = _host(r_ll, np.complex128)
    if r.ndim != 4 or r.shape[1:] != (4, lmax + 1, lmax + 1):
        raise ValueError("r_ll must be [n_species, 4, lmax+1, lmax+1]")
    K = (lmax + 1) ** 2
    J = np.zeros((r.shape[0], 4, 3, K, K), dtype=np.complex128)
    _check(lib().lsms_dipole_current(lmax, rp, r.shape[0], J.ctypes.data_as(_P)))
    return J


def tau_workspace_bytes(liz, lmax, n_energy, precision):
    a, b = _SZ(), _SZ()
    _check(lib().lsms_tau_workspace_bytes(liz.handle, lmax, n_energy, precision, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def backward_workspace_bytes(liz, lmax, n_energy, precision):
    a, b = _SZ(), _SZ()
    _check(lib().lsms_backward_workspace_bytes(liz.handle, lmax, n_energy, precision, ctypes.byref(a),
                                               ctypes.byref(b)))
    return a.value, b.value


def lu_store_bytes(liz, lmax, n_energy, precision):
    a = _SZ()
    _check(lib().lsms_lu_store_bytes(liz.handle, lmax, n_energy, precision, ctypes.byref(a)))
    return a.value


LSMS_CONJ_PAIRS = 0x100
LSMS_WS_STORE = 0x200  # workspace sizes for a call given an lu_store


def _prec(precision, conj_pairs=False):
    """Precision argument of the C ABI: "fp64"/"mixed" (or the enum), | LSMS_CONJ_PAIRS."""
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return p | (LSMS_CONJ_PAIRS if conj_pairs else 0)


def tau_blocks(liz, lmax, species, tinv, z, precision="fp64", tau=None, unit_status=None, workspace=None,
               lu_store=None, stream=None, conj_pairs=False):
    """lsms_tau_blocks.  species int32 [N] (cuda), tinv complex128 [n_species, n_energy, K, K] (cuda),
    z host complex [n_energy].  Returns (tau [n_energy, S_total, K, K], unit_status [n_energy, N]).
    conj_pairs: LSMS_CONJ_PAIRS (energies in (z, conj z) pairs; only z is factored)."""
    import torch
    K = (lmax + 1) ** 2
    zh, zp = _host(z, np.complex128)
    nE = zh.shape[0]
    n_species = tinv.shape[0]
    dev = tinv.device
    if tau is None:
        tau = torch.empty((nE, liz.total_sites, K, K), dtype=torch.complex128, device=dev)
    if unit_status is None:
        unit_status = torch.empty((nE, liz.n_atoms), dtype=torch.int32, device=dev)
    ws_p, ws_n = (_P(0), 0) if workspace is None else (_dev(workspace, torch.uint8, None, "workspace"),
                                                         workspace.numel())
    st_p, st_n = (_P(0), 0) if lu_store is None else (_dev(lu_store, torch.uint8, None, "lu_store"), lu_store.numel())
    _check(lib().lsms_tau_blocks(liz.handle, lmax, _dev(species, torch.int32, (liz.n_atoms,), "species"), n_species,
                                 _dev(tinv, torch.complex128, (n_species, nE, K, K), "tinv"), zp, nE,
                                 _prec(precision, conj_pairs),
                                 _dev(tau, torch.complex128, (nE, liz.total_sites, K, K), "tau"),
                                 _dev(unit_status, torch.int32, (nE, liz.n_atoms), "unit_status"), ws_p, ws_n, st_p,
                                 st_n, _stream(stream)))
    return tau, unit_status


def kubo_sigma(liz, lmax, species, J, tau, n_delta, volume, J_delta_stride=0, sigma=None, sigma_tilde=None,
               rho=None, stream=None, precision="fp64", conj_pairs=False):
    """lsms_kubo_sigma.  Returns (sigma [n_delta,3,3] c128, sigma_tilde [n_delta,4,3,3] c128, rho [n_delta,3,3] f64).
    conj_pairs: tau holds conjugate pairs; the (-,+) and (-,-) traces are conjugates when J allows."""
    import torch
    K = (lmax + 1) ** 2
    dev = tau.device
    if sigma is None:
        sigma = torch.empty((n_delta, 3, 3), dtype=torch.complex128, device=dev)
    if sigma_tilde is None:
        sigma_tilde = torch.empty((n_delta, 4, 3, 3), dtype=torch.complex128, device=dev)
    if rho is None:
        rho = torch.empty((n_delta, 3, 3), dtype=torch.float64, device=dev)
    n_species = J.shape[-5]
    _check(lib().lsms_kubo_sigma(liz.handle, lmax, _dev(species, torch.int32, (liz.n_atoms,), "species"), n_species,
                                 _dev(J, torch.complex128, None, "J"), int(J_delta_stride),
                                 _dev(tau, torch.complex128, (2 * n_delta, liz.total_sites, K, K), "tau"), n_delta,
                                 float(volume), _prec(precision, conj_pairs),
                                 _dev(sigma_tilde, torch.complex128, (n_delta, 4, 3, 3), "sigma_tilde"),
                                 _dev(sigma, torch.complex128, (n_delta, 3, 3), "sigma"),
                                 _dev(rho, torch.float64, (n_delta, 3, 3), "rho"), _stream(stream)))
    return sigma, sigma_tilde, rho


def kubo_sigma_atoms(liz, lmax, species, J, tau, n_delta, volume, J_delta_stride=0, out=None, stream=None,
                     precision="fp64"):
    """lsms_kubo_sigma_atoms: the per-centre-atom terms of sigma~, [n_delta, 4, n_atoms, 3, 3] complex128
    (their sum over atoms is sigma~)."""
    import torch
    K = (lmax + 1) ** 2
    dev = tau.device
    shape = (n_delta, 4, liz.n_atoms, 3, 3)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex128, device=dev)
    n_species = J.shape[-5]
    _check(lib().lsms_kubo_sigma_atoms(
        liz.handle, lmax, _dev(species, torch.int32, (liz.n_atoms,), "species"), n_species,
        _dev(J, torch.complex128, None, "J"), int(J_delta_stride),
        _dev(tau, torch.complex128, (2 * n_delta, liz.total_sites, K, K), "tau"), n_delta, float(volume),
        _prec(precision), _dev(out, torch.complex128, shape, "out"), _stream(stream)))
    return out


STATS_FIELDS = ("units", "zero_pivot", "noconv", "nonfinite", "bad_input", "tinv_asym", "growth",
                "fp64_fallback", "timeout", "invalid", "sweeps_sum", "sweeps_max", "probes_sum", "probes_max",
                "growth_code_max")


def unit_stats(unit_status, stream=None):
    """lsms_unit_stats: the status words (device int32 tensor) reduced on the device; returns a dict
    (flag counts, refinement sweeps and probes, the largest pivot-growth code and, decoded from it,
    growth_max ~ 2^(code - 64), None when none was recorded)."""
    import torch
    st = unit_status.contiguous()
    out = torch.empty(len(STATS_FIELDS), dtype=torch.int64, device=st.device)
    _check(lib().lsms_unit_stats(_dev(st, torch.int32, name="unit_status"), st.numel(),
                                 _dev(out, torch.int64, name="stats"), _stream(stream)))
    vals = out.cpu().tolist()
    d = dict(zip(STATS_FIELDS, vals))
    d["growth_max"] = None if d["growth_code_max"] == 0 else 2.0 ** (d["growth_code_max"] - 64)
    return d


def set_option(name, value):
    """lsms_set_option (process-wide): growth_limit, fallback_slots, ir_max_sweeps, streams, residual_tc,
    solve_cols, solve_regs, solve_steps, nvtx."""
    _check(lib().lsms_set_option(name.encode(), float(value)))


def get_option(name):
    v = _D()
    _check(lib().lsms_get_option(name.encode(), ctypes.byref(v)))
    return v.value


def kubo_sigma_noalloc(liz, lmax, species, J, tau, n_delta, volume, J_delta_stride=0, sigma=None, sigma_tilde=None,
                       rho=None, stream=None, precision="fp64"):
    """lsms_kubo_sigma_noalloc: as kubo_sigma, but the library allocates nothing during the
    call (its scratch is a fixed 16 MiB device array; see include/lsmskubo.h).  The output
    tensors are allocated here by PyTorch unless passed in."""
    import torch
    K = (lmax + 1) ** 2
    dev = tau.device
    if sigma is None:
        sigma = torch.empty((n_delta, 3, 3), dtype=torch.complex128, device=dev)
    if sigma_tilde is None:
        sigma_tilde = torch.empty((n_delta, 4, 3, 3), dtype=torch.complex128, device=dev)
    if rho is None:
        rho = torch.empty((n_delta, 3, 3), dtype=torch.float64, device=dev)
    n_species = J.shape[-5]
    _check(lib().lsms_kubo_sigma_noalloc(
        liz.handle, lmax, _dev(species, torch.int32, (liz.n_atoms,), "species"), n_species,
        _dev(J, torch.complex128, None, "J"), int(J_delta_stride),
        _dev(tau, torch.complex128, (2 * n_delta, liz.total_sites, K, K), "tau"), n_delta, float(volume),
        _prec(precision), _dev(sigma_tilde, torch.complex128, (n_delta, 4, 3, 3), "sigma_tilde"),
        _dev(sigma, torch.complex128, (n_delta, 3, 3), "sigma"), _dev(rho, torch.float64, (n_delta, 3, 3), "rho"),
        _stream(stream)))
    return sigma, sigma_tilde, rho


def kubo_sigma_backward(liz, lmax, species, tinv, z, J, tau, volume, grad_sigma, precision="fp64", lu_store=None,
                        J_delta_stride=0, grad_tinv=None, grad_tinv_species=None, unit_status=None, workspace=None,
                        stream=None, conj_pairs=False):
    """lsms_kubo_sigma_backward.  Returns (grad_tinv [n_energy, N, K, K], grad_tinv_species [n_species, n_energy, K, K])."""
    import torch
    K = (lmax + 1) ** 2
    zh, zp = _host(z, np.complex128)
    nE = zh.shape[0]
    n_species = tinv.shape[0]
    dev = tinv.device
    if grad_tinv is None:
        grad_tinv = torch.empty((nE, liz.n_atoms, K, K), dtype=torch.complex128, device=dev)
    if grad_tinv_species is None:
        grad_tinv_species = torch.empty((n_species, nE, K, K), dtype=torch.complex128, device=dev)
    ws_p, ws_n = (_P(0), 0) if workspace is None else (_dev(workspace, torch.uint8, None, "workspace"),
                                                         workspace.numel())
    st_p, st_n = (_P(0), 0) if lu_store is None else (_dev(lu_store, torch.uint8, None, "lu_store"), lu_store.numel())
    _check(lib().lsms_kubo_sigma_backward(
        liz.handle, lmax, _dev(species, torch.int32, (liz.n_atoms,), "species"), n_species,
        _dev(tinv, torch.complex128, (n_species, nE, K, K), "tinv"), zp, nE, _prec(precision, conj_pairs),
        _dev(J, torch.complex128, None, "J"), int(J_delta_stride),
        _dev(tau, torch.complex128, (nE, liz.total_sites, K, K), "tau"), float(volume),
        _dev(grad_sigma, torch.complex128, (nE // 2, 3, 3), "grad_sigma"), st_p, st_n,
        _dev(grad_tinv, torch.complex128, (nE, liz.n_atoms, K, K), "grad_tinv"),
        _dev(grad_tinv_species, torch.complex128, (n_species, nE, K, K), "grad_tinv_species"),
        _opt(unit_status, torch.int32, (nE, liz.n_atoms), "unit_status"), ws_p, ws_n, _stream(stream)))
    return grad_tinv, grad_tinv_species


def kernel_timer_start():
    _check(lib().lsms_kernel_timer_enable(1))


def kernel_timer_stop(steps=1):
    """Call after synchronizing.  Returns {kernel: (ms per step, launches per step)}."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().lsms_kernel_timer_report(buf, len(buf)))
    _check(lib().lsms_kernel_timer_enable(0))
    out = {}
    for line in buf.value.decode().splitlines():
        name, ms, cnt = line.split("\t")
        out[name.strip("()")] = (float(ms) / steps, int(cnt) / steps)
    return out


def launch_count():
    return int(lib().lsms_launch_count())


def version():
    return int(lib().lsms_version())
