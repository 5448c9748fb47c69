"""Shared helpers for the tests (no method arithmetic)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    from paper_2311_12134_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.lib()


def header_functions():
    names = []
    with open(os.path.join(ROOT, "include", "lsmskubo.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(lsms_\w+)\s*\(", text, flags=re.M):
        names.append(m.group(1))
    return sorted(set(names))


def rel_err_blocks(a, b):
    """max over leading index of ||a - b||_F / ||b||_F (norm-wise per block set)."""
    a = np.asarray(a)
    b = np.asarray(b)
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=tuple(range(1, a.ndim))))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=tuple(range(1, b.ndim))))
    return float(np.max(num / np.maximum(den, 1e-300)))


def unit_rel_errors(tau_a, tau_b, offsets):
    """Per (energy, atom) unit: ||tau_a^{.0} - tau_b^{.0}||_F / ||tau_b^{.0}||_F."""
    nE = tau_a.shape[0]
    N = len(offsets) - 1
    out = np.zeros((nE, N))
    for e in range(nE):
        for m in range(N):
            s = slice(offsets[m], offsets[m + 1])
            d = np.linalg.norm(tau_a[e, s] - tau_b[e, s])
            out[e, m] = d / np.linalg.norm(tau_b[e, s])
    return out
