"""Spherical Hankel functions for complex argument (oracle, test infrastructure).

The free-electron propagator of Eq. (tau-inverse) needs h_l(kappa R) with
complex kappa = sqrt(z), z = E_F +- i delta.  The paper names g but gives no
formula; this module evaluates the finite closed form

    h_l^(1)(x) = (-i)^{l+1} (e^{ix}/x) sum_{k=0}^{l} (l+k)! / (k! (l-k)!) (i/(2x))^k
    h_l^(2)(x) = ( i)^{l+1} (e^{-ix}/x) sum_{k=0}^{l} (l+k)! / (k! (l-k)!) (-i/(2x))^k

directly (no recurrence).  h^(2)_l(x) = conj(h^(1)_l(conj x)).
"""
from math import factorial

import numpy as np


def _poly(l, w):
    s = np.zeros_like(w)
    for k in range(l + 1):
        s = s + factorial(l + k) / (factorial(k) * factorial(l - k)) * w ** k
    return s


def h1(l, x):
    x = np.asarray(x, dtype=np.complex128)
    return (-1j) ** (l + 1) * np.exp(1j * x) / x * _poly(l, 1j / (2 * x))


def h2(l, x):
    x = np.asarray(x, dtype=np.complex128)
    return (1j) ** (l + 1) * np.exp(-1j * x) / x * _poly(l, -1j / (2 * x))
