"""Exact initial state mu0 = [y0, y'(0), ..., y^(q)(0)] (Eq. mu0, Section 2.1).

Test infrastructure only.  Taylor-mode recursion: write y(t) = sum_k c_k t^k; the ODE
y' = f(y) gives (k+1) c_{k+1} = [f(y)]_k, and the k-th coefficient of f(y) only depends on
c_0..c_k.  The derivatives are y^(k)(0) = k! c_k (raw derivatives, not Taylor coefficients).
"""
from __future__ import annotations

import math

import numpy as np

from .odes import f_series
from .taylor_series import Series


def taylor_coefficients(kind: int, params: np.ndarray, y0: np.ndarray, q: int) -> np.ndarray:
    """Coefficients c_0..c_q of every component, shape (d, q+1)."""
    y0 = np.asarray(y0, dtype=np.float64)
    d = y0.shape[0]
    C = np.zeros((d, q + 1))
    C[:, 0] = y0
    for k in range(q):
        Y = [Series(C[i]) for i in range(d)]
        F = f_series(kind, params, Y)
        for i in range(d):
            C[i, k + 1] = F[i].c[k] / (k + 1)
    return C


def initial_state(kind: int, params: np.ndarray, y0: np.ndarray, q: int) -> np.ndarray:
    """mu0 in the dimension-major layout: mu0[k (q+1) + i] = d^i y_k / dt^i (0)."""
    C = taylor_coefficients(kind, params, y0, q)
    d = C.shape[0]
    mu0 = np.zeros(d * (q + 1))
    for k in range(d):
        for i in range(q + 1):
            mu0[k * (q + 1) + i] = math.factorial(i) * C[k, i]
    return mu0
