"""Vector fields f(y, t) and Jacobians dF/dy of the test families, float64.

Test infrastructure only (see the package docstring).  Parameter layouts are the ones of the
``workloads`` module.  Each family also provides ``f_series``: f evaluated on truncated Taylor
series (used by ``taylor`` for the exact initial state, Eq. mu0).
"""
from __future__ import annotations

import numpy as np

import workloads as W
from .taylor_series import Series


def f(kind: int, params: np.ndarray, y: np.ndarray, t: float = 0.0) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    p = params
    if kind == W.LOGISTIC:
        r = p[0]
        return np.array([r * y[0] * (1.0 - y[0])])
    if kind == W.FITZHUGH_NAGUMO:
        a, b, c = p
        v, w = y
        return np.array([c * (v - v ** 3 / 3.0 + w), -(v - a + b * w) / c])
    if kind == W.LOTKA_VOLTERRA:
        al, be, ga, de = p
        x, z = y
        return np.array([al * x - be * x * z, de * x * z - ga * z])
    if kind == W.VAN_DER_POL:
        mu = p[0]
        return np.array([y[1], mu * ((1.0 - y[0] ** 2) * y[1] - y[0])])
    if kind == W.RIGID_BODY:
        return np.array([-2.0 * y[1] * y[2], 1.25 * y[0] * y[2], -0.5 * y[0] * y[1]])
    if kind == W.AFFINE:
        d = y.shape[0]
        L = p[: d * d].reshape(d, d)
        c = p[d * d: d * d + d]
        return L @ y + c
    if kind == W.LORENZ96:
        F = p[0]
        return (np.roll(y, -1) - np.roll(y, 2)) * np.roll(y, 1) - y + F
    raise ValueError(f"unknown ODE family {kind}")


def jac(kind: int, params: np.ndarray, y: np.ndarray, t: float = 0.0) -> np.ndarray:
    y = np.asarray(y, dtype=np.float64)
    p = params
    if kind == W.LOGISTIC:
        r = p[0]
        return np.array([[r * (1.0 - 2.0 * y[0])]])
    if kind == W.FITZHUGH_NAGUMO:
        a, b, c = p
        v, w = y
        return np.array([[c * (1.0 - v * v), c], [-1.0 / c, -b / c]])
    if kind == W.LOTKA_VOLTERRA:
        al, be, ga, de = p
        x, z = y
        return np.array([[al - be * z, -be * x], [de * z, de * x - ga]])
    if kind == W.VAN_DER_POL:
        mu = p[0]
        return np.array([[0.0, 1.0], [mu * (-2.0 * y[0] * y[1] - 1.0), mu * (1.0 - y[0] ** 2)]])
    if kind == W.RIGID_BODY:
        return np.array([[0.0, -2.0 * y[2], -2.0 * y[1]],
                         [1.25 * y[2], 0.0, 1.25 * y[0]],
                         [-0.5 * y[1], -0.5 * y[0], 0.0]])
    if kind == W.AFFINE:
        d = y.shape[0]
        return p[: d * d].reshape(d, d).copy()
    if kind == W.LORENZ96:
        d = y.shape[0]
        J = np.zeros((d, d))
        for i in range(d):
            ip1, im1, im2 = (i + 1) % d, (i - 1) % d, (i - 2) % d
            J[i, ip1] += y[im1]
            J[i, im2] -= y[im1]
            J[i, im1] += y[ip1] - y[im2]
            J[i, i] -= 1.0
        return J
    raise ValueError(f"unknown ODE family {kind}")


def f_series(kind: int, params: np.ndarray, Y: list) -> list:
    """f applied to a list of d truncated Taylor series (one per component)."""
    p = params
    if kind == W.LOGISTIC:
        r = p[0]
        y = Y[0]
        return [(y * (Series.const(1.0, y.order) - y)) * r]
    if kind == W.FITZHUGH_NAGUMO:
        a, b, c = p
        v, w = Y
        return [(v - v * v * v * (1.0 / 3.0) + w) * c,
                (v - Series.const(a, v.order) + w * b) * (-1.0 / c)]
    if kind == W.LOTKA_VOLTERRA:
        al, be, ga, de = p
        x, z = Y
        return [x * al - x * z * be, x * z * de - z * ga]
    if kind == W.VAN_DER_POL:
        mu = p[0]
        y1, y2 = Y
        one = Series.const(1.0, y1.order)
        return [y2, ((one - y1 * y1) * y2 - y1) * mu]
    if kind == W.RIGID_BODY:
        y1, y2, y3 = Y
        return [y2 * y3 * (-2.0), y1 * y3 * 1.25, y1 * y2 * (-0.5)]
    if kind == W.AFFINE:
        d = len(Y)
        L = p[: d * d].reshape(d, d)
        c = p[d * d: d * d + d]
        out = []
        for i in range(d):
            acc = Series.const(c[i], Y[0].order)
            for j in range(d):
                acc = acc + Y[j] * L[i, j]
            out.append(acc)
        return out
    if kind == W.LORENZ96:
        F = p[0]
        d = len(Y)
        return [(Y[(i + 1) % d] - Y[(i - 2) % d]) * Y[(i - 1) % d] - Y[i]
                + Series.const(F, Y[0].order) for i in range(d)]
    raise ValueError(f"unknown ODE family {kind}")
