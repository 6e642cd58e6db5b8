"""Pins of the exact initial state mu0 = [y0, y'(0), ..., y^(q)(0)] (Eq. mu0).

Independent routes: the logistic derivatives in closed form, symbolic Lie derivatives
y^(k+1) = (d y^(k) / d y) f computed by sympy for every family, and the affine closed form
y^(k+1)(0) = L y^(k)(0) (+ c for k = 0).
"""
import math

import numpy as np
import pytest
import sympy as sp

import workloads as W
from oracle.taylor import initial_state


def test_logistic_closed_form():
    r, y = 3.0, 0.01
    mu = initial_state(W.LOGISTIC, np.array([r]), np.array([y]), 3)
    y1 = r * y * (1 - y)
    y2 = r * (1 - 2 * y) * y1
    y3 = r * (1 - 2 * y) * y2 - 2 * r * y1 ** 2
    np.testing.assert_allclose(mu, [y, y1, y2, y3], rtol=1e-14)


def _symbolic_f(kind, params, ys):
    p = [sp.Rational(float(x)) for x in params]
    if kind == W.LOGISTIC:
        return [p[0] * ys[0] * (1 - ys[0])]
    if kind == W.FITZHUGH_NAGUMO:
        a, b, c = p
        v, w = ys
        return [c * (v - v ** 3 / 3 + w), -(v - a + b * w) / c]
    if kind == W.LOTKA_VOLTERRA:
        al, be, ga, de = p
        x, z = ys
        return [al * x - be * x * z, de * x * z - ga * z]
    if kind == W.VAN_DER_POL:
        mu = p[0]
        return [ys[1], mu * ((1 - ys[0] ** 2) * ys[1] - ys[0])]
    if kind == W.RIGID_BODY:
        y1, y2, y3 = ys
        return [-2 * y2 * y3, sp.Rational(5, 4) * y1 * y3, -sp.Rational(1, 2) * y1 * y2]
    if kind == W.LORENZ96:
        F = p[0]
        d = len(ys)
        return [(ys[(i + 1) % d] - ys[(i - 2) % d]) * ys[(i - 1) % d] - ys[i] + F
                for i in range(d)]
    raise ValueError(kind)


def _lie_derivatives(problem, q):
    d = problem.d
    ys = sp.symbols(f"y0:{d}")
    f = sp.Matrix(_symbolic_f(problem.kind, problem.params, ys))
    J = f.jacobian(ys)
    derivs = [sp.Matrix(ys), f]
    for _ in range(2, q + 1):
        prev = derivs[-1]
        derivs.append(prev.jacobian(ys) * f)
    subs = {ys[i]: sp.Rational(float(problem.y0[i])) for i in range(d)}
    out = np.zeros(d * (q + 1))
    for i in range(q + 1):
        vals = derivs[i].subs(subs)
        for k in range(d):
            out[k * (q + 1) + i] = float(vals[k])
    return out


@pytest.mark.parametrize("problem", [
    W.logistic(q=4), W.logistic_paper(q=3), W.fitzhugh_nagumo(q=4), W.van_der_pol(q=4),
    W.rigid_body(q=4), W.lotka_volterra(q=4), W.lotka_volterra_batch(count=3, seed=5)[2],
    W.lorenz96(d=6, q=3)],
    ids=lambda p: p.name)
def test_matches_symbolic_lie_derivatives(problem):
    q = problem.q
    mu = initial_state(problem.kind, problem.params, problem.y0, q)
    ref = _lie_derivatives(problem, q)
    np.testing.assert_allclose(mu, ref, rtol=1e-12, atol=1e-12)


def test_affine_closed_form():
    L = np.array([[0.0, 1.0], [-2.0, -0.3]])
    c = np.array([0.5, -1.0])
    p = W.affine(L, c, [1.0, 0.25], q=3)
    mu = initial_state(p.kind, p.params, p.y0, 3)
    ders = [p.y0, L @ p.y0 + c]
    for _ in range(2):
        ders.append(L @ ders[-1])
    ref = np.array([[ders[i][k] for i in range(4)] for k in range(2)]).reshape(-1)
    np.testing.assert_allclose(mu, ref, rtol=1e-14)
