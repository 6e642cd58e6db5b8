"""Pin of the oracle's Jacobians dF/dy (oracle/odes.py::jac), which the linearisation of Section
3.2.1 evaluates at E0 eta_n.

The reference is independent of the hand-written derivatives: sympy differentiates the symbolic
vector field of each family (the same field the Taylor-mode initial state is pinned against)
and the result is evaluated at random points.  A Gauss-Newton fixed point does not depend on
the Jacobian, so the fixed-point pins cannot catch a slip here; this test can, including a
wrong index in Lorenz-96's cyclic coupling.  The vector fields themselves are checked against
the symbolic ones too, and the Jacobians against central differences of f.
"""
import numpy as np
import pytest
import sympy as sp

import workloads as W
from oracle import odes

from test_oracle_taylor import _symbolic_f

FAMILIES = [W.logistic(), W.logistic_paper(), W.fitzhugh_nagumo(), W.van_der_pol(),
            W.rigid_body(), W.lotka_volterra(), W.lotka_volterra_batch(count=3, seed=5)[2],
            W.lorenz96(d=6, q=2), W.lorenz96(d=64, q=2)]


def _symbolic_jacobian(problem):
    ys = sp.symbols(f"y0:{problem.d}")
    f = sp.Matrix(_symbolic_f(problem.kind, problem.params, ys))
    J = f.jacobian(ys)
    return sp.lambdify([ys], f, "numpy"), sp.lambdify([ys], J, "numpy")


@pytest.mark.parametrize("problem", FAMILIES, ids=lambda p: f"{p.name}-d{p.d}")
def test_jacobian_matches_symbolic(problem):
    f_sym, J_sym = _symbolic_jacobian(problem)
    rng = np.random.default_rng(7 + problem.d)
    for _ in range(5):
        y = problem.y0 + rng.uniform(-2.0, 2.0, problem.d)
        Jref = np.asarray(J_sym(y), dtype=np.float64)
        Jgot = odes.jac(problem.kind, problem.params, y)
        assert Jgot.shape == (problem.d, problem.d)
        np.testing.assert_allclose(Jgot, Jref, rtol=1e-13, atol=1e-13 * max(1.0, np.abs(Jref).max()))
        fref = np.asarray(f_sym(y), dtype=np.float64).reshape(-1)
        np.testing.assert_allclose(odes.f(problem.kind, problem.params, y), fref, rtol=1e-13,
                                   atol=1e-13 * max(1.0, np.abs(fref).max()))


def test_affine_jacobian_is_the_matrix():
    L = np.array([[0.3, -0.5, 0.1], [0.8, -0.2, 0.0], [1.5, 0.25, -2.0]])
    p = W.affine(L, [0.1, -0.4, 0.0], [0.5, 1.0, -1.0])
    np.testing.assert_array_equal(odes.jac(p.kind, p.params, np.array([3.0, -1.0, 2.0])), L)


@pytest.mark.parametrize("problem", FAMILIES[:7] + [W.lorenz96(d=8, q=2)],
                         ids=lambda p: f"{p.name}-d{p.d}")
def test_jacobian_matches_central_differences(problem):
    """A route without sympy: (f(y + e_j h) - f(y - e_j h)) / 2h is exact for the quadratic
    fields and within O(h^2) for the cubic FitzHugh-Nagumo term."""
    rng = np.random.default_rng(3)
    y = problem.y0 + rng.uniform(-1.0, 1.0, problem.d)
    J = odes.jac(problem.kind, problem.params, y)
    h = 1e-4
    for j in range(problem.d):
        e = np.zeros(problem.d)
        e[j] = h
        col = (odes.f(problem.kind, problem.params, y + e)
               - odes.f(problem.kind, problem.params, y - e)) / (2 * h)
        np.testing.assert_allclose(J[:, j], col, rtol=1e-7, atol=1e-7)
