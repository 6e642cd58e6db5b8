"""Pins of the oracle's IWP prior (Section 2.1) and preconditioner (Section 2.4).

Each check uses a route independent of the closed form being tested: the matrix exponential of
the SDE drift, numerical quadrature of the noise integral, the semigroup law of the Markov
transition, and the exact rational entries of the printed Q formula at h = 1.
"""
import math
from fractions import Fraction
import os

import numpy as np
import pytest
import scipy.linalg
from scipy.integrate import quad

from oracle.prior import (iwp_1d, iwp_transition, preconditioned_1d, preconditioner_1d,
                          projection)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def drift(q):
    """Drift of dY^(i) = Y^(i+1) dt, i < q; dY^(q) = sigma dW (Section 2.1)."""
    F = np.zeros((q + 1, q + 1))
    for i in range(q):
        F[i, i + 1] = 1.0
    return F


@pytest.mark.parametrize("q", [1, 2, 3, 4])
@pytest.mark.parametrize("h", [1e-3, 0.1, 0.7, 2.0])
def test_phi_is_matrix_exponential_of_drift(q, h):
    Phi, _ = iwp_1d(q, h)
    np.testing.assert_allclose(Phi, scipy.linalg.expm(drift(q) * h), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("h", [0.05, 0.5, 1.5])
def test_q_is_noise_integral(q, h):
    """Q(h) = int_0^h Phi(s) e_q e_q^T Phi(s)^T ds (diffusion enters the last derivative)."""
    _, Q = iwp_1d(q, h)
    F = drift(q)
    ref = np.zeros((q + 1, q + 1))
    for i in range(q + 1):
        for j in range(q + 1):
            def integrand(s, i=i, j=j):
                E = scipy.linalg.expm(F * s)
                return E[i, q] * E[j, q]
            ref[i, j] = quad(integrand, 0.0, h, epsabs=0, epsrel=1e-13, limit=200)[0]
    np.testing.assert_allclose(Q, ref, rtol=1e-10, atol=1e-16)


@pytest.mark.parametrize("q", [1, 2, 3])
def test_semigroup(q):
    a, b = 0.3, 0.45
    Pa, Qa = iwp_1d(q, a)
    Pb, Qb = iwp_1d(q, b)
    Pab, Qab = iwp_1d(q, a + b)
    np.testing.assert_allclose(Pa @ Pb, Pab, rtol=1e-14)
    np.testing.assert_allclose(Pb @ Qa @ Pb.T + Qb, Qab, rtol=1e-13)


def test_q_nu1_textbook():
    h = 0.37
    _, Q = iwp_1d(1, h)
    np.testing.assert_allclose(Q, [[h ** 3 / 3, h ** 2 / 2], [h ** 2 / 2, h]], rtol=1e-15)


def test_q_at_h1_matches_printed_formula_exactly():
    """tests/golden/iwp_q_h1.txt holds [Q(1)]_ij = 1 / ((2q+1-i-j) (q-i)! (q-j)!) as exact
    fractions (Section 2.1, closed form of Q)."""
    rows = {}
    with open(os.path.join(GOLDEN, "iwp_q_h1.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            q, i, j, frac = line.split()
            rows[(int(q), int(i), int(j))] = Fraction(frac)
    seen = set()
    for (q, i, j), val in rows.items():
        _, Q = iwp_1d(q, 1.0)
        assert Q[i, j] == pytest.approx(float(val), rel=1e-15)
        seen.add(q)
    assert seen == {1, 2, 3}


@pytest.mark.parametrize("q", [1, 2, 3])
def test_kron_layout(q):
    d = 3
    Phi, Q = iwp_transition(q, 0.2, d)
    P1, Q1 = iwp_1d(q, 0.2)
    K = q + 1
    for k in range(d):
        np.testing.assert_array_equal(Phi[k * K:(k + 1) * K, k * K:(k + 1) * K], P1)
        np.testing.assert_array_equal(Q[k * K:(k + 1) * K, k * K:(k + 1) * K], Q1)
    E0, E1 = projection(0, q, d), projection(1, q, d)
    x = np.arange(d * K, dtype=float)
    np.testing.assert_array_equal(E0 @ x, x[0::K])
    np.testing.assert_array_equal(E1 @ x, x[1::K])


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("h", [1e-5, 3e-3, 0.25])
def test_preconditioner_makes_transitions_step_size_free(q, h):
    Phi, Q = iwp_1d(q, h)
    T = preconditioner_1d(q, h)
    Pb, Qb = preconditioned_1d(q)
    np.testing.assert_allclose(np.diag(1 / T) @ Phi @ np.diag(T), Pb, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(np.diag(1 / T) @ Q @ np.diag(1 / T), Qb, rtol=1e-12)
    # Q_bar is the Hilbert-type matrix 1 / (2q+1-i-j): symmetric positive definite
    assert np.all(np.linalg.eigvalsh(Qb) > 0)
    for i in range(q + 1):
        for j in range(q + 1):
            assert Qb[i, j] == pytest.approx(1.0 / (2 * q + 1 - i - j))
            if j >= i:
                assert Pb[i, j] == math.comb(q - i, j - i)
