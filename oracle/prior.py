"""IWP(q) prior transitions (Section 2.1) and the preconditioned form (Section 2.4).

Test infrastructure only (see the package docstring).

State layout: Y = [Y^(0), ..., Y^(q)] per ODE dimension, stacked dimension-major, so that
E_i = I_d (x) e_i selects the i-th derivative (Section 2.1).  Index of derivative i of
dimension k is k (q + 1) + i.
"""
from __future__ import annotations

import math

import numpy as np


def iwp_1d(q: int, h: float):
    """Closed-form transition of one dimension of the IWP(q) prior (Section 2.1).

    [Phi(h)]_ij = h^(j-i) / (j-i)!  for j >= i, else 0     (upper-triangular Taylor shift)
    [Q(h)]_ij   = h^(2q+1-i-j) / ((2q+1-i-j) (q-i)! (q-j)!)
    with 0-based indices i, j in {0..q}.  The printed Phi formula is garbled (it shows an
    indicator 1_{i=j}); the upper-triangular reading is the one that makes Phi the flow of
    dY^(i) = Y^(i+1) dt and is pinned in the tests by the semigroup identity and by quadrature
    of Q.
    """
    K = q + 1
    Phi = np.zeros((K, K))
    Q = np.zeros((K, K))
    for i in range(K):
        for j in range(K):
            if j >= i:
                Phi[i, j] = h ** (j - i) / math.factorial(j - i)
            p = 2 * q + 1 - i - j
            Q[i, j] = h ** p / (p * math.factorial(q - i) * math.factorial(q - j))
    return Phi, Q


def iwp_transition(q: int, h: float, d: int = 1):
    """Phi(h) = I_d (x) Phi1(h), Q(h) = I_d (x) Q1(h)  (Section 2.1), with sigma = 1."""
    Phi1, Q1 = iwp_1d(q, h)
    I = np.eye(d)
    return np.kron(I, Phi1), np.kron(I, Q1)


def projection(i: int, q: int, d: int) -> np.ndarray:
    """E_i = I_d (x) e_i^T, a d x d(q+1) matrix selecting the i-th derivative (Section 2.1)."""
    e = np.zeros((1, q + 1))
    e[0, i] = 1.0
    return np.kron(np.eye(d), e)


def preconditioner_1d(q: int, h: float) -> np.ndarray:
    """Diagonal of the coordinate change x = T x_bar that makes the transitions step-size
    free (Section 2.4 names the preconditioner but prints no formula; this is the Nordsieck
    scaling T = sqrt(h) diag(h^(q-i) / (q-i)!), i = 0..q)."""
    return np.array([math.sqrt(h) * h ** (q - i) / math.factorial(q - i) for i in range(q + 1)])


def preconditioned_1d(q: int):
    """Step-size free transition in preconditioned coordinates:
    Phi_bar_ij = binom(q-i, j-i) (j >= i), Q_bar_ij = 1 / (2q+1-i-j).
    Derived from the closed forms above: Phi_bar = T^-1 Phi(h) T, Q_bar = T^-1 Q(h) T^-1."""
    K = q + 1
    Pb = np.zeros((K, K))
    Qb = np.zeros((K, K))
    for i in range(K):
        for j in range(K):
            if j >= i:
                Pb[i, j] = math.comb(q - i, j - i)
            Qb[i, j] = 1.0 / (2 * q + 1 - i - j)
    return Pb, Qb
