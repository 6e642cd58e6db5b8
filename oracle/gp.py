"""Exact dense Gaussian conditioning for affine ODEs on tiny grids (Section 3.1).

Test infrastructure only.  For y' = L y + c the observation model is affine,
Z_n | Y_n ~ delta(H Y_n - c) with H = E1 - L E0, so Gaussian filtering and smoothing is exact
(Section 3.1).  This module builds the joint Gaussian of Y_0:N under the prior
Y_0 = mu0 (Sigma0 = 0), Y_{n+1} = Phi Y_n + w_n, w_n ~ N(0, Q), and conditions it on
H Y_n = c, n = 1..N, by a dense solve -- an independent route to the same posterior that pins
the whole square-root filter/smoother.  It also returns the exact maximum-likelihood diffusion
(z^T (B Sigma B^T)^-1 z) / (N d), which the prediction-error form of the quasi-MLE must equal.
"""
from __future__ import annotations

import numpy as np

from .prior import iwp_transition, projection
from .taylor import initial_state


def dense_posterior(problem):
    """Works on uniform and non-uniform grids: step k (into t_k) has its own Phi_k, Q_k, and
    Y_n = Phi_n ... Phi_1 Y_0 + sum_{k <= n} Phi_n ... Phi_{k+1} w_k."""
    d, q, N, D = problem.d, problem.q, problem.N, problem.D
    steps = problem.steps
    Phis, Qs = [None], [None]
    for h in steps:
        Phi, Q = iwp_transition(q, float(h), d)
        Phis.append(Phi)
        Qs.append(Q)
    mu0 = initial_state(problem.kind, problem.params, problem.y0, q)
    L = problem.params[: d * d].reshape(d, d)
    c = problem.params[d * d: d * d + d]
    H = projection(1, q, d) - L @ projection(0, q, d)

    def flow(n, k):
        """Phi_n ... Phi_{k+1} (identity for n == k)."""
        M = np.eye(D)
        for j in range(k + 1, n + 1):
            M = Phis[j] @ M
        return M

    # prior mean and covariance of the stacked state [Y_0, ..., Y_N]
    n_tot = (N + 1) * D
    mean = np.zeros(n_tot)
    cov = np.zeros((n_tot, n_tot))
    for n in range(N + 1):
        mean[n * D:(n + 1) * D] = flow(n, 0) @ mu0
    for n in range(N + 1):
        for m in range(N + 1):
            acc = np.zeros((D, D))
            for k in range(1, min(n, m) + 1):
                acc += flow(n, k) @ Qs[k] @ flow(m, k).T
            cov[n * D:(n + 1) * D, m * D:(m + 1) * D] = acc
    # constraints B Y = rhs
    B = np.zeros((N * d, n_tot))
    rhs = np.zeros(N * d)
    for n in range(1, N + 1):
        B[(n - 1) * d:n * d, n * D:(n + 1) * D] = H
        rhs[(n - 1) * d:n * d] = c
    S = B @ cov @ B.T
    z = rhs - B @ mean
    gain = np.linalg.solve(S, B @ cov).T
    post_mean = mean + gain @ z
    post_cov = cov - gain @ B @ cov
    sigma2 = float(z @ np.linalg.solve(S, z)) / (N * d)
    means = post_mean.reshape(N + 1, D)
    covs = np.stack([post_cov[n * D:(n + 1) * D, n * D:(n + 1) * D] for n in range(N + 1)])
    return means, covs, sigma2
