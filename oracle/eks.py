"""Sequential extended Kalman smoother with local linearisation (Section 2.3 / Section 4.3).

Test infrastructure only.  The established sequential probabilistic solver: one forward pass
that linearises the observation model at the predicted mean m-_n (not along a global
trajectory), then one square-root RTS pass.  No iteration.
"""
from __future__ import annotations

import numpy as np

from .filtering import predict, rts_smoother, step_matrix, update
from .ieks import linearize, prior_factors, sigma2_hat
from .taylor import initial_state


def eks(problem, calibrate: bool = True):
    d, q, N, D = problem.d, problem.q, problem.N, problem.D
    Phi, Q, sQ = prior_factors(problem)
    mu0 = initial_state(problem.kind, problem.params, problem.y0, q)
    ts = problem.times
    mf = np.zeros((N + 1, D))
    sPf = np.zeros((N + 1, D, D))
    sS = np.zeros((N + 1, d, d))
    res = np.zeros((N + 1, d))
    mf[0] = mu0
    for n in range(1, N + 1):
        mp, sPp = predict(mf[n - 1], sPf[n - 1], step_matrix(Phi, n), step_matrix(sQ, n))
        H, dv = linearize(problem.kind, problem.params, mp, ts[n], q, d)
        mf[n], sPf[n], sS[n], res[n] = update(mp, sPp, H, dv)
    ms, sPs = rts_smoother(mf, sPf, Phi, sQ)
    s2 = sigma2_hat(sS, res, N, d) if calibrate else 1.0
    return ms, sPs * np.sqrt(s2), s2
