"""Iterated extended Kalman smoother (Algorithm 2, Section 3.2), run sequentially.

Test infrastructure only.  The parallel solver computes the same numbers as the sequential
IEKS (Section 4.1); this is that sequential IEKS, in float64 and original coordinates:

    mu0 <- exact initial state (Eq. mu0), Sigma0 = 0
    eta_n <- mu0 for n = 0..N                        (constant initial trajectory)
    repeat
        H_n, d_n <- first-order Taylor linearisation at eta_n, n = 1..N
                    H_n = E1 - F_y(E0 eta_n) E0,  d_n = f(E0 eta_n) - F_y(E0 eta_n) E0 eta_n
        (m^s, P^s) <- square-root Kalman filter + RTS smoother in the linearised model
        delta <- max over n and over the d solution components of |E0 m^s_n - E0 eta_n|
        eta <- m^s
    until delta <= atol + rtol max|E0 m^s| or max_iter iterations

Stopping rule reading: Section 3.2.2 stops when the change of the trajectory estimate is small
but fixes neither the norm nor the components.  The change is measured on the solution
estimate E0 m (what Algorithm 2 returns), in original coordinates: the derivative components
carry a round-off floor far above 1e-10 in original coordinates (about 5e-8 for
FitzHugh-Nagumo with q = 3, N = 4096, observed with this oracle), so a rule over all state
components would never stop.

Then the quasi-maximum-likelihood diffusion sigma^2 (Section 2.4; formula not printed in the
paper, read as the prediction-error estimate (1 / (N d)) sum_n r_n^T S_n^-1 r_n of the final
filter pass with sigma = 1, r_n = H_n m-_n - d_n) rescales the square-root covariances by
sigma-hat; the means do not depend on sigma.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

from . import odes
from .filtering import rts_smoother, sequential_filter
from .linalg import solve_lower
from .prior import iwp_transition, projection
from .taylor import initial_state


LINEARIZATIONS = ("ek1", "diag", "ek0")


def approximate_jacobian(F, mode: str):
    """The Jacobian used by the linearisation: exact (EK1), its diagonal (DiagonalEK1) or zero
    (EK0) -- the approximate-Jacobian linearisations of Section 3.2.1 (remark on approximate
    Jacobians)."""
    if mode == "ek1":
        return F
    if mode == "diag":
        return np.diag(np.diag(F))
    if mode == "ek0":
        return np.zeros_like(F)
    raise ValueError(mode)


def linearize(kind, params, eta_n, t, q, d, mode: str = "ek1"):
    """H_n, d_n of Eq. linearized-observation-model (with the Jacobian of `mode`)."""
    E0 = projection(0, q, d)
    E1 = projection(1, q, d)
    y = E0 @ eta_n
    F = approximate_jacobian(odes.jac(kind, params, y, t), mode)
    fy = odes.f(kind, params, y, t)
    return E1 - F @ E0, fy - F @ y


def linearize_all(problem, traj, mode: str = "ek1"):
    d, q = problem.d, problem.q
    ts = problem.times
    Hs = [None]
    ds = [None]
    for n in range(1, problem.N + 1):
        H, dv = linearize(problem.kind, problem.params, traj[n], ts[n], q, d, mode)
        Hs.append(H)
        ds.append(dv)
    return Hs, ds


def prior_factors(problem):
    """Phi, Q, sqrt(Q) of the IWP prior (Section 2.1): one triple on a uniform grid; per-step
    lists (index n = 1..N for the step into t_n, index 0 unused) on a non-uniform grid."""
    if problem.uniform:
        Phi, Q = iwp_transition(problem.q, problem.h, problem.d)
        sQ = np.linalg.cholesky(Q)
        return Phi, Q, sQ
    Phis, Qs, sQs = [None], [None], [None]
    for h in problem.steps:
        Phi, Q = iwp_transition(problem.q, float(h), problem.d)
        Phis.append(Phi)
        Qs.append(Q)
        sQs.append(np.linalg.cholesky(Q))
    return Phis, Qs, sQs


def linear_smoother(problem, traj, mu0, Phi, sQ, want_cov=True, mode: str = "ek1"):
    """One linearise + filter + smoother pass (Alg. 1 in the linearised model)."""
    D = problem.D
    Hs, ds = linearize_all(problem, traj, mode)
    mf, sPf, sS, res = sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    ms, sPs = rts_smoother(mf, sPf, Phi, sQ)
    return dict(Hs=Hs, ds=ds, mf=mf, sPf=sPf, sS=sS, res=res, ms=ms, sPs=sPs)


def sigma2_hat(sS, res, N, d):
    """(1 / (N d)) sum_{n=1..N} || sqrtS_n^-1 r_n ||^2."""
    tot = 0.0
    for n in range(1, N + 1):
        z = solve_lower(sS[n], res[n])
        tot += float(z @ z)
    return tot / (N * d)


def objective(traj, Phi, sQ):
    """V(eta_0:N) = 1/2 sum_n || eta_n - Phi eta_{n-1} ||^2_{Q^-1}  (Eq. objective-value)."""
    from .filtering import step_matrix
    tot = 0.0
    for n in range(1, traj.shape[0]):
        z = solve_lower(step_matrix(sQ, n), traj[n] - step_matrix(Phi, n) @ traj[n - 1])
        tot += float(z @ z)
    return 0.5 * tot


def coarse_initial_trajectory(problem, coarse_n: int):
    """Initial trajectory from a sequential method on a coarse grid (Section 3.2.2, remark on
    other choices for the initial trajectory): the sequential EKS (local linearisation) on
    coarse_n uniform steps over the same interval, then between coarse nodes the prior's
    mean propagated from the node at or before t: eta_n = Phi(t_n - t_k) m^s_k with
    k = floor(n coarse_n / N) (an exact integer index; t_n - t_k = (n coarse_n - k N) T / (N coarse_n)).
    Parity with the GPU path fixes this reading of the interpolation, which the paper leaves
    open."""
    from .eks import eks
    from .prior import iwp_transition
    N, D = problem.N, problem.D
    pc = dataclasses.replace(problem, N=int(coarse_n))
    ms, _, _ = eks(pc, calibrate=False)
    span = problem.t1 - problem.t0
    traj = np.zeros((N + 1, D))
    for n in range(N + 1):
        k = min((n * coarse_n) // N, coarse_n)
        tau = float(n * coarse_n - k * N) * (span / (float(N) * float(coarse_n)))
        Phi_tau, _ = iwp_transition(problem.q, tau, problem.d)
        traj[n] = Phi_tau @ ms[k]
    return traj


@dataclasses.dataclass
class IEKSResult:
    means: np.ndarray            # (N+1, D) smoothing means of the final iteration
    sqrtcovs: np.ndarray         # (N+1, D, D) calibrated square-root covariances
    sigma2: float                # quasi-MLE diffusion
    iterations: int
    deltas: List[float]          # max |change| per iteration
    iterates: Optional[List[np.ndarray]] = None   # means after each iteration (if recorded)
    mu0: Optional[np.ndarray] = None
    last_pass: Optional[dict] = None
    objectives: Optional[List[float]] = None      # V of the initial trajectory and each iterate


def ieks(problem, atol: float = 1e-10, max_iter: int = 20, fixed_iters: Optional[int] = None,
         calibrate: bool = True, record_iterates: bool = False, init: str = "mu0",
         want_cov: bool = True, rtol: float = 0.0, init_traj=None, linearization: str = "ek1",
         obj_atol: Optional[float] = None, obj_rtol: float = 0.0,
         record_objective: bool = False, coarse_n: int = 0) -> IEKSResult:
    """Algorithm 2.  ``fixed_iters`` runs exactly that many iterations (no stopping rule);
    ``init='y0'`` starts from eta_n = [y0, 0, ..., 0] instead of mu0 (Section 3.2.2 notes that
    only E0 eta matters for the linearisation); ``init_traj`` ((N+1) x D) replaces the constant
    initial trajectory (a warm start).  ``linearization`` picks the Jacobian (EK1, diagonal EK1
    or EK0, Section 3.2.1).  ``obj_atol`` enables the second stopping criterion of Section 3.2.2:
    stop when |V(eta^k) - V(eta^(k-1))| <= obj_atol + obj_rtol |V(eta^k)| (Eq. objective-value),
    in addition to the change rule; ``record_objective`` records V without using it.
    ``coarse_n`` > 0 starts from coarse_initial_trajectory(problem, coarse_n)."""
    d, q, N, D = problem.d, problem.q, problem.N, problem.D
    Phi, Q, sQ = prior_factors(problem)
    mu0 = initial_state(problem.kind, problem.params, problem.y0, q)
    if init == "mu0":
        start = mu0
    else:
        start = np.zeros(D)
        start[0::q + 1] = problem.y0
    if init_traj is not None:
        traj = np.array(init_traj, dtype=float)
    elif coarse_n > 0:
        traj = coarse_initial_trajectory(problem, coarse_n)
    else:
        traj = np.tile(start, (N + 1, 1))
    deltas = []
    iterates = [] if record_iterates else None
    use_obj = obj_atol is not None
    objectives = [objective(traj, Phi, sQ)] if (use_obj or record_objective) else None
    k = 0
    last = None
    limit = fixed_iters if fixed_iters is not None else max_iter
    while k < limit:
        last = linear_smoother(problem, traj, mu0, Phi, sQ, mode=linearization)
        new = last["ms"]
        delta = float(np.max(np.abs(new[:, 0::q + 1] - traj[:, 0::q + 1])))
        deltas.append(delta)
        traj = new
        k += 1
        if record_iterates:
            iterates.append(new.copy())
        if objectives is not None:
            objectives.append(objective(traj, Phi, sQ))
        if fixed_iters is not None:
            continue
        if delta <= atol + rtol * float(np.max(np.abs(new[:, 0::q + 1]))):
            break
        if use_obj and abs(objectives[-1] - objectives[-2]) <= obj_atol + obj_rtol * abs(objectives[-1]):
            break
    s2 = sigma2_hat(last["sS"], last["res"], N, d) if calibrate else 1.0
    scale = np.sqrt(s2)
    return IEKSResult(means=traj, sqrtcovs=last["sPs"] * scale if want_cov else None,
                      sigma2=s2, iterations=k, deltas=deltas, iterates=iterates, mu0=mu0,
                      last_pass=last, objectives=objectives)
