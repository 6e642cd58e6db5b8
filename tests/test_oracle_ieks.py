"""Pins of the oracle's iterated extended Kalman smoother (Algorithm 2) and calibration.

* Affine ODEs (Section 3.1): the IEKS is exact inference, so one iteration must equal dense
  Gaussian conditioning of the joint prior on the observations, the second iteration must not
  move, and the quasi-MLE diffusion must equal the exact maximum-likelihood value.
* Logistic ODE of Section 4.1 (rate 1): the converged MAP approaches the analytic solution at
  least at the polynomial rate h^q as the grid is refined (Section 3.2.2, convergence of the
  MAP estimate).
* Every iterate satisfies the linearised constraint H_n m^s_n = d_n (noiseless observation);
  at convergence E1 m_n = f(E0 m_n) on the grid.
* Starting from [y0, 0, ..., 0] instead of mu0 gives the same iterates (only E0 eta matters for
  the linearisation, Section 3.2.2).
* The sequential EKS is exact on affine problems (local linearisation is exact there).
* The objective value (Eq. objective-value) is minimised by the posterior mean under the
  constraints: perturbations that keep the constraints only increase it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eks, gp, ieks
from oracle.odes import f as ode_f
from oracle.prior import projection

AFFINE_CASES = [
    W.affine([[-1.0]], [0.0], [1.0], t1=1.5, N=7, q=1),
    W.affine([[-1.0]], [1.0], [0.2], t1=2.0, N=6, q=2),
    W.affine([[0.0, 1.0], [-1.0, 0.0]], [0.0, 0.0], [1.0, 0.0], t1=3.0, N=5, q=2),
    W.affine([[0.3, -0.5], [0.8, -0.2]], [0.1, -0.4], [0.5, 1.0], t1=1.0, N=4, q=3),
]


@pytest.mark.parametrize("problem", AFFINE_CASES)
def test_affine_one_iteration_is_exact_posterior(problem):
    r = ieks.ieks(problem, fixed_iters=2)
    means, covs, s2 = gp.dense_posterior(problem)
    it1 = ieks.ieks(problem, fixed_iters=1)
    np.testing.assert_allclose(it1.means, means, atol=1e-10, rtol=1e-9)
    assert r.deltas[1] < 1e-12 * max(1.0, np.max(np.abs(means)))
    assert r.sigma2 == pytest.approx(s2, rel=1e-9)
    got = np.einsum("nij,nkj->nik", r.sqrtcovs, r.sqrtcovs)
    np.testing.assert_allclose(got, covs * s2, atol=1e-10 * max(1.0, np.max(np.abs(covs * s2))))


def test_logistic_converges_at_polynomial_rate():
    errs = {}
    for q in (1, 2):
        Ns = (512, 1024, 2048) if q == 1 else (64, 128, 256)
        e = []
        for N in Ns:
            p = W.logistic_paper(N=N, q=q)
            r = ieks.ieks(p)
            t = np.linspace(p.t0, p.t1, N + 1)
            exact = 1.0 / (1.0 + (1.0 / 0.01 - 1.0) * np.exp(-t))
            e.append(np.max(np.abs(r.means[:, 0] - exact)))
        slope = np.polyfit(np.log([p.t1 / N for N in Ns]), np.log(e), 1)[0]
        errs[q] = (e, slope)
        assert slope >= q - 0.3, (q, e, slope)
    # observed on the grid: order q + 1 for these problems
    assert errs[2][1] > 2.5


@pytest.mark.parametrize("problem", [W.logistic(N=96, q=2), W.fitzhugh_nagumo(N=64, q=2),
                                     W.van_der_pol(N=60, q=3)], ids=lambda p: p.name)
def test_constraint_identity_every_iteration(problem):
    r = ieks.ieks(problem, fixed_iters=3, record_iterates=True)
    traj_prev = np.tile(r.mu0, (problem.N + 1, 1))
    for new in r.iterates:
        Hs, ds = ieks.linearize_all(problem, traj_prev)
        for n in range(1, problem.N + 1):
            res = Hs[n] @ new[n] - ds[n]
            assert np.max(np.abs(res)) <= 1e-9 * max(1.0, np.max(np.abs(new[n])))
        traj_prev = new


def test_converged_mean_solves_ode_on_grid():
    p = W.logistic_paper(N=256, q=2)
    r = ieks.ieks(p)
    assert r.deltas[-1] < 1e-10
    E0, E1 = projection(0, p.q, p.d), projection(1, p.q, p.d)
    for n in range(p.N + 1):
        y = E0 @ r.means[n]
        assert np.max(np.abs(E1 @ r.means[n] - ode_f(p.kind, p.params, y))) < 1e-8


def test_init_with_y0_only_gives_same_iterates():
    p = W.van_der_pol(N=40, q=2)
    a = ieks.ieks(p, fixed_iters=4, record_iterates=True)
    b = ieks.ieks(p, fixed_iters=4, record_iterates=True, init="y0")
    for x, y in zip(a.iterates, b.iterates):
        np.testing.assert_allclose(x, y, atol=1e-12, rtol=1e-12)


@pytest.mark.parametrize("problem", AFFINE_CASES[:3])
def test_eks_exact_on_affine(problem):
    ms, sPs, s2 = eks.eks(problem)
    means, covs, s2ref = gp.dense_posterior(problem)
    np.testing.assert_allclose(ms, means, atol=1e-10)
    assert s2 == pytest.approx(s2ref, rel=1e-9)


def test_posterior_mean_minimises_objective_under_constraints():
    p = AFFINE_CASES[2]
    r = ieks.ieks(p, fixed_iters=1)
    Phi, Q, sQ = ieks.prior_factors(p)
    V0 = ieks.objective(r.means, Phi, sQ)
    # a trajectory propagated exactly by Phi has zero cost
    traj = np.zeros_like(r.means)
    traj[0] = r.mu0
    for n in range(1, p.N + 1):
        traj[n] = Phi @ traj[n - 1]
    assert ieks.objective(traj, Phi, sQ) == pytest.approx(0.0, abs=1e-20)
    # feasible perturbations (kept in the null space of H_n, x_0 fixed) increase V
    H = projection(1, p.q, p.d) - p.params[:4].reshape(2, 2) @ projection(0, p.q, p.d)
    _, _, Vt = np.linalg.svd(H)
    null = Vt[H.shape[0]:]
    rng = np.random.default_rng(0)
    for _ in range(5):
        pert = np.zeros_like(r.means)
        for n in range(1, p.N + 1):
            pert[n] = null.T @ rng.standard_normal(null.shape[0])
        for eps in (1e-3, -1e-3):
            assert ieks.objective(r.means + eps * pert, Phi, sQ) > V0


# ---- approximate Jacobians (Section 3.2.1, remark on EK0 and DiagonalEK1) -----------------------
def test_diagonal_ek1_equals_ek1_for_scalar_odes():
    """For d = 1 the Jacobian is its own diagonal: DiagonalEK1 iterates are EK1's."""
    p = W.logistic_paper(N=60, q=2)
    a = ieks.ieks(p, fixed_iters=4, want_cov=False, calibrate=False, record_iterates=True)
    b = ieks.ieks(p, fixed_iters=4, want_cov=False, calibrate=False, record_iterates=True,
                  linearization="diag")
    for x, y in zip(a.iterates, b.iterates):
        np.testing.assert_array_equal(x, y)


def test_ek0_equals_ek1_when_the_field_does_not_depend_on_y():
    """y' = c (affine with L = 0): the Jacobian is zero, so EK0 is EK1."""
    p = W.affine(np.zeros((2, 2)), [0.5, -1.0], [1.0, 2.0], t1=2.0, N=9, q=2)
    a = ieks.ieks(p, fixed_iters=2, want_cov=True, calibrate=True)
    b = ieks.ieks(p, fixed_iters=2, want_cov=True, calibrate=True, linearization="ek0")
    np.testing.assert_allclose(a.means, b.means, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p,mode", [
    (W.logistic_paper(N=100, q=2), "ek0"),
    (W.lotka_volterra(N=500, q=2, t1=2.0), "ek0"),
    (W.lotka_volterra(N=500, q=2, t1=2.0), "diag"),
    (W.van_der_pol(N=300, q=2), "diag"),
])
def test_approximate_jacobian_fixed_points_solve_the_ode_on_the_grid(p, mode):
    """A fixed point of the approximate-Jacobian iteration satisfies the linearised constraint
    at itself, H(eta) eta = d(eta), i.e. E1 eta_n = f(E0 eta_n) for every n >= 1 whatever the
    Jacobian; it is feasible, so its objective V is not below EK1's (the MAP)."""
    from oracle import odes
    r = ieks.ieks(p, atol=1e-12, max_iter=200, want_cov=False, calibrate=False,
                  linearization=mode, record_objective=True)
    assert r.deltas[-1] <= 1e-12
    q1 = p.q + 1
    for n in range(1, p.N + 1):
        np.testing.assert_allclose(r.means[n, 1::q1], odes.f(p.kind, p.params, r.means[n, 0::q1], 0.0),
                                   rtol=0, atol=1e-9)
    e = ieks.ieks(p, atol=1e-12, max_iter=200, want_cov=False, calibrate=False,
                  record_objective=True)
    assert r.objectives[-1] >= e.objectives[-1] * (1 - 1e-10)
    # the approximate Jacobian does change the iteration
    a1 = ieks.ieks(p, fixed_iters=1, want_cov=False, calibrate=False, linearization=mode)
    b1 = ieks.ieks(p, fixed_iters=1, want_cov=False, calibrate=False)
    assert np.max(np.abs(a1.means - b1.means)) > 1e-6


# ---- the objective value V (Eq. objective-value) and its stopping rule ---------------------------
def test_objective_closed_form_iwp1_one_step():
    """IWP(1), one step h: Q(h)^-1 = [[12/h^3, -6/h^2], [-6/h^2, 4/h]] (the textbook inverse of
    [[h^3/3, h^2/2], [h^2/2, h]]), so V = 1/2 w^T Q^-1 w with w = eta_1 - Phi eta_0."""
    h = 0.37
    p = W.Problem(W.AFFINE, 1, np.array([0.0, 0.0]), np.array([0.0]), 0.0, h, 1, 1)
    Phi, Q, sQ = ieks.prior_factors(p)
    e0 = np.array([0.3, -1.2])
    e1 = np.array([0.9, 0.4])
    w = np.array([e1[0] - e0[0] - h * e0[1], e1[1] - e0[1]])
    Qi = np.array([[12 / h ** 3, -6 / h ** 2], [-6 / h ** 2, 4 / h]])
    V = 0.5 * w @ Qi @ w
    assert ieks.objective(np.stack([e0, e1]), Phi, sQ) == pytest.approx(V, rel=1e-12)


def test_objective_stopping_rule():
    """Affine ODE: one iteration reaches the posterior mean, so V does not change in the second
    and the objective rule (with the change rule disabled) stops there."""
    p = W.affine([[-1.0]], [1.0], [0.0], t1=3.0, N=12, q=2)
    r = ieks.ieks(p, atol=-1.0, max_iter=10, obj_atol=1e-9, obj_rtol=1e-6, want_cov=False,
                  calibrate=False)
    assert r.iterations == 2
    assert len(r.objectives) == 3
    assert abs(r.objectives[2] - r.objectives[1]) <= 1e-9
    assert r.objectives[0] > r.objectives[1]


# ---- coarse-grid initial trajectory (Section 3.2.2, remark on the initial trajectory) ------------
def test_coarse_initial_trajectory_special_cases():
    """coarse_n = N: the trajectory is the sequential EKS itself (tau = 0 at every node).
    Affine ODE: the coarse EKS is exact at its nodes, and between nodes the trajectory is the
    prior mean Phi(tau) m_k; one IEKS iteration from any start reaches the posterior."""
    p = W.van_der_pol(N=40, q=2)
    traj = ieks.coarse_initial_trajectory(p, 40)
    ms, _, _ = eks.eks(p, calibrate=False)
    np.testing.assert_allclose(traj, ms, rtol=0, atol=1e-13)
    # nodes of a coarser grid coincide with every (N / coarse_n)-th fine point
    traj4 = ieks.coarse_initial_trajectory(p, 8)
    import dataclasses
    ms8, _, _ = eks.eks(dataclasses.replace(p, N=8), calibrate=False)
    np.testing.assert_allclose(traj4[::5], ms8, rtol=0, atol=1e-13)
    # between nodes: the Taylor shift of the node's state (tau = 2 h after node 1)
    from oracle.prior import iwp_transition
    Phi2, _ = iwp_transition(p.q, 2 * p.h, p.d)
    np.testing.assert_allclose(traj4[7], Phi2 @ ms8[1], rtol=1e-14, atol=1e-14)
    a = W.affine([[-1.0]], [1.0], [0.0], t1=3.0, N=12, q=2)
    r1 = ieks.ieks(a, fixed_iters=1, want_cov=False, calibrate=False)
    r2 = ieks.ieks(a, fixed_iters=1, want_cov=False, calibrate=False, coarse_n=3)
    np.testing.assert_allclose(r1.means, r2.means, rtol=0, atol=1e-12)


def test_coarse_init_converges_to_the_same_fixed_point_in_fewer_iterations():
    p = W.fitzhugh_nagumo(N=400, q=3)
    a = ieks.ieks(p, atol=1e-10, max_iter=80, want_cov=False, calibrate=False)
    b = ieks.ieks(p, atol=1e-10, max_iter=80, want_cov=False, calibrate=False, coarse_n=100)
    assert b.iterations < a.iterations
    np.testing.assert_allclose(a.means[:, 0::4], b.means[:, 0::4], rtol=0, atol=1e-8)
