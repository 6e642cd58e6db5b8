"""Pins of the oracle on non-uniform grids (Sections 2.3 and 3.1 state the method on a general
grid, with the IWP transitions of Section 2.1 for each step length)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import eks, gp, ieks


def test_explicit_uniform_grid_equals_uniform():
    """A grid given point by point with equal steps reproduces the uniform-grid solve."""
    p = W.van_der_pol(N=30, q=2)
    pg = W.on_grid(p, p.t0 + p.h * np.arange(p.N + 1))
    a = ieks.ieks(p, fixed_iters=3)
    b = ieks.ieks(pg, fixed_iters=3)
    assert np.max(np.abs(a.means - b.means)) <= 1e-12 * np.max(np.abs(a.means))
    assert np.max(np.abs(a.sqrtcovs @ a.sqrtcovs.transpose(0, 2, 1)
                         - b.sqrtcovs @ b.sqrtcovs.transpose(0, 2, 1))) <= 1e-12
    assert b.sigma2 == pytest.approx(a.sigma2, rel=1e-12)


@pytest.mark.parametrize("ratio", [0.1, 8.0])
def test_affine_graded_grid_equals_dense_conditioning(ratio):
    """Affine ODE on a graded grid: one IEKS iteration is the exact posterior of the
    non-uniform Markov prior conditioned on the ODE at every grid point (a dense solve of the
    joint Gaussian built from the per-step transitions), with the exact MLE diffusion; the
    second iteration does not move."""
    rng = np.random.Generator(np.random.PCG64(11))
    d = 2
    L = rng.standard_normal((d, d)) * 0.4 - 0.5 * np.eye(d)
    p = W.affine(L, rng.standard_normal(d), rng.standard_normal(d), t1=2.0, N=11, q=2)
    p = W.on_grid(p, W.graded_grid(0.0, 2.0, 11, ratio))
    r = ieks.ieks(p, fixed_iters=2, calibrate=True, record_iterates=True)
    means, covs, s2 = gp.dense_posterior(p)
    scale = np.max(np.abs(means))
    assert np.max(np.abs(r.iterates[0] - means)) <= 1e-9 * scale
    assert np.max(np.abs(r.iterates[1] - r.iterates[0])) <= 1e-9 * scale
    P = r.sqrtcovs @ r.sqrtcovs.transpose(0, 2, 1)
    assert np.max(np.abs(P - s2 * covs)) <= 1e-8 * np.max(np.abs(s2 * covs))
    assert r.sigma2 == pytest.approx(s2, rel=1e-8)


def test_graded_grid_dense_posterior_differs_from_uniform():
    """The grid matters: the same affine problem on a uniform and on a graded grid gives
    different posteriors at the shared end point (guards against a grid that is silently
    ignored)."""
    p = W.affine([[-1.0]], [1.0], [0.0], t1=2.0, N=8, q=1)
    pg = W.on_grid(p, W.graded_grid(0.0, 2.0, 8, 6.0))
    a = ieks.ieks(p, fixed_iters=1)
    b = ieks.ieks(pg, fixed_iters=1)
    assert abs(a.means[-1, 0] - b.means[-1, 0]) > 1e-6


def test_logistic_graded_grids_converge():
    """Logistic (rate 1) on grids refined near t = 0 (ratio 8): the error against the analytic
    solution falls by at least 2^q per halving of the steps (q = 2)."""
    errs = []
    for N in (40, 80, 160):
        p = W.on_grid(W.logistic_paper(N=N, q=2), W.graded_grid(0.0, 10.0, N, 8.0))
        r = ieks.ieks(p, atol=1e-12, max_iter=40)
        t = p.times
        exact = 1.0 / (1.0 + (1.0 / 0.01 - 1.0) * np.exp(-t))
        errs.append(np.max(np.abs(r.means[:, 0] - exact)))
    assert errs[1] < errs[0] / 4 and errs[2] < errs[1] / 4


def test_sequential_eks_graded_affine_is_exact():
    """The sequential EKS is exact on affine problems on any grid."""
    p = W.affine([[-0.7, 0.3], [-0.2, -0.4]], [0.5, -1.0], [1.0, 2.0], t1=3.0, N=10, q=1)
    p = W.on_grid(p, W.graded_grid(0.0, 3.0, 10, 0.2))
    ms, sPs, s2 = eks.eks(p)
    means, covs, s2d = gp.dense_posterior(p)
    assert np.max(np.abs(ms - means)) <= 1e-9 * np.max(np.abs(means))
    assert s2 == pytest.approx(s2d, rel=1e-8)
