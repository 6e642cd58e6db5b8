"""GPU parity on non-uniform grids (pit_solve_grid with per-step preconditioning: the lane-group
kernels for d <= 3, the large-state kernels for d > 3 or variant 3) against the FP64 oracle's
per-step IWP transitions.  Bars as in test_gpu_parity.py."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from oracle import gp, ieks  # noqa: E402


@pytest.fixture(scope="module")
def pit():
    import paper_2310_01145_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    P.load()
    return P


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, np.max(np.abs(b))))


def cov(s):
    return np.einsum("nij,nkj->nik", s, s)


def _np(t):
    return t.double().cpu().numpy()


def graded(p, ratio):
    return W.on_grid(p, W.graded_grid(p.t0, p.t1, p.N, ratio))


@pytest.mark.parametrize("p,tm,chain_len", [
    (graded(W.lorenz96(d=8, N=40, q=2), 0.25), 1e-10, 0),
    (graded(W.lorenz96(d=8, N=41, q=2), 4.0), 1e-10, 3),
    (graded(W.fitzhugh_nagumo(N=301, q=3), 0.3), 1e-9, 0),
    (graded(W.van_der_pol(N=120, q=1), 5.0), 1e-10, 7),
    (graded(W.logistic(N=97, q=2), 0.1), 1e-10, 0),
], ids=lambda x: getattr(x, "name", str(x)))
@pytest.mark.parametrize("variant", [0, 3], ids=["lane-group", "large-state"])
def test_fixed_iterations_fp64(pit, p, tm, chain_len, variant):
    orc = ieks.ieks(p, fixed_iters=2, want_cov=True, calibrate=True)
    r = pit.solve_problem(p, dtype=torch.float64, fixed_iters=2, want_cov=True,
                          chain_len=chain_len, variant=variant)
    torch.cuda.synchronize()
    assert rel(_np(r.mean), orc.means) < tm
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    assert r.sigma2 == pytest.approx(orc.sigma2, rel=10 * tm)


def test_affine_one_iteration_is_the_dense_posterior(pit):
    """Affine ODE on a graded grid: the first iteration equals dense Gaussian conditioning of the
    non-uniform Markov prior, and the second does not move."""
    rng = np.random.Generator(np.random.PCG64(11))
    d = 2
    L = rng.standard_normal((d, d)) * 0.4 - 0.5 * np.eye(d)
    p = graded(W.affine(L, rng.standard_normal(d), rng.standard_normal(d), t1=2.0, N=11, q=2), 8.0)
    means, covs, s2 = gp.dense_posterior(p)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=2, atol_delta=0.0, want_cov=True)
    torch.cuda.synchronize()
    assert r.iterations == 2 and r.deltas[1] <= 1e-11 * np.max(np.abs(means))
    assert rel(_np(r.mean), means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), s2 * covs) < 1e-8
    assert r.sigma2 == pytest.approx(s2, rel=1e-9)


def test_converged_fp64_and_fp32(pit):
    """Logistic (rate 1) on a grid refined near t = 0: the converged solve takes the oracle's
    iterations; FP32 (FP64 trajectory, per-step scale factors in FP64 in the residuals) meets
    the FP32 bar."""
    p = graded(W.logistic_paper(N=400, q=2), 8.0)
    orc = ieks.ieks(p, atol=1e-10, max_iter=40, want_cov=True)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=40, want_cov=True)
    r32 = pit.solve_problem(p, dtype=torch.float32, fixed_iters=orc.iterations + 2,
                            want_cov=True)
    torch.cuda.synchronize()
    assert r.converged and r.iterations == orc.iterations
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(_np(r32.mean)[:, 0::3], orc.means[:, 0::3]) < 1e-5
    assert rel(cov(_np(r32.sqrtcov)), cov(orc.sqrtcovs)) < 1e-3


@pytest.mark.parametrize("variant", [0, 3], ids=["lane-group", "large-state"])
def test_explicit_uniform_grid_equals_uniform_solve(pit, variant):
    """An explicit grid with equal steps reproduces the uniform solve of the same kernels (the
    per-point scales are 1 and the per-point preconditioner is the constant one)."""
    p = W.van_der_pol(N=200, q=2)
    pg = W.on_grid(p, p.t0 + p.h * np.arange(p.N + 1))
    a = pit.solve_problem(pg, dtype=torch.float64, fixed_iters=3, want_cov=True, variant=variant,
                          scan=1)
    b = pit.solve_problem(p, dtype=torch.float64, fixed_iters=3, want_cov=True, variant=variant,
                          scan=1)
    torch.cuda.synchronize()
    assert rel(_np(a.mean), _np(b.mean)) < 1e-13
    assert rel(cov(_np(a.sqrtcov)), cov(_np(b.sqrtcov))) < 1e-12


@pytest.mark.parametrize("p", [graded(W.fitzhugh_nagumo(N=400, q=3), 0.3),
                               graded(W.van_der_pol(N=300, q=2), 6.0),
                               graded(W.rigid_body(N=200, q=2), 0.2)],
                         ids=lambda x: x.name)
def test_lane_kernels_converged_fp64_fp32(pit, p):
    """d = 2 and 3 on graded grids with the lane-group kernels: FP64 converges in the oracle's
    iterations to its fixed point (1e-10), FP32 meets the FP32 bars there."""
    orc = ieks.ieks(p, atol=1e-10, max_iter=60, want_cov=True)
    assert orc.deltas[-1] <= 1e-10
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=60, want_cov=True)
    r32 = pit.solve_problem(p, dtype=torch.float32, fixed_iters=orc.iterations + 2,
                            want_cov=True)
    torch.cuda.synchronize()
    assert r.converged and r.iterations == orc.iterations
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    ys = slice(0, None, p.q + 1)
    assert rel(_np(r32.mean)[:, ys], orc.means[:, ys]) < 1e-5
    assert rel(cov(_np(r32.sqrtcov)), cov(orc.sqrtcovs)) < 1e-3


def test_grid_rejections(pit):
    p = graded(W.lorenz96(d=8, N=20, q=2), 2.0)
    with pytest.raises(pit.PitError) as ei:
        pit.solve_problem(p, dtype=torch.float64, init_coarse=5)
    assert ei.value.status == 8
