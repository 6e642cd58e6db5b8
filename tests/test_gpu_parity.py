"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (relative errors as max_n |x_gpu - x_orc| / max_n |x_orc| per quantity):
  FP64: means 1e-10, covariances (S S^T) 1e-8.
  FP32: solution means E0 m 1e-5 on problems of modest length, covariances 1e-3; the full
  state in preconditioned FP32 is compared with 1e-4 (higher derivatives are the
  least accurate components).
Covariances are compared as S S^T: tria's factor is unique only up to column signs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from oracle import eks as oeks  # noqa: E402
from oracle import filtering, gp, ieks  # noqa: E402
from oracle.taylor import initial_state  # noqa: E402


@pytest.fixture(scope="module")
def pit():
    import paper_2310_01145_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    P.load()
    return P


DEV = "cuda"
U32 = 2.0 ** -24   # unit roundoff of FP32


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(1e-300, np.max(np.abs(b))))


def cov(s):
    return np.einsum("nij,nkj->nik", s, s)


def ysl(p):
    return slice(0, None, p.q + 1)


def solve(pit, p, dtype, **kw):
    r = pit.solve_problem(p, dtype=dtype, **kw)
    torch.cuda.synchronize()
    return r


# ---------------------------------------------------------------------------------------------
# element scans (pit_filter_scan / pit_smooth_scan) on oracle-built elements
# ---------------------------------------------------------------------------------------------
def _elements(p):
    D, q, N = p.D, p.q, p.N
    Phi, Q, sQ = ieks.prior_factors(p)
    mu0 = initial_state(p.kind, p.params, p.y0, q)
    Hs, ds = ieks.linearize_all(p, np.tile(mu0, (N + 1, 1)))
    el = filtering.filtering_elements(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    mf, sPf, _, _ = filtering.sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    ms, sPs = filtering.rts_smoother(mf, sPf, Phi, sQ)
    be = filtering.smoothing_elements(mf, sPf, Phi, sQ)
    return el, mf, sPf, be, ms, sPs


@pytest.mark.parametrize("p,dtype,tm,tc", [
    (W.logistic(N=37, q=2), torch.float64, 1e-12, 1e-12),
    (W.logistic_paper(N=2500, q=2), torch.float64, 1e-10, 1e-10),
    (W.fitzhugh_nagumo(N=301, q=3), torch.float64, 1e-10, 1e-10),
    (W.van_der_pol(N=777, q=2), torch.float64, 1e-10, 1e-10),
    (W.van_der_pol(N=777, q=1), torch.float32, 2 * 777 * U32, 2 * 777 * U32),
    (W.van_der_pol(N=3000, q=2), torch.float32, 2 * 3000 * U32, 2 * 3000 * U32),
], ids=lambda x: getattr(x, "name", str(x)))
def test_filter_and_smooth_scans(pit, p, dtype, tm, tc):
    """The element scans on caller-built elements in original coordinates.  FP64: 1e-10.  FP32:
    2 N u32 (u32 = 2^-24): these entry points have no preconditioning and no increment
    formulation, each of the ~2N combines rounds at u32, and the error grows linearly in N
    (measured on GB300 for Van der Pol IWP(1)/IWP(2): 6e-6 / 3e-5 at N = 1000, 3e-5 / 3e-4 at
    N = 10^4)."""
    el, mf, sPf, be, ms, sPs = _elements(p)
    T = lambda k: torch.tensor(np.stack([e[k] for e in el[1:]]), dtype=dtype, device=DEV)
    A, b, C, eta, J = (T(k) for k in range(5))
    pit.pit_filter_scan(A, b, C, eta, J)
    torch.cuda.synchronize()
    assert rel(b.cpu().double().numpy(), mf[1:]) < tm
    assert rel(cov(C.cpu().double().numpy()), cov(sPf[1:])) < tc
    U = lambda k: torch.tensor(np.stack([x[k] for x in be]), dtype=dtype, device=DEV)
    E, g, L = U(0), U(1), U(2)
    pit.pit_smooth_scan(E, g, L)
    torch.cuda.synchronize()
    assert rel(g.cpu().double().numpy(), ms) < tm
    assert rel(cov(L.cpu().double().numpy()), cov(sPs)) < tc
    # means-only variant
    E2, g2 = U(0), U(1)
    pit.pit_smooth_scan(E2, g2, None)
    torch.cuda.synchronize()
    assert rel(g2.cpu().double().numpy(), ms) < tm


# ---------------------------------------------------------------------------------------------
# ParaIEKS per iteration (same linearisation trajectory on both sides)
# ---------------------------------------------------------------------------------------------
FP64_CASES = [
    (W.logistic(N=64, q=2), 3, 0),
    (W.logistic_paper(N=200, q=1), 5, 3),
    (W.fitzhugh_nagumo(N=333, q=2), 3, 11),
    (W.van_der_pol(N=100, q=3), 4, 7),
    (W.rigid_body(N=150, q=2), 3, 5),
    (W.rigid_body(N=90, q=1), 3, 0),
    (W.fitzhugh_nagumo(N=400, q=3), 42, 0),     # runs to the oracle's convergence
]


@pytest.mark.parametrize("p,iters,L", FP64_CASES, ids=lambda x: getattr(x, "name", str(x)))
def test_solve_fp64_matches_oracle(pit, p, iters, L):
    ref = ieks.ieks(p, fixed_iters=iters)
    r = solve(pit, p, torch.float64, fixed_iters=iters, chain_len=L)
    m = r.mean.cpu().numpy()
    assert rel(m, ref.means) < 1e-10
    assert rel(cov(r.sqrtcov.cpu().numpy()), cov(ref.sqrtcovs)) < 1e-8
    assert r.sigma2 == pytest.approx(ref.sigma2, rel=1e-9)
    assert r.iterations == iters


@pytest.mark.parametrize("p,iters", [(W.fitzhugh_nagumo(N=512, q=3), 3),
                                     (W.lotka_volterra(N=257, q=2), 3),
                                     (W.logistic(N=1024, q=2), 4)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_solve_fp64_early_iterates(pit, p, iters):
    """Early Gauss-Newton iterates from the constant initial trajectory: the linearised models
    are far from the solution (FitzHugh-Nagumo needs about 40 iterations on [0, 20], the
    Lotka-Volterra problem does not converge on this grid, the rate-3 logistic model grows by
    e^29 in its first linearisation), so the FP64 agreement is limited by their conditioning
    rather than by the arithmetic of either side."""
    ref = ieks.ieks(p, fixed_iters=iters)
    r = solve(pit, p, torch.float64, fixed_iters=iters)
    assert rel(r.mean.cpu().numpy(), ref.means) < 1e-7
    assert rel(cov(r.sqrtcov.cpu().numpy()), cov(ref.sqrtcovs)) < 1e-7


@pytest.mark.parametrize("N,L", [(1, 0), (2, 0), (5, 1), (12, 4), (13, 4), (64, 64), (64, 65),
                                 (100, 7)])
def test_solve_edge_sizes(pit, N, L):
    """Tiny grids, chain length 1, N a multiple of the chain length (the last chain then holds
    only b_N), a single chain covering everything."""
    p = W.van_der_pol(N=N, q=2)
    ref = ieks.ieks(p, fixed_iters=2)
    r = solve(pit, p, torch.float64, fixed_iters=2, chain_len=L)
    assert rel(r.mean.cpu().numpy(), ref.means) < 1e-10
    assert rel(cov(r.sqrtcov.cpu().numpy()), cov(ref.sqrtcovs)) < 1e-8


@pytest.mark.parametrize("p", [W.van_der_pol(N=255, q=2), W.van_der_pol(N=256, q=2),
                               W.van_der_pol(N=511, q=2), W.van_der_pol(N=127, q=3),
                               W.van_der_pol(N=128, q=3), W.van_der_pol(N=385, q=3)],
                         ids=lambda x: f"{x.name}-{x.N}-q{x.q}")
def test_residual_tile_boundaries(pit, p):
    """The residual kernel works on tiles of 256 time points (128 for FP64 with D = 8): N + 1
    exactly one or two tiles, a last tile holding only the final point, a ragged last tile.
    The bar is ten times the oracle's own sensitivity to a 1e-15 relative perturbation of its
    initial trajectory (at least 1e-10, at most 1e-9): the second Gauss-Newton iterate of the
    q = 3 model on the finest of these grids moves by ~2e-11 under that perturbation."""
    ref = ieks.ieks(p, fixed_iters=2)
    rng = np.random.default_rng(0)
    pert = np.tile(ref.mu0, (p.N + 1, 1)) * (1 + 1e-15 * rng.standard_normal((p.N + 1, p.D)))
    sens = rel(ieks.ieks(p, fixed_iters=2, init_traj=pert).means, ref.means)
    bar = min(1e-9, max(1e-10, 10 * sens))
    r = solve(pit, p, torch.float64, fixed_iters=2)
    assert rel(r.mean.cpu().numpy(), ref.means) < bar
    assert rel(cov(r.sqrtcov.cpu().numpy()), cov(ref.sqrtcovs)) < 1e-8
    if p.q == 2:
        conv = ieks.ieks(p, max_iter=60)
        r32 = solve(pit, p, torch.float32, fixed_iters=conv.iterations)
        m = r32.mean.cpu().double().numpy()
        assert rel(m[:, ysl(p)], conv.means[:, ysl(p)]) < 1e-5


def test_logistic_config_converges_like_oracle(pit):
    """logistic r = 3, y0 = 0.01, [0, 10], q = 2, N = 1024, FP64, stop at max|dy| < 1e-10 or
    20 iterations.  From the constant initial trajectory both reach the same fixed point."""
    p = W.logistic(N=1024, q=2)
    ref = ieks.ieks(p, atol=1e-10, max_iter=20)
    r = solve(pit, p, torch.float64, atol_delta=1e-10, max_iter=20)
    assert r.iterations == ref.iterations
    assert r.converged
    # both sides stop at |dy| ~ 5e-12, not yet at the fixed point; compare the fixed point
    # itself after running past convergence (quadratic phase: changes at round-off level)
    ref8 = ieks.ieks(p, fixed_iters=8)
    r8 = solve(pit, p, torch.float64, fixed_iters=8)
    m = r8.mean.cpu().numpy()
    # This fixed point is ill-conditioned (the rate-3 model grows by e^29): perturbing the
    # oracle's own initial trajectory by 1e-15 (relative) moves its result by ~6e-11.  The
    # GPU, which rounds in a different order, must agree to within a small multiple of that
    # sensitivity (and never worse than 1e-9).
    rng = np.random.default_rng(0)
    pert = np.tile(ref8.mu0, (p.N + 1, 1)) * (1 + 1e-15 * rng.standard_normal((p.N + 1, p.D)))
    sens = rel(ieks.ieks(p, fixed_iters=8, init_traj=pert).means[:, ysl(p)],
               ref8.means[:, ysl(p)])
    bar = min(1e-9, max(1e-10, 10 * sens))
    assert rel(m[:, ysl(p)], ref8.means[:, ysl(p)]) < bar        # the solution estimate
    assert rel(m, ref8.means) < 1e-8                             # whole state (diagnostic)
    assert rel(cov(r8.sqrtcov.cpu().numpy()), cov(ref8.sqrtcovs)) < 1e-8


@pytest.mark.parametrize("p", [W.logistic_paper(N=300, q=2), W.van_der_pol(N=256, q=2),
                               W.rigid_body(N=300, q=2), W.fitzhugh_nagumo(N=400, q=3)],
                         ids=lambda x: f"{x.name}-{x.N}-q{x.q}")
def test_solve_fp32_matches_oracle_at_convergence(pit, p):
    """FP32 (preconditioned coordinates) against the FP64 oracle, with the GPU running the
    oracle's iteration count to convergence.  Early Gauss-Newton iterates from the constant
    initial trajectory can be far from the solution and ill-conditioned; the FP32 bar applies to
    the converged MAP estimate."""
    ref = ieks.ieks(p, max_iter=60)
    assert ref.deltas[-1] < 1e-10
    r = solve(pit, p, torch.float32, fixed_iters=ref.iterations)
    m = r.mean.cpu().double().numpy()
    assert np.all(np.isfinite(m))
    assert rel(m[:, ysl(p)], ref.means[:, ysl(p)]) < 1e-5
    assert rel(cov(r.sqrtcov.cpu().double().numpy()), cov(ref.sqrtcovs)) < 1e-3
    assert r.sigma2 == pytest.approx(ref.sigma2, rel=1e-3)


@pytest.mark.parametrize("problem", [
    W.affine([[-1.0]], [1.0], [0.2], t1=2.0, N=6, q=2),
    W.affine([[0.0, 1.0], [-1.0, 0.0]], [0.0, 0.0], [1.0, 0.0], t1=3.0, N=5, q=2),
    W.affine([[0.3, -0.5], [0.8, -0.2]], [0.1, -0.4], [0.5, 1.0], t1=1.0, N=4, q=3),
])
def test_affine_matches_dense_gaussian_conditioning(pit, problem):
    means, covs, s2 = gp.dense_posterior(problem)
    r = solve(pit, problem, torch.float64, fixed_iters=1)
    assert rel(r.mean.cpu().numpy(), means) < 1e-9
    got = cov(r.sqrtcov.cpu().numpy())
    assert np.max(np.abs(got - covs * s2)) < 1e-9 * max(1.0, np.max(np.abs(covs * s2)))
    assert r.sigma2 == pytest.approx(s2, rel=1e-9)
    # exact inference: a second iteration does not move
    r2 = solve(pit, problem, torch.float64, fixed_iters=2)
    assert rel(r2.mean.cpu().numpy(), means) < 1e-9


def test_means_only_and_uncalibrated(pit):
    p = W.fitzhugh_nagumo(N=300, q=3)
    ref = ieks.ieks(p, fixed_iters=2, calibrate=False)
    r = solve(pit, p, torch.float64, fixed_iters=2, want_cov=False, calibrate=False)
    assert r.sqrtcov is None
    assert rel(r.mean.cpu().numpy(), ref.means) < 1e-10
    assert r.sigma2 == 1.0


def test_warm_start_trajectory(pit):
    """init_traj replaces the constant initial guess (resume / warm start)."""
    p = W.logistic(N=512, q=2)
    t = np.linspace(p.t0, p.t1, p.N + 1)
    y = 1.0 / (1.0 + (1.0 / 0.01 - 1.0) * np.exp(-3.0 * t))
    init = np.zeros((p.N + 1, p.D))
    init[:, 0] = y
    ref = ieks.ieks(p, fixed_iters=3, init_traj=init)
    init_t = torch.tensor(init, dtype=torch.float64, device=DEV)
    r = pit.pit_solve(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                      pit.make_opts(dtype=torch.float64, fixed_iters=3), init_traj=init_t)
    torch.cuda.synchronize()
    assert rel(r.mean.cpu().numpy(), ref.means) < 1e-10
    # warm start reaches the true solution of the rate-3 logistic ODE
    assert np.max(np.abs(r.mean.cpu().numpy()[:, 0] - y)) < 1e-6


def test_linearize_matches_oracle(pit):
    p = W.fitzhugh_nagumo(N=333, q=3)
    rng = np.random.default_rng(0)
    traj = rng.standard_normal((p.N + 1, p.D))
    Hs, ds = ieks.linearize_all(p, traj)
    H, dv = pit.pit_linearize(pit.ode_from_problem(p), p.t0, p.t1, p.N, p.q,
                              torch.tensor(traj, dtype=torch.float64, device=DEV))
    torch.cuda.synchronize()
    np.testing.assert_allclose(H.cpu().numpy(), np.stack(Hs[1:]), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(dv.cpu().numpy(), np.stack(ds[1:]), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p,dtype,tm", [(W.van_der_pol(N=200, q=2), torch.float64, 1e-10),
                                        (W.fitzhugh_nagumo(N=300, q=3), torch.float64, 1e-10),
                                        (W.logistic_paper(N=300, q=2), torch.float32, 1e-5)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_sequential_eks_matches_oracle(pit, p, dtype, tm):
    ms, sPs, s2 = oeks.eks(p)
    r = pit.pit_eks_sequential(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                               pit.make_opts(dtype=dtype))
    torch.cuda.synchronize()
    m = r.mean.cpu().double().numpy()
    assert rel(m[:, ysl(p)], ms[:, ysl(p)]) < tm
    assert r.sigma2 == pytest.approx(s2, rel=1e-8 if dtype == torch.float64 else 1e-3)


def test_workspace_errors(pit):
    """A workspace smaller than the query, or misaligned, is rejected before any launch."""
    import ctypes
    p = W.logistic(N=100, q=2)
    lib = pit.load()
    ode = pit.ode_from_problem(p).c()
    grid = pit._Grid(p.t0, p.t1, p.N)
    opts = pit.make_opts()
    sz = ctypes.c_size_t(0)
    assert lib.pit_solve_workspace_size(ctypes.byref(ode), ctypes.byref(grid), p.q,
                                        ctypes.byref(opts), ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value + 512, dtype=torch.uint8, device=DEV)
    mean = torch.empty((p.N + 1, p.D), dtype=torch.float64, device=DEV)
    cov = torch.empty((p.N + 1, p.D, p.D), dtype=torch.float64, device=DEV)
    y0 = np.ascontiguousarray(p.y0)
    info = pit._Info()
    args = lambda w, nbytes: (ctypes.byref(ode), ctypes.byref(grid), p.q, pit._dptr(y0),
                              ctypes.byref(opts), None, ctypes.c_void_p(mean.data_ptr()),
                              ctypes.c_void_p(cov.data_ptr()), ctypes.byref(info),
                              ctypes.c_void_p(w), nbytes, None)
    before = pit.pit_launch_count()
    assert lib.pit_solve(*args(ws.data_ptr(), sz.value - 1)) == 2
    assert lib.pit_solve(*args(ws.data_ptr() + 8, sz.value)) == 1
    assert pit.pit_launch_count() == before
    assert lib.pit_solve(*args(ws.data_ptr(), sz.value)) == 0


def test_launch_count_is_reported(pit):
    p = W.logistic(N=256, q=2)
    before = pit.pit_launch_count()
    r = solve(pit, p, torch.float64, fixed_iters=2)
    assert r.kernel_launches > 0
    assert pit.pit_launch_count() - before == r.kernel_launches
