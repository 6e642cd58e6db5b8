"""GPU parity of the large-state solver (one thread block per chain, block-level dense tria and
products; any d with D = d (q+1) <= 256) against the FP64 oracle, and against the lane-group
kernels where both apply.

Bars as in test_gpu_parity.py: FP64 means 1e-10 and covariances (S S^T) 1e-8 relative; FP32
solution means 1e-5 and covariances 1e-3 at convergence.  Chain lengths are chosen so that the
trees have padded levels and the chain that owns n = N sometimes has no leaves.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402
from oracle import ieks  # noqa: E402


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


@pytest.mark.parametrize("tcores", [0, 2], ids=["fp64-pipe", "tensor-cores"])
@pytest.mark.parametrize("d,N,chain_len", [(8, 40, 0), (8, 41, 3), (16, 25, 4), (64, 12, 0),
                                           (64, 13, 5)])
def test_lorenz96_fixed_iterations_fp64(pit, d, N, chain_len, tcores):
    """Lorenz-96 (d = 64: D = 192) per iteration against the oracle's sequential IEKS, with the
    D x D products on the FP64 pipes and as exact digit products on the tensor cores (forced for
    every D here; by default only for D >= 64)."""
    p = W.lorenz96(d=d, N=N, q=2)
    orc = ieks.ieks(p, fixed_iters=2, want_cov=True, calibrate=True)
    r = pit.solve_problem(p, dtype=torch.float64, fixed_iters=2, want_cov=True,
                          chain_len=chain_len, tensor_cores=tcores)
    torch.cuda.synchronize()
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    assert r.sigma2 == pytest.approx(orc.sigma2, rel=1e-9)


@pytest.mark.parametrize("d,N", [(8, 300), (64, 40)])
def test_lorenz96_converged(pit, d, N):
    """Converged solves: FP64 takes the oracle's iterations and matches it; FP32 (scans on the
    Gauss-Newton increment, double-float trajectory) matches it at the FP32 bars."""
    p = W.lorenz96(d=d, N=N, q=2)
    orc = ieks.ieks(p, atol=1e-10, max_iter=30, want_cov=True, calibrate=True)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=30, want_cov=True)
    r32 = pit.solve_problem(p, dtype=torch.float32, fixed_iters=orc.iterations + 2,
                            want_cov=True)
    torch.cuda.synchronize()
    assert r.converged and r.iterations == orc.iterations
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    ys = slice(0, None, p.q + 1)
    assert rel(_np(r32.mean)[:, ys], orc.means[:, ys]) < 1e-5
    assert rel(cov(_np(r32.sqrtcov)), cov(orc.sqrtcovs)) < 1e-3


@pytest.mark.parametrize("p,tm", [(W.fitzhugh_nagumo(N=301, q=3), 1e-9), (W.logistic(N=97, q=2), 1e-10),
                                  (W.rigid_body(N=150, q=2), 1e-10), (W.van_der_pol(N=64, q=1), 1e-10)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_large_state_solver_equals_lane_group_kernels(pit, p, tm):
    """variant 3 forces the large-state solver for d <= 3: the same iterates as the lane-group
    kernels (and the oracle) in FP64.  FitzHugh-Nagumo's third iterate from the constant start
    (values up to 1.5e4) carries the 1e-9 means bar of the element-scan parity tests."""
    a = pit.solve_problem(p, dtype=torch.float64, fixed_iters=3, want_cov=True, variant=3)
    b = pit.solve_problem(p, dtype=torch.float64, fixed_iters=3, want_cov=True)
    torch.cuda.synchronize()
    orc = ieks.ieks(p, fixed_iters=3, want_cov=True, calibrate=True)
    for r in (a, b):
        assert rel(_np(r.mean), orc.means) < tm
        assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    for r in (a, b):
        assert r.sigma2 == pytest.approx(orc.sigma2, rel=10 * tm)


def test_affine_one_iteration_is_exact(pit):
    """An affine ODE (d = 5, D = 10): the first iteration is the exact linear smoother, so the
    second does not move it (Section 3.1)."""
    rng = np.random.Generator(np.random.PCG64(3))
    d = 5
    L = rng.standard_normal((d, d)) * 0.5 - np.eye(d)
    p = W.affine(L, rng.standard_normal(d), rng.standard_normal(d), t1=2.0, N=33, q=1)
    orc = ieks.ieks(p, fixed_iters=1, want_cov=True, calibrate=True)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=2, atol_delta=0.0, want_cov=True,
                          chain_len=4)
    torch.cuda.synchronize()
    assert r.iterations == 2
    assert r.deltas[1] <= 1e-11 * np.max(np.abs(orc.means))
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8


@pytest.mark.parametrize("p,dtype,tm", [(W.lorenz96(d=8, N=30, q=2), torch.float64, 1e-10),
                                        (W.lorenz96(d=64, N=12, q=2), torch.float64, 1e-10),
                                        (W.lorenz96(d=16, N=200, q=2, F=0.5), torch.float32, 1e-5)],
                         ids=["l96_d8_f64", "l96_d64_f64", "l96_d16_F05_f32"])
def test_sequential_eks(pit, p, dtype, tm):
    """The sequential EKS (local linearisation at the predicted mean, one block walking all
    steps) against the oracle's.  The FP32 case uses the forcing F = 0.5, whose equilibrium is
    stable: at F = 8 Lorenz-96 is chaotic and its linearisation at the initial state grows like
    e^(8 t), so FP32 rounding of any solve is amplified far beyond 1e-5 (8.9e-5 on [0, 1], 1.7e-2
    on [0, 5] against the FP64 oracle, measured on GB300)."""
    from oracle import eks as oeks
    ms, sPs, _ = oeks.eks(p, calibrate=False)
    _, _, s2 = oeks.eks(p, calibrate=True)
    r = pit.pit_eks_sequential(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                               pit.make_opts(dtype=dtype, calibrate=False))
    rc = pit.pit_eks_sequential(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                                pit.make_opts(dtype=dtype, want_cov=False))
    torch.cuda.synchronize()
    ys = slice(0, None, p.q + 1)
    assert rel(_np(r.mean)[:, ys], ms[:, ys]) < tm
    assert rel(cov(_np(r.sqrtcov)), cov(sPs)) < (1e-8 if dtype == torch.float64 else 1e-3)
    # the sequential EKS runs the plain (not the increment) model: in FP32 its innovations
    # H m- - d cancel terms of the size of the state, which the diffusion estimate inherits
    assert rc.sigma2 == pytest.approx(s2, rel=1e-8 if dtype == torch.float64 else 1e-2)


def test_sequential_eks_equals_lane_group_kernels(pit):
    p = W.fitzhugh_nagumo(N=200, q=3)
    a = pit.pit_eks_sequential(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                               pit.make_opts(dtype=torch.float64, variant=3))
    b = pit.pit_eks_sequential(pit.ode_from_problem(p), p.y0, p.t0, p.t1, p.N, p.q,
                               pit.make_opts(dtype=torch.float64))
    torch.cuda.synchronize()
    assert rel(_np(a.mean), _np(b.mean)) < 1e-10
    assert rel(cov(_np(a.sqrtcov)), cov(_np(b.sqrtcov))) < 1e-8


@pytest.mark.parametrize("N,nc", [(60, 15), (61, 61)])
def test_coarse_initial_trajectory(pit, N, nc):
    """Coarse-grid start (sequential EKS on nc steps, prior-mean interpolation) against the
    oracle's, two IEKS iterations, Lorenz-96 d = 8."""
    p = W.lorenz96(d=8, N=N, q=2)
    orc = ieks.ieks(p, fixed_iters=2, want_cov=True, calibrate=True, coarse_n=nc)
    r = pit.solve_problem(p, dtype=torch.float64, fixed_iters=2, want_cov=True, init_coarse=nc)
    torch.cuda.synchronize()
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8


def test_large_state_rejections(pit):
    p = W.lorenz96(d=8, N=10, q=2)
    with pytest.raises(pit.PitError) as ei:
        pit.solve_problem(p, dtype=torch.float64, objective=1)
    assert ei.value.status == 8
    with pytest.raises(pit.PitError) as ei:
        pit.solve_problem(p, dtype=torch.float64, init_coarse=11)
    assert ei.value.status == 1


def _golden(N):
    import os
    return np.load(os.path.join(os.path.dirname(__file__), "golden", f"lorenz96_d64_N{N}_it1.npz"))


def _bar(g):
    """1e-10, or 10x the oracle's own change when every entry of its initial trajectory is
    perturbed by a relative 1e-15 (stored with the fixture), whichever is larger: on this chaotic
    workload rounding-level differences of the computation order grow by orders of magnitude
    over [0, 5], so a bar below that sensitivity would test rounding, not the method."""
    return max(1e-10, 10.0 * float(g["sens"]))


@pytest.mark.parametrize("N", [4096])
def test_lorenz96_full_size_kernels(pit, N):
    """The benchmark's Lorenz-96 workload (d = 64, D = 192, FP64) at full size with the large-state
    kernels run as one chain (the sequential square-root filter and smoother, no tree): the first
    IEKS iterate at sampled grid points, its maximal change and diffusion estimate against the
    oracle's (tests/golden/make_lorenz96_first_iterate.py); measured 2.4e-11 at N = 4096 and
    3.8e-11 at N = 16384 (one block walking 16384 FP64 steps takes about 4 minutes, so the suite
    runs the 4096-step case)."""
    g = _golden(N)
    p = W.lorenz96(d=64, N=N, q=2)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=1, atol_delta=0.0, want_cov=False,
                          chain_len=N)
    torch.cuda.synchronize()
    assert rel(_np(r.mean)[g["n"]], g["means"]) < _bar(g)
    assert r.deltas[0] == pytest.approx(float(g["delta"]), rel=_bar(g))
    assert r.sigma2 == pytest.approx(float(g["sigma2"]), rel=1e-9)


@pytest.mark.parametrize("tcores", [0, 1], ids=["fp64-pipe", "tensor-cores"])
@pytest.mark.parametrize("N", [4096, 16384])
def test_lorenz96_full_size_parallel_shape(pit, N, tcores):
    """The same first iterate in the benchmark's launch shape (about one chain per SM, the chain
    aggregates combined by tree levels inside groups of 8 and a sequential look-back across the
    groups).  On this chaotic workload (linearisation growing like e^(8 t)) a tree over all
    chains combined elements whose flow maps spanned most of [0, 5] and missed the oracle by
    2.7e-6 (N = 4096) and 2.9e-4 (N = 16384); with span-limited combines the parallel result
    keeps the FP64 bar.  Both with the D x D products on the FP64 pipes and as exact digit
    products on the tensor cores: the two orders of rounding give 7.7e-11 and 1.0e-10 at
    N = 16384, a spread the oracle's own sensitivity to rounding-level perturbations (_bar)
    accounts for."""
    g = _golden(N)
    p = W.lorenz96(d=64, N=N, q=2)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=1, atol_delta=0.0, want_cov=False,
                          tensor_cores=tcores)
    torch.cuda.synchronize()
    assert rel(_np(r.mean)[g["n"]], g["means"]) < _bar(g)
    assert r.deltas[0] == pytest.approx(float(g["delta"]), rel=_bar(g))
    assert r.sigma2 == pytest.approx(float(g["sigma2"]), rel=1e-9)


# ---- generic element scans on the large-state kernels (D outside the lane-group set) -----------
def _elements(p):
    from oracle import filtering
    from oracle.taylor import initial_state
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
    (W.lorenz96(d=8, N=300, q=2), torch.float64, 1e-10, 1e-10),
    (W.lorenz96(d=16, N=77, q=2), torch.float64, 1e-10, 1e-10),
    (W.affine([[-1.0, 0.3, 0.0, 0.2, 0.1], [0.1, -0.5, 0.2, 0.0, 0.0], [0.0, 0.1, -0.7, 0.3, 0.0],
               [0.0, 0.0, 0.2, -0.4, 0.1], [0.2, 0.0, 0.0, 0.1, -0.9]],
              [0.1, -0.2, 0.3, 0.0, 0.5], [1.0, 0.5, -0.5, 0.2, 0.0], t1=3.0, N=500, q=2),
     torch.float64, 1e-10, 1e-10),
    (W.lorenz96(d=8, N=300, q=2, F=0.5), torch.float32, 1e-4, 1e-4),
], ids=["l96_d8_f64", "l96_d16_f64", "affine_d5_f64", "l96_d8_F05_f32"])
def test_filter_and_smooth_scans_large_state(pit, p, dtype, tm, tc):
    """pit_filter_scan / pit_smooth_scan for D = 24, 48, 15 (the large-state kernels) on
    elements the oracle builds (Eqs. sqrt-filtering-elements, sqrt-smoothing-elements): the
    prefixes are the oracle's sequential filter and smoother marginals."""
    el, mf, sPf, be, ms, sPs = _elements(p)
    dev = "cuda"
    T = lambda k: torch.tensor(np.stack([e[k] for e in el[1:]]), dtype=dtype, device=dev)
    A, b, C, eta, J = (T(k) for k in range(5))
    pit.pit_filter_scan(A, b, C, eta, J)
    torch.cuda.synchronize()
    assert rel(_np(b), mf[1:]) < tm
    assert rel(cov(_np(C)), cov(sPf[1:])) < tc
    U = lambda k: torch.tensor(np.stack([x[k] for x in be]), dtype=dtype, device=dev)
    E, g, L = U(0), U(1), U(2)
    pit.pit_smooth_scan(E, g, L)
    torch.cuda.synchronize()
    assert rel(_np(g), ms) < tm
    assert rel(cov(_np(L)), cov(sPs)) < tc
    E2, g2 = U(0), U(1)
    pit.pit_smooth_scan(E2, g2, None)
    torch.cuda.synchronize()
    assert rel(_np(g2), ms) < tm


@pytest.mark.parametrize("p", [W.lorenz96(d=8, N=50, q=2), W.lorenz96(d=64, N=20, q=2),
                               W.affine([[-1.0, 0.2, 0.0, 0.1], [0.3, -0.5, 0.1, 0.0],
                                         [0.0, 0.2, -0.3, 0.1], [0.1, 0.0, 0.2, -0.8]],
                                        [0.1, 0.2, -0.1, 0.0], [1.0, 0.0, 0.5, -0.5], N=30, q=3)],
                         ids=["l96_d8", "l96_d64", "affine_d4"])
def test_linearize_any_d(pit, p):
    """pit_linearize for d > 3 (H_n = E1 - F E0, d_n = f - F y; Section 3.2.1) against the
    oracle's, at a random trajectory."""
    rng = np.random.default_rng(1)
    traj = rng.standard_normal((p.N + 1, p.D))
    Hs, ds = ieks.linearize_all(p, traj)
    H, dv = pit.pit_linearize(pit.ode_from_problem(p), p.t0, p.t1, p.N, p.q,
                              torch.tensor(traj, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    np.testing.assert_allclose(H.cpu().numpy(), np.stack(Hs[1:]), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(dv.cpu().numpy(), np.stack(ds[1:]), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("d,N", [(8, 200), (64, 30)])
def test_tensor_core_products_converged_and_sequential(pit, d, N):
    """Converged FP64 solves and the sequential EKS with the products on the tensor cores take
    the oracle's iterations and match it at the FP64 bars."""
    p = W.lorenz96(d=d, N=N, q=2)
    orc = ieks.ieks(p, atol=1e-10, max_iter=30, want_cov=True, calibrate=True)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=30, want_cov=True, tensor_cores=2)
    torch.cuda.synchronize()
    assert r.converged and r.iterations == orc.iterations
    assert rel(_np(r.mean), orc.means) < 1e-10
    assert rel(cov(_np(r.sqrtcov)), cov(orc.sqrtcovs)) < 1e-8
    assert r.sigma2 == pytest.approx(orc.sigma2, rel=1e-9)
