"""Accuracy of the solver at the benchmarked shapes, against the FP64 oracle.

The benchmark workload is FitzHugh-Nagumo (d = 2, IWP(3), D = 8) on N = 2^12 .. 2^20 uniform
steps, FP32, from the constant initial trajectory to max|dy| <= 1e-10, with the launch shape the
autotuner table gives (the same call the benchmark times).  Its result is compared with the
oracle's converged solution (tests/golden/fhn_q3_N*_converged.npz, written by
tests/golden/make_fhn_q3_converged.py from oracle/ only), which the parallel method must
reproduce (Section 4.1: parallel and sequential IEKS agree numerically).  The oracle started
from the coarse-grid trajectory of Section 3.2.2 to keep it affordable; Gauss-Newton reaches the
same fixed point from either start.

Bars (relative, max over the sampled points / max |oracle|):
  FP32: solution estimate E0 m 1e-5; covariances S S^T 1e-3, also with the diffusion divided
  out (unit covariances); sigma^2 1e-3.
  FP64: solution estimate 1e-10; derivative order i of the means max(1e-10, 10 s_i), where s_i
  is the oracle's own change under a 1e-15 relative perturbation of its fixed point (stored
  with the fixture): at fine grids the higher derivatives are set by FP64 rounding; unit
  covariances (the diffusion divided out) 1e-8.  sigma^2 max(1e-9, u |y'|max / T_1(h)): the
  quasi-MLE diffusion (Section 2.4) is a mean of squared innovations normalised by sqrt(S_n),
  whose scale is T_1(h) = sqrt(h) h^(q-1) / (q-1)!; one FP64 ulp (u = 2^-53) of a derivative
  of size |y'|max is already that fraction of an innovation, on either side (about 4e-4 at
  N = 2^20, 1e-9 at N = 2^14).  Chain length 1 at N = 4096 makes the scans over chain
  aggregates three levels deep, as in the N = 2^20 benchmark's tree path.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SIZES = [4096, 16384, 65536, 262144, 1048576]


@pytest.fixture(scope="module")
def pit():
    import paper_2310_01145_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    P.load()
    return P


def fixture(N):
    path = os.path.join(GOLDEN, f"fhn_q3_N{N}_converged.npz")
    if not os.path.exists(path):
        pytest.fail(f"missing oracle fixture {path}")
    return np.load(path)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def errors(r, ref):
    idx = lambda k: torch.as_tensor(ref[k], device=r.mean.device)
    m = r.mean[idx("n_mean")].double().cpu().numpy()
    S = r.sqrtcov[idx("n_cov")].double().cpu().numpy()
    c = np.einsum("nij,nkj->nik", S, S)
    s2, s2_ref = r.sigma2, float(ref["sigma2"])
    return {"solution": rel(m[:, 0::4], ref["means"][:, 0::4]),
            "orders": [rel(m[:, i::4], ref["means"][:, i::4]) for i in range(4)],
            "cov": rel(c, ref["covs"]),
            "unit_cov": rel(c / s2, ref["covs"] / s2_ref),
            "sigma2": abs(s2 - s2_ref) / s2_ref}


def fp64_bars(ref, q=3):
    N = int(ref["N"])
    h = 20.0 / N
    T1 = math.sqrt(h) * h ** (q - 1) / math.factorial(q - 1)
    dy = float(np.max(np.abs(ref["means"][:, 1::q + 1])))
    return ([max(1e-10, 10 * float(x)) for x in ref["sens_order"]],
            max(1e-9, 10 * float(ref["sens_sigma2"]), 2.0 ** -53 * dy / T1))


@pytest.mark.parametrize("N", SIZES)
def test_fp32_benchmark_shape_matches_oracle(pit, N):
    """The benchmark's call (FP32, constant initial trajectory, stop at 1e-10 or 64 iterations,
    tuned launch shape) against the oracle's fixed point."""
    from paper_2310_01145_gb300 import autotune
    ref = fixture(N)
    p = W.fitzhugh_nagumo(N=N, q=3)
    variant, chain_len = autotune.lookup(p, "f32")
    r = pit.solve_problem(p, dtype=torch.float32, max_iter=64, atol_delta=1e-10,
                          chain_len=chain_len, variant=variant)
    torch.cuda.synchronize()
    assert r.converged, r.deltas
    e = errors(r, ref)
    assert e["solution"] < 1e-5, e
    assert e["cov"] < 1e-3, e
    assert e["unit_cov"] < 1e-3, e
    assert e["sigma2"] < 1e-3, e


@pytest.mark.parametrize("N", SIZES)
def test_fp64_matches_oracle_per_size(pit, N):
    """FP64 from the same coarse-grid start as the oracle, the library's default launch shape."""
    ref = fixture(N)
    p = W.fitzhugh_nagumo(N=N, q=3)
    r = pit.solve_problem(p, dtype=torch.float64, max_iter=60, atol_delta=1e-10,
                          init_coarse=int(ref["coarse_n"]))
    torch.cuda.synchronize()
    assert r.converged
    e = errors(r, ref)
    bars, s2bar = fp64_bars(ref)
    assert e["solution"] < 1e-10, e
    assert all(x < b for x, b in zip(e["orders"], bars)), (e, bars)
    assert e["unit_cov"] < 1e-8, e
    assert e["sigma2"] < s2bar, (e, s2bar)


@pytest.mark.parametrize("scan", [1, 0], ids=["tree", "single-launch"])
@pytest.mark.parametrize("dtype,tm,tc", [(torch.float64, 1e-10, 1e-8), (torch.float32, 1e-5, 1e-3)],
                         ids=["f64", "f32"])
def test_three_level_scan_trees(pit, dtype, tm, tc, scan):
    """Chain length 1 at N = 4096: 4097 chain aggregates per scan.  The tree path reduces them
    by block trees of 64 items over three levels (4097 -> 65 -> 2) and sweeps back down; the
    single-launch path groups them into 65 (FP32) or 129 (FP64) thread blocks whose totals are
    combined across blocks in 7 or 8 look-back rounds.  Both scans, filtering and smoothing;
    the converged result must still be the oracle's.  Both start from the oracle's coarse-grid
    trajectory: from the constant trajectory the first Gauss-Newton steps are chaotic in FP32
    (changes of 1e6 at iteration 2, where two scan orders already differ by tens of percent;
    FP64 agrees to 1e-9), and whether 64 iterations reach the fixed point then depends on
    rounding, not on the scan."""
    ref = fixture(4096)
    p = W.fitzhugh_nagumo(N=4096, q=3)
    r = pit.solve_problem(p, dtype=dtype, max_iter=64, atol_delta=1e-10, chain_len=1,
                          scan=scan, init_coarse=int(ref["coarse_n"]))
    torch.cuda.synchronize()
    assert r.converged
    e = errors(r, ref)
    assert e["solution"] < tm, e
    assert e["unit_cov"] < tc, e
    if dtype == torch.float64:
        bars, s2bar = fp64_bars(ref)
        assert all(x < b for x, b in zip(e["orders"], bars)), (e, bars)
        assert e["sigma2"] < s2bar, (e, s2bar)
