"""Kernel layout variant 1 (two state rows per lane, d = 2, q = 2 and 3) against the oracle.

The autotuner sweeps the compiled layout variants; each one it may pick must compute the same
numbers.  Variant 0 gives each lane of a group one row of every D-row matrix, variant 1 gives it
two (half the lanes per group, twice the rows per lane) while the tree kernels keep one row per
lane.  Same bars as the other parity tests: FP64 means 1e-10 and covariances 1e-8 per
iteration; FP32 solution means 1e-5 and covariances 1e-3 at convergence.
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
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


def cov(s):
    return np.einsum("nij,nkj->nik", s, s)


@pytest.mark.parametrize("p,iters,L", [(W.fitzhugh_nagumo(N=333, q=2), 3, 11),
                                       (W.van_der_pol(N=100, q=3), 4, 7),
                                       (W.van_der_pol(N=1000, q=2), 3, 0),
                                       (W.fitzhugh_nagumo(N=400, q=3), 42, 0)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_variant1_fp64_per_iteration(pit, p, iters, L):
    ref = ieks.ieks(p, fixed_iters=iters)
    r = pit.solve_problem(p, dtype=torch.float64, fixed_iters=iters, chain_len=L, variant=1)
    torch.cuda.synchronize()
    assert rel(r.mean.cpu().numpy(), ref.means) < 1e-10
    assert rel(cov(r.sqrtcov.cpu().numpy()), cov(ref.sqrtcovs)) < 1e-8
    assert r.sigma2 == pytest.approx(ref.sigma2, rel=1e-9)
    r0 = pit.solve_problem(p, dtype=torch.float64, fixed_iters=iters, chain_len=L, variant=0)
    torch.cuda.synchronize()
    assert rel(r.mean.cpu().numpy(), r0.mean.cpu().numpy()) < 1e-11


@pytest.mark.parametrize("p", [W.van_der_pol(N=256, q=2), W.fitzhugh_nagumo(N=400, q=3),
                               W.fitzhugh_nagumo(N=2000, q=2)],
                         ids=lambda x: f"{x.name}-{x.N}-q{x.q}")
def test_variant1_fp32_at_convergence(pit, p):
    ref = ieks.ieks(p, max_iter=60)
    assert ref.deltas[-1] < 1e-10
    r = pit.solve_problem(p, dtype=torch.float32, fixed_iters=ref.iterations, variant=1)
    torch.cuda.synchronize()
    m = r.mean.cpu().double().numpy()
    ys = slice(0, None, p.q + 1)
    assert rel(m[:, ys], ref.means[:, ys]) < 1e-5
    assert rel(cov(r.sqrtcov.cpu().double().numpy()), cov(ref.sqrtcovs)) < 1e-3
    assert r.sigma2 == pytest.approx(ref.sigma2, rel=1e-3)


def test_variant1_rejected_where_not_compiled(pit):
    """Variant 1 exists for d = 2, q = 2 and 3 only; other shapes refuse it on the host."""
    p = W.logistic(N=64, q=2)
    with pytest.raises(pit.PitError):
        pit.solve_problem(p, dtype=torch.float64, fixed_iters=1, variant=1)
