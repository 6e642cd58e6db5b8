"""The FP64-accurate tensor-core product of the large-state solver (tcgen05, bf16 digit slices
of 56-bit fixed-point operands, exact FP32 accumulation, integer recombination), checked on its
own through pit_check_dgemm_tc against extended-precision products of the same FP64 inputs.

Bars: integer matrices whose products are exact in FP64 must come out bit-exact (any error in
the operand layouts, digit split or recombination breaks this); random matrices with rows and
columns of very different magnitude must meet the method's bound |C - AB| <= 2^-56 k
max|row of op(A)| max|column of op(B)| (the FP64 GEMM's own bound is 2^-53 k sum |a||b|).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pit():
    import paper_2310_01145_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    P.load()
    return P


DEV = "cuda:0"


def _op(X, t):
    return X.T if t else X


def _run(pit, A, B, C0, alpha, beta, ta, tb):
    At = torch.tensor(A, device=DEV)
    Bt = torch.tensor(B, device=DEV)
    Ct = torch.tensor(C0, device=DEV)
    pit.pit_check_dgemm_tc(At, Bt, Ct, alpha=alpha, beta=beta, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    return Ct.cpu().numpy()


def _ref(A, B, C0, alpha, beta, ta, tb):
    L = np.longdouble
    return (L(alpha) * (_op(A, ta).astype(L) @ _op(B, tb).astype(L)) + L(beta) * C0.astype(L))


SHAPES = [(1, 1, 1), (7, 5, 3), (128, 32, 32), (129, 33, 129), (192, 192, 192), (300, 70, 257),
          (64, 200, 31), (130, 65, 450)]


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", SHAPES)
def test_integer_products_bit_exact(pit, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n * 3 + k + 11 * ta + 5 * tb)
    A = rng.integers(-1000, 1001, size=(k, m) if ta else (m, k)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(n, k) if tb else (k, n)).astype(np.float64)
    C0 = rng.integers(-50, 51, size=(m, n)).astype(np.float64)
    got = _run(pit, A, B, C0, 1.0, 1.0, ta, tb)
    want = _op(A, ta) @ _op(B, tb) + C0        # exact: every partial sum is an integer < 2^53
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("m,n,k", SHAPES[1:])
def test_wide_range_within_bound(pit, m, n, k, ta, tb):
    rng = np.random.default_rng(1000 + m + n + k + ta + 2 * tb)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-30, 31, size=(m, 1)))
    A *= np.exp2(rng.integers(-12, 13, size=(m, k)))          # entries far below their row max
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-30, 31, size=(1, n)))
    C0 = rng.standard_normal((m, n))
    Ast = np.ascontiguousarray(A.T) if ta else A
    Bst = np.ascontiguousarray(B.T) if tb else B
    alpha, beta = -0.75, 0.5
    got = _run(pit, Ast, Bst, C0, alpha, beta, ta, tb)
    ref = _ref(Ast, Bst, C0, alpha, beta, ta, tb)
    scale = np.abs(alpha) * (np.abs(A) @ np.abs(B)) + np.abs(beta * C0)
    bound = 2.0 ** -56 * k * np.abs(alpha) * np.outer(np.abs(A).max(1), np.abs(B).max(0))
    bound += 2.0 ** -50 * scale      # FP64 roundings: the value, windows of 192 terms, alpha v + beta C
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.max(err / scale) < 1e-14


def test_special_values(pit):
    rng = np.random.default_rng(5)
    m, n, k = 40, 36, 50
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((k, n))
    A[3, :] = 0.0                       # zero row -> beta C only
    A[7, 11] = np.nan                   # non-finite row -> NaN row
    B[:, 5] = 1e-310                    # subnormal column -> treated as zero (< 2^-1022)
    C0 = rng.standard_normal((m, n))
    got = _run(pit, A, B, C0, 1.0, 2.0, 0, 0)
    assert np.all(np.isnan(got[7]))
    np.testing.assert_array_equal(got[3], 2.0 * C0[3])
    ok = np.ones(m, bool)
    ok[[3, 7]] = False
    np.testing.assert_allclose(got[ok, 5], 2.0 * C0[ok, 5], rtol=0, atol=1e-300)
    ref = A[ok] @ B + 2.0 * C0[ok]
    cols = np.arange(n) != 5
    np.testing.assert_allclose(got[ok][:, cols], ref[:, cols], rtol=1e-13, atol=1e-13)


def test_empty_k_and_beta_zero(pit):
    C0 = np.full((5, 6), np.nan)        # beta == 0 must not read C
    got = _run(pit, np.zeros((5, 0)), np.zeros((0, 6)), C0, 1.0, 0.0, 0, 0)
    np.testing.assert_array_equal(got, np.zeros((5, 6)))


def test_rejects_bad_arguments(pit):
    A = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    with pytest.raises(pit.PitError) as ei:
        pit.pit_check_dgemm_tc(A, A, torch.zeros((4, 5000), dtype=torch.float64, device=DEV))
    assert ei.value.status == 1


def test_bounded_wait_gives_up(pit):
    """An mbarrier that nothing arrives on: the wait gives up after its limit (50 ms here), sets
    the timeout bit and the block still frees its tensor memory; the context stays usable."""
    assert pit.pit_check_tc_wait(50_000_000) == 5
    rng = np.random.default_rng(0)
    A = rng.integers(-9, 10, size=(16, 16)).astype(np.float64)
    np.testing.assert_array_equal(_run(pit, A, A, np.zeros((16, 16)), 1.0, 0.0, 0, 0), A @ A)
