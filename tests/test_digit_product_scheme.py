"""The arithmetic of the FP64-accurate tensor-core product (csrc/pit_tc.cuh), emulated on the CPU
in exact integer arithmetic, independently of the CUDA code: the claims its design rests on.

* Every digit d_s 2^(-7 s) of a 63-bit fixed-point value is a bf16 number (8 significant bits,
  exponent in range), so the tensor cores see the digits exactly.
* The weight groups kept exact (g = s + t <= 5) never exceed 2^24 in their accumulators over a
  readout window of 160 terms (integer multiples of 2^(-7 g)), so FP32 accumulation is exact.
* With the digits of groups 0..8 formed (45 pairs), groups >= 6 summed in one FP32 accumulator
  and the dropped groups ignored, the product meets |C - AB| <= 2^-56 k max|row of A| max|col of B|
  for rows and columns spanning many binades.

The emulation follows the method's description (Ozaki, Ogita, Oishi, Rump 2012, in fixed-point
form); a plausible slip (a digit shift off by one, a dropped exact group, the wrong scale
exponent) breaks one of these checks.
"""
import math

import numpy as np

NDIG, GMAX, NEXACT, KACC = 9, 8, 6, 160


def _scale_exp(row):
    """Largest biased exponent of the entries (0 for an all-zero row)."""
    e = 0
    for x in row:
        if x != 0.0:
            e = max(e, math.frexp(abs(x))[1] + 1022)
    return e


def _fixed(x, emax):
    """trunc(x 2^(63 - (emax - 1022))) as a Python integer (|.| < 2^63)."""
    if x == 0.0:
        return 0
    m, e = math.frexp(x)               # x = m 2^e, 0.5 <= |m| < 1
    M = int(abs(m) * 2 ** 53)           # 53-bit integer mantissa, x = M 2^(e - 53)
    sh = e - 53 + 63 - (emax - 1022)    # <= 10
    v = M << sh if sh >= 0 else M >> (-sh)
    return -v if x < 0 else v


def _digits(a):
    s = -1 if a < 0 else 1
    u = abs(a)
    return [s * ((u >> (7 * (NDIG - 1 - k))) & 127) for k in range(NDIG)]


def _bf16_exact(v):
    """True when v (a float) is exactly a bf16 number: at most 8 significant bits."""
    if v == 0.0:
        return True
    m, e = math.frexp(v)
    return float(m * 256).is_integer() and -125 <= e <= 128


def _product(A, B):
    """The scheme's result for A (m x k) B (k x n) in exact arithmetic, the shared accumulator
    of groups >= NEXACT rounded as FP32 sums."""
    m, k = A.shape
    n = B.shape[1]
    ea = [_scale_exp(A[i]) for i in range(m)]
    eb = [_scale_exp(B[:, j]) for j in range(n)]
    da = [[_digits(_fixed(A[i, l], ea[i])) for l in range(k)] for i in range(m)]
    db = [[_digits(_fixed(B[l, j], eb[j])) for j in range(n)] for l in range(k)]
    C = np.zeros((m, n))
    peak = 0
    for i in range(m):
        for j in range(n):
            total = 0                                        # units of 2^-(7 GMAX)
            for w0 in range(0, k, KACC):
                exact = [0] * NEXACT                         # group sums as integers
                shared = np.float32(0.0)
                for l in range(w0, min(k, w0 + KACC)):
                    for s in range(NDIG):
                        for t in range(NDIG):
                            g = s + t
                            if g > GMAX:
                                continue
                            p = da[i][l][s] * db[l][j][t]
                            if g < NEXACT:
                                exact[g] += p
                                peak = max(peak, abs(exact[g]))
                            else:
                                shared = np.float32(shared + np.float32(p * 2.0 ** (-7 * g)))
                total += sum(exact[g] << (7 * (GMAX - g)) for g in range(NEXACT))
                total += int(round(float(shared) * 2.0 ** (7 * GMAX)))
            # value = total 2^(-7 GMAX) 2^112 2^(ea - 1022 - 63) 2^(eb - 1022 - 63)
            C[i, j] = math.ldexp(float(total), ea[i] + eb[j] - 2044 - 126 + 112 - 7 * GMAX)
    return C, peak


def test_digits_are_bf16_numbers():
    rng = np.random.default_rng(0)
    for x in rng.standard_normal(200) * np.exp2(rng.integers(-40, 41, size=200)):
        emax = _scale_exp([x])
        for s, d in enumerate(_digits(_fixed(x, emax))):
            assert abs(d) <= 127
            assert _bf16_exact(d * 2.0 ** (-7 * s))


def test_exact_groups_stay_below_2_24():
    # worst case: every digit 127 over a full window, the largest exact group (6 pairs)
    assert NEXACT * KACC * 127 * 127 < 2 ** 24
    assert (NEXACT + 1) * KACC * 127 * 127 >= 2 ** 24     # one more pair would not be exact


def test_fixed_point_split_is_exact_to_63_bits():
    rng = np.random.default_rng(1)
    row = rng.standard_normal(16) * np.exp2(rng.integers(-10, 11, size=16))
    emax = _scale_exp(row)
    for x in row:
        a = _fixed(x, emax)
        assert abs(a) < 2 ** 63
        back = math.ldexp(a, emax - 1022 - 63)
        assert abs(back - x) <= 2.0 ** -63 * 2.0 ** (emax - 1022)
        # the digits reassemble the fixed-point value
        assert sum(d << (7 * (NDIG - 1 - s)) for s, d in enumerate(_digits(a))) == a


def test_product_meets_its_bound_on_wide_range_inputs():
    from fractions import Fraction
    rng = np.random.default_rng(2)
    m, n, k = 5, 4, 170                                       # two readout windows
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-20, 21, size=(m, 1)))
    A *= np.exp2(rng.integers(-12, 13, size=(m, k)))
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-20, 21, size=(1, n)))
    C, peak = _product(A, B)
    assert peak < 2 ** 24
    for i in range(m):
        for j in range(n):
            exact = sum(Fraction(A[i, l]) * Fraction(B[l, j]) for l in range(k))
            err = abs(float(Fraction(C[i, j]) - exact))
            bound = 2.0 ** -56 * k * np.abs(A[i]).max() * np.abs(B[:, j]).max()
            assert err <= bound + 2.0 ** -52 * abs(float(exact)), (i, j, err / bound)


def test_integer_matrices_come_out_exact():
    rng = np.random.default_rng(3)
    A = rng.integers(-1000, 1001, size=(3, 40)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(40, 3)).astype(np.float64)
    C, _ = _product(A, B)
    np.testing.assert_array_equal(C, A @ B)
