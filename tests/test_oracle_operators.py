"""Pins of the oracle's prefix-sum elements and operators (Sections 3.1.1-3.1.3).

* a plain covariance-form Kalman filter / RTS smoother (textbook, no square roots) equals the
  square-root sequential filter/smoother;
* folding the filtering elements with (x)_f gives the filtering marginals (Section 3.1.2,
  "the filtering marginals"); folding the smoothing elements with (x)_s gives the smoothing
  marginals (Section 3.1.3);
* (x)_f and (x)_s are associative and have the stated neutral elements;
* the square-root operator agrees with the covariance-form operator of the element algebra
  (A_ij = A_j (I + C_i J_j)^-1 A_i, ...), a different formula for the same composition;
* an element with A = 0 restarts the scan: anything folded in before it is forgotten.
"""
import numpy as np
import pytest

from oracle.filtering import (filter_combine, filter_identity, filtering_elements,
                              fold_filter, fold_smooth, rts_smoother, sequential_filter,
                              smooth_combine, smooth_identity, smoothing_elements)
from oracle.linalg import tria
from oracle.prior import iwp_transition, projection


def random_linear_model(seed, d=2, q=2, N=9, h=0.3):
    rng = np.random.default_rng(seed)
    D = d * (q + 1)
    Phi, Q = iwp_transition(q, h, d)
    sQ = np.linalg.cholesky(Q)
    mu0 = rng.standard_normal(D)
    Hs, ds = [None], [None]
    for _ in range(N):
        F = rng.standard_normal((d, d))
        Hs.append(projection(1, q, d) - F @ projection(0, q, d))
        ds.append(rng.standard_normal(d))
    return mu0, Phi, Q, sQ, Hs, ds


def covariance_kalman(mu0, Sigma0, Phi, Q, Hs, ds):
    N = len(Hs) - 1
    m, P = mu0.copy(), Sigma0.copy()
    ms, Ps, mps, Pps = [m], [P], [None], [None]
    for n in range(1, N + 1):
        mp, Pp = Phi @ m, Phi @ P @ Phi.T + Q
        H = Hs[n]
        S = H @ Pp @ H.T
        K = Pp @ H.T @ np.linalg.inv(S)
        m = mp + K @ (ds[n] - H @ mp)
        P = Pp - K @ S @ K.T
        ms.append(m); Ps.append(P); mps.append(mp); Pps.append(Pp)
    # RTS
    msm, Psm = [None] * (N + 1), [None] * (N + 1)
    msm[N], Psm[N] = ms[N], Ps[N]
    for n in range(N - 1, -1, -1):
        G = Ps[n] @ Phi.T @ np.linalg.inv(Pps[n + 1])
        msm[n] = ms[n] + G @ (msm[n + 1] - mps[n + 1])
        Psm[n] = Ps[n] + G @ (Psm[n + 1] - Pps[n + 1]) @ G.T
    return np.array(ms), np.array(Ps), np.array(msm), np.array(Psm)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sqrt_filter_smoother_equal_covariance_form(seed):
    mu0, Phi, Q, sQ, Hs, ds = random_linear_model(seed)
    D = mu0.shape[0]
    mf, sPf, _, _ = sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    ms, sPs = rts_smoother(mf, sPf, Phi, sQ)
    cm, cP, cms, cPs = covariance_kalman(mu0, np.zeros((D, D)), Phi, Q, Hs, ds)
    np.testing.assert_allclose(mf, cm, atol=1e-9)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", sPf, sPf), cP, atol=1e-9)
    np.testing.assert_allclose(ms, cms, atol=1e-9)
    np.testing.assert_allclose(np.einsum("nij,nkj->nik", sPs, sPs), cPs, atol=1e-9)


def _cov(x):
    return x @ x.T


def assert_filter_elem_close(x, y, atol=1e-9):
    for a, b in [(x[0], y[0]), (x[1], y[1]), (_cov(x[2]), _cov(y[2])), (x[3], y[3]),
                 (_cov(x[4]), _cov(y[4]))]:
        np.testing.assert_allclose(a, b, atol=atol, rtol=1e-9)


@pytest.mark.parametrize("seed", [3, 4])
def test_fold_of_filtering_elements_gives_filter_marginals(seed):
    mu0, Phi, Q, sQ, Hs, ds = random_linear_model(seed)
    D = mu0.shape[0]
    mf, sPf, _, _ = sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    elems = filtering_elements(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    pref = fold_filter(elems)
    for n in range(1, len(Hs)):
        A, b, sC, _, _ = pref[n]
        np.testing.assert_allclose(A, 0.0, atol=1e-12)
        np.testing.assert_allclose(b, mf[n], atol=1e-9)
        np.testing.assert_allclose(_cov(sC), _cov(sPf[n]), atol=1e-9)


@pytest.mark.parametrize("seed", [5, 6])
def test_fold_of_smoothing_elements_gives_smoother_marginals(seed):
    mu0, Phi, Q, sQ, Hs, ds = random_linear_model(seed)
    D = mu0.shape[0]
    mf, sPf, _, _ = sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    ms, sPs = rts_smoother(mf, sPf, Phi, sQ)
    belems = smoothing_elements(mf, sPf, Phi, sQ)
    suf = fold_smooth(belems)
    for n in range(len(Hs)):
        E, g, sL = suf[n]
        np.testing.assert_allclose(E, 0.0, atol=1e-12)
        np.testing.assert_allclose(g, ms[n], atol=1e-9)
        np.testing.assert_allclose(_cov(sL), _cov(sPs[n]), atol=1e-9)


def random_filter_element(rng, D, rank_J=None):
    A = rng.standard_normal((D, D)) * 0.5
    b = rng.standard_normal(D)
    sC = np.tril(rng.standard_normal((D, D)))
    eta = rng.standard_normal(D)
    sJ = rng.standard_normal((D, D if rank_J is None else rank_J))
    if rank_J is not None:
        sJ = np.hstack([sJ, np.zeros((D, D - rank_J))])
    return A, b, sC, eta, sJ


def covariance_form_combine(ai, aj):
    """Composition of filtering elements with full covariances (element algebra of the
    prefix-sum formulation): A_ij = A_j (I + C_i J_j)^-1 A_i, etc."""
    Ai, bi, sCi, etai, sJi = ai
    Aj, bj, sCj, etaj, sJj = aj
    D = Ai.shape[0]
    Ci, Cj, Ji, Jj = _cov(sCi), _cov(sCj), _cov(sJi), _cov(sJj)
    I = np.eye(D)
    W = np.linalg.inv(I + Ci @ Jj)
    A = Aj @ W @ Ai
    b = Aj @ W @ (bi + Ci @ etaj) + bj
    C = Aj @ W @ Ci @ Aj.T + Cj
    V = np.linalg.inv(I + Jj @ Ci)
    eta = Ai.T @ V @ (etaj - Jj @ bi) + etai
    J = Ai.T @ V @ Jj @ Ai + Ji
    return A, b, C, eta, J


@pytest.mark.parametrize("seed", range(4))
def test_sqrt_operator_equals_covariance_form(seed):
    rng = np.random.default_rng(seed)
    D = 5
    ai = random_filter_element(rng, D)
    aj = random_filter_element(rng, D, rank_J=2)
    A, b, sC, eta, sJ = filter_combine(ai, aj)
    rA, rb, rC, reta, rJ = covariance_form_combine(ai, aj)
    np.testing.assert_allclose(A, rA, atol=1e-10)
    np.testing.assert_allclose(b, rb, atol=1e-10)
    np.testing.assert_allclose(_cov(sC), rC, atol=1e-10)
    np.testing.assert_allclose(eta, reta, atol=1e-10)
    np.testing.assert_allclose(_cov(sJ), rJ, atol=1e-10)


@pytest.mark.parametrize("seed", range(3))
def test_filter_operator_associative_and_neutral(seed):
    rng = np.random.default_rng(10 + seed)
    D = 4
    a, b, c = (random_filter_element(rng, D, rank_J=r) for r in (4, 2, 1))
    left = filter_combine(filter_combine(a, b), c)
    right = filter_combine(a, filter_combine(b, c))
    assert_filter_elem_close(left, right, atol=1e-9)
    e = filter_identity(D)
    assert_filter_elem_close(filter_combine(e, a), a, atol=1e-12)
    assert_filter_elem_close(filter_combine(a, e), a, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_smooth_operator_associative_and_neutral(seed):
    rng = np.random.default_rng(20 + seed)
    D = 4
    mk = lambda: (rng.standard_normal((D, D)) * 0.7, rng.standard_normal(D),
                  np.tril(rng.standard_normal((D, D))))
    a, b, c = mk(), mk(), mk()
    left = smooth_combine(smooth_combine(a, b), c)
    right = smooth_combine(a, smooth_combine(b, c))
    np.testing.assert_allclose(left[0], right[0], atol=1e-12)
    np.testing.assert_allclose(left[1], right[1], atol=1e-12)
    np.testing.assert_allclose(_cov(left[2]), _cov(right[2]), atol=1e-10)
    e = smooth_identity(D)
    for x, y in [(smooth_combine(e, a), a), (smooth_combine(a, e), a)]:
        np.testing.assert_allclose(x[0], y[0], atol=1e-14)
        np.testing.assert_allclose(x[1], y[1], atol=1e-14)
        np.testing.assert_allclose(_cov(x[2]), _cov(y[2]), atol=1e-12)


def test_segment_restart():
    """An element with A = 0 (a segment start) forgets everything folded in before it: its
    b and C are those of x (x) a_start for any x, and so is every later prefix."""
    mu0, Phi, Q, sQ, Hs, ds = random_linear_model(7, N=5)
    D = mu0.shape[0]
    elems = filtering_elements(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    rng = np.random.default_rng(99)
    garbage = random_filter_element(rng, D)
    clean = fold_filter(elems)
    acc = garbage
    for n in range(1, len(elems)):
        acc = filter_combine(acc, elems[n])
        np.testing.assert_allclose(acc[0], 0.0, atol=1e-12)
        np.testing.assert_allclose(acc[1], clean[n][1], atol=1e-9)
        np.testing.assert_allclose(_cov(acc[2]), _cov(clean[n][2]), atol=1e-9)
    # a smoothing element with E = 0 ends a segment for the reverse scan
    mf, sPf, _, _ = sequential_filter(mu0, np.zeros((D, D)), Phi, sQ, Hs, ds)
    belems = smoothing_elements(mf, sPf, Phi, sQ)
    junk = (rng.standard_normal((D, D)), rng.standard_normal(D), np.tril(rng.standard_normal((D, D))))
    x = smooth_combine(belems[-1], junk)
    np.testing.assert_allclose(x[1], belems[-1][1], atol=1e-14)
    np.testing.assert_allclose(_cov(x[2]), _cov(belems[-1][2]), atol=1e-12)
