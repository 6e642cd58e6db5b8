"""Square-root Kalman filtering and smoothing, sequential and in prefix-sum form (Section 3.1).

Test infrastructure only.  Covariances are carried as left square roots (Section 2.4,
square-root formulation); every covariance sum goes through ``tria``.  Observations are the
noiseless affine model Z_n | Y_n ~ delta(H_n Y_n - d_n) with data Z_n = 0 (Eq.
affine-estimation / linearized-inference-problem), i.e. sqrt(R_n) = 0.

Sequential part (the definition the parallel solver must reproduce):
    predict   m-_n = Phi m_{n-1},  sqrtP-_n = tria([Phi sqrtP_{n-1}, sqrtQ])
    update    Psi = tria([[H sqrtP-, 0], [sqrtP-, 0]]),  sqrtS = Psi11,  K = Psi21 Psi11^-1,
              m_n = m-_n - K (H m-_n - d_n),  sqrtP_n = Psi22
    RTS       Pi = tria([[Phi sqrtP_n, sqrtQ], [sqrtP_n, 0]]),  G = Pi21 Pi11^-1,
              m^s_n = m_n + G (m^s_{n+1} - Phi m_n),  sqrtP^s_n = tria([G sqrtP^s_{n+1}, Pi22])

Prefix-sum part (for pinning the operators): the filtering elements
(A, b, sqrtC, eta, sqrtJ) of Eq. sqrt-filtering-elements, the operator of Eq.
sqrt-associative-filtering, the smoothing elements (E, g, sqrtL) of Eq.
sqrt-smoothing-elements and the operator of Eq. sqrt-associative-smoothing.  All square-root
factors are stored as square D x D matrices, padded with zero columns where the paper's block
is narrower (sqrtJ is D x d in the paper).
"""
from __future__ import annotations

import numpy as np

from .linalg import right_solve, solve_lower, tria


# ------------------------------------------------------------------------------------------
# sequential square-root filter / smoother
# ------------------------------------------------------------------------------------------
def predict(m, sP, Phi, sQ):
    return Phi @ m, tria(np.hstack([Phi @ sP, sQ]))


def update(m_pred, sP_pred, H, dvec):
    """Square-root update with the Psi-tria of Section 3.1.2 (sqrt(R) = 0).

    Returns (m, sqrtP, sqrtS, r) with r = H m- - d the prediction residual."""
    dd, D = H.shape
    M = np.block([[H @ sP_pred, np.zeros((dd, dd))],
                  [sP_pred, np.zeros((D, dd))]])
    Psi = tria(M)
    sS = Psi[:dd, :dd]
    Psi21 = Psi[dd:, :dd]
    Psi22 = Psi[dd:, dd:]
    K = right_solve(Psi21, sS)
    r = H @ m_pred - dvec
    return m_pred - K @ r, Psi22, sS, r


def step_matrix(M, n):
    """Transition quantity of step n (from t_{n-1} to t_n): M itself on a uniform grid, M[n]
    when M is a per-step list (index 0 unused) on a non-uniform grid."""
    return M[n] if isinstance(M, (list, tuple)) else M


def sequential_filter(mu0, sSigma0, Phi, sQ, Hs, ds):
    """Filter marginals n = 0..N (n = 0 is the initial distribution).

    Hs[n], ds[n] for n = 1..N (index 0 unused); Phi, sQ one matrix each (uniform grid) or
    per-step lists (Phi[n], sQ[n] for the step into t_n).  Returns mf (N+1, D), sPf (N+1, D, D),
    sS (N+1, d, d) and residuals r (N+1, d) (index 0 unused)."""
    N = len(Hs) - 1
    D = mu0.shape[0]
    dd = Hs[1].shape[0]
    mf = np.zeros((N + 1, D))
    sPf = np.zeros((N + 1, D, D))
    sS = np.zeros((N + 1, dd, dd))
    res = np.zeros((N + 1, dd))
    mf[0] = mu0
    sPf[0] = sSigma0
    for n in range(1, N + 1):
        mp, sPp = predict(mf[n - 1], sPf[n - 1], step_matrix(Phi, n), step_matrix(sQ, n))
        mf[n], sPf[n], sS[n], res[n] = update(mp, sPp, Hs[n], ds[n])
    return mf, sPf, sS, res


def rts_smoother(mf, sPf, Phi, sQ):
    """Square-root Rauch-Tung-Striebel smoother (backward pass over n = N-1..0); Phi, sQ as in
    sequential_filter."""
    N = mf.shape[0] - 1
    D = mf.shape[1]
    ms = np.zeros_like(mf)
    sPs = np.zeros_like(sPf)
    ms[N] = mf[N]
    sPs[N] = sPf[N]
    for n in range(N - 1, -1, -1):
        F, sq = step_matrix(Phi, n + 1), step_matrix(sQ, n + 1)
        Pi = tria(np.block([[F @ sPf[n], sq], [sPf[n], np.zeros((D, D))]]))
        Pi11, Pi21, Pi22 = Pi[:D, :D], Pi[D:, :D], Pi[D:, D:]
        G = right_solve(Pi21, Pi11)
        ms[n] = mf[n] + G @ (ms[n + 1] - F @ mf[n])
        sPs[n] = tria(np.hstack([G @ sPs[n + 1], Pi22]))
    return ms, sPs


# ------------------------------------------------------------------------------------------
# prefix-sum elements and operators
# ------------------------------------------------------------------------------------------
def _pad(M, D):
    out = np.zeros((M.shape[0], D))
    out[:, : M.shape[1]] = M
    return out


def filtering_elements(mu0, sSigma0, Phi, sQ, Hs, ds):
    """Elements a_n = (A_n, b_n, sqrtC_n, eta_n, sqrtJ_n), n = 1..N (Eq.
    sqrt-filtering-elements).  m_0 = mu0, P_0 = Sigma0 and m_n = 0, P_n = 0 for n >= 1 enter
    the prediction.  For n = 1 the element does not depend on Y_0 (Section 3.1.1), so A_1,
    eta_1 and sqrtJ_1 are zero."""
    N = len(Hs) - 1
    D = mu0.shape[0]
    out = [None]
    for n in range(1, N + 1):
        H, dv = Hs[n], ds[n]
        dd = H.shape[0]
        if n == 1:
            m_prev, sP_prev = mu0, sSigma0
        else:
            m_prev, sP_prev = np.zeros(D), np.zeros((D, D))
        mp, sPp = predict(m_prev, sP_prev, Phi, sQ)
        Psi = tria(np.block([[H @ sPp, np.zeros((dd, dd))], [sPp, np.zeros((D, dd))]]))
        sS, Psi21, Psi22 = Psi[:dd, :dd], Psi[dd:, :dd], Psi[dd:, dd:]
        K = right_solve(Psi21, sS)
        A = (np.eye(D) - K @ H) @ Phi
        b = mp - K @ (H @ mp - dv)
        sC = Psi22
        sJ = right_solve(Phi.T @ H.T, sS.T)          # Phi^T H^T sqrtS^-T   (D x d)
        eta = sJ @ solve_lower(sS, dv)                # sqrtJ sqrtS^-1 d
        if n == 1:
            A = np.zeros((D, D))
            sJ = np.zeros_like(sJ)
            eta = np.zeros(D)
        out.append((A, b, sC, eta, _pad(sJ, D)))
    return out


def filter_combine(ai, aj):
    """a_i (x)_f a_j, Eq. sqrt-associative-filtering."""
    Ai, bi, sCi, etai, sJi = ai
    Aj, bj, sCj, etaj, sJj = aj
    D = Ai.shape[0]
    I = np.eye(D)
    Xi = tria(np.block([[sCi.T @ sJj, I], [sJj, np.zeros((D, D))]]))
    X11, X21, X22 = Xi[:D, :D], Xi[D:, :D], Xi[D:, D:]
    M = right_solve(sCi, X11.T)                        # sqrtC_i Xi11^-T
    Amid = I - M @ X21.T                               # I - sqrtC_i Xi11^-T Xi21^T
    A = Aj @ Ai - Aj @ M @ X21.T @ Ai
    b = Aj @ Amid @ (bi + sCi @ (sCi.T @ etaj)) + bj
    sC = tria(np.hstack([Aj @ M, sCj]))
    Bmid = I - X21 @ np.linalg.solve(X11, sCi.T)        # I - Xi21 Xi11^-1 sqrtC_i^T
    eta = Ai.T @ Bmid @ (etaj - sJj @ (sJj.T @ bi)) + etai
    sJ = tria(np.hstack([Ai.T @ X22, sJi]))
    return A, b, sC, eta, sJ


def filter_identity(D):
    """Neutral element of (x)_f: A = I and everything else zero."""
    Z = np.zeros((D, D))
    return np.eye(D), np.zeros(D), Z.copy(), np.zeros(D), Z.copy()


def smoothing_elements(mf, sPf, Phi, sQ):
    """Elements b_n = (E_n, g_n, sqrtL_n), n = 0..N (Eq. sqrt-smoothing-elements);
    b_N = p(Y_N | Z_1:N): E_N = 0, g_N = m^f_N, sqrtL_N = sqrtP^f_N."""
    N = mf.shape[0] - 1
    D = mf.shape[1]
    out = []
    for n in range(N):
        Pi = tria(np.block([[Phi @ sPf[n], sQ], [sPf[n], np.zeros((D, D))]]))
        Pi11, Pi21, Pi22 = Pi[:D, :D], Pi[D:, :D], Pi[D:, D:]
        E = right_solve(Pi21, Pi11)
        g = mf[n] - E @ Phi @ mf[n]
        out.append((E, g, Pi22))
    out.append((np.zeros((D, D)), mf[N].copy(), sPf[N].copy()))
    return out


def smooth_combine(bi, bj):
    """b_i (x)_s b_j, Eq. sqrt-associative-smoothing."""
    Ei, gi, sLi = bi
    Ej, gj, sLj = bj
    return Ei @ Ej, Ei @ gj + gi, tria(np.hstack([Ei @ sLj, sLi]))


def smooth_identity(D):
    return np.eye(D), np.zeros(D), np.zeros((D, D))


def fold_filter(elems):
    """Inclusive prefix results a_1 (x) ... (x) a_n, n = 1..N, by a plain left fold."""
    acc = elems[1]
    out = [None, acc]
    for n in range(2, len(elems)):
        acc = filter_combine(acc, elems[n])
        out.append(acc)
    return out


def fold_smooth(elems):
    """Reverse inclusive results b_n (x) ... (x) b_N, n = 0..N, by a plain right fold."""
    N = len(elems) - 1
    out = [None] * (N + 1)
    acc = elems[N]
    out[N] = acc
    for n in range(N - 1, -1, -1):
        acc = smooth_combine(elems[n], acc)
        out[n] = acc
    return out
