"""The triangularisation operator of Section 3.1.2 (test infrastructure only).

tria(M), for M of shape n x m with m >= n: take the QR decomposition M^T = Q R with R square
upper-triangular (n x n) and return R^T, a lower-triangular left square root of M M^T.  The
factor is unique up to the signs of its columns; this implementation fixes them so that the
diagonal is non-negative.  A tall M (m < n) is padded with zero columns first.
"""
from __future__ import annotations

import numpy as np


def tria(M: np.ndarray) -> np.ndarray:
    M = np.asarray(M, dtype=np.float64)
    n, m = M.shape
    if m < n:
        M = np.hstack([M, np.zeros((n, n - m))])
    R = np.linalg.qr(M.T, mode="r")  # n x n upper triangular (reduced QR of an m x n matrix)
    L = R.T.copy()
    s = np.sign(np.diag(L))
    s[s == 0] = 1.0
    return L * s[None, :]


def solve_lower(Lmat: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve Lmat X = B for lower-triangular Lmat (plain forward substitution)."""
    n = Lmat.shape[0]
    B = np.asarray(B, dtype=np.float64)
    vec = B.ndim == 1
    X = np.array(B.reshape(n, -1), dtype=np.float64)
    for i in range(n):
        X[i] -= Lmat[i, :i] @ X[:i]
        X[i] /= Lmat[i, i]
    return X.reshape(-1) if vec else X


def right_solve(B: np.ndarray, Mmat: np.ndarray) -> np.ndarray:
    """X = B Mmat^-1 (solve X Mmat = B) with a library solve."""
    return np.linalg.solve(Mmat.T, np.asarray(B, dtype=np.float64).T).T
