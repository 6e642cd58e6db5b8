"""Truncated Taylor series arithmetic (test infrastructure only).

A Series holds coefficients c_0..c_K of y(t) = sum_k c_k t^k.  Products are Cauchy products
truncated at order K.  This is the arithmetic behind Taylor-mode automatic differentiation
(Griewank & Walther), which Section 2.1 uses for the exact initial state.
"""
from __future__ import annotations

import numpy as np


class Series:
    __slots__ = ("c",)

    def __init__(self, coeffs):
        self.c = np.asarray(coeffs, dtype=np.float64).copy()

    @property
    def order(self) -> int:
        return self.c.shape[0] - 1

    @staticmethod
    def const(value: float, order: int) -> "Series":
        c = np.zeros(order + 1)
        c[0] = value
        return Series(c)

    def _coerce(self, other):
        if isinstance(other, Series):
            return other
        return Series.const(float(other), self.order)

    def __add__(self, other):
        o = self._coerce(other)
        return Series(self.c + o.c)

    def __sub__(self, other):
        o = self._coerce(other)
        return Series(self.c - o.c)

    def __mul__(self, other):
        if not isinstance(other, Series):
            return Series(self.c * float(other))
        K = self.order
        out = np.zeros(K + 1)
        for k in range(K + 1):
            s = 0.0
            for j in range(k + 1):
                s += self.c[j] * other.c[k - j]
            out[k] = s
        return Series(out)

    __rmul__ = __mul__
