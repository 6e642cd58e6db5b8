"""Seeded synthetic problem instances shared by the CUDA path, the oracle and the benchmark.

This module only *describes* problems: ODE family, parameters, initial value, time interval,
grid size and prior order.  It holds none of the solver's arithmetic (no vector fields, no
priors, no filtering), so that the oracle and the CUDA library, which must share no code, can
both read the same inputs from it.

The problems are shaped like the paper's test problems (Section 4.1: logistic, rigid body,
Van der Pol; Section 4.2: logistic with h = 2^0 ... 2^-14) and like the configurations the
benchmark runs (logistic r=3, FitzHugh-Nagumo, batched Lotka-Volterra).  Random draws use
numpy's PCG64 generator with the stated seeds.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Family identifiers.  The integer values are the ones the C ABI uses (pit_ode_kind).
LOGISTIC = 0
FITZHUGH_NAGUMO = 1
LOTKA_VOLTERRA = 2
LORENZ96 = 3
AFFINE = 4
RIGID_BODY = 5
VAN_DER_POL = 6

FAMILY_NAMES = {
    LOGISTIC: "logistic",
    FITZHUGH_NAGUMO: "fitzhugh_nagumo",
    LOTKA_VOLTERRA: "lotka_volterra",
    LORENZ96: "lorenz96",
    AFFINE: "affine",
    RIGID_BODY: "rigid_body",
    VAN_DER_POL: "van_der_pol",
}


@dataclasses.dataclass(frozen=True)
class Problem:
    """One initial value problem y' = f(y), y(t0) = y0 on a uniform grid of N steps.

    kind    -- family identifier (one of the constants above)
    d       -- ODE dimension
    params  -- family parameters, float64 (layout documented per family below)
    y0      -- initial value, float64, shape (d,)
    t0, t1  -- time interval
    N       -- number of steps; the grid is t_n = t0 + n (t1 - t0) / N, n = 0..N
    q       -- order of the integrated-Wiener-process prior (the paper's nu)
    ts      -- optional non-uniform grid t_0 = t0 < t_1 < ... < t_N = t1 (float64, N+1 values);
               None means the uniform grid above
    """

    kind: int
    d: int
    params: np.ndarray
    y0: np.ndarray
    t0: float
    t1: float
    N: int
    q: int
    ts: np.ndarray | None = None

    @property
    def uniform(self) -> bool:
        return self.ts is None

    @property
    def times(self) -> np.ndarray:
        """Grid points t_0 .. t_N."""
        if self.ts is not None:
            return np.asarray(self.ts, dtype=np.float64)
        return self.t0 + self.h * np.arange(self.N + 1)

    @property
    def steps(self) -> np.ndarray:
        """Step lengths h_n = t_n - t_{n-1}, n = 1..N (index 0 of the returned array is h_1)."""
        if self.ts is not None:
            return np.diff(np.asarray(self.ts, dtype=np.float64))
        return np.full(self.N, self.h)

    @property
    def D(self) -> int:
        return self.d * (self.q + 1)

    @property
    def h(self) -> float:
        """Step length of the uniform grid (the mean step of a non-uniform one)."""
        return (self.t1 - self.t0) / self.N

    @property
    def name(self) -> str:
        return FAMILY_NAMES[self.kind]

    def with_grid(self, N: int | None = None, q: int | None = None) -> "Problem":
        return dataclasses.replace(self, N=self.N if N is None else int(N),
                                   q=self.q if q is None else int(q))


def _p(*xs) -> np.ndarray:
    return np.asarray(xs, dtype=np.float64)


# ---- parameter layouts -------------------------------------------------------------------
# logistic         params = [r]                      y' = r y (1 - y)
# fitzhugh_nagumo  params = [a, b, c]                v' = c (v - v^3/3 + w),  w' = -(v - a + b w) / c
# lotka_volterra   params = [alpha, beta, gamma, delta]
#                                                    x' = alpha x - beta x y,  y' = delta x y - gamma y
# van_der_pol      params = [mu]                     y1' = y2,  y2' = mu ((1 - y1^2) y2 - y1)
# rigid_body       params = []                       y' = (-2 y2 y3, 1.25 y1 y3, -0.5 y1 y2)
# affine           params = [L (d*d, row-major), c (d)]   y' = L y + c
# lorenz96         params = [F]                      x_i' = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F


def logistic(N: int = 1024, q: int = 2, rate: float = 3.0, y0: float = 0.01,
             t1: float = 10.0) -> Problem:
    """Logistic ODE; rate 3 is the benchmark's small case, rate 1 the paper's Eq. (logistic)."""
    return Problem(LOGISTIC, 1, _p(rate), _p(y0), 0.0, float(t1), int(N), int(q))


def logistic_paper(N: int = 30, q: int = 2) -> Problem:
    """Section 4.1: y' = y (1 - y), y(0) = 0.01, t in [0, 10]."""
    return logistic(N=N, q=q, rate=1.0)


def fitzhugh_nagumo(N: int = 4096, q: int = 3) -> Problem:
    """FitzHugh-Nagumo with a = b = 0.2, c = 3, y0 = (-1, 1), t in [0, 20]."""
    return Problem(FITZHUGH_NAGUMO, 2, _p(0.2, 0.2, 3.0), _p(-1.0, 1.0), 0.0, 20.0,
                   int(N), int(q))


def rigid_body(N: int = 150, q: int = 2) -> Problem:
    """Section 4.1 rigid body dynamics, t in [0, 20], y0 = (1, 0, 0.9)."""
    return Problem(RIGID_BODY, 3, _p(), _p(1.0, 0.0, 0.9), 0.0, 20.0, int(N), int(q))


def van_der_pol(N: int = 100, q: int = 2, mu: float = 1.0) -> Problem:
    """Section 4.1 Van der Pol oscillator (non-stiff, mu = 1), t in [0, 6.3], y0 = (2, 0)."""
    return Problem(VAN_DER_POL, 2, _p(mu), _p(2.0, 0.0), 0.0, 6.3, int(N), int(q))


def affine(L: Sequence[Sequence[float]], c: Sequence[float], y0: Sequence[float],
           t1: float = 1.0, N: int = 8, q: int = 1) -> Problem:
    """Affine ODE y' = L y + c (Section 3.1, Eq. affine-ivp with constant L and d)."""
    L = np.asarray(L, dtype=np.float64)
    d = L.shape[0]
    params = np.concatenate([L.reshape(-1), np.asarray(c, dtype=np.float64).reshape(d)])
    return Problem(AFFINE, d, params, np.asarray(y0, dtype=np.float64).reshape(d), 0.0,
                   float(t1), int(N), int(q))


def lotka_volterra(alpha=1.5, beta=1.0, gamma=3.0, delta=1.0, y0=(1.0, 1.0), N: int = 1024,
                   q: int = 2, t1: float = 10.0) -> Problem:
    return Problem(LOTKA_VOLTERRA, 2, _p(alpha, beta, gamma, delta), _p(*y0), 0.0, float(t1),
                   int(N), int(q))


def lotka_volterra_batch(count: int = 4096, seed: int = 0, n_min: int = 256,
                         n_max: int = 16384, q: int = 2) -> List[Problem]:
    """Batched Lotka-Volterra: (alpha, beta, gamma, delta) = (1.5, 1, 3, 1) * U[0.8, 1.2]
    (independently), y0 ~ U[0.5, 2]^2, N log-uniform in [n_min, n_max], t in [0, 10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = np.array([1.5, 1.0, 3.0, 1.0])
    out = []
    for _ in range(count):
        prm = base * rng.uniform(0.8, 1.2, size=4)
        y0 = rng.uniform(0.5, 2.0, size=2)
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append(Problem(LOTKA_VOLTERRA, 2, prm, y0, 0.0, 10.0, N, q))
    return out


def lorenz96(d: int = 64, N: int = 16384, q: int = 2, F: float = 8.0, seed: int = 0) -> Problem:
    """Lorenz-96, cyclic, y0 = F + 0.01 N(0, 1), t in [0, 5]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    y0 = F + 0.01 * rng.standard_normal(d)
    return Problem(LORENZ96, d, _p(F), y0, 0.0, 5.0, int(N), int(q))


def graded_grid(t0: float, t1: float, N: int, ratio: float) -> np.ndarray:
    """Geometrically graded grid on [t0, t1]: N steps whose lengths grow by the constant factor
    ratio^(1/(N-1)) from the first to the last (the last step is `ratio` times the first)."""
    if N == 1:
        return np.array([t0, t1], dtype=np.float64)
    g = ratio ** (1.0 / (N - 1))
    w = g ** np.arange(N)
    ts = t0 + (t1 - t0) * np.concatenate([[0.0], np.cumsum(w) / np.sum(w)])
    ts[-1] = t1
    return ts


def on_grid(p: Problem, ts) -> Problem:
    """The same problem on the non-uniform grid ts (t0 and t1 are taken from its ends)."""
    ts = np.asarray(ts, dtype=np.float64)
    return dataclasses.replace(p, ts=ts, t0=float(ts[0]), t1=float(ts[-1]), N=len(ts) - 1)


def params_array(p: Problem) -> np.ndarray:
    """Parameters as a contiguous float64 array (what the C ABI receives)."""
    return np.ascontiguousarray(p.params, dtype=np.float64)


def serving_requests(count: int, seed: int = 0, n_min: int = 256, n_max: int = 65536,
                     families=("logistic", "fitzhugh_nagumo", "lotka_volterra")) -> List[Problem]:
    """Request stream of the serving workload: family uniform over `families`, q ~ U{1, 2, 3},
    N log-uniform in [n_min, n_max]; parameters and y0 around each family's benchmark values
    (logistic r = 3 U[0.8, 1.2], y0 = 0.01 U[0.5, 2] on [0, 10]; FitzHugh-Nagumo a, b, c scaled
    by U[0.8, 1.2], y0 = (-1, 1) + 0.1 U[-1, 1]^2 on [0, 20]; Lotka-Volterra as the batched
    workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        fam = families[int(rng.integers(len(families)))]
        q = int(rng.integers(1, 4))
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        if fam == "logistic":
            out.append(Problem(LOGISTIC, 1, _p(3.0 * rng.uniform(0.8, 1.2)),
                               _p(0.01 * rng.uniform(0.5, 2.0)), 0.0, 10.0, N, q))
        elif fam == "fitzhugh_nagumo":
            prm = np.array([0.2, 0.2, 3.0]) * rng.uniform(0.8, 1.2, size=3)
            y0 = np.array([-1.0, 1.0]) + 0.1 * rng.uniform(-1.0, 1.0, size=2)
            out.append(Problem(FITZHUGH_NAGUMO, 2, prm, y0, 0.0, 20.0, N, q))
        else:
            prm = np.array([1.5, 1.0, 3.0, 1.0]) * rng.uniform(0.8, 1.2, size=4)
            y0 = rng.uniform(0.5, 2.0, size=2)
            out.append(Problem(LOTKA_VOLTERRA, 2, prm, y0, 0.0, 10.0, N, q))
    return out
