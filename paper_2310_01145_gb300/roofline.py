"""Algorithmic work per time step of each kernel class, for the roofline report.

Counts are of the algorithm the kernels run (operations that change a result), not of the
instructions they issue: zero blocks of Phibar, rows already reduced by earlier reflections
and the redundant copies of small quantities that every lane of a group evaluates are not
counted.  A fused multiply-add counts as 2 flops; a square root or division counts as 1.

Notation: D = d (q+1) state dimension, d ODE dimension, Q1 = q + 1, W = D - d (width of the
filtering square-root factor after an update).
"""
from __future__ import annotations


def _phi_fma(D, d, Q1, ncols):
    # Phibar (I_d (x) upper-triangular Q1 x Q1 with all entries on and above the diagonal
    # non-zero) times a D x ncols matrix
    return d * (Q1 * (Q1 + 1) // 2) * ncols


def _lq_tri_ext_fma(D, NE, rows_other):
    """D reflections on [L | X]: reflection i has support 1 + NE, updates rows i+1..D-1 of the
    pivot set and `rows_other` rows of the other sets (dot + axpy each) plus its norm."""
    fma = 0
    for i in range(D):
        rows = (D - 1 - i) + rows_other
        fma += (NE + 1) * (1 + 2 * rows)
    return fma


def _lq_dense_fma(npiv, nc, rows_after_pivot_set, rows_other):
    fma = 0
    for k in range(npiv):
        supp = nc - k
        rows = (rows_after_pivot_set - 1 - k) + rows_other
        fma += supp * (1 + 2 * rows)
    return fma


def filter_down_flops(D: int, d: int, Q1: int, with_cov: bool = False) -> float:
    """One square-root Kalman step with the Pi-triangularisation that also yields the
    smoothing element b_{n-1}, folded into the chain's smoothing aggregate."""
    W = D - d
    fma = 0
    fma += _phi_fma(D, d, Q1, D) + _phi_fma(D, d, Q1, 1)           # Phi sqrtP, Phi m (+ u)
    # Pi: [sqrtQ | Phi sqrtP] / [0 | sqrtP]; sqrtP has W columns after an update (only the first
    # step of a chain starts from the tree's D-column prefix factor, 1 step in L)
    fma += _lq_tri_ext_fma(D, W, rows_other=D)
    fma += D * D * (D - 1) // 2 + D * D                              # E = Pi21 Pi11^-1 (back subst.)
    fma += D * D                                                     # g = m - E m-
    fma += D * D * D + D * D                                         # aggregate E~ E, x += E~ g
    fma += d * D * (d + 1) + d * (d + 1)                             # Htilde Pi11, residual
    fma += _lq_dense_fma(d, D, d, D)                                 # Psi: d reflections
    fma += D * d * (d + 1) // 2 + D * d                              # K, m update
    fma += d * (d + 1) // 2 + d                                      # calibration term
    other = D + 2 * d + d + 10 * d                                   # sqrt/div per reflection, linearisation
    if with_cov:
        fma += _lq_dense_fma(D, D, D, 0)                             # sqrtL = tria(remainder)
        fma += D * D * D + _lq_tri_ext_fma(D, D, rows_other=0)       # aggregate sqrtL~
    return 2.0 * fma + other


def filter_reduce_flops(D: int, d: int, Q1: int) -> float:
    """One fold of a leaf into the chain's conditional-filter aggregate."""
    W = D - d
    fma = 0
    fma += _phi_fma(D, d, Q1, D) + _phi_fma(D, d, Q1, W) + _phi_fma(D, d, Q1, 1)
    fma += _lq_tri_ext_fma(D, W, rows_other=0)                       # predicted sqrtC
    fma += d * D * (d + 1) * 2 + d * (d + 1)                         # Htilde C-, Htilde A', residual
    fma += _lq_dense_fma(d, D, d, D)                                 # Psi
    fma += D * d * (d + 1) // 2 + D * d                              # K, b update
    fma += D * D * d                                                 # A = A' - K (H A')
    fma += D * d * (d + 1) // 2 + d * (d + 1) // 2 + D * d           # G^T, sqrtS^-1 nu, eta
    fma += _lq_tri_ext_fma(D, d, rows_other=0)                       # sqrtJ update
    other = D + 2 * d + D + 10 * d
    return 2.0 * fma + other


def smooth_down_flops(D: int, with_cov: bool = False) -> float:
    fma = D * D
    if with_cov:
        fma += D * D * D + _lq_tri_ext_fma(D, D, rows_other=0)
    return 2.0 * fma


def residuals_flops(D: int, d: int, Q1: int) -> float:
    # FP64 arithmetic of the increment model's inputs
    return 2.0 * _phi_fma(D, d, Q1, 1) + D + 12 * d


def iteration_flops(D: int, d: int, Q1: int, with_cov: bool = False) -> float:
    """One time step of a whole IEKS iteration in the single-launch kernel: filter fold, Kalman
    step with the smoothing element, smoothing step.  The residuals are FP64 work and the scans
    over chain aggregates add a few combines per chain; neither is counted here."""
    return (filter_reduce_flops(D, d, Q1) + filter_down_flops(D, d, Q1, with_cov)
            + smooth_down_flops(D, with_cov))


# ---- bytes (algorithmic: each array element moved once per kernel) -------------------------
def bytes_per_step(kernel: str, D: int, d: int, elem: int, traj_elem: int,
                   with_cov: bool = False) -> float:
    """HBM bytes per time step a kernel must move.

    residuals:     read lin (D traj), write u (D), r (d), y (d)
    filter_reduce: read u (D), r (d), y (d)
    filter_down:   read u, r, y; write E (D^2), g (D) [+ sqrtL (D^2)]
    smooth_down:   read E, g [+ sqrtL], lin; write lin' [or mean (D) + sqrt cov (D^2)]
    """
    if kernel == "residuals":
        return D * traj_elem + (D + 2 * d) * elem
    if kernel == "filter_reduce":
        return (D + 2 * d) * elem
    if kernel == "filter_down":
        return (D + 2 * d) * elem + (D * D + D + (D * D if with_cov else 0)) * elem
    if kernel == "smooth_down":
        rd = (D * D + D + (D * D if with_cov else 0)) * elem + D * traj_elem
        wr = (D + D * D) * elem if with_cov else D * traj_elem
        return rd + wr
    raise ValueError(kernel)


def fp32_alu_peak_tflops(sm_count: int, clock_mhz: float, fp32_lanes_per_sm: int = 128) -> float:
    """Nominal FP32 FMA peak: SMs x FP32 lanes x 2 flops x clock (the SM count is the device's,
    the clock its maximum)."""
    return sm_count * fp32_lanes_per_sm * 2.0 * clock_mhz * 1e6 / 1e12


def fp64_alu_peak_tflops(sm_count: int, clock_mhz: float, fma_per_clk_per_sm: int = 2) -> float:
    """Nominal FP64 peak of GB300 (its FP64 rate is cut to 1.25 TFLOP/s at 152 SMs): SMs x FP64
    FMA per clock x 2 flops x clock."""
    return sm_count * fma_per_clk_per_sm * 2.0 * clock_mhz * 1e6 / 1e12
