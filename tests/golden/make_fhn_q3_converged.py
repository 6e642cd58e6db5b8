"""Writes tests/golden/fhn_q3_N{N}_converged.npz: the FP64 oracle's converged IEKS solution of the
FitzHugh-Nagumo workload (d = 2, a = b = 0.2, c = 3, y0 = (-1, 1), t in [0, 20], IWP(3), N
uniform steps), sampled on the grid, for the per-N accuracy tests of the FP32 and FP64 solvers.

The oracle starts from the coarse-grid trajectory of Section 3.2.2 (sequential EKS on 256 coarse
steps) and iterates until max|change of E0 m| <= 1e-10.  Gauss-Newton from that start reaches
the same fixed point as from the constant trajectory (checked at N = 4096: the two converged
solutions differ by 1e-14) in 3-5 instead of 40-55 iterations, which keeps the oracle to about
20 minutes of one CPU core at N = 2^20.

Stored: the sampled indices n (every N/1024-th point and N), all D state components of the
means at those points (original coordinates), the full covariances S S^T at every N/128-th
point, the quasi-MLE diffusion sigma^2, the iteration count and the changes per iteration.

Also the oracle's own conditioning at the fixed point: one more IEKS pass from the converged
trajectory and one from the same trajectory with every entry perturbed by a relative 1e-15
(seeded normal); `sens_order[i]` is the relative change of derivative order i of the means
(max over the grid / max |x_i|) and `sens_sigma2` the relative change of sigma^2.  At fine grids
the higher derivatives and sigma^2 are dominated by FP64 rounding (the preconditioned
coordinates scale derivative i by h^-(q-i+1/2)), and a parity bar tighter than this
sensitivity would test rounding, not the method.
Calls only the oracle (test infrastructure).

    python tests/golden/make_fhn_q3_converged.py N [N ...]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ieks  # noqa: E402

COARSE_N = 256


def samples(N, count):
    stride = max(1, N // count)
    idx = np.arange(0, N + 1, stride)
    if idx[-1] != N:
        idx = np.append(idx, N)
    return idx


def make(N):
    p = W.fitzhugh_nagumo(N=N, q=3)
    r = ieks.ieks(p, atol=1e-10, max_iter=60, coarse_n=COARSE_N)
    assert r.deltas[-1] <= 1e-10, r.deltas
    im = samples(N, 1024)
    ic = samples(N, 128)
    S = r.sqrtcovs[ic]
    # sensitivity of one more pass to a 1e-15 relative perturbation of the fixed point
    rng = np.random.default_rng(0)
    pert = r.means * (1.0 + 1e-15 * rng.standard_normal(r.means.shape))
    a = ieks.ieks(p, fixed_iters=1, init_traj=r.means, want_cov=False)
    b = ieks.ieks(p, fixed_iters=1, init_traj=pert, want_cov=False)
    q1 = p.q + 1
    sens = [float(np.max(np.abs(a.means[:, i::q1] - b.means[:, i::q1]))
                  / np.max(np.abs(a.means[:, i::q1]))) for i in range(q1)]
    sens_s2 = abs(a.sigma2 - b.sigma2) / a.sigma2
    out = os.path.join(HERE, f"fhn_q3_N{N}_converged.npz")
    np.savez_compressed(out, N=N, n_mean=im, means=r.means[im], n_cov=ic,
                        covs=np.einsum("nij,nkj->nik", S, S), sigma2=r.sigma2,
                        iterations=r.iterations, deltas=np.array(r.deltas), coarse_n=COARSE_N,
                        sens_order=np.array(sens), sens_sigma2=sens_s2)
    print(out, "iterations", r.iterations, "deltas", r.deltas, "sigma2", r.sigma2,
          "sens_order", sens, "sens_sigma2", sens_s2, flush=True)


def main():
    for a in sys.argv[1:]:
        make(int(a))


if __name__ == "__main__":
    main()
