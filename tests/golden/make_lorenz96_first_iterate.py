"""Writes tests/golden/lorenz96_d64_N{N}_it1.npz: the FP64 oracle's first IEKS iterate for the
Lorenz-96 workload (d = 64, F = 8, IWP(2), t in [0, 5], constant initial trajectory) at the
benchmark's grid size, sampled every `stride` steps, with the maximal change and the
quasi-MLE diffusion of that iteration, and `sens`: the relative change of the sampled means
(max / max |means|) when every entry of the constant initial trajectory is perturbed by a relative
1e-15 (seeded normal) -- the amplification of rounding-level perturbations on this chaotic
workload, against which GPU results computed in another order are compared.  Calls only the
oracle (test infrastructure); takes a few minutes of one CPU core per 16384 steps and run.

    python tests/golden/make_lorenz96_first_iterate.py [N] [stride]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import ieks  # noqa: E402
from oracle.taylor import initial_state  # noqa: E402


def main():
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 16384
    stride = int(sys.argv[2]) if len(sys.argv) > 2 else 256
    p = W.lorenz96(d=64, N=N, q=2)
    r = ieks.ieks(p, fixed_iters=1, want_cov=False, calibrate=True)
    idx = np.arange(0, N + 1, stride)
    if idx[-1] != N:
        idx = np.append(idx, N)
    mu0 = initial_state(p.kind, p.params, p.y0, p.q)
    rng = np.random.default_rng(1)
    traj = np.tile(mu0, (N + 1, 1))
    traj = traj * (1.0 + 1e-15 * rng.standard_normal(traj.shape))
    rp = ieks.ieks(p, fixed_iters=1, want_cov=False, calibrate=True, init_traj=traj)
    sens = float(np.max(np.abs(rp.means[idx] - r.means[idx])) / np.max(np.abs(r.means[idx])))
    out = os.path.join(HERE, f"lorenz96_d64_N{N}_it1.npz")
    np.savez_compressed(out, n=idx, means=r.means[idx], delta=r.deltas[0], sigma2=r.sigma2,
                        N=N, sens=sens)
    print(out, "delta", r.deltas[0], "sigma2", r.sigma2, "sens", sens)


if __name__ == "__main__":
    main()
