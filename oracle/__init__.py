"""Plain, slow FP64 CPU oracle for the parallel-in-time probabilistic ODE solver.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the benchmark's CPU
baseline leg may import or run anything in this package.  The CUDA library never calls it and
shares no code, constants or helpers with it; the only thing both sides read is the problem
description in the ``workloads`` module.

What it computes (Bosch et al., "Parallel-in-Time Probabilistic Numerical ODE Solvers"):

* ``prior``      -- IWP(q) transition matrices Phi(h), Q(h) in closed form (Section 2.1) and the
                    step-size-free preconditioned form (Section 2.4, preconditioned transitions).
* ``taylor``     -- the exact initial state mu0 = [y0, y'(0), ..., y^(q)(0)] (Eq. mu0) by
                    Taylor-series recursion.
* ``odes``       -- vector fields and Jacobians of the test families, in float64.
* ``linalg``     -- the ``tria`` operator (Section 3.1.2).
* ``filtering``  -- the sequential square-root Kalman filter and RTS smoother, the paper's
                    square-root filtering/smoothing elements and associative operators
                    (Eqs. sqrt-filtering-elements, sqrt-associative-filtering,
                    sqrt-smoothing-elements, sqrt-associative-smoothing).
* ``ieks``       -- the iterated extended Kalman smoother (Algorithm 2), run sequentially: the
                    parallel solver computes the same numbers (Section 4.1), so a sequential
                    implementation is the definition the CUDA path is compared against; also
                    the quasi-maximum-likelihood diffusion estimate and the objective value
                    (Eq. objective-value).
* ``eks``        -- the sequential extended Kalman smoother with local linearisation (the
                    established sequential solver the paper compares against, Section 4.3).
* ``gp``         -- exact dense Gaussian conditioning for affine ODEs on tiny grids: an
                    independent pin of the whole linear smoother (Section 3.1).

Everything works in the paper's original (unpreconditioned) coordinates and in float64.
"""
