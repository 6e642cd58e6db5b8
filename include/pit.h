/*
 * pit.h -- C ABI of the GB300 parallel-in-time probabilistic ODE solver.
 *
 * Bosch, Corenflos, Yaghoobi, Tronarp, Hennig, Saerkkae: "Parallel-in-Time Probabilistic
 * Numerical ODE Solvers" (JMLR 25, 2024).  The solver computes the probabilistic numerical
 * solution p(y(t_n) | y(0) = y0, {y'(t_m) = f(y(t_m), t_m)}) (Section 2, Eq. pnsol) of an
 * initial value problem y' = f(y, t), y(t0) = y0 (Eq. ivp) on a uniform grid, by the iterated
 * extended Kalman smoother of Algorithm 2 (ParaIEKS), whose linear smoothing step is the
 * time-parallel square-root Rauch-Tung-Striebel smoother of Algorithm 1 (ParaRTS).
 *
 * Conventions (all entry points):
 *  - Plain pointers and sizes only.  "host" pointers are CPU memory, "device" pointers are
 *    CUDA global memory of the current device.  The caller owns every buffer; the library
 *    never frees caller memory and never allocates device memory on the calls below: scratch
 *    space is a caller-provided device workspace whose size the *_workspace_size functions
 *    return.  A workspace that is too small gives PIT_ENOMEM.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Device
 *    work is enqueued on it.  Unless stated otherwise a call returns once its work is
 *    enqueued; pit_solve synchronises the stream (see there).
 *  - Matrices are row-major.  A state vector of an ODE of dimension d under an IWP(q) prior
 *    has D = d (q+1) entries ordered dimension-major, derivative-minor: entry k (q+1) + i is
 *    the i-th derivative of component k (E_i = I_d (x) e_i, Section 2.1).
 *  - Square-root factors are D x D matrices S with S S^T the covariance (left square roots,
 *    Section 3.1.2); narrower factors are zero-padded to D columns.
 *  - Floating point arithmetic on the device is in the dtype the call names (PIT_F32 or
 *    PIT_F64); device buffers have that element type.  Prior construction, the initial state
 *    and the diffusion sum are always computed in FP64.
 *  - Errors: a non-zero pit_status; pit_last_error() gives a one-line, thread-local detail.
 *    Invalid arguments are rejected on the host before any device work (PIT_EINVAL).  No C++
 *    exception crosses the ABI.
 */
#ifndef PIT_H_
#define PIT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PIT_OK = 0,
  PIT_EINVAL = 1,       /* invalid argument (checked on the host)                        */
  PIT_ENOMEM = 2,       /* workspace smaller than the *_workspace_size value              */
  PIT_ECUDA = 3,        /* a CUDA runtime call failed                                     */
  PIT_ENOCONV = 4,      /* stopping rule not met within max_iter (outputs hold last iterate)*/
  PIT_ETIMEOUT = 5,     /* a bounded device-side wait expired                             */
  PIT_ENONFINITE = 6,   /* a non-finite value appeared in the device computation          */
  PIT_EINTERNAL = 7,    /* internal consistency check failed                             */
  PIT_EUNSUPPORTED = 8  /* valid request outside the compiled kernel set (e.g. d, q)      */
} pit_status;

typedef enum { PIT_F32 = 0, PIT_F64 = 1 } pit_dtype;

/* ODE families with device-side vector fields and Jacobians.  Parameter layouts:
 *   PIT_ODE_LOGISTIC         d=1  params = [r]               y' = r y (1 - y)            (Eq. logistic)
 *   PIT_ODE_FITZHUGH_NAGUMO  d=2  params = [a, b, c]         v' = c (v - v^3/3 + w), w' = -(v - a + b w)/c
 *   PIT_ODE_LOTKA_VOLTERRA   d=2  params = [al, be, ga, de]  x' = al x - be x y, y' = de x y - ga y
 *   PIT_ODE_LORENZ96         d>=4 params = [F]               x_i' = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F
 *   PIT_ODE_AFFINE           d    params = [L (d*d), c (d)]  y' = L y + c                (Eq. affine-ivp)
 *   PIT_ODE_RIGID_BODY       d=3  params = []                y' = (-2 y2 y3, 1.25 y1 y3, -0.5 y1 y2)
 *   PIT_ODE_VAN_DER_POL      d=2  params = [mu]              y1' = y2, y2' = mu ((1 - y1^2) y2 - y1)
 */
typedef enum {
  PIT_ODE_LOGISTIC = 0,
  PIT_ODE_FITZHUGH_NAGUMO = 1,
  PIT_ODE_LOTKA_VOLTERRA = 2,
  PIT_ODE_LORENZ96 = 3,
  PIT_ODE_AFFINE = 4,
  PIT_ODE_RIGID_BODY = 5,
  PIT_ODE_VAN_DER_POL = 6
} pit_ode_kind;

/* An initial value problem's vector field (Eq. ivp).  `params` is host memory, FP64. */
typedef struct {
  int32_t kind;          /* pit_ode_kind */
  int32_t d;             /* ODE dimension */
  const double* params;  /* host, n_params values (layout above) */
  int32_t n_params;
} pit_ode;

/* Uniform grid t_n = t0 + n (t1 - t0) / N, n = 0..N (N >= 1 steps, N observations). */
typedef struct {
  double t0;
  double t1;
  int64_t N;
} pit_grid;

/* Solver options.  pit_opts_default() fills the defaults given in brackets. */
typedef struct {
  int32_t max_iter;     /* [20]  iteration cap (>= 1)                                        */
  int32_t fixed_iters;  /* [0]   > 0: run exactly this many iterations, ignore the stop rule  */
  double atol_delta;    /* [1e-10] stop when max_n,k |y_n,k(new) - y_n,k(old)| <=            */
  double rtol_delta;    /* [0]     atol + rtol * max_n,k |y_n,k(new)|, y = E0 mean, original  */
                        /*         coordinates (the change in the solution estimate, Sec. 3.2.2)*/
  int32_t dtype;        /* [PIT_F64] device arithmetic and output element type              */
  int32_t calibrate;    /* [1]   quasi-MLE diffusion (Section 2.4) rescales the covariances */
  int32_t want_cov;     /* [1]   write square-root covariances (needs `sqrtcov`)            */
  int32_t chain_len;    /* [0]   time steps per sequential chain inside the scans, 0 = auto  */
  int32_t variant;      /* [0]   kernel layout: 0 = one state row per lane; 1 = two rows per
                                 lane (half the lanes per chain); 2 = approximate Jacobians as
                                 d decoupled components; 3 = the large-state kernels (one
                                 thread block per chain, any d with D <= 256; always used for
                                 d > 3 with the exact Jacobian); others PIT_EUNSUPPORTED      */
  int32_t linearization;/* [PIT_LIN_EK1] Jacobian of the linearisation (Sec. 3.2.1, remark on
                                 approximate Jacobians): exact, its diagonal, or zero         */
  int32_t objective;    /* [0]   1: evaluate the objective V (Eq. objective-value) of the
                                 initial trajectory and of every iterate (pit_solve_info)     */
  double atol_objective;/* [0]   second stopping criterion of Sec. 3.2.2: also stop when      */
  double rtol_objective;/* [0]   |V(k) - V(k-1)| <= atol_objective + rtol_objective |V(k)|;
                                 enabled (and V evaluated) when either is > 0                 */
  int32_t init_coarse;  /* [0]   > 0: initial trajectory from the sequential EKS on a coarse
                                 uniform grid of this many steps (<= N) over the same interval,
                                 the prior mean Phi(t - t_k) m_k between coarse nodes (Sec.
                                 3.2.2, remark on the initial trajectory); 0: constant mu0     */
  int32_t scan;         /* [0]   0: each IEKS iteration of a single-problem solve is one
                                 cooperative launch (residuals, chain folds, decoupled
                                 cross-block scans, down-sweeps) when the layout is variant 0,
                                 d <= 3 and the chains fit one resident wave, and all means
                                 iterations of a batched solve are one cooperative launch
                                 (stopping rules and compaction of the active instances on
                                 the device); else as 1.  1: one launch per scan phase with
                                 block-level scan trees, host-driven iteration loop          */
  int32_t tensor_cores; /* [1]   FP64 large-state solves (variant 3, d > 3 with EK1): 1 = the
                                 D x D products run on the tcgen05 tensor cores as exact
                                 products of 7-bit fixed-point digits (FP64 accuracy) when
                                 D >= 64; 2 = for any D; 0 = on the FP64 pipes.  No effect on
                                 FP32 solves or on the small-state kernels                    */
} pit_opts;

/* Linearisation of the vector field (pit_opts.linearization). */
typedef enum { PIT_LIN_EK1 = 0, PIT_LIN_DIAGONAL_EK1 = 1, PIT_LIN_EK0 = 2 } pit_linearization;

/* Per-solve report, written by pit_solve (host memory). */
typedef struct {
  int32_t iterations;   /* IEKS iterations performed (Algorithm 2 loop trips)               */
  int32_t converged;    /* 1 if the stopping rule was met (or fixed_iters was requested)    */
  double last_delta;    /* max |change of E0 mean| in the last iteration                    */
  double sigma2;        /* quasi-MLE diffusion sigma^2 (1 when calibrate == 0)              */
  int64_t kernel_launches; /* CUDA kernels this call launched                               */
  double deltas[64];    /* max |change of E0 mean| of iterations 1..min(iterations, 64) (0 when
                           fixed_iters skips the per-iteration readback)                     */
  double objective;     /* V of the returned means (0 unless V is evaluated, see pit_opts)  */
  double objectives[65];/* V of the initial trajectory and of iterations 1..64 (same)       */
} pit_solve_info;

/* ---- library ------------------------------------------------------------------------- */

/* Version string, e.g. "pit 0.1 sm_103a". */
const char* pit_version(void);
/* Static description of a status code. */
const char* pit_status_string(int32_t status);
/* Thread-local detail of the last error on this thread ("" if none). */
const char* pit_last_error(void);
/* Total CUDA kernels launched by this process through the library (monotone counter). */
int64_t pit_launch_count(void);
/* Fill `opts` with the defaults documented in pit_opts. */
void pit_opts_default(pit_opts* opts);

/* Opt-in launch profiler.  While enabled, each kernel launch of the library is bracketed by two
 * CUDA events recorded on its stream.  pit_profile_read waits for outstanding events and
 * reports, per kernel class, the accumulated device time (ms) and launch count since the last
 * pit_profile_reset: names (may be NULL) receives max_classes entries of 32 chars each,
 * total_ms and launches (may be NULL) max_classes values.  Returns the number of classes the
 * library defines (fill up to min(max_classes, that number)).  Host only, thread-safe. */
void pit_profile_enable(int32_t on);
void pit_profile_reset(void);
int32_t pit_profile_read(int32_t max_classes, char* names, double* total_ms, int64_t* launches);

/* ---- prior and initial state (host, FP64) --------------------------------------------- */

/* IWP(q) prior of one ODE dimension (Section 2.1) and its preconditioned form (Section 2.4,
 * "preconditioned state transitions").  Outputs (host, each may be NULL):
 *   Phi, Q        (q+1) x (q+1)  closed-form transition and process-noise covariance, sigma = 1:
 *                                [Phi]_ij = h^(j-i)/(j-i)! (j >= i), [Q]_ij = h^(2q+1-i-j) /
 *                                ((2q+1-i-j) (q-i)! (q-j)!)
 *   Phibar        (q+1) x (q+1)  binom(q-i, j-i) (j >= i): step-size free transition
 *   sqrtQbar      (q+1) x (q+1)  lower Cholesky factor of Qbar_ij = 1/(2q+1-i-j)
 *   Tdiag         (q+1)          diagonal of T(h) = sqrt(h) diag(h^(q-i)/(q-i)!), so that
 *                                Phi = T Phibar T^-1 and Q = T Qbar T
 * The full D x D matrices are I_d (x) these blocks.  Errors: PIT_EINVAL if q < 1, q > 8 or
 * h is not a positive finite number. */
int32_t pit_prior(int32_t q, double h, double* Phi, double* Q, double* Phibar, double* sqrtQbar,
                  double* Tdiag);

/* Exact initial state mu0 = [y0, y'(t0), ..., y^(q)(t0)] (Eq. mu0) by Taylor-mode recursion on
 * the family's polynomial vector field.  y0: host, d values; mu0: host, D = d (q+1) values in
 * the state layout above.  Errors: PIT_EINVAL for an unknown family, a bad d or n_params, or a
 * non-finite y0. */
int32_t pit_init_state(const pit_ode* ode, int32_t q, const double* y0, double* mu0);

/* ---- device building blocks -------------------------------------------------------------- */

/* First-order Taylor linearisation of the information operator at all grid points at once
 * (Section 3.2.1, Eq. linearized-observation-model):
 *   H_n = E1 - F_y(E0 traj_n, t_n) E0,   d_n = f(E0 traj_n, t_n) - F_y(E0 traj_n, t_n) E0 traj_n
 * for n = 1..N.  traj: device, (N+1) x D, original coordinates (row n = linearisation point at
 * t_n; row 0 is not read).  H: device, N x d x D (row n-1 holds H_n); dvec: device, N x d.
 * Asynchronous.  Errors: PIT_EINVAL for bad sizes/pointers, PIT_EUNSUPPORTED for a family with
 * more than 32 parameters (the affine family beyond d = 5; pit_solve linearises it itself). */
int32_t pit_linearize(const pit_ode* ode, const pit_grid* grid, int32_t q, int32_t dtype,
                      const void* traj, void* H, void* dvec, void* stream);
/* pit_linearize with an approximate Jacobian (Section 3.2.1, remark on approximate Jacobians):
 * F_y is replaced by its diagonal (PIT_LIN_DIAGONAL_EK1) or by zero (PIT_LIN_EK0) in both H_n and
 * d_n; PIT_LIN_EK1 is pit_linearize.  Other arguments, layouts and errors as pit_linearize, plus
 * PIT_EINVAL for an unknown linearization. */
int32_t pit_linearize_approx(const pit_ode* ode, const pit_grid* grid, int32_t q, int32_t dtype,
                             int32_t linearization, const void* traj, void* H, void* dvec,
                             void* stream);

/* Bytes of device workspace pit_filter_scan needs for N elements of dimension D. */
int32_t pit_filter_scan_workspace_size(int64_t N, int32_t D, int32_t dtype, size_t* bytes);

/* Inclusive time-parallel scan of square-root filtering elements with the associative
 * operator of Eq. sqrt-associative-filtering (Section 3.1.2):
 *   a_1, ..., a_N  ->  a_1 (x)_f a_2 (x)_f ... (x)_f a_n,  n = 1..N  (in place).
 * Element n is (A_n, b_n, C_n = sqrt(C_n), eta_n, J_n = sqrt(J_n)); device arrays
 * A, C, J: N x D x D, b, eta: N x D, all of `dtype`.  For elements built as in Eq.
 * sqrt-filtering-elements the outputs b, C are the filtering means and square-root
 * covariances m^f_n, sqrt(P^f_n).  Output factors C, J are lower-triangular; they are
 * square roots of the same matrices as the paper's but their column signs are not fixed.
 * Asynchronous.  Errors: PIT_EINVAL (N < 1, D < 1, null pointer), PIT_EUNSUPPORTED (D not
 * 1..256), PIT_ENOMEM (workspace too small).  D in {2, 3, 4, 6, 8} runs on lane-group kernels,
 * every other D on the large-state kernels (one thread block per chain of elements; chain
 * aggregates scanned by tree levels inside groups of 8 chains and a look-back across groups). */
int32_t pit_filter_scan(int64_t N, int32_t D, int32_t dtype, void* A, void* b, void* C,
                        void* eta, void* J, void* workspace, size_t ws_bytes, void* stream);

/* Bytes of device workspace pit_smooth_scan needs. */
int32_t pit_smooth_scan_workspace_size(int64_t N, int32_t D, int32_t dtype, int32_t want_L,
                                       size_t* bytes);

/* Reverse inclusive time-parallel scan of square-root smoothing elements with the operator of
 * Eq. sqrt-associative-smoothing (Section 3.1.3):
 *   b_n (x)_s b_{n+1} (x)_s ... (x)_s b_{N-1},  n = 0..N-1  (in place; N elements here).
 * Element n is (E_n, g_n, L_n = sqrt(L_n)); device arrays E, L: N x D x D, g: N x D.  For
 * smoothing elements built as in Eq. sqrt-smoothing-elements the outputs g, L are the
 * smoothing means and square-root covariances.  want_L = 0 skips the covariance part (L may be
 * NULL).  Asynchronous.  Errors as pit_filter_scan. */
int32_t pit_smooth_scan(int64_t N, int32_t D, int32_t dtype, void* E, void* g, void* L,
                        int32_t want_L, void* workspace, size_t ws_bytes, void* stream);

/* ---- the solver (Algorithm 2) ------------------------------------------------------------ */

/* Bytes of device workspace pit_solve needs for this problem. */
int32_t pit_solve_workspace_size(const pit_ode* ode, const pit_grid* grid, int32_t q,
                                 const pit_opts* opts, size_t* bytes);

/* ParaIEKS (Algorithm 2): exact initial state (Eq. mu0), constant initial trajectory
 * eta_n = mu0 (or `init_traj`), then repeat { linearise at all n (Section 3.2.1); time-parallel
 * square-root filter and smoother (Algorithm 1) } until the stopping rule of pit_opts holds or
 * max_iter iterations ran.  The quasi-MLE diffusion sigma^2 = (1/(N d)) sum_n ||sqrtS_n^-1 r_n||^2
 * of the final iteration's filter pass (Section 2.4) rescales the covariances when calibrate
 * is set; means do not depend on sigma.
 *   ode, grid, q, y0   problem (host); y0 has d values; 1 <= q <= 3 for the compiled kernels
 *   opts               host, NULL = defaults
 *   init_traj          optional device (N+1) x D warm-start trajectory in original
 *                      coordinates, of `dtype`; NULL = Algorithm 2's constant guess
 *   mean               device, (N+1) x D, `dtype`: smoothing means E[Y(t_n)], original coords
 *   sqrtcov            device, (N+1) x D x D, `dtype` (or NULL when want_cov = 0): square-root
 *                      covariances (calibrated), original coordinates
 *   info               host, may be NULL
 *   workspace          device, >= pit_solve_workspace_size bytes, 256-byte aligned
 * Work runs on `stream`; the call synchronises the stream once per iteration to read the
 * convergence scalar (once at the end with fixed_iters) and returns when the outputs are
 * complete.  Errors: PIT_EINVAL, PIT_EUNSUPPORTED (family/d/q without compiled kernels),
 * PIT_ENOMEM, PIT_ECUDA, PIT_ENONFINITE; PIT_ENOCONV when max_iter ran out (outputs hold the
 * last iterate). */
int32_t pit_solve(const pit_ode* ode, const pit_grid* grid, int32_t q, const double* y0,
                  const pit_opts* opts, const void* init_traj, void* mean, void* sqrtcov,
                  pit_solve_info* info, void* workspace, size_t ws_bytes, void* stream);

/* ParaIEKS (Algorithm 2) on a non-uniform grid t_0 < t_1 < ... < t_N (the method is stated on a
 * general grid: Sections 2.3 and 3.1 take the IWP transitions Phi(t_{n+1} - t_n),
 * Q(t_{n+1} - t_n) of Section 2.1 per step, Algorithm 2 a time grid).  Solved by the large-state kernels for any d, with
 * per-step preconditioning: in coordinates x_n = T(h_n) xbar_n (Section 2.4) the step into t_n
 * is xbar_n = Phibar diag(T(h_{n-1}) / T(h_n)) xbar_{n-1} + w, w ~ N(0, Qbar), h_0 = h_1.
 *   t                  host, N+1 grid points, finite and strictly increasing
 *   other arguments    as pit_solve (grid replaced by t, N); init_traj rows are at the t_n
 * Workspace size from pit_solve_grid_workspace_size.  Errors: as pit_solve; PIT_EINVAL for a
 * grid that is not strictly increasing (the message names the first bad index);
 * PIT_EUNSUPPORTED for init_coarse > 0 or the objective value (uniform grids only). */
int32_t pit_solve_grid_workspace_size(const pit_ode* ode, const double* t, int64_t N, int32_t q,
                                      const pit_opts* opts, size_t* bytes);
int32_t pit_solve_grid(const pit_ode* ode, const double* t, int64_t N, int32_t q,
                       const double* y0, const pit_opts* opts, const void* init_traj,
                       void* mean, void* sqrtcov, pit_solve_info* info, void* workspace,
                       size_t ws_bytes, void* stream);

/* Check of the bounded wait that the single-launch iterations (pit_opts.scan = 0) use between
 * thread blocks (no counterpart in the paper).  Launches one thread group that polls the flag
 * words[0] (device memory, 3 x uint32, 4-byte aligned: flag, status, result) until it is >=
 * target, at most poll_limit times.  Returns PIT_OK when the flag was seen, PIT_ETIMEOUT when
 * the wait gave up and set its timeout bit (a flag that nothing sets), PIT_EINVAL for bad
 * arguments.  words[1..2] are overwritten.  Synchronises `stream`. */
int32_t pit_check_wait(int64_t poll_limit, uint32_t target, void* words, void* stream);

/* Check of the FP64-accurate tensor-core product that the large-state solver uses for its dense
 * D x D products (Section 3.1.2's operators; the method itself is not in the paper).  One thread
 * block computes C = alpha op(A) op(B) + beta C in FP64 from 7-bit fixed-point digits of the
 * operands multiplied on the tcgen05 tensor cores (bf16 digits, exact FP32 accumulation, integer
 * recombination); the error of an output is below about 2^-52 k max|row of op(A)| max|column of
 * op(B)|.  op(A) = A (m x k, row-major, row stride lda) or, trans_a = 1, A^T with A k x m;
 * op(B) = B (k x n, stride ldb) or, trans_b = 1, B^T with B n x k; C m x n, stride ldc.  All
 * matrices are FP64 device memory owned by the caller; C must not alias A or B; beta == 0 does
 * not read C.  status: 2 x uint32 device words (overwritten: timeout bit 4, the product whose
 * wait gave up).  Returns PIT_OK, PIT_ETIMEOUT when a wait for the tensor cores gave up (after 4
 * s; the outputs are then NaN), PIT_EINVAL for sizes outside 0..4096, trans flags other than 0/1,
 * leading dimensions below the row lengths or null pointers.  Synchronises `stream`. */
int32_t pit_check_dgemm_tc(int32_t m, int32_t n, int32_t k, int32_t trans_a, int32_t trans_b,
                           double alpha, const void* A, int32_t lda, const void* B, int32_t ldb,
                           double beta, void* C, int32_t ldc, void* status, void* stream);

/* Check of the bounded wait of the tensor-core product (no counterpart in the paper): one block
 * allocates its tensor memory, waits on an mbarrier that nothing arrives on and frees the tensor
 * memory.  The wait must give up after wait_ns nanoseconds (0 .. 4e9) and set the timeout bit.
 * status: 2 x uint32 device words (overwritten).  Returns PIT_ETIMEOUT when it did so,
 * PIT_EINTERNAL otherwise, PIT_EINVAL for bad arguments.  Synchronises `stream`. */
int32_t pit_check_tc_wait(int64_t wait_ns, void* status, void* stream);

/* pit_solve for callers that cannot allocate device memory (no counterpart in the paper: this
 * is a deployment convenience).  Serving loops whose device memory budget is fixed at start-up,
 * plug-ins that run inside another framework's memory manager and have no device allocator of
 * their own, and real-time hosts that forbid allocation (and the synchronisation cudaMalloc may
 * bring) after initialisation cannot obtain a workspace for pit_solve; this entry point takes
 * none and uses a fixed 64 MiB scratch array in device memory that the library defines instead
 * (held by every GPU that loads the library until the process exits).  It allocates nothing
 * itself.  Arguments and outputs are those of pit_solve without workspace/ws_bytes.  The first
 * call on a device looks up the array's address on that device (with that device current) and
 * keeps it for the life of the process; do not reset the device (cudaDeviceReset) after it.  Every call shares the array (the solver
 * initialises all scratch it reads, so the previous call's contents are harmless); calls whose
 * device work overlaps race on it and must be serialised by the caller.  Errors: as pit_solve,
 * plus PIT_ENOMEM (with a message giving both sizes) when the problem needs more scratch than
 * the array holds. */
int32_t pit_solve_noalloc(const pit_ode* ode, const pit_grid* grid, int32_t q, const double* y0,
                          const pit_opts* opts, const void* init_traj, void* mean,
                          void* sqrtcov, pit_solve_info* info, void* stream);

/* Sequential extended Kalman smoother with local linearisation at the predicted mean (the
 * established sequential solver the paper compares against, Sections 2.3 and 4.3): one
 * forward filter pass and one backward RTS pass, strictly in time order, one thread group on
 * the GPU.  Same arguments and outputs as pit_solve (no iteration; opts->max_iter and the stop
 * rule are ignored); workspace size from pit_eks_workspace_size. */
int32_t pit_eks_workspace_size(const pit_ode* ode, const pit_grid* grid, int32_t q,
                               const pit_opts* opts, size_t* bytes);
int32_t pit_eks_sequential(const pit_ode* ode, const pit_grid* grid, int32_t q,
                           const double* y0, const pit_opts* opts, void* mean, void* sqrtcov,
                           pit_solve_info* info, void* workspace, size_t ws_bytes,
                           void* stream);

/* ---- batched (segmented) solves ------------------------------------------------------- */

/* Per-instance report of a batched solve (host memory). */
typedef struct {
  int32_t iterations;   /* IEKS iterations this instance took part in                      */
  int32_t converged;    /* 1 if its stopping rule was met (or fixed_iters was requested)    */
  int32_t status;       /* PIT_OK, PIT_ENOCONV, or PIT_ENONFINITE (diverged, see below)     */
  int32_t pad;
  double last_delta;    /* max |change of E0 mean| of its last iteration                    */
  double sigma2;        /* its quasi-MLE diffusion sigma^2 (1 when calibrate == 0)          */
  double objective;     /* V of its last iterate (Eq. objective-value) when pit_opts.objective
                           or the objective stopping rule asks for it, else 0               */
} pit_batch_info;

/* ParaIEKS (Algorithm 2) on B independent initial value problems of one ODE family, dimension
 * d and prior order q, each with its own parameters, initial value and uniform grid (any N).
 * No counterpart in the paper, which solves one problem at a time: the instances are laid end
 * to end on one time axis and solved by the same associative scans (Algorithm 1) in the same
 * kernel launches.  Each instance's first point enters the filtering scan as an element with
 * A = 0, sqrtC = 0, eta = 0, sqrtJ = 0 and its last point the smoothing scan as an element with
 * E = 0 (the boundary elements of Section 3.1.3, Eqs. filtering-elements and
 * smoothing-elements), so no value of one instance depends on another's and every instance gets
 * the result a single solve would give, up to the rounding of a different chain partition.
 * Each instance stops on its own rule (as pit_solve, including the objective rule of Section
 * 3.2.2 on its own V when atol_objective or rtol_objective is set) and then leaves the active
 * set; later iterations run on the remaining instances only.  Evaluating V (objective, or the
 * objective rule) runs the host-driven iteration loop whatever pit_opts.scan says.
 *   B                  number of instances (>= 1)
 *   odes               host, B entries; all of the same kind and d (parameters may differ)
 *   grids              host, B entries (t0 < t1, N >= 1 each)
 *   q                  prior order, shared
 *   y0                 host, B x d initial values
 *   opts               host, NULL = defaults (as pit_solve; init_traj is not supported)
 *   mean               device, sum_i (N_i + 1) rows of D values, `dtype`: instance i's
 *                      smoothing means start at row sum_{j<i} (N_j + 1); original coordinates
 *   sqrtcov            device, the same rows of D x D values, or NULL when want_cov = 0
 *   info               host, B entries, may be NULL
 *   workspace          device, >= pit_solve_batched_workspace_size bytes, 256-byte aligned
 * The call synchronises `stream` once per iteration (to read the per-instance change
 * statistics) and returns when the outputs are complete.  An instance whose change exceeds
 * 1e12 or turns non-finite is stopped with status PIT_ENONFINITE (its outputs hold its last
 * finite iterate); an overflow inside a pass can make the values of instances that share a
 * chain or tree node with it non-finite in that pass, which are then reported the same way.
 * Returns PIT_ENONFINITE if any instance diverged, else PIT_ENOCONV if any instance hit
 * max_iter, else PIT_OK; PIT_EINVAL (arguments, mixed kinds), PIT_EUNSUPPORTED, PIT_ENOMEM,
 * PIT_ECUDA as pit_solve. */
int32_t pit_solve_batched_workspace_size(int32_t B, const pit_ode* odes, const pit_grid* grids,
                                         int32_t q, const pit_opts* opts, size_t* bytes);
int32_t pit_solve_batched(int32_t B, const pit_ode* odes, const pit_grid* grids, int32_t q,
                          const double* y0, const pit_opts* opts, void* mean, void* sqrtcov,
                          pit_batch_info* info, void* workspace, size_t ws_bytes, void* stream);

/* ---- serving with continuous batching --------------------------------------------------- */

/* A solve server (no counterpart in the paper, which solves one problem at a time).  Requests
 * (an IVP, its grid and q) wait in a FIFO queue per (ODE family, d, q) class.  Each
 * pit_server_step admits queued requests into their class's batch while the class's point and
 * request capacity and the device memory budget allow (the head of a queue blocks the requests
 * behind it), runs ONE IEKS iteration (the loop body of Algorithm 2: linearisation and the
 * parallel filter and smoother of Algorithm 1, as pit_solve_batched) over every request in
 * flight -- each class on its own CUDA stream, so the classes' kernels overlap -- and retires
 * the requests whose stopping rule holds (as pit_solve: max|change of E0 mean| <= atol + rtol
 * max|E0 mean|, or max_iter iterations, or divergence as in pit_solve_batched).  Classes with
 * d > 3 (e.g. Lorenz-96) run on the large-state kernels: each such request has its own workspace
 * in the budget and takes one iteration per step on its class's stream.  A request's
 * trajectory stays in device memory from admission to retirement; the host reads back only
 * the per-request change statistics once per step.  Retired requests deliver their smoothing
 * means (original coordinates) and diffusion estimate, and on request (pit_server_submit_cov)
 * their square-root covariances.
 * The server allocates its whole device memory budget once, at creation, and never more.
 * Calls on one server must not overlap (they are serialised by a mutex). */
typedef struct pit_server pit_server;

typedef struct {
  int32_t dtype;            /* [PIT_F32] arithmetic and output element type                 */
  int32_t max_iter;         /* [20]    iteration cap per request                             */
  double atol_delta;        /* [1e-10] stopping rule (as pit_opts)                           */
  double rtol_delta;        /* [1e-6]                                                         */
  int32_t calibrate;        /* [1]     quasi-MLE diffusion estimate per request               */
  int32_t chain_len;        /* [0]     chain length inside the scans, 0 = auto               */
  int64_t max_points;       /* [2^22]  per class: sum of (N + 1) over requests in flight      */
  int32_t max_requests;     /* [1024]  per class: requests in flight                          */
  int32_t pad;
  size_t hbm_budget_bytes;  /* [8 GiB] device memory the server allocates at creation: the
                               classes' workspaces and the requests' trajectories (2 (N+1) D
                               values each, 8 bytes per value in FP32, 16 in FP64 rounded)     */
  double atol_objective;    /* [0]     objective rule of Sec. 3.2.2 per request (classes with
                               d <= 3): also stop when |V(k) - V(k-1)| <= atol_objective +  */
  double rtol_objective;    /* [0]     rtol_objective |V(k)|; enabled when either is > 0     */
} pit_server_config;

typedef struct {
  int64_t request_id;       /* id returned by pit_server_submit                              */
  uint64_t tag;             /* caller's tag                                                   */
  int32_t status;           /* PIT_OK (converged), PIT_ENOCONV (max_iter), PIT_ENONFINITE     */
  int32_t iterations;
  double last_delta;
  double sigma2;            /* quasi-MLE diffusion sigma^2 (1 when calibrate == 0)           */
  double t_submit;          /* pit_server_clock() at submission, admission and retirement   */
  double t_admit;
  double t_done;            /* the request's means are complete in its buffer at this time   */
  double objective;         /* V of its last iterate (Eq. objective-value) when the objective
                               rule is enabled and its class has d <= 3, else 0             */
} pit_server_result;

/* Fill `cfg` with the defaults in brackets above. */
void pit_server_config_default(pit_server_config* cfg);
/* Monotonic clock of the server's timestamps, in seconds. */
double pit_server_clock(void);
/* Create a server (allocates cfg->hbm_budget_bytes of device memory on the current device).
 * Errors: PIT_EINVAL (config), PIT_ENOMEM (allocation failed). */
int32_t pit_server_create(const pit_server_config* cfg, pit_server** out);
/* Queue a request.  ode, grid, y0: host, as pit_solve.  mean_out: device, (N+1) x D values of
 * the server's dtype, written when the request retires; the caller keeps it alive until then.
 * request_id (host, may be NULL) receives the request's id.  The first request of a class sets
 * up its kernels and workspace.  Errors: PIT_EINVAL (arguments, N + 1 above max_points),
 * PIT_EUNSUPPORTED (no compiled kernels), PIT_ENOMEM (budget cannot hold another class, or a
 * d > 3 request needs more device memory than the whole budget). */
int32_t pit_server_submit(pit_server* server, const pit_ode* ode, const pit_grid* grid,
                          int32_t q, const double* y0, void* mean_out, uint64_t tag,
                          int64_t* request_id);
/* pit_server_submit that also delivers square-root covariances.  sqrtcov_out: device,
 * (N+1) x D x D values of the server's dtype (row-major per grid point, original coordinates,
 * as pit_solve's sqrtcov), owned by the caller until the request retires.  When the request
 * retires with PIT_OK or PIT_ENOCONV, the server runs the covariance pass on the class's stream
 * before delivering the result: one IEKS iteration of Algorithm 1 linearised at the delivered
 * means, with the covariance recursions and, with calibrate, that pass's quasi-MLE diffusion
 * (Section 2.4).  This is the pass pit_solve ends with, taken at the final iterate.  The pass's
 * workspace and scratch means are reserved from the budget at admission, with the request's
 * trajectory.  Errors: as pit_server_submit, plus PIT_EINVAL for a NULL sqrtcov_out and
 * PIT_ENOMEM when the pass needs more than the whole budget.  A failing pass (e.g.
 * PIT_ENONFINITE) becomes the result's status. */
int32_t pit_server_submit_cov(pit_server* server, const pit_ode* ode, const pit_grid* grid,
                              int32_t q, const double* y0, void* mean_out, void* sqrtcov_out,
                              uint64_t tag, int64_t* request_id);
/* Admit, iterate once, retire (see above); waits for the iteration.  in_flight and queued
 * (host, may be NULL) receive the counts after the step. */
int32_t pit_server_step(pit_server* server, int32_t* in_flight, int32_t* queued);
/* Move up to `max` retired requests' results into out (host); *n receives the count. */
int32_t pit_server_poll(pit_server* server, pit_server_result* out, int32_t max, int32_t* n);
/* Device memory of the budget in use (bytes) and number of classes set up. */
int32_t pit_server_stats(pit_server* server, size_t* pool_used, int32_t* classes);
/* Wait for outstanding work and free the server and its device memory. */
void pit_server_destroy(pit_server* server);

#ifdef __cplusplus
}
#endif

#endif /* PIT_H_ */
