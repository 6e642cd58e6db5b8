// Internal host-side interface between the C ABI (pit_abi.cu) and the per-configuration
// kernel instantiations (pit_inst_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "../../include/pit.h"

namespace pit {

constexpr int kMaxOdeDim = 64;  // largest ODE dimension d accepted at the boundary

// Problem description after host-side validation.
struct Problem {
  int kind;
  int d;
  int q;
  double params[32];
  int n_params;
  double t0, t1;
  int64_t N;
  double y0[kMaxOdeDim];
};

struct SolveArgs {
  Problem pb;
  pit_opts opts;
  const double* grid;   // host, N+1 grid points of a non-uniform grid (null: uniform)
  const void* init_traj;
  void* mean;
  void* sqrtcov;
  pit_solve_info* info;
  void* workspace;
  size_t ws_bytes;
  cudaStream_t stream;
};

struct ScanArgs {
  int64_t N;
  int D;       // state dimension of the elements
  void* x0;  // A or E
  void* x1;  // b or g
  void* x2;  // C or L
  void* x3;  // eta
  void* x4;  // J
  int want_L;
  void* workspace;
  size_t ws_bytes;
  cudaStream_t stream;
};

// Error reporting (thread-local message) and launch accounting.
void set_error(const std::string& msg);
void count_launches(int64_t n);
int64_t launches_total();
// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// Kernel classes for the opt-in launch profiler (pit_profile_enable / pit_profile_read).
enum KernelClass {
  KC_INIT = 0, KC_RESIDUALS, KC_FILTER_REDUCE, KC_FILTER_DOWN, KC_SMOOTH_DOWN,
  KC_TREE_FILTER_UP, KC_TREE_FILTER_DOWN, KC_TREE_SMOOTH_UP, KC_TREE_SMOOTH_DOWN,
  KC_EXPORT, KC_SCAN_FILTER, KC_SCAN_SMOOTH, KC_LINEARIZE, KC_EKS_FILTER, KC_EKS_SMOOTH,
  KC_ITERATION, KC_COUNT
};
// Brackets one kernel launch: counts it and, when profiling is on, records CUDA events on the
// launch stream around it.
struct LaunchScope {
  int cls;
  cudaStream_t stream;
  cudaEvent_t begin;
  LaunchScope(int c, cudaStream_t s);
  ~LaunchScope();
};
#define PIT_LAUNCH(cls, stream, ...)            \
  do {                                           \
    ::pit::LaunchScope pit_scope_((cls), (stream)); \
    __VA_ARGS__;                                 \
  } while (0)

// Host-side validation of the C ABI arguments (PIT_OK or PIT_EINVAL with a message).
int fill_problem(const pit_ode* ode, int q, const double* y0, Problem& pb, bool need_y0 = true);
int fill_grid(const pit_grid* grid, Problem& pb);
int check_opts(const pit_opts* in, pit_opts& o);

// Host FP64 helpers shared by the instantiations.
int prior_blocks(int q, double h, double* Phi, double* Q, double* Phibar, double* sqrtQbar,
                 double* Tdiag);
int taylor_init(const Problem& pb, double* mu0);
// Per-point data of a non-uniform grid t[0..N] for IWP(q) with per-step preconditioning: SW =
// 2 (q+1) + 3 values per point n, [T(h_n) | T(h_{n-1}) / T(h_n) | h_n / q | T_0(h_n) |
// 1 / T_1(h_n)], h_n = t_n - t_{n-1} (h_0 = h_1).
int grid_step_data(const double* t, int64_t N, int q, double* out, int* SW);

// Per-configuration entry points (defined in the pit_inst_*.cu files).
using SolveFn = int (*)(const SolveArgs&, size_t* ws_query, bool eks);
using ScanFn = int (*)(const ScanArgs&, size_t* ws_query);

SolveFn find_solver(int dtype, int d, int q, int variant);
// The large-state solver (pit_dense_impl.cuh): any family and d with D = d (q+1) <= 256, EK1.
SolveFn find_dense_solver(int dtype);
ScanFn find_filter_scan(int dtype, int D);
ScanFn find_smooth_scan(int dtype, int D);

// Registration (each instantiation file registers its functions at static-init time).
struct Registrar {
  Registrar(int dtype, int d, int q, int variant, SolveFn fn);
};
struct DenseRegistrar {
  DenseRegistrar(int dtype, SolveFn fn);
  DenseRegistrar(int dtype, ScanFn filter_fn, ScanFn smooth_fn);  // generic element scans
};
// One request of the serving loop on the large-state kernels (d > 3): its workspace (from the
// server's pool) holds the trajectory and all scratch between iterations; each iterate() enqueues
// one IEKS iteration (residuals + filter and smoother passes) and the read-back of its
// reductions into `host` (page-locked, LargeScalars layout); advance() makes the new iterate the
// linearisation trajectory; export_means writes the means of the last iterate (or, after a
// diverged pass, of the one before) in original coordinates.
struct LargeScalars {
  double sigma2_sum, delta_max, y_max;
  unsigned int flags, pad;
  double objective;
};
class LargeSession {
 public:
  virtual ~LargeSession() {}
  virtual int start(const Problem& pb, const pit_opts& o, void* ws, size_t bytes,
                    cudaStream_t s) = 0;
  virtual int iterate(LargeScalars* host, cudaStream_t s) = 0;
  virtual void advance() = 0;
  virtual int export_means(void* mean, bool diverged, cudaStream_t s) = 0;
};
using LargeSessionFactory = LargeSession* (*)();
struct LargeSessionRegistrar {
  LargeSessionRegistrar(int dtype, LargeSessionFactory f);
};
LargeSessionFactory find_large_session(int dtype);
// Workspace bytes of a large-state session (0 with the error set when the problem is invalid).
size_t large_session_bytes(int dtype, const Problem& pb, const pit_opts& o);

// pit_linearize for any d (families with at most 32 parameters).
int dense_linearize_f32(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                        cudaStream_t s);
int dense_linearize_f64(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                        cudaStream_t s);
// Element scans of the large-state kernels (any D <= 256; ScanArgs::D gives D).
ScanFn find_dense_scan(int dtype, bool filter);
struct ScanRegistrar {
  ScanRegistrar(int dtype, int D, ScanFn filter_fn, ScanFn smooth_fn);
};

// ---- segmented (batched) solves -------------------------------------------------------------
// A layout slot: instance `id` occupies global points off .. off + N_id of the current pass and
// its linearisation trajectory is lin[cur].
struct SegSlot {
  int32_t id;
  int32_t cur;
  int64_t off;
};
// Per-instance reductions of one pass (same layout as the device-side InstAcc).
struct SegResult {
  double sigma2_sum;
  double delta_max;
  double y_max;
  unsigned int flags;
  unsigned int pad;
};
// Per-instance state of a batched solve iterated on the device (SegEngine::run_iterations);
// the same layout on host and device.
struct SegIterState {
  int32_t cur;        // lin[cur] is the instance's current linearisation trajectory
  int32_t iters;      // IEKS iterations it took part in
  int32_t active;     // still iterating
  int32_t converged;  // its stopping rule was met (or fixed_iters ran out)
  int32_t failed;     // non-finite or diverging values
  int32_t pad;
  double last_delta;  // max |change of E0 mean| of its last iteration
  double sigma2;      // quasi-MLE diffusion of its last pass (1 without calibration)
};

// Engine of one (dtype, d, q): device state of up to max_inst instances and the per-point
// buffers of passes over up to max_points global points.
class SegEngine {
 public:
  virtual ~SegEngine() {}
  virtual int state_dim() const = 0;
  virtual size_t traj_bytes(int64_t N) const = 0;   // one trajectory buffer, (N+1) x D
  virtual size_t workspace_bytes(int64_t max_points, int max_inst, bool want_cov,
                                 int chain_len) const = 0;
  virtual int bind(void* ws, size_t bytes, int64_t max_points, int max_inst, bool want_cov,
                   int chain_len) = 0;
  // Jacobian of the linearisation for every instance (pit_linearization)
  virtual void set_linearization(int mode) = 0;
  // host-side constants of instance `id` (prior, exact initial state, parameters) -> device
  virtual int set_instance(int id, const Problem& pb, void* lin0, void* lin1, void* mean,
                           void* cov, cudaStream_t s) = 0;
  // decoupled solves (approximate Jacobians, see solve_decoupled): instance `id` is component
  // k of the d-dimensional problem pb, with its (q+1)-block mu0k of the exact initial state;
  // outputs are written into the full (N+1) x d(q+1) mean and (N+1) x D x D covariance arrays
  virtual int set_component(int id, const Problem& pb, int k, const double* mu0k, void* lin0,
                            void* lin1, void* mean, void* cov, cudaStream_t s) = 0;
  // lin[cur] <- the constant initial trajectory mu0, for every slot
  virtual int init_traj(const SegSlot* slots, int n, cudaStream_t s) = 0;
  // one IEKS filter/smoother pass over the layout; means passes write lin[1 - cur], with_L
  // passes write the instance outputs (mean, cov).  Returns the per-slot reductions (host).
  virtual int pass(const SegSlot* slots, int n, bool with_L, int calibrate, SegResult* res,
                   cudaStream_t s) = 0;
  // the same pass split in two: pass_begin enqueues it (and the read-back of the reductions)
  // without waiting; pass_end waits for it and returns the reductions of the begun layout
  virtual int pass_begin(const SegSlot* slots, int n, bool with_L, int calibrate,
                         cudaStream_t s) = 0;
  // decoupled residuals: component instances read the whole state of their problem
  virtual void set_decoupled(bool on) = 0;
  virtual int pass_end(SegResult* res, cudaStream_t s) = 0;
  // page-locked host staging for slots, descriptors and reductions (optional; without it the
  // transfers go through pageable memory and pass_begin waits for the stream)
  virtual int use_pinned_staging() = 0;
  // mean <- T lin[1 - cur] (the last means pass), for every slot
  virtual int export_means(const SegSlot* slots, int n, cudaStream_t s) = 0;
  // Objective value (Eq. objective-value) of trajectory lin[slot.cur] of each slot, into out
  // (host, n values).  Synchronises s.
  virtual int objective(const SegSlot* slots, int n, double* out, cudaStream_t s) = 0;
  // All means iterations of instances 0..n-1 (trajectories initialised) in one cooperative
  // launch: per iteration the segmented IEKS pass, every instance's stopping rule and the
  // compaction of the active instances run on the device.  Fills out[0..n-1].  Returns
  // PIT_EUNSUPPORTED (nothing launched) when the layout does not fit one resident wave.
  virtual int run_iterations(int n, const pit_opts& o, double diverged_delta,
                             SegIterState* out, cudaStream_t s) = 0;
};
using SegFactory = SegEngine* (*)();
struct SegRegistrar {
  SegRegistrar(int dtype, int d, int q, SegFactory f);
};
SegFactory find_seg_engine(int dtype, int d, int q);

// ParaIEKS with an approximate (diagonal or zero) Jacobian, solved as d decoupled
// (q+1)-dimensional problems on the segmented engine (pit_seg.cu).
int solve_decoupled(const SolveArgs& a, size_t* ws_query);

// Workspace carving: 256-byte aligned bump allocator over a caller buffer.
struct Carver {
  char* base;
  size_t cap;
  size_t off;
  explicit Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c), off(0) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
  size_t used() const { return (off + 255) & ~size_t(255); }
};

#define PIT_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::pit::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));         \
      return PIT_ECUDA;                                                             \
    }                                                                               \
  } while (0)

}  // namespace pit
