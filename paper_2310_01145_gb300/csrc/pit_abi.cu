// C ABI of the solver (declared in include/pit.h): validation, host FP64 prior and initial
// state, dispatch to the per-configuration kernel sets, pit_linearize.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pit_internal.h"
#include "pit_ode.cuh"

namespace pit {

// ---- error state and accounting ----------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }

// ---- device geometry ---------------------------------------------------------------------------
// Streaming multiprocessors of the current device, queried once per device.  Launch shapes
// (chain lengths, grid caps) are derived from it.  Without a queryable device (a workspace-size
// query on a host with no GPU) GB300's count is assumed; the solve itself then fails at its
// first CUDA call.
int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 152;
  }
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
    cudaGetLastError();
    return 152;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

// ---- opt-in launch profiler ------------------------------------------------------------------
// When enabled, every kernel launch is bracketed by two CUDA events recorded on its stream;
// pit_profile_read() waits for the pending events and accumulates elapsed device time per
// kernel class.  Events are pooled and reused.
static const char* kClassNames[KC_COUNT] = {
    "init_traj",       "residuals",        "filter_reduce",    "filter_down",
    "smooth_down",     "tree_filter_up",   "tree_filter_down", "tree_smooth_up",
    "tree_smooth_down", "export_mean",     "scan_filter",      "scan_smooth",
    "linearize",       "eks_filter",       "eks_smooth",       "iteration"};
struct Profiler {
  std::atomic<bool> on{false};
  std::mutex mu;
  std::vector<cudaEvent_t> pool;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  double total_ms[KC_COUNT] = {};
  int64_t count[KC_COUNT] = {};
  cudaEvent_t take() {
    std::lock_guard<std::mutex> lk(mu);
    if (pool.empty()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
};
static Profiler& profiler() {
  static Profiler p;
  return p;
}

LaunchScope::LaunchScope(int c, cudaStream_t s) : cls(c), stream(s), begin(nullptr) {
  Profiler& p = profiler();
  if (p.on.load(std::memory_order_relaxed)) {
    begin = p.take();
    if (begin) cudaEventRecord(begin, s);
  }
}
LaunchScope::~LaunchScope() {
  count_launches(1);
  if (!begin) return;
  Profiler& p = profiler();
  cudaEvent_t end = p.take();
  if (!end) return;
  cudaEventRecord(end, stream);
  std::lock_guard<std::mutex> lk(p.mu);
  p.pending.push_back({cls, begin, end});
}

static void profile_flush() {
  Profiler& p = profiler();
  std::lock_guard<std::mutex> lk(p.mu);
  for (auto& r : p.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p.total_ms[r.cls] += ms;
      p.count[r.cls] += 1;
    }
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
}

// ---- registry -------------------------------------------------------------------------------
struct Registry {
  std::mutex mu;
  std::map<int, SolveFn> solvers;  // key variant*100000 + dtype*10000 + d*100 + q
  std::map<int, SolveFn> dense;    // key dtype
  std::map<int, ScanFn> dense_scans;  // key dtype*2 + (filter ? 1 : 0)
  std::map<int, LargeSessionFactory> sessions;  // key dtype
  std::map<int, ScanFn> fscans;    // key dtype*100 + D
  std::map<int, ScanFn> sscans;
};
static Registry& registry() {
  static Registry r;
  return r;
}
Registrar::Registrar(int dtype, int d, int q, int variant, SolveFn fn) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.solvers[variant * 100000 + dtype * 10000 + d * 100 + q] = fn;
}
DenseRegistrar::DenseRegistrar(int dtype, SolveFn fn) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.dense[dtype] = fn;
}
DenseRegistrar::DenseRegistrar(int dtype, ScanFn f, ScanFn sm) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.dense_scans[dtype * 2 + 1] = f;
  r.dense_scans[dtype * 2] = sm;
}
ScanFn find_dense_scan(int dtype, bool filter) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.dense_scans.find(dtype * 2 + (filter ? 1 : 0));
  return it == r.dense_scans.end() ? nullptr : it->second;
}
LargeSessionRegistrar::LargeSessionRegistrar(int dtype, LargeSessionFactory f) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.sessions[dtype] = f;
}
LargeSessionFactory find_large_session(int dtype) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.sessions.find(dtype);
  return it == r.sessions.end() ? nullptr : it->second;
}
size_t large_session_bytes_f32(const Problem& pb, const pit_opts& o);
size_t large_session_bytes_f64(const Problem& pb, const pit_opts& o);
size_t large_session_bytes(int dtype, const Problem& pb, const pit_opts& o) {
  return dtype == PIT_F64 ? large_session_bytes_f64(pb, o) : large_session_bytes_f32(pb, o);
}
SolveFn find_dense_solver(int dtype) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.dense.find(dtype);
  return it == r.dense.end() ? nullptr : it->second;
}
ScanRegistrar::ScanRegistrar(int dtype, int D, ScanFn f, ScanFn s) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.fscans[dtype * 100 + D] = f;
  r.sscans[dtype * 100 + D] = s;
}
SolveFn find_solver(int dtype, int d, int q, int variant) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.solvers.find(variant * 100000 + dtype * 10000 + d * 100 + q);
  return it == r.solvers.end() ? nullptr : it->second;
}
ScanFn find_filter_scan(int dtype, int D) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.fscans.find(dtype * 100 + D);
  return it == r.fscans.end() ? nullptr : it->second;
}
ScanFn find_smooth_scan(int dtype, int D) {
  Registry& r = registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.sscans.find(dtype * 100 + D);
  return it == r.sscans.end() ? nullptr : it->second;
}

// ---- host FP64 prior (Section 2.1) and preconditioner (Section 2.4) -----------------------
static double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}
static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  return factorial(n) / (factorial(k) * factorial(n - k));
}

int prior_blocks(int q, double h, double* Phi, double* Q, double* Phibar, double* sqrtQbar,
                 double* Tdiag) {
  if (q < 1 || q > 8 || !(h > 0.0) || !std::isfinite(h)) return PIT_EINVAL;
  const int K = q + 1;
  double Qb[81];
  for (int i = 0; i < K; ++i) {
    for (int j = 0; j < K; ++j) {
      const int p = 2 * q + 1 - i - j;
      if (Phi) Phi[i * K + j] = (j >= i) ? std::pow(h, j - i) / factorial(j - i) : 0.0;
      if (Q) Q[i * K + j] = std::pow(h, p) / (p * factorial(q - i) * factorial(q - j));
      if (Phibar) Phibar[i * K + j] = (j >= i) ? binom(q - i, j - i) : 0.0;
      Qb[i * K + j] = 1.0 / p;
    }
    if (Tdiag) Tdiag[i] = std::sqrt(h) * std::pow(h, q - i) / factorial(q - i);
  }
  if (sqrtQbar) {
    // Cholesky factor of the (well-conditioned for q <= 8) matrix Qbar, lower-triangular
    for (int i = 0; i < K * K; ++i) sqrtQbar[i] = 0.0;
    for (int j = 0; j < K; ++j) {
      double s = Qb[j * K + j];
      for (int k = 0; k < j; ++k) s -= sqrtQbar[j * K + k] * sqrtQbar[j * K + k];
      if (!(s > 0.0)) return PIT_EINTERNAL;
      const double djj = std::sqrt(s);
      sqrtQbar[j * K + j] = djj;
      for (int i = j + 1; i < K; ++i) {
        double t = Qb[i * K + j];
        for (int k = 0; k < j; ++k) t -= sqrtQbar[i * K + k] * sqrtQbar[j * K + k];
        sqrtQbar[i * K + j] = t / djj;
      }
    }
  }
  return PIT_OK;
}

// ---- exact initial state by Taylor-series recursion (Eq. mu0) ------------------------------
namespace {
constexpr int kMaxOrd = 10;
struct Ser {
  double c[kMaxOrd];
};
Ser s_const(double v) {
  Ser s{};
  s.c[0] = v;
  return s;
}
Ser s_add(const Ser& a, const Ser& b) {
  Ser s;
  for (int k = 0; k < kMaxOrd; ++k) s.c[k] = a.c[k] + b.c[k];
  return s;
}
Ser s_sub(const Ser& a, const Ser& b) {
  Ser s;
  for (int k = 0; k < kMaxOrd; ++k) s.c[k] = a.c[k] - b.c[k];
  return s;
}
Ser s_scale(const Ser& a, double f) {
  Ser s;
  for (int k = 0; k < kMaxOrd; ++k) s.c[k] = a.c[k] * f;
  return s;
}
Ser s_mul(const Ser& a, const Ser& b) {
  Ser s{};
  for (int k = 0; k < kMaxOrd; ++k)
    for (int j = 0; j <= k; ++j) s.c[k] += a.c[j] * b.c[k - j];
  return s;
}
// f applied to series y[0..d-1]
void f_series(const Problem& pb, const Ser* y, Ser* out) {
  const double* p = pb.params;
  switch (pb.kind) {
    case PIT_ODE_LOGISTIC:
      out[0] = s_scale(s_mul(y[0], s_sub(s_const(1.0), y[0])), p[0]);
      break;
    case PIT_ODE_FITZHUGH_NAGUMO: {
      const double a = p[0], b = p[1], c = p[2];
      Ser v3 = s_mul(s_mul(y[0], y[0]), y[0]);
      out[0] = s_scale(s_add(s_sub(y[0], s_scale(v3, 1.0 / 3.0)), y[1]), c);
      out[1] = s_scale(s_add(s_sub(y[0], s_const(a)), s_scale(y[1], b)), -1.0 / c);
      break;
    }
    case PIT_ODE_LOTKA_VOLTERRA: {
      Ser xy = s_mul(y[0], y[1]);
      out[0] = s_sub(s_scale(y[0], p[0]), s_scale(xy, p[1]));
      out[1] = s_sub(s_scale(xy, p[3]), s_scale(y[1], p[2]));
      break;
    }
    case PIT_ODE_VAN_DER_POL: {
      Ser one_m = s_sub(s_const(1.0), s_mul(y[0], y[0]));
      out[0] = y[1];
      out[1] = s_scale(s_sub(s_mul(one_m, y[1]), y[0]), p[0]);
      break;
    }
    case PIT_ODE_RIGID_BODY:
      out[0] = s_scale(s_mul(y[1], y[2]), -2.0);
      out[1] = s_scale(s_mul(y[0], y[2]), 1.25);
      out[2] = s_scale(s_mul(y[0], y[1]), -0.5);
      break;
    case PIT_ODE_AFFINE: {
      const int d = pb.d;
      for (int i = 0; i < d; ++i) {
        Ser acc = s_const(p[d * d + i]);
        for (int j = 0; j < d; ++j) acc = s_add(acc, s_scale(y[j], p[i * d + j]));
        out[i] = acc;
      }
      break;
    }
    case PIT_ODE_LORENZ96: {
      const int d = pb.d;
      for (int i = 0; i < d; ++i) {
        Ser t = s_mul(s_sub(y[(i + 1) % d], y[(i - 2 + d) % d]), y[(i - 1 + d) % d]);
        out[i] = s_add(s_sub(t, y[i]), s_const(p[0]));
      }
      break;
    }
    default:
      break;
  }
}
}  // namespace

int taylor_init(const Problem& pb, double* mu0) {
  const int d = pb.d, q = pb.q;
  if (q + 1 > kMaxOrd || d > kMaxOdeDim) return PIT_EINVAL;
  Ser y[kMaxOdeDim], fy[kMaxOdeDim];
  for (int i = 0; i < d; ++i) y[i] = s_const(pb.y0[i]);
  for (int k = 0; k < q; ++k) {
    f_series(pb, y, fy);
    for (int i = 0; i < d; ++i) y[i].c[k + 1] = fy[i].c[k] / (k + 1);
  }
  for (int i = 0; i < d; ++i)
    for (int k = 0; k <= q; ++k) mu0[i * (q + 1) + k] = factorial(k) * y[i].c[k];
  return PIT_OK;
}

// ---- validation ------------------------------------------------------------------------------
static int expected_params(int kind, int d) {
  switch (kind) {
    case PIT_ODE_LOGISTIC: return 1;
    case PIT_ODE_FITZHUGH_NAGUMO: return 3;
    case PIT_ODE_LOTKA_VOLTERRA: return 4;
    case PIT_ODE_LORENZ96: return 1;
    case PIT_ODE_AFFINE: return d * d + d;
    case PIT_ODE_RIGID_BODY: return 0;
    case PIT_ODE_VAN_DER_POL: return 1;
    default: return -1;
  }
}
static int expected_d(int kind, int d) {
  switch (kind) {
    case PIT_ODE_LOGISTIC: return 1;
    case PIT_ODE_FITZHUGH_NAGUMO:
    case PIT_ODE_LOTKA_VOLTERRA:
    case PIT_ODE_VAN_DER_POL: return 2;
    case PIT_ODE_RIGID_BODY: return 3;
    case PIT_ODE_AFFINE: return (d >= 1 && d <= 16) ? d : -1;
    case PIT_ODE_LORENZ96: return (d >= 4 && d <= kMaxOdeDim) ? d : -1;
    default: return -1;
  }
}

int fill_problem(const pit_ode* ode, int q, const double* y0, Problem& pb, bool need_y0) {
  if (!ode) {
    set_error("ode is NULL");
    return PIT_EINVAL;
  }
  std::memset(&pb, 0, sizeof(pb));
  pb.kind = ode->kind;
  pb.d = ode->d;
  pb.q = q;
  if (expected_d(ode->kind, ode->d) != ode->d) {
    set_error("unknown ODE family or dimension d not valid for it");
    return PIT_EINVAL;
  }
  const int np = expected_params(ode->kind, ode->d);
  if (np < 0 || ode->n_params != np || (np > 0 && !ode->params) || np > 32) {
    set_error("n_params / params do not match the ODE family");
    return PIT_EINVAL;
  }
  for (int i = 0; i < np; ++i) {
    if (!std::isfinite(ode->params[i])) {
      set_error("non-finite ODE parameter");
      return PIT_EINVAL;
    }
    pb.params[i] = ode->params[i];
  }
  pb.n_params = np;
  if (q < 1 || q > 8) {
    set_error("prior order q must be in 1..8");
    return PIT_EINVAL;
  }
  if (need_y0) {
    if (!y0) {
      set_error("y0 is NULL");
      return PIT_EINVAL;
    }
    for (int i = 0; i < ode->d; ++i) {
      if (!std::isfinite(y0[i])) {
        set_error("non-finite y0");
        return PIT_EINVAL;
      }
      pb.y0[i] = y0[i];
    }
  }
  return PIT_OK;
}

int fill_grid(const pit_grid* grid, Problem& pb) {
  if (!grid) {
    set_error("grid is NULL");
    return PIT_EINVAL;
  }
  if (!(grid->N >= 1) || grid->N > (int64_t(1) << 31) - 2) {
    set_error("grid N must be in 1..2^31-2");
    return PIT_EINVAL;
  }
  if (!std::isfinite(grid->t0) || !std::isfinite(grid->t1) || !(grid->t1 > grid->t0)) {
    set_error("grid needs finite t0 < t1");
    return PIT_EINVAL;
  }
  pb.t0 = grid->t0;
  pb.t1 = grid->t1;
  pb.N = grid->N;
  return PIT_OK;
}

int check_opts(const pit_opts* in, pit_opts& o) {
  pit_opts_default(&o);
  if (in) o = *in;
  if (o.max_iter < 1 || o.fixed_iters < 0 || !(o.atol_delta >= 0) || !(o.rtol_delta >= 0) ||
      (o.dtype != PIT_F32 && o.dtype != PIT_F64) || o.chain_len < 0 || o.chain_len > (1 << 20) ||
      o.variant < 0 || o.variant > 9 || o.linearization < 0 || o.linearization > 2 ||
      !(o.atol_objective >= 0) || !(o.rtol_objective >= 0) || o.init_coarse < 0 || o.scan < 0 || o.scan > 1 ||
      o.tensor_cores < 0 || o.tensor_cores > 2) {
    set_error("invalid pit_opts");
    return PIT_EINVAL;
  }
  return PIT_OK;
}

int grid_step_data(const double* t, int64_t N, int q, double* out, int* SW) {
  const int Q1 = q + 1;
  *SW = 2 * Q1 + 3;
  double Phib[64], sqb[64], Td[8], Tprev[8];
  for (int64_t n = 0; n <= N; ++n) {
    const double h = n == 0 ? t[1] - t[0] : t[n] - t[n - 1];
    if (prior_blocks(q, h, nullptr, nullptr, Phib, sqb, Td) != PIT_OK) return PIT_EINVAL;
    double* g = out + n * *SW;
    for (int i = 0; i < Q1; ++i) {
      g[i] = Td[i];
      g[Q1 + i] = n == 0 ? 1.0 : Tprev[i] / Td[i];
      Tprev[i] = Td[i];
    }
    g[2 * Q1] = h / q;
    g[2 * Q1 + 1] = Td[0];
    g[2 * Q1 + 2] = 1.0 / Td[1];
  }
  return PIT_OK;
}

// ---- pit_linearize kernel ---------------------------------------------------------------------
template <typename T, int DD>
__global__ void k_linearize(OdeParams<T> ode, int64_t N, int Q1, double t0, double h,
                            int lin_mode, const T* __restrict__ traj, T* __restrict__ H,
                            T* __restrict__ dv) {
  const int D = DD * Q1;
  for (int64_t n = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= N;
       n += (int64_t)gridDim.x * blockDim.x) {
    T y[DD], f[DD], F[DD][DD];
    for (int k = 0; k < DD; ++k) y[k] = traj[n * D + k * Q1];
    ode_eval<T, DD>(ode, y, f, F);
    approximate_jacobian<T, DD>(lin_mode, F);
    T* Hn = H + (n - 1) * DD * D;
    for (int k = 0; k < DD; ++k) {
      T acc = f[k];
      for (int c = 0; c < D; ++c) Hn[k * D + c] = T(0);
      Hn[k * D + k * Q1 + 1] = T(1);
      for (int m = 0; m < DD; ++m) {
        Hn[k * D + m * Q1] -= F[k][m];
        acc -= F[k][m] * y[m];
      }
      dv[(n - 1) * DD + k] = acc;
    }
  }
}

template <typename T, int DD>
static int launch_linearize(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                            cudaStream_t s) {
  OdeParams<T> op;
  std::memset(&op, 0, sizeof(op));
  op.kind = pb.kind;
  op.d = pb.d;
  for (int i = 0; i < pb.n_params; ++i) op.p[i] = static_cast<T>(pb.params[i]);
  const double h = (pb.t1 - pb.t0) / static_cast<double>(pb.N);
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>((pb.N + 255) / 256, int64_t(sm_count()) * 16));
  PIT_LAUNCH(KC_LINEARIZE, s, 
             k_linearize<T, DD><<<grid, 256, 0, s>>>(op, pb.N, pb.q + 1, pb.t0, h, lin_mode,
                                           static_cast<const T*>(traj), static_cast<T*>(H),
                                           static_cast<T*>(dv)););
  PIT_CUDA_TRY(cudaGetLastError());
  return PIT_OK;
}

}  // namespace pit

using namespace pit;

extern "C" {

const char* pit_version(void) { return "pit 0.1 sm_103a"; }

const char* pit_status_string(int32_t s) {
  switch (s) {
    case PIT_OK: return "ok";
    case PIT_EINVAL: return "invalid argument";
    case PIT_ENOMEM: return "workspace too small";
    case PIT_ECUDA: return "CUDA runtime error";
    case PIT_ENOCONV: return "stopping rule not met within max_iter";
    case PIT_ETIMEOUT: return "bounded device wait expired";
    case PIT_ENONFINITE: return "non-finite value in the computation";
    case PIT_EINTERNAL: return "internal error";
    case PIT_EUNSUPPORTED: return "configuration not compiled";
    default: return "unknown status";
  }
}

const char* pit_last_error(void) { return g_err.c_str(); }

int64_t pit_launch_count(void) { return launches_total(); }

void pit_profile_enable(int32_t on) {
  if (!on) profile_flush();
  profiler().on.store(on != 0);
}

void pit_profile_reset(void) {
  profile_flush();
  Profiler& p = profiler();
  std::lock_guard<std::mutex> lk(p.mu);
  for (int i = 0; i < KC_COUNT; ++i) {
    p.total_ms[i] = 0.0;
    p.count[i] = 0;
  }
}

int32_t pit_profile_read(int32_t max_classes, char* names, double* total_ms, int64_t* launches) {
  profile_flush();
  Profiler& p = profiler();
  std::lock_guard<std::mutex> lk(p.mu);
  const int n = std::min<int>(max_classes, KC_COUNT);
  for (int i = 0; i < n; ++i) {
    if (names) {
      std::memset(names + 32 * i, 0, 32);
      std::strncpy(names + 32 * i, kClassNames[i], 31);
    }
    if (total_ms) total_ms[i] = p.total_ms[i];
    if (launches) launches[i] = p.count[i];
  }
  return KC_COUNT;
}

void pit_opts_default(pit_opts* o) {
  if (!o) return;
  o->max_iter = 20;
  o->fixed_iters = 0;
  o->atol_delta = 1e-10;
  o->rtol_delta = 0.0;
  o->dtype = PIT_F64;
  o->calibrate = 1;
  o->want_cov = 1;
  o->chain_len = 0;
  o->variant = 0;
  o->linearization = PIT_LIN_EK1;
  o->objective = 0;
  o->atol_objective = 0.0;
  o->rtol_objective = 0.0;
  o->init_coarse = 0;
  o->scan = 0;
  o->tensor_cores = 1;
}

int32_t pit_prior(int32_t q, double h, double* Phi, double* Q, double* Phibar, double* sqrtQbar,
                  double* Tdiag) {
  g_err.clear();
  const int st = prior_blocks(q, h, Phi, Q, Phibar, sqrtQbar, Tdiag);
  if (st != PIT_OK) set_error("pit_prior: need 1 <= q <= 8 and finite h > 0");
  return st;
}

int32_t pit_init_state(const pit_ode* ode, int32_t q, const double* y0, double* mu0) {
  g_err.clear();
  Problem pb;
  int st = fill_problem(ode, q, y0, pb);
  if (st != PIT_OK) return st;
  if (!mu0) {
    set_error("mu0 is NULL");
    return PIT_EINVAL;
  }
  return taylor_init(pb, mu0);
}

int32_t pit_linearize(const pit_ode* ode, const pit_grid* grid, int32_t q, int32_t dtype,
                      const void* traj, void* H, void* dvec, void* stream) {
  return pit_linearize_approx(ode, grid, q, dtype, PIT_LIN_EK1, traj, H, dvec, stream);
}

int32_t pit_linearize_approx(const pit_ode* ode, const pit_grid* grid, int32_t q, int32_t dtype,
                             int32_t linearization, const void* traj, void* H, void* dvec,
                             void* stream) {
  g_err.clear();
  if (linearization < PIT_LIN_EK1 || linearization > PIT_LIN_EK0) {
    set_error("pit_linearize_approx: linearization must be EK1, DiagonalEK1 or EK0");
    return PIT_EINVAL;
  }
  Problem pb;
  int st = fill_problem(ode, q, nullptr, pb, false);
  if (st != PIT_OK) return st;
  st = fill_grid(grid, pb);
  if (st != PIT_OK) return st;
  if (!traj || !H || !dvec || (dtype != PIT_F32 && dtype != PIT_F64)) {
    set_error("pit_linearize: null buffer or bad dtype");
    return PIT_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool f64 = dtype == PIT_F64;
  switch (pb.d) {
    case 1: return f64 ? launch_linearize<double, 1>(pb, linearization, traj, H, dvec, s)
                       : launch_linearize<float, 1>(pb, linearization, traj, H, dvec, s);
    case 2: return f64 ? launch_linearize<double, 2>(pb, linearization, traj, H, dvec, s)
                       : launch_linearize<float, 2>(pb, linearization, traj, H, dvec, s);
    case 3: return f64 ? launch_linearize<double, 3>(pb, linearization, traj, H, dvec, s)
                       : launch_linearize<float, 3>(pb, linearization, traj, H, dvec, s);
    default:
      return f64 ? dense_linearize_f64(pb, linearization, traj, H, dvec, s)
                 : dense_linearize_f32(pb, linearization, traj, H, dvec, s);
  }
}

static int32_t scan_common(bool filter, int64_t N, int32_t D, int32_t dtype, void* x0, void* x1,
                           void* x2, void* x3, void* x4, int want_L, void* ws, size_t wsb,
                           void* stream, size_t* query) {
  if (N < 1 || D < 1 || (dtype != PIT_F32 && dtype != PIT_F64)) {
    set_error("scan: need N >= 1, D >= 1, dtype F32/F64");
    return PIT_EINVAL;
  }
  ScanFn fn = filter ? find_filter_scan(dtype, D) : find_smooth_scan(dtype, D);
  // other D up to 256: the large-state kernels' block-level operators
  if (!fn && D <= 256) fn = find_dense_scan(dtype, filter);
  if (!fn) {
    set_error("scan: D=" + std::to_string(D) + " not supported (1..256)");
    return PIT_EUNSUPPORTED;
  }
  ScanArgs a{N, D, x0, x1, x2, x3, x4, want_L, ws, wsb, static_cast<cudaStream_t>(stream)};
  if (query) return fn(a, query);
  if (!x0 || !x1 || (filter && (!x2 || !x3 || !x4)) || (!filter && want_L && !x2) || !ws) {
    set_error("scan: null buffer");
    return PIT_EINVAL;
  }
  return fn(a, nullptr);
}

int32_t pit_filter_scan_workspace_size(int64_t N, int32_t D, int32_t dtype, size_t* bytes) {
  g_err.clear();
  if (!bytes) return PIT_EINVAL;
  return scan_common(true, N, D, dtype, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr,
                     0, nullptr, bytes);
}

int32_t pit_filter_scan(int64_t N, int32_t D, int32_t dtype, void* A, void* b, void* C,
                        void* eta, void* J, void* workspace, size_t ws_bytes, void* stream) {
  g_err.clear();
  return scan_common(true, N, D, dtype, A, b, C, eta, J, 0, workspace, ws_bytes, stream,
                     nullptr);
}

int32_t pit_smooth_scan_workspace_size(int64_t N, int32_t D, int32_t dtype, int32_t want_L,
                                       size_t* bytes) {
  g_err.clear();
  if (!bytes) return PIT_EINVAL;
  return scan_common(false, N, D, dtype, nullptr, nullptr, nullptr, nullptr, nullptr, want_L,
                     nullptr, 0, nullptr, bytes);
}

int32_t pit_smooth_scan(int64_t N, int32_t D, int32_t dtype, void* E, void* g, void* L,
                        int32_t want_L, void* workspace, size_t ws_bytes, void* stream) {
  g_err.clear();
  return scan_common(false, N, D, dtype, E, g, L, nullptr, nullptr, want_L, workspace, ws_bytes,
                     stream, nullptr);
}

static int32_t solve_common(const pit_ode* ode, const pit_grid* grid, int32_t q,
                            const double* y0, const pit_opts* opts, const void* init_traj,
                            void* mean, void* sqrtcov, pit_solve_info* info, void* workspace,
                            size_t ws_bytes, void* stream, size_t* query, bool eks) {
  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  int st = fill_problem(ode, q, y0, a.pb, query == nullptr);
  if (st != PIT_OK) return st;
  st = fill_grid(grid, a.pb);
  if (st != PIT_OK) return st;
  st = check_opts(opts, a.opts);
  if (st != PIT_OK) return st;
  // approximate Jacobians decouple the components (variant 2, and always for d > 3)
  if (!eks && a.opts.linearization != PIT_LIN_EK1 && (a.opts.variant == 2 || a.pb.d > 3)) {
    a.init_traj = init_traj;
    a.mean = mean;
    a.sqrtcov = sqrtcov;
    a.info = info;
    a.workspace = workspace;
    a.ws_bytes = ws_bytes;
    a.stream = static_cast<cudaStream_t>(stream);
    if (query) return solve_decoupled(a, query);
    if (!mean || (a.opts.want_cov && !sqrtcov) || !workspace) {
      set_error("null output or workspace buffer");
      return PIT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) {
      set_error("workspace must be 256-byte aligned");
      return PIT_EINVAL;
    }
    return solve_decoupled(a, nullptr);
  }
  if (a.opts.variant == 2) {
    set_error("variant 2 (decoupled components) needs an approximate Jacobian");
    return PIT_EINVAL;
  }
  // the large-state solver: every d > 3 (exact Jacobian), and any d with variant 3
  SolveFn fn = (a.pb.d > 3 || a.opts.variant == 3) ? find_dense_solver(a.opts.dtype)
                                                   : find_solver(a.opts.dtype, a.pb.d, q, a.opts.variant);
  if (!fn) {
    set_error("no compiled kernels for this (dtype, d, q, variant); compiled: d in 1..3, q in 1..3 "
              "(d=3: q <= 2), variant 1 for D = d (q+1) in {6, 8}");
    return PIT_EUNSUPPORTED;
  }
  a.init_traj = init_traj;
  a.mean = mean;
  a.sqrtcov = sqrtcov;
  a.info = info;
  a.workspace = workspace;
  a.ws_bytes = ws_bytes;
  a.stream = static_cast<cudaStream_t>(stream);
  if (query) {
    if (query) *query = 0;
    return fn(a, query, eks);
  }
  if (!mean || (a.opts.want_cov && !sqrtcov) || !workspace) {
    set_error("null output or workspace buffer");
    return PIT_EINVAL;
  }
  return fn(a, nullptr, eks);
}

int32_t pit_solve_workspace_size(const pit_ode* ode, const pit_grid* grid, int32_t q,
                                 const pit_opts* opts, size_t* bytes) {
  g_err.clear();
  if (!bytes) return PIT_EINVAL;
  return solve_common(ode, grid, q, nullptr, opts, nullptr, nullptr, nullptr, nullptr, nullptr,
                      0, nullptr, bytes, false);
}

int32_t pit_solve(const pit_ode* ode, const pit_grid* grid, int32_t q, const double* y0,
                  const pit_opts* opts, const void* init_traj, void* mean, void* sqrtcov,
                  pit_solve_info* info, void* workspace, size_t ws_bytes, void* stream) {
  g_err.clear();
  return solve_common(ode, grid, q, y0, opts, init_traj, mean, sqrtcov, info, workspace,
                      ws_bytes, stream, nullptr, false);
}

// ParaIEKS on a non-uniform grid: the large-state kernels with per-step preconditioning.
static int32_t solve_grid_common(const pit_ode* ode, const double* t, int64_t N, int32_t q,
                                 const double* y0, const pit_opts* opts, const void* init_traj,
                                 void* mean, void* sqrtcov, pit_solve_info* info,
                                 void* workspace, size_t ws_bytes, void* stream, size_t* query) {
  if (!t) {
    set_error("grid points are NULL");
    return PIT_EINVAL;
  }
  if (!(N >= 1) || N > (int64_t(1) << 31) - 2) {
    set_error("grid N must be in 1..2^31-2");
    return PIT_EINVAL;
  }
  for (int64_t n = 0; n <= N; ++n) {
    if (!std::isfinite(t[n]) || (n > 0 && !(t[n] > t[n - 1]))) {
      set_error("grid points must be finite and strictly increasing (index " +
                std::to_string(n) + ")");
      return PIT_EINVAL;
    }
  }
  SolveArgs a;
  std::memset(&a, 0, sizeof(a));
  int st = fill_problem(ode, q, y0, a.pb, query == nullptr);
  if (st != PIT_OK) return st;
  a.pb.t0 = t[0];
  a.pb.t1 = t[N];
  a.pb.N = N;
  st = check_opts(opts, a.opts);
  if (st != PIT_OK) return st;
  // small states (d <= 3, layout variants 0 and 1, exact or approximate Jacobian in the dense
  // d x d form) run on the lane-group kernels with per-point preconditioning; everything else,
  // and variant 3, on the large-state kernels
  SolveFn fn = nullptr;
  if (a.pb.d <= 3 && (a.opts.variant == 0 || a.opts.variant == 1))
    fn = find_solver(a.opts.dtype, a.pb.d, q, a.opts.variant);
  if (!fn) fn = find_dense_solver(a.opts.dtype);
  if (!fn) {
    set_error("large-state kernels not compiled for this dtype");
    return PIT_EUNSUPPORTED;
  }
  a.grid = t;
  a.init_traj = init_traj;
  a.mean = mean;
  a.sqrtcov = sqrtcov;
  a.info = info;
  a.workspace = workspace;
  a.ws_bytes = ws_bytes;
  a.stream = static_cast<cudaStream_t>(stream);
  if (query) return fn(a, query, false);
  if (!mean || (a.opts.want_cov && !sqrtcov) || !workspace) {
    set_error("null output or workspace buffer");
    return PIT_EINVAL;
  }
  return fn(a, nullptr, false);
}

int32_t pit_solve_grid_workspace_size(const pit_ode* ode, const double* t, int64_t N, int32_t q,
                                      const pit_opts* opts, size_t* bytes) {
  g_err.clear();
  if (!bytes) return PIT_EINVAL;
  return solve_grid_common(ode, t, N, q, nullptr, opts, nullptr, nullptr, nullptr, nullptr,
                           nullptr, 0, nullptr, bytes);
}

int32_t pit_solve_grid(const pit_ode* ode, const double* t, int64_t N, int32_t q,
                       const double* y0, const pit_opts* opts, const void* init_traj,
                       void* mean, void* sqrtcov, pit_solve_info* info, void* workspace,
                       size_t ws_bytes, void* stream) {
  g_err.clear();
  return solve_grid_common(ode, t, N, q, y0, opts, init_traj, mean, sqrtcov, info, workspace,
                           ws_bytes, stream, nullptr);
}

int32_t pit_eks_workspace_size(const pit_ode* ode, const pit_grid* grid, int32_t q,
                               const pit_opts* opts, size_t* bytes) {
  g_err.clear();
  if (!bytes) return PIT_EINVAL;
  return solve_common(ode, grid, q, nullptr, opts, nullptr, nullptr, nullptr, nullptr, nullptr,
                      0, nullptr, bytes, true);
}

int32_t pit_eks_sequential(const pit_ode* ode, const pit_grid* grid, int32_t q,
                           const double* y0, const pit_opts* opts, void* mean, void* sqrtcov,
                           pit_solve_info* info, void* workspace, size_t ws_bytes,
                           void* stream) {
  g_err.clear();
  return solve_common(ode, grid, q, y0, opts, nullptr, mean, sqrtcov, info, workspace, ws_bytes,
                      stream, nullptr, true);
}

}  // extern "C"
