// Host side of the segmented (batched) solves: engine registry, the active-set iteration of
// pit_solve_batched (Algorithm 2 per instance, all instances in the same launches), and its C ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pit_internal.h"

namespace pit {

namespace {
struct SegRegistry {
  std::mutex mu;
  std::map<int, SegFactory> f;  // key dtype*10000 + d*100 + q
};
SegRegistry& seg_registry() {
  static SegRegistry r;
  return r;
}
}  // namespace

SegRegistrar::SegRegistrar(int dtype, int d, int q, SegFactory fn) {
  SegRegistry& r = seg_registry();
  std::lock_guard<std::mutex> lk(r.mu);
  r.f[dtype * 10000 + d * 100 + q] = fn;
}

SegFactory find_seg_engine(int dtype, int d, int q) {
  SegRegistry& r = seg_registry();
  std::lock_guard<std::mutex> lk(r.mu);
  auto it = r.f.find(dtype * 10000 + d * 100 + q);
  return it == r.f.end() ? nullptr : it->second;
}

// An instance whose change per iteration exceeds this is treated as diverged (before FP32 cubes
// of its trajectory can overflow).
constexpr double kDivergedDelta = 1e12;

namespace {

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchState {
  int cur = 0;
  int iters = 0;
  bool active = true;
  bool converged = false;
  bool failed = false;
  double last_delta = 0.0;
  double sigma2 = 1.0;
  double objective = 0.0;   // V of the last iterate (Eq. objective-value), when evaluated
};

int batched(int32_t B, const pit_ode* odes, const pit_grid* grids, int32_t q, const double* y0,
            const pit_opts* opts_in, void* mean, void* sqrtcov, pit_batch_info* info,
            void* workspace, size_t ws_bytes, cudaStream_t s, size_t* query) {
  if (B < 1 || !odes || !grids) {
    set_error("batched solve needs B >= 1 and non-NULL odes, grids");
    return PIT_EINVAL;
  }
  pit_opts o;
  int st = check_opts(opts_in, o);
  if (st != PIT_OK) return st;
  if (o.variant != 0) {
    set_error("batched solves support variant 0 only");
    return PIT_EUNSUPPORTED;
  }
  const bool need_y0 = (query == nullptr);
  if (need_y0 && !y0) {
    set_error("y0 is NULL");
    return PIT_EINVAL;
  }
  std::vector<Problem> pbs(B);
  for (int i = 0; i < B; ++i) {
    st = fill_problem(&odes[i], q, need_y0 ? y0 + static_cast<size_t>(i) * odes[0].d : nullptr,
                      pbs[i], need_y0);
    if (st == PIT_OK) st = fill_grid(&grids[i], pbs[i]);
    if (st != PIT_OK) {
      set_error("instance " + std::to_string(i) + ": " + std::string(pit_last_error()));
      return st;
    }
    if (pbs[i].kind != pbs[0].kind || pbs[i].d != pbs[0].d) {
      set_error("all instances of a batched solve must share the ODE kind and d");
      return PIT_EINVAL;
    }
  }
  SegFactory fac = find_seg_engine(o.dtype, pbs[0].d, q);
  if (!fac) {
    set_error("no compiled segmented kernels for this (dtype, d, q); compiled: d in 1..3, q in "
              "1..3 (d=3: q <= 2)");
    return PIT_EUNSUPPORTED;
  }
  std::unique_ptr<SegEngine> e(fac());
  const int D = e->state_dim();
  const size_t esz = (o.dtype == PIT_F32) ? sizeof(float) : sizeof(double);
  int64_t M = 0;
  std::vector<int64_t> row(B);
  for (int i = 0; i < B; ++i) {
    row[i] = M;
    M += pbs[i].N + 1;
  }
  const bool want_cov = o.want_cov != 0;
  const size_t eng = round256(e->workspace_bytes(M, B, want_cov, o.chain_len));
  size_t total = eng;
  for (int i = 0; i < B; ++i) total += 2 * round256(e->traj_bytes(pbs[i].N));
  if (query) {
    *query = total;
    return PIT_OK;
  }
  if (!mean || (want_cov && !sqrtcov) || !workspace) {
    set_error("null output or workspace buffer");
    return PIT_EINVAL;
  }
  if (ws_bytes < total) {
    set_error("workspace too small: need " + std::to_string(total) + " bytes, got " +
              std::to_string(ws_bytes));
    return PIT_ENOMEM;
  }
  st = e->bind(workspace, eng, M, B, want_cov, o.chain_len);
  if (st != PIT_OK) return st;
  e->set_linearization(o.linearization);
  char* lp = static_cast<char*>(workspace) + eng;
  for (int i = 0; i < B; ++i) {
    const size_t tb = round256(e->traj_bytes(pbs[i].N));
    void* l0 = lp;
    void* l1 = lp + tb;
    lp += 2 * tb;
    char* mo = static_cast<char*>(mean) + static_cast<size_t>(row[i]) * D * esz;
    char* co = want_cov ? static_cast<char*>(sqrtcov) + static_cast<size_t>(row[i]) * D * D * esz
                        : nullptr;
    st = e->set_instance(i, pbs[i], l0, l1, mo, co, s);
    if (st != PIT_OK) return st;
  }
  std::vector<BatchState> bs(B);
  std::vector<SegSlot> slots;
  slots.reserve(B);
  for (int i = 0; i < B; ++i) slots.push_back(SegSlot{i, 0, row[i]});
  st = e->init_traj(slots.data(), B, s);
  if (st != PIT_OK) return st;

  const int fixed = o.fixed_iters;
  const int limit = fixed > 0 ? fixed : o.max_iter;
  std::vector<SegResult> res(B);
  // objective value V (Eq. objective-value) per instance: evaluated when requested or used by
  // the second stopping rule of Section 3.2.2 (host-driven loop only)
  const bool obj_rule = o.atol_objective > 0 || o.rtol_objective > 0;
  const bool want_obj = obj_rule || o.objective != 0;
  std::vector<double> vals(B);
  if (want_obj) {
    st = e->objective(slots.data(), B, vals.data(), s);
    if (st != PIT_OK) return st;
    for (int i = 0; i < B; ++i) bs[i].objective = vals[i];
  }
  // all means iterations in one cooperative launch (stopping rules and compaction on the
  // device) where the layout fits one resident wave; otherwise the host-driven loop below
  bool on_device = false;
  if (o.scan == 0 && !want_obj) {
    std::vector<SegIterState> ds(B);
    st = e->run_iterations(B, o, kDivergedDelta, ds.data(), s);
    if (st == PIT_OK) {
      on_device = true;
      for (int i = 0; i < B; ++i) {
        BatchState& b = bs[i];
        b.cur = ds[i].cur;
        b.iters = ds[i].iters;
        b.active = false;
        b.converged = ds[i].converged != 0;
        b.failed = ds[i].failed != 0;
        b.last_delta = ds[i].last_delta;
        b.sigma2 = ds[i].sigma2;
      }
    } else if (st != PIT_EUNSUPPORTED) {
      return st;
    }
  }
  for (int k = 1; k <= limit && !on_device; ++k) {
    slots.clear();
    int64_t off = 0;
    for (int i = 0; i < B; ++i) {
      if (!bs[i].active) continue;
      slots.push_back(SegSlot{i, bs[i].cur, off});
      off += pbs[i].N + 1;
    }
    if (slots.empty()) break;
    const int n = static_cast<int>(slots.size());
    st = e->pass(slots.data(), n, false, o.calibrate, res.data(), s);
    if (st != PIT_OK) return st;
    if (want_obj) {   // V of the new iterates lin[1 - cur]
      std::vector<SegSlot> nxt(slots);
      for (SegSlot& x : nxt) x.cur ^= 1;
      st = e->objective(nxt.data(), n, vals.data(), s);
      if (st != PIT_OK) return st;
    }
    for (int j = 0; j < n; ++j) {
      const int i = slots[j].id;
      BatchState& b = bs[i];
      const SegResult& r = res[j];
      bool obj_stop = false;
      if (want_obj) {
        obj_stop = obj_rule && std::fabs(vals[j] - b.objective) <=
                                   o.atol_objective + o.rtol_objective * std::fabs(vals[j]);
        b.objective = vals[j];
      }
      b.iters = k;
      b.last_delta = r.delta_max;
      b.sigma2 = o.calibrate ? r.sigma2_sum / (static_cast<double>(pbs[i].N) * pbs[i].d) : 1.0;
      if ((r.flags & 1u) || !(r.delta_max <= kDivergedDelta)) {
        b.failed = true;
        b.active = false;
      } else if (fixed > 0) {
        if (k == limit) {
          b.active = false;
          b.converged = true;
        } else {
          b.cur ^= 1;
        }
      } else if (r.delta_max <= o.atol_delta + o.rtol_delta * r.y_max || obj_stop) {
        b.active = false;
        b.converged = true;
      } else if (k == limit) {
        b.active = false;
      } else {
        b.cur ^= 1;
      }
    }
  }
  // outputs: covariance pass (means = lin + delta, the last iterate) or export of the last means
  slots.clear();
  std::vector<SegSlot> failed;
  int64_t off = 0;
  for (int i = 0; i < B; ++i) {
    if (bs[i].failed) {
      // export the last finite iterate lin[cur] (export reads lin[1 - slot.cur])
      failed.push_back(SegSlot{i, bs[i].cur ^ 1, 0});
      continue;
    }
    slots.push_back(SegSlot{i, bs[i].cur, off});
    off += pbs[i].N + 1;
  }
  if (!slots.empty()) {
    if (want_cov) {
      st = e->pass(slots.data(), static_cast<int>(slots.size()), true, o.calibrate, res.data(), s);
    } else {
      st = e->export_means(slots.data(), static_cast<int>(slots.size()), s);
    }
    if (st != PIT_OK) return st;
  }
  if (!failed.empty()) {
    st = e->export_means(failed.data(), static_cast<int>(failed.size()), s);
    if (st != PIT_OK) return st;
  }
  PIT_CUDA_TRY(cudaStreamSynchronize(s));
  bool anyfail = false, anync = false;
  for (int i = 0; i < B; ++i) {
    const BatchState& b = bs[i];
    anyfail = anyfail || b.failed;
    anync = anync || (!b.failed && !b.converged);
    if (info) {
      info[i].iterations = b.iters;
      info[i].converged = b.converged ? 1 : 0;
      info[i].status = b.failed ? PIT_ENONFINITE : (b.converged ? PIT_OK : PIT_ENOCONV);
      info[i].pad = 0;
      info[i].last_delta = b.last_delta;
      info[i].sigma2 = b.sigma2;
      info[i].objective = want_obj ? b.objective : 0.0;
    }
  }
  if (anyfail) {
    set_error("at least one instance diverged (see its pit_batch_info.status)");
    return PIT_ENONFINITE;
  }
  return anync ? PIT_ENOCONV : PIT_OK;
}

}  // namespace

// Approximate Jacobians make the linearised model of a d-dimensional problem block diagonal:
// the prior is I_d (x) IWP(q), H_n = E1 - F E0 with F diagonal (or zero) acts on each
// component's block alone, and Sigma_0 = 0.  The filter and smoother of one iteration are then
// d independent (q+1)-dimensional ones (Section 3.2.1, remark on approximate Jacobians), coupled
// only through the residuals f(E0 lin) of the common trajectory.  They run as d segments of one
// scan on the d = 1 segmented engine, iterated together under the global stopping rule.
int solve_decoupled(const SolveArgs& a, size_t* wsq) {
  const Problem& pb = a.pb;
  const pit_opts& o = a.opts;
  const int d = pb.d, q = pb.q, Q1 = q + 1, Dfull = d * Q1;
  if (o.linearization == PIT_LIN_EK1) {
    set_error("the decoupled solve needs an approximate Jacobian (DiagonalEK1 or EK0)");
    return PIT_EINVAL;
  }
  if (a.init_traj || o.init_coarse > 0 || o.objective || o.atol_objective > 0 ||
      o.rtol_objective > 0) {
    set_error("decoupled solves support neither warm starts, coarse initialisation nor the "
              "objective value");
    return PIT_EINVAL;
  }
  SegFactory fac = find_seg_engine(o.dtype, 1, q);
  if (!fac) {
    set_error("no compiled kernels for the decoupled components (q in 1..3)");
    return PIT_EUNSUPPORTED;
  }
  std::unique_ptr<SegEngine> e(fac());
  const int64_t M = static_cast<int64_t>(d) * (pb.N + 1);
  const bool want_cov = o.want_cov != 0;
  const size_t eng = round256(e->workspace_bytes(M, d, want_cov, o.chain_len));
  const size_t tb = round256(e->traj_bytes(pb.N));
  const size_t total = eng + static_cast<size_t>(d) * 2 * tb;
  if (wsq) {
    *wsq = total;
    return PIT_OK;
  }
  if (a.ws_bytes < total) {
    set_error("workspace too small: need " + std::to_string(total) + " bytes, got " +
              std::to_string(a.ws_bytes));
    return PIT_ENOMEM;
  }
  cudaStream_t s = a.stream;
  const int64_t launches0 = launches_total();
  int st = e->bind(a.workspace, eng, M, d, want_cov, o.chain_len);
  if (st != PIT_OK) return st;
  e->set_linearization(o.linearization);
  e->set_decoupled(true);
  std::vector<double> mu0(Dfull);
  st = taylor_init(pb, mu0.data());
  if (st != PIT_OK) {
    set_error("exact initial state: unsupported problem size");
    return st;
  }
  const size_t esz = (o.dtype == PIT_F32) ? sizeof(float) : sizeof(double);
  if (want_cov)
    PIT_CUDA_TRY(cudaMemsetAsync(a.sqrtcov, 0,
                                 static_cast<size_t>(pb.N + 1) * Dfull * Dfull * esz, s));
  char* lp = static_cast<char*>(a.workspace) + eng;
  std::vector<SegSlot> slots(d);
  for (int k = 0; k < d; ++k) {
    st = e->set_component(k, pb, k, mu0.data() + static_cast<size_t>(k) * Q1, lp, lp + tb,
                          a.mean, want_cov ? a.sqrtcov : nullptr, s);
    if (st != PIT_OK) return st;
    lp += 2 * tb;
    slots[k] = SegSlot{k, 0, static_cast<int64_t>(k) * (pb.N + 1)};
  }
  st = e->init_traj(slots.data(), d, s);
  if (st != PIT_OK) return st;
  pit_solve_info info;
  std::memset(&info, 0, sizeof(info));
  std::vector<SegResult> res(d);
  const int fixed = o.fixed_iters;
  const int limit = fixed > 0 ? fixed : std::max(1, o.max_iter);
  bool converged = fixed > 0;
  int k = 0;
  double s2sum = 0.0;
  while (k < limit) {
    st = e->pass(slots.data(), d, false, o.calibrate, res.data(), s);
    if (st != PIT_OK) return st;
    ++k;
    double dmax = 0.0, ymax = 0.0;
    unsigned flags = 0;
    s2sum = 0.0;
    for (int j = 0; j < d; ++j) {
      dmax = std::max(dmax, res[j].delta_max);
      ymax = std::max(ymax, res[j].y_max);
      flags |= res[j].flags;
      s2sum += res[j].sigma2_sum;
    }
    if ((flags & 1u) || !(dmax == dmax)) {
      set_error("non-finite value in the smoothing means at iteration " + std::to_string(k));
      return PIT_ENONFINITE;
    }
    info.last_delta = dmax;
    if (k <= 64) info.deltas[k - 1] = dmax;
    bool stop = (k == limit);
    if (fixed <= 0 && dmax <= o.atol_delta + o.rtol_delta * ymax) {
      converged = true;
      stop = true;
    }
    if (stop) break;
    for (auto& sl : slots) sl.cur ^= 1;
  }
  if (want_cov) {
    st = e->pass(slots.data(), d, true, o.calibrate, res.data(), s);
  } else {
    st = e->export_means(slots.data(), d, s);
  }
  if (st != PIT_OK) return st;
  PIT_CUDA_TRY(cudaStreamSynchronize(s));
  info.iterations = k;
  info.converged = converged ? 1 : 0;
  info.sigma2 = o.calibrate ? s2sum / (static_cast<double>(pb.N) * d) : 1.0;
  info.kernel_launches = launches_total() - launches0;
  if (a.info) *a.info = info;
  return converged ? PIT_OK : PIT_ENOCONV;
}

}  // namespace pit

using namespace pit;

extern "C" {

int32_t pit_solve_batched_workspace_size(int32_t B, const pit_ode* odes, const pit_grid* grids,
                                         int32_t q, const pit_opts* opts, size_t* bytes) {
  set_error("");
  if (!bytes) {
    set_error("bytes is NULL");
    return PIT_EINVAL;
  }
  *bytes = 0;
  return batched(B, odes, grids, q, nullptr, opts, nullptr, nullptr, nullptr, nullptr, 0,
                 nullptr, bytes);
}

int32_t pit_solve_batched(int32_t B, const pit_ode* odes, const pit_grid* grids, int32_t q,
                          const double* y0, const pit_opts* opts, void* mean, void* sqrtcov,
                          pit_batch_info* info, void* workspace, size_t ws_bytes, void* stream) {
  set_error("");
  return batched(B, odes, grids, q, y0, opts, mean, sqrtcov, info, workspace, ws_bytes,
                 static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
