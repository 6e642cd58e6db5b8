// Host side of the segmented (batched) solves: engine registry, the active-set iteration of
// pit_solve_batched (Algorithm 2 per instance, all instances in the same launches), and its C ABI.
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
  for (int k = 1; k <= limit; ++k) {
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
    for (int j = 0; j < n; ++j) {
      const int i = slots[j].id;
      BatchState& b = bs[i];
      const SegResult& r = res[j];
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
      } else if (r.delta_max <= o.atol_delta + o.rtol_delta * r.y_max) {
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
    }
  }
  if (anyfail) {
    set_error("at least one instance diverged (see its pit_batch_info.status)");
    return PIT_ENONFINITE;
  }
  return anync ? PIT_ENOCONV : PIT_OK;
}

}  // namespace
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
