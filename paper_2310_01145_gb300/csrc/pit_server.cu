// Serving loop with continuous batching (no counterpart in the paper, which solves one problem
// at a time): requests of any ODE family, d, q and length wait in a FIFO queue per (family, d, q)
// class; every step admits queued requests into the class's batch while its point and request
// capacity and the device memory pool allow, runs one IEKS iteration (Algorithm 2's loop body:
// linearise, then the parallel filter and smoother of Algorithm 1) over all requests in flight of
// every class -- classes on their own CUDA streams, so their kernels overlap -- and retires the
// requests whose stopping rule holds.  A request's trajectory stays in device memory between
// iterations; only the per-request change statistics come back to the host each step.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "pit_internal.h"

struct pit_server;  // opaque handle of the C ABI

namespace pit {
namespace {

constexpr double kDiverged = 1e12;  // change per iteration treated as divergence (as batched)

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over one device region (offsets, 256-byte granularity, coalescing).
class Pool {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

struct Request {
  int64_t id = 0;
  uint64_t tag = 0;
  Problem pb{};
  void* mean_out = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int key = 0;
  // in flight
  int slot = -1;
  size_t lin_off = 0, lin_bytes = 0;
  int cur = 0;
  int iters = 0;
  double last_delta = 0, sigma2 = 1;
  double objective = 0;   // V of the current trajectory (objective rule, d <= 3 classes)
  // large-state request (d > 3): its own session and workspace in the pool
  std::unique_ptr<LargeSession> sess;
  // square-root covariances on request: the covariance pass's workspace and scratch means,
  // reserved from the pool at admission
  void* cov_out = nullptr;
  size_t cov_ws = 0, cov_bytes = 0, cov_off = 0;
  bool cov_held = false;
};

struct ClassState {
  int kind = 0, d = 0, q = 0;
  // large: requests run on the large-state kernels, one session each (no segmented engine)
  bool large = false;
  LargeScalars* hres = nullptr;  // page-locked, one slot per request in flight
  std::unique_ptr<SegEngine> eng;
  cudaStream_t stream = nullptr;
  size_t ws_off = 0, ws_bytes = 0;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;  // request ids in flight, in layout order
  std::vector<int> free_slots;
  int64_t active_points = 0;
  bool begun = false;
  std::vector<SegSlot> slots;
  std::vector<SegResult> res;
};

}  // namespace
}  // namespace pit

struct pit_server {
  pit_server_config cfg{};
  void* pool = nullptr;
  pit::Pool alloc;
  std::map<int, pit::ClassState> classes;
  std::unordered_map<int64_t, pit::Request> reqs;
  std::deque<pit_server_result> done;
  int64_t next_id = 1;
  std::mutex mu;
};

namespace pit {
namespace {

int class_key(int kind, int d, int q) { return kind * 10000 + d * 100 + q; }

int ensure_class(pit_server* sv, const Problem& pb, ClassState** out) {
  const int key = class_key(pb.kind, pb.d, pb.q);
  auto it = sv->classes.find(key);
  if (it != sv->classes.end()) {
    *out = &it->second;
    return PIT_OK;
  }
  SegFactory fac = find_seg_engine(sv->cfg.dtype, pb.d, pb.q);
  if (!fac && pb.d > 3 && find_large_session(sv->cfg.dtype)) {
    // large-state class: per-request sessions, one stream, page-locked reductions
    ClassState cs;
    cs.kind = pb.kind;
    cs.d = pb.d;
    cs.q = pb.q;
    cs.large = true;
    if (cudaHostAlloc(reinterpret_cast<void**>(&cs.hres),
                      sizeof(LargeScalars) * static_cast<size_t>(sv->cfg.max_requests),
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaHostAlloc of the reduction buffer failed");
      return PIT_ECUDA;
    }
    if (cudaStreamCreateWithFlags(&cs.stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaFreeHost(cs.hres);
      set_error("cudaStreamCreateWithFlags failed");
      return PIT_ECUDA;
    }
    for (int i = sv->cfg.max_requests - 1; i >= 0; --i) cs.free_slots.push_back(i);
    auto res = sv->classes.emplace(key, std::move(cs));
    *out = &res.first->second;
    return PIT_OK;
  }
  if (!fac) {
    set_error("no compiled segmented kernels for this (dtype, d, q)");
    return PIT_EUNSUPPORTED;
  }
  ClassState cs;
  cs.kind = pb.kind;
  cs.d = pb.d;
  cs.q = pb.q;
  cs.eng.reset(fac());
  cs.ws_bytes = round256(cs.eng->workspace_bytes(sv->cfg.max_points, sv->cfg.max_requests, false,
                                                 sv->cfg.chain_len));
  if (!sv->alloc.alloc(cs.ws_bytes, &cs.ws_off)) {
    set_error("device memory budget too small for another request class (needs " +
              std::to_string(cs.ws_bytes) + " bytes)");
    return PIT_ENOMEM;
  }
  int st = cs.eng->bind(static_cast<char*>(sv->pool) + cs.ws_off, cs.ws_bytes, sv->cfg.max_points,
                        sv->cfg.max_requests, false, sv->cfg.chain_len);
  if (st == PIT_OK) st = cs.eng->use_pinned_staging();
  if (st != PIT_OK) {
    sv->alloc.release(cs.ws_off, cs.ws_bytes);
    return st;
  }
  if (cudaStreamCreateWithFlags(&cs.stream, cudaStreamNonBlocking) != cudaSuccess) {
    sv->alloc.release(cs.ws_off, cs.ws_bytes);
    set_error("cudaStreamCreateWithFlags failed");
    return PIT_ECUDA;
  }
  for (int i = sv->cfg.max_requests - 1; i >= 0; --i) cs.free_slots.push_back(i);
  auto res = sv->classes.emplace(key, std::move(cs));
  *out = &res.first->second;
  return PIT_OK;
}

pit_opts session_opts(const pit_server* sv) {
  pit_opts o;
  pit_opts_default(&o);
  o.dtype = sv->cfg.dtype;
  o.calibrate = sv->cfg.calibrate;
  o.chain_len = sv->cfg.chain_len;
  o.want_cov = 0;
  return o;
}

// The covariance pass of a retiring request: the request's problem as the C ABI describes it,
// and options for one IEKS iteration linearised at the delivered means with the covariance
// recursions (host-driven scan trees: no cooperative launch beside the other classes' kernels).
pit_ode ode_of(const Problem& pb) {
  pit_ode o;
  o.kind = pb.kind;
  o.d = pb.d;
  o.params = pb.params;
  o.n_params = pb.n_params;
  return o;
}
pit_grid grid_of(const Problem& pb) {
  pit_grid g;
  g.t0 = pb.t0;
  g.t1 = pb.t1;
  g.N = pb.N;
  return g;
}
pit_opts cov_opts(const pit_server* sv) {
  pit_opts o = session_opts(sv);
  o.fixed_iters = 1;
  o.want_cov = 1;
  o.scan = 1;
  return o;
}
// Workspace of the covariance pass and the bytes reserved for it (+ its scratch means).
int cov_sizes(const pit_server* sv, const Problem& pb, size_t* ws, size_t* total) {
  const pit_ode o = ode_of(pb);
  const pit_grid g = grid_of(pb);
  const pit_opts op = cov_opts(sv);
  size_t w = 0;
  const int st = pit_solve_workspace_size(&o, &g, pb.q, &op, &w);
  if (st != PIT_OK) return st;
  const size_t esz = sv->cfg.dtype == PIT_F64 ? 8 : 4;
  *ws = round256(w);
  *total = *ws + round256(static_cast<size_t>(pb.N + 1) * pb.d * (pb.q + 1) * esz);
  return PIT_OK;
}
// Runs the covariance pass of a retiring request on `s` (synchronises it) and frees its
// reservation.  Returns the pass's status.
int cov_pass(pit_server* sv, Request& r, cudaStream_t s) {
  const pit_ode o = ode_of(r.pb);
  const pit_grid g = grid_of(r.pb);
  const pit_opts op = cov_opts(sv);
  char* base = static_cast<char*>(sv->pool) + r.cov_off;
  const int st = pit_solve(&o, &g, r.pb.q, r.pb.y0, &op, r.mean_out, base + r.cov_ws, r.cov_out,
                           nullptr, base, r.cov_ws, s);
  sv->alloc.release(r.cov_off, r.cov_bytes);
  r.cov_held = false;
  return st;
}
// Reserves the covariance pass's memory at admission (false: the pool cannot hold it now).
bool cov_reserve(pit_server* sv, Request& r) {
  if (!r.cov_out) return true;
  if (!sv->alloc.alloc(r.cov_bytes, &r.cov_off)) return false;
  r.cov_held = true;
  return true;
}

bool obj_rule(const pit_server* sv) {
  return sv->cfg.atol_objective > 0 || sv->cfg.rtol_objective > 0;
}

// Large-state class: admit (FIFO, by slots, points and pool memory), then enqueue one IEKS
// iteration of every request in flight on the class stream.
int begin_large(pit_server* sv, ClassState& cs) {
  const pit_opts o = session_opts(sv);
  while (!cs.queue.empty()) {
    Request& r = sv->reqs[cs.queue.front()];
    const int64_t pts = r.pb.N + 1;
    if (cs.free_slots.empty() || cs.active_points + pts > sv->cfg.max_points) break;
    const size_t bytes = large_session_bytes(sv->cfg.dtype, r.pb, o);
    if (bytes == 0) return PIT_EINVAL;
    size_t off = 0;
    if (!sv->alloc.alloc(bytes, &off)) break;
    if (!cov_reserve(sv, r)) {
      sv->alloc.release(off, bytes);
      break;
    }
    std::unique_ptr<LargeSession> ss(find_large_session(sv->cfg.dtype)());
    const int st = ss->start(r.pb, o, static_cast<char*>(sv->pool) + off, round256(bytes), cs.stream);
    if (st != PIT_OK) {
      sv->alloc.release(off, bytes);
      if (r.cov_held) sv->alloc.release(r.cov_off, r.cov_bytes);
      r.cov_held = false;
      return st;
    }
    r.sess = std::move(ss);
    r.lin_off = off;
    r.lin_bytes = bytes;
    r.slot = cs.free_slots.back();
    cs.free_slots.pop_back();
    r.t_admit = now_s();
    cs.active.push_back(r.id);
    cs.active_points += pts;
    cs.queue.pop_front();
  }
  if (cs.active.empty()) return PIT_OK;
  for (int64_t id : cs.active) {
    Request& r = sv->reqs[id];
    const int st = r.sess->iterate(cs.hres + r.slot, cs.stream);
    if (st != PIT_OK) return st;
  }
  cs.begun = true;
  return PIT_OK;
}

// Admit queued requests of one class (FIFO; the head blocks until it fits) and start its pass.
int begin_class(pit_server* sv, ClassState& cs) {
  if (cs.large) return begin_large(sv, cs);
  std::vector<SegSlot> fresh;
  while (!cs.queue.empty()) {
    Request& r = sv->reqs[cs.queue.front()];
    const int64_t pts = r.pb.N + 1;
    if (cs.free_slots.empty() || cs.active_points + pts > sv->cfg.max_points) break;
    const size_t tb = round256(cs.eng->traj_bytes(r.pb.N));
    size_t off = 0;
    if (!sv->alloc.alloc(2 * tb, &off)) break;
    if (!cov_reserve(sv, r)) {
      sv->alloc.release(off, 2 * tb);
      break;
    }
    r.lin_off = off;
    r.lin_bytes = 2 * tb;
    r.slot = cs.free_slots.back();
    cs.free_slots.pop_back();
    char* base = static_cast<char*>(sv->pool) + off;
    int st = cs.eng->set_instance(r.slot, r.pb, base, base + tb, r.mean_out, nullptr, cs.stream);
    if (st != PIT_OK) return st;
    r.cur = 0;
    r.t_admit = now_s();
    cs.active.push_back(r.id);
    cs.active_points += pts;
    fresh.push_back(SegSlot{r.slot, 0, 0});
    cs.queue.pop_front();
  }
  if (!fresh.empty()) {
    int st = cs.eng->init_traj(fresh.data(), static_cast<int>(fresh.size()), cs.stream);
    if (st != PIT_OK) return st;
    if (obj_rule(sv)) {
      std::vector<double> v(fresh.size());
      st = cs.eng->objective(fresh.data(), static_cast<int>(fresh.size()), v.data(), cs.stream);
      if (st != PIT_OK) return st;
      for (size_t j = 0; j < fresh.size(); ++j)
        for (int64_t id : cs.active)
          if (sv->reqs[id].slot == fresh[j].id) sv->reqs[id].objective = v[j];
    }
  }
  if (cs.active.empty()) return PIT_OK;
  cs.slots.clear();
  int64_t off = 0;
  for (int64_t id : cs.active) {
    const Request& r = sv->reqs[id];
    cs.slots.push_back(SegSlot{r.slot, r.cur, off});
    off += r.pb.N + 1;
  }
  int st = cs.eng->pass_begin(cs.slots.data(), static_cast<int>(cs.slots.size()), false,
                              sv->cfg.calibrate, cs.stream);
  if (st != PIT_OK) return st;
  cs.begun = true;
  return PIT_OK;
}

// Wait for a large-state class's iteration, apply the stopping rules, retire finished requests.
int end_large(pit_server* sv, ClassState& cs) {
  PIT_CUDA_TRY(cudaStreamSynchronize(cs.stream));
  std::vector<int64_t> keep;
  for (int64_t id : cs.active) {
    Request& r = sv->reqs[id];
    const LargeScalars& a = cs.hres[r.slot];
    r.iters += 1;
    r.last_delta = a.delta_max;
    r.sigma2 = sv->cfg.calibrate ? a.sigma2_sum / (static_cast<double>(r.pb.N) * r.pb.d) : 1.0;
    int status = -1;
    if ((a.flags & 1u) || !(a.delta_max <= kDiverged)) {
      status = PIT_ENONFINITE;
    } else if (a.delta_max <= sv->cfg.atol_delta + sv->cfg.rtol_delta * a.y_max) {
      status = PIT_OK;
    } else if (r.iters >= sv->cfg.max_iter) {
      status = PIT_ENOCONV;
    }
    if (status < 0) {
      r.sess->advance();
      keep.push_back(id);
      continue;
    }
    const int st = r.sess->export_means(r.mean_out, status == PIT_ENONFINITE, cs.stream);
    if (st != PIT_OK) return st;
    PIT_CUDA_TRY(cudaStreamSynchronize(cs.stream));
    if (r.cov_held) {
      if (status != PIT_ENONFINITE) {
        const int cst = cov_pass(sv, r, cs.stream);
        if (cst != PIT_OK) status = cst;
      } else {
        sv->alloc.release(r.cov_off, r.cov_bytes);
        r.cov_held = false;
      }
    }
    pit_server_result out;
    std::memset(&out, 0, sizeof(out));
    out.request_id = r.id;
    out.tag = r.tag;
    out.status = status;
    out.iterations = r.iters;
    out.last_delta = r.last_delta;
    out.sigma2 = r.sigma2;
    out.t_submit = r.t_submit;
    out.t_admit = r.t_admit;
    out.t_done = now_s();
    sv->done.push_back(out);
    sv->alloc.release(r.lin_off, r.lin_bytes);
    cs.free_slots.push_back(r.slot);
    cs.active_points -= r.pb.N + 1;
    sv->reqs.erase(id);
  }
  cs.active.swap(keep);
  return PIT_OK;
}

// Wait for a class's pass, apply each request's stopping rule, retire the finished ones.
int end_class(pit_server* sv, ClassState& cs) {
  if (!cs.begun) return PIT_OK;
  cs.begun = false;
  if (cs.large) return end_large(sv, cs);
  cs.res.resize(cs.slots.size());
  int st = cs.eng->pass_end(cs.res.data(), cs.stream);
  if (st != PIT_OK) return st;
  std::vector<double> vnew;
  if (obj_rule(sv)) {   // V of the new iterates lin[1 - cur] (Eq. objective-value)
    std::vector<SegSlot> nxt(cs.slots);
    for (SegSlot& x : nxt) x.cur ^= 1;
    vnew.resize(nxt.size());
    st = cs.eng->objective(nxt.data(), static_cast<int>(nxt.size()), vnew.data(), cs.stream);
    if (st != PIT_OK) return st;
  }
  std::vector<SegSlot> fin;
  std::vector<int64_t> fin_ids, keep;
  std::vector<int> fin_status;
  for (size_t j = 0; j < cs.active.size(); ++j) {
    Request& r = sv->reqs[cs.active[j]];
    const SegResult& a = cs.res[j];
    r.iters += 1;
    r.last_delta = a.delta_max;
    r.sigma2 = sv->cfg.calibrate ? a.sigma2_sum / (static_cast<double>(r.pb.N) * r.pb.d) : 1.0;
    bool obj_stop = false;
    if (!vnew.empty()) {
      obj_stop = std::fabs(vnew[j] - r.objective) <=
                 sv->cfg.atol_objective + sv->cfg.rtol_objective * std::fabs(vnew[j]);
      r.objective = vnew[j];
    }
    int status = -1;
    if ((a.flags & 1u) || !(a.delta_max <= kDiverged)) {
      status = PIT_ENONFINITE;
    } else if (a.delta_max <= sv->cfg.atol_delta + sv->cfg.rtol_delta * a.y_max || obj_stop) {
      status = PIT_OK;
    } else if (r.iters >= sv->cfg.max_iter) {
      status = PIT_ENOCONV;
    }
    if (status < 0) {
      r.cur ^= 1;
      keep.push_back(r.id);
      continue;
    }
    // finished: the last means are in lin[1 - cur] (lin[cur] when the last pass diverged)
    fin.push_back(SegSlot{r.slot, status == PIT_ENONFINITE ? (r.cur ^ 1) : r.cur, 0});
    fin_ids.push_back(r.id);
    fin_status.push_back(status);
  }
  if (!fin.empty()) {
    st = cs.eng->export_means(fin.data(), static_cast<int>(fin.size()), cs.stream);
    if (st != PIT_OK) return st;
    PIT_CUDA_TRY(cudaStreamSynchronize(cs.stream));
    for (size_t k = 0; k < fin_ids.size(); ++k) {
      Request& r = sv->reqs[fin_ids[k]];
      if (!r.cov_held) continue;
      if (fin_status[k] != PIT_ENONFINITE) {
        const int cst = cov_pass(sv, r, cs.stream);
        if (cst != PIT_OK) fin_status[k] = cst;
      } else {
        sv->alloc.release(r.cov_off, r.cov_bytes);
        r.cov_held = false;
      }
    }
    const double t = now_s();
    for (size_t k = 0; k < fin_ids.size(); ++k) {
      Request& r = sv->reqs[fin_ids[k]];
      pit_server_result out;
      std::memset(&out, 0, sizeof(out));
      out.request_id = r.id;
      out.tag = r.tag;
      out.status = fin_status[k];
      out.iterations = r.iters;
      out.last_delta = r.last_delta;
      out.sigma2 = r.sigma2;
      out.t_submit = r.t_submit;
      out.t_admit = r.t_admit;
      out.t_done = t;
      out.objective = obj_rule(sv) ? r.objective : 0.0;
      sv->done.push_back(out);
      sv->alloc.release(r.lin_off, r.lin_bytes);
      cs.free_slots.push_back(r.slot);
      cs.active_points -= r.pb.N + 1;
      sv->reqs.erase(fin_ids[k]);
    }
  }
  cs.active.swap(keep);
  return PIT_OK;
}

}  // namespace
}  // namespace pit

namespace pit {
namespace {
int submit_common(pit_server* sv, const pit_ode* ode, const pit_grid* grid, int32_t q,
                  const double* y0, void* mean_out, void* cov_out, uint64_t tag,
                  int64_t* request_id) {
  std::lock_guard<std::mutex> lk(sv->mu);
  Request r;
  int st = fill_problem(ode, q, y0, r.pb, true);
  if (st == PIT_OK) st = fill_grid(grid, r.pb);
  if (st != PIT_OK) return st;
  if (r.pb.N + 1 > sv->cfg.max_points) {
    set_error("request longer than the server's per-class point capacity");
    return PIT_EINVAL;
  }
  ClassState* cs = nullptr;
  st = ensure_class(sv, r.pb, &cs);
  if (st != PIT_OK) return st;
  if (cs->large) {
    // a request whose workspace can never fit the budget would block its queue for good
    const size_t bytes = large_session_bytes(sv->cfg.dtype, r.pb, session_opts(sv));
    if (bytes == 0) return PIT_EINVAL;
    if (bytes > sv->cfg.hbm_budget_bytes) {
      set_error("request needs " + std::to_string(bytes) + " bytes of device memory, more than the "
                "server's budget of " + std::to_string(sv->cfg.hbm_budget_bytes));
      return PIT_ENOMEM;
    }
  }
  if (cov_out) {
    st = cov_sizes(sv, r.pb, &r.cov_ws, &r.cov_bytes);
    if (st != PIT_OK) return st;
    if (r.cov_bytes > sv->cfg.hbm_budget_bytes) {
      set_error("the request's covariance pass needs " + std::to_string(r.cov_bytes) +
                " bytes of device memory, more than the server's budget");
      return PIT_ENOMEM;
    }
    r.cov_out = cov_out;
  }
  r.id = sv->next_id++;
  r.tag = tag;
  r.mean_out = mean_out;
  r.key = class_key(r.pb.kind, r.pb.d, r.pb.q);
  r.t_submit = now_s();
  const int64_t rid = r.id;
  cs->queue.push_back(rid);
  sv->reqs.emplace(rid, std::move(r));
  if (request_id) *request_id = rid;
  return PIT_OK;
}
}  // namespace
}  // namespace pit

using namespace pit;

extern "C" {

void pit_server_config_default(pit_server_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->dtype = PIT_F32;
  c->max_iter = 20;
  c->atol_delta = 1e-10;
  c->rtol_delta = 1e-6;
  c->calibrate = 1;
  c->chain_len = 0;
  c->max_points = int64_t(1) << 22;
  c->max_requests = 1024;
  c->hbm_budget_bytes = size_t(8) << 30;
}

double pit_server_clock(void) { return now_s(); }

int32_t pit_server_create(const pit_server_config* cfg, pit_server** out) {
  set_error("");
  if (!out) {
    set_error("out is NULL");
    return PIT_EINVAL;
  }
  *out = nullptr;
  pit_server_config c;
  pit_server_config_default(&c);
  if (cfg) c = *cfg;
  if ((c.dtype != PIT_F32 && c.dtype != PIT_F64) || c.max_iter < 1 || !(c.atol_delta >= 0) ||
      !(c.rtol_delta >= 0) || c.chain_len < 0 || c.max_points < 2 || c.max_requests < 1 ||
      c.hbm_budget_bytes < (size_t(1) << 20) || !(c.atol_objective >= 0) ||
      !(c.rtol_objective >= 0)) {
    set_error("invalid pit_server_config");
    return PIT_EINVAL;
  }
  std::unique_ptr<pit_server> sv(new pit_server());
  sv->cfg = c;
  if (cudaMalloc(&sv->pool, c.hbm_budget_bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of the server's device memory budget failed");
    return PIT_ENOMEM;
  }
  sv->alloc.reset(c.hbm_budget_bytes);
  *out = sv.release();
  return PIT_OK;
}


int32_t pit_server_submit(pit_server* sv, const pit_ode* ode, const pit_grid* grid, int32_t q,
                          const double* y0, void* mean_out, uint64_t tag, int64_t* request_id) {
  set_error("");
  if (!sv || !mean_out) {
    set_error("server or mean_out is NULL");
    return PIT_EINVAL;
  }
  return submit_common(sv, ode, grid, q, y0, mean_out, nullptr, tag, request_id);
}

int32_t pit_server_submit_cov(pit_server* sv, const pit_ode* ode, const pit_grid* grid, int32_t q,
                              const double* y0, void* mean_out, void* sqrtcov_out, uint64_t tag,
                              int64_t* request_id) {
  set_error("");
  if (!sv || !mean_out || !sqrtcov_out) {
    set_error("server, mean_out or sqrtcov_out is NULL");
    return PIT_EINVAL;
  }
  return submit_common(sv, ode, grid, q, y0, mean_out, sqrtcov_out, tag, request_id);
}

int32_t pit_server_step(pit_server* sv, int32_t* in_flight, int32_t* queued) {
  set_error("");
  if (!sv) {
    set_error("server is NULL");
    return PIT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  int first_err = PIT_OK;
  for (auto& kv : sv->classes) {
    const int st = begin_class(sv, kv.second);
    if (st != PIT_OK && first_err == PIT_OK) first_err = st;
  }
  for (auto& kv : sv->classes) {
    const int st = end_class(sv, kv.second);
    if (st != PIT_OK && first_err == PIT_OK) first_err = st;
  }
  int fl = 0, qu = 0;
  for (auto& kv : sv->classes) {
    fl += static_cast<int>(kv.second.active.size());
    qu += static_cast<int>(kv.second.queue.size());
  }
  if (in_flight) *in_flight = fl;
  if (queued) *queued = qu;
  return first_err;
}

int32_t pit_server_poll(pit_server* sv, pit_server_result* out, int32_t max, int32_t* n) {
  set_error("");
  if (!sv || !n || (max > 0 && !out)) {
    set_error("invalid poll arguments");
    return PIT_EINVAL;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  int k = 0;
  while (k < max && !sv->done.empty()) {
    out[k++] = sv->done.front();
    sv->done.pop_front();
  }
  *n = k;
  return PIT_OK;
}

int32_t pit_server_stats(pit_server* sv, size_t* pool_used, int32_t* classes) {
  if (!sv) return PIT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (pool_used) *pool_used = sv->alloc.used();
  if (classes) *classes = static_cast<int32_t>(sv->classes.size());
  return PIT_OK;
}

void pit_server_destroy(pit_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto& kv : sv->classes) {
      if (kv.second.stream) {
        cudaStreamSynchronize(kv.second.stream);
        cudaStreamDestroy(kv.second.stream);
      }
      if (kv.second.hres) cudaFreeHost(kv.second.hres);
      kv.second.eng.reset();
    }
    if (sv->pool) cudaFree(sv->pool);
  }
  delete sv;
}

}  // extern "C"
