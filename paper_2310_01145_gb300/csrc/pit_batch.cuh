// Segmented (batched) IEKS: many instances of one ODE family, of any lengths, solved by the same
// scans over one global time axis (Section 3.1's operators, unchanged).  Instance i occupies
// global points off_i .. off_i + N_i; its n = 0 point enters the filter scan as a reset element
// (A = 0, b = delta_0, C = 0, eta = 0, J = 0) and its n = N point leaves the smoothing scan as an
// element with E = 0, so every prefix value (filtering means and factors) and every smoothing
// value of an instance depends on that instance's data only.  Included by the pit_batch_*.cu
// instantiation files.
#pragma once

#include <cstddef>
#include <vector>

#include "pit_solve_impl.cuh"

namespace pit {

static_assert(sizeof(InstAcc) == sizeof(SegResult), "InstAcc and SegResult must match");
static_assert(offsetof(InstAcc, delta_max) == offsetof(SegResult, delta_max), "layout");
static_assert(offsetof(InstAcc, flags) == offsetof(SegResult, flags), "layout");

// Layout of one pass: per slot, the instance's offset and current trajectory; per global point,
// the instance code (id, or ~id at n = 0).
template <typename T>
__global__ void k_seg_layout(const SegSlot* __restrict__ slots, InstDesc<T>* __restrict__ desc,
                             int* __restrict__ inst_of) {
  const SegSlot sl = slots[blockIdx.x];
  InstDesc<T>& d = desc[sl.id];
  if (threadIdx.x == 0) {
    d.off = sl.off;
    d.cur = sl.cur;
  }
  const int64_t npts = d.N + 1;
  for (int64_t n = threadIdx.x; n < npts; n += blockDim.x)
    inst_of[sl.off + n] = (n == 0) ? ~sl.id : sl.id;
}

// lin[cur] <- mu0 (preconditioned) at every point, for every slot (blockIdx.y).
template <class C>
__global__ void k_seg_init(const SegSlot* __restrict__ slots,
                           const InstDesc<typename C::Tp>* __restrict__ desc) {
  using V = typename TrajType<typename C::Tp>::type;
  const SegSlot sl = slots[blockIdx.y];
  const InstDesc<typename C::Tp>& d = desc[sl.id];
  V* lin = static_cast<V*>(d.lin[sl.cur]);
  const int64_t total = (d.N + 1) * C::D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    lin[i] = v_from_double<V>(d.mu0d[i % C::D]);
}

// mean <- T lin[1 - cur] (original coordinates), for every slot (blockIdx.y).
template <class C>
__global__ void k_seg_export(const SegSlot* __restrict__ slots,
                             const InstDesc<typename C::Tp>* __restrict__ desc) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  const SegSlot sl = slots[blockIdx.y];
  const InstDesc<T>& d = desc[sl.id];
  const V* lin = static_cast<const V*>(d.lin[1 - sl.cur]);
  const int64_t total = (d.N + 1) * C::D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(i % C::D);
    d.mean[(i / C::D) * d.mean_ld + r] = d.Tdiag[r % C::Q1] * v_to_T<T>(lin[i]);
  }
}

// Objective value (Eq. objective-value) of trajectory lin[cur] of every slot (blockIdx.y):
// out[slot] += 1/2 sum_{n=1..N} || sqrt(Qbar)^-1 (xbar_n - Phibar xbar_{n-1}) ||^2 per dimension
// block, as k_objective for a single solve (Phibar, Qbar are step-free, shared by the instances).
template <class C>
__global__ void __launch_bounds__(256)
k_seg_objective(const SegSlot* __restrict__ slots, const InstDesc<typename C::Tp>* __restrict__ desc,
                const IeksParams<typename C::Tp> p, double* __restrict__ out) {
  using V = typename TrajType<typename C::Tp>::type;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  const SegSlot sl = slots[blockIdx.y];
  const InstDesc<typename C::Tp>& d = desc[sl.id];
  const V* lin = static_cast<const V*>(d.lin[sl.cur]);
  double acc = 0.0;
  for (int64_t n = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= d.N;
       n += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < DD; ++k) {
      double w[Q1];
#pragma unroll
      for (int i = 0; i < Q1; ++i) {
        V a = lin[n * D + k * Q1 + i] - lin[(n - 1) * D + k * Q1 + i];
#pragma unroll
        for (int j = i + 1; j < Q1; ++j)
          a = a - lin[(n - 1) * D + k * Q1 + j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
        w[i] = v_to_double(a);
      }
#pragma unroll
      for (int i = 0; i < Q1; ++i) {
        double z = w[i];
        // forward substitution with the lower-triangular sqrt(Qbar); z_i kept in w[i]
#pragma unroll
        for (int j = 0; j < i; ++j) z -= p.sqbd[i * kMaxQ1 + j] * w[j];
        w[i] = z / p.sqbd[i * kMaxQ1 + i];
        acc += w[i] * w[i];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out + blockIdx.y, 0.5 * acc);
}

// Decoupled residuals: every instance is component k = id of one d-dimensional problem solved
// with an approximate (diagonal or zero) Jacobian, laid out at offset k (N + 1); component k's
// residual reads the whole state y_j(n) = T_0 lin_j(n) of that problem.  Writes U, R as
// k_seg_residuals and, in place of the state, the diagonal Jacobian entry dF_kk/dy_k (Yv),
// which the chain kernels read through the kOdeDiagJacobian family.
template <class C>
__global__ void __launch_bounds__(256)
k_dec_residuals(const IeksParams<typename C::Tp> p, int d_full, int kind_full,
                typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
                typename C::Tp* __restrict__ Yv, typename C::Tp* __restrict__ d0) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  constexpr int D = C::D, Q1 = C::Q1;
  static_assert(C::DD == 1, "decoupled components are one-dimensional");
  for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp <= p.N;
       gp += (int64_t)gridDim.x * blockDim.x) {
    const int id = seg_id(p.seg.inst_of[gp]);
    const InstDesc<T>& d = p.seg.desc[id];
    const int64_t n = gp - d.off;
    const V* lin = static_cast<const V*>(d.lin[d.cur]);
    V x[D];
#pragma unroll
    for (int r = 0; r < D; ++r) x[r] = lin[n * D + r];
    if (n < d.N) {
#pragma unroll
      for (int i = 0; i < Q1; ++i) {
        V acc = x[i];
#pragma unroll
        for (int j = i + 1; j < Q1; ++j)
          acc = acc + x[j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
        acc = acc - lin[(n + 1) * D + i];
        U[gp * D + i] = v_to_T<T>(acc);
      }
    } else {
#pragma unroll
      for (int r = 0; r < D; ++r) U[gp * D + r] = T(0);
    }
    const V T0v = v_from_double<V>(d.T0d);
    const V T1iv = v_from_double<V>(d.T1invd);
    auto yv = [&](int j) -> V {
      const InstDesc<T>& e = p.seg.desc[j];
      return T0v * static_cast<const V*>(e.lin[e.cur])[n * D];
    };
    const V f = component_f<V, T>(kind_full, d.pd, d_full, id, yv);
    auto yt = [&](int j) -> T { return v_to_T<T>(yv(j)); };
    Yv[gp] = component_jac_diag<T>(kind_full, d.pd, d_full, id, yt);
    R[gp] = v_to_T<T>(f * T1iv - x[1]);
    if (n == 0) {
#pragma unroll
      for (int r = 0; r < D; ++r)
        d0[static_cast<int64_t>(id) * D + r] = v_to_T<T>(v_from_double<V>(d.mu0d[r]) - x[r]);
    }
  }
}

// Inputs of the increment model (as k_residuals) for every global point of the layout, with the
// instance's own constants: u_n = Phibar lin_n - lin_{n+1} (n < N_i; 0 at n = N_i), r_n, y_n, and
// delta_0 = mu0 - lin_0 of instance i at d0[i D ..].
template <class C>
__global__ void __launch_bounds__(256)
k_seg_residuals(const IeksParams<typename C::Tp> p, typename C::Tp* __restrict__ U,
                typename C::Tp* __restrict__ R, typename C::Tp* __restrict__ Yv,
                typename C::Tp* __restrict__ d0) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  for (int64_t gp = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gp <= p.N;
       gp += (int64_t)gridDim.x * blockDim.x) {
    const int id = seg_id(p.seg.inst_of[gp]);
    const InstDesc<T>& d = p.seg.desc[id];
    const int64_t n = gp - d.off;
    const V* lin = static_cast<const V*>(d.lin[d.cur]);
    V x[D];
#pragma unroll
    for (int r = 0; r < D; ++r) x[r] = lin[n * D + r];
    if (n < d.N) {
#pragma unroll
      for (int k = 0; k < DD; ++k) {
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
          V acc = x[k * Q1 + i];
#pragma unroll
          for (int j = i + 1; j < Q1; ++j)
            acc = acc + x[k * Q1 + j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
          acc = acc - lin[(n + 1) * D + k * Q1 + i];
          U[gp * D + k * Q1 + i] = v_to_T<T>(acc);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < D; ++r) U[gp * D + r] = T(0);
    }
    OdeConstsV<V> oc;
    ode_consts_v<V, T, DD>(p.ode, d.pd, oc);
    const V T0v = v_from_double<V>(d.T0d);
    const V T1iv = v_from_double<V>(d.T1invd);
    V y[DD], f[DD];
#pragma unroll
    for (int k = 0; k < DD; ++k) y[k] = T0v * x[k * Q1];
    ode_f_v<V, DD>(oc, y, f);
#pragma unroll
    for (int k = 0; k < DD; ++k) {
      Yv[gp * DD + k] = v_to_T<T>(y[k]);
      R[gp * DD + k] = v_to_T<T>(f[k] * T1iv - x[k * Q1 + 1]);
    }
    if (n == 0) {
#pragma unroll
      for (int r = 0; r < D; ++r)
        d0[static_cast<int64_t>(id) * D + r] = v_to_T<T>(v_from_double<V>(d.mu0d[r]) - x[r]);
    }
  }
}

// ---- all means iterations of a batch in one cooperative launch ------------------------------
// Arguments of k_batch_iterations.
template <typename T>
struct BatchRun {
  InstDesc<T>* desc;     // by instance id (offsets and current trajectories are rewritten)
  InstAcc* acc;          // per-instance reductions of the pass
  int* inst_of;          // per global point of the current layout
  int* ids;              // active instance ids in layout order
  SegIterState* st;      // per instance id
  int64_t* ctl;          // [0] points of the current layout, [1] active instances
  unsigned* bar;         // grid-barrier arrivals (cleared before the launch)
  T *U, *R, *Yv, *d0, *Es, *gs;
  int limit, fixed, calibrate, d, chain_len;
  double atol, rtol, diverged;
  int64_t cap;           // chains one launch holds
};

// Block 0 rewrites the layout after the stopping decisions: the active instances keep their
// order, each gets its new offset (exclusive prefix sum of N + 1 over the instances before it),
// and ctl receives the new point and instance counts.  Chunks of NT instances, prefix sums in
// shared memory; within a chunk every read happens before any write.
template <typename T, int NT>
__device__ void batch_compact(const BatchRun<T>& r, unsigned char* smem_raw) {
  int64_t* s_sz = reinterpret_cast<int64_t*>(smem_raw);
  int* s_ct = reinterpret_cast<int*>(smem_raw + 2 * NT * sizeof(int64_t));
  const int t = threadIdx.x;
  const int nact = static_cast<int>(r.ctl[1]);
  int out = 0;
  int64_t off = 0;
  for (int c0 = 0; c0 < nact; c0 += NT) {
    const int j = c0 + t;
    const int id = j < nact ? r.ids[j] : -1;
    const bool keep = id >= 0 && r.st[id].active;
    const int64_t sz = keep ? r.desc[id].N + 1 : 0;
    s_sz[t] = sz;
    s_ct[t] = keep ? 1 : 0;
    __syncthreads();
    // inclusive Hillis-Steele scans (ping-pong halves of the buffers)
    int src = 0;
    for (int o = 1; o < NT; o <<= 1) {
      const int64_t a = s_sz[src * NT + t] + (t >= o ? s_sz[src * NT + t - o] : 0);
      const int b = s_ct[src * NT + t] + (t >= o ? s_ct[src * NT + t - o] : 0);
      s_sz[(1 - src) * NT + t] = a;
      s_ct[(1 - src) * NT + t] = b;
      __syncthreads();
      src = 1 - src;
    }
    if (keep) {
      r.ids[out + s_ct[src * NT + t] - 1] = id;
      r.desc[id].off = off + s_sz[src * NT + t] - sz;
    }
    out += s_ct[src * NT + NT - 1];
    off += s_sz[src * NT + NT - 1];
    __syncthreads();
  }
  if (t == 0) {
    r.ctl[0] = off;
    r.ctl[1] = out;
  }
}

// All means iterations of a batch (Algorithm 2 per instance) in one cooperative launch.  Per
// iteration: the segmented IEKS pass over the current layout (iteration_body, chain length
// chosen so that the chains fill the resident blocks), a grid barrier, every active
// instance's stopping rule (the host loop's rule: non-finite or diverging values, fixed
// iteration count, max|dy| <= atol + rtol max|y|, iteration cap), a grid barrier, compaction of
// the active instances by block 0, a grid barrier, the new per-point instance map and cleared
// reductions, a grid barrier.  Every barrier and every cross-block wait is bounded (see
// group_wait); after a timeout the launch runs to its end without waiting and the host reports
// PIT_ETIMEOUT.
template <class C>
__global__ void __launch_bounds__(FusedShape<C>::NT, 1)
k_batch_iterations(const IeksParams<typename C::Tp> p0, const BatchRun<typename C::Tp> r,
                   const FusedXchg<typename C::Tp> x0) {
  using T = typename C::Tp;
  using FS = FusedShape<C>;
  constexpr int NT = FS::NT, NGB = FS::NGB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  unsigned gen = 0;
  auto grid_barrier = [&](unsigned k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(r.bar, 1u);
    }
    ++gen;
    if (grp == 0) {
      group_wait(g, r.bar, gen * gridDim.x, x0.status, x0.spin_limit, x0.where,
                 wait_tag(3u, blockIdx.x, k));
      __threadfence();
    }
    __syncthreads();
  };
  for (int k = 1; k <= r.limit; ++k) {
    const int64_t M = r.ctl[0];
    const int nact = static_cast<int>(r.ctl[1]);
    if (nact <= 0 || (ld_acquire_u32(x0.status) & kStatusTimeout)) break;
    // the iteration's parameters: the layout changes N, L and P (a local copy, whose hot fields
    // stay in registers; measured faster than a shared-memory copy)
    IeksParams<T> p = p0;
    p.N = M - 1;
    if (r.chain_len > 0) {
      p.L = r.chain_len;
    } else {
      const int64_t L = (M + r.cap - 1) / r.cap;
      p.L = static_cast<int>(L > 4 ? L : 4);
    }
    p.P = p.N / p.L + 1;
    const int nb = static_cast<int>((p.P + NGB - 1) / NGB);
    FusedXchg<T> x = x0;
    x.NB = nb;
    x.K = 0;
    while ((1 << x.K) < nb) ++x.K;
    x.epoch = static_cast<unsigned>(k);
    if (static_cast<int>(blockIdx.x) < nb)
      iteration_body<C, false, true>(p, blockIdx.x, nullptr, nullptr, r.U, r.R, r.Yv, r.d0, r.Es,
                                     r.gs, nullptr, nullptr, nullptr, nullptr, x, smem_raw);
    grid_barrier(k);
    // stopping rule of every instance of the pass
    for (int j = blockIdx.x * NT + threadIdx.x; j < nact; j += gridDim.x * NT) {
      const int id = r.ids[j];
      const InstAcc a = r.acc[id];
      SegIterState& s = r.st[id];
      const double Ni = static_cast<double>(r.desc[id].N);
      s.iters = k;
      s.last_delta = a.delta_max;
      s.sigma2 = r.calibrate ? a.sigma2_sum / (Ni * r.d) : 1.0;
      bool stop = false, conv = false, fail = false;
      if ((a.flags & 1u) || !(a.delta_max <= r.diverged)) {
        stop = fail = true;
      } else if (r.fixed > 0) {
        stop = conv = (k == r.limit);
      } else if (a.delta_max <= r.atol + r.rtol * a.y_max) {
        stop = conv = true;
      } else if (k == r.limit) {
        stop = true;
      }
      if (!stop) {
        s.cur ^= 1;
        r.desc[id].cur = s.cur;
      }
      s.active = stop ? 0 : 1;
      s.converged = conv ? 1 : 0;
      s.failed = fail ? 1 : 0;
    }
    grid_barrier(k);
    if (blockIdx.x == 0) batch_compact<T, NT>(r, smem_raw);
    grid_barrier(k);
    // the next layout: per-point instance codes, cleared reductions
    const int nnext = static_cast<int>(r.ctl[1]);
    for (int j = blockIdx.x; j < nnext; j += gridDim.x) {
      const int id = r.ids[j];
      const int64_t off = r.desc[id].off;
      const int64_t Ni = r.desc[id].N;
      for (int64_t n = threadIdx.x; n <= Ni; n += NT) r.inst_of[off + n] = (n == 0) ? ~id : id;
      if (threadIdx.x == 0) {
        InstAcc z = {};
        r.acc[id] = z;
      }
    }
    grid_barrier(k);
  }
}

template <typename T, int DD, int Q1, int G, int RL>
class SegEngineImpl final : public SegEngine {
 public:
  using C = Cfg<T, DD, Q1, G, RL>;
  using V = typename TrajType<T>::type;
  using Base = SolverImpl<T, DD, Q1, G, RL>;
  static constexpr int D = C::D;
  static constexpr int NG = kThreads / G;

  int state_dim() const override { return D; }
  size_t traj_bytes(int64_t N) const override {
    return static_cast<size_t>(N + 1) * D * sizeof(V);
  }

  static int64_t max_chains(int64_t max_points, int chain_len) {
    if (chain_len > 0) return (max_points - 1) / chain_len + 1;
    // default chain length (SolverImpl::default_chain_len) gives at most target + 1 chains, or
    // max_points / 512 + 1 when the length is clamped at 512
    const int64_t target = int64_t(sm_count()) * 8 * NG;
    return std::max<int64_t>(target + 2, max_points / 512 + 2);
  }

  struct Bufs {
    T *U, *R, *Yv, *d0, *Es, *gs, *Ls, *fagg, *fup, *sagg, *sup;
    SolveScalars* scal;
    InstDesc<T>* desc;
    InstAcc* acc;
    int* inst_of;
    SegSlot* slots;
    // device-iterated batches (run_iterations)
    SegIterState* st;
    int* ids;
    int64_t* ctl;
    unsigned* words;  // [0] status, [1] first timeout, [2] grid-barrier arrivals
    double* obj;      // objective values of the slots of one evaluation
    T *xf, *xs;
    unsigned* xflags;
    int xNB, xK;
  };

  // Blocks of k_batch_iterations that are resident at once (0 where it cannot run).
  static int persistent_blocks() {
    static std::atomic<int> cached{0};
    const int c = cached.load(std::memory_order_relaxed);
    if (c > 0) return c;
    using FS = FusedShape<C>;
    int nb = 0;
    if (cudaFuncSetAttribute(k_batch_iterations<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(FS::smem)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_iterations<C>, FS::NT,
                                                      FS::smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    const int v = nb * sm_count();
    cached.store(v, std::memory_order_relaxed);
    return v;
  }

  size_t carve(void* ws, size_t bytes, int64_t max_points, int max_inst, bool want_cov,
               int chain_len, Bufs& b) const {
    Carver cv(ws, bytes);
    const int64_t M = max_points;
    const int64_t P = max_chains(max_points, chain_len);
    b.U = cv.take<T>(M * D);
    b.R = cv.take<T>(M * DD);
    b.Yv = cv.take<T>(M * DD);
    b.d0 = cv.take<T>(static_cast<int64_t>(max_inst) * D);
    b.Es = cv.take<T>(M * D * D);
    b.gs = cv.take<T>(M * D);
    b.Ls = want_cov ? cv.take<T>(M * D * D) : nullptr;
    b.fagg = cv.take<T>(P * C::FA);
    b.fup = cv.take<T>(Tree<C, true, false, false, true>::upper_bytes(P) / sizeof(T) + 1);
    b.sagg = cv.take<T>(P * C::SA);
    const size_t sup_bytes = std::max(Tree<C, false, false, true>::upper_bytes(P),
                                      Tree<C, false, true, true>::upper_bytes(P));
    b.sup = cv.take<T>(sup_bytes / sizeof(T) + 1);
    b.scal = cv.take<SolveScalars>(1);
    b.desc = cv.take<InstDesc<T>>(max_inst);
    b.acc = cv.take<InstAcc>(max_inst);
    b.inst_of = cv.take<int>(M);
    b.slots = cv.take<SegSlot>(max_inst);
    b.st = cv.take<SegIterState>(max_inst);
    b.ids = cv.take<int>(max_inst);
    b.ctl = cv.take<int64_t>(2);
    b.words = cv.take<unsigned>(4);
    b.obj = cv.take<double>(max_inst);
    b.xNB = persistent_blocks();
    b.xK = 0;
    while ((1 << b.xK) < b.xNB) ++b.xK;
    const size_t lv = static_cast<size_t>(b.xK + 1) * b.xNB;
    b.xf = b.xNB ? cv.take<T>(lv * C::FA) : nullptr;
    b.xs = b.xNB ? cv.take<T>(lv * C::SA) : nullptr;
    b.xflags = b.xNB ? cv.take<unsigned>(2 * static_cast<size_t>(b.xNB)) : nullptr;
    return cv.used();
  }

  size_t workspace_bytes(int64_t max_points, int max_inst, bool want_cov,
                         int chain_len) const override {
    Bufs b;
    return carve(nullptr, 0, max_points, max_inst, want_cov, chain_len, b);
  }

  int bind(void* ws, size_t bytes, int64_t max_points, int max_inst, bool want_cov,
           int chain_len) override {
    const size_t need = carve(ws, bytes, max_points, max_inst, want_cov, chain_len, b_);
    if (bytes < need || !ws) {
      set_error("segmented workspace too small: need " + std::to_string(need) + " bytes");
      return PIT_ENOMEM;
    }
    if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) {
      set_error("workspace must be 256-byte aligned");
      return PIT_EINVAL;
    }
    max_points_ = max_points;
    max_inst_ = max_inst;
    want_cov_ = want_cov;
    chain_len_ = chain_len;
    h_desc_.assign(max_inst, InstDesc<T>{});
    h_acc_.assign(max_inst, InstAcc{});
    Ns_.assign(max_inst, 0);
    kind_ = -1;
    return Base::set_smem_attrs_seg();
  }

  int set_instance(int id, const Problem& pb, void* lin0, void* lin1, void* mean, void* cov,
                   cudaStream_t s) override {
    if (id < 0 || id >= max_inst_) {
      set_error("instance id out of range");
      return PIT_EINVAL;
    }
    if (kind_ < 0) {
      // constants shared by all instances: family, Phibar, sqrt(Qbar) (step-size free)
      SolveArgs a;
      std::memset(&a, 0, sizeof(a));
      a.pb = pb;
      pit_opts_default(&a.opts);
      int st = Base::fill_params(a, shared_, 0);
      if (st != PIT_OK) return st;
      kind_ = pb.kind;
    } else if (pb.kind != kind_) {
      set_error("all instances of a segmented solve must share the ODE family");
      return PIT_EINVAL;
    }
    if (pb.n_params > kMaxInstParams) {
      set_error("too many ODE parameters for a segmented solve");
      return PIT_EINVAL;
    }
    SolveArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pb = pb;
    pit_opts_default(&a.opts);
    IeksParams<T> pi;
    int st = Base::fill_params(a, pi, 0);
    if (st != PIT_OK) return st;
    InstDesc<T>& d = desc_host(id);
    std::memset(&d, 0, sizeof(d));
    d.off = 0;
    d.N = pb.N;
    d.lin[0] = lin0;
    d.lin[1] = lin1;
    d.cur = 0;
    d.mean = static_cast<T*>(mean);
    d.cov = static_cast<T*>(cov);
    d.mean_ld = D;
    d.cov_ld = D * D;
    d.cov_rld = D;
    for (int j = 0; j < pb.n_params; ++j) {
      d.pd[j] = pb.params[j];
      d.p[j] = static_cast<T>(pb.params[j]);
    }
    for (int r = 0; r < D; ++r) d.mu0d[r] = pi.mu0d[r];
    d.T0d = pi.T0d;
    d.T1invd = pi.T1invd;
    for (int i = 0; i < Q1; ++i) {
      d.Tdiagd[i] = pi.Tdiagd[i];
      d.Tdiag[i] = pi.Tdiag[i];
    }
    d.T0 = pi.T0;
    d.T1inv = pi.T1inv;
    d.hq = pi.hq;
    Ns_[id] = pb.N;
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.desc + id, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    return PIT_OK;
  }

  void set_linearization(int mode) override { lin_mode_ = mode; }
  void set_decoupled(bool on) override { decoupled_ = on; }

  int set_component(int id, const Problem& pb, int k, const double* mu0k, void* lin0,
                    void* lin1, void* mean, void* cov, cudaStream_t s) override {
    if constexpr (DD != 1) {
      set_error("internal: decoupled components need the d = 1 engine");
      return PIT_EINTERNAL;
    } else {
      if (id < 0 || id >= max_inst_) {
        set_error("instance id out of range");
        return PIT_EINVAL;
      }
      if (pb.n_params > kMaxInstParams) {
        set_error("too many ODE parameters for a decoupled solve");
        return PIT_EINVAL;
      }
      const int Dfull = pb.d * Q1;
      // prior blocks and preconditioner of the common step size (the component problem is the
      // 1-dimensional IWP(q) with the full problem's grid)
      Problem p1 = pb;
      p1.kind = PIT_ODE_LOGISTIC;
      p1.d = 1;
      p1.n_params = 1;
      p1.params[0] = 0.0;
      p1.y0[0] = 0.0;
      SolveArgs a;
      std::memset(&a, 0, sizeof(a));
      a.pb = p1;
      pit_opts_default(&a.opts);
      IeksParams<T> pi;
      int st = Base::fill_params(a, pi, 0);
      if (st != PIT_OK) return st;
      if (kind_ < 0) {
        shared_ = pi;
        shared_.ode.kind = kOdeDiagJacobian;
        shared_.ode.d = 1;
        kind_ = kOdeDiagJacobian;
      }
      InstDesc<T>& d = desc_host(id);
      std::memset(&d, 0, sizeof(d));
      d.N = pb.N;
      d.lin[0] = lin0;
      d.lin[1] = lin1;
      d.mean = static_cast<T*>(mean) + static_cast<int64_t>(k) * Q1;
      d.cov = cov ? static_cast<T*>(cov) + static_cast<int64_t>(k) * Q1 * Dfull +
                        static_cast<int64_t>(k) * Q1
                  : nullptr;
      d.mean_ld = Dfull;
      d.cov_ld = static_cast<int64_t>(Dfull) * Dfull;
      d.cov_rld = Dfull;
      for (int j = 0; j < pb.n_params; ++j) {
        d.pd[j] = pb.params[j];
        d.p[j] = static_cast<T>(pb.params[j]);
      }
      for (int r = 0; r < Q1; ++r) d.mu0d[r] = mu0k[r] / pi.Tdiagd[r];
      d.T0d = pi.T0d;
      d.T1invd = pi.T1invd;
      for (int i = 0; i < Q1; ++i) {
        d.Tdiagd[i] = pi.Tdiagd[i];
        d.Tdiag[i] = pi.Tdiag[i];
      }
      d.T0 = pi.T0;
      d.T1inv = pi.T1inv;
      d.hq = pi.hq;
      Ns_[id] = pb.N;
      dec_kind_ = pb.kind;
      dec_d_ = pb.d;
      PIT_CUDA_TRY(cudaMemcpyAsync(b_.desc + id, &d, sizeof(d), cudaMemcpyHostToDevice, s));
      return PIT_OK;
    }
  }

  int use_pinned_staging() override {
    if (pin_desc_) return PIT_OK;
    PIT_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&pin_desc_),
                                sizeof(InstDesc<T>) * max_inst_));
    PIT_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&pin_slots_),
                                sizeof(SegSlot) * max_inst_));
    PIT_CUDA_TRY(cudaMallocHost(reinterpret_cast<void**>(&pin_acc_), sizeof(InstAcc) * max_inst_));
    return PIT_OK;
  }

  ~SegEngineImpl() override {
    if (pin_desc_) cudaFreeHost(pin_desc_);
    if (pin_slots_) cudaFreeHost(pin_slots_);
    if (pin_acc_) cudaFreeHost(pin_acc_);
  }

  int upload_slots(const SegSlot* slots, int n, cudaStream_t s) {
    if (n < 1 || n > max_inst_) {
      set_error("slot count out of range");
      return PIT_EINVAL;
    }
    const SegSlot* src = slots;
    if (pin_slots_) {
      // the previous upload from the staging buffer must have been consumed
      PIT_CUDA_TRY(cudaStreamSynchronize(s));
      std::memcpy(pin_slots_, slots, sizeof(SegSlot) * n);
      src = pin_slots_;
    }
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.slots, src, sizeof(SegSlot) * n, cudaMemcpyHostToDevice, s));
    return PIT_OK;
  }

  unsigned per_slot_grid(const SegSlot* slots, int n) const {
    int64_t mx = 1;
    for (int i = 0; i < n; ++i) mx = std::max<int64_t>(mx, (Ns_[slots[i].id] + 1) * D);
    return static_cast<unsigned>(std::min<int64_t>((mx + 255) / 256, 64));
  }

  int init_traj(const SegSlot* slots, int n, cudaStream_t s) override {
    int st = upload_slots(slots, n, s);
    if (st != PIT_OK) return st;
    dim3 grid(per_slot_grid(slots, n), static_cast<unsigned>(n));
    PIT_LAUNCH(KC_INIT, s, k_seg_init<C><<<grid, 256, 0, s>>>(b_.slots, b_.desc););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  int objective(const SegSlot* slots, int n, double* out, cudaStream_t s) override {
    int st = upload_slots(slots, n, s);
    if (st != PIT_OK) return st;
    PIT_CUDA_TRY(cudaMemsetAsync(b_.obj, 0, sizeof(double) * n, s));
    dim3 grid(per_slot_grid(slots, n), static_cast<unsigned>(n));
    PIT_LAUNCH(KC_EXPORT, s, k_seg_objective<C><<<grid, 256, 0, s>>>(b_.slots, b_.desc, shared_, b_.obj););
    PIT_CUDA_TRY(cudaGetLastError());
    PIT_CUDA_TRY(cudaMemcpyAsync(out, b_.obj, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    return PIT_OK;
  }

  int export_means(const SegSlot* slots, int n, cudaStream_t s) override {
    int st = upload_slots(slots, n, s);
    if (st != PIT_OK) return st;
    dim3 grid(per_slot_grid(slots, n), static_cast<unsigned>(n));
    PIT_LAUNCH(KC_EXPORT, s, k_seg_export<C><<<grid, 256, 0, s>>>(b_.slots, b_.desc););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  template <bool WITH_L>
  int pass_t(int64_t M, int calibrate, cudaStream_t s) {
    IeksParams<T> p = shared_;
    p.N = M - 1;
    p.L = chain_len_ > 0 ? chain_len_ : Base::default_chain_len(p.N);
    p.P = p.N / p.L + 1;
    p.want_cov = WITH_L ? 1 : 0;
    p.calibrate = calibrate;
    p.lin_mode = lin_mode_;
    p.want_sigma = 1;
    p.sigma_pool = decoupled_ ? dec_d_ : 0;
    p.seg.desc = b_.desc;
    p.seg.inst_of = b_.inst_of;
    p.seg.acc = b_.acc;
    if (p.P > max_chains(max_points_, chain_len_)) {
      set_error("internal: chain count exceeds the bound");
      return PIT_EINTERNAL;
    }
    const unsigned grid = static_cast<unsigned>((p.P + NG - 1) / NG);
    const size_t sm = Base::chain_smem();
    if (decoupled_) {
      if constexpr (DD == 1) {
        PIT_LAUNCH(KC_RESIDUALS, s,
                   k_dec_residuals<C><<<Base::elem_grid(M, 256), 256, 0, s>>>(
                       p, dec_d_, dec_kind_, b_.U, b_.R, b_.Yv, b_.d0););
      }
    } else {
      PIT_LAUNCH(KC_RESIDUALS, s,
                 k_seg_residuals<C><<<Base::elem_grid(M, 256), 256, 0, s>>>(p, b_.U, b_.R, b_.Yv,
                                                                           b_.d0););
    }
    PIT_LAUNCH(KC_FILTER_REDUCE, s,
               k_filter_reduce<C, true><<<grid, kThreads, sm, s>>>(p, b_.U, b_.R, b_.Yv, b_.d0,
                                                                  b_.fagg););
    int st = Tree<C, true, false, false, true>::run(b_.fagg, p.P, b_.fup, false, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_FILTER_DOWN, s,
               k_filter_down<C, WITH_L, false, true><<<grid, kThreads, sm, s>>>(
                   p, b_.U, b_.R, b_.Yv, b_.d0, b_.fagg, b_.Es, b_.gs, b_.Ls, b_.sagg, b_.scal););
    st = Tree<C, false, WITH_L, true>::run(b_.sagg, p.P, b_.sup, true, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SMOOTH_DOWN, s,
               k_smooth_down<C, WITH_L, true><<<grid, kThreads, sm, s>>>(
                   p, b_.Es, b_.gs, b_.Ls, b_.sagg, nullptr, nullptr, nullptr, nullptr, b_.scal););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  int pass_begin(const SegSlot* slots, int n, bool with_L, int calibrate,
                 cudaStream_t s) override {
    if (with_L && !want_cov_) {
      set_error("covariance pass on an engine bound without covariance buffers");
      return PIT_EINVAL;
    }
    int64_t M = 0;
    for (int i = 0; i < n; ++i) {
      if (slots[i].off != M) {
        set_error("internal: slots must tile the global points in order");
        return PIT_EINTERNAL;
      }
      M += Ns_[slots[i].id] + 1;
    }
    if (M > max_points_ || M < 2) {
      set_error("layout exceeds the engine's point capacity");
      return PIT_EINVAL;
    }
    int st = upload_slots(slots, n, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_INIT, s,
               k_seg_layout<T><<<static_cast<unsigned>(n), 256, 0, s>>>(b_.slots, b_.desc,
                                                                       b_.inst_of););
    PIT_CUDA_TRY(cudaMemsetAsync(b_.acc, 0, sizeof(InstAcc) * max_inst_, s));
    st = with_L ? pass_t<true>(M, calibrate, s) : pass_t<false>(M, calibrate, s);
    if (st != PIT_OK) return st;
    begun_.assign(slots, slots + n);
    if (pin_acc_) {
      PIT_CUDA_TRY(cudaMemcpyAsync(pin_acc_, b_.acc, sizeof(InstAcc) * max_inst_,
                                   cudaMemcpyDeviceToHost, s));
    }
    return PIT_OK;
  }

  int pass_end(SegResult* res, cudaStream_t s) override {
    const InstAcc* src = pin_acc_;
    if (!pin_acc_) {
      // pageable destination: returns once the copy (and everything before it) has completed
      PIT_CUDA_TRY(cudaMemcpyAsync(h_acc_.data(), b_.acc, sizeof(InstAcc) * max_inst_,
                                   cudaMemcpyDeviceToHost, s));
      src = h_acc_.data();
    }
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t i = 0; i < begun_.size(); ++i)
      std::memcpy(&res[i], &src[begun_[i].id], sizeof(SegResult));
    return PIT_OK;
  }

  int pass(const SegSlot* slots, int n, bool with_L, int calibrate, SegResult* res,
           cudaStream_t s) override {
    int st = pass_begin(slots, n, with_L, calibrate, s);
    if (st != PIT_OK) return st;
    return pass_end(res, s);
  }

  int run_iterations(int n, const pit_opts& o, double diverged_delta, SegIterState* out,
                     cudaStream_t s) override {
    using FS = FusedShape<C>;
    if (decoupled_ || b_.xNB <= 0 || n < 1 || n > max_inst_) return PIT_EUNSUPPORTED;
    const int64_t cap = static_cast<int64_t>(b_.xNB) * FS::NGB;
    std::vector<SegSlot> slots(n);
    std::vector<int> ids(n);
    std::vector<SegIterState> st(n);
    int64_t M = 0;
    for (int i = 0; i < n; ++i) {
      slots[i] = SegSlot{i, 0, M};
      ids[i] = i;
      st[i] = SegIterState{0, 0, 1, 0, 0, 0, 0.0, 1.0};
      M += Ns_[i] + 1;
    }
    if (M > max_points_ || M < 2) {
      set_error("layout exceeds the engine's point capacity");
      return PIT_EINVAL;
    }
    if (o.chain_len > 0 && (M - 2) / o.chain_len + 1 > cap) return PIT_EUNSUPPORTED;
    // the first layout (every instance, trajectories lin[0]) and cleared state
    int st0 = upload_slots(slots.data(), n, s);
    if (st0 != PIT_OK) return st0;
    PIT_LAUNCH(KC_INIT, s,
               k_seg_layout<T><<<static_cast<unsigned>(n), 256, 0, s>>>(b_.slots, b_.desc,
                                                                       b_.inst_of););
    PIT_CUDA_TRY(cudaMemsetAsync(b_.acc, 0, sizeof(InstAcc) * max_inst_, s));
    PIT_CUDA_TRY(cudaMemsetAsync(b_.words, 0, 4 * sizeof(unsigned), s));
    PIT_CUDA_TRY(cudaMemsetAsync(b_.xflags, 0, 2 * sizeof(unsigned) * b_.xNB, s));
    const int64_t ctl[2] = {M, n};
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.ids, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.st, st.data(), sizeof(SegIterState) * n,
                                 cudaMemcpyHostToDevice, s));
    IeksParams<T> p = shared_;
    p.want_cov = 0;
    p.calibrate = o.calibrate;
    p.lin_mode = lin_mode_;
    p.want_sigma = 1;
    p.sigma_pool = 0;
    p.seg.desc = b_.desc;
    p.seg.inst_of = b_.inst_of;
    p.seg.acc = b_.acc;
    BatchRun<T> r;
    r.desc = b_.desc;
    r.acc = b_.acc;
    r.inst_of = b_.inst_of;
    r.ids = b_.ids;
    r.st = b_.st;
    r.ctl = b_.ctl;
    r.bar = b_.words + 2;
    r.U = b_.U;
    r.R = b_.R;
    r.Yv = b_.Yv;
    r.d0 = b_.d0;
    r.Es = b_.Es;
    r.gs = b_.gs;
    r.limit = o.fixed_iters > 0 ? o.fixed_iters : o.max_iter;
    r.fixed = o.fixed_iters;
    r.calibrate = o.calibrate;
    r.d = DD;
    r.chain_len = o.chain_len;
    r.atol = o.atol_delta;
    r.rtol = o.rtol_delta;
    r.diverged = diverged_delta;
    r.cap = cap;
    FusedXchg<T> x;
    std::memset(&x, 0, sizeof(x));
    x.fbuf = b_.xf;
    x.sbuf = b_.xs;
    x.fflag = b_.xflags;
    x.sflag = b_.xflags + b_.xNB;
    x.status = b_.words;
    x.where = b_.words + 1;
    x.NB = b_.xNB;
    x.K = b_.xK;
    x.spin_limit = Base::kSpinLimit;
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_batch_iterations<C>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(FS::smem)));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(b_.xNB));
    cfg.blockDim = dim3(FS::NT);
    cfg.dynamicSmemBytes = FS::smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    PIT_LAUNCH(KC_ITERATION, s, e = cudaLaunchKernelEx(&cfg, k_batch_iterations<C>, p, r, x));
    if (e != cudaSuccess) {
      set_error(std::string("cooperative launch of the batched iterations: ") +
                cudaGetErrorString(e));
      return PIT_ECUDA;
    }
    unsigned words[4];
    PIT_CUDA_TRY(cudaMemcpyAsync(out, b_.st, sizeof(SegIterState) * n, cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(words, b_.words, sizeof(words), cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    if (words[0] & kStatusTimeout) {
      static const char* phases[] = {"filter scan", "smoothing scan", "calibration barrier",
                                     "grid barrier"};
      const unsigned w = words[1];
      set_error(std::string("a cross-block wait of the batched iterations ran out (") +
                phases[(w >> 28) & 3u] + ", block position " + std::to_string(w & 0xffffu) +
                ", iteration/level " + std::to_string((w >> 16) & 0xffu) + ")");
      return PIT_ETIMEOUT;
    }
    return PIT_OK;
  }

  static SegEngine* make() { return new SegEngineImpl(); }

 private:
  Bufs b_{};
  int64_t max_points_ = 0;
  int max_inst_ = 0;
  bool want_cov_ = false;
  int chain_len_ = 0;
  int kind_ = -1;
  int lin_mode_ = 0;
  bool decoupled_ = false;
  int dec_kind_ = 0, dec_d_ = 1;
  IeksParams<T> shared_{};
  InstDesc<T>& desc_host(int id) { return pin_desc_ ? pin_desc_[id] : h_desc_[id]; }
  std::vector<InstDesc<T>> h_desc_;
  std::vector<InstAcc> h_acc_;
  std::vector<int64_t> Ns_;
  std::vector<SegSlot> begun_;
  InstDesc<T>* pin_desc_ = nullptr;
  SegSlot* pin_slots_ = nullptr;
  InstAcc* pin_acc_ = nullptr;
};

}  // namespace pit
