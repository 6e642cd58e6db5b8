// One IEKS iteration in a single cooperative launch (Algorithms 1 and 2 for small D).
//
// The multi-launch form of an iteration runs the residuals, the filter chains, a tree of block
// launches over the chain aggregates, the filter down-sweep, a second tree for the smoothing
// scan and the smoothing down-sweep: fourteen launches whose scan trees are latency-bound (a
// few combines per launch and a launch gap each).  Here one launch does all of it.  A block of
// NT threads owns NGB consecutive chains; all blocks are resident at once (cooperative launch),
// and blocks exchange scan values through global memory with per-block flags:
//   0. residuals of the increment model for the block's time steps (data-parallel, staged in
//      shared memory);
//   A. every group folds its chain's filtering elements into the chain aggregate (Section
//      3.1.2, Eq. sqrt-associative-filtering applied leaf by leaf);
//   B. the block reduces its NGB aggregates with a Brent-Kung up-sweep in shared memory;
//   C. the blocks compute the prefix over the block totals by a decoupled cross-block scan:
//      in round k every block looks back 2^k blocks, waits for that block's round-k value and
//      combines it with its own (log2 of the block count rounds, each value posted to global
//      memory behind a release flag).  A look-back that walked one predecessor at a time would
//      put all block combines on one chain, because every block reaches this point at the same
//      moment (one resident wave); doubling the distance keeps the chain logarithmic;
//   D. a Blelloch down-sweep in shared memory turns the block's exclusive prefix into every
//      chain's exclusive prefix (values only: every prefix starts at the initial state);
//   E. every group runs its chain's square-root Kalman steps from that prefix, emitting the
//      smoothing elements and folding them into the chain's smoothing aggregate;
//   F. B-D again for the reverse smoothing scan (Section 3.1.3), block order and chain order
//      reversed;
//   G. every group walks its chain backwards from its smoothing prefix: new trajectory (or
//      outputs) and the stopping-rule reductions.
// Every wait on another block's flag is bounded (spin_limit polls); when one runs out the
// kernel sets the timeout bit in the status word, every later wait returns at once, and the
// host reports PIT_ETIMEOUT after the launch.
#pragma once

#include "pit_chains.cuh"

namespace pit {

constexpr unsigned kStatusTimeout = 2u;  // SolveScalars::flags bit: a cross-block wait ran out

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kWaitNs = 4000000000ull;  // a wait gives up after 4 s

// A trajectory value (FP64) from its 8-byte bit pattern.
__device__ __forceinline__ void bits_to(uint2 w, double& v) { v = __hiloint2double(w.y, w.x); }

// Cross-block exchange state of one launch.
template <typename T>
struct FusedXchg {
  T* fbuf;             // filter scan values, (K + 1) levels x NB positions x FA
  T* sbuf;             // smoothing scan values, (K + 1) x NB x SA
  unsigned* fflag;     // per position: epoch * 64 + (highest level posted + 1)
  unsigned* sflag;
  unsigned* status;    // timeout bit (cleared once per solve)
  unsigned* where;     // first wait that ran out: wait_tag() code (cleared once per solve)
  unsigned* barrier;   // arrivals at the calibration barrier (cleared once per solve)
  unsigned bar_target; // arrivals to wait for in this launch (NB x covariance launches so far)
  unsigned epoch;      // >= 1, distinct for every launch since the flags were cleared
  int K;               // rounds: 2^K >= NB
  int NB;              // blocks
  long long spin_limit;  // polls per wait before giving up
};

// Identifies a wait for the error report: the phase (0 filter scan, 1 smoothing scan,
// 2 calibration barrier), the scan position of the waiting block and the level it waited for.
__device__ __forceinline__ unsigned wait_tag(unsigned phase, unsigned pos, unsigned level) {
  return 0x80000000u | (phase << 28) | ((level & 0xffu) << 16) | (pos & 0xffffu);
}

// Every lane of the group polls `flag` until it reaches `target` (all lanes agree on the
// result).  A wait gives up after `limit` polls or kWaitNs of wall time, whichever comes
// first, or as soon as another wait has given up; the first wait that gives up records `tag`
// in *where.  Returns false when it gave up.
template <class GR>
__device__ bool group_wait(const GR& g, const unsigned* flag, unsigned target, unsigned* status,
                           long long limit, unsigned* where = nullptr, unsigned tag = 0) {
  bool ok = false;
  const unsigned long long t0 = global_ns();
  for (long long it = 0;; ++it) {
    if (ld_acquire_u32(flag) >= target) {
      ok = true;
      break;
    }
    if (ld_acquire_u32(status) & kStatusTimeout) break;
    if (it >= limit || global_ns() - t0 > kWaitNs) {
      if (where) atomicCAS(where, 0u, tag);
      atomicOr(status, kStatusTimeout);
      break;
    }
    __nanosleep(128);
  }
  return __all_sync(g.mask, ok);
}

// Store an item to global memory and publish it: every lane's stores are fenced before the
// group's release of the flag.
template <class C, int SZ>
__device__ __forceinline__ void post_item(const typename C::GR& g, const typename C::Tp* src,
                                          typename C::Tp* dst, unsigned* flag, unsigned value) {
  for (int i = g.gl; i < SZ; i += C::G) dst[i] = src[i];
  __threadfence();
  g.sync();
  if (g.gl == 0) st_release_u32(flag, value);
  g.sync();
}

template <class C, int SZ>
__device__ __forceinline__ void fetch_item(const typename C::GR& g, const typename C::Tp* src,
                                           typename C::Tp* dst) {
  for (int i = g.gl; i < SZ; i += C::G) dst[i] = __ldcg(src + i);
  g.sync();
}

// The decoupled cross-block scan, run by one group of each block.  `cur` (shared memory) holds
// the block's total on entry; on return `xpre` holds the block's exclusive prefix (the combined
// totals of all positions before `pos`; untouched for pos == 0).  Position pos of the scan is
// the block index (filter) or the reversed block index (smoothing); OPS/REVERSE as in the tree
// kernels.  Returns false after a timed-out wait.
template <class C, class OPS, bool REVERSE>
__device__ bool cross_block_scan(const typename C::GR& g, int pos, typename C::Tp* cur,
                                 typename C::Tp* xpre, typename C::Tp* tmp, typename C::Tp* scr,
                                 typename C::Tp* buf, unsigned* flags,
                                 const FusedXchg<typename C::Tp>& x, unsigned phase) {
  constexpr int SZ = OPS::SZ;
  const unsigned base = x.epoch * 64u;
  const size_t lvl = static_cast<size_t>(x.NB) * SZ;
  post_item<C, SZ>(g, cur, buf + static_cast<size_t>(pos) * SZ, flags + pos, base + 1);
  bool ok = true;
  for (int k = 0; k < x.K; ++k) {
    const int s = 1 << k;
    if (pos >= s) {
      ok = ok && group_wait(g, flags + (pos - s), base + k + 1, x.status, x.spin_limit, x.where,
                            wait_tag(phase, pos, k));
      if (ok) {
        fetch_item<C, SZ>(g, buf + k * lvl + static_cast<size_t>(pos - s) * SZ, tmp);
        OPS::template op<REVERSE>(g, tmp, cur, cur, scr);
      }
    }
    post_item<C, SZ>(g, cur, buf + (k + 1) * lvl + static_cast<size_t>(pos) * SZ, flags + pos,
                     base + k + 2);
  }
  if (pos > 0) {
    ok = ok && group_wait(g, flags + (pos - 1), base + x.K + 1, x.status, x.spin_limit, x.where,
                          wait_tag(phase, pos, x.K + 1));
    if (ok) fetch_item<C, SZ>(g, buf + x.K * lvl + static_cast<size_t>(pos - 1) * SZ, xpre);
  }
  return ok;
}

// Launch geometry of the fused kernel for configuration C.
template <class C>
struct FusedShape {
  using T = typename C::Tp;
  static constexpr int NT = sizeof(T) == 4 ? 512 : 256;  // threads per block
  static constexpr int NGB = NT / C::G;                   // chains (groups) per block
  // residual phase: one time step per thread, NT steps per tile
  static constexpr int SV = C::D | 1, SU = C::D | 1, SR = C::DD | 1;
  static constexpr size_t res_bytes =
      static_cast<size_t>(NT + 1) * SV * 8 + static_cast<size_t>(NT) * (SU + 2 * SR) * sizeof(T);
  // chain phases: group scratch, NGB items, one temporary item per group, the block prefix
  static constexpr size_t chain_bytes =
      (static_cast<size_t>(NGB) * (C::SCR + 2 * C::FA) + C::FA) * sizeof(T);
  static constexpr size_t smem = res_bytes > chain_bytes ? res_bytes : chain_bytes;
};

// Residuals of the increment model for the time steps n in [lo, hi] (see k_residuals): u_{n-1},
// r_n and y_n, and delta_0 when lo == 1.  Tiles of NT steps; the trajectory rows n-1 .. n of a
// tile are staged in shared memory so that global loads and stores are contiguous.
template <class C, int NT>
__device__ void residual_steps(const IeksParams<typename C::Tp>& p,
                               const typename TrajType<typename C::Tp>::type* __restrict__ lin,
                               typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
                               typename C::Tp* __restrict__ Yv, typename C::Tp* __restrict__ d0,
                               int64_t lo, int64_t hi, unsigned char* s_raw) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  using FS = FusedShape<C>;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  constexpr int SV = FS::SV, SU = FS::SU, SR = FS::SR;
  uint2* s_lin = reinterpret_cast<uint2*>(s_raw);
  T* s_u = reinterpret_cast<T*>(s_raw + static_cast<size_t>(NT + 1) * SV * 8);
  T* s_r = s_u + NT * SU;
  T* s_y = s_r + NT * SR;
  const uint2* lin_w = reinterpret_cast<const uint2*>(lin);
  OdeConstsV<V> oc;
  ode_consts_v<V, T, DD>(p.ode, p.pd, oc);
  const V T0v = v_from_double<V>(p.T0d);
  const V T1iv = v_from_double<V>(p.T1invd);
  const int t = threadIdx.x;
  for (int64_t n0 = lo; n0 <= hi; n0 += NT) {
    const int cnt = static_cast<int>(hi - n0 + 1 < NT ? hi - n0 + 1 : NT);
    // rows n0 - 1 .. n0 + cnt - 1
    for (int i = t; i < (cnt + 1) * D; i += NT)
      s_lin[(i / D) * SV + i % D] = lin_w[(n0 - 1) * D + i];
    __syncthreads();
    if (t < cnt) {
      V xp[D], x[D];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        bits_to(s_lin[t * SV + r], xp[r]);
        bits_to(s_lin[(t + 1) * SV + r], x[r]);
      }
#pragma unroll
      for (int k = 0; k < DD; ++k) {
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
          V acc = xp[k * Q1 + i];
#pragma unroll
          for (int j = i + 1; j < Q1; ++j)
            acc = acc + xp[k * Q1 + j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
          acc = acc - x[k * Q1 + i];
          s_u[t * SU + k * Q1 + i] = v_to_T<T>(acc);
        }
      }
      V y[DD], f[DD];
#pragma unroll
      for (int k = 0; k < DD; ++k) y[k] = T0v * x[k * Q1];
      ode_f_v<V, DD>(oc, y, f);
#pragma unroll
      for (int k = 0; k < DD; ++k) {
        s_y[t * SR + k] = v_to_T<T>(y[k]);
        s_r[t * SR + k] = v_to_T<T>(f[k] * T1iv - x[k * Q1 + 1]);
      }
      if (n0 + t == 1) {
#pragma unroll
        for (int r = 0; r < D; ++r) d0[r] = v_to_T<T>(v_from_double<V>(p.mu0d[r]) - xp[r]);
      }
    }
    __syncthreads();
    for (int i = t; i < cnt * D; i += NT) U[(n0 - 1) * D + i] = s_u[(i / D) * SU + i % D];
    for (int i = t; i < cnt * DD; i += NT) {
      const int o = (i / DD) * SR + i % DD;
      R[n0 * DD + i] = s_r[o];
      Yv[n0 * DD + i] = s_y[o];
    }
    __syncthreads();
  }
}

// Residuals of the increment model for the time steps n in [lo, hi] of a segmented layout (see
// k_seg_residuals): instance id = the owner of point n, local index m = n - off_id.  Step n reads
// rows m-1 and m of the instance's own trajectory; at an instance's first point (m = 0) it
// writes that instance's delta_0 instead of u (the point is a reset element).  Block 0 also
// writes delta_0 of the instance at global point 0.  One thread per step.
template <class C, int NT>
__device__ void residual_steps_seg(const IeksParams<typename C::Tp>& p,
                                   typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
                                   typename C::Tp* __restrict__ Yv,
                                   typename C::Tp* __restrict__ d0, int64_t lo, int64_t hi) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  auto start = [&](int id, const InstDesc<T>& d) {
    const V* lin = static_cast<const V*>(d.lin[d.cur]);
#pragma unroll
    for (int r = 0; r < D; ++r)
      d0[static_cast<int64_t>(id) * D + r] = v_to_T<T>(v_from_double<V>(d.mu0d[r]) - lin[r]);
  };
  if (lo == 1 && threadIdx.x == 0) {
    const int id = seg_id(p.seg.inst_of[0]);
    start(id, p.seg.desc[id]);
  }
  for (int64_t n = lo + threadIdx.x; n <= hi; n += NT) {
    const int id = seg_id(p.seg.inst_of[n]);
    const InstDesc<T>& d = p.seg.desc[id];
    const int64_t m = n - d.off;
    const V* lin = static_cast<const V*>(d.lin[d.cur]);
    V x[D];
#pragma unroll
    for (int r = 0; r < D; ++r) x[r] = lin[m * D + r];
    if (m == 0) {
      start(id, d);
    } else {
#pragma unroll
      for (int k = 0; k < DD; ++k) {
#pragma unroll
        for (int i = 0; i < Q1; ++i) {
          V acc = lin[(m - 1) * D + k * Q1 + i];
#pragma unroll
          for (int j = i + 1; j < Q1; ++j)
            acc = acc + lin[(m - 1) * D + k * Q1 + j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
          acc = acc - x[k * Q1 + i];
          U[(n - 1) * D + k * Q1 + i] = v_to_T<T>(acc);
        }
      }
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
      Yv[n * DD + k] = v_to_T<T>(y[k]);
      R[n * DD + k] = v_to_T<T>(f[k] * T1iv - x[k * Q1 + 1]);
    }
  }
  __syncthreads();
}

// One IEKS iteration of the chains of block `blk` (phases 0 and A-G above).  SEG: the time axis
// is a segmented layout of many instances (segment boundaries absorb in the operators, see
// InstDesc).  Every thread of the block calls it.
template <class C, bool WITH_L, bool SEG>
__device__ __forceinline__ void iteration_body(
    const IeksParams<typename C::Tp>& p, int blk,
    const typename TrajType<typename C::Tp>::type* __restrict__ lin,
    typename TrajType<typename C::Tp>::type* __restrict__ lin_out,
    typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
    typename C::Tp* __restrict__ Yv, typename C::Tp* __restrict__ d0,
    typename C::Tp* __restrict__ Es, typename C::Tp* __restrict__ gs,
    typename C::Tp* __restrict__ Ls, typename C::Tp* __restrict__ mean_out,
    typename C::Tp* __restrict__ cov_out, SolveScalars* __restrict__ scal,
    const FusedXchg<typename C::Tp>& x, unsigned char* smem_raw) {
  using T = typename C::Tp;
  using GR = typename C::GR;
  using FS = FusedShape<C>;
  using OPF = TreeOps<C, true, false, true>;
  using OPS = TreeOps<C, false, WITH_L>;
  constexpr int NGB = FS::NGB, FA = C::FA, SA = C::SA;
  T* smem = reinterpret_cast<T*>(smem_raw);
  GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t base = static_cast<int64_t>(blk) * NGB;
  const int64_t chain = base + grp;
  const int nv = static_cast<int>(p.P - base < NGB ? p.P - base : NGB);  // chains of this block
  T* scr = smem + grp * C::SCR;
  T* items = smem + NGB * C::SCR;
  T* tmp = items + NGB * FA + grp * FA;
  T* xpre = items + 2 * NGB * FA;

  // 0. residuals for the steps of this block's chains
  {
    const int64_t lo = base * p.L + 1;
    int64_t hi = (base + nv) * p.L;
    hi = hi < p.N ? hi : p.N;
    if constexpr (SEG) residual_steps_seg<C, FS::NT>(p, U, R, Yv, d0, lo, hi);
    else residual_steps<C, FS::NT>(p, lin, U, R, Yv, d0, lo, hi, smem_raw);
  }
  // (the last __syncthreads of the residual phase orders its global stores before the chains)

  // A. filter chain aggregates
  if (chain < p.P) filter_reduce_chain<C, SEG>(g, p, U, R, Yv, d0, chain, scr, items + grp * FA);
  else set_identity_f<C>(g, items + grp * FA);
  __syncthreads();
  // B. block up-sweep; C. cross-block scan; D. down-sweep to chain prefixes
  block_tree<C, OPF, false>(items, NGB, nv, tmp, scr, g, grp, NGB, true, false, nullptr);
  if (grp == 0)
    cross_block_scan<C, OPF, false>(g, blk, items + (NGB - 1) * FA, xpre, tmp, scr, x.fbuf,
                                    x.fflag, x, 0u);
  __syncthreads();
  block_tree<C, OPF, false>(items, NGB, nv, tmp, scr, g, grp, NGB, false, true,
                            blk > 0 ? xpre : nullptr);
  __syncthreads();
  // E. filter down-sweep of every chain; its smoothing aggregate goes to position nv-1-grp
  // (reverse order for the smoothing scan)
  if (chain < p.P)
    filter_down_chain<C, WITH_L, false, SEG>(g, p, U, R, Yv, d0, items + grp * FA, Es, gs, Ls,
                                             tmp, scal, chain, scr);
  __syncthreads();
  // the aggregates were written to each group's temporary slot; move them into scan positions
  if (chain < p.P) copy_item<C, SA>(g, tmp, items + (nv - 1 - grp) * SA);
  else set_identity_s<C>(g, items + grp * SA);
  __syncthreads();
  // F. reverse smoothing scan over the block's aggregates and across blocks
  const int rpos = x.NB - 1 - blk;
  block_tree<C, OPS, true>(items, NGB, nv, tmp, scr, g, grp, NGB, true, false, nullptr);
  if (grp == 0)
    cross_block_scan<C, OPS, true>(g, rpos, items + (NGB - 1) * SA, xpre, tmp, scr, x.sbuf,
                                   x.sflag, x, 1u);
  __syncthreads();
  block_tree<C, OPS, true>(items, NGB, nv, tmp, scr, g, grp, NGB, false, true,
                           rpos > 0 ? xpre : nullptr);
  __syncthreads();
  // The covariance pass scales its outputs by the quasi-MLE sigma-hat, a sum over every
  // block's filter steps (phase E): wait until all blocks have added their part.  The reverse
  // scan above only orders this block after the blocks later in time.
  if constexpr (WITH_L && !SEG) {
    if (p.calibrate) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(x.barrier, 1u);
      }
      if (grp == 0)
        group_wait(g, x.barrier, x.bar_target, x.status, x.spin_limit, x.where,
                   wait_tag(2u, blk, 0u));
      __syncthreads();
    }
  }
  // G. smoothing down-sweep of every chain from its prefix
  if (chain < p.P)
    smooth_down_chain<C, WITH_L, SEG>(g, p, Es, gs, Ls, items + (nv - 1 - grp) * SA, lin,
                                      lin_out, mean_out, cov_out, scal, chain, scr);
}

template <class C, bool WITH_L>
__global__ void __launch_bounds__(FusedShape<C>::NT, 1)
k_iteration(const IeksParams<typename C::Tp> p,
            const typename TrajType<typename C::Tp>::type* __restrict__ lin,
            typename TrajType<typename C::Tp>::type* __restrict__ lin_out,
            typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
            typename C::Tp* __restrict__ Yv, typename C::Tp* __restrict__ d0,
            typename C::Tp* __restrict__ Es, typename C::Tp* __restrict__ gs,
            typename C::Tp* __restrict__ Ls, typename C::Tp* __restrict__ mean_out,
            typename C::Tp* __restrict__ cov_out, SolveScalars* __restrict__ scal,
            const FusedXchg<typename C::Tp> x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  iteration_body<C, WITH_L, false>(p, blockIdx.x, lin, lin_out, U, R, Yv, d0, Es, gs, Ls,
                                   mean_out, cov_out, scal, x, smem_raw);
}

}  // namespace pit
