// Chain kernels of one IEKS iteration and the block-level/grid-level tree scans.
#pragma once

#include <type_traits>

#include "pit_kernels.cuh"

namespace pit {

constexpr int kThreads = 128;  // threads per block of every chain / tree kernel
// Minimum resident blocks per SM requested for the chain kernels: FP32 groups fit 4 blocks of
// 128 threads (128 registers per thread) with negligible spilling, which measured 15% faster
// than the compiler's unconstrained choice (about 135 registers, 3 blocks) for D = 8.
template <class C>
struct ChainOcc {
  static constexpr int value = (sizeof(typename C::Tp) == 4 && C::D <= 8) ? 4 : 1;
};

template <class C>
__device__ __forceinline__ int64_t chain_index(int grp_in_block) {
  return static_cast<int64_t>(blockIdx.x) * (kThreads / C::G) + grp_in_block;
}

// ---------------------------------------------------------------------------------------------
// Per-step model inputs.  The IEKS solves for the Gauss-Newton increment delta = Y - lin of
// iteration k (lin = the linearisation trajectory, kept in FP64):
//   delta_0 = mu0 - lin_0,   delta_n = Phibar delta_{n-1} + u_{n-1} + w,   u_{n-1} = Phibar lin_{n-1} - lin_n,
//   Htilde_n delta_n = r_n,  r_n = (f(E0 lin_n) - E1 lin_n) / T_1      (scaled preconditioned form)
// which is the linearised model of Section 3.2.1 shifted by lin (its posterior mean is
// m^s - lin).  u, r and y = E0 lin are evaluated once per iteration in extended precision by
// k_residuals; the scans then handle only increment-sized numbers in FP32.
// ---------------------------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ void load_forcing(const typename C::GR& g,
                                             const typename C::Tp* __restrict__ U, int64_t n,
                                             typename C::Tp (&uf)[C::RL]) {
#pragma unroll
  for (int l = 0; l < C::RL; ++l) uf[l] = g.valid(l) ? U[n * C::D + g.row(l)] : typename C::Tp(0);
}

// Raw per-step inputs (loaded one step ahead to hide their latency).  SEG: also the point's
// instance code (instance id, or ~id at the instance's n = 0).  GRID: also the transition scale
// of the step into point n and its h_n / q (non-uniform grids).
template <class C, bool SEG = false, bool GRID = false>
struct StepIn {
  using T = typename C::Tp;
  T y[C::DD];  // solution components of lin_n (original coordinates, for the Jacobian)
  T r[C::DD];  // residual r_n
  T u[C::RL];  // forcing u_{n-1}, this lane's rows
  T sc[C::Q1];  // GRID: T(h_{n-1}) / T(h_n)
  T hq;         // GRID: h_n / q
  int code;
  __device__ __forceinline__ void load(const typename C::GR& g, const IeksParams<T>& p,
                                       const T* __restrict__ Yv, const T* __restrict__ R,
                                       const T* __restrict__ U, int64_t n) {
#pragma unroll
    for (int k = 0; k < C::DD; ++k) {
      y[k] = Yv[n * C::DD + k];
      r[k] = R[n * C::DD + k];
    }
    load_forcing<C>(g, U, n - 1, u);
    code = SEG ? p.seg.inst_of[n] : 0;
    if constexpr (GRID) {
#pragma unroll
      for (int j = 0; j < C::Q1; ++j) sc[j] = p.gst[n * p.SW + C::Q1 + j];
      hq = gp_hq(p, n);
    }
  }
  __device__ __forceinline__ void jacobian(const OdeParams<T>& ode, T hq, int lin_mode,
                                           T (&Ft)[C::DD][C::DD]) const {
    T f[C::DD], F[C::DD][C::DD];
    ode_eval<T, C::DD>(ode, y, f, F);
    approximate_jacobian<T, C::DD>(lin_mode, F);
#pragma unroll
    for (int k = 0; k < C::DD; ++k)
#pragma unroll
      for (int m = 0; m < C::DD; ++m) Ft[k][m] = F[k][m] * hq;
  }
};

// ODE parameters of the instance that owns the current step (segmented solves switch them at
// instance boundaries; single solves use the kernel parameters).
template <class C, bool SEG>
struct StepModel {
  using T = typename C::Tp;
  OdeParams<T> ode;
  T hq;
  int id = -1;
  __device__ __forceinline__ const OdeParams<T>& params(const IeksParams<T>& p) const {
    if constexpr (SEG) return ode; else return p.ode;
  }
  __device__ __forceinline__ T scale(const IeksParams<T>& p) const {
    if constexpr (SEG) return hq; else return p.hq;
  }
  // SEG: make instance `nid` current; returns the previous id (or -1)
  __device__ __forceinline__ void select(const IeksParams<T>& p, int nid) {
    if constexpr (SEG) {
      const InstDesc<T>& d = p.seg.desc[nid];
      ode.kind = p.ode.kind;
      ode.d = p.ode.d;
#pragma unroll
      for (int j = 0; j < kMaxInstParams; ++j) ode.p[j] = d.p[j];
      hq = d.hq;
      id = nid;
    }
  }
};

// Initial increment delta_0 of the instance that starts at global point 0.
template <class C, bool SEG>
__device__ __forceinline__ const typename C::Tp* first_d0(const IeksParams<typename C::Tp>& p,
                                                          const typename C::Tp* d0) {
  if constexpr (SEG) return d0 + static_cast<int64_t>(seg_id(p.seg.inst_of[0])) * C::D;
  else return d0;
}

#ifndef PIT_JBATCH
#define PIT_JBATCH 4
#endif
constexpr int kJBatch = PIT_JBATCH;  // leaves whose information rows are folded into sqrtJ at once

// ---------------------------------------------------------------------------------------------
// Filter reduce: chain c folds its leaves n = cL+1 .. min(cL+L, N) into the aggregate
// a_{cL+1} (x)_f ... (x)_f a_{end}; chain 0 starts from the initial state (A = 0, b = delta_0,
// C = 0), the others from the neutral element.  Output: one filter item per chain, with C and J
// lower-triangular.
// ---------------------------------------------------------------------------------------------
template <class C, bool SEG = false, bool GRID = false>
__device__ __forceinline__ void filter_reduce_chain(
    const typename C::GR& g, const IeksParams<typename C::Tp>& p,
    const typename C::Tp* __restrict__ U, const typename C::Tp* __restrict__ R,
    const typename C::Tp* __restrict__ Yv, const typename C::Tp* __restrict__ d0, int64_t chain,
    typename C::Tp* scr, typename C::Tp* out) {
  using T = typename C::Tp;
  using GR = typename C::GR;
  constexpr int D = C::D, DD = C::DD, W = C::W, RL = C::RL, LDM = C::LDM;
  LaneConst<C> lc;
  lc.init(g, p);
  T phibase[RL][C::Q1];
  if constexpr (GRID) {
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int j = 0; j < C::Q1; ++j) phibase[l][j] = lc.phirow[l][j];
  }

  T A[RL][D], b[RL], sC[RL][W], eta[RL], sJ[1][RL][D];
  const T* d0c = first_d0<C, SEG>(p, d0);
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      A[l][c] = (chain != 0 && c == r) ? T(1) : T(0);
      sJ[0][l][c] = T(0);
    }
#pragma unroll
    for (int c = 0; c < W; ++c) sC[l][c] = T(0);
    b[l] = (chain == 0 && r < D) ? d0c[r] : T(0);
    eta[l] = T(0);
  }
  StepModel<C, SEG> mdl;
  // information rows G^T of the last kJBatch leaves, folded into sqrtJ by one structured LQ
  T Gbuf[1][RL][kJBatch * DD];
#pragma unroll
  for (int l = 0; l < RL; ++l)
#pragma unroll
    for (int j = 0; j < kJBatch * DD; ++j) Gbuf[0][l][j] = T(0);
  int nbuf = 0;
  const int64_t n0 = chain * p.L + 1;
  const int64_t n1 = min(chain * p.L + p.L, p.N);
  StepIn<C, SEG, GRID> cur, nxt;
  if (n0 <= n1) cur.load(g, p, Yv, R, U, n0);
  for (int64_t n = n0; n <= n1; ++n) {
    if (n + 1 <= n1) nxt.load(g, p, Yv, R, U, n + 1);
    if constexpr (SEG) {
      if (cur.code < 0) {
        // first point of an instance: the reset element (A = 0, b = delta_0, C = 0); the
        // information part is dropped too, since no later value depends on it
        const T* d0i = d0 + static_cast<int64_t>(~cur.code) * D;
#pragma unroll
        for (int l = 0; l < RL; ++l) {
          const int r = g.row(l);
#pragma unroll
          for (int c = 0; c < D; ++c) {
            A[l][c] = T(0);
            sJ[0][l][c] = T(0);
          }
#pragma unroll
          for (int c = 0; c < W; ++c) sC[l][c] = T(0);
#pragma unroll
          for (int j = 0; j < kJBatch * DD; ++j) Gbuf[0][l][j] = T(0);
          b[l] = (r < D) ? d0i[r] : T(0);
          eta[l] = T(0);
        }
        nbuf = 0;
        cur = nxt;
        continue;
      }
      if (cur.code != mdl.id) mdl.select(p, cur.code);
    }
    T Ft[DD][DD], rr[DD], uf[RL];
    if constexpr (GRID) lc.scale_step(phibase, cur.sc);
    cur.jacobian(mdl.params(p), GRID ? cur.hq : mdl.scale(p), p.lin_mode, Ft);
#pragma unroll
    for (int k = 0; k < DD; ++k) rr[k] = cur.r[k];
#pragma unroll
    for (int l = 0; l < RL; ++l) uf[l] = cur.u[l];
    // predict the conditional filter: A' = Phi A, b' = Phi b + u, C- = tria([sqrtQ | Phi sqrtC])
    publish<GR, D, LDM>(g, A, scr + C::MAT0);
    publish<GR, W, LDM>(g, sC, scr + C::MAT1);
    publish_vec(g, b, scr + C::VEC0);
    g.sync();
    T Ap[RL][D], bp[RL], tri[1][RL][D], ext[1][RL][W];
    phi_rows<C, D>(lc, scr + C::MAT0, Ap);
    phi_rows<C, W>(lc, scr + C::MAT1, ext[0]);
    phi_vec<C>(lc, scr + C::VEC0, bp);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      bp[l] += uf[l];
#pragma unroll
      for (int c = 0; c < D; ++c) tri[0][l][c] = lc.sqrow[l][c];
    }
    g.sync();
    lq_tri_ext<GR, 1, W>(g, tri, ext, scr + C::PIV);
    // update with the linearised observation
    publish<GR, D, LDM>(g, tri[0], scr + C::MAT0);
    publish<GR, D, LDM>(g, Ap, scr + C::MAT1);
    publish_vec(g, bp, scr + C::VEC0);
    g.sync();
    T HA[DD][D];
#pragma unroll
    for (int kk = 0; kk < DD; ++kk)
#pragma unroll
      for (int c = 0; c < D; ++c) HA[kk][c] = hrow_entry<C>(scr + C::MAT1, Ft, kk, c);
    T HAcol[RL][DD];
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const int r = g.valid(l) ? g.row(l) : 0;
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) HAcol[l][kk] = hrow_entry<C>(scr + C::MAT1, Ft, kk, r);
    }
    UpdateOut<C> u;
    sqrt_update<C>(g, scr, tri[0], Ft, rr, sC, u);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      T acc = bp[l];
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) acc += u.K[l][kk] * u.nu[kk];
      b[l] = acc;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        T a = Ap[l][c];
#pragma unroll
        for (int kk = 0; kk < DD; ++kk) a -= u.K[l][kk] * HA[kk][c];
        A[l][c] = a;
      }
    }
    // information part: G = sqrtS^-1 Htilde A';  J += G^T G (square root), eta += G^T sqrtS^-1 nu
    T znu[DD];
    solve_sS<C>(u.sS, u.rS, u.nu, znu);
    T Gt[1][RL][DD];
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      T z[DD];
      solve_sS<C>(u.sS, u.rS, HAcol[l], z);
      T acc = eta[l];
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) {
        Gt[0][l][kk] = g.valid(l) ? z[kk] : T(0);
        acc += z[kk] * znu[kk];
      }
      eta[l] = acc;
    }
    // shift the batch left by one leaf and append this leaf's rows
#pragma unroll
    for (int l = 0; l < RL; ++l) {
#pragma unroll
      for (int j = 0; j < (kJBatch - 1) * DD; ++j) Gbuf[0][l][j] = Gbuf[0][l][j + DD];
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) Gbuf[0][l][(kJBatch - 1) * DD + kk] = Gt[0][l][kk];
    }
    if (++nbuf == kJBatch || n == n1) {
      lq_tri_ext<GR, 1, kJBatch * DD>(g, sJ, Gbuf, scr + C::PIV);
#pragma unroll
      for (int l = 0; l < RL; ++l)
#pragma unroll
        for (int j = 0; j < kJBatch * DD; ++j) Gbuf[0][l][j] = T(0);
      nbuf = 0;
    }
    cur = nxt;
  }
  // triangularise sqrtC (D x W -> D x D lower) and write the chain item
  T Cfull[1][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l)
#pragma unroll
    for (int c = 0; c < D; ++c) Cfull[0][l][c] = (c < W) ? sC[l][c] : T(0);
  lq_dense<GR, 1, D, 0, D, 0>(g, Cfull, scr + C::PIV);
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      out[C::F_A + r * D + c] = A[l][c];
      out[C::F_C + r * D + c] = Cfull[0][l][c];
      out[C::F_J + r * D + c] = sJ[0][l][c];
    }
    out[C::F_B + r] = b[l];
    out[C::F_ETA + r] = eta[l];
  }
  g.sync();
}

template <class C, bool SEG = false, bool GRID = false>
__global__ void __launch_bounds__(kThreads, ChainOcc<C>::value)
k_filter_reduce(const IeksParams<typename C::Tp> p, const typename C::Tp* __restrict__ U,
                const typename C::Tp* __restrict__ R, const typename C::Tp* __restrict__ Yv,
                const typename C::Tp* __restrict__ d0, typename C::Tp* __restrict__ agg) {
  using T = typename C::Tp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t chain = chain_index<C>(grp);
  if (chain >= p.P) return;
  filter_reduce_chain<C, SEG, GRID>(g, p, U, R, Yv, d0, chain, smem + grp * C::SCR,
                                    agg + chain * C::FA);
}

// ---------------------------------------------------------------------------------------------
// Filter down-sweep: chain c starts from the filtering marginal at n = cL (its exclusive
// prefix, or the initial state for c = 0) and runs square-root Kalman steps over its leaves.
// Step n also forms the smoothing element b_{n-1} from the Pi-triangularisation of Eq.
// sqrt-smoothing-elements (whose top block is the prediction of step n) and folds it into the
// chain's smoothing aggregate.  The chain owning n = N also emits b_N = (0, m^f_N, sqrtP^f_N).
// Accumulates the calibration sum sum_n ||sqrtS_n^-1 nu_n||^2 in FP64.
// LOCAL_LIN: the sequential EKS; linearise at the predicted mean (plain model, no increment).
// ---------------------------------------------------------------------------------------------
template <class C, bool WITH_L, bool LOCAL_LIN, bool SEG = false, bool GRID = false>
__device__ __forceinline__ void filter_down_chain(
    const typename C::GR& g, const IeksParams<typename C::Tp>& p,
    const typename C::Tp* __restrict__ U, const typename C::Tp* __restrict__ R,
    const typename C::Tp* __restrict__ Yv, const typename C::Tp* __restrict__ d0,
    const typename C::Tp* pre, typename C::Tp* __restrict__ Es, typename C::Tp* __restrict__ gs,
    typename C::Tp* __restrict__ Ls, typename C::Tp* sout, SolveScalars* __restrict__ scal,
    int64_t chain, typename C::Tp* scr) {
  using T = typename C::Tp;
  using GR = typename C::GR;
  constexpr int D = C::D, DD = C::DD, W = C::W, RL = C::RL, LDM = C::LDM;
  static_assert(!(GRID && LOCAL_LIN), "the sequential EKS runs on uniform grids");
  LaneConst<C> lc;
  lc.init(g, p);
  T phibase[RL][C::Q1];
  if constexpr (GRID) {
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int j = 0; j < C::Q1; ++j) phibase[l][j] = lc.phirow[l][j];
  }

  // filter state (m, sqrtP) with sqrtP kept D wide (zero-padded)
  T m[RL], sP[RL][D];
  {
    const T* d0c = first_d0<C, SEG>(p, d0);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const int r = g.valid(l) ? g.row(l) : 0;
      const bool v = g.valid(l);
      if (chain == 0) {
        m[l] = v ? (LOCAL_LIN ? p.mu0[r] : d0c[r]) : T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) sP[l][c] = T(0);
      } else {
        m[l] = v ? pre[C::F_B + r] : T(0);
#pragma unroll
        for (int c = 0; c < D; ++c) sP[l][c] = v ? pre[C::F_C + r * D + c] : T(0);
      }
    }
  }
  // smoothing aggregate (E~, x, L~), starts neutral
  T Ea[RL][D], xa[RL], La[1][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      Ea[l][c] = (c == r) ? T(1) : T(0);
      La[0][l][c] = T(0);
    }
    xa[l] = T(0);
  }
  double s2acc = 0.0;
  bool closed = false;  // the smoothing aggregate holds a segment's last element (E = 0)
  StepModel<C, SEG> mdl;
  // calibration sum of the current instance (segmented) or of the solve
  auto flush_s2 = [&]() {
    if (g.gl == 0 && s2acc != 0.0) {
      if constexpr (SEG) atomicAdd(&p.seg.acc[mdl.id].sigma2_sum, s2acc);
      else atomicAdd(&scal->sigma2_sum, s2acc);
    }
    s2acc = 0.0;
  };

  // fold one smoothing element (rows e, entry gg, rows lrow) into the chain aggregate and store it
  auto emit = [&](int64_t idx, const T (&e)[RL][D], const T (&gg)[RL], const T (&lrow)[RL][D]) {
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      if (!g.valid(l)) continue;
      const int r = g.row(l);
#pragma unroll
      for (int c = 0; c < D; ++c) Es[idx * D * D + r * D + c] = e[l][c];
      gs[idx * D + r] = gg[l];
      if constexpr (WITH_L) {
#pragma unroll
        for (int c = 0; c < D; ++c) Ls[idx * D * D + r * D + c] = lrow[l][c];
      }
    }
    // after a segment's last element the aggregate is final (its E is 0): later elements,
    // which belong to the next segment, are not folded in
    if (closed) return;
    g.sync();
    publish<GR, D, LDM>(g, e, scr + C::MAT2);
    publish_vec(g, gg, scr + C::VEC2);
    if constexpr (WITH_L) publish<GR, D, LDM>(g, lrow, scr + C::MAT1);
    g.sync();
    T Enew[RL][D], ext[1][RL][D];
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      T acc = xa[l];
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Ea[l][k] * scr[C::VEC2 + k];
      xa[l] = acc;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          a1 += Ea[l][k] * scr[C::MAT2 + k * LDM + c];
          if constexpr (WITH_L) a2 += Ea[l][k] * scr[C::MAT1 + k * LDM + c];
        }
        Enew[l][c] = a1;
        ext[0][l][c] = g.valid(l) ? a2 : T(0);
      }
    }
    g.sync();
    if constexpr (WITH_L) lq_tri_ext<GR, 1, D>(g, La, ext, scr + C::PIV);
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) Ea[l][c] = Enew[l][c];
  };

  // the last smoothing element of a segment: b_N = (E = 0, g = m^f_N, sqrtL = tria(sqrtP^f_N))
  auto emit_end = [&](int64_t idx) {
    T e[RL][D], lrow[RL][D];
    T Rm[1][RL][D];
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) {
        e[l][c] = T(0);
        Rm[0][l][c] = sP[l][c];
      }
    if constexpr (WITH_L) lq_dense<GR, 1, D, 0, D, 0>(g, Rm, scr + C::PIV);
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) lrow[l][c] = WITH_L ? Rm[0][l][c] : T(0);
    T gg[RL];
#pragma unroll
    for (int l = 0; l < RL; ++l) gg[l] = g.valid(l) ? m[l] : T(0);
    emit(idx, e, gg, lrow);
    closed = true;
  };

  const int64_t n0 = chain * p.L + 1;
  const int64_t n1 = min(chain * p.L + p.L, p.N);
  StepIn<C, SEG, GRID> cur, nxt;
  if (!LOCAL_LIN && n0 <= n1) cur.load(g, p, Yv, R, U, n0);
  // One Kalman step n.  NE = number of columns of sqrtP in use: D for a prefix that comes from
  // the tree (a full triangular factor), W = D - d after any update (rank D - d).
  auto step = [&](auto ne_tag, int64_t n) {
    constexpr int NE = decltype(ne_tag)::value;
    if constexpr (!LOCAL_LIN) {
      if (n + 1 <= n1) nxt.load(g, p, Yv, R, U, n + 1);
    }
    if constexpr (SEG) {
      if (cur.code < 0) {
        // first point of an instance: close the previous instance with its last smoothing
        // element and restart the filter from the reset element (delta_0, zero covariance)
        emit_end(n - 1);
        const T* d0i = d0 + static_cast<int64_t>(~cur.code) * D;
#pragma unroll
        for (int l = 0; l < RL; ++l) {
          m[l] = g.valid(l) ? d0i[g.row(l)] : T(0);
#pragma unroll
          for (int cc = 0; cc < D; ++cc) sP[l][cc] = T(0);
        }
        cur = nxt;
        return;
      }
      if (cur.code != mdl.id) {
        flush_s2();
        mdl.select(p, cur.code);
      }
    }
    T Ft[DD][DD], rr[DD], uf[RL];
    if constexpr (GRID) lc.scale_step(phibase, cur.sc);
    if constexpr (!LOCAL_LIN) {
      cur.jacobian(mdl.params(p), GRID ? cur.hq : mdl.scale(p), p.lin_mode, Ft);
#pragma unroll
      for (int k = 0; k < DD; ++k) rr[k] = cur.r[k];
#pragma unroll
      for (int l = 0; l < RL; ++l) uf[l] = cur.u[l];
    } else {
#pragma unroll
      for (int l = 0; l < RL; ++l) uf[l] = T(0);
    }
    publish_cols<GR, NE, LDM>(g, sP, scr + C::MAT0);
    publish_vec(g, m, scr + C::VEC0);
    g.sync();
    // Pi input: top rows [sqrtQ | Phi sqrtP], bottom rows [0 | sqrtP]
    T tri[2][RL][D], ext[2][RL][NE], mp[RL];
    phi_rows<C, NE>(lc, scr + C::MAT0, ext[0]);
    phi_vec<C>(lc, scr + C::VEC0, mp);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      mp[l] += uf[l];
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        tri[0][l][cc] = lc.sqrow[l][cc];
        tri[1][l][cc] = T(0);
      }
#pragma unroll
      for (int cc = 0; cc < NE; ++cc) ext[1][l][cc] = sP[l][cc];
    }
    g.sync();
    lq_tri_ext<GR, 2, NE>(g, tri, ext, scr + C::PIV);
    // Pi11 = tri[0] (= predicted factor of step n), Pi21 = tri[1], remainder ext[1]
    publish<GR, D, LDM>(g, tri[0], scr + C::MAT0);
    publish_vec(g, mp, scr + C::VEC0);
    g.sync();
    // smoothing element n-1: E = Pi21 Pi11^-1, g = m^f - E m-
    T e[RL][D], gg[RL], lrow[RL][D];
    T rinv[D];
    inv_diag<D, LDM>(scr + C::MAT0, rinv);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      solve_xL<D, LDM>(scr + C::MAT0, rinv, tri[1][l], e[l]);
      const T acc = m[l] - sum4<T, D>([&](int cc) { return e[l][cc] * scr[C::VEC0 + cc]; });
      gg[l] = g.valid(l) ? acc : T(0);
#pragma unroll
      for (int cc = 0; cc < D; ++cc) {
        if (!g.valid(l)) e[l][cc] = T(0);
        lrow[l][cc] = T(0);
      }
    }
    if constexpr (WITH_L) {
      // sqrtL = Pi22 = tria(remainder)
      T Rm[1][RL][D];
#pragma unroll
      for (int l = 0; l < RL; ++l)
#pragma unroll
        for (int cc = 0; cc < D; ++cc) Rm[0][l][cc] = (cc < NE) ? ext[1][l][cc < NE ? cc : 0] : T(0);
      lq_dense<GR, 1, D, 0, D, 0>(g, Rm, scr + C::PIV);
#pragma unroll
      for (int l = 0; l < RL; ++l)
#pragma unroll
        for (int cc = 0; cc < D; ++cc) lrow[l][cc] = Rm[0][l][cc];
    }
    emit(n - 1, e, gg, lrow);
    if constexpr (LOCAL_LIN) {
      // sequential EKS: linearise at the predicted mean m-_n (published at VEC0)
      T y[DD];
#pragma unroll
      for (int k = 0; k < DD; ++k) y[k] = p.T0 * scr[C::VEC0 + k * C::Q1];
      linearize_y<C>(p, y, Ft, rr);
    }
    // Kalman update of step n (Pi11 is still published at MAT0, m- at VEC0)
    T sPn[RL][W];
    UpdateOut<C> u;
    sqrt_update<C>(g, scr, tri[0], Ft, rr, sPn, u);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      T acc = mp[l];
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) acc += u.K[l][kk] * u.nu[kk];
      m[l] = acc;
#pragma unroll
      for (int cc = 0; cc < D; ++cc) sP[l][cc] = (cc < W) ? sPn[l][cc < W ? cc : 0] : T(0);
    }
    if (p.want_sigma && g.gl == 0) {
      T z[DD];
      solve_sS<C>(u.sS, u.rS, u.nu, z);
      double s = 0.0;
#pragma unroll
      for (int kk = 0; kk < DD; ++kk) s += static_cast<double>(z[kk]) * static_cast<double>(z[kk]);
      s2acc += s;
    }
    if constexpr (!LOCAL_LIN) cur = nxt;
  };
  int64_t n = n0;
  if (chain != 0 && n <= n1) {
    step(std::integral_constant<int, D>{}, n);
    ++n;
  }
  for (; n <= n1; ++n) step(std::integral_constant<int, W>{}, n);
  // the chain owning n = N emits b_N
  if (chain == p.N / p.L) emit_end(p.N);
  // write the chain's smoothing aggregate
  T* out = sout;
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      out[C::S_E + r * D + c] = Ea[l][c];
      out[C::S_L + r * D + c] = WITH_L ? La[0][l][c] : T(0);
    }
    out[C::S_G + r] = xa[l];
  }
  flush_s2();
  g.sync();
}

template <class C, bool WITH_L, bool LOCAL_LIN, bool SEG = false, bool GRID = false>
__global__ void __launch_bounds__(kThreads, ChainOcc<C>::value)
k_filter_down(const IeksParams<typename C::Tp> p, const typename C::Tp* __restrict__ U,
              const typename C::Tp* __restrict__ R, const typename C::Tp* __restrict__ Yv,
              const typename C::Tp* __restrict__ d0,
              const typename C::Tp* __restrict__ fprefix, typename C::Tp* __restrict__ Es,
              typename C::Tp* __restrict__ gs, typename C::Tp* __restrict__ Ls,
              typename C::Tp* __restrict__ sagg, SolveScalars* __restrict__ scal) {
  using T = typename C::Tp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t chain = chain_index<C>(grp);
  if (chain >= p.P) return;
  filter_down_chain<C, WITH_L, LOCAL_LIN, SEG, GRID>(g, p, U, R, Yv, d0, fprefix + chain * C::FA, Es,
                                               gs, Ls, sagg + chain * C::SA, scal, chain,
                                               smem + grp * C::SCR);
}

// ---------------------------------------------------------------------------------------------
// Smoothing down-sweep: chain c starts from the smoothing mean at its right end (the reverse
// exclusive prefix, or nothing for the chain holding n = N) and walks its elements backwards:
//   delta^s_n = E_n delta^s_{n+1} + g_n,   sqrtP^s_n = tria([sqrtL_n | E_n sqrtP^s_{n+1}])
// Means passes write lin_new = lin + delta^s and reduce max|change of y| = max|T_0 delta^s_0|;
// the covariance pass writes the outputs in original coordinates.  lin == nullptr means a zero
// trajectory (the sequential EKS).
// ---------------------------------------------------------------------------------------------
template <class C, bool WITH_L, bool SEG = false, bool GRID = false>
__device__ __forceinline__ void smooth_down_chain(
    const typename C::GR& g, const IeksParams<typename C::Tp>& p,
    const typename C::Tp* __restrict__ Es, const typename C::Tp* __restrict__ gs,
    const typename C::Tp* __restrict__ Ls, const typename C::Tp* pre,
    const typename TrajType<typename C::Tp>::type* __restrict__ lin,
    typename TrajType<typename C::Tp>::type* __restrict__ lin_new,
    typename C::Tp* __restrict__ mean_out, typename C::Tp* __restrict__ cov_out,
    SolveScalars* __restrict__ scal, int64_t chain, typename C::Tp* scr) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  using GR = typename C::GR;
  constexpr int D = C::D, RL = C::RL, LDM = C::LDM;
  int rr[RL];
  bool vv[RL];
  T Trow[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    vv[l] = g.valid(l);
    rr[l] = vv[l] ? g.row(l) : 0;
    Trow[l] = p.Tdiag[rr[l] % C::Q1];
  }
  const bool last = (chain == p.N / p.L);
  T m[RL], sPs[RL][D];
  {
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      m[l] = (!last && vv[l]) ? pre[C::S_G + rr[l]] : T(0);
#pragma unroll
      for (int c = 0; c < D; ++c)
        sPs[l][c] = (WITH_L && !last && vv[l]) ? pre[C::S_L + rr[l] * D + c] : T(0);
    }
  }
  T dmax = T(0), ymax = T(0);
  bool bad = false;
  // quasi-MLE diffusion of this (final) pass: sigma^2 = sum / (N d)
  T sigma = static_cast<T>(
      (!SEG && WITH_L && p.calibrate) ? sqrt(__ldcg(&scal->sigma2_sum) / (static_cast<double>(p.N) * C::DD))
                                      : 1.0);
  T T0 = p.T0;
  // segmented: the instance being written (outputs, scalings, reductions) ...
  int sid = -1;
  int64_t soff = 0;
  V* snew = lin_new;
  T* smean = mean_out;
  T* scov = cov_out;
  int64_t mld = D, cld = D * D, crld = D;  // output strides (point, point, row)
  // ... and the instance being loaded (one step ahead)
  int lid = -1;
  int64_t loff = 0;
  const V* lbase = lin;
  // reduce the change statistics over the group: one atomic per group and instance
  auto flush = [&]() {
    if constexpr (!WITH_L) {
#pragma unroll
      for (int o = C::G / 2; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(g.mask, dmax, o));
        ymax = fmax(ymax, __shfl_xor_sync(g.mask, ymax, o));
      }
      const unsigned anybad = __any_sync(g.mask, bad);
      if (g.gl == 0) {
        double* dm = SEG ? &p.seg.acc[sid].delta_max : &scal->delta_max;
        double* ym = SEG ? &p.seg.acc[sid].y_max : &scal->y_max;
        unsigned* fl = SEG ? &p.seg.acc[sid].flags : &scal->flags;
        if (anybad) atomicOr(fl, 1u);
        atomic_max_nonneg(dm, static_cast<double>(dmax));
        atomic_max_nonneg(ym, static_cast<double>(ymax));
      }
      dmax = T(0);
      ymax = T(0);
      bad = false;
    }
  };
  const int64_t s0 = chain * p.L;
  const int64_t s1 = min(chain * p.L + p.L - 1, p.N);
  // E row, g entry and trajectory entry of step n for this lane's rows (prefetched one step
  // ahead: the walk is a dependent chain, the loads are not)
  auto load = [&](int64_t n, T (&E_)[RL][D], T (&g_)[RL], V (&l_)[RL], int& id_, int& code_) {
    int64_t ln = n;
    if constexpr (SEG) {
      code_ = p.seg.inst_of[n];
      id_ = seg_id(code_);
      if (id_ != lid) {
        const InstDesc<T>& d = p.seg.desc[id_];
        lid = id_;
        loff = d.off;
        lbase = static_cast<const V*>(d.lin[d.cur]);
      }
      ln = n - loff;
    }
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const T* Er = Es + n * D * D + rr[l] * D;
#pragma unroll
      for (int k = 0; k < D; ++k) E_[l][k] = Er[k];
      g_[l] = gs[n * D + rr[l]];
      l_[l] = lbase ? lbase[ln * D + rr[l]] : v_from_zero<V>();
    }
  };
  T Ec[RL][D], gc[RL];
  V lc[RL];
  int ic = 0, cc_ = 0;
  if (s1 >= s0) load(s1, Ec, gc, lc, ic, cc_);
  // segmented: the point after n starts another instance (or n = N), so n is a segment's last
  // point with E_n = 0; its successor state is taken as exactly zero (E_n m = 0 for finite m,
  // and another instance's non-finite values stay out)
  bool succ_start = SEG && (s1 == p.N || p.seg.inst_of[s1 + 1 <= p.N ? s1 + 1 : s1] < 0);
  for (int64_t n = s1; n >= s0; --n) {
    T En[RL][D], gn[RL];
    V ln_[RL];
    int in_ = 0, cn_ = 0;
    if (n - 1 >= s0) load(n - 1, En, gn, ln_, in_, cn_);
    if constexpr (SEG) {
      if (succ_start) {
#pragma unroll
        for (int l = 0; l < RL; ++l) {
          m[l] = T(0);
#pragma unroll
          for (int c = 0; c < D; ++c) sPs[l][c] = T(0);
        }
      }
      succ_start = cc_ < 0;
      if (ic != sid) {
        if (sid >= 0) flush();
        const InstDesc<T>& d = p.seg.desc[ic];
        sid = ic;
        soff = d.off;
        snew = static_cast<V*>(d.lin[1 - d.cur]);
        smean = d.mean;
        scov = d.cov;
        mld = d.mean_ld;
        cld = d.cov_ld;
        crld = d.cov_rld;
        T0 = d.T0;
#pragma unroll
        for (int l = 0; l < RL; ++l) Trow[l] = d.Tdiag[rr[l] % C::Q1];
        if constexpr (WITH_L) {
          double s2 = 1.0;
          if (p.calibrate) {
            if (p.sigma_pool > 0) {
              double tot = 0.0;
              for (int j = 0; j < p.sigma_pool; ++j) tot += p.seg.acc[j].sigma2_sum;
              s2 = tot / (static_cast<double>(d.N) * p.sigma_pool * C::DD);
            } else {
              s2 = p.seg.acc[ic].sigma2_sum / (static_cast<double>(d.N) * C::DD);
            }
          }
          sigma = static_cast<T>(sqrt(s2));
        }
      }
    }
    if constexpr (GRID) {
      // per-point preconditioner of a non-uniform grid
#pragma unroll
      for (int l = 0; l < RL; ++l) Trow[l] = gp_T(p, n, rr[l] % C::Q1);
      T0 = gp_T0(p, n);
    }
    const int64_t on = SEG ? n - soff : n;  // index within the output arrays
    publish_vec(g, m, scr + C::VEC0);
    if constexpr (WITH_L) publish<GR, D, LDM>(g, sPs, scr + C::MAT0);
    g.sync();
    T mn[RL];
    T tri[1][RL][D], ext[1][RL][D];
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const T acc = gc[l] + sum4<T, D>([&](int k) { return Ec[l][k] * scr[C::VEC0 + k]; });
      mn[l] = vv[l] ? acc : T(0);
      if constexpr (WITH_L) {
        const T* Lr = Ls + n * D * D + rr[l] * D;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const T a2 = sum4<T, D>([&](int k) { return Ec[l][k] * scr[C::MAT0 + k * LDM + c]; });
          ext[0][l][c] = vv[l] ? a2 : T(0);
          tri[0][l][c] = vv[l] ? Lr[c] : T(0);
        }
      }
    }
    g.sync();
    if constexpr (WITH_L) {
      lq_tri_ext<GR, 1, D>(g, tri, ext, scr + C::PIV);
#pragma unroll
      for (int l = 0; l < RL; ++l)
#pragma unroll
        for (int c = 0; c < D; ++c) sPs[l][c] = tri[0][l][c];
    }
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      m[l] = mn[l];
      if (!vv[l]) continue;
      const int r = rr[l];
      const V lnew = v_add_small(lc[l], mn[l]);
      if constexpr (WITH_L) {
        smean[on * mld + r] = Trow[l] * v_to_T<T>(lnew);
#pragma unroll
        for (int c = 0; c < D; ++c) scov[on * cld + r * crld + c] = sigma * Trow[l] * sPs[l][c];
      } else {
        snew[on * D + r] = lnew;
        if (r % C::Q1 == 0) {
          const T dd = fabs(T0 * mn[l]);
          bad = bad || !(dd == dd);
          dmax = fmax(dmax, dd);
          ymax = fmax(ymax, fabs(T0 * v_to_T<T>(lnew)));
        }
      }
    }
#pragma unroll
    for (int l = 0; l < RL; ++l) {
#pragma unroll
      for (int k = 0; k < D; ++k) Ec[l][k] = En[l][k];
      gc[l] = gn[l];
      lc[l] = ln_[l];
    }
    ic = in_;
    cc_ = cn_;
  }
  // groups past the last chain have returned; every lane of a live group reaches here
  if (!SEG || sid >= 0) flush();
  g.sync();
}

template <class C, bool WITH_L, bool SEG = false, bool GRID = false>
__global__ void __launch_bounds__(kThreads, ChainOcc<C>::value)
k_smooth_down(const IeksParams<typename C::Tp> p, const typename C::Tp* __restrict__ Es,
              const typename C::Tp* __restrict__ gs, const typename C::Tp* __restrict__ Ls,
              const typename C::Tp* __restrict__ sprefix,
              const typename TrajType<typename C::Tp>::type* __restrict__ lin,
              typename TrajType<typename C::Tp>::type* __restrict__ lin_new,
              typename C::Tp* __restrict__ mean_out, typename C::Tp* __restrict__ cov_out,
              SolveScalars* __restrict__ scal) {
  using T = typename C::Tp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t chain = chain_index<C>(grp);
  if (chain >= p.P) return;
  smooth_down_chain<C, WITH_L, SEG, GRID>(g, p, Es, gs, Ls, sprefix + chain * C::SA, lin, lin_new,
                                    mean_out, cov_out, scal, chain, smem + grp * C::SCR);
}
// ---------------------------------------------------------------------------------------------
// Tree scans over items (filter: FA elements, smoothing: SA elements) in blocks of B items.
// Position p of a level maps to item index p, or to n-1-p when `rev_index` is set (only the
// bottom level of a reverse scan; upper levels hold block totals in position order).  With
// REVERSE the operator's operands are swapped so that the result at item k is
// item_k (x) item_{k+1} (x) ... (the reverse scan of Section 3.1.3).
// ---------------------------------------------------------------------------------------------
template <class C, bool FILTER, bool WITH_L, bool VALUES_DOWN = false>
struct TreeOps {
  using T = typename C::Tp;
  static constexpr int SZ = FILTER ? C::FA : C::SA;
  static __device__ __forceinline__ void identity(const typename C::GR& g, T* x) {
    if constexpr (FILTER) set_identity_f<C>(g, x); else set_identity_s<C>(g, x);
  }
  // out = earlier (x) later   (forward);  out = later (x)_s earlier  in reverse mode.
  // DOWN: a down-sweep combine (prefix (x) left sum).  With VALUES_DOWN the filter down-sweep
  // forms only b and C of the result: every prefix of the IEKS scan starts at the initial
  // state, and b, C of (prefix (x) x) depend on the prefix only through its b, C.
  template <bool REVERSE, bool DOWN = false>
  static __device__ __forceinline__ void op(const typename C::GR& g, const T* earlier,
                                            const T* later, T* out, T* scr) {
    if constexpr (FILTER) {
      combine_f<C, DOWN && VALUES_DOWN>(g, earlier, later, out, scr);
    } else {
      if constexpr (REVERSE) combine_s<C, WITH_L>(g, later, earlier, out, scr);
      else combine_s<C, WITH_L>(g, earlier, later, out, scr);
    }
  }
};

__device__ __forceinline__ int64_t tree_item_index(int64_t n, int64_t pos, bool reverse) {
  return reverse ? (n - 1 - pos) : pos;
}

// Brent-Kung up-sweep over B items in shared memory (`items`), then (DOWN) Blelloch down-sweep
// with `prefix` as the block's exclusive prefix.  ngroups groups of the block take the combines.
// Positions >= nv hold neutral padding: combines whose right operand covers only padding become
// copies, combines of two padding nodes are skipped.
template <class C, class OPS, bool REVERSE>
__device__ void block_tree(typename C::Tp* items, int B, int nv, typename C::Tp* tmp,
                           typename C::Tp* scr, const typename C::GR& g, int grp, int ngroups,
                           bool up, bool down, const typename C::Tp* prefix) {
  using T = typename C::Tp;
  constexpr int SZ = OPS::SZ;
  if (up) {
    for (int stride = 1; stride < B; stride *= 2) {
      const int npairs = B / (2 * stride);
      for (int pr = grp; pr < npairs; pr += ngroups) {
        const int i = (pr + 1) * 2 * stride - 1;
        const int j = i - stride;
        if (j - stride + 1 >= nv) continue;            // both subtrees padding
        if (j + 1 >= nv) {                             // right subtree padding
          copy_item<C, SZ>(g, items + j * SZ, items + i * SZ);
          g.sync();
          continue;
        }
        OPS::template op<REVERSE>(g, items + j * SZ, items + i * SZ, items + i * SZ, scr);
      }
      __syncthreads();
    }
  }
  if (down) {
    if (grp == 0) {
      if (prefix) copy_item<C, SZ>(g, prefix, items + (B - 1) * SZ);
      else OPS::identity(g, items + (B - 1) * SZ);
    }
    __syncthreads();
    for (int stride = B / 2; stride >= 1; stride /= 2) {
      const int npairs = B / (2 * stride);
      for (int pr = grp; pr < npairs; pr += ngroups) {
        const int i = (pr + 1) * 2 * stride - 1;
        const int j = i - stride;
        if (j - stride + 1 >= nv) {                    // left subtree padding: prefix passes
          copy_item<C, SZ>(g, items + i * SZ, items + j * SZ);
          g.sync();
          continue;
        }
        T* tj = tmp;
        copy_item<C, SZ>(g, items + j * SZ, tj);
        g.sync();
        copy_item<C, SZ>(g, items + i * SZ, items + j * SZ);
        g.sync();
        OPS::template op<REVERSE, true>(g, items + j * SZ, tj, items + i * SZ, scr);
      }
      __syncthreads();
    }
  }
}

// Up-sweep kernel: block b loads items [b B, (b+1) B) (identity padding), reduces, writes the
// up-swept block back in place and its total to `totals[b]`.  If `single` (one block covers all
// items) it also runs the down-sweep with the neutral prefix and writes exclusive prefixes.
template <class C, class OPS, bool REVERSE>
__global__ void __launch_bounds__(kThreads)
k_tree_up(typename C::Tp* __restrict__ items, int64_t n, int B,
          typename C::Tp* __restrict__ totals, int single, int rev_index) {
  using T = typename C::Tp;
  constexpr int SZ = OPS::SZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int ngroups = kThreads / C::G;
  T* sitems = sm;
  T* scr = sm + (size_t)B * SZ + grp * (C::SCR + SZ);
  T* tmp = scr + C::SCR;
  const int64_t base = (int64_t)blockIdx.x * B;
  for (int pos = grp; pos < B; pos += ngroups) {
    const int64_t gp = base + pos;
    if (gp < n) copy_item<C, SZ>(g, items + tree_item_index(n, gp, rev_index != 0) * SZ, sitems + pos * SZ);
    else OPS::identity(g, sitems + pos * SZ);
  }
  __syncthreads();
  const int nv = static_cast<int>((n - base) < B ? (n - base) : B);
  block_tree<C, OPS, REVERSE>(sitems, B, nv, tmp, scr, g, grp, ngroups, true, single != 0, nullptr);
  for (int pos = grp; pos < B; pos += ngroups) {
    const int64_t gp = base + pos;
    if (gp < n) copy_item<C, SZ>(g, sitems + pos * SZ, items + tree_item_index(n, gp, rev_index != 0) * SZ);
  }
  if (!single && grp == 0) copy_item<C, SZ>(g, sitems + (B - 1) * SZ, totals + blockIdx.x * SZ);
}

// Down-sweep kernel: block b loads its up-swept items and its exclusive prefix
// `block_prefix[b]`, and writes exclusive prefixes in place.
template <class C, class OPS, bool REVERSE>
__global__ void __launch_bounds__(kThreads)
k_tree_down(typename C::Tp* __restrict__ items, int64_t n, int B,
            const typename C::Tp* __restrict__ block_prefix, int rev_index) {
  using T = typename C::Tp;
  constexpr int SZ = OPS::SZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int ngroups = kThreads / C::G;
  T* sitems = sm;
  T* scr = sm + (size_t)B * SZ + grp * (C::SCR + SZ);
  T* tmp = scr + C::SCR;
  const int64_t base = (int64_t)blockIdx.x * B;
  for (int pos = grp; pos < B; pos += ngroups) {
    const int64_t gp = base + pos;
    if (gp < n) copy_item<C, SZ>(g, items + tree_item_index(n, gp, rev_index != 0) * SZ, sitems + pos * SZ);
    else OPS::identity(g, sitems + pos * SZ);
  }
  __syncthreads();
  const int nv = static_cast<int>((n - base) < B ? (n - base) : B);
  block_tree<C, OPS, REVERSE>(sitems, B, nv, tmp, scr, g, grp, ngroups, false, true,
                              block_prefix + blockIdx.x * SZ);
  for (int pos = grp; pos < B; pos += ngroups) {
    const int64_t gp = base + pos;
    if (gp < n) copy_item<C, SZ>(g, sitems + pos * SZ, items + tree_item_index(n, gp, rev_index != 0) * SZ);
  }
}

}  // namespace pit
