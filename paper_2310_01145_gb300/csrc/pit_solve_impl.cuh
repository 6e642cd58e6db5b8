// Host orchestration of the time-parallel IEKS (Algorithm 2) and of the element scans, templated
// on the configuration.  Included only by the pit_inst_*.cu instantiation files.
#pragma once

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pit_chains.cuh"
#include "pit_fused.cuh"
#include "pit_internal.h"

namespace pit {

// ---- small elementwise kernels ---------------------------------------------------------------
// Initial linearisation trajectory (preconditioned, trajectory number type V): the constant
// mu0 of Algorithm 2, or a caller-provided warm start in original coordinates.
template <class C, bool GRID = false>
__global__ void k_init_traj(const IeksParams<typename C::Tp> p,
                            const typename C::Tp* __restrict__ init,
                            typename TrajType<typename C::Tp>::type* __restrict__ lin) {
  using V = typename TrajType<typename C::Tp>::type;
  const int64_t total = (p.N + 1) * C::D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(i % C::D);
    double x;
    if constexpr (GRID) {
      // original coordinates (mu0 was preconditioned with T(h_0)), then the point's T(h_n)
      const double orig = init ? static_cast<double>(init[i]) : p.mu0d[r] * p.Tdiagd[r % C::Q1];
      x = orig / gp_Td(p, i / C::D, r % C::Q1);
    } else {
      x = init ? static_cast<double>(init[i]) / p.Tdiagd[r % C::Q1] : p.mu0d[r];
    }
    lin[i] = v_from_double<V>(x);
  }
}

// Inputs of the increment model of one iteration, in FP64: u_n = Phibar lin_n - lin_{n+1} (n < N), r_n = f(y_n)/T_1 - xbar_{1,n} (n >= 1)
// with y_n = T_0 xbar_{0,n} (the solution components of lin_n, also stored in T for the
// Jacobian), and delta_0 = mu0 - lin_0.  One thread per time step.  A block takes a tile of
// consecutive steps and stages their trajectory rows (and the row after them) and its outputs
// in shared memory, so that every global load and store is a contiguous run: a thread reading
// its own row of D 8-byte values from global memory would make each warp load touch 32 rows.
// Shared rows use odd strides, which keeps the per-thread row accesses free of bank conflicts;
// the tile is 256 steps, or 128 where that staging would not fit 48 KB.
template <class C>
struct ResTile {
  using T = typename C::Tp;
  static constexpr int SV = C::D | 1, SU = C::D | 1, SR = C::DD | 1;
  static constexpr int lin_bytes(int tile) { return (tile + 1) * SV * 8; }
  static constexpr int u_bytes(int tile) { return tile * SU * static_cast<int>(sizeof(T)); }
  static constexpr int r_bytes(int tile) { return tile * SR * static_cast<int>(sizeof(T)); }
  static constexpr int bytes(int tile) { return lin_bytes(tile) + u_bytes(tile) + 2 * r_bytes(tile); }
  static constexpr int size = bytes(256) <= 48 * 1024 ? 256 : 128;
};


template <class C, bool GRID = false>
__global__ void __launch_bounds__(ResTile<C>::size)
k_residuals(const IeksParams<typename C::Tp> p,
            const typename TrajType<typename C::Tp>::type* __restrict__ lin,
            typename C::Tp* __restrict__ U, typename C::Tp* __restrict__ R,
            typename C::Tp* __restrict__ Yv, typename C::Tp* __restrict__ d0) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  using RT = ResTile<C>;
  static_assert(sizeof(V) == sizeof(uint2), "trajectory values are 8 bytes");
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  constexpr int TILE = RT::size, SV = RT::SV, SU = RT::SU, SR = RT::SR;
  __shared__ __align__(16) unsigned char s_raw[RT::bytes(TILE)];
  uint2* s_lin = reinterpret_cast<uint2*>(s_raw);
  T* s_u = reinterpret_cast<T*>(s_raw + RT::lin_bytes(TILE));
  T* s_r = reinterpret_cast<T*>(s_raw + RT::lin_bytes(TILE) + RT::u_bytes(TILE));
  T* s_y = reinterpret_cast<T*>(s_raw + RT::lin_bytes(TILE) + RT::u_bytes(TILE) + RT::r_bytes(TILE));
  const uint2* lin_w = reinterpret_cast<const uint2*>(lin);

  OdeConstsV<V> oc;
  ode_consts_v<V, T, DD>(p.ode, p.pd, oc);
  const V T0v = v_from_double<V>(p.T0d);
  const V T1iv = v_from_double<V>(p.T1invd);
  const int t = threadIdx.x;
  const int64_t tiles = (p.N + TILE) / TILE;  // ceil((N + 1) / TILE)
  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t n0 = tile * TILE;
    // rows n0 .. n0 + rows - 1 (the last one is the next tile's first when it exists)
    const int64_t left = p.N + 1 - n0;
    const int rows = left < TILE + 1 ? static_cast<int>(left) : TILE + 1;
    const int steps = rows < TILE ? rows : TILE;
    const int usteps = left - 1 < steps ? static_cast<int>(left - 1) : steps;  // steps with u_n
    for (int i = t; i < rows * D; i += TILE) s_lin[(i / D) * SV + i % D] = lin_w[n0 * D + i];
    __syncthreads();
    if (t < steps) {
      V x[D];
#pragma unroll
      for (int r = 0; r < D; ++r) bits_to(s_lin[t * SV + r], x[r]);
      double sc[Q1];  // GRID: scale of the step into point n + 1
#pragma unroll
      for (int i = 0; i < Q1; ++i) sc[i] = (GRID && t < usteps) ? gp_scaled(p, n0 + t + 1, i) : 1.0;
      if (t < usteps) {
#pragma unroll
        for (int k = 0; k < DD; ++k) {
#pragma unroll
          for (int i = 0; i < Q1; ++i) {
            V acc = GRID ? x[k * Q1 + i] * sc[i] : x[k * Q1 + i];
#pragma unroll
            for (int j = i + 1; j < Q1; ++j)
              acc = acc + x[k * Q1 + j] * (GRID ? static_cast<double>(p.phib[i * kMaxQ1 + j]) * sc[j]
                                                : static_cast<double>(p.phib[i * kMaxQ1 + j]));
            V next;
            bits_to(s_lin[(t + 1) * SV + k * Q1 + i], next);
            acc = acc - next;
            s_u[t * SU + k * Q1 + i] = v_to_T<T>(acc);
          }
        }
      }
      V y[DD], f[DD];
      const V t0n = GRID ? v_from_double<V>(gp_T0d(p, n0 + t)) : T0v;
      const V t1n = GRID ? v_from_double<V>(gp_T1invd(p, n0 + t)) : T1iv;
#pragma unroll
      for (int k = 0; k < DD; ++k) y[k] = t0n * x[k * Q1];
      ode_f_v<V, DD>(oc, y, f);
#pragma unroll
      for (int k = 0; k < DD; ++k) {
        s_y[t * SR + k] = v_to_T<T>(y[k]);
        s_r[t * SR + k] = v_to_T<T>(f[k] * t1n - x[k * Q1 + 1]);
      }
      if (n0 + t == 0) {
#pragma unroll
        for (int r = 0; r < D; ++r) d0[r] = v_to_T<T>(v_from_double<V>(p.mu0d[r]) - x[r]);
      }
    }
    __syncthreads();
    for (int i = t; i < usteps * D; i += TILE) U[n0 * D + i] = s_u[(i / D) * SU + i % D];
    for (int i = t; i < steps * DD; i += TILE) {
      const int o = (i / DD) * SR + i % DD;
      R[n0 * DD + i] = s_r[o];
      Yv[n0 * DD + i] = s_y[o];
    }
    __syncthreads();  // the next tile restages the shared buffers
  }
}

// Objective value of a trajectory (Eq. objective-value), V = 1/2 sum_{n=1..N}
// || lin_n - Phi lin_{n-1} ||^2_{Q^-1}.  In preconditioned coordinates Phi, Q become Phibar,
// Qbar and the quadratic form is unchanged, so each dimension block contributes
// || sqrt(Qbar)^-1 (xbar_n - Phibar xbar_{n-1}) ||^2 (differences in the trajectory's number
// type, the triangular solve and the sum in FP64).
template <class C>
__global__ void __launch_bounds__(256)
k_objective(const IeksParams<typename C::Tp> p,
            const typename TrajType<typename C::Tp>::type* __restrict__ lin,
            SolveScalars* __restrict__ scal) {
  using T = typename C::Tp;
  using V = typename TrajType<T>::type;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  double acc = 0.0;
  for (int64_t n = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= p.N;
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
      double z[Q1];
#pragma unroll
      for (int i = 0; i < Q1; ++i) {
        double s = w[i];
#pragma unroll
        for (int j = 0; j < i; ++j) s -= p.sqbd[i * kMaxQ1 + j] * z[j];
        z[i] = s / p.sqbd[i * kMaxQ1 + i];
        acc += z[i] * z[i];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(&scal->objective, 0.5 * acc);
}

// Initial trajectory from a coarse-grid solution (Section 3.2.2, remark on the initial
// trajectory): fine point n takes the coarse smoothing mean at node k = floor(n Nc / N),
// propagated by the prior mean over tau = t_n - t_k, x = Phi(tau) m_k with
// Phi(tau)_ij = tau^(j-i) / (j-i)! per dimension block (original coordinates, FP64), then
// preconditioned.
template <class C>
__global__ void k_coarse_init(const IeksParams<typename C::Tp> p,
                              const typename C::Tp* __restrict__ cm, int64_t Nc, double span,
                              typename TrajType<typename C::Tp>::type* __restrict__ lin) {
  using V = typename TrajType<typename C::Tp>::type;
  constexpr int D = C::D, DD = C::DD, Q1 = C::Q1;
  const double scale = span / (static_cast<double>(p.N) * static_cast<double>(Nc));
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= p.N;
       n += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = (n * Nc) / p.N;
    k = k < Nc ? k : Nc;
    const double tau = static_cast<double>(n * Nc - k * p.N) * scale;
    double pw[Q1];  // tau^m / m!
    pw[0] = 1.0;
#pragma unroll
    for (int m = 1; m < Q1; ++m) pw[m] = pw[m - 1] * tau / static_cast<double>(m);
#pragma unroll
    for (int b = 0; b < DD; ++b) {
#pragma unroll
      for (int i = 0; i < Q1; ++i) {
        double x = 0.0;
#pragma unroll
        for (int j = i; j < Q1; ++j) x += pw[j - i] * static_cast<double>(cm[k * D + b * Q1 + j]);
        lin[n * D + b * Q1 + i] = v_from_double<V>(x / p.Tdiagd[i]);
      }
    }
  }
}

template <class C, bool GRID = false>
__global__ void k_export_mean(const IeksParams<typename C::Tp> p,
                              const typename TrajType<typename C::Tp>::type* __restrict__ lin,
                              typename C::Tp* __restrict__ mean) {
  const int64_t total = (p.N + 1) * C::D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(i % C::D);
    const typename C::Tp tr = GRID ? gp_T(p, i / C::D, r % C::Q1) : p.Tdiag[r % C::Q1];
    mean[i] = tr * v_to_T<typename C::Tp>(lin[i]);
  }
}

// ---- generic element scans (pit_filter_scan / pit_smooth_scan) -------------------------------
template <class C>
__device__ void load_filter_elem(const typename C::GR& g, int64_t n, const typename C::Tp* A,
                                 const typename C::Tp* b, const typename C::Tp* Cm,
                                 const typename C::Tp* eta, const typename C::Tp* J,
                                 typename C::Tp* item, typename C::Tp* scr) {
  using T = typename C::Tp;
  constexpr int D = C::D, RL = C::RL;
  T Cr[1][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const bool v = g.valid(l);
    const int r = v ? g.row(l) : 0;
#pragma unroll
    for (int c = 0; c < D; ++c) Cr[0][l][c] = v ? Cm[(n * D + r) * D + c] : T(0);
  }
  lq_dense<typename C::GR, 1, D, 0, D, 0>(g, Cr, scr + C::PIV);
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      item[C::F_A + r * D + c] = A[(n * D + r) * D + c];
      item[C::F_C + r * D + c] = Cr[0][l][c];
      item[C::F_J + r * D + c] = J[(n * D + r) * D + c];
    }
    item[C::F_B + r] = b[n * D + r];
    item[C::F_ETA + r] = eta[n * D + r];
  }
  g.sync();
}

template <class C>
__global__ void __launch_bounds__(kThreads)
k_gen_filter(int64_t N, int L, int64_t P, typename C::Tp* A, typename C::Tp* b,
             typename C::Tp* Cm, typename C::Tp* eta, typename C::Tp* J,
             typename C::Tp* items, int down) {
  using T = typename C::Tp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t chain = chain_index<C>(grp);
  if (chain >= P) return;
  T* scr = smem + grp * (C::SCR + 2 * C::FA);
  T* acc = scr + C::SCR;
  T* el = acc + C::FA;
  if (down) copy_item<C, C::FA>(g, items + chain * C::FA, acc);
  else set_identity_f<C>(g, acc);
  g.sync();
  const int64_t n0 = chain * L, n1 = min(chain * L + L, N);
  for (int64_t n = n0; n < n1; ++n) {
    load_filter_elem<C>(g, n, A, b, Cm, eta, J, el, scr);
    combine_f<C, false>(g, acc, el, acc, scr);
    if (down) {
      for (int i = g.gl; i < C::D * C::D; i += C::G) {
        A[n * C::D * C::D + i] = acc[C::F_A + i];
        Cm[n * C::D * C::D + i] = acc[C::F_C + i];
        J[n * C::D * C::D + i] = acc[C::F_J + i];
      }
      for (int i = g.gl; i < C::D; i += C::G) {
        b[n * C::D + i] = acc[C::F_B + i];
        eta[n * C::D + i] = acc[C::F_ETA + i];
      }
      g.sync();
    }
  }
  if (!down) copy_item<C, C::FA>(g, acc, items + chain * C::FA);
}

template <class C, bool WITH_L>
__global__ void __launch_bounds__(kThreads)
k_gen_smooth(int64_t N, int L, int64_t P, typename C::Tp* E, typename C::Tp* gv,
             typename C::Tp* Lm, typename C::Tp* items, int down) {
  using T = typename C::Tp;
  constexpr int D = C::D, RL = C::RL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  typename C::GR g;
  g.init();
  const int grp = threadIdx.x / C::G;
  const int64_t chain = chain_index<C>(grp);
  if (chain >= P) return;
  T* scr = smem + grp * (C::SCR + 2 * C::SA);
  T* acc = scr + C::SCR;
  T* el = acc + C::SA;
  if (down) copy_item<C, C::SA>(g, items + chain * C::SA, acc);
  else set_identity_s<C>(g, acc);
  g.sync();
  const int64_t n0 = chain * L, n1 = min(chain * L + L, N);
  auto load = [&](int64_t n) {
    T Lr[1][RL][D];
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const bool v = g.valid(l);
      const int r = v ? g.row(l) : 0;
#pragma unroll
      for (int c = 0; c < D; ++c) Lr[0][l][c] = (WITH_L && v) ? Lm[(n * D + r) * D + c] : T(0);
    }
    if constexpr (WITH_L) lq_dense<typename C::GR, 1, D, 0, D, 0>(g, Lr, scr + C::PIV);
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      if (!g.valid(l)) continue;
      const int r = g.row(l);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        el[C::S_E + r * D + c] = E[(n * D + r) * D + c];
        el[C::S_L + r * D + c] = Lr[0][l][c];
      }
      el[C::S_G + r] = gv[n * D + r];
    }
    g.sync();
  };
  if (!down) {
    // forward fold acc = b_n0 (x) ... (x) b_{n1-1}
    for (int64_t n = n0; n < n1; ++n) {
      load(n);
      combine_s<C, WITH_L>(g, acc, el, acc, scr);
    }
    copy_item<C, C::SA>(g, acc, items + chain * C::SA);
  } else {
    for (int64_t n = n1 - 1; n >= n0; --n) {
      load(n);
      combine_s<C, WITH_L>(g, el, acc, acc, scr);
      for (int i = g.gl; i < D * D; i += C::G) {
        E[n * D * D + i] = acc[C::S_E + i];
        if (WITH_L) Lm[n * D * D + i] = acc[C::S_L + i];
      }
      for (int i = g.gl; i < D; i += C::G) gv[n * D + i] = acc[C::S_G + i];
      g.sync();
    }
  }
}

// ---- tree driver -----------------------------------------------------------------------------
template <class C, bool FILTER, bool WITH_L, bool REVERSE, bool VALUES_DOWN = false>
struct Tree {
  using T = typename C::Tp;
  using OPS = TreeOps<C, FILTER, WITH_L, VALUES_DOWN>;
  static constexpr int SZ = OPS::SZ;
  static constexpr int NG = kThreads / C::G;
  static int block_items() {
    int B = 64;
    while (B > 2 && smem_bytes(B) > 200 * 1024) B /= 2;
    return B;
  }
  static size_t smem_bytes(int B) {
    return (static_cast<size_t>(B) * SZ + static_cast<size_t>(NG) * (C::SCR + SZ)) * sizeof(T);
  }
  // element counts of the upper levels for n bottom items
  static std::vector<int64_t> levels(int64_t n, int B) {
    std::vector<int64_t> v;
    int64_t cur = n;
    while (cur > B) {
      cur = (cur + B - 1) / B;
      v.push_back(cur);
    }
    return v;
  }
  static size_t upper_bytes(int64_t n) {
    const int B = block_items();
    size_t tot = 0;
    for (int64_t c : levels(n, B)) tot += ((c * SZ * sizeof(T) + 255) / 256) * 256;
    return tot;
  }
  // Exclusive scan of items[0..n) in place (rev_bottom: bottom level indexed in reverse).
  static int run(T* items, int64_t n, T* upper, bool rev_bottom, cudaStream_t s) {
    const int B = block_items();
    const size_t smem = smem_bytes(B);
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_tree_up<C, OPS, REVERSE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_tree_down<C, OPS, REVERSE>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    std::vector<int64_t> lv = levels(n, B);
    std::vector<T*> arr;
    std::vector<int64_t> cnt;
    arr.push_back(items);
    cnt.push_back(n);
    char* up = reinterpret_cast<char*>(upper);
    for (int64_t c : lv) {
      arr.push_back(reinterpret_cast<T*>(up));
      cnt.push_back(c);
      up += ((c * SZ * sizeof(T) + 255) / 256) * 256;
    }
    const int top = static_cast<int>(arr.size()) - 1;
    for (int lvl = 0; lvl < top; ++lvl) {
      const unsigned grid = static_cast<unsigned>((cnt[lvl] + B - 1) / B);
      PIT_LAUNCH(FILTER ? KC_TREE_FILTER_UP : KC_TREE_SMOOTH_UP, s, 
                 k_tree_up<C, OPS, REVERSE><<<grid, kThreads, smem, s>>>(arr[lvl], cnt[lvl], B,
                                                              arr[lvl + 1], 0,
                                                              (lvl == 0 && rev_bottom) ? 1 : 0););
    }
    PIT_LAUNCH(FILTER ? KC_TREE_FILTER_UP : KC_TREE_SMOOTH_UP, s, 
               k_tree_up<C, OPS, REVERSE><<<1, kThreads, smem, s>>>(arr[top], cnt[top], B, nullptr, 1,
                                                         (top == 0 && rev_bottom) ? 1 : 0););
    for (int lvl = top - 1; lvl >= 0; --lvl) {
      const unsigned grid = static_cast<unsigned>((cnt[lvl] + B - 1) / B);
      PIT_LAUNCH(FILTER ? KC_TREE_FILTER_DOWN : KC_TREE_SMOOTH_DOWN, s, 
                 k_tree_down<C, OPS, REVERSE><<<grid, kThreads, smem, s>>>(
          arr[lvl], cnt[lvl], B, arr[lvl + 1], (lvl == 0 && rev_bottom) ? 1 : 0););
    }
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }
};

// ---- the solver ------------------------------------------------------------------------------
// C: layout of the chain kernels; CT: layout of the tree kernels (items are layout-free).
template <typename T, int DD, int Q1, int G, int RL, int GT = G, int RLT = RL>
struct SolverImpl {
  using C = Cfg<T, DD, Q1, G, RL>;
  using CT = Cfg<T, DD, Q1, GT, RLT>;
  using V = typename TrajType<T>::type;
  static constexpr int D = C::D;
  static constexpr int NG = kThreads / G;

  static int default_chain_len(int64_t N) {
    // enough chains to fill every SM with several resident groups
    const int64_t target_chains = int64_t(sm_count()) * 8 * NG;
    int64_t L = (N + target_chains - 1) / target_chains;
    L = std::max<int64_t>(L, 4);
    L = std::min<int64_t>(L, 512);
    return static_cast<int>(L);
  }

  // Single-launch iterations (k_iteration) exist for the one-row-per-lane layout only.
  static constexpr bool kFusable = (G == GT) && (RL == RLT);
  static constexpr long long kSpinLimit = 1LL << 30;  // polls per cross-block wait (the 4 s
                                                      // wall-time bound comes first)

  // Chains that one cooperative launch of k_iteration can hold (all blocks resident), or 0
  // when it cannot run here (shared memory, no device).
  static int64_t fused_capacity() {
    if constexpr (!kFusable) {
      return 0;
    } else {
      static std::atomic<int64_t> cached{0};
      const int64_t c = cached.load(std::memory_order_relaxed);
      if (c > 0) return c;
      using FS = FusedShape<C>;
      const int smem = static_cast<int>(FS::smem);
      int n0 = 0, n1 = 0;
      if (cudaFuncSetAttribute(k_iteration<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem) != cudaSuccess ||
          cudaFuncSetAttribute(k_iteration<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_iteration<C, false>, FS::NT,
                                                        smem) != cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_iteration<C, true>, FS::NT,
                                                        smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      const int64_t cap = static_cast<int64_t>(std::min(n0, n1)) * sm_count() * FS::NGB;
      cached.store(cap, std::memory_order_relaxed);
      return cap;
    }
  }

  static int fill_params(const SolveArgs& a, IeksParams<T>& p, int want_cov,
                         bool allow_fused = false) {
    const Problem& pb = a.pb;
    std::memset(&p, 0, sizeof(p));
    p.ode.kind = pb.kind;
    p.ode.d = pb.d;
    for (int i = 0; i < pb.n_params && i < kMaxParams; ++i) {
      p.ode.p[i] = static_cast<T>(pb.params[i]);
      p.pd[i] = pb.params[i];
    }
    p.N = pb.N;
    p.lin_mode = a.opts.linearization;
    p.want_sigma = 1;
    const int64_t cap = (allow_fused && a.opts.scan == 0 && !a.grid) ? fused_capacity() : 0;
    if (a.opts.chain_len > 0) {
      p.L = a.opts.chain_len;
    } else if (cap > 0) {
      // the shortest chains whose count fits one resident wave of the fused kernel
      p.L = static_cast<int>(std::max<int64_t>(4, (pb.N + 1 + cap - 1) / cap));
    } else {
      p.L = default_chain_len(pb.N);
    }
    p.P = pb.N / p.L + 1;
    p.fused = (cap > 0 && p.P <= cap) ? 1 : 0;
    p.want_cov = want_cov;
    p.calibrate = a.opts.calibrate;
    // uniform grid: its step; non-uniform: the first step (T at t_0 preconditions mu0), the
    // per-point data come from grid_step_data
    const double h = a.grid ? a.grid[1] - a.grid[0] : (pb.t1 - pb.t0) / static_cast<double>(pb.N);
    double Phib[64], sqb[64], Td[8];
    if (prior_blocks(pb.q, h, nullptr, nullptr, Phib, sqb, Td) != PIT_OK) return PIT_EINVAL;
    for (int i = 0; i < Q1; ++i) {
      p.Tdiag[i] = static_cast<T>(Td[i]);
      p.Tdiagd[i] = Td[i];
      for (int j = 0; j < Q1; ++j) {
        p.phib[i * kMaxQ1 + j] = static_cast<T>(Phib[i * Q1 + j]);
        p.sqb[i * kMaxQ1 + j] = static_cast<T>(sqb[i * Q1 + j]);
        p.sqbd[i * kMaxQ1 + j] = sqb[i * Q1 + j];
      }
    }
    p.t0 = static_cast<T>(pb.t0);
    p.h = static_cast<T>(h);
    p.T0 = static_cast<T>(Td[0]);
    p.T1inv = static_cast<T>(1.0 / Td[1]);
    p.T0d = Td[0];
    p.T1invd = 1.0 / Td[1];
    p.hq = static_cast<T>(h / pb.q);
    double mu0[kMaxD];
    if (taylor_init(pb, mu0) != PIT_OK) return PIT_EINVAL;
    for (int r = 0; r < D; ++r) {
      p.mu0d[r] = mu0[r] / Td[r % Q1];
      p.mu0[r] = static_cast<T>(p.mu0d[r]);
    }
    return PIT_OK;
  }

  // Scalars of a solve: the per-pass reductions (cleared before every pass) followed by the
  // status word of the single-launch iterations (cleared once per solve), read back together.
  struct ScalBlock {
    SolveScalars s;
    unsigned status;
    unsigned where;  // first cross-block wait that ran out (wait_tag code), or 0
    unsigned pad[2];
  };
  static std::string wait_report(unsigned w) {
    static const char* phases[] = {"filter scan", "smoothing scan", "calibration barrier", "?"};
    return std::string(" (") + phases[(w >> 28) & 3u] + ", block position " +
           std::to_string(w & 0xffffu) + ", level " + std::to_string((w >> 16) & 0xffu) + ")";
  }

  struct Buffers {
    V *linA, *linB;
    T *U, *R, *Yv, *d0;
    T *Es, *gs, *Ls, *fagg, *fup, *sagg, *sup;
    SolveScalars* scal;
    ScalBlock* sblock;
    // non-uniform grid: per-point data (FP64 and arithmetic type)
    double* gsd;
    T* gst;
    // single-launch iterations: cross-block scan values and flags
    T *xf, *xs;
    unsigned* xflags;  // 2 x NB
    int xNB, xK;
    T* coarse_mean;       // coarse-grid initialisation: EKS means and its workspace
    char* coarse_ws;
    size_t coarse_ws_bytes;
  };

  // The sequential EKS on the coarse grid of the initial trajectory.
  static SolveArgs coarse_args(const SolveArgs& a) {
    SolveArgs c = a;
    c.pb.N = a.opts.init_coarse;
    c.opts.init_coarse = 0;
    c.opts.want_cov = 0;
    c.opts.calibrate = 0;
    c.opts.objective = 0;
    c.opts.atol_objective = c.opts.rtol_objective = 0;
    c.opts.chain_len = 0;
    c.init_traj = nullptr;
    c.info = nullptr;
    c.sqrtcov = nullptr;
    return c;
  }

  static size_t carve(const SolveArgs& a, const IeksParams<T>& p, bool want_cov, Buffers& b) {
    Carver cv(a.workspace, a.ws_bytes);
    const int64_t N1 = p.N + 1;
    b.linA = cv.take<V>(N1 * D);
    b.linB = cv.take<V>(N1 * D);
    b.U = cv.take<T>(N1 * D);
    b.R = cv.take<T>(N1 * DD);
    b.Yv = cv.take<T>(N1 * DD);
    b.d0 = cv.take<T>(D);
    b.Es = cv.take<T>(N1 * D * D);
    b.gs = cv.take<T>(N1 * D);
    b.Ls = want_cov ? cv.take<T>(N1 * D * D) : nullptr;
    b.fagg = cv.take<T>(p.P * C::FA);
    b.fup = cv.take<T>(Tree<CT, true, false, false, true>::upper_bytes(p.P) / sizeof(T) + 1);
    b.sagg = cv.take<T>(p.P * C::SA);
    const size_t sup_bytes = std::max(Tree<CT, false, false, true>::upper_bytes(p.P),
                                      Tree<CT, false, true, true>::upper_bytes(p.P));
    b.sup = cv.take<T>(sup_bytes / sizeof(T) + 1);
    b.sblock = cv.take<ScalBlock>(1);
    b.scal = b.sblock ? &b.sblock->s : nullptr;
    b.gsd = a.grid ? cv.take<double>(N1 * (2 * Q1 + 3)) : nullptr;
    b.gst = a.grid ? cv.take<T>(N1 * (2 * Q1 + 3)) : nullptr;
    b.xNB = 0;
    b.xK = 0;
    b.xf = b.xs = nullptr;
    b.xflags = nullptr;
    if (p.fused) {
      b.xNB = static_cast<int>((p.P + FusedShape<C>::NGB - 1) / FusedShape<C>::NGB);
      while ((1 << b.xK) < b.xNB) ++b.xK;
      const size_t lv = static_cast<size_t>(b.xK + 1) * b.xNB;
      b.xf = cv.take<T>(lv * C::FA);
      b.xs = cv.take<T>(lv * C::SA);
      b.xflags = cv.take<unsigned>(2 * static_cast<size_t>(b.xNB) + 1);  // + calibration barrier
    }
    b.coarse_mean = nullptr;
    b.coarse_ws = nullptr;
    b.coarse_ws_bytes = 0;
    if (a.opts.init_coarse > 0) {
      size_t cw = 0;
      run(coarse_args(a), &cw, true);
      b.coarse_mean = cv.take<T>(static_cast<size_t>(a.opts.init_coarse + 1) * D);
      b.coarse_ws = cv.take<char>(cw);
      b.coarse_ws_bytes = cw;
    }
    return cv.used();
  }

  static size_t chain_smem() { return static_cast<size_t>(NG) * C::SCR * sizeof(T); }

  static unsigned elem_grid(int64_t count, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((count + threads - 1) / threads, int64_t(sm_count()) * 16)));
  }

  // Residuals of the increment model at trajectory `lin` (once per iteration).
  template <bool GRID = false>
  static int residuals(const IeksParams<T>& p, const Buffers& b, const V* lin, cudaStream_t s) {
    PIT_LAUNCH(KC_RESIDUALS, s,
               k_residuals<C, GRID><<<elem_grid(p.N + 1, ResTile<C>::size), ResTile<C>::size, 0, s>>>(
                   p, lin, b.U, b.R, b.Yv, b.d0););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  // One filter pass + smoother pass at trajectory `lin` (Algorithm 1 in the linearised model);
  // needs residuals(lin) to have run.
  template <bool WITH_L, bool GRID = false>
  static int pass(const IeksParams<T>& p_in, const Buffers& b, const V* lin, V* lin_out,
                  T* mean_out, T* cov_out, cudaStream_t s) {
    // the diffusion sum is needed by the pass that reports it: the covariance pass, or every
    // means pass of a solve without covariances (its last one is the final iteration)
    IeksParams<T> p = p_in;
    p.want_sigma = (WITH_L || !p.want_cov) ? 1 : 0;
    const unsigned grid = static_cast<unsigned>((p.P + NG - 1) / NG);
    const size_t sm = chain_smem();
    PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
    PIT_LAUNCH(KC_FILTER_REDUCE, s, 
               k_filter_reduce<C, false, GRID><<<grid, kThreads, sm, s>>>(p, b.U, b.R, b.Yv, b.d0,
                                                                          b.fagg););
    int st = Tree<CT, true, false, false, true>::run(b.fagg, p.P, b.fup, false, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_FILTER_DOWN, s, 
               k_filter_down<C, WITH_L, false, false, GRID><<<grid, kThreads, sm, s>>>(
                   p, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs, b.Ls, b.sagg, b.scal););
    st = Tree<CT, false, WITH_L, true>::run(b.sagg, p.P, b.sup, true, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SMOOTH_DOWN, s, 
               k_smooth_down<C, WITH_L, false, GRID><<<grid, kThreads, sm, s>>>(
                   p, b.Es, b.gs, b.Ls, b.sagg, lin, lin_out, mean_out, cov_out, b.scal););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  // One IEKS iteration (or the covariance pass) as a single cooperative launch of k_iteration:
  // residuals at `lin`, both scans and both down-sweeps.  `epoch` must differ for every launch
  // since the exchange flags were cleared.
  template <bool WITH_L>
  static int fused_pass(const IeksParams<T>& p_in, const Buffers& b, const V* lin, V* lin_out,
                        T* mean_out, T* cov_out, unsigned epoch, unsigned cov_launch,
                        cudaStream_t s) {
    if constexpr (!kFusable) {
      set_error("single-launch iterations are not compiled for this layout");
      return PIT_EINTERNAL;
    } else {
      using FS = FusedShape<C>;
      IeksParams<T> p = p_in;
      p.want_sigma = (WITH_L || !p.want_cov) ? 1 : 0;
      PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
      FusedXchg<T> x;
      x.fbuf = b.xf;
      x.sbuf = b.xs;
      x.fflag = b.xflags;
      x.sflag = b.xflags + b.xNB;
      x.status = &b.sblock->status;
      x.where = &b.sblock->where;
      x.barrier = b.xflags + 2 * b.xNB;
      x.bar_target = cov_launch * static_cast<unsigned>(b.xNB);
      x.epoch = epoch;
      x.K = b.xK;
      x.NB = b.xNB;
      x.spin_limit = kSpinLimit;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(static_cast<unsigned>(b.xNB));
      cfg.blockDim = dim3(FS::NT);
      cfg.dynamicSmemBytes = FS::smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaError_t e = cudaSuccess;
      PIT_LAUNCH(KC_ITERATION, s,
                 e = cudaLaunchKernelEx(&cfg, k_iteration<C, WITH_L>, p, lin, lin_out, b.U, b.R,
                                        b.Yv, b.d0, b.Es, b.gs, b.Ls, mean_out, cov_out, b.scal,
                                        x));
      if (e != cudaSuccess) {
        set_error(std::string("cooperative launch of the iteration kernel: ") +
                  cudaGetErrorString(e));
        return PIT_ECUDA;
      }
      return PIT_OK;
    }
  }

  static int set_smem_attrs() {
    const int sm = static_cast<int>(chain_smem());
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_reduce<C>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, false, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, true, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, true, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return PIT_OK;
  }

  // kernels of non-uniform grids
  static int set_smem_attrs_grid() {
    const int sm = static_cast<int>(chain_smem());
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_reduce<C, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, false, false, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, true, false, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, false, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, true, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return PIT_OK;
  }

  // kernels of the segmented (batched) solve
  static int set_smem_attrs_seg() {
    const int sm = static_cast<int>(chain_smem());
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_reduce<C, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, false, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_filter_down<C, true, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, false, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_smooth_down<C, true, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    return PIT_OK;
  }

  static int run(const SolveArgs& a, size_t* wsq, bool eks) {
    const bool want_cov = a.opts.want_cov != 0;
    if (a.grid && (eks || a.opts.init_coarse > 0 || a.opts.objective ||
                   a.opts.atol_objective > 0 || a.opts.rtol_objective > 0)) {
      set_error("non-uniform grids support neither the sequential EKS, coarse initialisation nor "
                "the objective value");
      return PIT_EUNSUPPORTED;
    }
    IeksParams<T> p;
    int st = fill_params(a, p, want_cov ? 1 : 0, !eks);
    if (st != PIT_OK) return st;
    Buffers b;
    const size_t need = carve(a, p, want_cov, b);
    if (wsq) {
      *wsq = need;
      return PIT_OK;
    }
    if (a.ws_bytes < need) {
      set_error("workspace too small: need " + std::to_string(need) + " bytes, got " +
                std::to_string(a.ws_bytes));
      return PIT_ENOMEM;
    }
    if (reinterpret_cast<uintptr_t>(a.workspace) % 256 != 0) {
      set_error("workspace must be 256-byte aligned");
      return PIT_EINVAL;
    }
    st = set_smem_attrs();
    if (st != PIT_OK) return st;
    cudaStream_t s = a.stream;
    const int64_t total = (p.N + 1) * D;
    const unsigned eg = elem_grid(total, 256);
    T* mean = static_cast<T*>(a.mean);
    T* cov = static_cast<T*>(a.sqrtcov);
    pit_solve_info info;
    std::memset(&info, 0, sizeof(info));
    const int64_t launches0 = launches_total();
    ScalBlock hb;
    std::memset(&hb, 0, sizeof(hb));
    SolveScalars& hs = hb.s;
    unsigned epoch = 0;  // single-launch iterations: launches since the flags were cleared
    // the status words are read back with the reductions on either path: clear them per solve
    PIT_CUDA_TRY(cudaMemsetAsync(&b.sblock->status, 0, 2 * sizeof(unsigned), s));
    if (p.fused)
      PIT_CUDA_TRY(cudaMemsetAsync(b.xflags, 0, (2 * b.xNB + 1) * sizeof(unsigned), s));
    if (a.grid) {
      // per-point preconditioner and transition scales of the non-uniform grid
      st = set_smem_attrs_grid();
      if (st != PIT_OK) return st;
      int SW = 0;
      std::vector<double> gs(static_cast<size_t>(p.N + 1) * (2 * Q1 + 3));
      if (grid_step_data(a.grid, p.N, Q1 - 1, gs.data(), &SW) != PIT_OK) return PIT_EINVAL;
      std::vector<T> gt(gs.size());
      for (size_t i = 0; i < gs.size(); ++i) gt[i] = static_cast<T>(gs[i]);
      PIT_CUDA_TRY(cudaMemcpyAsync(b.gsd, gs.data(), sizeof(double) * gs.size(),
                                   cudaMemcpyHostToDevice, s));
      PIT_CUDA_TRY(cudaMemcpyAsync(b.gst, gt.data(), sizeof(T) * gt.size(),
                                   cudaMemcpyHostToDevice, s));
      PIT_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
      p.gsd = b.gsd;
      p.gst = b.gst;
      p.SW = SW;
    }

    if (eks) {
      // sequential EKS: one chain, local linearisation at the predicted mean, plain model
      const size_t sm = chain_smem();
      PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
      IeksParams<T> ps = p;
      ps.L = static_cast<int>(p.N + 1);  // one chain: leaves n = 1..N, owns b_N
      ps.P = 1;
      if (want_cov)
        PIT_LAUNCH(KC_EKS_FILTER, s,
                   k_filter_down<C, true, true><<<1, kThreads, sm, s>>>(
                       ps, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs, b.Ls, b.sagg, b.scal));
      else
        PIT_LAUNCH(KC_EKS_FILTER, s,
                   k_filter_down<C, false, true><<<1, kThreads, sm, s>>>(
                       ps, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs, b.Ls, b.sagg, b.scal));
      if (want_cov) {
        PIT_LAUNCH(KC_EKS_SMOOTH, s, 
                   k_smooth_down<C, true><<<1, kThreads, sm, s>>>(ps, b.Es, b.gs, b.Ls, b.sagg, nullptr,
                                                       nullptr, mean, cov, b.scal););
      } else {
        PIT_LAUNCH(KC_EKS_SMOOTH, s, 
                   k_smooth_down<C, false><<<1, kThreads, sm, s>>>(ps, b.Es, b.gs, b.Ls, b.sagg, nullptr,
                                                        b.linB, mean, cov, b.scal););
        PIT_LAUNCH(KC_EXPORT, s, 
                   k_export_mean<C><<<eg, 256, 0, s>>>(p, b.linB, mean););
      }
      PIT_CUDA_TRY(cudaGetLastError());
      PIT_CUDA_TRY(cudaMemcpyAsync(&hs, b.scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
      PIT_CUDA_TRY(cudaStreamSynchronize(s));
      info.iterations = 1;
      info.converged = 1;
      info.sigma2 = a.opts.calibrate ? hs.sigma2_sum / (static_cast<double>(p.N) * DD) : 1.0;
      info.kernel_launches = launches_total() - launches0;
      if (a.info) *a.info = info;
      return PIT_OK;
    }

    if (a.opts.init_coarse > 0) {
      if (a.opts.init_coarse > p.N || a.init_traj) {
        set_error("init_coarse must be <= N and excludes init_traj");
        return PIT_EINVAL;
      }
      SolveArgs c = coarse_args(a);
      c.mean = b.coarse_mean;
      c.workspace = b.coarse_ws;
      c.ws_bytes = b.coarse_ws_bytes;
      st = run(c, nullptr, true);
      if (st != PIT_OK) return st;
      PIT_LAUNCH(KC_INIT, s,
                 k_coarse_init<C><<<elem_grid(p.N + 1, 256), 256, 0, s>>>(
                     p, b.coarse_mean, static_cast<int64_t>(a.opts.init_coarse),
                     a.pb.t1 - a.pb.t0, b.linA););
    } else {
      if (p.gsd)
        PIT_LAUNCH(KC_INIT, s,
                   k_init_traj<C, true><<<eg, 256, 0, s>>>(p, static_cast<const T*>(a.init_traj),
                                                          b.linA););
      else
        PIT_LAUNCH(KC_INIT, s,
                   k_init_traj<C><<<eg, 256, 0, s>>>(p, static_cast<const T*>(a.init_traj),
                                                    b.linA););
    }
    PIT_CUDA_TRY(cudaGetLastError());
    V* cur = b.linA;  // linearisation trajectory of the current iteration
    V* nxt = b.linB;  // its smoothing means
    const int fixed = a.opts.fixed_iters;
    const int limit = fixed > 0 ? fixed : std::max(1, a.opts.max_iter);
    // objective value V (Eq. objective-value): evaluated when requested or used by the rule
    const bool obj_rule = a.opts.atol_objective > 0 || a.opts.rtol_objective > 0;
    const bool want_obj = obj_rule || a.opts.objective != 0;
    const unsigned og = elem_grid(p.N, 256);
    double v_prev = 0.0;
    if (want_obj) {
      PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
      PIT_LAUNCH(KC_EXPORT, s, k_objective<C><<<og, 256, 0, s>>>(p, cur, b.scal););
      PIT_CUDA_TRY(cudaMemcpyAsync(&hs, b.scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
      PIT_CUDA_TRY(cudaStreamSynchronize(s));
      v_prev = hs.objective;
      info.objectives[0] = v_prev;
      info.objective = v_prev;
    }
    bool converged = fixed > 0;
    int k = 0;
    while (k < limit) {
      if (p.fused) {
        st = fused_pass<false>(p, b, cur, nxt, nullptr, nullptr, ++epoch, 0, s);
      } else if (p.gsd) {
        st = residuals<true>(p, b, cur, s);
        if (st != PIT_OK) return st;
        st = pass<false, true>(p, b, cur, nxt, nullptr, nullptr, s);
      } else {
        st = residuals(p, b, cur, s);
        if (st != PIT_OK) return st;
        st = pass<false>(p, b, cur, nxt, nullptr, nullptr, s);
      }
      if (st != PIT_OK) return st;
      if (want_obj) PIT_LAUNCH(KC_EXPORT, s, k_objective<C><<<og, 256, 0, s>>>(p, nxt, b.scal););
      ++k;
      bool stop = (k == limit);
      if (fixed <= 0 || want_obj) {
        PIT_CUDA_TRY(cudaMemcpyAsync(&hb, b.sblock, sizeof(hb), cudaMemcpyDeviceToHost, s));
        PIT_CUDA_TRY(cudaStreamSynchronize(s));
        if (p.fused && (hb.status & kStatusTimeout)) {
          set_error("a cross-block wait of the iteration kernel ran out at iteration " +
                    std::to_string(k) + wait_report(hb.where));
          return PIT_ETIMEOUT;
        }
        if (hs.flags & 1u) {
          set_error("non-finite value in the smoothing means at iteration " + std::to_string(k));
          return PIT_ENONFINITE;
        }
        info.last_delta = hs.delta_max;
        if (k <= 64) info.deltas[k - 1] = hs.delta_max;
        if (want_obj) {
          if (k <= 64) info.objectives[k] = hs.objective;
          info.objective = hs.objective;
        }
        if (fixed <= 0) {
          if (hs.delta_max <= a.opts.atol_delta + a.opts.rtol_delta * hs.y_max) {
            converged = true;
            stop = true;
          }
          if (obj_rule && std::fabs(hs.objective - v_prev) <=
                              a.opts.atol_objective + a.opts.rtol_objective * std::fabs(hs.objective)) {
            converged = true;
            stop = true;
          }
        }
        v_prev = hs.objective;
      }
      if (stop) break;
      std::swap(cur, nxt);
    }
    // outputs: the last iteration's means (nxt) and, if requested, covariances from a pass with
    // the same linearisation trajectory (cur, whose residuals are still in U, R, Yv); that pass
    // reproduces the same means.
    if (want_cov) {
      st = p.fused ? fused_pass<true>(p, b, cur, nullptr, mean, cov, ++epoch, 1, s)
           : p.gsd ? pass<true, true>(p, b, cur, nullptr, mean, cov, s)
                   : pass<true>(p, b, cur, nullptr, mean, cov, s);
      if (st != PIT_OK) return st;
    } else {
      if (p.gsd)
        PIT_LAUNCH(KC_EXPORT, s, k_export_mean<C, true><<<eg, 256, 0, s>>>(p, nxt, mean););
      else
        PIT_LAUNCH(KC_EXPORT, s, k_export_mean<C><<<eg, 256, 0, s>>>(p, nxt, mean););
    }
    PIT_CUDA_TRY(cudaGetLastError());
    ScalBlock hb2;
    PIT_CUDA_TRY(cudaMemcpyAsync(&hb2, b.sblock, sizeof(hb2), cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    const SolveScalars& hs2 = hb2.s;
    if (p.fused && (hb2.status & kStatusTimeout)) {
      set_error("a cross-block wait of the iteration kernel ran out" + wait_report(hb2.where));
      return PIT_ETIMEOUT;
    }
    if (fixed > 0 && !want_cov) info.last_delta = hs2.delta_max;
    info.iterations = k;
    info.converged = converged ? 1 : 0;
    info.sigma2 = a.opts.calibrate ? hs2.sigma2_sum / (static_cast<double>(p.N) * DD) : 1.0;
    info.kernel_launches = launches_total() - launches0;
    if (a.info) *a.info = info;
    return converged ? PIT_OK : PIT_ENOCONV;
  }
};

// ---- generic scans ---------------------------------------------------------------------------
template <typename T, int D, int G, int RL>
struct ScanImpl {
  using C = Cfg<T, 1, D, G, RL>;
  static constexpr int NG = kThreads / G;
  static int chain_len(int64_t N) {
    const int64_t per = int64_t(sm_count()) * 4 * NG;
    int64_t L = (N + per - 1) / per;
    return static_cast<int>(std::max<int64_t>(4, std::min<int64_t>(L, 256)));
  }
  static int filter(const ScanArgs& a, size_t* wsq) {
    const int L = chain_len(a.N);
    const int64_t P = (a.N + L - 1) / L;
    Carver cv(a.workspace, a.ws_bytes);
    T* items = cv.take<T>(P * C::FA);
    T* up = cv.take<T>(Tree<C, true, false, false>::upper_bytes(P) / sizeof(T) + 1);
    if (wsq) {
      *wsq = cv.used();
      return PIT_OK;
    }
    if (a.ws_bytes < cv.used()) {
      set_error("workspace too small");
      return PIT_ENOMEM;
    }
    const size_t sm = static_cast<size_t>(NG) * (C::SCR + 2 * C::FA) * sizeof(T);
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_gen_filter<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm));
    const unsigned grid = static_cast<unsigned>((P + NG - 1) / NG);
    T *A = (T*)a.x0, *b = (T*)a.x1, *Cm = (T*)a.x2, *eta = (T*)a.x3, *J = (T*)a.x4;
    PIT_LAUNCH(KC_SCAN_FILTER, a.stream, 
               k_gen_filter<C><<<grid, kThreads, sm, a.stream>>>(a.N, L, P, A, b, Cm, eta, J, items, 0););
    int st = Tree<C, true, false, false>::run(items, P, up, false, a.stream);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SCAN_FILTER, a.stream, 
               k_gen_filter<C><<<grid, kThreads, sm, a.stream>>>(a.N, L, P, A, b, Cm, eta, J, items, 1););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }
  template <bool WITH_L>
  static int smooth_t(const ScanArgs& a, size_t* wsq) {
    const int L = chain_len(a.N);
    const int64_t P = (a.N + L - 1) / L;
    Carver cv(a.workspace, a.ws_bytes);
    T* items = cv.take<T>(P * C::SA);
    T* up = cv.take<T>(Tree<C, false, WITH_L, true>::upper_bytes(P) / sizeof(T) + 1);
    if (wsq) {
      *wsq = cv.used();
      return PIT_OK;
    }
    if (a.ws_bytes < cv.used()) {
      set_error("workspace too small");
      return PIT_ENOMEM;
    }
    const size_t sm = static_cast<size_t>(NG) * (C::SCR + 2 * C::SA) * sizeof(T);
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_gen_smooth<C, WITH_L>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const unsigned grid = static_cast<unsigned>((P + NG - 1) / NG);
    T *E = (T*)a.x0, *g = (T*)a.x1, *Lm = (T*)a.x2;
    PIT_LAUNCH(KC_SCAN_SMOOTH, a.stream, 
               k_gen_smooth<C, WITH_L><<<grid, kThreads, sm, a.stream>>>(a.N, L, P, E, g, Lm, items, 0););
    int st = Tree<C, false, WITH_L, true>::run(items, P, up, true, a.stream);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SCAN_SMOOTH, a.stream, 
               k_gen_smooth<C, WITH_L><<<grid, kThreads, sm, a.stream>>>(a.N, L, P, E, g, Lm, items, 1););
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }
  static int smooth(const ScanArgs& a, size_t* wsq) {
    return a.want_L ? smooth_t<true>(a, wsq) : smooth_t<false>(a, wsq);
  }
};

}  // namespace pit
