// Large-state ParaIEKS (Algorithm 2 with Algorithm 1's parallel square-root filter and smoother)
// for ODE dimensions where the state D = d (q+1) is too large for the lane-group kernels of
// pit_chains.cuh: Lorenz-96 with d = 64 (D = 192) and any family with D <= 256.
//
// Same method, model and conventions as the small-state solver (pit_solve_impl.cuh): the scans
// run in preconditioned coordinates on the Gauss-Newton increment delta = Y - lin of each
// iteration (trajectory and residuals in FP64), time steps are cut into chains
// of L consecutive steps, each chain is walked sequentially, and the chain aggregates are
// combined with the full square-root operators of Eqs. sqrt-associative-filtering and
// sqrt-associative-smoothing in a work-efficient (Brent-Kung up-sweep, Blelloch down-sweep)
// tree.  The difference is the granularity: one thread block of dn::NT threads walks a chain and
// every D x D block operation is a block-level dense routine (pit_dense.cuh) on matrices held in
// the chain's scratch area in global memory (L2-resident), instead of rows in lane registers.
//
// Per step of a chain (one time step n, d observations):
//   filter reduce:  A' = Phibar A, b' = Phibar b + u, sqrtC- = tria([sqrtQbar | Phibar sqrtC]);
//                   Psi = tria([[Ht sqrtC-], [sqrtC-]]) (d reflections): sqrtS, K = Psi21 sqrtS^-1,
//                   sqrtC = Psi22; b = b' + K nu, A = A' - K Ht A'; G = sqrtS^-1 Ht A',
//                   eta += G^T sqrtS^-1 nu, sqrtJ = tria([sqrtJ | G^T ...]) every kJ steps
//   filter down:    Pi = tria([[sqrtQbar, Phibar sqrtP], [0, sqrtP]]) (D reflections):
//                   E_{n-1} = Pi21 Pi11^-1, g_{n-1} = m - E m-, sqrtL_{n-1} = tria(Pi22 part);
//                   the chain's smoothing aggregate absorbs (E, g, sqrtL); then the Kalman update
//                   with the Psi-tria of the predicted factor Pi11 (Eq. sqrt-filtering-elements)
//   smooth down:    m^s_n = E_n m^s_{n+1} + g_n, sqrtP^s_n = tria([sqrtL_n | E_n sqrtP^s_{n+1}])
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <type_traits>

#include "pit_dense.cuh"
#include "pit_kernels.cuh"
#include "pit_internal.h"
#include "pit_tc.cuh"

namespace pit {

// FP32 values of the vector field for the sequential EKS's local linearisation
template <>
__device__ __forceinline__ float v_from_double<float>(double x) {
  return static_cast<float>(x);
}

namespace dn {

constexpr int kMaxDenseD = 256;
constexpr int kJBatchDense = 3;  // information rows of kJ steps are folded into sqrtJ at once
#ifndef PIT_TREE_GROUP
#define PIT_TREE_GROUP 8
#endif
constexpr int kTreeGroup = PIT_TREE_GROUP;  // chain aggregates combined by tree levels before the look-back

template <typename T>
struct DenseParams {
  int d, q, Q1, D, W;
  int64_t N, P;
  int L;
  int kind;
  int lin_mode;
  int kJ;
  int want_sigma;
  int calibrate;
  int wsmax;
  int64_t chain_elems;   // scratch elements per chain (and per tree combine)
  T hq, T0, T1inv;
  T Tdiag[kMaxQ1];
  T phib[kMaxQ1 * kMaxQ1];
  T sqb[kMaxQ1 * kMaxQ1];
  double T0d, T1invd;
  double Tdiagd[kMaxQ1];
  const double* pd;      // device: ODE parameters, FP64
  const T* pt;           // device: ODE parameters, arithmetic type
  int n_params;
  const double* mu0d;    // device: preconditioned exact initial state (D)
  // Non-uniform grid (null on a uniform grid): per grid point n = 0..N, SW = 2 Q1 + 3 values
  // [T(h_n) (Q1) | T(h_{n-1}) / T(h_n) (Q1) | h_n / q | T_0(h_n) | 1 / T_1(h_n)], h_n the step
  // into t_n (h_0 = h_1).  In preconditioned coordinates x_n = T(h_n) xbar_n the step into t_n
  // is xbar_n = Phibar diag(T(h_{n-1}) / T(h_n)) xbar_{n-1} + w, w ~ N(0, Qbar) (Section 2.4's
  // step-free Phibar, Qbar), and the observation rows are scaled by 1 / T_1(h_n).
  const double* mu0o;    // device: exact initial state in original coordinates (D)
  const double* gsd;     // FP64
  const T* gst;          // arithmetic type
  int SW;
  // FP64 solves: 1 = the D x D products run on the tensor cores as exact digit products
  // (pit_tc.cuh); tc_status receives the timeout bit of their bounded waits
  int tc;
  unsigned* tc_status;
  int64_t wbuf_off;      // tc: offset of the tria's product buffer in a block's scratch
};

// ---- per-step quantities (uniform grid: the constants) ------------------------------------------
template <typename T>
__device__ __forceinline__ T st_T(const DenseParams<T>& p, int64_t n, int i) {
  return p.gst ? p.gst[n * p.SW + i] : p.Tdiag[i];
}
template <typename T>
__device__ __forceinline__ double st_Td(const DenseParams<T>& p, int64_t n, int i) {
  return p.gsd ? p.gsd[n * p.SW + i] : p.Tdiagd[i];
}
// scale vector of the step into t_n (null: all ones)
template <typename T>
__device__ __forceinline__ const T* st_sc(const DenseParams<T>& p, int64_t n) {
  return p.gst ? p.gst + n * p.SW + p.Q1 : nullptr;
}
template <typename T>
__device__ __forceinline__ T st_hq(const DenseParams<T>& p, int64_t n) {
  return p.gst ? p.gst[n * p.SW + 2 * p.Q1] : p.hq;
}
template <typename T>
__device__ __forceinline__ T st_T0(const DenseParams<T>& p, int64_t n) {
  return p.gst ? p.gst[n * p.SW + 2 * p.Q1 + 1] : p.T0;
}
template <typename T>
__device__ __forceinline__ double st_T0d(const DenseParams<T>& p, int64_t n) {
  return p.gsd ? p.gsd[n * p.SW + 2 * p.Q1 + 1] : p.T0d;
}
template <typename T>
__device__ __forceinline__ double st_T1invd(const DenseParams<T>& p, int64_t n) {
  return p.gsd ? p.gsd[n * p.SW + 2 * p.Q1 + 2] : p.T1invd;
}

// ---- per-step model inputs ------------------------------------------------------------------
// Component k of the vector field in number type V, the state read through y(j): the affine
// family for any d here, every other family through component_f.
template <typename V, typename T, typename Get>
__device__ __forceinline__ V dense_f(int kind, const double* pd, int d, int k, Get y) {
  if (kind == 4 && d > 3) {  // y' = L y + c, params [L (d x d), c (d)]
    V acc = v_from_double<V>(pd[d * d + k]);
    for (int j = 0; j < d; ++j) acc = acc + v_from_double<V>(pd[k * d + j]) * y(j);
    return acc;
  }
  return component_f<V, T>(kind, pd, d, k, y);
}

// Jacobian of the vector field at y (original coordinates), entry (i, j), arithmetic type T.
template <typename T, int DD>
__device__ __forceinline__ T small_jac(const DenseParams<T>& p, const T* y, int i, int j) {
  OdeParams<T> P;
  P.kind = p.kind;
  P.d = DD;
  for (int k = 0; k < kMaxParams; ++k) P.p[k] = k < p.n_params ? p.pt[k] : T(0);
  T yy[DD], f[DD], F[DD][DD];
#pragma unroll
  for (int k = 0; k < DD; ++k) yy[k] = y[k];
  ode_eval<T, DD>(P, yy, f, F);
  T out = T(0);
#pragma unroll
  for (int a = 0; a < DD; ++a)
#pragma unroll
    for (int b = 0; b < DD; ++b)
      if (a == i && b == j) out = F[a][b];
  return out;
}

template <typename T>
__device__ __forceinline__ T jac_entry(const DenseParams<T>& p, const T* y, int i, int j) {
  const int d = p.d;
  if (p.lin_mode == 2 || (p.lin_mode == 1 && i != j)) return T(0);
  switch (p.kind) {
    case 3: {  // Lorenz-96: f_i = (y_{i+1} - y_{i-2}) y_{i-1} - y_i + F, cyclic, d >= 4
      const int ip = (i + 1) % d, im1 = (i - 1 + d) % d, im2 = (i - 2 + d) % d;
      T v = T(0);
      if (j == ip) v += y[im1];
      if (j == im2) v -= y[im1];
      if (j == im1) v += y[ip] - y[im2];
      if (j == i) v -= T(1);
      return v;
    }
    case 4:  // affine: F = L
      return p.pt[i * d + j];
    default:
      if (d == 1) return small_jac<T, 1>(p, y, i, j);
      if (d == 2) return small_jac<T, 2>(p, y, i, j);
      if (d == 3) return small_jac<T, 3>(p, y, i, j);
      return T(0);
  }
}

// Ft = (h/q) F_y(y) (d x d, row-major) for the scaled observation model Ht = E1 - Ft E0.
template <typename T>
__device__ __forceinline__ void cta_jacobian(const DenseParams<T>& p, const T* y, T* Ft, T hq) {
  const int d = p.d;
  for (int e = threadIdx.x; e < d * d; e += NT) {
    const int i = e / d, j = e - i * d;
    Ft[e] = hq * jac_entry<T>(p, y, i, j);
  }
  __syncthreads();
}

// ---- tensor-core products of the FP64 kernels ---------------------------------------------------
// Products with all three dimensions at least kTcMinDim run as FP64-accurate digit products on
// the tensor cores when p.tc is set (FP64 solves); the others, and every FP32 product, on the
// FP64/FP32 pipes (cta_gemm).  Every kernel that reaches dgemm opens a TcScope first.
constexpr int kTcMinDim = 32;

template <typename T, bool TA, bool TB>
__device__ __forceinline__ void dgemm(const DenseParams<T>& p, int m, int n, int k, T alpha,
                                      const T* A, int lda, const T* B, int ldb, T beta, T* C,
                                      int ldc, T* sm) {
  if constexpr (std::is_same<T, double>::value) {
    if (p.tc && m >= kTcMinDim && n >= kTcMinDim && k >= kTcMinDim) {
      const tc::TcCtx c{reinterpret_cast<unsigned char*>(sm), p.tc_status, tc::kTcWaitNs};
      tc::cta_dgemm<TA, TB>(c, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
      return;
    }
  }
  cta_gemm<T, TA, TB>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, sm);
}

// The tensor-core products for a solve: FP64 only; pit_opts.tensor_cores 1 = when D >= 64,
// 2 = for any D, 0 = never.
constexpr int kTcMinD = 64;
template <typename T>
inline int use_tensor_cores(int opt, int D) {
  if (!std::is_same<T, double>::value) return 0;
  return (opt == 2 || (opt == 1 && D >= kTcMinD)) ? 1 : 0;
}

// tria of Section 3.1.2 (cta_lq) with, for FP64 solves with p.tc, the trailing-row products on
// the tensor cores (their buffer in the block's scratch area scr).
template <typename T>
__device__ __forceinline__ void dlq(const DenseParams<T>& p, T* scr, T* M, int ld, int rows,
                                    int rf, int ctri, int ncols, T* sm) {
  if constexpr (std::is_same<T, double>::value) {
    if (p.tc) {
      const tc::TcCtx c{nullptr, p.tc_status, tc::kTcWaitNs};
      cta_lq<T>(M, ld, rows, rf, ctri, ncols, sm, p.wsmax, &c, scr + p.wbuf_off);
      return;
    }
  }
  cta_lq<T>(M, ld, rows, rf, ctri, ncols, sm, p.wsmax);
}

// X op(L) = B (cta_trsm_right) with, for FP64 solves with p.tc, the coupling products on the
// tensor cores.
template <typename T, bool TRANS>
__device__ __forceinline__ void dtrsm_right(const DenseParams<T>& p, int m, int n, const T* L,
                                            int ldl, T* X, int ldx, T* sm) {
  if constexpr (std::is_same<T, double>::value) {
    if (p.tc) {
      const tc::TcCtx c{nullptr, p.tc_status, tc::kTcWaitNs};
      cta_trsm_right<T, TRANS>(m, n, L, ldl, X, ldx, sm, &c);
      return;
    }
  }
  cta_trsm_right<T, TRANS>(m, n, L, ldl, X, ldx, sm);
}

// Holds the block's tensor memory for the lifetime of a kernel (FP64 solves with p.tc only).
// Open it after the kernel's block-uniform early returns; every thread leaves through its end.
template <typename T>
struct TcScope {
  bool on;
  __device__ explicit TcScope(const DenseParams<T>& p)
      : on(std::is_same<T, double>::value && p.tc != 0) {
    if (on) tc::tc_setup();
  }
  __device__ ~TcScope() {
    if (on) tc::tc_teardown();
  }
};

// OUT (d x ncol) = Ht X = E1 X - Ft E0 X for X with D rows (row stride ldx).
template <typename T>
__device__ __forceinline__ void cta_hx(const DenseParams<T>& p, const T* Ft, const T* X, int ldx,
                                       int ncol, T* OUT, int ldo, T* sm) {
  const int d = p.d, Q1 = p.Q1;
  for (int e = threadIdx.x; e < d * ncol; e += NT) {
    const int k = e / ncol, c = e - k * ncol;
    OUT[static_cast<size_t>(k) * ldo + c] = X[static_cast<size_t>(k * Q1 + 1) * ldx + c];
  }
  __syncthreads();
  // E0 X = rows 0, Q1, 2 Q1, ... of X: a matrix with row stride Q1 ldx
  dgemm<T, false, false>(p, d, ncol, d, T(-1), Ft, d, X, Q1 * ldx, T(1), OUT, ldo, sm);
}

// nu = r - Ht x for a state vector x (d values)
template <typename T>
__device__ __forceinline__ void cta_innovation(const DenseParams<T>& p, const T* Ft, const T* x,
                                               const T* r, T* nu) {
  const int d = p.d, Q1 = p.Q1;
  for (int k = threadIdx.x; k < d; k += NT) {
    T acc = x[k * Q1 + 1];
    for (int m = 0; m < d; ++m) acc -= Ft[k * d + m] * x[m * Q1];
    nu[k] = r[k] - acc;
  }
  __syncthreads();
}

// z = sqrtS^-1 x (forward substitution, one thread; d <= 64)
template <typename T>
__device__ __forceinline__ void cta_solve_small(int d, const T* S, int lds, const T* x, T* z) {
  if (threadIdx.x == 0) {
    for (int a = 0; a < d; ++a) {
      T acc = x[a];
      for (int b = 0; b < a; ++b) acc -= S[static_cast<size_t>(a) * lds + b] * z[b];
      z[a] = acc / S[static_cast<size_t>(a) * lds + a];
    }
  }
  __syncthreads();
}

// Entry (i, j) of the step's transition Phibar diag(sc) in one dimension block (sc null: Phibar).
template <typename T>
__device__ __forceinline__ T phi_entry(const DenseParams<T>& p, const T* sc, int i, int j) {
  return sc ? p.phib[i * kMaxQ1 + j] * sc[j] : p.phib[i * kMaxQ1 + j];
}

// y = Phibar diag(sc) x + u   (block upper-triangular, I_d (x) Phibar1); y must not alias x
template <typename T>
__device__ __forceinline__ void cta_phi_vec(const DenseParams<T>& p, const T* x, const T* u, T* y,
                                            const T* sc = nullptr) {
  const int Q1 = p.Q1;
  for (int r = threadIdx.x; r < p.D; r += NT) {
    const int ir = r % Q1, b = r - ir;
    T acc = u ? u[r] : T(0);
    for (int j = ir; j < Q1; ++j) acc += phi_entry(p, sc, ir, j) * x[b + j];
    y[r] = acc;
  }
  __syncthreads();
}

// Y (D x nc) = Phibar diag(sc) X; Y must not alias X
template <typename T>
__device__ __forceinline__ void cta_phi_mat(const DenseParams<T>& p, const T* X, int ldx, int nc,
                                            T* Y, int ldy, const T* sc = nullptr) {
  const int Q1 = p.Q1;
  for (int e = threadIdx.x; e < p.D * nc; e += NT) {
    const int r = e / nc, c = e - r * nc;
    const int ir = r % Q1, b = r - ir;
    T acc = T(0);
    for (int j = ir; j < Q1; ++j) acc += phi_entry(p, sc, ir, j) * X[static_cast<size_t>(b + j) * ldx + c];
    Y[static_cast<size_t>(r) * ldy + c] = acc;
  }
  __syncthreads();
}

// A <- Phibar A in place (D x nc): each thread owns one (dimension block, column) and updates the
// block's rows in increasing order, each reading only rows not yet overwritten.
template <typename T>
__device__ __forceinline__ void cta_phi_inplace(const DenseParams<T>& p, T* A, int lda, int nc,
                                                const T* sc = nullptr) {
  const int Q1 = p.Q1, d = p.d;
  for (int e = threadIdx.x; e < d * nc; e += NT) {
    const int k = e / nc, c = e - k * nc;
    T* col = A + static_cast<size_t>(k * Q1) * lda + c;
    for (int i = 0; i < Q1; ++i) {
      T acc = T(0);
      for (int j = i; j < Q1; ++j) acc += phi_entry(p, sc, i, j) * col[static_cast<size_t>(j) * lda];
      col[static_cast<size_t>(i) * lda] = acc;
    }
  }
  __syncthreads();
}

// X (D x D block of a wider matrix) = sqrt(Qbar) = I_d (x) sqrt(Qbar1)
template <typename T>
__device__ __forceinline__ void cta_sqrtq(const DenseParams<T>& p, T* X, int ldx) {
  const int Q1 = p.Q1, D = p.D;
  for (int e = threadIdx.x; e < D * D; e += NT) {
    const int r = e / D, c = e - r * D;
    const int br = r / Q1, bc = c / Q1, ir = r % Q1, jc = c % Q1;
    X[static_cast<size_t>(r) * ldx + c] = (br == bc && jc <= ir) ? p.sqb[ir * kMaxQ1 + jc] : T(0);
  }
  __syncthreads();
}

// ---- scratch layout of one chain ------------------------------------------------------------
// All matrices row-major; `ldw` = 2 D.  Sizes in elements of T.
struct ChainLayout {
  int64_t Wk, Jw, HA;                           // filter reduce
  int64_t Wk2, Ea0, Ea1, LaW;                   // filter down
  int64_t Pw;                                   // smooth down
  int64_t K, Ft, vec;                           // shared by the passes
  int64_t total;
  int ldw, ldj;
  __host__ __device__ ChainLayout(int d, int D, int kJ) {
    ldw = 2 * D;
    ldj = D + kJ * d;
    int64_t o = 0;
    auto take = [&](int64_t n) {
      const int64_t at = o;
      o += (n + 63) & ~int64_t(63);
      return at;
    };
    Wk = take(int64_t(d + D) * ldw);
    Jw = take(int64_t(D) * ldj);
    HA = take(int64_t(d) * D);
    const int64_t red = o;
    o = 0;
    Wk2 = take(int64_t(d + 2 * D) * ldw);
    Ea0 = take(int64_t(D) * D);
    Ea1 = take(int64_t(D) * D);
    LaW = take(int64_t(D) * 2 * D);
    const int64_t down = o;
    Pw = 0;  // D x 2D, inside either region above
    o = red > down ? red : down;
    K = take(int64_t(D) * d);
    Ft = take(int64_t(d) * d);
    vec = take(int64_t(16) * D);
    total = o;
  }
};
// vector slots inside `vec` (each D long)
enum { V_B = 0, V_ETA, V_BP, V_NU, V_ZNU, V_U, V_R, V_Y, V_M, V_MP, V_XA, V_G, V_MN, V_T0, V_T1 };

// ---- kernels ------------------------------------------------------------------------------------
template <typename T>
using Vt = typename TrajType<T>::type;

template <typename T>
__global__ void k_dinit_traj(const DenseParams<T> p, const T* __restrict__ init,
                             Vt<T>* __restrict__ lin) {
  const int64_t total = (p.N + 1) * p.D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(i % p.D);
    double x;
    if (p.gsd) {
      const int64_t n = i / p.D;
      x = (init ? static_cast<double>(init[i]) : p.mu0o[r]) / st_Td(p, n, r % p.Q1);
    } else {
      x = init ? static_cast<double>(init[i]) / p.Tdiagd[r % p.Q1] : p.mu0d[r];
    }
    lin[i] = v_from_double<Vt<T>>(x);
  }
}

// Residuals of the increment model at trajectory lin (one thread per time step and component):
// u_n = Phibar lin_n - lin_{n+1}, r_n = f(y_n)/T_1 - xbar_{1,n}, y_n = T_0 xbar_{0,n}, delta_0.
template <typename T>
__global__ void __launch_bounds__(256)
k_dres(const DenseParams<T> p, const Vt<T>* __restrict__ lin, T* __restrict__ U,
       T* __restrict__ R, T* __restrict__ Yv, T* __restrict__ d0) {
  using V = Vt<T>;
  const int d = p.d, Q1 = p.Q1, D = p.D;
  const int64_t total = (p.N + 1) * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / d;
    const int k = static_cast<int>(e - n * d);
    const V T0v = v_from_double<V>(st_T0d(p, n));
    const V T1iv = v_from_double<V>(st_T1invd(p, n));
    const V* x = lin + n * D;
    if (n < p.N) {
      if (!p.gsd) {
        for (int i = 0; i < Q1; ++i) {
          V acc = x[k * Q1 + i];
          for (int j = i + 1; j < Q1; ++j) acc = acc + x[k * Q1 + j] * static_cast<float>(p.phib[i * kMaxQ1 + j]);
          acc = acc - lin[(n + 1) * D + k * Q1 + i];
          U[n * D + k * Q1 + i] = v_to_T<T>(acc);
        }
      } else {
        // u_n = Phibar diag(sc_{n+1}) lin_n - lin_{n+1}, the scale factors in extended precision
        const double* sc = p.gsd + (n + 1) * p.SW + Q1;
        for (int i = 0; i < Q1; ++i) {
          V acc = x[k * Q1 + i] * v_from_double<V>(sc[i]);
          for (int j = i + 1; j < Q1; ++j)
            acc = acc + x[k * Q1 + j] * v_from_double<V>(static_cast<double>(p.phib[i * kMaxQ1 + j]) * sc[j]);
          acc = acc - lin[(n + 1) * D + k * Q1 + i];
          U[n * D + k * Q1 + i] = v_to_T<T>(acc);
        }
      }
    }
    const V fk = dense_f<V, T>(p.kind, p.pd, d, k, [&](int j) { return T0v * x[j * Q1]; });
    Yv[n * d + k] = v_to_T<T>(T0v * x[k * Q1]);
    R[n * d + k] = v_to_T<T>(fk * T1iv - x[k * Q1 + 1]);
    if (n == 0)
      for (int i = 0; i < Q1; ++i)
        d0[k * Q1 + i] = v_to_T<T>(v_from_double<V>(p.mu0d[k * Q1 + i]) - x[k * Q1 + i]);
  }
}

// Item layouts (elements of T): filter [A | b | C | eta | J], smoothing [E | g | L].
__host__ __device__ inline int64_t fitem(int D) { return 3LL * D * D + 2LL * D; }
__host__ __device__ inline int64_t sitem(int D) { return 2LL * D * D + D; }

// Model inputs of step n into the vector slots (y_n, r_n, u_{n-1}) and its Jacobian.
template <typename T>
__device__ __forceinline__ void load_step(const DenseParams<T>& p, int64_t n, const T* U,
                                          const T* R, const T* Yv, T* vec, T* Ft) {
  const int d = p.d, D = p.D;
  for (int i = threadIdx.x; i < D; i += NT) vec[V_U * D + i] = U[(n - 1) * D + i];
  for (int i = threadIdx.x; i < d; i += NT) {
    vec[V_Y * D + i] = Yv[n * d + i];
    vec[V_R * D + i] = R[n * d + i];
  }
  __syncthreads();
  cta_jacobian<T>(p, vec + V_Y * D, Ft, st_hq(p, n));
}

// Filter reduce: chain c folds leaves n = cL+1 .. min(cL+L, N) into its aggregate (chain 0 from
// the initial element A = 0, b = delta_0, C = 0; the others from the neutral element).
template <typename T>
__global__ void __launch_bounds__(NT, 1)
k_dreduce(const DenseParams<T> p, const T* __restrict__ U, const T* __restrict__ R,
          const T* __restrict__ Yv, const T* __restrict__ d0, T* __restrict__ fagg,
          T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int64_t chain = blockIdx.x;
  if (chain >= p.P) return;
  TcScope<T> tc_scope(p);
  const int d = p.d, D = p.D, W = p.W;
  const ChainLayout lay(d, D, p.kJ);
  const int ldw = lay.ldw, ldj = lay.ldj;
  T* scr = scratch + chain * p.chain_elems;
  T* item = fagg + chain * fitem(D);
  T* A = item;                      // aggregate A, kept in place in the item
  T* Wk = scr + lay.Wk;
  T* Jw = scr + lay.Jw;
  T* HA = scr + lay.HA;
  T* K = scr + lay.K;
  T* Ft = scr + lay.Ft;
  T* vec = scr + lay.vec;
  T* b = vec + V_B * D;
  T* eta = vec + V_ETA * D;
  T* bp = vec + V_BP * D;
  T* nu = vec + V_NU * D;
  T* znu = vec + V_ZNU * D;
  T* Csq = Wk + static_cast<size_t>(d) * ldw + d;  // sqrtC (D x W) sits where Psi22 lands

  cta_set<T>(D, D, A, D, chain != 0 ? T(1) : T(0));
  for (int i = threadIdx.x; i < D; i += NT) {
    b[i] = chain == 0 ? d0[i] : T(0);
    eta[i] = T(0);
  }
  for (int e = threadIdx.x; e < D * W; e += NT) Csq[static_cast<size_t>(e / W) * ldw + e % W] = T(0);
  for (int e = threadIdx.x; e < D * ldj; e += NT) Jw[e] = T(0);
  __syncthreads();
  int slot = 0;
  const int64_t n0 = chain * p.L + 1;
  const int64_t n1 = min(chain * p.L + p.L, p.N);
  for (int64_t n = n0; n <= n1; ++n) {
    load_step<T>(p, n, U, R, Yv, vec, Ft);
    // predict: A' = Phibar A, b' = Phibar b + u, sqrtC- = tria([sqrtQbar | Phibar sqrtC])
    const T* sc = st_sc(p, n);
    cta_phi_inplace<T>(p, A, D, D, sc);
    cta_phi_vec<T>(p, b, vec + V_U * D, bp, sc);
    T* Pr = Wk + static_cast<size_t>(d) * ldw;  // rows d .. d+D-1
    cta_phi_mat<T>(p, Csq, ldw, W, Pr + D, ldw, sc);
    cta_sqrtq<T>(p, Pr, ldw);
    dlq<T>(p, scr, Pr, ldw, D, D, D, D + W, sm);
    // update: Psi = tria([[Ht sqrtC-], [sqrtC-]]), d reflections
    cta_hx<T>(p, Ft, Pr, ldw, D, Wk, ldw, sm);
    dlq<T>(p, scr, Wk, ldw, d + D, d, 0, D, sm);
    // sqrtS = Wk[0:d, 0:d], Psi21 = Pr[:, 0:d], sqrtC = Psi22 = Pr[:, d:D] (= Csq)
    cta_innovation<T>(p, Ft, bp, vec + V_R * D, nu);
    cta_copy<T>(D, d, Pr, ldw, K, d);
    dtrsm_right<T, false>(p, D, d, Wk, ldw, K, d, sm);
    for (int i = threadIdx.x; i < D; i += NT) b[i] = bp[i];
    __syncthreads();
    cta_gemv<T, false>(D, d, T(1), K, d, nu, T(1), b);
    // A = A' - K Ht A';  G = sqrtS^-1 Ht A'
    cta_hx<T>(p, Ft, A, D, D, HA, D, sm);
    dgemm<T, false, false>(p, D, D, d, T(-1), K, d, HA, D, T(1), A, D, sm);
    cta_trsm_left<T>(d, D, Wk, ldw, HA, D, sm);
    cta_solve_small<T>(d, Wk, ldw, nu, znu);
    cta_gemv<T, true>(D, d, T(1), HA, D, znu, T(1), eta);
    // information rows G^T of this step into the batch; fold the batch into sqrtJ
    cta_copy_t<T>(d, D, HA, D, Jw + D + slot * d, ldj);
    ++slot;
    if (slot == p.kJ || n == n1) {
      dlq<T>(p, scr, Jw, ldj, D, D, D, D + slot * d, sm);
      slot = 0;
    }
  }
  // item: A (in place), b, C = tria(sqrtC) (D x W -> lower-trapezoidal D x D), eta, J
  T* Ci = item + static_cast<int64_t>(D) * D + D;
  for (int e = threadIdx.x; e < D * D; e += NT) {
    const int r = e / D, c = e - r * D;
    Ci[e] = c < W ? Csq[static_cast<size_t>(r) * ldw + c] : T(0);
  }
  for (int i = threadIdx.x; i < D; i += NT) {
    item[static_cast<int64_t>(D) * D + i] = b[i];
    item[2LL * D * D + D + i] = eta[i];
  }
  __syncthreads();
  if (W > 0) dlq<T>(p, scr, Ci, D, D, W, 0, W, sm);
  cta_copy<T>(D, D, Jw, ldj, item + 2LL * D * D + 2 * D, D);
}

// ---- tree operators (block-level, on items in global memory) --------------------------------
// Scratch of one combine (elements of T): X (2D x 2D), M, Y, U (D x D each), CW, JW (D x 2D each),
// vectors, and the output item.
struct TreeLayout {
  int64_t X, M, Y, U, CW, JW, vec, out, total;
  __host__ __device__ TreeLayout(int D) {
    int64_t o = 0;
    auto take = [&](int64_t n) {
      const int64_t at = o;
      o += (n + 63) & ~int64_t(63);
      return at;
    };
    X = take(4LL * D * D);
    M = take(int64_t(D) * D);
    Y = take(int64_t(D) * D);
    U = take(int64_t(D) * D);
    CW = take(2LL * D * D);
    JW = take(2LL * D * D);
    vec = take(8LL * D);
    out = take(fitem(D));
    total = o;
  }
};

// out = a_l (x)_f a_r  (Eq. sqrt-associative-filtering), same steps as combine_f of the
// lane-group kernels.  VALUES: b and C of the result only (the down-sweep).  C_r and J_l must be
// lower-triangular.  `out` must not alias the operands.
template <typename T, bool VALUES>
__device__ void dcombine_f(const DenseParams<T>& p, const T* al, const T* ar, T* out, T* scr,
                           T* sm) {
  const int D = p.D;
  const int64_t DD = static_cast<int64_t>(D) * D;
  const T *Ai = al, *bi = al + DD, *Ci = al + DD + D, *ei = al + 2 * DD + D, *Ji = al + 2 * DD + 2 * D;
  const T *Aj = ar, *bj = ar + DD, *Cj = ar + DD + D, *ej = ar + 2 * DD + D, *Jj = ar + 2 * DD + 2 * D;
  const TreeLayout tl(D);
  T* X = scr + tl.X;  // 2D x 2D, ld 2D
  const int l2 = 2 * D;
  T* M = scr + tl.M;
  T* Y = scr + tl.Y;
  T* Um = scr + tl.U;
  T* CW = scr + tl.CW;
  T* JW = scr + tl.JW;
  T* tv = scr + tl.vec;
  T* sv = tv + D;
  T* vv = sv + D;
  T* uu = vv + D;
  T* wv = uu + D;
  // 1. Xi from the rows [I | Ci^T Jj] over [0 | Jj] (a column permutation of the paper's block)
  cta_set<T>(D, D, X, l2, T(1));
  cta_set<T>(D, D, X + static_cast<size_t>(D) * l2, l2, T(0));
  cta_copy<T>(D, D, Jj, D, X + static_cast<size_t>(D) * l2 + D, l2);
  dgemm<T, true, false>(p, D, D, D, T(1), Ci, D, Jj, D, T(0), X + D, l2, sm);
  dlq<T>(p, scr, X, l2, 2 * D, D, D, 2 * D, sm);
  const T* X11 = X;
  const T* X21 = X + static_cast<size_t>(D) * l2;
  T* X22 = X + static_cast<size_t>(D) * l2 + D;
  if (!VALUES) dlq<T>(p, scr, X22, l2, D, D, 0, D, sm);
  // 2. M = Ci Xi11^-T; Y = I - M Xi21^T
  cta_copy<T>(D, D, Ci, D, M, D);
  dtrsm_right<T, true>(p, D, D, X11, l2, M, D, sm);
  cta_set<T>(D, D, Y, D, T(1));
  dgemm<T, false, true>(p, D, D, D, T(-1), M, D, X21, l2, T(1), Y, D, sm);
  // 3. vectors: t = Ci^T eta_j, v = b_i + Ci t, w = Y v, b_new = b_j + Aj w
  cta_gemv<T, true>(D, D, T(1), Ci, D, ej, T(0), tv);
  for (int i = threadIdx.x; i < D; i += NT) vv[i] = bi[i];
  __syncthreads();
  cta_gemv<T, false>(D, D, T(1), Ci, D, tv, T(1), vv);
  cta_gemv<T, false>(D, D, T(1), Y, D, vv, T(0), wv);
  T* ob = out + DD;
  for (int i = threadIdx.x; i < D; i += NT) ob[i] = bj[i];
  __syncthreads();
  cta_gemv<T, false>(D, D, T(1), Aj, D, wv, T(1), ob);
  // 4. C_new = tria([Cj | Aj M])
  cta_copy<T>(D, D, Cj, D, CW, l2);
  dgemm<T, false, false>(p, D, D, D, T(1), Aj, D, M, D, T(0), CW + D, l2, sm);
  dlq<T>(p, scr, CW, l2, D, D, D, 2 * D, sm);
  cta_copy<T>(D, D, CW, l2, out + DD + D, D);
  if (VALUES) return;
  // 5. U = Y Ai, A_new = Aj U; s = Jj^T b_i, u = eta_j - Jj s, eta_new = U^T u + eta_i
  dgemm<T, false, false>(p, D, D, D, T(1), Y, D, Ai, D, T(0), Um, D, sm);
  dgemm<T, false, false>(p, D, D, D, T(1), Aj, D, Um, D, T(0), out, D, sm);
  cta_gemv<T, true>(D, D, T(1), Jj, D, bi, T(0), sv);
  for (int i = threadIdx.x; i < D; i += NT) uu[i] = ej[i];
  __syncthreads();
  cta_gemv<T, false>(D, D, T(-1), Jj, D, sv, T(1), uu);
  T* oe = out + 2 * DD + D;
  for (int i = threadIdx.x; i < D; i += NT) oe[i] = ei[i];
  __syncthreads();
  cta_gemv<T, true>(D, D, T(1), Um, D, uu, T(1), oe);
  // 6. J_new = tria([Ji | Ai^T Xi22])
  cta_copy<T>(D, D, Ji, D, JW, l2);
  dgemm<T, true, false>(p, D, D, D, T(1), Ai, D, X22, l2, T(0), JW + D, l2, sm);
  dlq<T>(p, scr, JW, l2, D, D, D, 2 * D, sm);
  cta_copy<T>(D, D, JW, l2, out + 2 * DD + 2 * D, D);
}

// out = b_l (x)_s b_r  (Eq. sqrt-associative-smoothing); L_l lower-triangular.
template <typename T, bool WITH_L>
__device__ void dcombine_s(const DenseParams<T>& p, const T* bl, const T* br, T* out, T* scr,
                           T* sm) {
  const int D = p.D;
  const int64_t DD = static_cast<int64_t>(D) * D;
  const TreeLayout tl(D);
  dgemm<T, false, false>(p, D, D, D, T(1), bl, D, br, D, T(0), out, D, sm);
  for (int i = threadIdx.x; i < D; i += NT) out[DD + i] = bl[DD + i];
  __syncthreads();
  cta_gemv<T, false>(D, D, T(1), bl, D, br + DD, T(1), out + DD);
  if (WITH_L) {
    T* LW = scr + tl.CW;
    cta_copy<T>(D, D, bl + DD + D, D, LW, 2 * D);
    dgemm<T, false, false>(p, D, D, D, T(1), bl, D, br + DD + D, D, T(0), LW + D, 2 * D, sm);
    dlq<T>(p, scr, LW, 2 * D, D, D, D, 2 * D, sm);
    cta_copy<T>(D, D, LW, 2 * D, out + DD + D, D);
  } else {
    for (int e = threadIdx.x; e < D * D; e += NT) out[DD + D + e] = T(0);
    __syncthreads();
  }
}

// Tree position -> item index: the filter scan runs in chain order; the smoothing scan runs
// over reversed chains (position 0 = last chain); padding positions >= P map to themselves.
__device__ __forceinline__ int64_t tree_idx(int64_t pos, int64_t P, bool rev) {
  return (rev && pos < P) ? P - 1 - pos : pos;
}

// Neutral elements into the padding items P .. P2-1 (and, with root, into position P2-1).
template <typename T, bool FILTER>
__global__ void __launch_bounds__(NT)
k_dtree_neutral(const DenseParams<T> p, T* __restrict__ items, int64_t first, int64_t last) {
  const int D = p.D;
  const int64_t sz = FILTER ? fitem(D) : sitem(D);
  for (int64_t it = first + blockIdx.x; it < last; it += gridDim.x) {
    T* x = items + it * sz;
    for (int64_t e = threadIdx.x; e < sz; e += NT) {
      T v = T(0);
      if (e < static_cast<int64_t>(D) * D) v = (e / D == e % D) ? T(1) : T(0);
      x[e] = v;
    }
  }
}

// One level of the tree.  UP: item[i] = item[j] (op) item[i]; DOWN: t = item[j], item[j] =
// item[i], item[i] = item[i] (op) t.  Pair k of the level: i = (k+1) 2 s - 1, j = i - s.
// Position order op: filter x (x)_f y; smoothing (reversed chains) y (x)_s x.
// FULL: the filter's down-sweep forms whole prefixes (A, b, C, eta, J) instead of b and C only
// (the generic element scan, whose outputs are the prefixes themselves).
template <typename T, bool FILTER, bool UP, bool WITH_L, bool FULL = false>
__global__ void __launch_bounds__(NT, 1)
k_dtree_level(const DenseParams<T> p, T* __restrict__ items, int64_t s, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int D = p.D;
  const int64_t P = p.P;
  const int64_t sz = FILTER ? fitem(D) : sitem(D);
  const int64_t k = blockIdx.x;
  const int64_t i = (k + 1) * 2 * s - 1, j = i - s;
  if (j - s + 1 >= P) return;  // both subtrees are padding
  TcScope<T> tc_scope(p);
  T* scr = scratch + k * p.chain_elems;
  const TreeLayout tl(D);
  T* res = scr + tl.out;
  T* xi = items + tree_idx(i, P, !FILTER) * sz;
  T* xj = items + tree_idx(j, P, !FILTER) * sz;
  if (UP) {
    if (j + 1 >= P) {  // right subtree padding: the total is the left one
      for (int64_t e = threadIdx.x; e < sz; e += NT) xi[e] = xj[e];
      return;
    }
    if (FILTER) dcombine_f<T, false>(p, xj, xi, res, scr, sm);
    else dcombine_s<T, WITH_L>(p, xi, xj, res, scr, sm);
  } else {
    if (j + 1 >= P) {  // right subtree padding: only the left child's prefix matters
      for (int64_t e = threadIdx.x; e < sz; e += NT) xj[e] = xi[e];
      return;
    }
    if (FILTER) dcombine_f<T, !FULL>(p, xi, xj, res, scr, sm);
    else dcombine_s<T, WITH_L>(p, xj, xi, res, scr, sm);
    for (int64_t e = threadIdx.x; e < sz; e += NT) xj[e] = xi[e];
    __syncthreads();
  }
  if (FILTER && !UP && !FULL) {
    // values-only result: b and C
    const int64_t DD = static_cast<int64_t>(D) * D;
    for (int64_t e = threadIdx.x; e < DD + D; e += NT) xi[DD + e] = res[DD + e];
  } else {
    for (int64_t e = threadIdx.x; e < sz; e += NT) xi[e] = res[e];
  }
}

// Look-back across groups of G tree positions.  After the up-sweep inside the groups, position
// (g+1) G - 1 holds group g's total; one block walks the groups in order, stores each group's
// exclusive prefix at that position (the root of the group's down-sweep) and extends the running
// prefix with the group's total (values-only for the filter).  Applying a short-span aggregate
// to a running prefix is conditioned like the sequential filter; tree levels above the groups
// would instead form elements whose flow maps span up to the whole interval, whose rounding
// strongly unstable linearisations amplify.  pre, tot: two item-sized buffers.
template <typename T, bool FILTER, bool WITH_L, bool FULL = false>
__global__ void __launch_bounds__(NT, 1)
k_dtree_seq(const DenseParams<T> p, T* __restrict__ items, int64_t G, int64_t ngroups,
            T* __restrict__ pre, T* __restrict__ tot, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  TcScope<T> tc_scope(p);
  const int D = p.D;
  const int64_t P = p.P;
  const int64_t sz = FILTER ? fitem(D) : sitem(D);
  const TreeLayout tl(D);
  T* res = scratch + tl.out;
  for (int64_t e = threadIdx.x; e < sz; e += NT) {
    T v = T(0);
    if (e < static_cast<int64_t>(D) * D) v = (e / D == e % D) ? T(1) : T(0);
    pre[e] = v;
  }
  __syncthreads();
  for (int64_t g = 0; g < ngroups; ++g) {
    const int64_t pos = (g + 1) * G - 1;
    if (pos - G + 1 >= P) break;  // this group and all later ones are padding
    T* root = items + tree_idx(pos, P, !FILTER) * sz;
    for (int64_t e = threadIdx.x; e < sz; e += NT) {
      tot[e] = root[e];
      root[e] = pre[e];
    }
    __syncthreads();
    if (pos + 1 >= P) break;      // no later group holds a chain
    if (FILTER && !FULL) {
      dcombine_f<T, true>(p, pre, tot, res, scratch, sm);
      const int64_t DD = static_cast<int64_t>(D) * D;
      for (int64_t e = threadIdx.x; e < DD + D; e += NT) pre[DD + e] = res[DD + e];
    } else if (FILTER) {
      dcombine_f<T, false>(p, pre, tot, res, scratch, sm);
      for (int64_t e = threadIdx.x; e < sz; e += NT) pre[e] = res[e];
    } else {
      dcombine_s<T, WITH_L>(p, tot, pre, res, scratch, sm);
      for (int64_t e = threadIdx.x; e < sz; e += NT) pre[e] = res[e];
    }
    __syncthreads();
  }
}

// Filter down: chain c starts from its exclusive prefix (the filtering marginal at n = cL; chain
// 0 from the initial state) and runs square-root Kalman steps; step n emits the smoothing element
// b_{n-1} and folds it into the chain's smoothing aggregate; the chain owning n = N also emits
// b_N = (0, m^f_N, tria(sqrtP^f_N)).  Accumulates the calibration sum in FP64.
// LOCAL_LIN: the sequential EKS (one chain over all steps, plain model, linearisation at the
// predicted mean of each step).
template <typename T, bool WITH_L, bool LOCAL_LIN = false>
__global__ void __launch_bounds__(NT, 1)
k_ddown(const DenseParams<T> p, const T* __restrict__ U, const T* __restrict__ R,
        const T* __restrict__ Yv, const T* __restrict__ d0, const T* __restrict__ fprefix,
        T* __restrict__ Es, T* __restrict__ gs, T* __restrict__ Ls, T* __restrict__ sagg,
        SolveScalars* __restrict__ scal, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int64_t chain = blockIdx.x;
  if (chain >= p.P) return;
  TcScope<T> tc_scope(p);
  const int d = p.d, D = p.D, W = p.W;
  const int64_t DD = static_cast<int64_t>(D) * D;
  const ChainLayout lay(d, D, p.kJ);
  const int ldw = lay.ldw;
  T* scr = scratch + chain * p.chain_elems;
  T* Wk = scr + lay.Wk2;
  T* Top = Wk + static_cast<size_t>(d) * ldw;       // Pi rows 0 .. D-1
  T* Bot = Top + static_cast<size_t>(D) * ldw;      // Pi rows D .. 2D-1
  T* Ea = scr + lay.Ea0;
  T* Eb = scr + lay.Ea1;
  T* LaW = scr + lay.LaW;
  T* K = scr + lay.K;
  T* Ft = scr + lay.Ft;
  T* vec = scr + lay.vec;
  T* m = vec + V_M * D;
  T* mp = vec + V_MP * D;
  T* xa = vec + V_XA * D;
  T* nu = vec + V_NU * D;
  T* znu = vec + V_ZNU * D;
  T* Psl = Top + d;  // sqrtP^f (D x W) after an update: Psi22's place

  // filter state: chain 0 starts at the initial state (delta_0, zero covariance); the others
  // at the prefix (m = b, sqrtP = C, D columns)
  const T* psrc;
  int psld, ne;
  if (chain == 0) {
    for (int i = threadIdx.x; i < D; i += NT) m[i] = LOCAL_LIN ? static_cast<T>(p.mu0d[i]) : d0[i];
    for (int e = threadIdx.x; e < D * W; e += NT) Psl[static_cast<size_t>(e / W) * ldw + e % W] = T(0);
    psrc = Psl;
    psld = ldw;
    ne = W;
  } else {
    const T* pre = fprefix + chain * fitem(D);
    for (int i = threadIdx.x; i < D; i += NT) m[i] = pre[DD + i];
    psrc = pre + DD + D;
    psld = D;
    ne = D;
  }
  // smoothing aggregate (E~, x, L~) starts neutral
  cta_set<T>(D, D, Ea, D, T(1));
  for (int i = threadIdx.x; i < D; i += NT) xa[i] = T(0);
  if (WITH_L) cta_set<T>(D, D, LaW, 2 * D, T(0));
  __syncthreads();
  double s2acc = 0.0;

  // fold the element (E at Enew, g, sqrtL at Lnew) into the aggregate
  auto fold = [&](const T* Enew, const T* gnew, const T* Lnew) {
    cta_gemv<T, false>(D, D, T(1), Ea, D, gnew, T(1), xa);
    if (WITH_L) {
      dgemm<T, false, false>(p, D, D, D, T(1), Ea, D, Lnew, D, T(0), LaW + D, 2 * D, sm);
      dlq<T>(p, scr, LaW, 2 * D, D, D, D, 2 * D, sm);
    }
    dgemm<T, false, false>(p, D, D, D, T(1), Ea, D, Enew, D, T(0), Eb, D, sm);
    T* t = Ea;
    Ea = Eb;
    Eb = t;
  };

  const int64_t n0 = chain * p.L + 1;
  const int64_t n1 = min(chain * p.L + p.L, p.N);
  for (int64_t n = n0; n <= n1; ++n) {
    if (!LOCAL_LIN) load_step<T>(p, n, U, R, Yv, vec, Ft);
    // Pi input: top [sqrtQbar | Phibar sqrtP], bottom [0 | sqrtP]
    const T* sc = st_sc(p, n);
    cta_phi_mat<T>(p, psrc, psld, ne, Top + D, ldw, sc);
    cta_copy<T>(D, ne, psrc, psld, Bot + D, ldw);
    cta_sqrtq<T>(p, Top, ldw);
    cta_set<T>(D, D, Bot, ldw, T(0));
    cta_phi_vec<T>(p, m, LOCAL_LIN ? nullptr : vec + V_U * D, mp, sc);
    dlq<T>(p, scr, Top, ldw, 2 * D, D, D, D + ne, sm);
    // smoothing element n-1: E = Pi21 Pi11^-1, g = m^f - E m-, sqrtL = tria(remainder)
    T* En = Es + (n - 1) * DD;
    T* gn = gs + (n - 1) * D;
    cta_copy<T>(D, D, Bot, ldw, En, D);
    dtrsm_right<T, false>(p, D, D, Top, ldw, En, D, sm);
    for (int i = threadIdx.x; i < D; i += NT) gn[i] = m[i];
    __syncthreads();
    cta_gemv<T, false>(D, D, T(-1), En, D, mp, T(1), gn);
    T* Ln = nullptr;
    if (WITH_L) {
      Ln = Ls + (n - 1) * DD;
      for (int e = threadIdx.x; e < D * D; e += NT) {
        const int r = e / D, c = e - r * D;
        Ln[e] = c < ne ? Bot[static_cast<size_t>(r) * ldw + D + c] : T(0);
      }
      __syncthreads();
      dlq<T>(p, scr, Ln, D, D, min(D, ne), 0, ne, sm);
    }
    fold(En, gn, Ln);
    if (LOCAL_LIN) {
      // linearise at the predicted mean: y = T_0 E0 m-, Ft = (h/q) F_y(y),
      // r = (f(y) - F_y(y) y) / T_1 (the plain model's scaled observation)
      T* y = vec + V_Y * D;
      T* rr = vec + V_R * D;
      for (int k = threadIdx.x; k < d; k += NT) y[k] = p.T0 * mp[k * p.Q1];
      __syncthreads();
      cta_jacobian<T>(p, y, Ft, p.hq);
      for (int k = threadIdx.x; k < d; k += NT) {
        T acc = dense_f<T, T>(p.kind, p.pd, d, k, [&](int j) { return y[j]; });
        for (int j = 0; j < d; ++j) acc -= jac_entry<T>(p, y, k, j) * y[j];
        rr[k] = acc * p.T1inv;
      }
      __syncthreads();
    }
    // Kalman update of step n with Psi = tria([[Ht Pi11], [Pi11]])
    cta_hx<T>(p, Ft, Top, ldw, D, Wk, ldw, sm);
    dlq<T>(p, scr, Wk, ldw, d + D, d, 0, D, sm);
    cta_innovation<T>(p, Ft, mp, vec + V_R * D, nu);
    cta_copy<T>(D, d, Top, ldw, K, d);
    dtrsm_right<T, false>(p, D, d, Wk, ldw, K, d, sm);
    for (int i = threadIdx.x; i < D; i += NT) m[i] = mp[i];
    __syncthreads();
    cta_gemv<T, false>(D, d, T(1), K, d, nu, T(1), m);
    if (p.want_sigma) {
      cta_solve_small<T>(d, Wk, ldw, nu, znu);
      if (threadIdx.x == 0)
        for (int k = 0; k < d; ++k) s2acc += static_cast<double>(znu[k]) * static_cast<double>(znu[k]);
    }
    psrc = Psl;
    psld = ldw;
    ne = W;
  }
  if (chain == p.N / p.L) {
    // b_N = (E = 0, g = m^f_N, sqrtL = tria(sqrtP^f_N))
    T* En = Es + p.N * DD;
    T* gn = gs + p.N * D;
    for (int e = threadIdx.x; e < D * D; e += NT) En[e] = T(0);
    for (int i = threadIdx.x; i < D; i += NT) gn[i] = m[i];
    __syncthreads();
    T* Ln = nullptr;
    if (WITH_L) {
      Ln = Ls + p.N * DD;
      for (int e = threadIdx.x; e < D * D; e += NT) {
        const int r = e / D, c = e - r * D;
        Ln[e] = c < ne ? psrc[static_cast<size_t>(r) * psld + c] : T(0);
      }
      __syncthreads();
      dlq<T>(p, scr, Ln, D, D, min(D, ne), 0, ne, sm);
    }
    fold(En, gn, Ln);
  }
  T* out = sagg + chain * sitem(D);
  cta_copy<T>(D, D, Ea, D, out, D);
  for (int i = threadIdx.x; i < D; i += NT) out[DD + i] = xa[i];
  if (WITH_L) {
    cta_copy<T>(D, D, LaW, 2 * D, out + DD + D, D);
  } else {
    for (int e = threadIdx.x; e < D * D; e += NT) out[DD + D + e] = T(0);
  }
  if (threadIdx.x == 0 && s2acc != 0.0) atomicAdd(&scal->sigma2_sum, s2acc);
}

// Smoothing down: chain c starts from its reverse exclusive prefix (nothing for the chain that
// holds n = N) and walks its elements backwards.  Means passes write lin_new = lin + delta^s and
// reduce max |change of y|; the covariance pass writes the outputs in original coordinates.
template <typename T, bool WITH_L>
__global__ void __launch_bounds__(NT, 1)
k_dsmooth(const DenseParams<T> p, const T* __restrict__ Es, const T* __restrict__ gs,
          const T* __restrict__ Ls, const T* __restrict__ sprefix, const Vt<T>* __restrict__ lin,
          Vt<T>* __restrict__ lin_new, T* __restrict__ mean_out, T* __restrict__ cov_out,
          SolveScalars* __restrict__ scal, T* __restrict__ scratch) {
  using V = Vt<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  __shared__ T red[2][NWARPS];
  __shared__ int redbad;
  const int64_t chain = blockIdx.x;
  if (chain >= p.P) return;
  TcScope<T> tc_scope(p);
  const int d = p.d, D = p.D, Q1 = p.Q1;
  const int64_t DD = static_cast<int64_t>(D) * D;
  const ChainLayout lay(d, D, p.kJ);
  T* scr = scratch + chain * p.chain_elems;
  T* Pw = scr + lay.Pw;  // [Pss | E Pss], D x 2D
  T* vec = scr + lay.vec;
  T* m = vec + V_M * D;
  T* mn = vec + V_MN * D;
  const bool last = (chain == p.N / p.L);
  const T* pre = sprefix + chain * sitem(D);
  for (int i = threadIdx.x; i < D; i += NT) m[i] = last ? T(0) : pre[DD + i];
  if (threadIdx.x == 0) redbad = 0;
  if (WITH_L) {
    for (int e = threadIdx.x; e < D * D; e += NT) {
      const int r = e / D, c = e - r * D;
      Pw[static_cast<size_t>(r) * 2 * D + c] = last ? T(0) : pre[DD + D + e];
    }
  }
  __syncthreads();
  const T sigma = static_cast<T>(
      (WITH_L && p.calibrate) ? sqrt(scal->sigma2_sum / (static_cast<double>(p.N) * d)) : 1.0);
  T dmax = T(0), ymax = T(0);
  bool bad = false;
  const int64_t s0 = chain * p.L;
  const int64_t s1 = min(chain * p.L + p.L - 1, p.N);
  for (int64_t n = s1; n >= s0; --n) {
    const T* En = Es + n * DD;
    for (int i = threadIdx.x; i < D; i += NT) mn[i] = gs[n * D + i];
    __syncthreads();
    cta_gemv<T, false>(D, D, T(1), En, D, m, T(1), mn);
    if (WITH_L) {
      dgemm<T, false, false>(p, D, D, D, T(1), En, D, Pw, 2 * D, T(0), Pw + D, 2 * D, sm);
      cta_copy<T>(D, D, Ls + n * DD, D, Pw, 2 * D);
      dlq<T>(p, scr, Pw, 2 * D, D, D, D, 2 * D, sm);
    }
    for (int r = threadIdx.x; r < D; r += NT) {
      const V lnew = v_add_small(lin ? lin[n * D + r] : v_from_zero<V>(), mn[r]);
      if (WITH_L) {
        const T tr = st_T(p, n, r % Q1);
        mean_out[n * D + r] = tr * v_to_T<T>(lnew);
        for (int c = 0; c < D; ++c)
          cov_out[n * DD + static_cast<int64_t>(r) * D + c] = sigma * tr * Pw[static_cast<size_t>(r) * 2 * D + c];
      } else {
        lin_new[n * D + r] = lnew;
        if (r % Q1 == 0) {
          const T t0n = st_T0(p, n);
          const T dd = fabs(t0n * mn[r]);
          bad = bad || !(dd == dd);
          dmax = fmax(dmax, dd);
          ymax = fmax(ymax, fabs(t0n * v_to_T<T>(lnew)));
        }
      }
    }
    for (int i = threadIdx.x; i < D; i += NT) m[i] = mn[i];
    __syncthreads();
  }
  if (!WITH_L) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    dmax = warp_max(dmax);
    ymax = warp_max(ymax);
    if (bad) atomicOr(&redbad, 1);
    if (lane == 0) {
      red[0][warp] = dmax;
      red[1][warp] = ymax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T a = T(0), b = T(0);
      for (int w = 0; w < NWARPS; ++w) {
        a = fmax(a, red[0][w]);
        b = fmax(b, red[1][w]);
      }
      if (redbad) atomicOr(&scal->flags, 1u);
      atomic_max_nonneg(&scal->delta_max, static_cast<double>(a));
      atomic_max_nonneg(&scal->y_max, static_cast<double>(b));
    }
  }
}

// Initial trajectory from a coarse-grid solution (Section 3.2.2, remark on the initial
// trajectory): fine point n takes the coarse smoothing mean at node k = floor(n Nc / N),
// propagated by the prior mean over tau = t_n - t_k (Phi(tau)_ij = tau^(j-i)/(j-i)! per
// dimension block, original coordinates, FP64), then preconditioned.
template <typename T>
__global__ void k_dcoarse_init(const DenseParams<T> p, const T* __restrict__ cm, int64_t Nc,
                               double span, Vt<T>* __restrict__ lin) {
  using V = Vt<T>;
  const int d = p.d, Q1 = p.Q1, D = p.D;
  const double scale = span / (static_cast<double>(p.N) * static_cast<double>(Nc));
  const int64_t total = (p.N + 1) * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / d;
    const int b = static_cast<int>(e - n * d);
    int64_t k = (n * Nc) / p.N;
    k = k < Nc ? k : Nc;
    const double tau = static_cast<double>(n * Nc - k * p.N) * scale;
    double pw[kMaxQ1];
    pw[0] = 1.0;
    for (int m = 1; m < Q1; ++m) pw[m] = pw[m - 1] * tau / static_cast<double>(m);
    for (int i = 0; i < Q1; ++i) {
      double x = 0.0;
      for (int j = i; j < Q1; ++j) x += pw[j - i] * static_cast<double>(cm[k * D + b * Q1 + j]);
      lin[n * D + b * Q1 + i] = v_from_double<V>(x / p.Tdiagd[i]);
    }
  }
}

template <typename T>
__global__ void k_dexport(const DenseParams<T> p, const Vt<T>* __restrict__ lin, T* __restrict__ mean) {
  const int64_t total = (p.N + 1) * p.D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(i % p.D);
    mean[i] = st_T(p, i / p.D, r % p.Q1) * v_to_T<T>(lin[i]);
  }
}

// ---- host solver ---------------------------------------------------------------------------------
template <typename T>
struct DenseSolver {
  using V = Vt<T>;

  struct Buffers {
    V *linA, *linB;
    T *U, *R, *Yv, *d0;
    T *Es, *gs, *Ls;
    T *fagg, *sagg, *scratch, *seq;
    SolveScalars* scal;
    unsigned* tcs;   // tensor-core status word (timeout bit), cleared once per solve
    double* pd;
    T* pt;
    double* mu0d;
    double* mu0o;
    double* gsd;
    T* gst;
  };

  static int default_chain_len(int64_t N) {
    // about one chain per SM
    const int64_t sms = sm_count();
    const int64_t L = (N + sms - 1) / sms;
    return static_cast<int>(std::max<int64_t>(1, L));
  }

  static int64_t pow2_at_least(int64_t x) {
    int64_t v = 1;
    while (v < x) v <<= 1;
    return v;
  }

  // Per-point step data of a non-uniform grid (see DenseParams::gsd); FP64 on the host.
  static int grid_steps(const SolveArgs& a, int q, std::vector<double>& gs, int* SW) {
    const int Q1 = q + 1;
    *SW = 2 * Q1 + 3;
    const int64_t N = a.pb.N;
    gs.assign(static_cast<size_t>(N + 1) * *SW, 0.0);
    std::vector<double> Tprev(Q1), Tn(Q1);
    double Phib[64], sqb[64], Td[8];
    for (int64_t n = 0; n <= N; ++n) {
      const double h = n == 0 ? a.grid[1] - a.grid[0] : a.grid[n] - a.grid[n - 1];
      if (prior_blocks(q, h, nullptr, nullptr, Phib, sqb, Td) != PIT_OK) return PIT_EINVAL;
      double* g = gs.data() + n * *SW;
      for (int i = 0; i < Q1; ++i) {
        Tn[i] = Td[i];
        g[i] = Td[i];
        g[Q1 + i] = n == 0 ? 1.0 : Tprev[i] / Td[i];
      }
      g[2 * Q1] = h / q;
      g[2 * Q1 + 1] = Td[0];
      g[2 * Q1 + 2] = 1.0 / Td[1];
      Tprev = Tn;
    }
    return PIT_OK;
  }

  static int fill_params(const SolveArgs& a, DenseParams<T>& p, std::vector<double>& mu0pre,
                         std::vector<double>* mu0orig = nullptr) {
    const Problem& pb = a.pb;
    std::memset(&p, 0, sizeof(p));
    p.d = pb.d;
    p.q = pb.q;
    p.Q1 = pb.q + 1;
    p.D = p.d * p.Q1;
    p.W = p.D - p.d;
    p.N = pb.N;
    p.kind = pb.kind;
    p.lin_mode = a.opts.linearization;
    p.kJ = std::min(kJBatchDense, p.Q1);
    p.want_sigma = 1;
    p.calibrate = a.opts.calibrate;
    p.L = a.opts.chain_len > 0 ? a.opts.chain_len : default_chain_len(pb.N);
    p.P = pb.N / p.L + 1;
    p.n_params = pb.n_params;
    p.wsmax = NB + std::max(p.D, p.kJ * p.d);
    p.tc = use_tensor_cores<T>(a.opts.tensor_cores, p.D);
    if (p.D > kMaxDenseD || p.wsmax > MAXWS) {
      set_error("large-state solver: D = d (q+1) must be <= " + std::to_string(kMaxDenseD));
      return PIT_EUNSUPPORTED;
    }
    // uniform grid: its step; non-uniform: the first step (T at t_0, the scale of mu0's
    // preconditioning); the per-step data come from grid_steps
    const double h = a.grid ? a.grid[1] - a.grid[0] : (pb.t1 - pb.t0) / static_cast<double>(pb.N);
    double Phib[64], sqb[64], Td[8];
    if (prior_blocks(pb.q, h, nullptr, nullptr, Phib, sqb, Td) != PIT_OK) return PIT_EINVAL;
    for (int i = 0; i < p.Q1; ++i) {
      p.Tdiag[i] = static_cast<T>(Td[i]);
      p.Tdiagd[i] = Td[i];
      for (int j = 0; j < p.Q1; ++j) {
        p.phib[i * kMaxQ1 + j] = static_cast<T>(Phib[i * p.Q1 + j]);
        p.sqb[i * kMaxQ1 + j] = static_cast<T>(sqb[i * p.Q1 + j]);
      }
    }
    p.hq = static_cast<T>(h / pb.q);
    p.T0 = static_cast<T>(Td[0]);
    p.T1inv = static_cast<T>(1.0 / Td[1]);
    p.T0d = Td[0];
    p.T1invd = 1.0 / Td[1];
    std::vector<double> mu0(p.D);
    if (taylor_init(pb, mu0.data()) != PIT_OK) return PIT_EINVAL;
    mu0pre.resize(p.D);
    for (int r = 0; r < p.D; ++r) mu0pre[r] = mu0[r] / Td[r % p.Q1];
    if (mu0orig) *mu0orig = mu0;
    const ChainLayout lay(p.d, p.D, p.kJ);
    const TreeLayout tl(p.D);
    p.chain_elems = std::max(lay.total, tl.total);
    if (p.tc) {   // the tria's W and W T (2 x (2 D) x NB values, the tallest tria has 2 D rows)
      p.wbuf_off = (p.chain_elems + 31) / 32 * 32;
      p.chain_elems = p.wbuf_off + 4LL * p.D * NB;
    }
    return PIT_OK;
  }

  static size_t carve(const SolveArgs& a, const DenseParams<T>& p, bool want_cov, Buffers& b) {
    Carver cv(a.workspace, a.ws_bytes);
    const int64_t N1 = p.N + 1;
    const int64_t D = p.D, d = p.d;
    const int64_t P2 = pow2_at_least(p.P);
    b.linA = cv.take<V>(N1 * D);
    b.linB = cv.take<V>(N1 * D);
    b.U = cv.take<T>(N1 * D);
    b.R = cv.take<T>(N1 * d);
    b.Yv = cv.take<T>(N1 * d);
    b.d0 = cv.take<T>(D);
    b.Es = cv.take<T>(N1 * D * D);
    b.gs = cv.take<T>(N1 * D);
    b.Ls = want_cov ? cv.take<T>(N1 * D * D) : nullptr;
    b.fagg = cv.take<T>(P2 * fitem(p.D));
    b.sagg = cv.take<T>(P2 * sitem(p.D));
    b.scratch = cv.take<T>(std::max<int64_t>(p.P, P2 / 2) * p.chain_elems);
    b.seq = cv.take<T>(2 * fitem(p.D));
    b.scal = cv.take<SolveScalars>(1);
    b.tcs = cv.take<unsigned>(4);
    b.pd = cv.take<double>(std::max(1, a.pb.n_params));
    b.pt = cv.take<T>(std::max(1, a.pb.n_params));
    b.mu0d = cv.take<double>(D);
    b.mu0o = cv.take<double>(D);
    if (a.grid) {
      const int64_t SW = 2 * (a.pb.q + 1) + 3;
      b.gsd = cv.take<double>(N1 * SW);
      b.gst = cv.take<T>(N1 * SW);
    } else {
      b.gsd = nullptr;
      b.gst = nullptr;
    }
    return cv.used();
  }

  static size_t smem_bytes(const DenseParams<T>& p) {
    return std::max(lq_smem_elems<T>(p.wsmax) * sizeof(T), p.tc ? lq_tc_smem_bytes(p.wsmax) : size_t(0));
  }

  // Reads the tensor-core status word (one small copy; synchronises the stream).
  static int tc_check(const DenseParams<T>& p, const Buffers& b, cudaStream_t s) {
    if (!p.tc) return PIT_OK;
    unsigned w = 0;
    PIT_CUDA_TRY(cudaMemcpyAsync(&w, b.tcs, sizeof(w), cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    if (w & tc::kTcTimeoutBit) {
      set_error("large-state solver: a wait for the tensor cores gave up after 4 s");
      return PIT_ETIMEOUT;
    }
    return PIT_OK;
  }

  // The attribute is a per-kernel cap shared by every solve, session and scan in the process,
  // so it is always raised to the largest panel width the engine accepts: a call with a smaller
  // D must not lower it under another (e.g. a serving class with larger D) still launching.
  static size_t max_smem_bytes() {
    return std::max(lq_smem_elems<T>(MAXWS) * sizeof(T),
                    std::is_same<T, double>::value ? lq_tc_smem_bytes(MAXWS) : size_t(0));
  }
  static int set_attrs(size_t) {
    const int s = static_cast<int>(max_smem_bytes());
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dreduce<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_ddown<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_ddown<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_ddown<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_ddown<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dsmooth<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dsmooth<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, true, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, false, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_level<T, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_seq<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_seq<T, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    PIT_CUDA_TRY(cudaFuncSetAttribute(k_dtree_seq<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s));
    return PIT_OK;
  }

  // Chain-aggregate scan: Brent-Kung up-sweep inside groups of kTreeGroup positions, a
  // sequential look-back over the group totals (k_dtree_seq), Blelloch down-sweep inside groups.
  template <bool FILTER, bool WITH_L, bool FULL = false>
  static int tree(const DenseParams<T>& p, T* items, T* seq, T* scratch, size_t sm,
                  cudaStream_t s) {
    const int64_t P2 = pow2_at_least(p.P);
    const int64_t G = std::min<int64_t>(P2, kTreeGroup);
    const int kc = FILTER ? KC_TREE_FILTER_UP : KC_TREE_SMOOTH_UP;
    const int kd = FILTER ? KC_TREE_FILTER_DOWN : KC_TREE_SMOOTH_DOWN;
    if (P2 > p.P)
      PIT_LAUNCH(kc, s, (k_dtree_neutral<T, FILTER><<<static_cast<unsigned>(std::min<int64_t>(P2 - p.P, 1024)), NT, 0, s>>>(p, items, p.P, P2)));
    for (int64_t st = 1; st < G; st *= 2) {
      const unsigned grid = static_cast<unsigned>(P2 / (2 * st));
      PIT_LAUNCH(kc, s, (k_dtree_level<T, FILTER, true, WITH_L, FULL><<<grid, NT, sm, s>>>(p, items, st, scratch)));
    }
    const int64_t fs = fitem(p.D);
    PIT_LAUNCH(kd, s, (k_dtree_seq<T, FILTER, WITH_L, FULL><<<1, NT, sm, s>>>(p, items, G, P2 / G, seq, seq + fs, scratch)));
    for (int64_t st = G / 2; st >= 1; st /= 2) {
      const unsigned grid = static_cast<unsigned>(P2 / (2 * st));
      PIT_LAUNCH(kd, s, (k_dtree_level<T, FILTER, false, WITH_L, FULL><<<grid, NT, sm, s>>>(p, items, st, scratch)));
    }
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  template <bool WITH_L>
  static int pass(const DenseParams<T>& p_in, const Buffers& b, const V* lin, V* lin_out,
                  T* mean_out, T* cov_out, bool want_cov, size_t sm, cudaStream_t s) {
    DenseParams<T> p = p_in;
    p.want_sigma = (WITH_L || !want_cov) ? 1 : 0;
    const unsigned grid = static_cast<unsigned>(p.P);
    PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
    PIT_LAUNCH(KC_FILTER_REDUCE, s,
               (k_dreduce<T><<<grid, NT, sm, s>>>(p, b.U, b.R, b.Yv, b.d0, b.fagg, b.scratch)));
    int st = tree<true, false>(p, b.fagg, b.seq, b.scratch, sm, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_FILTER_DOWN, s,
               (k_ddown<T, WITH_L><<<grid, NT, sm, s>>>(p, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs,
                                                       b.Ls, b.sagg, b.scal, b.scratch)));
    st = tree<false, WITH_L>(p, b.sagg, b.seq, b.scratch, sm, s);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SMOOTH_DOWN, s,
               (k_dsmooth<T, WITH_L><<<grid, NT, sm, s>>>(p, b.Es, b.gs, b.Ls, b.sagg, lin, lin_out,
                                                         mean_out, cov_out, b.scal, b.scratch)));
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

  // The sequential EKS on the coarse grid of the initial trajectory.
  static SolveArgs coarse_args(const SolveArgs& a) {
    SolveArgs c = a;
    c.pb.N = a.opts.init_coarse;
    c.opts.init_coarse = 0;
    c.opts.want_cov = 0;
    c.opts.calibrate = 0;
    c.opts.chain_len = 0;
    c.init_traj = nullptr;
    c.info = nullptr;
    c.sqrtcov = nullptr;
    return c;
  }

  static unsigned elem_grid(int64_t count, int threads) {
    return static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((count + threads - 1) / threads, int64_t(sm_count()) * 16)));
  }

  static int run(const SolveArgs& a, size_t* wsq, bool eks) {
    if (a.opts.objective || a.opts.atol_objective > 0 || a.opts.rtol_objective > 0) {
      set_error("the objective value is not evaluated by the large-state solver");
      return PIT_EUNSUPPORTED;
    }
    const bool want_cov = a.opts.want_cov != 0;
    if (a.grid && (eks || a.opts.init_coarse > 0)) {
      set_error("the sequential EKS and the coarse-grid start are implemented for uniform grids");
      return PIT_EUNSUPPORTED;
    }
    DenseParams<T> p;
    std::vector<double> mu0pre, mu0orig;
    int st = fill_params(a, p, mu0pre, &mu0orig);
    if (st != PIT_OK) return st;
    if (eks) {
      // one chain over all steps (leaves 1..N, owner of b_N)
      p.L = static_cast<int>(std::min<int64_t>(p.N + 1, 0x7fffffff));
      p.P = 1;
    }
    Buffers b;
    size_t need = carve(a, p, want_cov, b);
    T* coarse_mean = nullptr;
    char* coarse_ws = nullptr;
    size_t coarse_ws_bytes = 0;
    if (!eks && a.opts.init_coarse > 0) {
      if (a.opts.init_coarse > p.N || a.init_traj) {
        set_error("init_coarse must be <= N and excludes init_traj");
        return PIT_EINVAL;
      }
      size_t cw = 0;
      const SolveArgs c = coarse_args(a);
      st = run(c, &cw, true);
      if (st != PIT_OK) return st;
      Carver cv(a.workspace, a.ws_bytes);
      cv.off = need;
      coarse_mean = cv.take<T>(static_cast<size_t>(a.opts.init_coarse + 1) * p.D);
      coarse_ws = cv.take<char>(cw);
      coarse_ws_bytes = cw;
      need = cv.used();
    }
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
    const size_t sm = smem_bytes(p);
    st = set_attrs(sm);
    if (st != PIT_OK) return st;
    cudaStream_t s = a.stream;
    p.tc_status = b.tcs;
    PIT_CUDA_TRY(cudaMemsetAsync(b.tcs, 0, 4 * sizeof(unsigned), s));
    // ODE parameters and the exact initial state to the device
    std::vector<T> pt(std::max(1, a.pb.n_params));
    for (int i = 0; i < a.pb.n_params; ++i) pt[i] = static_cast<T>(a.pb.params[i]);
    PIT_CUDA_TRY(cudaMemcpyAsync(b.pd, a.pb.params, sizeof(double) * std::max(1, a.pb.n_params),
                                 cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b.pt, pt.data(), sizeof(T) * pt.size(), cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b.mu0d, mu0pre.data(), sizeof(double) * p.D, cudaMemcpyHostToDevice, s));
    p.pd = b.pd;
    p.pt = b.pt;
    p.mu0d = b.mu0d;
    std::vector<double> gs;
    std::vector<T> gst;
    if (a.grid) {
      int SW = 0;
      st = grid_steps(a, p.q, gs, &SW);
      if (st != PIT_OK) return st;
      gst.resize(gs.size());
      for (size_t i = 0; i < gs.size(); ++i) gst[i] = static_cast<T>(gs[i]);
      PIT_CUDA_TRY(cudaMemcpyAsync(b.gsd, gs.data(), sizeof(double) * gs.size(), cudaMemcpyHostToDevice, s));
      PIT_CUDA_TRY(cudaMemcpyAsync(b.gst, gst.data(), sizeof(T) * gst.size(), cudaMemcpyHostToDevice, s));
      p.gsd = b.gsd;
      p.gst = b.gst;
      p.SW = SW;
    }
    PIT_CUDA_TRY(cudaMemcpyAsync(b.mu0o, mu0orig.data(), sizeof(double) * p.D, cudaMemcpyHostToDevice, s));
    p.mu0o = b.mu0o;
    const int64_t total = (p.N + 1) * p.D;
    const unsigned eg = elem_grid(total, 256);
    T* mean = static_cast<T*>(a.mean);
    T* cov = static_cast<T*>(a.sqrtcov);
    pit_solve_info info;
    std::memset(&info, 0, sizeof(info));
    const int64_t launches0 = launches_total();
    SolveScalars hs;
    std::memset(&hs, 0, sizeof(hs));
    if (eks) {
      const unsigned one = 1;
      PIT_CUDA_TRY(cudaMemsetAsync(b.scal, 0, sizeof(SolveScalars), s));
      if (want_cov)
        PIT_LAUNCH(KC_EKS_FILTER, s, (k_ddown<T, true, true><<<one, NT, sm, s>>>(p, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs, b.Ls, b.sagg, b.scal, b.scratch)));
      else
        PIT_LAUNCH(KC_EKS_FILTER, s, (k_ddown<T, false, true><<<one, NT, sm, s>>>(p, b.U, b.R, b.Yv, b.d0, b.fagg, b.Es, b.gs, b.Ls, b.sagg, b.scal, b.scratch)));
      if (want_cov) {
        PIT_LAUNCH(KC_EKS_SMOOTH, s, (k_dsmooth<T, true><<<one, NT, sm, s>>>(p, b.Es, b.gs, b.Ls, b.sagg, nullptr, nullptr, mean, cov, b.scal, b.scratch)));
      } else {
        PIT_LAUNCH(KC_EKS_SMOOTH, s, (k_dsmooth<T, false><<<one, NT, sm, s>>>(p, b.Es, b.gs, b.Ls, b.sagg, nullptr, b.linB, mean, cov, b.scal, b.scratch)));
        PIT_LAUNCH(KC_EXPORT, s, (k_dexport<T><<<eg, 256, 0, s>>>(p, b.linB, mean)));
      }
      PIT_CUDA_TRY(cudaGetLastError());
      PIT_CUDA_TRY(cudaMemcpyAsync(&hs, b.scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
      PIT_CUDA_TRY(cudaStreamSynchronize(s));
      st = tc_check(p, b, s);
      if (st != PIT_OK) return st;
      info.iterations = 1;
      info.converged = 1;
      info.sigma2 = a.opts.calibrate ? hs.sigma2_sum / (static_cast<double>(p.N) * p.d) : 1.0;
      info.kernel_launches = launches_total() - launches0;
      if (a.info) *a.info = info;
      return PIT_OK;
    }
    if (coarse_mean) {
      SolveArgs c = coarse_args(a);
      c.mean = coarse_mean;
      c.workspace = coarse_ws;
      c.ws_bytes = coarse_ws_bytes;
      st = run(c, nullptr, true);
      if (st != PIT_OK) return st;
      PIT_LAUNCH(KC_INIT, s, (k_dcoarse_init<T><<<elem_grid((p.N + 1) * p.d, 256), 256, 0, s>>>(p, coarse_mean, static_cast<int64_t>(a.opts.init_coarse), a.pb.t1 - a.pb.t0, b.linA)));
    } else {
      PIT_LAUNCH(KC_INIT, s, (k_dinit_traj<T><<<eg, 256, 0, s>>>(p, static_cast<const T*>(a.init_traj), b.linA)));
    }
    PIT_CUDA_TRY(cudaGetLastError());
    V* cur = b.linA;
    V* nxt = b.linB;
    const int fixed = a.opts.fixed_iters;
    const int limit = fixed > 0 ? fixed : std::max(1, a.opts.max_iter);
    bool converged = fixed > 0;
    int k = 0;
    const unsigned rg = elem_grid((p.N + 1) * p.d, 256);
    while (k < limit) {
      PIT_LAUNCH(KC_RESIDUALS, s, (k_dres<T><<<rg, 256, 0, s>>>(p, cur, b.U, b.R, b.Yv, b.d0)));
      st = pass<false>(p, b, cur, nxt, nullptr, nullptr, want_cov, sm, s);
      if (st != PIT_OK) return st;
      ++k;
      bool stop = (k == limit);
      if (fixed <= 0) {
        PIT_CUDA_TRY(cudaMemcpyAsync(&hs, b.scal, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PIT_CUDA_TRY(cudaStreamSynchronize(s));
        st = tc_check(p, b, s);
        if (st != PIT_OK) return st;
        if (hs.flags & 1u) {
          set_error("non-finite value in the smoothing means at iteration " + std::to_string(k));
          return PIT_ENONFINITE;
        }
        info.last_delta = hs.delta_max;
        if (k <= 64) info.deltas[k - 1] = hs.delta_max;
        if (hs.delta_max <= a.opts.atol_delta + a.opts.rtol_delta * hs.y_max) {
          converged = true;
          stop = true;
        }
      }
      if (stop) break;
      std::swap(cur, nxt);
    }
    if (want_cov) {
      st = pass<true>(p, b, cur, nullptr, mean, cov, want_cov, sm, s);
      if (st != PIT_OK) return st;
    } else {
      PIT_LAUNCH(KC_EXPORT, s, (k_dexport<T><<<eg, 256, 0, s>>>(p, nxt, mean)));
    }
    PIT_CUDA_TRY(cudaGetLastError());
    SolveScalars hs2;
    PIT_CUDA_TRY(cudaMemcpyAsync(&hs2, b.scal, sizeof(hs2), cudaMemcpyDeviceToHost, s));
    PIT_CUDA_TRY(cudaStreamSynchronize(s));
    st = tc_check(p, b, s);
    if (st != PIT_OK) return st;
    if (fixed > 0 && !want_cov) info.last_delta = hs2.delta_max;
    info.iterations = k;
    info.converged = converged ? 1 : 0;
    info.sigma2 = a.opts.calibrate ? hs2.sigma2_sum / (static_cast<double>(p.N) * p.d) : 1.0;
    info.kernel_launches = launches_total() - launches0;
    if (a.info) *a.info = info;
    return converged ? PIT_OK : PIT_ENOCONV;
  }
};


// ---- a serving-loop request on the large-state kernels (see LargeSession) ----------------------
template <typename T>
class DenseSession final : public LargeSession {
 public:
  using S = DenseSolver<T>;
  using V = Vt<T>;
  static SolveArgs args(const Problem& pb, const pit_opts& o, void* ws, size_t bytes,
                        cudaStream_t s) {
    SolveArgs a;
    std::memset(&a, 0, sizeof(a));
    a.pb = pb;
    a.opts = o;
    a.opts.want_cov = 0;
    a.opts.init_coarse = 0;
    a.opts.objective = 0;
    a.opts.atol_objective = a.opts.rtol_objective = 0;
    a.workspace = ws;
    a.ws_bytes = bytes;
    a.stream = s;
    return a;
  }
  static size_t bytes(const Problem& pb, const pit_opts& o) {
    size_t need = 0;
    const SolveArgs a = args(pb, o, nullptr, 0, nullptr);
    if (S::run(a, &need, false) != PIT_OK) return 0;
    return need;
  }
  int start(const Problem& pb, const pit_opts& o, void* ws, size_t nbytes,
            cudaStream_t s) override {
    a_ = args(pb, o, ws, nbytes, s);
    std::vector<double> mu0pre, mu0orig;
    int st = S::fill_params(a_, p_, mu0pre, &mu0orig);
    if (st != PIT_OK) return st;
    const size_t need = S::carve(a_, p_, false, b_);
    if (nbytes < need) {
      set_error("large-state session: workspace too small");
      return PIT_ENOMEM;
    }
    sm_ = S::smem_bytes(p_);
    st = S::set_attrs(sm_);
    if (st != PIT_OK) return st;
    std::vector<T> pt(std::max(1, pb.n_params));
    for (int i = 0; i < pb.n_params; ++i) pt[i] = static_cast<T>(pb.params[i]);
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.pd, pb.params, sizeof(double) * std::max(1, pb.n_params),
                                 cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.pt, pt.data(), sizeof(T) * pt.size(), cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.mu0d, mu0pre.data(), sizeof(double) * p_.D, cudaMemcpyHostToDevice, s));
    PIT_CUDA_TRY(cudaMemcpyAsync(b_.mu0o, mu0orig.data(), sizeof(double) * p_.D, cudaMemcpyHostToDevice, s));
    p_.pd = b_.pd;
    p_.pt = b_.pt;
    p_.mu0d = b_.mu0d;
    p_.mu0o = b_.mu0o;
    p_.tc_status = &b_.scal->flags;
    const int64_t total = (p_.N + 1) * p_.D;
    PIT_LAUNCH(KC_INIT, s, (k_dinit_traj<T><<<S::elem_grid(total, 256), 256, 0, s>>>(p_, nullptr, b_.linA)));
    PIT_CUDA_TRY(cudaGetLastError());
    cur_ = b_.linA;
    nxt_ = b_.linB;
    return PIT_OK;
  }
  int iterate(LargeScalars* host, cudaStream_t s) override {
    static_assert(sizeof(LargeScalars) == sizeof(SolveScalars), "scalar layouts differ");
    PIT_LAUNCH(KC_RESIDUALS, s, (k_dres<T><<<S::elem_grid((p_.N + 1) * p_.d, 256), 256, 0, s>>>(p_, cur_, b_.U, b_.R, b_.Yv, b_.d0)));
    int st = S::template pass<false>(p_, b_, cur_, nxt_, nullptr, nullptr, false, sm_, s);
    if (st != PIT_OK) return st;
    PIT_CUDA_TRY(cudaMemcpyAsync(host, b_.scal, sizeof(SolveScalars), cudaMemcpyDeviceToHost, s));
    return PIT_OK;
  }
  void advance() override { std::swap(cur_, nxt_); }
  int export_means(void* mean, bool diverged, cudaStream_t s) override {
    const int64_t total = (p_.N + 1) * p_.D;
    PIT_LAUNCH(KC_EXPORT, s, (k_dexport<T><<<S::elem_grid(total, 256), 256, 0, s>>>(p_, diverged ? cur_ : nxt_, static_cast<T*>(mean))));
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }

 private:
  SolveArgs a_{};
  DenseParams<T> p_{};
  typename S::Buffers b_{};
  size_t sm_ = 0;
  V* cur_ = nullptr;
  V* nxt_ = nullptr;
};

// ---- generic element scans (pit_filter_scan / pit_smooth_scan for any D <= 256) -------------
// Inclusive scans of caller-built elements with the block-level operators of the solver's trees:
// each block folds its chain of elements, the chain aggregates are scanned (tree inside groups
// plus look-back, whole prefixes), and each block folds its chain again from its prefix,
// writing every prefix in place.  Element C (filter) and L (smoothing) are triangularised on
// load, which the operators need of the operands they take them from.
template <typename T>
__device__ __forceinline__ void load_felem(const DenseParams<T>& p, int64_t n, const T* A, const T* b,
                                           const T* Cm, const T* eta, const T* J, T* el, T* sm) {
  const int D = p.D;
  const int64_t DD = static_cast<int64_t>(D) * D;
  for (int64_t e = threadIdx.x; e < DD; e += NT) {
    el[e] = A[n * DD + e];
    el[DD + D + e] = Cm[n * DD + e];
    el[2 * DD + 2 * D + e] = J[n * DD + e];
  }
  for (int i = threadIdx.x; i < D; i += NT) {
    el[DD + i] = b[n * D + i];
    el[2 * DD + D + i] = eta[n * D + i];
  }
  __syncthreads();
  cta_lq<T>(el + DD + D, D, D, D, 0, D, sm, p.wsmax);
}

template <typename T>
__global__ void __launch_bounds__(NT, 1)
k_dgen_filter(const DenseParams<T> p, int64_t N, T* __restrict__ A, T* __restrict__ b,
              T* __restrict__ Cm, T* __restrict__ eta, T* __restrict__ J, T* __restrict__ items,
              int down, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int64_t chain = blockIdx.x;
  if (chain >= p.P) return;
  TcScope<T> tc_scope(p);
  const int D = p.D;
  const int64_t DD = static_cast<int64_t>(D) * D, sz = fitem(D);
  const TreeLayout tl(D);
  T* scr = scratch + chain * p.chain_elems;
  T* res = scr + tl.out;
  T* acc = scr + tl.total;
  T* el = acc + sz;
  for (int64_t e = threadIdx.x; e < sz; e += NT) {
    T v = down ? items[chain * sz + e] : T(0);
    if (!down && e < DD) v = (e / D == e % D) ? T(1) : T(0);
    acc[e] = v;
  }
  __syncthreads();
  const int64_t n0 = chain * p.L, n1 = min(chain * p.L + p.L, N);
  for (int64_t n = n0; n < n1; ++n) {
    load_felem<T>(p, n, A, b, Cm, eta, J, el, sm);
    dcombine_f<T, false>(p, acc, el, res, scr, sm);
    for (int64_t e = threadIdx.x; e < sz; e += NT) acc[e] = res[e];
    __syncthreads();
    if (down) {
      for (int64_t e = threadIdx.x; e < DD; e += NT) {
        A[n * DD + e] = acc[e];
        Cm[n * DD + e] = acc[DD + D + e];
        J[n * DD + e] = acc[2 * DD + 2 * D + e];
      }
      for (int i = threadIdx.x; i < D; i += NT) {
        b[n * D + i] = acc[DD + i];
        eta[n * D + i] = acc[2 * DD + D + i];
      }
      __syncthreads();
    }
  }
  if (!down)
    for (int64_t e = threadIdx.x; e < sz; e += NT) items[chain * sz + e] = acc[e];
}

template <typename T, bool WITH_L>
__global__ void __launch_bounds__(NT, 1)
k_dgen_smooth(const DenseParams<T> p, int64_t N, T* __restrict__ E, T* __restrict__ gv,
              T* __restrict__ Lm, T* __restrict__ items, int down, T* __restrict__ scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int64_t chain = blockIdx.x;
  if (chain >= p.P) return;
  TcScope<T> tc_scope(p);
  const int D = p.D;
  const int64_t DD = static_cast<int64_t>(D) * D, sz = sitem(D);
  const TreeLayout tl(D);
  T* scr = scratch + chain * p.chain_elems;
  T* res = scr + tl.out;
  T* acc = scr + tl.total;
  T* el = acc + fitem(D);
  for (int64_t e = threadIdx.x; e < sz; e += NT) {
    T v = down ? items[chain * sz + e] : T(0);
    if (!down && e < DD) v = (e / D == e % D) ? T(1) : T(0);
    acc[e] = v;
  }
  __syncthreads();
  auto load = [&](int64_t n) {
    for (int64_t e = threadIdx.x; e < DD; e += NT) {
      el[e] = E[n * DD + e];
      el[DD + D + e] = WITH_L ? Lm[n * DD + e] : T(0);
    }
    for (int i = threadIdx.x; i < D; i += NT) el[DD + i] = gv[n * D + i];
    __syncthreads();
    if (WITH_L) cta_lq<T>(el + DD + D, D, D, D, 0, D, sm, p.wsmax);
  };
  const int64_t n0 = chain * p.L, n1 = min(chain * p.L + p.L, N);
  if (!down) {
    for (int64_t n = n0; n < n1; ++n) {   // acc = b_n0 (x) ... (x) b_{n1-1}
      load(n);
      dcombine_s<T, WITH_L>(p, acc, el, res, scr, sm);
      for (int64_t e = threadIdx.x; e < sz; e += NT) acc[e] = res[e];
      __syncthreads();
    }
    for (int64_t e = threadIdx.x; e < sz; e += NT) items[chain * sz + e] = acc[e];
  } else {
    for (int64_t n = n1 - 1; n >= n0; --n) {  // acc = b_n (x) acc
      load(n);
      dcombine_s<T, WITH_L>(p, el, acc, res, scr, sm);
      for (int64_t e = threadIdx.x; e < sz; e += NT) acc[e] = res[e];
      __syncthreads();
      for (int64_t e = threadIdx.x; e < DD; e += NT) {
        E[n * DD + e] = acc[e];
        if (WITH_L) Lm[n * DD + e] = acc[DD + D + e];
      }
      for (int i = threadIdx.x; i < D; i += NT) gv[n * D + i] = acc[DD + i];
      __syncthreads();
    }
  }
}

template <typename T>
struct DenseScan {
  static DenseParams<T> params(int64_t N, int D) {
    DenseParams<T> p;
    std::memset(&p, 0, sizeof(p));
    p.D = D;
    p.N = N;
    p.L = static_cast<int>(std::max<int64_t>(1, (N + sm_count() - 1) / sm_count()));
    p.P = (N + p.L - 1) / p.L;
    p.wsmax = NB + D;
    const TreeLayout tl(D);
    p.chain_elems = tl.total + 2 * fitem(D);
    return p;
  }
  struct Bufs {
    T *items, *seq, *scratch;
  };
  static size_t carve(const ScanArgs& a, const DenseParams<T>& p, Bufs& b) {
    Carver cv(a.workspace, a.ws_bytes);
    int64_t P2 = 1;
    while (P2 < p.P) P2 <<= 1;
    b.items = cv.take<T>(P2 * fitem(p.D));
    b.seq = cv.take<T>(2 * fitem(p.D));
    b.scratch = cv.take<T>(std::max<int64_t>(p.P, P2 / 2) * p.chain_elems);
    return cv.used();
  }
  template <class K>
  static int attr(K k, size_t) {
    PIT_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(DenseSolver<T>::max_smem_bytes())));
    return PIT_OK;
  }
  static int check(const ScanArgs& a, int D, size_t need) {
    if (a.ws_bytes < need) {
      set_error("workspace too small: need " + std::to_string(need) + " bytes");
      return PIT_ENOMEM;
    }
    if (reinterpret_cast<uintptr_t>(a.workspace) % 256 != 0) {
      set_error("workspace must be 256-byte aligned");
      return PIT_EINVAL;
    }
    return PIT_OK;
  }
  static int filter(const ScanArgs& a, int D, size_t* wsq) {
    if (D > kMaxDenseD) {
      set_error("scan: D must be <= " + std::to_string(kMaxDenseD));
      return PIT_EUNSUPPORTED;
    }
    DenseParams<T> p = params(a.N, D);
    Bufs b;
    const size_t need = carve(a, p, b);
    if (wsq) {
      *wsq = need;
      return PIT_OK;
    }
    int st = check(a, D, need);
    if (st != PIT_OK) return st;
    const size_t sm = lq_smem_elems<T>(p.wsmax) * sizeof(T);
    if ((st = attr(k_dgen_filter<T>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_level<T, true, true, false, true>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_level<T, true, false, false, true>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_seq<T, true, false, true>, sm)) != PIT_OK) return st;
    T *A = (T*)a.x0, *bb = (T*)a.x1, *Cm = (T*)a.x2, *eta = (T*)a.x3, *J = (T*)a.x4;
    const unsigned grid = static_cast<unsigned>(p.P);
    PIT_LAUNCH(KC_SCAN_FILTER, a.stream, (k_dgen_filter<T><<<grid, NT, sm, a.stream>>>(p, a.N, A, bb, Cm, eta, J, b.items, 0, b.scratch)));
    st = DenseSolver<T>::template tree<true, false, true>(p, b.items, b.seq, b.scratch, sm, a.stream);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SCAN_FILTER, a.stream, (k_dgen_filter<T><<<grid, NT, sm, a.stream>>>(p, a.N, A, bb, Cm, eta, J, b.items, 1, b.scratch)));
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }
  template <bool WITH_L>
  static int smooth_t(const ScanArgs& a, int D, size_t* wsq) {
    if (D > kMaxDenseD) {
      set_error("scan: D must be <= " + std::to_string(kMaxDenseD));
      return PIT_EUNSUPPORTED;
    }
    DenseParams<T> p = params(a.N, D);
    Bufs b;
    const size_t need = carve(a, p, b);
    if (wsq) {
      *wsq = need;
      return PIT_OK;
    }
    int st = check(a, D, need);
    if (st != PIT_OK) return st;
    const size_t sm = lq_smem_elems<T>(p.wsmax) * sizeof(T);
    if ((st = attr(k_dgen_smooth<T, WITH_L>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_level<T, false, true, WITH_L>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_level<T, false, false, WITH_L>, sm)) != PIT_OK) return st;
    if ((st = attr(k_dtree_seq<T, false, WITH_L>, sm)) != PIT_OK) return st;
    T *E = (T*)a.x0, *g = (T*)a.x1, *Lm = (T*)a.x2;
    const unsigned grid = static_cast<unsigned>(p.P);
    PIT_LAUNCH(KC_SCAN_SMOOTH, a.stream, (k_dgen_smooth<T, WITH_L><<<grid, NT, sm, a.stream>>>(p, a.N, E, g, Lm, b.items, 0, b.scratch)));
    st = DenseSolver<T>::template tree<false, WITH_L>(p, b.items, b.seq, b.scratch, sm, a.stream);
    if (st != PIT_OK) return st;
    PIT_LAUNCH(KC_SCAN_SMOOTH, a.stream, (k_dgen_smooth<T, WITH_L><<<grid, NT, sm, a.stream>>>(p, a.N, E, g, Lm, b.items, 1, b.scratch)));
    PIT_CUDA_TRY(cudaGetLastError());
    return PIT_OK;
  }
  static int smooth(const ScanArgs& a, int D, size_t* wsq) {
    return a.want_L ? smooth_t<true>(a, D, wsq) : smooth_t<false>(a, D, wsq);
  }
};


// ---- linearisation for any d (pit_linearize beyond the lane-group families) -------------------
// H_n = E1 - F_y(E0 traj_n) E0 and d_n = f - F_y y at every n = 1..N (Section 3.2.1), one thread
// per (n, component); the family's parameters travel in the kernel argument.  lin_mode replaces
// F_y by its diagonal (1) or by zero (2), the approximate Jacobians of Section 3.2.1's remark.
struct LinArgs {
  int kind, d, Q1, n_params, lin_mode;
  double pd[kMaxParams];
};

template <typename T>
__global__ void __launch_bounds__(256)
k_dlinearize(const LinArgs a, int64_t N, const T* __restrict__ traj, T* __restrict__ H,
             T* __restrict__ dv) {
  double pd[kMaxParams];
  T pt[kMaxParams];
  for (int i = 0; i < kMaxParams; ++i) {
    pd[i] = a.pd[i];
    pt[i] = static_cast<T>(a.pd[i]);
  }
  DenseParams<T> p{};
  p.kind = a.kind;
  p.d = a.d;
  p.Q1 = a.Q1;
  p.D = a.d * a.Q1;
  p.n_params = a.n_params;
  p.lin_mode = 0;
  p.pd = pd;
  p.pt = pt;
  const int d = a.d, Q1 = a.Q1, D = d * Q1;
  const int64_t total = N * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = 1 + e / d;
    const int k = static_cast<int>(e % d);
    T y[kMaxOdeDim];
    for (int m = 0; m < d; ++m) y[m] = traj[n * D + m * Q1];
    T* Hr = H + ((n - 1) * d + k) * D;
    for (int c = 0; c < D; ++c) Hr[c] = T(0);
    Hr[k * Q1 + 1] = T(1);
    T acc = dense_f<T, T>(a.kind, pd, d, k, [&](int j) { return y[j]; });
    for (int m = 0; m < d; ++m) {
      const bool keep = a.lin_mode == 0 || (a.lin_mode == 1 && m == k);
      const T F = keep ? jac_entry<T>(p, y, k, m) : T(0);
      Hr[m * Q1] -= F;
      acc -= F * y[m];
    }
    dv[(n - 1) * d + k] = acc;
  }
}

template <typename T>
int dense_linearize(const Problem& pb, int lin_mode, const void* traj, void* H, void* dv,
                    cudaStream_t s) {
  if (pb.n_params > kMaxParams) {
    set_error("pit_linearize: families with more than " + std::to_string(kMaxParams) +
              " parameters (affine beyond d = 5) are linearised inside pit_solve only");
    return PIT_EUNSUPPORTED;
  }
  LinArgs a{};
  a.kind = pb.kind;
  a.d = pb.d;
  a.Q1 = pb.q + 1;
  a.n_params = pb.n_params;
  a.lin_mode = lin_mode;
  for (int i = 0; i < pb.n_params; ++i) a.pd[i] = pb.params[i];
  const int64_t total = pb.N * pb.d;
  const unsigned grid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 16)));
  PIT_LAUNCH(KC_LINEARIZE, s, (k_dlinearize<T><<<grid, 256, 0, s>>>(a, pb.N, static_cast<const T*>(traj), static_cast<T*>(H), static_cast<T*>(dv))));
  PIT_CUDA_TRY(cudaGetLastError());
  return PIT_OK;
}

}  // namespace dn
}  // namespace pit
