// Kernels of the time-parallel IEKS (Algorithms 1 and 2) for small state dimension D = d (q+1).
//
// Work decomposition.  The N filtering elements (and N+1 smoothing elements) are cut into
// chains of L consecutive time steps; one lane group (see pit_group.cuh) walks one chain.
// Inside a chain the associative operators are applied left to right, which the structure of
// the elements makes cheap:
//   * filter reduce:  aggregate (x)_f a_n, where a_n is a rank-d leaf element, is one
//     square-root Kalman prediction + update of the "conditional" filter (A, b, sqrtC) plus a
//     rank-d update of the information part (eta, sqrtJ);
//   * filter down:    (m^f_{n-1}, sqrtP^f_{n-1}) (x)_f a_n is one square-root Kalman step; the
//     same Pi-triangularisation yields the smoothing element b_{n-1} (Eq.
//     sqrt-smoothing-elements), which is written out, and the chain's smoothing aggregate;
//   * smooth down:    m^s_n = E_n m^s_{n+1} + g_n (and the square-root covariance with one
//     tria) walking the chain backwards.
// The chain aggregates are combined with the full square-root operators of Eqs.
// sqrt-associative-filtering / sqrt-associative-smoothing in a work-efficient
// (Brent-Kung/Blelloch) tree, first inside a thread block in shared memory, then across blocks.
//
// Coordinates.  The device works in preconditioned coordinates x = T xbar with
// T = I_d (x) sqrt(h) diag(h^(q-i)/(q-i)!) (Section 2.4): the transitions become the
// step-size-free Phibar = binom(q-i, j-i), Qbar = 1/(2q+1-i-j).  The observation rows are scaled
// by 1/T_1, which leaves the Dirac conditioning unchanged: Htilde = E1 - (h/q) F E0,
// dtilde = d / T_1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pit_group.cuh"
#include "pit_ode.cuh"

namespace pit {

constexpr int kMaxQ1 = 8;
constexpr int kMaxD = 16;

constexpr int kMaxInstParams = 12;  // ODE parameters per instance of a segmented solve

// One instance of a segmented (batched) solve, indexed by instance id.  Many instances share
// one global time axis: instance i occupies global points off .. off + N (its n = 0 .. N).  At
// its n = 0 the filter scan meets a "reset" element (A = 0, b = delta_0, C = 0, eta = 0,
// J = 0), and at its n = N the smoothing scan meets an element with E = 0, so neither scan
// carries anything across an instance boundary (the associative operators of Section 3.1 are
// applied unchanged; the instances form segments of one scan).
template <typename T>
struct InstDesc {
  int64_t off;                  // global point of n = 0 in the current layout
  int64_t N;                    // time steps
  void* lin[2];                 // linearisation trajectories (TrajType<T>), (N+1) x D each
  int cur;                      // lin[cur] is the trajectory of the current iteration
  int pad_;
  T* mean;                      // output means, original coordinates: point n, row r at
                                // mean[n * mean_ld + r]
  T* cov;                       // output square-root covariances, or null: point n, (r, c) at
                                // cov[n * cov_ld + r * cov_rld + c]
  int64_t mean_ld, cov_ld, cov_rld;
  double pd[kMaxInstParams];    // ODE parameters (FP64)
  double mu0d[kMaxD];           // preconditioned exact initial state
  double T0d, T1invd;
  double Tdiagd[kMaxQ1];
  T p[kMaxInstParams];          // ODE parameters (arithmetic type)
  T T0, T1inv, hq;
  T Tdiag[kMaxQ1];
};

// Per-instance reductions of one pass (device, zeroed before each pass).
struct InstAcc {
  double sigma2_sum;   // sum_n ||sqrtS_n^-1 r_n||^2
  double delta_max;    // max |change of E0 mean| (original coordinates)
  double y_max;        // max |E0 mean|
  unsigned int flags;  // bit 0: non-finite value seen
  unsigned int pad;
};

// Segment view of a batched solve (all null for a single problem).
template <typename T>
struct SegView {
  const InstDesc<T>* desc;   // by instance id
  const int* inst_of;        // per global point: instance id, or ~id at the instance's n = 0
  InstAcc* acc;              // by instance id
};

__device__ __forceinline__ int seg_id(int code) { return code < 0 ? ~code : code; }

// Per-solve constants (kernel argument).
template <typename T>
struct IeksParams {
  OdeParams<T> ode;
  int64_t N;        // time steps (observations at n = 1..N)
  int64_t P;        // chains = N / L + 1
  int L;            // chain length
  int want_cov;     // this pass produces square-root covariances
  int calibrate;    // scale square-root covariances by the quasi-MLE sigma
  T t0, h;
  T T0;             // T_0(h): y = T_0 xbar_{k(q+1)}
  T T1inv;          // 1 / T_1(h)
  T hq;             // h / q
  T Tdiag[kMaxQ1];  // T_i(h), i = 0..q
  T phib[kMaxQ1 * kMaxQ1];   // Phibar (q+1)x(q+1), row-major
  T sqb[kMaxQ1 * kMaxQ1];    // lower Cholesky factor of Qbar
  T mu0[kMaxD];              // preconditioned exact initial state
  // FP64 copies for the trajectory arithmetic
  double mu0d[kMaxD];
  double pd[kMaxParams];
  double T0d, T1invd;
  double Tdiagd[kMaxQ1];
  SegView<T> seg;   // segmented solve: instance table and point -> instance map
  int lin_mode;     // Jacobian: 0 exact (EK1), 1 diagonal (DiagonalEK1), 2 zero (EK0)
  int want_sigma;   // accumulate the quasi-MLE diffusion sum in this pass
  int fused;        // host only: iterations run as single cooperative launches
  // Non-uniform grid (null on a uniform grid): per grid point n = 0..N, SW = 2 Q1 + 3 values
  // [T(h_n) (Q1) | T(h_{n-1}) / T(h_n) (Q1) | h_n / q | T_0(h_n) | 1 / T_1(h_n)], h_n the step
  // into t_n (h_0 = h_1); FP64 (gsd) and the arithmetic type (gst).  In coordinates
  // x_n = T(h_n) xbar_n the step into t_n is xbar_n = Phibar diag(T(h_{n-1}) / T(h_n)) xbar_{n-1}
  // + w, w ~ N(0, Qbar) (Section 2.4's step-free Phibar, Qbar), and the observation rows of
  // point n are scaled by 1 / T_1(h_n).
  const double* gsd;
  const T* gst;
  int SW;
  int sigma_pool;   // segmented: > 0 pools the diffusion sums of instances 0..sigma_pool-1
                    // (the components of one decoupled problem) into one sigma-hat
  double sqbd[kMaxQ1 * kMaxQ1];   // sqrt(Qbar) in FP64 (objective value)
};

// Number type of the linearisation trajectory: FP64 for both solvers.  At fine grids the
// residuals r_n = (f(y_n) - y'_n) / T_1(h) of the increment model amplify the trajectory's
// representation error by 1 / T_1(h) (about 1e12 for IWP(3) at h = 2e-5), and the quasi-MLE
// diffusion is a mean of squared residuals: a 48-bit double-float trajectory left sigma-hat^2
// 1% off at N = 2^20 where FP64 keeps it within 2e-5.
template <typename T>
struct TrajType {
  using type = double;
};

// Scalars shared by the kernels of one solve (device memory, FP64).
struct SolveScalars {
  double sigma2_sum;   // sum_n ||sqrtS_n^-1 r_n||^2 of the current filter pass
  double delta_max;    // max |change of E0 mean| (original coordinates)
  double y_max;        // max |E0 mean| (original coordinates)
  unsigned int flags;  // bit 0: non-finite value seen
  unsigned int pad;
  double objective;    // V of the trajectory (Eq. objective-value), when evaluated
};

#ifndef PIT_LDM_PAD
#define PIT_LDM_PAD 0
#endif
#ifndef PIT_SCR_SHIFT
#define PIT_SCR_SHIFT 0
#endif

template <typename T, int DD_, int Q1_, int G_, int RL_>
struct Cfg {
  using Tp = T;
  static constexpr int DD = DD_;
  static constexpr int Q1 = Q1_;
  static constexpr int D = DD_ * Q1_;
  static constexpr int W = D - DD_;
  static constexpr int G = G_;
  static constexpr int RL = RL_;
  static constexpr int RP = G_ * RL_;
  // row stride of published matrices (FP32: optionally padded against bank conflicts)
  static constexpr int LDM = D + (sizeof(T) == 4 ? PIT_LDM_PAD : 0);
  // group scratch layout (elements of T)
  static constexpr int MAT0 = 0;
  static constexpr int MAT1 = MAT0 + RP * LDM;
  static constexpr int MAT2 = MAT1 + RP * LDM;
  static constexpr int VEC0 = MAT2 + RP * LDM;
  static constexpr int VEC1 = VEC0 + RP;
  static constexpr int VEC2 = VEC1 + RP;
  static constexpr int VEC3 = VEC2 + RP;
  static constexpr int SV = VEC3 + RP;
  static constexpr int PIV = SV + RoundUp<(DD_ * DD_ > 1 ? DD_ * DD_ : 1), 2>::value;
  static constexpr int SCR_RAW =
      RoundUp<PIV + 2 * ((2 * D > 4 * DD_ ? 2 * D : 4 * DD_) + 1), 4>::value;
  // group scratch size; PIT_SCR_SHIFT makes consecutive groups start G banks apart
  static constexpr int SCR = (PIT_SCR_SHIFT && sizeof(T) == 4)
                                 ? RoundUp<SCR_RAW, 32>::value + G_
                                 : SCR_RAW;
  // item sizes
  static constexpr int FA = 3 * D * D + 2 * D;   // filter element (A, b, C, eta, J)
  static constexpr int SA = 2 * D * D + D;       // smoothing element (E, g, L)
  static constexpr int F_A = 0, F_B = D * D, F_C = D * D + D, F_ETA = 2 * D * D + D,
                       F_J = 2 * D * D + 2 * D;
  static constexpr int S_E = 0, S_G = D * D, S_L = D * D + D;
  using GR = Grp<T, D, G_, RL_>;
};

// Per-point grid data (GRID kernels; the constants of IeksParams on a uniform grid).
template <typename T>
__device__ __forceinline__ T gp_T(const IeksParams<T>& p, int64_t n, int i) {
  return p.gst[n * p.SW + i];
}
template <typename T>
__device__ __forceinline__ T gp_scale(const IeksParams<T>& p, int64_t n, int i) {
  return p.gst[n * p.SW + (p.SW - 3) / 2 + i];
}
template <typename T>
__device__ __forceinline__ T gp_hq(const IeksParams<T>& p, int64_t n) {
  return p.gst[n * p.SW + p.SW - 3];
}
template <typename T>
__device__ __forceinline__ T gp_T0(const IeksParams<T>& p, int64_t n) {
  return p.gst[n * p.SW + p.SW - 2];
}
template <typename T>
__device__ __forceinline__ double gp_T0d(const IeksParams<T>& p, int64_t n) {
  return p.gsd[n * p.SW + p.SW - 2];
}
template <typename T>
__device__ __forceinline__ double gp_T1invd(const IeksParams<T>& p, int64_t n) {
  return p.gsd[n * p.SW + p.SW - 1];
}
template <typename T>
__device__ __forceinline__ double gp_scaled(const IeksParams<T>& p, int64_t n, int i) {
  return p.gsd[n * p.SW + (p.SW - 3) / 2 + i];
}
template <typename T>
__device__ __forceinline__ double gp_Td(const IeksParams<T>& p, int64_t n, int i) {
  return p.gsd[n * p.SW + i];
}

// Per-lane constant rows of Phibar and sqrt(Qbar) (I_d (x) blocks).
template <class C>
struct LaneConst {
  using T = typename C::Tp;
  T phirow[C::RL][C::Q1];  // Phibar1[r % Q1][j], j = 0..Q1-1 (row of the block)
  T sqrow[C::RL][C::D];    // row r of I_d (x) sqrt(Qbar1)
  int blk[C::RL];          // first row of r's block
  // non-uniform grid: the transition of the step into point n is Phibar diag(scale_n); the
  // unscaled rows are kept in base
  __device__ __forceinline__ void scale_step(const T (&base)[C::RL][C::Q1], const T (&sc)[C::Q1]) {
#pragma unroll
    for (int l = 0; l < C::RL; ++l)
#pragma unroll
      for (int j = 0; j < C::Q1; ++j) phirow[l][j] = base[l][j] * sc[j];
  }
  __device__ __forceinline__ void init(const typename C::GR& g, const IeksParams<T>& p) {
#pragma unroll
    for (int l = 0; l < C::RL; ++l) {
      const int r = g.row(l);
      const bool v = r < C::D;
      const int ir = v ? r % C::Q1 : 0;
      const int b = v ? (r / C::Q1) * C::Q1 : 0;
      blk[l] = b;
#pragma unroll
      for (int j = 0; j < C::Q1; ++j) phirow[l][j] = v ? p.phib[ir * kMaxQ1 + j] : T(0);
#pragma unroll
      for (int c = 0; c < C::D; ++c) {
        const int cb = (c / C::Q1) * C::Q1;
        const int jc = c % C::Q1;
        sqrow[l][c] = (v && cb == b && jc <= ir) ? p.sqb[ir * kMaxQ1 + jc] : T(0);
      }
    }
  }
};

// Linearisation of the information operator at trajectory row n (Section 3.2.1), returned in
// scaled preconditioned form: Ft = (h/q) F_y, dt = (f - F_y y) / T_1.
template <class C>
__device__ __forceinline__ void linearize_y(const IeksParams<typename C::Tp>& p,
                                            const typename C::Tp (&y)[C::DD],
                                            typename C::Tp (&Ft)[C::DD][C::DD],
                                            typename C::Tp (&dt)[C::DD]) {
  using T = typename C::Tp;
  T f[C::DD], F[C::DD][C::DD];
  ode_eval<T, C::DD>(p.ode, y, f, F);
  approximate_jacobian<T, C::DD>(p.lin_mode, F);
#pragma unroll
  for (int k = 0; k < C::DD; ++k) {
    T acc = f[k];
#pragma unroll
    for (int m = 0; m < C::DD; ++m) acc -= F[k][m] * y[m];
    dt[k] = acc * p.T1inv;
#pragma unroll
    for (int m = 0; m < C::DD; ++m) Ft[k][m] = F[k][m] * p.hq;
  }
}

template <class C>
__device__ __forceinline__ void linearize_at(const IeksParams<typename C::Tp>& p,
                                             const typename C::Tp* __restrict__ traj,
                                             int64_t n, typename C::Tp (&Ft)[C::DD][C::DD],
                                             typename C::Tp (&dt)[C::DD]) {
  typename C::Tp y[C::DD];
#pragma unroll
  for (int k = 0; k < C::DD; ++k) y[k] = p.T0 * traj[n * C::D + k * C::Q1];
  linearize_y<C>(p, y, Ft, dt);
}

// Row kk of Htilde X for X published in scratch (rows of length LDM).
template <class C>
__device__ __forceinline__ typename C::Tp hrow_entry(const typename C::Tp* X,
                                                     const typename C::Tp (&Ft)[C::DD][C::DD],
                                                     int kk, int c) {
  typename C::Tp v = X[(kk * C::Q1 + 1) * C::LDM + c];
#pragma unroll
  for (int m = 0; m < C::DD; ++m) v -= Ft[kk][m] * X[(m * C::Q1) * C::LDM + c];
  return v;
}

// Apply Phibar (block upper-triangular) to a published matrix: out[l][c] = (Phibar X)[r][c].
template <class C, int NC>
__device__ __forceinline__ void phi_rows(const LaneConst<C>& lc, const typename C::Tp* X,
                                         typename C::Tp (&out)[C::RL][NC]) {
#pragma unroll
  for (int l = 0; l < C::RL; ++l) {
#pragma unroll
    for (int c = 0; c < NC; ++c) out[l][c] = typename C::Tp(0);
#pragma unroll
    for (int j = 0; j < C::Q1; ++j) {
      const typename C::Tp ph = lc.phirow[l][j];
      const typename C::Tp* xr = X + (lc.blk[l] + j) * C::LDM;
#pragma unroll
      for (int c = 0; c < NC; ++c) out[l][c] += ph * xr[c];
    }
  }
}

template <class C>
__device__ __forceinline__ void phi_vec(const LaneConst<C>& lc, const typename C::Tp* x,
                                        typename C::Tp (&out)[C::RL]) {
#pragma unroll
  for (int l = 0; l < C::RL; ++l) {
    typename C::Tp acc = 0;
#pragma unroll
    for (int j = 0; j < C::Q1; ++j) acc += lc.phirow[l][j] * x[lc.blk[l] + j];
    out[l] = acc;
  }
}

// Square-root Kalman update in the scaled observation model (Psi-tria of Eq.
// sqrt-filtering-elements with sqrt(R) = 0).  Input: the lower-triangular predicted factor
// Lp (lane rows) already published at scr+MAT0 and the predicted mean published at scr+VEC0.
// Output: Psi21 columns -> K (gain rows), Psi22 -> sP_new (width W), sqrtS (all lanes),
// nu = dtilde - Htilde m- (all lanes).
template <class C>
struct UpdateOut {
  using T = typename C::Tp;
  T K[C::RL][C::DD];
  T sS[C::DD][C::DD];
  T rS[C::DD];   // reciprocals of sqrtS's diagonal
  T nu[C::DD];
};

template <class C>
__device__ __forceinline__ void sqrt_update(const typename C::GR& g, typename C::Tp* scr,
                                            const typename C::Tp (&Lp)[C::RL][C::D],
                                            const typename C::Tp (&Ft)[C::DD][C::DD],
                                            const typename C::Tp (&dt)[C::DD],
                                            typename C::Tp (&sPnew)[C::RL][C::W],
                                            UpdateOut<C>& u) {
  using T = typename C::Tp;
  constexpr int D = C::D, DD = C::DD, RL = C::RL;
  T U[2][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = g.row(l);
    // observation row r of Htilde Lp (lanes holding rows r < d); rows >= d stay zero
    const bool obs = r < DD;
    const int kk = obs ? r : 0;
    T Fr[DD];
#pragma unroll
    for (int m = 0; m < DD; ++m) {
      T f = T(0);
#pragma unroll
      for (int j = 0; j < DD; ++j) f = (j == kk) ? Ft[j][m] : f;
      Fr[m] = f;
    }
    const T* x1 = scr + C::MAT0 + (kk * C::Q1 + 1) * C::LDM;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      U[1][l][c] = Lp[l][c];
      T v = x1[c];
#pragma unroll
      for (int m = 0; m < DD; ++m) v -= Fr[m] * scr[C::MAT0 + (m * C::Q1) * C::LDM + c];
      U[0][l][c] = obs ? v : T(0);
    }
  }
#pragma unroll
  for (int kk = 0; kk < DD; ++kk) {
    T v = scr[C::VEC0 + kk * C::Q1 + 1];
#pragma unroll
    for (int m = 0; m < DD; ++m) v -= Ft[kk][m] * scr[C::VEC0 + m * C::Q1];
    u.nu[kk] = dt[kk] - v;
  }
  lq_dense<typename C::GR, 2, D, 0, DD, 0>(g, U, scr + C::PIV);
  // publish sqrtS (obs rows, first DD columns)
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = g.row(l);
#pragma unroll
    for (int kk = 0; kk < DD; ++kk)
      if (r == kk) {
#pragma unroll
        for (int c = 0; c < DD; ++c) scr[C::SV + kk * DD + c] = U[0][l][c];
      }
  }
  g.sync();
#pragma unroll
  for (int a = 0; a < DD; ++a)
#pragma unroll
    for (int b = 0; b < DD; ++b) u.sS[a][b] = (b <= a) ? scr[C::SV + a * DD + b] : T(0);
  g.sync();
#pragma unroll
  for (int a = 0; a < DD; ++a) u.rS[a] = recip<T>(u.sS[a][a]);
  // K = Psi21 sqrtS^-1 :  K[l] sqrtS = Psi21[l]  (backward substitution)
#pragma unroll
  for (int l = 0; l < RL; ++l) {
#pragma unroll
    for (int c = DD - 1; c >= 0; --c) {
      T acc = U[1][l][c];
#pragma unroll
      for (int k = c + 1; k < DD; ++k) acc -= u.K[l][k] * u.sS[k][c];
      u.K[l][c] = acc * u.rS[c];
    }
#pragma unroll
    for (int c = 0; c < C::W; ++c) sPnew[l][c] = U[1][l][DD + c];
  }
}

// Forward substitution with sqrtS: z = sqrtS^-1 x (rS: reciprocals of its diagonal).
template <class C>
__device__ __forceinline__ void solve_sS(const typename C::Tp (&sS)[C::DD][C::DD],
                                         const typename C::Tp (&rS)[C::DD],
                                         const typename C::Tp (&x)[C::DD],
                                         typename C::Tp (&z)[C::DD]) {
#pragma unroll
  for (int a = 0; a < C::DD; ++a) {
    typename C::Tp acc = x[a];
#pragma unroll
    for (int b = 0; b < a; ++b) acc -= sS[a][b] * z[b];
    z[a] = acc * rS[a];
  }
}

// =============================================================================================
// Full associative operators on items in shared memory (group-cooperative).
// =============================================================================================

template <class C, int SZ>
__device__ __forceinline__ void copy_item(const typename C::GR& g, const typename C::Tp* src,
                                          typename C::Tp* dst) {
  for (int i = g.gl; i < SZ; i += C::G) dst[i] = src[i];
}

// a_out = a_l (x)_f a_r   (Eq. sqrt-associative-filtering).  Items: [A | b | C | eta | J].
// C of the right operand and J of the left operand must be lower-triangular (true for every
// item the library produces: tria outputs, identity, triangularised inputs).
// a_out may alias a_r or a_l (writes happen after all reads).  VALUES_ONLY skips A, eta, J.
template <class C, bool VALUES_ONLY = false>
__device__ void combine_f(const typename C::GR& g, const typename C::Tp* al,
                          const typename C::Tp* ar, typename C::Tp* aout,
                          typename C::Tp* scr) {
  using T = typename C::Tp;
  constexpr int D = C::D, RL = C::RL, LDM = C::LDM;
  const T* Ai = al + C::F_A;
  const T* bi = al + C::F_B;
  const T* Ci = al + C::F_C;
  const T* ei = al + C::F_ETA;
  const T* Ji = al + C::F_J;
  const T* Aj = ar + C::F_A;
  const T* bj = ar + C::F_B;
  const T* Cj = ar + C::F_C;
  const T* ej = ar + C::F_ETA;
  const T* Jj = ar + C::F_J;
  int rr[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) rr[l] = g.valid(l) ? g.row(l) : 0;
  // A right operand with A_j = 0 (it contains the initial element of a segment) absorbs the
  // left one: (x) gives b_j, C_j, A = 0 whatever a_l holds.  Copying it keeps non-finite values
  // of another segment (0 * inf) out of this segment's values.
  {
    bool nz = false;
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) nz = nz || (g.valid(l) && !(Aj[rr[l] * D + c] == T(0)));
    if (!__any_sync(g.mask, nz)) {
      g.sync();
      if (aout != ar) copy_item<C, C::FA>(g, ar, aout);
      g.sync();
      return;
    }
  }
  // 1. Xi = tria([[Ci^T Jj, I], [Jj, 0]]).  tria is invariant under a permutation of the
  // columns, so the rows are taken as top [I | Ci^T Jj], bottom [0 | Jj]: a lower-triangular
  // block plus a dense block, which the structured LQ reduces with D reflections.  Afterwards
  // top = [Xi11 | 0], bottom = [Xi21 | R] with Xi22 = tria(R).
  T tri[2][RL][D], ext[2][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = rr[l];
    const bool v = g.valid(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const T w = sum4<T, D>([&](int kk) { return Ci[kk * D + r] * Jj[kk * D + c]; });
      tri[0][l][c] = (v && c == r) ? T(1) : T(0);
      ext[0][l][c] = v ? w : T(0);
      tri[1][l][c] = T(0);
      ext[1][l][c] = v ? Jj[r * D + c] : T(0);
    }
  }
  lq_tri_ext<typename C::GR, 2, D>(g, tri, ext, scr + C::PIV);
  T X11r[RL][D], X21r[RL][D], X22r[RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      X11r[l][c] = tri[0][l][c];
      X21r[l][c] = tri[1][l][c];
    }
  if constexpr (!VALUES_ONLY) {
    T Rm[1][RL][D];
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) Rm[0][l][c] = ext[1][l][c];
    lq_dense<typename C::GR, 1, D, 0, D, 0>(g, Rm, scr + C::PIV);
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) X22r[l][c] = Rm[0][l][c];
  }
  publish<typename C::GR, D, LDM>(g, X11r, scr + C::MAT0);
  publish<typename C::GR, D, LDM>(g, X21r, scr + C::MAT1);
  g.sync();
  // 2. M = Ci Xi11^-T (row r: solve M_r Xi11^T = Ci_r); Y = I - M Xi21^T
  T Mr[RL][D], Yr[RL][D];
  T rinv[D];
  inv_diag<D, LDM>(scr + C::MAT0, rinv);
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    T y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = Ci[rr[l] * D + c];
    solve_xLt<D, LDM>(scr + C::MAT0, rinv, y, Mr[l]);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Mr[l][k] * scr[C::MAT1 + c * LDM + k];
      Yr[l][c] = ((c == rr[l]) ? T(1) : T(0)) - acc;
    }
  }
  g.sync();
  // 3. U = Y Ai (rows), publish U -> MAT0, M -> MAT1
  T Ur[RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) acc += Yr[l][k] * Ai[k * D + c];
      Ur[l][c] = acc;
    }
  publish<typename C::GR, D, LDM>(g, Ur, scr + C::MAT0);
  publish<typename C::GR, D, LDM>(g, Mr, scr + C::MAT1);
  // vector t = Ci^T eta_j (entry r per lane)
  T tv[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Ci[k * D + rr[l]] * ej[k];
    tv[l] = acc;
  }
  publish_vec(g, tv, scr + C::VEC0);
  // s = Jj^T b_i (entry r)
  T sv[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Jj[k * D + rr[l]] * bi[k];
    sv[l] = acc;
  }
  publish_vec(g, sv, scr + C::VEC1);
  g.sync();
  // 4. new A row: Aj[r] U ; (Aj M) rows for C ; v = b_i + Ci t
  T Anew[RL][D], AjM[RL][D], vv[RL], uu[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = rr[l];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const T ajk = Aj[r * D + k];
        a1 += ajk * scr[C::MAT0 + k * LDM + c];
        a2 += ajk * scr[C::MAT1 + k * LDM + c];
      }
      Anew[l][c] = a1;
      AjM[l][c] = a2;
    }
    T acc = bi[r];
#pragma unroll
    for (int c = 0; c < D; ++c) acc += Ci[r * D + c] * scr[C::VEC0 + c];
    vv[l] = acc;
    T acc2 = ej[r];
#pragma unroll
    for (int c = 0; c < D; ++c) acc2 -= Jj[r * D + c] * scr[C::VEC1 + c];
    uu[l] = acc2;
  }
  g.sync();
  publish_vec(g, vv, scr + C::VEC2);
  publish_vec(g, uu, scr + C::VEC3);
  g.sync();
  // w = Y v (entry r), eta_new = U^T u + eta_i (entry r)
  T wv[RL], etan[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = rr[l];
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Yr[l][k] * scr[C::VEC2 + k];
    wv[l] = acc;
    T acc2 = ei[r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc2 += scr[C::MAT0 + k * LDM + r] * scr[C::VEC3 + k];
    etan[l] = acc2;
  }
  g.sync();
  publish_vec(g, wv, scr + C::VEC0);
  g.sync();
  T bnew[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = rr[l];
    T acc = bj[r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Aj[r * D + k] * scr[C::VEC0 + k];
    bnew[l] = acc;
  }
  // 5. sqrtC_new = tria([Cj | Aj M])  (Cj lower-triangular)
  T triC[1][RL][D], extC[1][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      triC[0][l][c] = g.valid(l) ? Cj[rr[l] * D + c] : T(0);
      extC[0][l][c] = g.valid(l) ? AjM[l][c] : T(0);
    }
  lq_tri_ext<typename C::GR, 1, D>(g, triC, extC, scr + C::PIV);
  // 6. sqrtJ_new = tria([Ji | Ai^T Xi22])  (Ji lower-triangular)
  T triJ[1][RL][D], extJ[1][RL][D];
  if constexpr (!VALUES_ONLY) {
    publish<typename C::GR, D, LDM>(g, X22r, scr + C::MAT1);
    g.sync();
#pragma unroll
    for (int l = 0; l < RL; ++l) {
      const int r = rr[l];
#pragma unroll
      for (int c = 0; c < D; ++c) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) acc += Ai[k * D + r] * scr[C::MAT1 + k * LDM + c];
        extJ[0][l][c] = g.valid(l) ? acc : T(0);
        triJ[0][l][c] = g.valid(l) ? Ji[r * D + c] : T(0);
      }
    }
    lq_tri_ext<typename C::GR, 1, D>(g, triJ, extJ, scr + C::PIV);
  }
  g.sync();
  // 7. write
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = rr[l];
#pragma unroll
    for (int c = 0; c < D; ++c) aout[C::F_C + r * D + c] = triC[0][l][c];
    aout[C::F_B + r] = bnew[l];
    if constexpr (!VALUES_ONLY) {
#pragma unroll
      for (int c = 0; c < D; ++c) {
        aout[C::F_A + r * D + c] = Anew[l][c];
        aout[C::F_J + r * D + c] = triJ[0][l][c];
      }
      aout[C::F_ETA + r] = etan[l];
    }
  }
  g.sync();
}

// b_out = b_l (x)_s b_r   (Eq. sqrt-associative-smoothing).  Items [E | g | L].
// L of the left operand must be lower-triangular.  WITH_L = false skips the L part.
template <class C, bool WITH_L>
__device__ void combine_s(const typename C::GR& g, const typename C::Tp* bl,
                          const typename C::Tp* br, typename C::Tp* bout,
                          typename C::Tp* scr) {
  using T = typename C::Tp;
  constexpr int D = C::D, RL = C::RL;
  const T* Ei = bl + C::S_E;
  const T* gi = bl + C::S_G;
  const T* Li = bl + C::S_L;
  const T* Ej = br + C::S_E;
  const T* gj = br + C::S_G;
  const T* Lj = br + C::S_L;
  int rr[RL];
#pragma unroll
  for (int l = 0; l < RL; ++l) rr[l] = g.valid(l) ? g.row(l) : 0;
  // A left operand with E_i = 0 (it contains the last element of a segment) absorbs the right
  // one; copying it keeps another segment's non-finite values out (see combine_f).
  {
    bool nz = false;
#pragma unroll
    for (int l = 0; l < RL; ++l)
#pragma unroll
      for (int c = 0; c < D; ++c) nz = nz || (g.valid(l) && !(Ei[rr[l] * D + c] == T(0)));
    if (!__any_sync(g.mask, nz)) {
      g.sync();
      if (bout != bl) copy_item<C, C::SA>(g, bl, bout);
      g.sync();
      return;
    }
  }
  T En[RL][D], gn[RL];
  T tri[1][RL][D], ext[1][RL][D];
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    const int r = rr[l];
    T acc = gi[r];
#pragma unroll
    for (int k = 0; k < D; ++k) acc += Ei[r * D + k] * gj[k];
    gn[l] = acc;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      T a1 = T(0), a2 = T(0);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        a1 += Ei[r * D + k] * Ej[k * D + c];
        if constexpr (WITH_L) a2 += Ei[r * D + k] * Lj[k * D + c];
      }
      En[l][c] = a1;
      ext[0][l][c] = g.valid(l) ? a2 : T(0);
      tri[0][l][c] = (WITH_L && g.valid(l)) ? Li[r * D + c] : T(0);
    }
  }
  if constexpr (WITH_L) lq_tri_ext<typename C::GR, 1, D>(g, tri, ext, scr + C::PIV);
  g.sync();
#pragma unroll
  for (int l = 0; l < RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = rr[l];
#pragma unroll
    for (int c = 0; c < D; ++c) {
      bout[C::S_E + r * D + c] = En[l][c];
      if constexpr (WITH_L) bout[C::S_L + r * D + c] = tri[0][l][c];
    }
    bout[C::S_G + r] = gn[l];
  }
  g.sync();
}

template <class C>
__device__ __forceinline__ void set_identity_f(const typename C::GR& g, typename C::Tp* a) {
  constexpr int D = C::D;
#pragma unroll
  for (int l = 0; l < C::RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      a[C::F_A + r * D + c] = (c == r) ? 1 : 0;
      a[C::F_C + r * D + c] = 0;
      a[C::F_J + r * D + c] = 0;
    }
    a[C::F_B + r] = 0;
    a[C::F_ETA + r] = 0;
  }
}

template <class C>
__device__ __forceinline__ void set_identity_s(const typename C::GR& g, typename C::Tp* b) {
  constexpr int D = C::D;
#pragma unroll
  for (int l = 0; l < C::RL; ++l) {
    if (!g.valid(l)) continue;
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      b[C::S_E + r * D + c] = (c == r) ? 1 : 0;
      b[C::S_L + r * D + c] = 0;
    }
    b[C::S_G + r] = 0;
  }
}


}  // namespace pit
