// Group-cooperative dense linear algebra on small square-root factors.
//
// A *group* is G consecutive lanes of one warp that work on one sequential chain of time steps
// or on one associative combine.  Every D-row matrix is distributed by rows: lane `gl` of the
// group owns rows gl*RL .. gl*RL+RL-1 and keeps them in registers.  Rows >= D (padding rows of
// the last lane) exist, stay zero and are never written to global memory.  Matrices that other
// lanes need are *published* to the group's shared-memory scratch, then read back after a
// warp barrier.
//
// The triangularisation tria(M) of Section 3.1.2 (QR of M^T, return R^T) is computed here as
// the equivalent LQ factorisation of M by Householder reflections from the right, one pivot row
// at a time: reflection i annihilates the entries of row i to the right of column i.  Two
// variants exploit the structure that occurs in the solver:
//   lq_tri_ext  -- M = [L | X] with L lower-triangular (D x D) and X dense (D x NE): reflection
//                  i touches only column i and the NE columns of X;
//   lq_dense    -- general pivot rows with support from the pivot column to the last column.
// Diagonal signs of the factors are left as the reflections produce them; every consumer only
// uses S S^T or solves with the (non-singular) factor, so the sign freedom of tria (its
// factor is unique only up to column signs) does not matter.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pit {

#ifndef PIT_RECIP_MODE
#define PIT_RECIP_MODE 2
#endif

// Reciprocal used by the reflections and triangular solves.  FP32: 0 = IEEE division,
// 1 = the correctly rounded reciprocal intrinsic (__frcp_rn), 2 = the fast approximate division
// intrinsic (__fdividef, about 2 ulp; measured 12% faster per FitzHugh-Nagumo iteration than 0
// or 1, well inside the FP32 rounding the scans carry anyway).  FP64 always divides.
template <typename T>
__device__ __forceinline__ T recip(T x) {
  return T(1) / x;
}
template <>
__device__ __forceinline__ float recip<float>(float x) {
#if PIT_RECIP_MODE == 1
  return __frcp_rn(x);
#elif PIT_RECIP_MODE == 2
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

#ifndef PIT_SQRT_MODE
#define PIT_SQRT_MODE 2
#endif

template <typename T>
__device__ __forceinline__ T dsqrt(T x);
// FP32 square root of the reflections' norms: 1 = IEEE sqrtf, 2 = x * rsqrtf(x) (about 2 ulp;
// the callers pass x in the safe range [1e-30, 1e30])
template <>
__device__ __forceinline__ float dsqrt<float>(float x) {
#if PIT_SQRT_MODE == 2
  return x * rsqrtf(x);
#else
  return sqrtf(x);
#endif
}
template <>
__device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <int N, int A>
struct RoundUp {
  static constexpr int value = ((N + A - 1) / A) * A;
};

// sum_{j<N} f(j) with four independent partial sums: shortens the dependent multiply-add chain
// of dot products and norms (the summation order differs from a left fold).
template <typename T, int N, class F>
__device__ __forceinline__ T sum4(F f) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    a0 += f(j);
    if (j + 1 < N) a1 += f(j + 1);
    if (j + 2 < N) a2 += f(j + 2);
    if (j + 3 < N) a3 += f(j + 3);
  }
  return (a0 + a1) + (a2 + a3);
}

// Group geometry.  D rows, G lanes, RL rows per lane.
template <typename T, int D_, int G_, int RL_>
struct Grp {
  static constexpr int D = D_;
  static constexpr int G = G_;
  static constexpr int RL = RL_;
  static constexpr int RP = G_ * RL_;  // padded row count
  static_assert(G_ * RL_ >= D_, "group too small for D");
  static_assert(32 % G_ == 0, "group size must divide 32");
  int gl;         // lane index inside the group
  unsigned mask;  // lanes of this group within the warp
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
  __device__ __forceinline__ void init() {
    const int lane = threadIdx.x & 31;
    gl = lane % G_;
    const unsigned base = (G_ == 32) ? 0xffffffffu : ((1u << G_) - 1u);
    mask = (G_ == 32) ? base : (base << (lane - gl));
  }
  __device__ __forceinline__ int row(int l) const { return gl * RL_ + l; }
  __device__ __forceinline__ bool valid(int l) const { return gl * RL_ + l < D_; }
};

// Publish RL rows of an NC-column register matrix into scratch with leading dimension LD.
template <class GR, int NC, int LD, typename T>
__device__ __forceinline__ void publish(const GR& g, const T (&x)[GR::RL][NC], T* buf) {
#pragma unroll
  for (int l = 0; l < GR::RL; ++l) {
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < NC; ++c) buf[r * LD + c] = x[l][c];
  }
}

// Publish the first NC columns of RL rows stored with NX >= NC columns.
template <class GR, int NC, int LD, int NX, typename T>
__device__ __forceinline__ void publish_cols(const GR& g, const T (&x)[GR::RL][NX], T* buf) {
  static_assert(NC <= NX, "too many columns");
#pragma unroll
  for (int l = 0; l < GR::RL; ++l) {
    const int r = g.row(l);
#pragma unroll
    for (int c = 0; c < NC; ++c) buf[r * LD + c] = x[l][c];
  }
}

template <class GR, typename T>
__device__ __forceinline__ void publish_vec(const GR& g, const T (&x)[GR::RL], T* buf) {
#pragma unroll
  for (int l = 0; l < GR::RL; ++l) buf[g.row(l)] = x[l];
}

// One Householder reflection from the right, normalised as in LAPACK's larfg: for the pivot
// row x = (x0, xe) it returns beta = -sign(x0) ||x||, tau = (beta - x0) / beta in [1, 2] and
// w = 1 / (x0 - beta), so that v = (1, w xe) and (I - tau v v^T) maps x to (beta, 0, ..., 0).
// With v0 = 1 and |w xe_j| <= 1 nothing overflows even when ||x|| is tiny (rank-deficient
// factors leave round-off-sized pivots).  ||x|| is computed with scaling when x0^2 + sum xe^2
// leaves the safe range of T.  A row y is transformed as
//   f = tau (y0 + w sum_j y_j xe_j),  y0 -= f,  y_j -= (f w) xe_j.
template <typename T>
struct Reflector {
  T beta, tau, w;
  bool active;
};

template <typename T>
struct SafeRange;
template <>
struct SafeRange<float> {
  static constexpr float lo = 1e-30f, hi = 1e30f;
};
template <>
struct SafeRange<double> {
  static constexpr double lo = 1e-280, hi = 1e280;
};

template <typename T, int NE, class GetX>
__device__ __forceinline__ Reflector<T> make_reflector_g(T x0, GetX xe) {
  T sig = sum4<T, NE>([&](int j) { return xe(j) * xe(j); });
  Reflector<T> h;
  T ss = x0 * x0 + sig;
  T nrm;
  if (ss > SafeRange<T>::lo && ss < SafeRange<T>::hi) {
    nrm = dsqrt<T>(ss);
  } else {
    T amax = fabs(x0);
#pragma unroll
    for (int j = 0; j < NE; ++j) amax = fmax(amax, fabs(xe(j)));
    if (amax > T(0)) {
      const T inv = T(1) / amax;
      T acc = (x0 * inv) * (x0 * inv);
#pragma unroll
      for (int j = 0; j < NE; ++j) acc += (xe(j) * inv) * (xe(j) * inv);
      nrm = amax * dsqrt<T>(acc);
    } else {
      nrm = T(0);
    }
    sig = (nrm > fabs(x0)) ? T(1) : T(0);  // only its sign (> 0) is used below
  }
  h.active = sig > T(0) && nrm > T(0);
  h.beta = (x0 >= T(0)) ? -nrm : nrm;
  h.tau = h.active ? (h.beta - x0) * recip<T>(h.beta) : T(0);
  h.w = h.active ? recip<T>(x0 - h.beta) : T(0);
  return h;
}

template <typename T, int NE>
__device__ __forceinline__ Reflector<T> make_reflector(T x0, const T (&xe)[NE]) {
  return make_reflector_g<T, NE>(x0, [&](int j) { return xe[j]; });
}

// ---- structured LQ: [L | X], L lower-triangular ------------------------------------------
// NS row sets; set 0 provides the D pivots.  tri[s][l][*] are the D "triangular" columns and
// ext[s][l][*] the NE extra columns of row (s, l).  After the call, set 0 holds the
// lower-triangular factor in tri and zeros in ext; the other sets hold the transformed rows.
// `piv` is group scratch of at least 2*(NE+1) elements.
template <class GR, int NS, int NE, typename T>
__device__ __forceinline__ void lq_tri_ext(const GR& g, T (&tri)[NS][GR::RL][GR::D],
                                           T (&ext)[NS][GR::RL][NE], T* piv) {
  constexpr int D = GR::D;
  constexpr int RL = GR::RL;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const int owner = i / RL;
    const int li = i % RL;
    T* pb = piv + (i & 1) * (NE + 1);
    if (g.gl == owner) {
#pragma unroll
      for (int l = 0; l < RL; ++l) {
        if (l == li) {
          pb[0] = tri[0][l][i];
#pragma unroll
          for (int j = 0; j < NE; ++j) pb[1 + j] = ext[0][l][j];
        }
      }
    }
    g.sync();
    T x0 = pb[0];
    T xe[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) xe[j] = pb[1 + j];
    const Reflector<T> h = make_reflector<T, NE>(x0, xe);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int l = 0; l < RL; ++l) {
        const T acc = sum4<T, NE>([&](int j) { return ext[s][l][j] * xe[j]; });
        const T f = h.tau * (tri[s][l][i] + h.w * acc);
        const T fw = f * h.w;
        tri[s][l][i] -= f;
#pragma unroll
        for (int j = 0; j < NE; ++j) ext[s][l][j] -= fw * xe[j];
        if (s == 0 && l == li && g.gl == owner && h.active) {
          tri[s][l][i] = h.beta;
#pragma unroll
          for (int j = 0; j < NE; ++j) ext[s][l][j] = T(0);
        }
      }
    }
  }
  g.sync();
}

// ---- dense LQ ----------------------------------------------------------------------------
// Rows of NS sets with NC columns each.  Pivot rows k = 0..NPIV-1 of set PS, pivot column
// PC0 + k, support columns PC0+k .. NC-1.  Every row of every set is transformed; after the
// call pivot row k is (..., beta_k at column PC0+k, 0, ..., 0).
template <class GR, int NS, int NC, int PS, int NPIV, int PC0, typename T>
__device__ __forceinline__ void lq_dense(const GR& g, T (&rows)[NS][GR::RL][NC], T* piv) {
  constexpr int RL = GR::RL;
  static_assert(PC0 + NPIV <= NC, "pivot columns out of range");
#pragma unroll
  for (int k = 0; k < NPIV; ++k) {
    const int c0 = PC0 + k;
    const int owner = k / RL;
    const int lk = k % RL;
    T* pb = piv + (k & 1) * NC;
    if (g.gl == owner) {
#pragma unroll
      for (int l = 0; l < RL; ++l) {
        if (l == lk) {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (c >= c0) pb[c] = rows[PS][l][c];
        }
      }
    }
    g.sync();
    T x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) x[c] = (c > c0) ? pb[c] : T(0);
    const T x0 = pb[c0];
    const Reflector<T> h = make_reflector_g<T, NC>(x0, [&](int j) { return x[j]; });
#pragma unroll
    for (int s = 0; s < NS; ++s) {
#pragma unroll
      for (int l = 0; l < RL; ++l) {
        const T acc = sum4<T, NC>([&](int c) { return (c > c0) ? rows[s][l][c] * x[c] : T(0); });
        const T f = h.tau * (rows[s][l][c0] + h.w * acc);
        const T fw = f * h.w;
        rows[s][l][c0] -= f;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c > c0) rows[s][l][c] -= fw * x[c];
        if (s == PS && l == lk && g.gl == owner && h.active) {
          rows[s][l][c0] = h.beta;
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (c > c0) rows[s][l][c] = T(0);
        }
      }
    }
  }
  g.sync();
}

// ---- small helpers -------------------------------------------------------------------------
// Reciprocals of the diagonal of a D x D matrix in scratch (ld LD); computed once so that the
// substitutions below run on multiply-adds only.
template <int D, int LD, typename T>
__device__ __forceinline__ void inv_diag(const T* Lm, T (&rinv)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) rinv[c] = recip<T>(Lm[c * LD + c]);
}

// Solve x * L^T = y for x (row vector), L lower-triangular D x D in scratch (ld LD):
//   x[c] = (y[c] - sum_{k<c} x[k] L[c][k]) / L[c][c]     (forward substitution)
template <int D, int LD, typename T>
__device__ __forceinline__ void solve_xLt(const T* Lm, const T (&rinv)[D], const T (&y)[D],
                                          T (&x)[D]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const T acc = y[c] - sum4<T, D>([&](int k) { return (k < c) ? x[k] * Lm[c * LD + k] : T(0); });
    x[c] = acc * rinv[c];
  }
}

// Solve x * L = y for x (row vector), L lower-triangular:
//   x[c] = (y[c] - sum_{k>c} x[k] L[k][c]) / L[c][c]      (backward substitution)
template <int D, int LD, typename T>
__device__ __forceinline__ void solve_xL(const T* Lm, const T (&rinv)[D], const T (&y)[D],
                                         T (&x)[D]) {
#pragma unroll
  for (int c = D - 1; c >= 0; --c) {
    const T acc = y[c] - sum4<T, D>([&](int k) { return (k > c) ? x[k] * Lm[k * LD + c] : T(0); });
    x[c] = acc * rinv[c];
  }
}

// Non-negative floating point values as monotone unsigned integers (for atomicMax).
__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr),
            static_cast<unsigned long long>(__double_as_longlong(v)));
}

}  // namespace pit
