// Device-side vector fields f(y) and Jacobians F_y(y) of the supported ODE families.
// Parameter layouts are those of pit.h (pit_ode_kind).  All families are autonomous
// polynomial vector fields, so no transcendental function is evaluated here.
#pragma once

#include <cuda_runtime.h>

namespace pit {

constexpr int kMaxParams = 32;
// Internal family code of the components of a decoupled solve (approximate Jacobians): the
// solver passes the precomputed diagonal Jacobian entry in place of the state.
constexpr int kOdeDiagJacobian = 100;

template <typename T>
struct OdeParams {
  int kind;
  int d;
  T p[kMaxParams];
};

// y: DD values (original coordinates).  Writes f (DD) and F (DD x DD, row-major).
template <typename T, int DD>
__device__ __forceinline__ void ode_eval(const OdeParams<T>& P, const T (&y)[DD], T (&f)[DD],
                                         T (&F)[DD][DD]) {
#pragma unroll
  for (int i = 0; i < DD; ++i) {
    f[i] = T(0);
#pragma unroll
    for (int j = 0; j < DD; ++j) F[i][j] = T(0);
  }
  switch (P.kind) {
    case 0: {  // logistic
      if constexpr (DD == 1) {
        const T r = P.p[0];
        f[0] = r * y[0] * (T(1) - y[0]);
        F[0][0] = r * (T(1) - T(2) * y[0]);
      }
      break;
    }
    case 1: {  // FitzHugh-Nagumo
      if constexpr (DD == 2) {
        const T a = P.p[0], b = P.p[1], c = P.p[2];
        const T v = y[0], w = y[1];
        f[0] = c * (v - v * v * v / T(3) + w);
        f[1] = -(v - a + b * w) / c;
        F[0][0] = c * (T(1) - v * v);
        F[0][1] = c;
        F[1][0] = T(-1) / c;
        F[1][1] = -b / c;
      }
      break;
    }
    case 2: {  // Lotka-Volterra
      if constexpr (DD == 2) {
        const T al = P.p[0], be = P.p[1], ga = P.p[2], de = P.p[3];
        const T x = y[0], z = y[1];
        f[0] = al * x - be * x * z;
        f[1] = de * x * z - ga * z;
        F[0][0] = al - be * z;
        F[0][1] = -be * x;
        F[1][0] = de * z;
        F[1][1] = de * x - ga;
      }
      break;
    }
    case 4: {  // affine y' = L y + c
      const T* L = P.p;
      const T* c = P.p + DD * DD;
#pragma unroll
      for (int i = 0; i < DD; ++i) {
        T acc = c[i];
#pragma unroll
        for (int j = 0; j < DD; ++j) {
          acc += L[i * DD + j] * y[j];
          F[i][j] = L[i * DD + j];
        }
        f[i] = acc;
      }
      break;
    }
    case 5: {  // rigid body
      if constexpr (DD == 3) {
        f[0] = T(-2) * y[1] * y[2];
        f[1] = T(1.25) * y[0] * y[2];
        f[2] = T(-0.5) * y[0] * y[1];
        F[0][1] = T(-2) * y[2];
        F[0][2] = T(-2) * y[1];
        F[1][0] = T(1.25) * y[2];
        F[1][2] = T(1.25) * y[0];
        F[2][0] = T(-0.5) * y[1];
        F[2][1] = T(-0.5) * y[0];
      }
      break;
    }
    case 6: {  // Van der Pol
      if constexpr (DD == 2) {
        const T mu = P.p[0];
        f[0] = y[1];
        f[1] = mu * ((T(1) - y[0] * y[0]) * y[1] - y[0]);
        F[0][1] = T(1);
        F[1][0] = mu * (T(-2) * y[0] * y[1] - T(1));
        F[1][1] = mu * (T(1) - y[0] * y[0]);
      }
      break;
    }
    case kOdeDiagJacobian:  // component of a decoupled solve: y[0] carries dF_kk/dy_k
      if constexpr (DD == 1) F[0][0] = y[0];
      break;
    default:
      break;
  }
}

}  // namespace pit

// ---------------------------------------------------------------------------------------------
// Trajectory arithmetic.  The linearisation trajectory and the residuals of the increment model
// are kept in FP64 for both solvers (the FP32 solver runs only its scans in FP32).  The helpers
// below are the conversions the kernels use between the trajectory type V and the arithmetic
// type T of the scans.
// ---------------------------------------------------------------------------------------------
namespace pit {

template <typename V>
__device__ __forceinline__ V v_from_double(double x);
template <>
__device__ __forceinline__ double v_from_double<double>(double x) { return x; }
__device__ __forceinline__ double v_to_double(double x) { return x; }
__device__ __forceinline__ double v_add_small(double x, double d) { return x + d; }
template <typename V>
__device__ __forceinline__ V v_from_zero() {
  return v_from_double<V>(0.0);
}
// round a trajectory value to the arithmetic type T of the scans
template <typename T>
__device__ __forceinline__ T v_to_T(double x) {
  return static_cast<T>(x);
}

// Constants of the vector field in the trajectory number type V.
template <typename V>
struct OdeConstsV {
  int kind;
  V k[8];
  V L[12];  // affine (d <= 3): L (d x d) then c (d)
};

// Vector field f(y) in number type V (no Jacobian); parameter layouts as in pit.h.
template <typename V, int DD>
__device__ __forceinline__ void ode_f_v(const OdeConstsV<V>& P, const V (&y)[DD], V (&f)[DD]) {
  switch (P.kind) {
    case 0:
      if constexpr (DD == 1) f[0] = P.k[0] * y[0] - P.k[0] * (y[0] * y[0]);
      break;
    case 1:  // k = [a, b, c, 1/c, 1/3]
      if constexpr (DD == 2) {
        const V v3 = y[0] * y[0] * y[0];
        f[0] = P.k[2] * (y[0] - v3 * P.k[4] + y[1]);
        f[1] = -((y[0] - P.k[0] + P.k[1] * y[1]) * P.k[3]);
      }
      break;
    case 2:  // k = [al, be, ga, de]
      if constexpr (DD == 2) {
        const V xz = y[0] * y[1];
        f[0] = P.k[0] * y[0] - P.k[1] * xz;
        f[1] = P.k[3] * xz - P.k[2] * y[1];
      }
      break;
    case 4:
#pragma unroll
      for (int i = 0; i < DD; ++i) {
        V acc = P.L[DD * DD + i];
#pragma unroll
        for (int j = 0; j < DD; ++j) acc = acc + P.L[i * DD + j] * y[j];
        f[i] = acc;
      }
      break;
    case 5:  // k = [-2, 1.25, -0.5]
      if constexpr (DD == 3) {
        f[0] = P.k[0] * (y[1] * y[2]);
        f[1] = P.k[1] * (y[0] * y[2]);
        f[2] = P.k[2] * (y[0] * y[1]);
      }
      break;
    case 6:  // k = [mu, 1]
      if constexpr (DD == 2) {
        f[0] = y[1];
        f[1] = P.k[0] * ((P.k[1] - y[0] * y[0]) * y[1] - y[0]);
      }
      break;
    default:
      break;
  }
}

template <typename V, typename T, int DD>
__device__ __forceinline__ void ode_consts_v(const OdeParams<T>& P, const double* pd,
                                             OdeConstsV<V>& c) {
  c.kind = P.kind;
  switch (P.kind) {
    case 0: c.k[0] = v_from_double<V>(pd[0]); break;
    case 1:
      c.k[0] = v_from_double<V>(pd[0]);
      c.k[1] = v_from_double<V>(pd[1]);
      c.k[2] = v_from_double<V>(pd[2]);
      c.k[3] = v_from_double<V>(1.0 / pd[2]);
      c.k[4] = v_from_double<V>(1.0 / 3.0);
      break;
    case 2:
      for (int i = 0; i < 4; ++i) c.k[i] = v_from_double<V>(pd[i]);
      break;
    case 4:
      for (int i = 0; i < DD * DD + DD; ++i) c.L[i] = v_from_double<V>(pd[i]);
      break;
    case 5:
      c.k[0] = v_from_double<V>(-2.0);
      c.k[1] = v_from_double<V>(1.25);
      c.k[2] = v_from_double<V>(-0.5);
      break;
    case 6:
      c.k[0] = v_from_double<V>(pd[0]);
      c.k[1] = v_from_double<V>(1.0);
      break;
    default: break;
  }
}


// Component k of the vector field f(y) of a d-dimensional problem, in number type V, with the
// state read through y(j) (decoupled solves).  Families with d <= 3 evaluate the full field;
// Lorenz-96 reads its three neighbours only.
template <typename V, typename T, typename Get>
__device__ __forceinline__ V component_f(int kind, const double* pd, int d, int k, Get y) {
  if (kind == 3) {  // Lorenz-96: (y_{k+1} - y_{k-2}) y_{k-1} - y_k + F
    const V a = y((k + 1) % d), b = y((k - 2 + d) % d), c = y((k - 1 + d) % d);
    return (a - b) * c - y(k) + v_from_double<V>(pd[0]);
  }
  OdeParams<T> P;
  P.kind = kind;
  P.d = d;
  V out = v_from_zero<V>();
  if (d == 1) {
    OdeConstsV<V> oc;
    ode_consts_v<V, T, 1>(P, pd, oc);
    V yy[1] = {y(0)}, f[1];
    ode_f_v<V, 1>(oc, yy, f);
    out = f[0];
  } else if (d == 2) {
    OdeConstsV<V> oc;
    ode_consts_v<V, T, 2>(P, pd, oc);
    V yy[2] = {y(0), y(1)}, f[2];
    ode_f_v<V, 2>(oc, yy, f);
    out = f[k];
  } else if (d == 3) {
    OdeConstsV<V> oc;
    ode_consts_v<V, T, 3>(P, pd, oc);
    V yy[3] = {y(0), y(1), y(2)}, f[3];
    ode_f_v<V, 3>(oc, yy, f);
    out = f[k];
  }
  return out;
}

// Diagonal entry dF_kk/dy_k of the Jacobian (arithmetic type T), state through y(j).
template <typename T, typename Get>
__device__ __forceinline__ T component_jac_diag(int kind, const double* pd, int d, int k, Get y) {
  if (kind == 3) return T(-1);  // Lorenz-96
  OdeParams<T> P;
  P.kind = kind;
  P.d = d;
#pragma unroll
  for (int i = 0; i < 12; ++i) P.p[i] = static_cast<T>(pd[i]);
  if (d == 1) {
    T yy[1] = {y(0)}, f[1], F[1][1];
    ode_eval<T, 1>(P, yy, f, F);
    return F[0][0];
  } else if (d == 2) {
    T yy[2] = {y(0), y(1)}, f[2], F[2][2];
    ode_eval<T, 2>(P, yy, f, F);
    return F[k][k];
  } else if (d == 3) {
    T yy[3] = {y(0), y(1), y(2)}, f[3], F[3][3];
    ode_eval<T, 3>(P, yy, f, F);
    return F[k][k];
  }
  return T(0);
}

// The Jacobian used by the linearisation (Section 3.2.1, remark on approximate Jacobians):
// exact, its diagonal, or zero.
template <typename T, int DD>
__device__ __forceinline__ void approximate_jacobian(int mode, T (&F)[DD][DD]) {
  if (mode == 0) return;
#pragma unroll
  for (int i = 0; i < DD; ++i)
#pragma unroll
    for (int j = 0; j < DD; ++j)
      if (mode == 2 || i != j) F[i][j] = T(0);
}

}  // namespace pit
