// Device-side vector fields f(y) and Jacobians F_y(y) of the supported ODE families.
// Parameter layouts are those of pit.h (pit_ode_kind).  All families are autonomous
// polynomial vector fields, so no transcendental function is evaluated here.
#pragma once

#include <cuda_runtime.h>

namespace pit {

constexpr int kMaxParams = 32;

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
    default:
      break;
  }
}

}  // namespace pit
