// curve_sphere.cuh — the 3-manifold of Example 3: the Fourier-embedded circle
// times a sphere, M = C(S^1) x S^2(a) in R^9,
//   C(phi) = R (cos phi, sin phi, cos 2phi / 2, sin 2phi / 2, cos 3phi / 3, sin 3phi / 3).
//   - closest point: the two factors separately; on the curve Newton's method on
//     C'(phi).(C(phi) - xh) = 0 from the angle of (x_1, x_2), on the sphere
//     normalisation to radius a;
//   - the data u = sum_t T_t(q_t phi) S_t(w), S_t = c_t + v_t.w + w^T A_t w, w the
//     unit vector of the sphere factor, and (-Delta_M + sigma) u in closed form:
//     the curve has constant speed sqrt(3) R, so -Delta_curve T(q phi) =
//     q^2 T / (3 R^2); on S^2(a) v.w has eigenvalue 2/a^2 and the trace-free part
//     of w^T A w 6/a^2.
#pragma once
#include <cmath>
#include "dev_common.cuh"

namespace mpwos {

template <typename T>
__device__ __forceinline__ void cs_sincos(T x, T& s, T& c) {
  if constexpr (sizeof(T) == 8) { s = sin(x); c = cos(x); } else { __sincosf(x, &s, &c); }
}

template <typename T>
__device__ __forceinline__ void fourier_curve(T R, T ph, T* C, T* C1, T* C2) {
#pragma unroll
  for (int k = 1; k <= 3; ++k) {
    T s, c;
    cs_sincos<T>(T(k) * ph, s, c);
    C[2 * k - 2] = R * c / T(k);
    C[2 * k - 1] = R * s / T(k);
    C1[2 * k - 2] = -R * s;
    C1[2 * k - 1] = R * c;
    C2[2 * k - 2] = -R * T(k) * c;
    C2[2 * k - 1] = -R * T(k) * s;
  }
}

// phi of the nearest curve point to x[0..5]: Newton's method from the angle of
// (x_1, x_2); where |C'|^2 + C''.(C - x) falls below 0.1 |C'|^2 the Gauss-Newton
// derivative |C'|^2 is used; stops at a step below tol (1 + |phi|) (1e-15 in
// FP64; 1e-6 in FP32, whose fast sine and cosine carry ~1e-6 absolute error) or
// after 60 (FP32: 16) steps.
template <typename T>
__device__ __forceinline__ T curve_cp_phi(T R, const T* x) {
  constexpr bool f64 = sizeof(T) == 8;
  const T tol = f64 ? T(1e-15) : T(1e-6);
  const int maxit = f64 ? 60 : 16;
  T ph = atan2(x[1], x[0]);
  for (int it = 0; it < maxit; ++it) {
    T C[6], C1[6], C2[6];
    fourier_curve<T>(R, ph, C, C1, C2);
    T F = T(0), g2 = T(0), h = T(0);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      F += C1[i] * (C[i] - x[i]);
      g2 += C1[i] * C1[i];
      h += C2[i] * (C[i] - x[i]);
    }
    T J = g2 + h;
    if (!(J > T(0.1) * g2)) J = g2;
    const T pn = ph - F / J;
    if (fabs(pn - ph) <= tol * (T(1) + fabs(ph))) { ph = pn; break; }
    ph = pn;
  }
  return ph;
}

// cp(x) for x in R^9
template <typename T>
__device__ __forceinline__ void curve_sphere_cp(T R, T a, const T* x, T* out) {
  const T ph = curve_cp_phi<T>(R, x);
  T C[6], C1[6], C2[6];
  fourier_curve<T>(R, ph, C, C1, C2);
#pragma unroll
  for (int i = 0; i < 6; ++i) out[i] = C[i];
  const T ns = sqrt(x[6] * x[6] + x[7] * x[7] + x[8] * x[8]);
#pragma unroll
  for (int i = 6; i < 9; ++i) out[i] = x[i] * (a / ns);
}

// u or (-Delta_M + sigma) u at y on M; v, A: 3 and 9 entries per term.
template <typename T>
__device__ __forceinline__ T curve_sphere_value(const DevFunc& fn, const T* v, const T* A, T R, T a, T sigma,
                                                const T* y) {
  const T ph = atan2(y[1], y[0]);
  const T ns = sqrt(y[6] * y[6] + y[7] * y[7] + y[8] * y[8]);
  const T w[3] = {y[6] / ns, y[7] / ns, y[8] / ns};
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    const int q = fn.modes[t][0];
    const T* vt = v + 3 * t;
    const T* At = A + 9 * t;
    const T lin = vt[0] * w[0] + vt[1] * w[1] + vt[2] * w[2];
    T quad = T(0);
    const T tr = At[0] + At[4] + At[8];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) quad += At[3 * i + j] * w[i] * w[j];
    const T St = pick<T>(fn.coef[t], fn.coef_f[t]) + lin + quad;
    T s, c;
    cs_sincos<T>(T(q) * ph, s, c);
    const T Tv = fn.modes[t][1] == 0 ? c : s;
    if (!fn.apply_op) {
      total += Tv * St;
    } else {
      const T a2 = a * a;
      const T lap = T(q * q) / (T(3) * R * R) * St + T(2) / a2 * lin + T(6) / a2 * (quad - tr / T(3));
      total += Tv * (lap + sigma * St);
    }
  }
  return total;
}

}  // namespace mpwos
