// revolution.cuh — the hypersurface of revolution about the last axis of
// Example 2: M = {x = (xh, t) in R^n : |xh| = R(t)}, with the dumbbell profile
//   R(t) = sqrt(1 - s^2) (1 - al + 2 al s^2),  s = t / k.
// Host and device (the host scans the curvature for the radius range).
//   - closest point: x's meridian half-plane holds it; t minimises
//     D(t) = (R(t) - rho0)^2 + (t - t0)^2, found by Newton's method on
//     D'/2 = (R - rho0) R' + (t - t0) from t0 (the paper's local Newton
//     iteration in the profile parameter);
//   - curvature indicator (eq. rho_geo_curvature): the largest absolute
//     principal curvature, max(|R''| / G^3, 1 / (R G)), G = sqrt(1 + R'^2);
//   - the data u = c0 + c1 t + c2 t^2 + v.xh + sum_j A_j xh_j^2 and its source
//     (-Delta_M + sigma) u in closed form (degree-0, 1, 2 spherical harmonics of
//     the unit vector w = xh/|xh| on S^{n-2}).
#pragma once
#include <cmath>
#include "dev_common.cuh"

namespace mpwos {

template <typename T> struct Profile { T R, R1, R2; };

template <typename T>
__host__ __device__ __forceinline__ Profile<T> rev_profile(T t, T al, T k) {
  const T s = t / k;
  const T w = sqrt(T(1) - s * s);
  const T q = T(1) - al + T(2) * al * s * s;
  const T dw = -s / w, ddw = T(-1) / (w * w * w);
  const T dq = T(4) * al * s, ddq = T(4) * al;
  Profile<T> P;
  P.R = w * q;
  P.R1 = (dw * q + w * dq) / k;
  P.R2 = (ddw * q + T(2) * dw * dq + w * ddq) / (k * k);
  return P;
}

template <typename T>
__host__ __device__ __forceinline__ T rev_kappa(const Profile<T>& P) {
  const T G = sqrt(T(1) + P.R1 * P.R1);
  const T km = fabs(P.R2) / (G * G * G), kp = T(1) / (P.R * G);
  return km > kp ? km : kp;
}

// t of cp(x) from rho0 = |xh| and t0 = x_{n-1}; |t| <= k (1 - 1e-6).  Where the
// Newton derivative R'^2 + (R - rho0) R'' + 1 falls below 0.1 the Gauss-Newton
// one R'^2 + 1 is used.  Stops when a step moves t by at most tol (1 + |t|)
// (1e-15 in FP64, 2e-7 in FP32) or after 60 steps.  P receives the profile at t.
template <typename T>
__host__ __device__ __forceinline__ T rev_cp_t(T rho0, T t0, T al, T k, Profile<T>& P) {
  const T tol = sizeof(T) == 8 ? T(1e-15) : T(2e-7);
  const T lim = k * (T(1) - T(1e-6));
  T t = t0 < -lim ? -lim : (t0 > lim ? lim : t0);
  for (int it = 0; it < 60; ++it) {
    const Profile<T> Q = rev_profile<T>(t, al, k);
    const T F = (Q.R - rho0) * Q.R1 + (t - t0);
    T J = Q.R1 * Q.R1 + (Q.R - rho0) * Q.R2 + T(1);
    if (!(J > T(0.1))) J = Q.R1 * Q.R1 + T(1);
    T tn = t - F / J;
    tn = tn < -lim ? -lim : (tn > lim ? lim : tn);
    if (fabs(tn - t) <= tol * (T(1) + fabs(t))) { t = tn; break; }
    t = tn;
  }
  P = rev_profile<T>(t, al, k);
  return t;
}

// u or (-Delta_M + sigma) u at the point (R(t) w, t) of M from vw = v.w and
// aw = w^T diag(A) w, mA = tr(A)/(n-1).  On M (metric (1 + R'^2) dt^2 +
// R^2 dw^2) Delta_M (h(t) Y_k) = [ (h'' + (n-2) R' h'/R - h' R' R''/(1+R'^2))
// / (1+R'^2) - lambda_k h/R^2 ] Y_k with lambda = 0, n-2, 2(n-1) for the
// degree-0 part h0 = c0 + c1 t + c2 t^2 + mA R^2, the degree-1 part R (v.w) and the
// degree-2 part R^2 (aw - mA).
template <typename T>
__host__ __device__ __forceinline__ T rev_quad_value(const Profile<T>& P, T t, T vw, T aw, T mA, T c0, T c1,
                                                     T c2, T sigma, int n, bool apply_op) {
  const T R = P.R, R1 = P.R1, R2 = P.R2;
  const T u = c0 + c1 * t + c2 * t * t + R * vw + R * R * aw;
  if (!apply_op) return u;
  const T md = T(n - 2), G2 = T(1) + R1 * R1;
  const T h0p = c1 + T(2) * c2 * t + T(2) * mA * R * R1;
  const T h0pp = T(2) * c2 + T(2) * mA * (R1 * R1 + R * R2);
  const T L0 = (h0pp + md * R1 * h0p / R - h0p * R1 * R2 / G2) / G2;
  const T L1 = (R2 + md * R1 * R1 / R - R1 * R1 * R2 / G2) / G2 - md / R;
  const T h2p = T(2) * R * R1, h2pp = T(2) * R1 * R1 + T(2) * R * R2;
  const T L2 = (h2pp + md * R1 * h2p / R - h2p * R1 * R2 / G2) / G2 - T(2) * (md + T(1));
  return -L0 - L1 * vw - L2 * (aw - mA) + sigma * u;
}

}  // namespace mpwos
