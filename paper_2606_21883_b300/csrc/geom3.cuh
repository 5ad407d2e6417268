// geom3.cuh — closest point (eq. cp_map), effective boundary distance (eq.
// delta_Gamma_general) and the problem data f, g for manifolds in R^3, in
// scalar type T (double for the FP64 walk, float for the FP32 walk).
#pragma once
#include "dev_common.cuh"

namespace mpwos {

template <typename T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }

template <typename T>
__device__ __forceinline__ T dot3(const T* a, const T* b) {
  T s = T(0);
  s += a[0] * b[0];
  s += a[1] * b[1];
  s += a[2] * b[2];
  return s;
}

// cp(x) for the R^3 manifolds.
template <int MK, typename T>
__device__ __forceinline__ void cp3(const DevProblem& pb, const T* x, T* out) {
  if (MK == kEuclid) {
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2];
  } else if (MK == kSphere) {
    const T nx = dsqrt<T>(dot3(x, x));
    out[0] = x[0] / nx; out[1] = x[1] / nx; out[2] = x[2] / nx;
  } else {  // torus: nearest point of the centre circle, then the tube around it
    const T R = pick<T>(pb.R, pb.sf.R), a = pick<T>(pb.a_tube, pb.sf.a);
    const T rho = dsqrt<T>(x[0] * x[0] + x[1] * x[1]);
    const T c0 = R * x[0] / rho, c1 = R * x[1] / rho;
    T w[3] = {x[0] - c0, x[1] - c1, x[2] - T(0)};
    const T nw = dsqrt<T>(dot3(w, w));
    const T s = a / nw;
    out[0] = c0 + s * w[0];
    out[1] = c1 + s * w[1];
    out[2] = T(0) + s * w[2];
  }
}

// delta_Gamma(y) = (|P_T r_G|^2 + (|P_N r_G| - ell)_+^2)^{1/2}, r_G = y_G - y, for
// Omega = M intersected with {e.x > h}; y_G = cp_Gamma(y) is written to yg.  A state
// with e.y <= h is outside Omega: distance 0.
template <int MK, typename T>
__device__ __forceinline__ T delta_gamma3(const DevProblem& pb, const T* y, T* yg) {
  T e[3];
  if constexpr (sizeof(T) == 4) {
    e[0] = pb.ef[0]; e[1] = pb.ef[1]; e[2] = pb.ef[2];
  } else {
    e[0] = pb.e[0]; e[1] = pb.e[1]; e[2] = pb.e[2];
  }
  const T h = pick<T>(pb.h, pb.sf.h);
  const T ey = dot3(e, y);
  if constexpr (MK == kEuclid) {
    for (int i = 0; i < 3; ++i) yg[i] = y[i] - (ey - h) * e[i];
    const T d = fabs(ey - h);
    return (ey <= h) ? T(0) : d;
  } else if constexpr (MK == kTorus) {
    // a plane through the axis (e_3 = 0, h = 0): Gamma is the two meridian
    // circles c_b + a (cos t u_b + sin t e_3), c_b = R u_b, u_0 = (-e_2, e_1, 0),
    // u_1 = -u_0.  Nearest point of circle b: c_b + a w/|w|, w the part of
    // y - c_b in span(u_b, e_3); the nearer circle wins (circle 0 on a tie); the
    // torus normal at y_G is w/|w|.
    const T R = pick<T>(pb.R, pb.sf.R), a = pick<T>(pb.a_tube, pb.sf.a);
    T best = T(INFINITY), nrm[3] = {T(0), T(0), T(0)};
    for (int b = 0; b < 2; ++b) {
      const T sgn = (b == 0) ? T(1) : T(-1);
      const T u[3] = {-sgn * e[1], sgn * e[0], T(0)};
      const T c[3] = {R * u[0], R * u[1], T(0)};
      const T wu = (y[0] - c[0]) * u[0] + (y[1] - c[1]) * u[1];
      const T wz = y[2];
      const T w[3] = {wu * u[0], wu * u[1], wz};
      const T nw = dsqrt<T>(wu * wu + wz * wz);
      T nb[3];
      if (nw > T(0)) {
        for (int i = 0; i < 3; ++i) nb[i] = w[i] / nw;
      } else {   // y on the circle's axis: take t = 0
        for (int i = 0; i < 3; ++i) nb[i] = u[i];
      }
      T q[3], d2 = T(0);
      for (int i = 0; i < 3; ++i) {
        q[i] = c[i] + a * nb[i];
        d2 += (q[i] - y[i]) * (q[i] - y[i]);
      }
      if (d2 < best) {
        best = d2;
        for (int i = 0; i < 3; ++i) { yg[i] = q[i]; nrm[i] = nb[i]; }
      }
    }
    T rn = T(0);
    for (int i = 0; i < 3; ++i) rn += (yg[i] - y[i]) * nrm[i];
    T rt2 = T(0);
    for (int i = 0; i < 3; ++i) {
      const T rti = (yg[i] - y[i]) - rn * nrm[i];
      rt2 += rti * rti;
    }
    if (ey <= h) return T(0);
    T ex = fabs(rn) - pick<T>(pb.rho_geo, pb.sf.rho_geo);
    if (ex < T(0)) ex = T(0);
    return dsqrt<T>(rt2 + ex * ex);
  } else {
  // unit sphere: y_G = h e + sqrt(1 - h^2) w/|w|, w = y - (e.y) e
  T w[3];
  for (int i = 0; i < 3; ++i) w[i] = y[i] - ey * e[i];
  T nw = dsqrt<T>(dot3(w, w));
  if (nw == T(0)) {  // pole: lowest-index axis not parallel to e
    for (int j = 0; j < 3; ++j) {
      for (int i = 0; i < 3; ++i) w[i] = ((i == j) ? T(1) : T(0)) - e[j] * e[i];
      nw = dsqrt<T>(dot3(w, w));
      if (nw > T(1e-8)) break;
    }
  }
  const T sh = dsqrt<T>(T(1) - h * h);
  for (int i = 0; i < 3; ++i) yg[i] = h * e[i] + sh * (w[i] / nw);
  T rn = T(0);
  for (int i = 0; i < 3; ++i) rn += (yg[i] - y[i]) * yg[i];
  T rt2 = T(0);
  for (int i = 0; i < 3; ++i) {
    const T rti = (yg[i] - y[i]) - rn * yg[i];
    rt2 += rti * rti;
  }
  if (ey <= h) return T(0);
  T ex = fabs(rn) - pick<T>(pb.rho_geo, pb.sf.rho_geo);
  if (ex < T(0)) ex = T(0);
  return dsqrt<T>(rt2 + ex * ex);
  }
}

// cos(m x), sin(m x) from c = cos x, s = sin x: closed forms for m <= 4 (the
// mode is uniform across the warp, so the switch does not diverge), repeated
// rotation above.
__device__ __forceinline__ void angle_multiple(int m, float c, float s, float& cm, float& sm) {
  switch (m) {
    case 0: cm = 1.0f; sm = 0.0f; return;
    case 1: cm = c; sm = s; return;
    case 2: cm = fmaf(2.0f * c, c, -1.0f); sm = 2.0f * s * c; return;
    case 3: {
      const float c2 = fmaf(2.0f * c, c, -1.0f);
      cm = c * fmaf(2.0f, c2, -1.0f);
      sm = s * fmaf(2.0f, c2, 1.0f);
      return;
    }
    case 4: {
      const float c2 = fmaf(2.0f * c, c, -1.0f), s2 = 2.0f * s * c;
      cm = fmaf(2.0f * c2, c2, -1.0f);
      sm = 2.0f * s2 * c2;
      return;
    }
    default: {
      float a = 1.0f, b = 0.0f;
      for (int j = 0; j < m; ++j) { const float a2 = a * c - b * s; b = b * c + a * s; a = a2; }
      cm = a; sm = b;
    }
  }
}

// Problem data at a point x of M (f(cp(Z)) and g(cp_Gamma(Y)) of Algorithm 1).
template <int MK, typename T>
__device__ __forceinline__ T func3(const DevProblem& pb, const DevFunc& fn, const T* x) {
  if (fn.kind == kPoly) {
    T total = T(0);
    for (int t = 0; t < fn.n_terms; ++t) {
      T prod = pick<T>(fn.coef[t], fn.coef_f[t]);
      for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
        const T xv = x[fn.var[q]];
        for (int e = 0; e < fn.pw[q]; ++e) prod *= xv;
      }
      total += prod;
    }
    return total;
  }
  if (fn.kind == kTorusFourier) {
    const T R = pick<T>(pb.R, pb.sf.R), a = pick<T>(pb.a_tube, pb.sf.a);
    const T rho = dsqrt<T>(x[0] * x[0] + x[1] * x[1]);
    const T dr = rho - R;
    const T nr = dsqrt<T>(dr * dr + x[2] * x[2]);
    const T ct = dr / nr, st = x[2] / nr;       // theta of the point
    const T cp = x[0] / rho, sp = x[1] / rho;    // phi of the point
    T total = T(0);
    for (int t = 0; t < fn.n_terms; ++t) {
      const int m = fn.modes[t][0], q = fn.modes[t][1];
      // cos/sin of m theta and q phi by angle addition
      T cm = T(1), sm = T(0), cq = T(1), sq = T(0);
      for (int j = 0; j < m; ++j) { const T c2 = cm * ct - sm * st; sm = sm * ct + cm * st; cm = c2; }
      for (int j = 0; j < q; ++j) { const T c2 = cq * cp - sq * sp; sq = sq * cp + cq * sp; cq = c2; }
      const T Tv = fn.modes[t][2] == 0 ? cm : sm;
      const T Pv = fn.modes[t][3] == 0 ? cq : sq;
      T val;
      if (!fn.apply_op) {
        val = Tv * Pv;
      } else {
        // -Delta_M(T P) = P [m^2 T/a^2 + sin(th) T'/(a (R + a cos th)) + q^2 T/(R + a cos th)^2]
        const T Tp = fn.modes[t][2] == 0 ? -T(m) * sm : T(m) * cm;
        const T rr = R + a * ct;
        const T lap = T(m * m) * Tv / (a * a) + st * Tp / (a * rr) + T(q * q) * Tv / (rr * rr);
        val = Pv * (lap + pick<T>(pb.sigma, pb.sf.sigma) * Tv);
      }
      total += pick<T>(fn.coef[t], fn.coef_f[t]) * val;
    }
    return total;
  }
  // sphere quad on the unit sphere of R^3 (s = x/|x|, d = 2)
  const T nx = dsqrt<T>(dot3(x, x));
  const T s[3] = {x[0] / nx, x[1] / nx, x[2] / nx};
  T lin = T(0), quad = T(0), tr = T(0);
  for (int i = 0; i < 3; ++i) {
    lin += T(fn.v[i]) * s[i];
    tr += T(fn.A[i * 3 + i]);
    for (int j = 0; j < 3; ++j) quad += T(fn.A[i * 3 + j]) * s[i] * s[j];
  }
  const T c0 = pick<T>(fn.c0, fn.c0_f);
  if (!fn.apply_op) return c0 + lin + quad;
  const T mean = tr / T(3);
  const T sg = pick<T>(pb.sigma, pb.sf.sigma);
  return sg * (c0 + mean) + (T(2) + sg) * lin + (T(6) + sg) * (quad - mean);
}

}  // namespace mpwos
