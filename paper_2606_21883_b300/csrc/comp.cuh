// comp.cuh — the compensation term m_* of Sec. 2.3.3 (m of eq.
// mismatch_definition) for the walks in R^3: the unit sphere and the torus.
//
// For x near M write x = y + eta n(y), y = cp(x), eta the signed normal
// distance.  With a predictor u_* and E u_* = u_* o cp,
//   R_*(s; y) = -Delta(E u_*)(y + s n(y)) + sigma u_*(y) - f(y),
//   NORMAL2: m_*(x) = eta m1 + eta^2 m2 / 2,
//            m1 = (R_*(h) - R_*(-h)) / (2h), m2 = (R_*(h) - 2 R_*(0) + R_*(-h)) / h^2;
//   EXACT:   m_*(x) = R_*(eta; y).
// E u_* is constant along normals, so -Delta(E u_*) at y + s n(y) is the
// Laplacian of a function of the tangential coordinates alone:
//   unit sphere (rho = 1 + s): Lambda(y) / rho^2, Lambda = -Delta_S u_*(y);
//   torus (rho = a + s, angles th, ph of y, rr = R + rho cos th):
//     -(u_thth / rho^2 - sin th u_th / (rho rr) + u_phph / rr^2).
// FP64 (parity with the CPU oracle): the definition evaluated in the
// oracle's order.  FP32: R_*(s) - R_*(0) = L(s) - L(0) (the sigma u_* - f
// part is common to every s), written per term without cancellation, e.g.
//   1/(a+s)^2 - 1/a^2 = -s (2a + s) / (a^2 (a+s)^2),
// so the h^-2 of m2 multiplies rounding of size ulp(h L') rather than ulp(L).
#pragma once
#include "dev_common.cuh"
#include "geom3.cuh"

namespace mpwos {

// ---------------------------------------------------------------- FP64 ----
template <int MK>
__device__ __forceinline__ double normal_coord64(const DevProblem& pb, const double* x) {
  if constexpr (MK == kTorus) {
    const double rxy = sqrt(x[0] * x[0] + x[1] * x[1]);
    const double dr = rxy - pb.R;
    return sqrt(dr * dr + x[2] * x[2]) - pb.a_tube;
  } else {
    return sqrt(dot3(x, x)) - 1.0;
  }
}

// The predictor's tangential data at y: torus (cos th, sin th, u_thth, u_th,
// u_phph, u_*); sphere (Lambda, u_*) in the first and last slots.
struct PredAt64 { double ct, st, utt, ut, upp, lam, u; };

template <int MK>
__device__ __forceinline__ PredAt64 pred_at64(const DevProblem& pb, const double* y) {
  const DevPredictor& P = pb.pred;
  PredAt64 o{};
  if constexpr (MK == kTorus) {
    const double rxy = sqrt(y[0] * y[0] + y[1] * y[1]);
    const double dr = rxy - pb.R;
    const double nr = sqrt(dr * dr + y[2] * y[2]);
    o.ct = dr / nr;
    o.st = y[2] / nr;
    const double cp = y[0] / rxy, sp = y[1] / rxy;
    for (int t = 0; t < P.n_terms; ++t) {
      const int m = P.modes[t][0], q = P.modes[t][1];
      double cm = 1.0, sm = 0.0, cq = 1.0, sq = 0.0;
      for (int j = 0; j < m; ++j) { const double c2 = cm * o.ct - sm * o.st; sm = sm * o.ct + cm * o.st; cm = c2; }
      for (int j = 0; j < q; ++j) { const double c2 = cq * cp - sq * sp; sq = sq * cp + cq * sp; cq = c2; }
      const bool tcos = P.modes[t][2] == 0;
      const double Tv = tcos ? cm : sm;
      const double Tp = tcos ? -static_cast<double>(m) * sm : static_cast<double>(m) * cm;
      const double Pv = P.modes[t][3] == 0 ? cq : sq;
      o.utt += P.coef[t] * (-static_cast<double>(m * m) * Tv * Pv);
      o.ut += P.coef[t] * (Tp * Pv);
      o.upp += P.coef[t] * (-static_cast<double>(q * q) * Tv * Pv);
      o.u += P.coef[t] * (Tv * Pv);
    }
  } else {
    // degree-1 part: -Delta_S eigenvalue 2; trace-free quadratic part: 6
    const double ny = sqrt(dot3(y, y));
    const double w[3] = {y[0] / ny, y[1] / ny, y[2] / ny};
    const double lin = dot3(P.v, w);
    double quad = 0.0, tr = 0.0;
    for (int i = 0; i < 3; ++i) {
      tr += P.A[i * 3 + i];
      for (int j = 0; j < 3; ++j) quad += P.A[i * 3 + j] * w[i] * w[j];
    }
    o.lam = 2.0 * lin + 6.0 * (quad - tr / 3.0);
    o.u = P.c0 + lin + quad;
  }
  return o;
}

// -Delta(E u_*) at normal coordinate s
template <int MK>
__device__ __forceinline__ double ext_neg_lap64(const DevProblem& pb, const PredAt64& o, double s) {
  if constexpr (MK == kTorus) {
    const double rho = pb.a_tube + s;
    const double rr = pb.R + rho * o.ct;
    return -(o.utt / (rho * rho) - o.st * o.ut / (rho * rr) + o.upp / (rr * rr));
  } else {
    const double rho = 1.0 + s;
    return o.lam / (rho * rho);
  }
}

// m_*(x), y = cp(x), fy = f(y)
template <int MK>
__device__ __forceinline__ double comp_m64(const DevProblem& pb, const double* x, const double* y, double fy) {
  const PredAt64 o = pred_at64<MK>(pb, y);
  const double eta = normal_coord64<MK>(pb, x);
  const double su = pb.sigma * o.u;
  if (pb.pred.comp == kCompExact) return (ext_neg_lap64<MK>(pb, o, eta) + su) - fy;
  const double h = pb.pred.h;
  const double Rp = (ext_neg_lap64<MK>(pb, o, h) + su) - fy;
  const double R0 = (ext_neg_lap64<MK>(pb, o, 0.0) + su) - fy;
  const double Rm = (ext_neg_lap64<MK>(pb, o, -h) + su) - fy;
  const double m1 = (Rp - Rm) / (2.0 * h);
  const double m2 = (Rp - 2.0 * R0 + Rm) / (h * h);
  return eta * m1 + 0.5 * eta * eta * m2;
}

// ---------------------------------------------------------------- FP32 ----
// L(s) - L(0) on the torus from the sums A = u_thth, B = u_th, C = u_phph.
__device__ __forceinline__ float torus_dL32(float a, float q0, float ct, float st, float A, float B, float C,
                                            float s) {
  const float as = a + s, qs = fmaf(s, ct, q0);
  const float dg1 = -s * (2.0f * a + s) / (a * a * as * as);
  const float dg2 = -s * fmaf(ct, as, q0) / (a * q0 * as * qs);
  const float dg3 = -s * ct * fmaf(s, ct, 2.0f * q0) / (q0 * q0 * qs * qs);
  return -(A * dg1 - st * B * dg2 + C * dg3);
}

// m_*(Z) in FP32; fz = f(cp(Z)) (used by the EXACT mode only).
template <int MK>
__device__ __forceinline__ float comp_m32(const DevProblem& pb, const float* Z, float fz) {
  const DevPredictor& P = pb.pred;
  const float h = P.hf;
  if constexpr (MK == kTorus) {
    const float R = pb.sf.R, a = pb.sf.a;
    const float rho2 = Z[0] * Z[0] + Z[1] * Z[1];
    const float irho = rsqrtf(rho2);
    const float dr = rho2 * irho - R;
    const float d2 = dr * dr + Z[2] * Z[2];
    const float iw = rsqrtf(d2);
    const float ct = dr * iw, st = Z[2] * iw;
    const float cph = Z[0] * irho, sph = Z[1] * irho;
    const float eta = d2 * iw - a;
    float A = 0.0f, B = 0.0f, C = 0.0f, U = 0.0f;
    for (int t = 0; t < P.n_terms; ++t) {
      float cm, sm, cq, sq;
      angle_multiple(P.modes[t][0], ct, st, cm, sm);
      angle_multiple(P.modes[t][1], cph, sph, cq, sq);
      const bool tcos = P.modes[t][2] == 0;
      const float m = P.mode_f[t][0], q = P.mode_f[t][1];
      const float Tv = tcos ? cm : sm;
      const float Tp = tcos ? -m * sm : m * cm;
      const float Pv = P.modes[t][3] == 0 ? cq : sq;
      const float cT = P.coef_f[t] * Tv * Pv;
      A = fmaf(-m * m, cT, A);
      B = fmaf(P.coef_f[t] * Tp, Pv, B);
      C = fmaf(-q * q, cT, C);
      U += cT;
    }
    const float q0 = fmaf(a, ct, R);
    if (P.comp == kCompExact) {
      const float L0 = -(A / (a * a) - st * B / (a * q0) + C / (q0 * q0));
      return torus_dL32(a, q0, ct, st, A, B, C, eta) + ((L0 + pb.sf.sigma * U) - fz);
    }
    const float dp = torus_dL32(a, q0, ct, st, A, B, C, h);
    const float dm = torus_dL32(a, q0, ct, st, A, B, C, -h);
    const float m1 = (dp - dm) / (2.0f * h);
    const float m2 = (dp + dm) / (h * h);
    return eta * fmaf(0.5f * eta, m2, m1);
  } else {
    const float nz2 = Z[0] * Z[0] + Z[1] * Z[1] + Z[2] * Z[2];
    const float inz = rsqrtf(nz2);
    const float w[3] = {Z[0] * inz, Z[1] * inz, Z[2] * inz};
    const float eta = nz2 * inz - 1.0f;
    const float lin = P.v_f[0] * w[0] + P.v_f[1] * w[1] + P.v_f[2] * w[2];
    float quad = 0.0f;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) quad = fmaf(P.A_f[i * 3 + j] * w[i], w[j], quad);
    const float tr = P.A_f[0] + P.A_f[4] + P.A_f[8];
    const float lam = 2.0f * lin + 6.0f * (quad - tr * (1.0f / 3.0f));
    if (P.comp == kCompExact) {
      const float g1 = 1.0f + eta;
      const float dL = lam * (-eta * (2.0f + eta) / (g1 * g1));   // Lambda ((1 + eta)^-2 - 1)
      return dL + ((lam + pb.sf.sigma * (P.c0_f + lin + quad)) - fz);
    }
    return lam * (eta * fmaf(0.5f * eta, P.sd2, P.sd1));
  }
}

}  // namespace mpwos
