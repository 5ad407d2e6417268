// green.cuh — screened factor c_{sigma,r}, the radial law of the interior
// sample Z ~ rho(y, .) = G(y, .)/omega(y), and its inverse.
//
//   c_{sigma,r} = 1 / I~_nu(a),  I~_nu(a) = sum_j (a^2/4)^j / (j! (nu+1)_j)
//       (Lemma 2.1, eq. def_c_sigma_r, through the Bessel-free series of
//        Lemma 3.1); a = sqrt(sigma) r, nu = (n-2)/2.
//   omega = (1 - c)/sigma  (Thm 2.2, eq. omega_explicit_formula).
//   Radial CDF of t = |Z - y|/r (eq. Z_sampling_density with the Remark's G):
//       F(t) = [ (1 - K~_{nu+1}(x)) - c K~_nu(a) I~_{nu+1}(x) (x/2)^2 t^{2nu}/(nu(nu+1)) ] / (1 - c),
//       F'(t) = (a x / (2 nu)) [ K~_nu(x) - c K~_nu(a) I~_nu(x) t^{2nu} ] / (1 - c),   x = a t,
//   where K~_mu(x) = 2 (x/2)^mu K_mu(x)/Gamma(mu).  For n = 3 these reduce to
//       F(t) = [P(x) - Q(x) e^{-a}/sinh a]/(1-c),  F'(t) = a x sinh(a - x)/(sinh a (1-c)),
//       P(x) = 1 - e^{-x}(1+x), Q(x) = x cosh x - sinh x.
// FP64 throughout (these are the FP64 parts of the walk in every precision).
#pragma once
#include <cuda_runtime.h>
#include "dev_common.cuh"

namespace mpwos {

constexpr double kEulerGamma = 0.57721566490153286;
constexpr double kPi = 3.141592653589793;

// I~_nu(a) - 1 with z = a^2/4.
__host__ __device__ __forceinline__ double em1_series(double nu, double z) {
  double term = 1.0, sum = 0.0;
  for (int j = 1; j < 10000; ++j) {
    term *= z / (static_cast<double>(j) * (nu + static_cast<double>(j)));
    sum += term;
    if (term <= 1e-17 * sum) break;
  }
  return sum;
}

// em1(z) from the FP32 polynomial of a problem (Horner).
__device__ __forceinline__ float em1_poly32(const DevProblem& pb, float z) {
  float acc = pb.em1_k[pb.em1_terms - 1];
  for (int j = pb.em1_terms - 2; j >= 0; --j) acc = fmaf(acc, z, pb.em1_k[j]);
  return acc * z;
}

// 1 - c from em1 without cancellation.
__host__ __device__ __forceinline__ double one_minus_c(double em1, double c) {
  return (em1 <= 1.0) ? em1 * c : 1.0 - c;
}

// 0F1(;b;z), b > 0.
__host__ __device__ inline double hyp0f1_dev(double b, double z) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 10000; ++k) {
    term *= z / (static_cast<double>(k) * (b + static_cast<double>(k) - 1.0));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

// K~_mu(x) - 1.  Non-integer mu: reflection formula K = (pi/2)(I_{-mu} - I_mu)/sin(pi mu);
// integer mu: the logarithmic expansion (Abramowitz & Stegun 9.6.11).
__host__ __device__ inline double kt_m1(double mu, double x) {
  const double z = 0.25 * (x * x);
  const double hx = log(0.5 * x);
  const double mr = floor(mu + 0.5);
  double s = 0.0, term = 1.0;
  if (fabs(mu - mr) < 1e-12) {
    const int m = static_cast<int>(mr);
    for (int k = 1; k <= m - 1; ++k) {
      term *= z / (static_cast<double>(k) * (static_cast<double>(k) - mr));
      s += term;
      if (fabs(term) <= 1e-18 * fabs(s)) break;
    }
    const double lg = 0.6931471805599453 + 2.0 * mr * hx - lgamma(mr) - lgamma(mr + 1.0);
    if (lg > -740.0) {
      double Hm = 0.0;
      for (int q = 1; q <= m; ++q) Hm += 1.0 / static_cast<double>(q);
      double inner = 0.0, tk = 1.0, Hk = 0.0, Hmk = Hm;
      for (int k = 0; k < 10000; ++k) {
        const double add = tk * (hx + kEulerGamma - 0.5 * (Hk + Hmk));
        inner += add;
        if (k > 2 && fabs(add) <= 1e-18 * fabs(inner)) break;
        tk *= z / (static_cast<double>(k + 1) * static_cast<double>(m + k + 1));
        Hk += 1.0 / static_cast<double>(k + 1);
        Hmk += 1.0 / static_cast<double>(m + k + 1);
      }
      s += (((m + 1) & 1) ? -1.0 : 1.0) * exp(lg) * inner;
    }
    return s;
  }
  for (int k = 1; k < 10000; ++k) {
    term *= z / (static_cast<double>(k) * (static_cast<double>(k) - mu));
    s += term;
    if (term == 0.0) break;
    if (static_cast<double>(k) > mu + 1.0 && fabs(term) <= 1e-18 * fabs(s)) break;
  }
  const double sp = sin(kPi * mu);
  const double lg = log(kPi) - log(fabs(sp)) - lgamma(mu) - lgamma(mu + 1.0) + 2.0 * mu * hx;
  if (lg > -740.0) s -= ((sp > 0.0) ? 1.0 : -1.0) * exp(lg) * hyp0f1_dev(1.0 + mu, z);
  return s;
}

// P(x) = 1 - e^{-x}(1+x) and Q(x) = x cosh x - sinh x for x < 1 (series).
__host__ __device__ __forceinline__ double p3_series(double x) {
  double term = x, sum = 0.0;
  for (int k = 2; k < 60; ++k) {
    term *= x / static_cast<double>(k);
    const double add = ((k & 1) ? -1.0 : 1.0) * static_cast<double>(k - 1) * term;
    sum += add;
    if (fabs(add) <= 1e-18 * fabs(sum)) break;
  }
  return sum;
}

__host__ __device__ __forceinline__ double q3_series(double x) {
  double term = x, sum = 0.0;
  for (int k = 1; k < 60; ++k) {
    term *= x * x / (static_cast<double>(2 * k) * static_cast<double>(2 * k + 1));
    const double add = 2.0 * static_cast<double>(k) * term;
    sum += add;
    if (add <= 1e-18 * sum) break;
  }
  return sum;
}

// Constants of one radial law (depend on n and a only).
struct GreenLaw {
  int n;
  double nu, a, c, omc, kta;   // kta = K~_nu(a) (general n)
};

__host__ __device__ inline GreenLaw green_law(int n, double a) {
  GreenLaw L;
  L.n = n;
  L.nu = 0.5 * static_cast<double>(n - 2);
  L.a = a;
  const double em1 = em1_series(L.nu, 0.25 * (a * a));
  L.c = 1.0 / (1.0 + em1);
  L.omc = one_minus_c(em1, L.c);
  L.kta = (n == 3 || a == 0.0) ? 1.0 : 1.0 + kt_m1(L.nu, a);
  return L;
}

// F(t) and F'(t).  a == 0 is the Laplace limit (n t^2 - 2 t^n)/(n - 2).
__host__ __device__ inline void green_cdf_pdf(const GreenLaw& L, double t, double& F, double& dF) {
  const double a = L.a, x = a * t;
  if (a == 0.0) {
    const double tn2 = pow(t, static_cast<double>(L.n - 2));
    F = (static_cast<double>(L.n) * t * t - 2.0 * t * t * tn2) / static_cast<double>(L.n - 2);
    dF = 2.0 * static_cast<double>(L.n) * t * (1.0 - tn2) / static_cast<double>(L.n - 2);
    return;
  }
  if (L.n == 3) {
    double second, ratio_d;
    if (x < 1.0) {
      const double k = 2.0 / expm1(2.0 * a);
      second = q3_series(x) * k;
      F = (p3_series(x) - second) / L.omc;
    } else {
      const double den = -expm1(-2.0 * a);
      second = ((x - 1.0) * exp(x - 2.0 * a) + (x + 1.0) * exp(-x - 2.0 * a)) / den;
      F = ((1.0 - exp(-x) * (1.0 + x)) - second) / L.omc;
    }
    // sinh(a - x)/sinh(a) = e^{-x} (1 - e^{-2(a-x)}) / (1 - e^{-2a})
    ratio_d = exp(-x) * (-expm1(-2.0 * (a - x))) / (-expm1(-2.0 * a));
    dF = a * x * ratio_d / L.omc;
    return;
  }
  const double nu = L.nu, zx = 0.25 * (x * x);
  const double t2nu = pow(t, 2.0 * nu);
  const double sk = -kt_m1(nu + 1.0, x);
  const double it1 = hyp0f1_dev(nu + 2.0, zx);
  F = (sk - L.c * L.kta * it1 * zx * t2nu / (nu * (nu + 1.0))) / L.omc;
  const double ktx = 1.0 + kt_m1(nu, x);
  const double itx = hyp0f1_dev(nu + 1.0, zx);
  dF = (a * x / (2.0 * nu)) * (ktx - L.c * L.kta * itx * t2nu) / L.omc;
}

// Safeguarded Newton for F(t) = U on [0, 1] from guess t0.
__host__ __device__ inline double green_invert64(const GreenLaw& L, double U, double t0) {
  if (U >= 1.0) return 1.0;
  double lo = 0.0, hi = 1.0;
  double t = (t0 > 0.0 && t0 < 1.0) ? t0 : 0.5;
  for (int it = 0; it < 100; ++it) {
    double F, dF;
    green_cdf_pdf(L, t, F, dF);
    const double res = F - U;
    if (res == 0.0) break;
    if (res < 0.0) lo = t; else hi = t;
    double tn = (dF > 0.0) ? t - res / dF : 0.5 * (lo + hi);
    if (!(tn >= lo && tn <= hi)) tn = 0.5 * (lo + hi);
    const bool conv = fabs(tn - t) <= 4e-16 * t || hi - lo <= 4e-16 * hi;
    t = tn;
    if (conv) break;
  }
  return t;
}

// Radius tables.  Each law (row) holds two sides of NS + 2 nodes: side A
// tabulates t over v = sqrt(U) for U <= 1/2, side B over v = sqrt(1 - U) for
// U > 1/2.  Both ends of t(U) behave like square roots (t ~ sqrt(U) at 0,
// 1 - t ~ sqrt(1 - U) at 1), so t is smooth in v on each side; nodes v_j = j h,
// h = sqrt(1/2)/(NS - 1), j = -1 .. NS (node j at offset j + 1; j = -1 from the
// odd symmetries t(-v) = -t(v), 1 - t(-v) = -(1 - t(v))).
constexpr double kTableVmax = 0.70710678118654752;

template <typename T>
__host__ __device__ __forceinline__ T catmull_rom(const T* row, int j, T f) {
  const T p0 = row[j], p1 = row[j + 1], p2 = row[j + 2], p3 = row[j + 3];
  return p1 + T(0.5) * f * (p2 - p0 + f * (T(2) * p0 - T(5) * p1 + T(4) * p2 - p3 +
                                           f * (T(3) * (p1 - p2) + p3 - p0)));
}

// Table lookup t(U; z), rows over z = a^2/4 in [0, z_max] (NA = 1: one law),
// Catmull-Rom along v, linear across rows.
template <typename T>
__host__ __device__ __forceinline__ T table_lookup(const T* tab, int NA, int NS, double z_max, T a, T U) {
  const int side_len = NS + 2;
  const bool upper = U > T(0.5);
  const T v = sqrt(upper ? T(1) - U : U);
  const T xs = v * T(static_cast<double>(NS - 1) / kTableVmax);
  int j = static_cast<int>(xs);
  j = j < 0 ? 0 : (j > NS - 2 ? NS - 2 : j);
  const T f = xs - T(j);
  const int side = upper ? side_len : 0;
  if (NA == 1) return catmull_rom(tab + side, j, f);
  const T fa = (a * a * T(0.25)) / T(z_max) * T(NA - 1);
  int ia = static_cast<int>(fa);
  ia = ia < 0 ? 0 : (ia > NA - 2 ? NA - 2 : ia);
  const T wa = fa - T(ia);
  const T* r0 = tab + static_cast<size_t>(ia) * (2 * side_len) + side;
  const T v0 = catmull_rom(r0, j, f);
  const T v1 = catmull_rom(r0 + 2 * side_len, j, f);
  return v0 + wa * (v1 - v0);
}

// FP32 lookup in the coefficient table: the Catmull-Rom cubic of interval j
// (nodes j-1 .. j+2 of the node table) stored as one float4 of monomial
// coefficients computed in FP64, so a lookup is one 16-byte load and three
// FMAs per row.  tab_scale = (NS - 1)/sqrt(1/2), z_scale = (NA - 1)/z_max.
__device__ __forceinline__ float table_lookup32(const float4* tabc, int NA, int NS, float tab_scale, float z_scale,
                                                float a, float U) {
  const int NI = NS - 1;   // intervals per side
  const bool upper = U > 0.5f;
  const float v = sqrtf(upper ? 1.0f - U : U);
  const float xs = v * tab_scale;
  int j = static_cast<int>(xs);
  j = j > NI - 1 ? NI - 1 : j;
  const float f = xs - static_cast<float>(j);
  const float4* tab = tabc + (upper ? NI : 0) + j;
  const float4 c = tab[0];
  const float t0 = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
  if (NA == 1) return t0;
  const float fa = a * a * 0.25f * z_scale;
  int ia = static_cast<int>(fa);
  ia = ia < 0 ? 0 : (ia > NA - 2 ? NA - 2 : ia);
  const float wa = fminf(fa - static_cast<float>(ia), 1.0f);
  const float4 c0 = tab[static_cast<size_t>(ia) * (2 * NI)];
  const float4 c1 = tab[static_cast<size_t>(ia + 1) * (2 * NI)];
  const float v0 = fmaf(f, fmaf(f, fmaf(f, c0.w, c0.z), c0.y), c0.x);
  const float v1 = fmaf(f, fmaf(f, fmaf(f, c1.w, c1.z), c1.y), c1.x);
  return v0 + wa * (v1 - v0);
}

__device__ __forceinline__ float table_lookup32(const DevProblem& pb, float a, float U) {
  return table_lookup32(pb.tabc, pb.NA, pb.NS, pb.sf.tab_scale, pb.sf.z_scale, a, U);
}

}  // namespace mpwos
