/*
 * mpwos_oracle.c — plain, slow, FP64 CPU oracle of the MPWoS walk.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code with the
 * CUDA path; it is compiled with -ffp-contract=off so that every + and * is
 * one IEEE operation.
 *
 * Arithmetic order is that of Algorithm 1 with the path score of eq.
 * path_score_definition: per step the radius (eq. radius_rule_unified), the
 * screened factor c_{sigma,r} and omega = (1 - c)/sigma (Thm 2.2, eq.
 * omega_explicit_formula), the sphere sample Theta = Y + r zeta (eq.
 * projected_chain_update), N_V interior samples Z ~ rho(Y, .) (eq.
 * Z_sampling_density) averaged into F_k (eq. local_average_source), the score
 * update S += W_k omega F_k, W_{k+1} = W_k c, Y_{k+1} = cp(Theta).
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): the stopping test is applied at k = 0 as well (K = inf{k >= 0 ...});
 * f at an off-manifold Z is the extension f(cp(Z)) (eq. cp_extension); the
 * interior sample's radius is drawn by inverting the radial CDF of the
 * Green density (derived from the Remark's G), its direction independently
 * uniform; m_* = 0 (the baseline variant of Sec. 2.3.3); a walk that reaches
 * max_steps is flagged, never silently cut; a boundary-case walk whose weight
 * has underflowed to exactly 0 stops (all later terms vanish).
 */
#include "mpwos_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TWO_PI 6.283185307179586
#define ORC_EULER_GAMMA 0.57721566490153286

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: round function and Weyl key schedule as published by        */
/* Salmon et al. (SC'11): multipliers 0xD2511F53, 0xCD9E8D57; key increments  */
/* 0x9E3779B9, 0xBB67AE85; ten rounds.                                         */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 53-bit uniform in (0, 1]: the top 53 bits of (hi:lo), plus one, times 2^-53. */
double orc_u53(uint32_t hi, uint32_t lo) {
  uint64_t m = (((uint64_t)hi << 32) | (uint64_t)lo) >> 11;
  return (double)(m + 1u) * 0x1p-53;
}

static void block(uint64_t seed, uint32_t j, uint32_t k, uint32_t i, uint32_t p, uint32_t out[4]) {
  uint32_t ctr[4] = {j, k, i, p};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* n standard Gaussians from blocks j0, j0+1, ... (two per block, Box-Muller:
 * sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b)); an odd n drops the last one. */
void orc_gaussians(uint64_t seed, uint32_t j0, uint32_t k, uint32_t i, uint32_t p, int n, double* g) {
  int nb = (n + 1) / 2;
  for (int b = 0; b < nb; ++b) {
    uint32_t x[4];
    block(seed, j0 + (uint32_t)b, k, i, p, x);
    double ua = orc_u53(x[0], x[1]);
    double ub = orc_u53(x[2], x[3]);
    double rad = sqrt(-2.0 * log(ua));
    double ang = ORC_TWO_PI * ub;
    g[2 * b] = rad * cos(ang);
    if (2 * b + 1 < n) g[2 * b + 1] = rad * sin(ang);
  }
}

static double uniform_at(uint64_t seed, uint32_t j, uint32_t k, uint32_t i, uint32_t p) {
  uint32_t x[4];
  block(seed, j, k, i, p, x);
  return orc_u53(x[0], x[1]);
}

/* ------------------------------------------------------------------------- */
/* Screened factor (Lemma 2.1, series of Lemma 3.1):                           */
/*   c_{sigma,r} = 1 / I~_nu(a),  I~_nu(a) = sum_j (a^2/4)^j / (j! (nu+1)_j),  */
/*   a = sqrt(sigma) r, nu = (n-2)/2.  em1 = I~_nu(a) - 1 (no leading 1).      */
/* ------------------------------------------------------------------------- */
double orc_em1(int n, double a) {
  double nu = 0.5 * (double)(n - 2);
  double z = 0.25 * (a * a);
  double term = 1.0, sum = 0.0;
  for (int j = 1; j < 100000; ++j) {
    term *= z / ((double)j * (nu + (double)j));
    sum += term;
    if (term <= 1e-17 * sum) break;
  }
  return sum;
}

double orc_c_sigma_r(int n, double a) { return 1.0 / (1.0 + orc_em1(n, a)); }

/* 0F1(;b;z) = sum_k z^k / (k! (b)_k), b > 0. */
static double hyp0f1(double b, double z) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 100000; ++k) {
    term *= z / ((double)k * (b + (double)k - 1.0));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

/* K~_mu(x) - 1, where K~_mu(x) = 2 (x/2)^mu K_mu(x) / Gamma(mu) (-> 1 as x -> 0).
 * Non-integer mu: K_mu = (pi/2)(I_{-mu} - I_mu)/sin(mu pi) gives
 *   K~_mu = 0F1(;1-mu;z) - [Gamma(1-mu)/Gamma(1+mu)] (x/2)^{2mu} 0F1(;1+mu;z).
 * Integer mu = m: Abramowitz & Stegun 9.6.11 gives
 *   K~_m = sum_{k<m} z^k/(k!(1-m)_k)
 *        + (-1)^{m+1} 2 (x/2)^{2m}/((m-1)! m!) sum_k z^k m!/(k!(m+k)!)
 *                     [ln(x/2) + gamma - (H_k + H_{m+k})/2].
 * z = x^2/4. */
double orc_kt_minus_one(double mu, double x) {
  double z = 0.25 * (x * x);
  double hx = log(0.5 * x);
  double m_round = floor(mu + 0.5);
  if (fabs(mu - m_round) < 1e-12) {
    int m = (int)m_round;
    double s = 0.0, term = 1.0;
    for (int k = 1; k <= m - 1; ++k) {
      term *= z / ((double)k * ((double)k - (double)m));
      s += term;
      if (term == 0.0) break;
    }
    double lg = log(2.0) + 2.0 * (double)m * hx - lgamma((double)m) - lgamma((double)m + 1.0);
    double lp = 0.0;
    if (lg > -740.0) {
      double Hm = 0.0;
      for (int q = 1; q <= m; ++q) Hm += 1.0 / (double)q;
      double inner = 0.0, tk = 1.0, Hk = 0.0, Hmk = Hm;
      for (int k = 0; k < 100000; ++k) {
        double add = tk * (hx + ORC_EULER_GAMMA - 0.5 * (Hk + Hmk));
        inner += add;
        if (k > 2 && fabs(add) <= 1e-18 * fabs(inner)) break;
        tk *= z / ((double)(k + 1) * (double)(m + k + 1));
        Hk += 1.0 / (double)(k + 1);
        Hmk += 1.0 / (double)(m + k + 1);
      }
      double sign = ((m + 1) % 2 == 0) ? 1.0 : -1.0;
      lp = sign * exp(lg) * inner;
    }
    return s + lp;
  } else {
    double s = 0.0, term = 1.0;
    for (int k = 1; k < 100000; ++k) {
      term *= z / ((double)k * ((double)k - mu));
      s += term;
      if (term == 0.0) break;
      if ((double)k > mu + 1.0 && fabs(term) <= 1e-18 * fabs(s)) break;
    }
    double sp = sin(M_PI * mu);
    double lg = log(M_PI) - log(fabs(sp)) - lgamma(mu) - lgamma(mu + 1.0) + 2.0 * mu * hx;
    double second = 0.0;
    if (lg > -740.0) second = -((sp > 0) ? 1.0 : -1.0) * exp(lg) * hyp0f1(1.0 + mu, z);
    return s + second;
  }
}

/* n = 3 closed forms (the Remark's G for n = 3):
 *   P(x) = 1 - e^{-x}(1+x),  Q(x) = x cosh x - sinh x. */
static double p3(double x) {
  if (x < 1.0) {
    double term = x, sum = 0.0;       /* term = x^k / k! */
    for (int k = 2; k < 200; ++k) {
      term *= x / (double)k;
      double add = ((k % 2 == 0) ? 1.0 : -1.0) * (double)(k - 1) * term;
      sum += add;
      if (fabs(add) <= 1e-18 * fabs(sum)) break;
    }
    return sum;
  }
  return 1.0 - exp(-x) * (1.0 + x);
}

static double q3(double x) {
  if (x < 1.0) {
    double term = x, sum = 0.0;       /* term = x^(2k+1)/(2k+1)! */
    for (int k = 1; k < 200; ++k) {
      term *= x * x / ((double)(2 * k) * (double)(2 * k + 1));
      double add = 2.0 * (double)k * term;
      sum += add;
      if (add <= 1e-18 * sum) break;
    }
    return sum;
  }
  return x * cosh(x) - sinh(x);
}

/* Radial CDF of |Z - y| / r under rho(y, .) (eq. Z_sampling_density).
 * With H(x) = x^{nu+1}[K_{nu+1}(x) + (K_nu(a)/I_nu(a)) I_{nu+1}(x)]/(2^nu Gamma(nu+1)),
 * Green's identity on the sub-ball of radius t r and the Wronskian
 * I_nu K_{nu+1} + I_{nu+1} K_nu = 1/x give F(t) = (1 - H(a t)) / (1 - c).
 * In normalised functions:
 *   1 - H(x) = [1 - K~_{nu+1}(x)] - c K~_nu(a) I~_{nu+1}(x) (x/2)^2 t^{2nu} / (nu(nu+1)).
 * n = 3 uses the elementary forms:
 *   1 - H(x) = P(x) - Q(x) e^{-a}/sinh(a),  e^{-a}/sinh(a) = 2/expm1(2a). */
double orc_green_cdf(int n, double a, double t) {
  if (t <= 0.0) return 0.0;
  if (t >= 1.0) return 1.0;
  double em1 = orc_em1(n, a);
  double c = 1.0 / (1.0 + em1);
  double omc = (em1 <= 1.0) ? em1 * c : 1.0 - c;
  double x = a * t;
  if (n == 3) {
    double second;
    if (x < 1.0) {
      second = q3(x) * (2.0 / expm1(2.0 * a));
    } else {
      /* Q(x) 2/(e^{2a}-1) = [(x-1) e^{x-2a} + (x+1) e^{-x-2a}] / (1 - e^{-2a}), no overflow */
      second = ((x - 1.0) * exp(x - 2.0 * a) + (x + 1.0) * exp(-x - 2.0 * a)) / (-expm1(-2.0 * a));
    }
    return (p3(x) - second) / omc;
  }
  double nu = 0.5 * (double)(n - 2);
  double sk = -orc_kt_minus_one(nu + 1.0, x);
  double kta = 1.0 + orc_kt_minus_one(nu, a);
  double it1 = hyp0f1(nu + 2.0, 0.25 * (x * x));
  double second = c * kta * it1 * (0.25 * (x * x)) * pow(t, 2.0 * nu) / (nu * (nu + 1.0));
  return (sk - second) / omc;
}

/* Inverse of the radial CDF by plain bisection on [0, 1] down to adjacent doubles. */
double orc_green_cdf_inv(int n, double a, double U) {
  if (U >= 1.0) return 1.0;
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 2000; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (orc_green_cdf(n, a, mid) < U) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------- */
/* Geometry: closest point (eq. cp_map), curvature indicator (eq.               */
/* rho_geo_curvature), effective boundary distance (eq. delta_Gamma_general).   */
/* ------------------------------------------------------------------------- */
static double dot(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void cloud_cp(const orc_manifold* m, const double* x, double* out);

/* ---- hypersurface of revolution (Example 2) ----------------------------- */
/* Profile R(t) = w(s) q(s), s = t/k, w = sqrt(1 - s^2), q = 1 - al + 2 al s^2,
 * and its first two t-derivatives (w' = -s/w, w'' = -1/w^3 in s). */
void orc_profile(const orc_manifold* m, double t, double* R, double* R1, double* R2) {
  double k = m->prof_kappa, al = m->prof_alpha;
  double s = t / k;
  double w = sqrt(1.0 - s * s);
  double q = 1.0 - al + 2.0 * al * s * s;
  double dw = -s / w, ddw = -1.0 / (w * w * w);
  double dq = 4.0 * al * s, ddq = 4.0 * al;
  *R = w * q;
  *R1 = (dw * q + w * dq) / k;
  *R2 = (ddw * q + 2.0 * dw * dq + w * ddq) / (k * k);
}

/* The closest point of M to x lies in x's meridian half-plane: minimise
 * D(t) = (R(t) - rho0)^2 + (t - t0)^2 (rho0 = |xh|, t0 = x_{n-1}) by Newton's
 * method on D'(t)/2 = (R - rho0) R' + (t - t0) from t = t0, kept inside
 * |t| <= k (1 - 1e-6); where the Newton derivative R'^2 + (R - rho0) R'' + 1
 * falls below 0.1 the Gauss-Newton one R'^2 + 1 is used.  Stops when a step
 * changes t by at most 1e-15 (1 + |t|), or after 60 steps. */
static double rev_cp_t(const orc_manifold* m, double rho0, double t0) {
  double lim = m->prof_kappa * (1.0 - 1e-6);
  double t = t0 < -lim ? -lim : (t0 > lim ? lim : t0);
  for (int it = 0; it < 60; ++it) {
    double R, R1, R2;
    orc_profile(m, t, &R, &R1, &R2);
    double F = (R - rho0) * R1 + (t - t0);
    double J = R1 * R1 + (R - rho0) * R2 + 1.0;
    if (!(J > 0.1)) J = R1 * R1 + 1.0;
    double tn = t - F / J;
    tn = tn < -lim ? -lim : (tn > lim ? lim : tn);
    if (fabs(tn - t) <= 1e-15 * (1.0 + fabs(t))) { t = tn; break; }
    t = tn;
  }
  return t;
}

/* ---- Fourier curve x sphere (Example 3) ----------------------------------- */
/* C(phi) = R (cos phi, sin phi, cos 2phi / 2, sin 2phi / 2, cos 3phi / 3, sin 3phi / 3)
 * and its first two phi-derivatives. */
static void fourier_curve(double R, double ph, double* C, double* C1, double* C2) {
  for (int k = 1; k <= 3; ++k) {
    double c = cos(k * ph), s = sin(k * ph);
    C[2 * k - 2] = R * c / k;
    C[2 * k - 1] = R * s / k;
    C1[2 * k - 2] = -R * s;
    C1[2 * k - 1] = R * c;
    C2[2 * k - 2] = -R * k * c;
    C2[2 * k - 1] = -R * k * s;
  }
}

/* Minimise |C(phi) - xh|^2 by Newton's method on C'.(C - xh) = 0 from the angle
 * of (x_1, x_2); where |C'|^2 + C''.(C - xh) falls below 0.1 |C'|^2 the
 * Gauss-Newton derivative |C'|^2 is used; stops at a step below 1e-15 (1 + |phi|)
 * or after 60 steps. */
double orc_curve_cp_phi(const orc_manifold* m, const double* x) {
  double ph = atan2(x[1], x[0]);
  for (int it = 0; it < 60; ++it) {
    double C[6], C1[6], C2[6];
    fourier_curve(m->R, ph, C, C1, C2);
    double F = 0.0, g2 = 0.0, h = 0.0;
    for (int i = 0; i < 6; ++i) {
      F += C1[i] * (C[i] - x[i]);
      g2 += C1[i] * C1[i];
      h += C2[i] * (C[i] - x[i]);
    }
    double J = g2 + h;
    if (!(J > 0.1 * g2)) J = g2;
    double pn = ph - F / J;
    if (fabs(pn - ph) <= 1e-15 * (1.0 + fabs(ph))) { ph = pn; break; }
    ph = pn;
  }
  return ph;
}

void orc_cp(const orc_manifold* m, const double* x, double* out) {
  int n = m->n;
  if (m->kind == ORC_EUCLID) {
    memcpy(out, x, sizeof(double) * (size_t)n);
  } else if (m->kind == ORC_SPHERE) {
    double nx = sqrt(dot(x, x, n));
    for (int i = 0; i < n; ++i) out[i] = x[i] / nx;
  } else if (m->kind == ORC_TORUS) {
    /* nearest point of the centre circle, then the tube of radius a around it */
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    double c[3] = {m->R * x[0] / rho, m->R * x[1] / rho, 0.0};
    double w[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    double nw = sqrt(dot(w, w, 3));
    double s = m->a / nw;
    for (int i = 0; i < 3; ++i) out[i] = c[i] + s * w[i];
  } else if (m->kind == ORC_POINT_CLOUD) {
    cloud_cp(m, x, out);
  } else if (m->kind == ORC_CURVE_SPHERE) {
    double ph = orc_curve_cp_phi(m, x);
    double C[6], C1[6], C2[6];
    fourier_curve(m->R, ph, C, C1, C2);
    for (int i = 0; i < 6; ++i) out[i] = C[i];
    double ns = sqrt(x[6] * x[6] + x[7] * x[7] + x[8] * x[8]);
    for (int i = 6; i < 9; ++i) out[i] = x[i] * (m->a / ns);
  } else if (m->kind == ORC_REVOLUTION) {
    double rho0 = 0.0;
    for (int i = 0; i < n - 1; ++i) rho0 += x[i] * x[i];
    rho0 = sqrt(rho0);
    double t = rev_cp_t(m, rho0, x[n - 1]);
    double R, R1, R2;
    orc_profile(m, t, &R, &R1, &R2);
    if (rho0 > 0.0) {
      for (int i = 0; i < n - 1; ++i) out[i] = x[i] * (R / rho0);
    } else {   /* on the axis: every direction is nearest; take e_1 */
      for (int i = 0; i < n - 1; ++i) out[i] = (i == 0) ? R : 0.0;
    }
    out[n - 1] = t;
  } else { /* embedded unit sphere: cp(x) = Q normalize(Q^T (x - b)) + b */
    int D = m->d + 1;
    double* s = (double*)malloc(sizeof(double) * (size_t)D);
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int i = 0; i < n; ++i) acc += m->Q[(size_t)i * D + j] * (x[i] - m->b[i]);
      s[j] = acc;
    }
    double ns = sqrt(dot(s, s, D));
    for (int j = 0; j < D; ++j) s[j] /= ns;
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < D; ++j) acc += m->Q[(size_t)i * D + j] * s[j];
      out[i] = acc + m->b[i];
    }
    free(s);
  }
}

/* ---- point cloud (Sec. 2.1 representation (iii); eq. rho_geo_spacing) ---- */
/* k nearest cloud points of x by brute force, ordered by (distance^2, index);
 * returns h(x), the mean distance to them. */
double orc_cloud_knn(const orc_manifold* m, const double* x, int64_t* idx, double* d2) {
  int k = m->k_nn;
  for (int j = 0; j < k; ++j) { d2[j] = INFINITY; idx[j] = -1; }
  for (int64_t i = 0; i < m->n_cloud; ++i) {
    const double* p = m->cloud + 3 * i;
    double dx = p[0] - x[0], dy = p[1] - x[1], dz = p[2] - x[2];
    double dd = dx * dx + dy * dy + dz * dz;
    if (dd < d2[k - 1]) {
      int j = k - 1;
      while (j > 0 && d2[j - 1] > dd) { d2[j] = d2[j - 1]; idx[j] = idx[j - 1]; --j; }
      d2[j] = dd;
      idx[j] = i;
    }
  }
  double h = 0.0;
  for (int j = 0; j < k; ++j) h += sqrt(d2[j]);
  return h / (double)k;
}

/* Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations;
 * V's columns are the eigenvectors. */
static void jacobi3(double A[3][3], double lam[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    if (off < 1e-300) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (A[p][q] == 0.0) continue;
        double th = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
        double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < 3; ++r) {          /* A <- A J */
          double arp = A[r][p], arq = A[r][q];
          A[r][p] = c * arp - s * arq;
          A[r][q] = s * arp + c * arq;
        }
        for (int r = 0; r < 3; ++r) {          /* A <- J^T A */
          double apr = A[p][r], aqr = A[q][r];
          A[p][r] = c * apr - s * aqr;
          A[q][r] = s * apr + c * aqr;
        }
        for (int r = 0; r < 3; ++r) {          /* V <- V J */
          double vrp = V[r][p], vrq = V[r][q];
          V[r][p] = c * vrp - s * vrq;
          V[r][q] = s * vrp + c * vrq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) lam[i] = A[i][i];
}

/* Solve the n x n system M a = b by Gaussian elimination with partial pivoting. */
static void gauss_solve(int n, double M[6][6], double b[6], double a[6]) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < n; ++j) { double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r][c] / M[c][c];
      for (int j = c; j < n; ++j) M[r][j] -= f * M[c][j];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < n; ++j) s -= M[r][j] * a[j];
    a[r] = s / M[r][r];
  }
}

/* cp on a point cloud: the k nearest points, their PCA plane at the centroid
 * (normal = eigenvector of the smallest covariance eigenvalue), an unweighted
 * least-squares quadratic height z = a0 + a1 u + a2 v + a3 u^2 + a4 uv + a5 v^2
 * in plane coordinates scaled by h(x), and the projection of x onto that graph:
 * the vertical foot point plus one Newton step on the squared distance.
 * Nearest mode: the nearest cloud point. */
static void cloud_cp(const orc_manifold* m, const double* x, double* out) {
  int k = m->k_nn;
  int64_t idx[64];
  double d2[64];
  double h = orc_cloud_knn(m, x, idx, d2);
  if (m->cp_mode == ORC_CP_NEAREST) {
    for (int i = 0; i < 3; ++i) out[i] = m->cloud[3 * idx[0] + i];
    return;
  }
  double c[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < 3; ++i) c[i] += m->cloud[3 * idx[j] + i];
  for (int i = 0; i < 3; ++i) c[i] /= (double)k;
  double C[3][3] = {{0}};
  for (int j = 0; j < k; ++j) {
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = m->cloud[3 * idx[j] + i] - c[i];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) C[a][b] += d[a] * d[b];
  }
  double lam[3], V[3][3];
  jacobi3(C, lam, V);
  int imin = 0, imax = 0;
  for (int i = 1; i < 3; ++i) {
    if (lam[i] < lam[imin]) imin = i;
    if (lam[i] > lam[imax]) imax = i;
  }
  double nrm[3] = {V[0][imin], V[1][imin], V[2][imin]};
  double u[3] = {V[0][imax], V[1][imax], V[2][imax]};
  double v[3] = {nrm[1] * u[2] - nrm[2] * u[1], nrm[2] * u[0] - nrm[0] * u[2], nrm[0] * u[1] - nrm[1] * u[0]};
  double s = h > 0.0 ? h : 1.0;
  double M[6][6] = {{0}}, rhs[6] = {0}, a[6];
  for (int j = 0; j < k; ++j) {
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = (m->cloud[3 * idx[j] + i] - c[i]) / s;
    double xi = dot(d, u, 3), et = dot(d, v, 3), ze = dot(d, nrm, 3);
    double row[6] = {1.0, xi, et, xi * xi, xi * et, et * et};
    for (int p = 0; p < 6; ++p) {
      rhs[p] += row[p] * ze;
      for (int q = 0; q < 6; ++q) M[p][q] += row[p] * row[q];
    }
  }
  gauss_solve(6, M, rhs, a);
  double d[3];
  for (int i = 0; i < 3; ++i) d[i] = (x[i] - c[i]) / s;
  double xi0 = dot(d, u, 3), et0 = dot(d, v, 3), ze0 = dot(d, nrm, 3);
  double hz = a[0] + a[1] * xi0 + a[2] * et0 + a[3] * xi0 * xi0 + a[4] * xi0 * et0 + a[5] * et0 * et0;
  double hx = a[1] + 2.0 * a[3] * xi0 + a[4] * et0;
  double hy = a[2] + a[4] * xi0 + 2.0 * a[5] * et0;
  double e = hz - ze0;
  double g0 = e * hx, g1 = e * hy;
  double H00 = 1.0 + hx * hx + e * 2.0 * a[3], H01 = hx * hy + e * a[4], H11 = 1.0 + hy * hy + e * 2.0 * a[5];
  double det = H00 * H11 - H01 * H01;
  double xi1 = xi0 - (H11 * g0 - H01 * g1) / det;
  double et1 = et0 - (H00 * g1 - H01 * g0) / det;
  double z1 = a[0] + a[1] * xi1 + a[2] * et1 + a[3] * xi1 * xi1 + a[4] * xi1 * et1 + a[5] * et1 * et1;
  for (int i = 0; i < 3; ++i) out[i] = c[i] + s * (xi1 * u[i] + et1 * v[i] + z1 * nrm[i]);
}

/* largest absolute principal curvature at y on a hypersurface of revolution:
 * the meridian |R''| / (1 + R'^2)^{3/2} and the n-2 parallel ones
 * 1 / (R (1 + R'^2)^{1/2}) */
double orc_kappa_at(const orc_manifold* m, const double* y);

static double kappa_of(const orc_manifold* m) {
  /* largest absolute principal curvature (constant on these manifolds) */
  if (m->kind == ORC_EUCLID) return 0.0;
  if (m->kind == ORC_TORUS) return 1.0 / m->a;
  if (m->kind == ORC_CURVE_SPHERE) {
    /* the curve has constant speed |C'| = sqrt(3) R and |C''| = sqrt(14) R, so its
     * curvature is sqrt(14) / (3 R); the sphere's is 1/a */
    double kc = sqrt(14.0) / (3.0 * m->R), ks = 1.0 / m->a;
    return kc > ks ? kc : ks;
  }
  return 1.0; /* unit sphere, embedded unit sphere */
}

double orc_kappa_at(const orc_manifold* m, const double* y) {
  if (m->kind != ORC_REVOLUTION) return kappa_of(m);
  double R, R1, R2;
  orc_profile(m, y[m->n - 1], &R, &R1, &R2);
  double G = sqrt(1.0 + R1 * R1);
  double km = fabs(R2) / (G * G * G), kp = 1.0 / (R * G);
  return km > kp ? km : kp;
}

/* delta_Gamma(y) = ( |P_T r_Gamma|^2 + (|P_N r_Gamma| - ell)_+^2 )^{1/2},
 * r_Gamma = y_Gamma - y, ell = rho_geo(y_Gamma).  Boundary: half-space
 * {e.x > h} intersected with M (unit sphere or Euclidean space).  A state with
 * e.y <= h is outside Omega and counts as inside the boundary layer (0). */
double orc_delta_gamma(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                       const double* y, double* yg) {
  int n = m->n;
  const double* e = pb->bnd_normal;
  double h = pb->bnd_offset;
  double ey = dot(e, y, n);
  double ell = pr->c_kappa / (1.0 + kappa_of(m));
  if (m->kind == ORC_EUCLID) {
    for (int i = 0; i < n; ++i) yg[i] = y[i] - (ey - h) * e[i];
    double d = fabs(ey - h);
    return (ey <= h) ? 0.0 : d;
  }
  if (m->kind == ORC_TORUS) {
    /* a plane through the torus axis (e_3 = 0, h = 0), as in Example 1's cut:
     * Gamma is the two meridian circles c_b + a (cos t u_b + sin t e_3), with
     * centres c_b = R u_b, u_0 = (-e_2, e_1, 0), u_1 = -u_0.  The nearest point
     * of circle b to y is c_b + a w/|w|, w = the part of y - c_b in the
     * circle's plane span(u_b, e_3); the nearer circle wins (circle 0 on a tie).
     * The torus normal at y_Gamma is w/|w|. */
    double best = INFINITY, nrm[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 2; ++b) {
      double sgn = (b == 0) ? 1.0 : -1.0;
      double u[3] = {-sgn * e[1], sgn * e[0], 0.0};
      double c[3] = {m->R * u[0], m->R * u[1], 0.0};
      double wu = (y[0] - c[0]) * u[0] + (y[1] - c[1]) * u[1];
      double wz = y[2];
      double w[3] = {wu * u[0], wu * u[1], wz};
      double nw = sqrt(wu * wu + wz * wz);
      double nb[3];
      if (nw > 0.0) {
        for (int i = 0; i < 3; ++i) nb[i] = w[i] / nw;
      } else {   /* y on the circle's axis: every point of the circle is nearest; take t = 0 */
        for (int i = 0; i < 3; ++i) nb[i] = u[i];
      }
      double q[3], d2 = 0.0;
      for (int i = 0; i < 3; ++i) {
        q[i] = c[i] + m->a * nb[i];
        d2 += (q[i] - y[i]) * (q[i] - y[i]);
      }
      if (d2 < best) {
        best = d2;
        for (int i = 0; i < 3; ++i) { yg[i] = q[i]; nrm[i] = nb[i]; }
      }
    }
    double rn = 0.0;
    for (int i = 0; i < 3; ++i) rn += (yg[i] - y[i]) * nrm[i];
    double rt2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      double rti = (yg[i] - y[i]) - rn * nrm[i];
      rt2 += rti * rti;
    }
    if (ey <= h) return 0.0;
    double ex = fabs(rn) - ell;
    if (ex < 0.0) ex = 0.0;
    return sqrt(rt2 + ex * ex);
  }
  /* unit sphere: y_Gamma = h e + sqrt(1-h^2) w/|w|, w = y - (e.y) e */
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i < n; ++i) w[i] = y[i] - ey * e[i];
  double nw = sqrt(dot(w, w, n));
  if (nw == 0.0) {
    /* non-unique nearest point: lowest-index axis not parallel to e */
    for (int j = 0; j < n; ++j) {
      for (int i = 0; i < n; ++i) w[i] = ((i == j) ? 1.0 : 0.0) - e[j] * e[i];
      nw = sqrt(dot(w, w, n));
      if (nw > 1e-8) break;
    }
  }
  double sh = sqrt(1.0 - h * h);
  for (int i = 0; i < n; ++i) yg[i] = h * e[i] + sh * (w[i] / nw);
  /* r_Gamma, its normal part along y_Gamma (the sphere's unit normal there) */
  double rn = 0.0;
  for (int i = 0; i < n; ++i) rn += (yg[i] - y[i]) * yg[i];
  double rt2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double rti = (yg[i] - y[i]) - rn * yg[i];
    rt2 += rti * rti;
  }
  free(w);
  if (ey <= h) return 0.0;
  double ex = fabs(rn) - ell;
  if (ex < 0.0) ex = 0.0;
  return sqrt(rt2 + ex * ex);
}

/* ------------------------------------------------------------------------- */
/* Problem data f, g evaluated at a point x of M.                              */
/* ------------------------------------------------------------------------- */
/* SPHERE_QUAD at the direction of s in R^{d+1} (normalised here):
 * u = c0 + v.s + s^T A s, or (-Delta_{S^d} + sigma) u when apply_op. */
static double quad_at(const orc_func* f, int d_dim, double sigma, const double* s_in) {
  int D = d_dim + 1;   /* <= 32 */
  double s[32];
  double ns = sqrt(dot(s_in, s_in, D));
  for (int j = 0; j < D; ++j) s[j] = s_in[j] / ns;
  double lin = dot(f->v, s, D);
  double quad = 0.0, tr = 0.0;
  for (int i = 0; i < D; ++i) {
    tr += f->A[(size_t)i * D + i];
    for (int j = 0; j < D; ++j) quad += f->A[(size_t)i * D + j] * s[i] * s[j];
  }
  if (!f->apply_op) return f->c0 + lin + quad;
  /* on S^d: degree-k harmonics have -Delta eigenvalue k(k+d-1); s^T A s splits
   * into its trace-free part (k = 2) and the constant tr(A)/(d+1). */
  double d = (double)d_dim;
  double mean = tr / (double)D;
  return sigma * (f->c0 + mean) + (d + sigma) * lin + (2.0 * (d + 1.0) + sigma) * (quad - mean);
}

static double trig(int kind, double v) { return kind == 0 ? cos(v) : sin(v); }

double orc_func_eval(const orc_manifold* m, const orc_func* f, double sigma, const double* x) {
  if (f->kind == ORC_POLY) {
    double total = 0.0;
    for (int t = 0; t < f->n_terms; ++t) {
      double prod = f->coef[t];
      for (int q = f->term_off[t]; q < f->term_off[t + 1]; ++q)
        for (int e = 0; e < f->pw[q]; ++e) prod *= x[f->var[q]];
      total += prod;
    }
    return total;
  }
  if (f->kind == ORC_TORUS_FOURIER) {
    double R = m->R, a = m->a;
    double rho = sqrt(x[0] * x[0] + x[1] * x[1]);
    double th = atan2(x[2], rho - R);
    double ph = atan2(x[1], x[0]);
    double ct = cos(th), st = sin(th);
    double total = 0.0;
    for (int t = 0; t < f->n_terms; ++t) {
      int mm = f->modes[4 * t], q = f->modes[4 * t + 1];
      int tk = f->modes[4 * t + 2], pk = f->modes[4 * t + 3];
      double T = trig(tk, mm * th);
      double P = trig(pk, q * ph);
      double val;
      if (!f->apply_op) {
        val = T * P;
      } else {
        /* -Delta_T of T(theta)P(phi) on the torus (R + a cos th) e_r + a sin th e_z:
         * P [ m^2 T / a^2 + sin th T' / (a (R + a cos th)) + q^2 T / (R + a cos th)^2 ] */
        double Tp = (tk == 0) ? -(double)mm * sin(mm * th) : (double)mm * cos(mm * th);
        double rr = R + a * ct;
        double lap = (double)(mm * mm) * T / (a * a) + st * Tp / (a * rr) + (double)(q * q) * T / (rr * rr);
        val = P * (lap + sigma * T);
      }
      total += f->coef[t] * val;
    }
    return total;
  }
  if (f->kind == ORC_REVOLUTION_QUAD) {
    /* u = c0 + c1 t + c2 t^2 + v.xh + sum_j A_j xh_j^2 on |xh| = R(t).  With xh = R w
     * (w on the unit sphere S^{n-2}), u = h0(t) + R (v.w) + R^2 (w^T A w - mA),
     * h0 = c0 + c1 t + c2 t^2 + mA R^2, mA = tr(A)/(n-1): degree-0, 1 and 2 spherical
     * harmonics with -Delta_{S^{n-2}} eigenvalues 0, n-2 and 2(n-1).  On the
     * surface of revolution (metric (1 + R'^2) dt^2 + R^2 dw^2),
     *   Delta_M (h(t) Y_k) = [ (h'' + (n-2) R' h'/R - h' R' R''/(1+R'^2)) / (1+R'^2)
     *                          - lambda_k h / R^2 ] Y_k. */
    int n = m->n;
    double t = x[n - 1];
    double R, R1, R2;
    orc_profile(m, t, &R, &R1, &R2);
    double rh = 0.0, vw = 0.0, aw = 0.0, trA = 0.0;
    for (int i = 0; i < n - 1; ++i) rh += x[i] * x[i];
    rh = sqrt(rh);
    for (int i = 0; i < n - 1; ++i) {
      double wi = x[i] / rh;
      vw += f->v[i] * wi;
      aw += f->A[i] * wi * wi;
      trA += f->A[i];
    }
    double c1 = f->coef[0], c2 = f->coef[1];
    double mA = trA / (double)(n - 1);
    double u = f->c0 + c1 * t + c2 * t * t + R * vw + R * R * aw;
    if (!f->apply_op) return u;
    double md = (double)(n - 2), G2 = 1.0 + R1 * R1;
    double h0p = c1 + 2.0 * c2 * t + 2.0 * mA * R * R1;
    double h0pp = 2.0 * c2 + 2.0 * mA * (R1 * R1 + R * R2);
    double L0 = (h0pp + md * R1 * h0p / R - h0p * R1 * R2 / G2) / G2;
    double L1 = (R2 + md * R1 * R1 / R - R1 * R1 * R2 / G2) / G2 - md / R;
    double h2p = 2.0 * R * R1, h2pp = 2.0 * R1 * R1 + 2.0 * R * R2;
    double L2 = (h2pp + md * R1 * h2p / R - h2p * R1 * R2 / G2) / G2 - 2.0 * (md + 1.0);
    return -L0 - L1 * vw - L2 * (aw - mA) + sigma * u;
  }
  if (f->kind == ORC_CURVE_SPHERE_FUNC) {
    /* at x = (C(phi), a w): u = sum_t T_t(q_t phi) S_t(w), S_t = c_t + v_t.w + w^T A_t w.
     * Delta_M = Delta_curve + Delta_{S^2(a)}; the curve has constant speed sqrt(3) R, so
     * -Delta_curve T(q phi) = q^2 T / (3 R^2); on S^2(a) v.w has -Delta eigenvalue 2/a^2,
     * the trace-free part of w^T A w 6/a^2, constants 0. */
    double ph = atan2(x[1], x[0]);
    double ns = sqrt(x[6] * x[6] + x[7] * x[7] + x[8] * x[8]);
    double w[3] = {x[6] / ns, x[7] / ns, x[8] / ns};
    double total = 0.0;
    for (int t = 0; t < f->n_terms; ++t) {
      int q = f->modes[4 * t], tk = f->modes[4 * t + 1];
      const double* v = f->v + 3 * t;
      const double* A = f->A + 9 * t;
      double lin = v[0] * w[0] + v[1] * w[1] + v[2] * w[2];
      double quad = 0.0, tr = A[0] + A[4] + A[8];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) quad += A[3 * i + j] * w[i] * w[j];
      double St = f->coef[t] + lin + quad;
      double T = trig(tk, q * ph);
      if (!f->apply_op) {
        total += T * St;
      } else {
        double a2 = m->a * m->a;
        double lap = (double)(q * q) / (3.0 * m->R * m->R) * St + 2.0 / a2 * lin + 6.0 / a2 * (quad - tr / 3.0);
        total += T * (lap + sigma * St);
      }
    }
    return total;
  }
  /* sphere quad: intrinsic unit vector s of the round sphere S^d */
  int D = m->d + 1;
  double* s = (double*)malloc(sizeof(double) * (size_t)D);
  if (m->kind == ORC_EMBEDDED_SPHERE) {
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int i = 0; i < m->n; ++i) acc += m->Q[(size_t)i * D + j] * (x[i] - m->b[i]);
      s[j] = acc;
    }
  } else {
    for (int j = 0; j < D; ++j) s[j] = x[j];
  }
  double val = quad_at(f, m->d, sigma, s);
  free(s);
  return val;
}

/* ------------------------------------------------------------------------- */
/* Compensation term (Sec. 2.3.3).  For x near M write x = y + eta n(y), y =   */
/* cp(x), eta the signed normal distance (n the outward unit normal).  With a  */
/* predictor u_*,                                                             */
/*   R_*(s; y) = -Delta(E u_*)(y + s n(y)) + sigma u_*(y) - f(y),             */
/*   m1 = (R_*(h) - R_*(-h)) / (2h),  m2 = (R_*(h) - 2 R_*(0) + R_*(-h)) / h^2, */
/*   m_*(x) = eta m1(y) + eta^2 m2(y) / 2,                                     */
/* and the source of a step becomes f(cp(Z)) + m_*(Z).  E u_* = u_* o cp is   */
/* constant along normals, so its ambient Laplacian at y + s n(y) is the      */
/* Laplacian of a function of the tangential coordinates alone:               */
/*   unit sphere of R^3 (normal coordinate rho = 1 + s):                      */
/*     -Delta(E u)(rho y) = (-Delta_S u)(y) / rho^2;                          */
/*   torus (rho = a + s the distance from the centre circle, angles th, ph):  */
/*     -Delta(E u) = -[u_thth / rho^2 - sin th u_th / (rho (R + rho cos th))  */
/*                     + u_phph / (R + rho cos th)^2]                         */
/*   (the Laplacian in the coordinates (rho, th, ph), whose metric is         */
/*   d rho^2 + rho^2 d th^2 + (R + rho cos th)^2 d ph^2).                     */
/* ------------------------------------------------------------------------- */
double orc_normal_coord(const orc_manifold* m, const double* x) {
  if (m->kind == ORC_TORUS) {
    double rxy = sqrt(x[0] * x[0] + x[1] * x[1]);
    double dr = rxy - m->R;
    return sqrt(dr * dr + x[2] * x[2]) - m->a;
  }
  return sqrt(dot(x, x, 3)) - 1.0;   /* unit sphere of R^3 */
}

/* -Delta(E u_*) at y + s n(y), y on M */
static double ext_neg_lap(const orc_manifold* m, const orc_func* u, const double* y, double s) {
  if (m->kind == ORC_TORUS) {
    double R = m->R;
    double rxy = sqrt(y[0] * y[0] + y[1] * y[1]);
    double dr = rxy - R;
    double nr = sqrt(dr * dr + y[2] * y[2]);
    double ct = dr / nr, st = y[2] / nr;
    double th = atan2(y[2], dr), ph = atan2(y[1], y[0]);
    double utt = 0.0, ut = 0.0, upp = 0.0;
    for (int t = 0; t < u->n_terms; ++t) {
      int mm = u->modes[4 * t], q = u->modes[4 * t + 1];
      int tk = u->modes[4 * t + 2], pk = u->modes[4 * t + 3];
      double T = trig(tk, mm * th);
      double Tp = (tk == 0) ? -(double)mm * sin(mm * th) : (double)mm * cos(mm * th);
      double P = trig(pk, q * ph);
      utt += u->coef[t] * (-(double)(mm * mm) * T * P);
      ut += u->coef[t] * (Tp * P);
      upp += u->coef[t] * (-(double)(q * q) * T * P);
    }
    double rho = m->a + s;
    double rr = R + rho * ct;
    return -(utt / (rho * rho) - st * ut / (rho * rr) + upp / (rr * rr));
  }
  /* unit sphere of R^3, quadratic u = c0 + v.y + y^T A y: the degree-1 part is
   * an eigenfunction of -Delta_S with eigenvalue 2, the trace-free quadratic
   * part with eigenvalue 6 (the constant tr(A)/3 with 0) */
  double ny = sqrt(dot(y, y, 3));
  double w[3] = {y[0] / ny, y[1] / ny, y[2] / ny};
  double lin = dot(u->v, w, 3), quad = 0.0, tr = 0.0;
  for (int i = 0; i < 3; ++i) {
    tr += u->A[i * 3 + i];
    for (int j = 0; j < 3; ++j) quad += u->A[i * 3 + j] * w[i] * w[j];
  }
  double lam = 2.0 * lin + 6.0 * (quad - tr / 3.0);
  double rho = 1.0 + s;
  return lam / (rho * rho);
}

static double comp_R(const orc_manifold* m, const orc_problem* pb, const double* y, double s, double fy) {
  return (ext_neg_lap(m, &pb->u_star, y, s) + pb->sigma * orc_func_eval(m, &pb->u_star, pb->sigma, y)) - fy;
}

/* m_*(x) with y = cp(x) and fy = f(y) already known */
static double comp_m(const orc_manifold* m, const orc_problem* pb, const double* x, const double* y, double fy) {
  double eta = orc_normal_coord(m, x);
  if (pb->comp == ORC_COMP_EXACT) return comp_R(m, pb, y, eta, fy);
  double h = pb->h_eta;
  double Rp = comp_R(m, pb, y, h, fy);
  double R0 = comp_R(m, pb, y, 0.0, fy);
  double Rm = comp_R(m, pb, y, -h, fy);
  double m1 = (Rp - Rm) / (2.0 * h);
  double m2 = (Rp - 2.0 * R0 + Rm) / (h * h);
  return eta * m1 + 0.5 * eta * eta * m2;
}

double orc_comp_R(const orc_manifold* m, const orc_problem* pb, const double* y, double s) {
  return comp_R(m, pb, y, s, orc_func_eval(m, &pb->f, pb->sigma, y));
}

double orc_comp_m(const orc_manifold* m, const orc_problem* pb, const double* x) {
  double y[3];
  orc_cp(m, x, y);
  return comp_m(m, pb, x, y, orc_func_eval(m, &pb->f, pb->sigma, y));
}

/* ------------------------------------------------------------------------- */
/* One walk (Algorithm 1 + eq. path_score_definition).                          */
/*   blocks of step k: Theta direction [0, nb); Z_l direction                   */
/*   [nb(1+l), nb(2+l)); U_l at nb(1+N_V) + l;  nb = ceil(n/2).                 */
/* ------------------------------------------------------------------------- */
typedef struct {
  double *Y, *Th, *Z, *cZ, *g, *yg;
} work_t;

static void work_alloc(work_t* w, int n) {
  w->Y = (double*)malloc(sizeof(double) * (size_t)n * 6);
  w->Th = w->Y + n; w->Z = w->Th + n; w->cZ = w->Z + n; w->g = w->cZ + n; w->yg = w->g + n;
}
static void work_free(work_t* w) { free(w->Y); }

static int run_walk(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                    const double* y0, uint32_t p, uint32_t i, work_t* w,
                    double* S_out, int64_t* K_out, orc_trace_rec* rec, int64_t cap, int64_t* nrec) {
  int n = m->n;
  uint32_t nb = (uint32_t)((n + 1) / 2);
  double sqs = sqrt(pb->sigma);
  memcpy(w->Y, y0, sizeof(double) * (size_t)n);
  double W = 1.0, S = 0.0;
  int64_t k = 0;
  int flag = 0;
  for (;;) {
    double dG = INFINITY;
    if (!pb->closed) {
      dG = orc_delta_gamma(m, pb, pr, w->Y, w->yg);
      if (dG < pr->eps) {
        S += W * orc_func_eval(m, &pb->g, pb->sigma, w->yg);
        break;
      }
      /* W = 0 (underflow): every later term of the score is multiplied by W,
       * so stopping is exact. */
      if (W == 0.0) break;
    } else if (W < pr->tau_w) {
      break;
    }
    if (k >= pr->max_steps) { flag = 1; break; }
    double rgeo;
    if (m->kind == ORC_POINT_CLOUD) {
      int64_t idx[64];
      double d2[64];
      rgeo = m->c_h * orc_cloud_knn(m, w->Y, idx, d2);   /* eq. rho_geo_spacing */
    } else {
      rgeo = pr->c_kappa / (1.0 + orc_kappa_at(m, w->Y));   /* eq. rho_geo_curvature */
    }
    double r = pr->theta * (dG < rgeo ? dG : rgeo);
    double a = sqs * r;
    double em1 = orc_em1(n, a);
    double c = 1.0 / (1.0 + em1);
    /* 1 - c = em1/(1+em1) without cancellation; 1 - c directly once c <= 1/2 */
    double omega = ((em1 <= 1.0) ? em1 * c : 1.0 - c) / pb->sigma;
    /* Theta = Y + r g/|g| */
    orc_gaussians(pr->seed, 0u, (uint32_t)k, i, p, n, w->g);
    double gn = sqrt(dot(w->g, w->g, n));
    double sc = r / gn;
    for (int q = 0; q < n; ++q) w->Th[q] = w->Y[q] + sc * w->g[q];
    /* F_k: N_V interior samples */
    double F = 0.0, U0 = 0.0, t0 = 0.0;
    for (int l = 0; l < pr->n_v; ++l) {
      double U = uniform_at(pr->seed, nb * (uint32_t)(1 + pr->n_v) + (uint32_t)l, (uint32_t)k, i, p);
      double t = orc_green_cdf_inv(n, a, U);
      if (l == 0) { U0 = U; t0 = t; }
      orc_gaussians(pr->seed, nb * (uint32_t)(1 + l), (uint32_t)k, i, p, n, w->g);
      double zn = sqrt(dot(w->g, w->g, n));
      double zs = (r * t) / zn;
      for (int q = 0; q < n; ++q) w->Z[q] = w->Y[q] + zs * w->g[q];
      orc_cp(m, w->Z, w->cZ);
      double fz = orc_func_eval(m, &pb->f, pb->sigma, w->cZ);
      if (pb->comp != ORC_COMP_NONE) fz = fz + comp_m(m, pb, w->Z, w->cZ, fz);   /* f + m_* */
      F += fz;
    }
    if (pr->n_v > 1) F /= (double)pr->n_v;
    S += (W * omega) * F;
    W *= c;
    orc_cp(m, w->Th, w->Y);
    if (rec && *nrec < cap) {
      orc_trace_rec* R = &rec[*nrec];
      R->k = k; R->r = r; R->c = c; R->omega = omega; R->delta_gamma = dG; R->W = W; R->S = S;
      R->F = F; R->U0 = U0; R->t0 = t0; R->theta_norm = gn;
      for (int q = 0; q < 3; ++q) R->y[q] = q < n ? w->Y[q] : 0.0;
      (*nrec)++;
    }
    k++;
  }
  *S_out = S;
  *K_out = k;
  return flag;
}

/* ------------------------------------------------------------------------- */
/* Dimension-reduced exact sampler (an exact reformulation of the same walk;  */
/* the paper draws full n-dimensional directions).  A step uses the n        */
/* Gaussians g of a direction only through                                    */
/*   - embedded sphere Q S^d + b: Q^T g (the intrinsic step) and |g|^2;       */
/*   - sphere / R^n: the coordinates T that f, g and the boundary normal      */
/*     read, |g|^2, and (sphere) the component of g along Y's part outside T. */
/* For g ~ N(0, I_n) these are independent N(0,1) variables and a chi^2 with  */
/* the remaining number of dimensions (n - D, n - |T| - 1 or n - |T|), so     */
/* drawing them directly gives the same law of the walk.  The state kept is   */
/* s (embedded sphere), or Y with T coordinates and, for the sphere, the norm */
/* of the rest in one spare coordinate (which keeps |Y| and e.Y exact).       */
/*   draws of vector v (0: Theta, 1 + l: Z_l) at step k:                      */
/*     Gaussians: blocks 64 v, 64 v + 1, ... (two per block, orc_gaussians);  */
/*       on a sphere the first is the component along Y's rest, then T's      */
/*     chi^2:     from block 64 v + 32 (orc_chi2)                             */
/*     U_l:       block 64 (1 + N_V) + l, u53(words 0, 1)                     */
/* ------------------------------------------------------------------------- */
#define ORC_CHI2_ATTEMPTS 16

double orc_chi2(uint64_t seed, uint32_t j0, uint32_t k, uint32_t i, uint32_t p, int m) {
  if (m <= 0) return 0.0;
  double x;
  if (m == 1) {
    orc_gaussians(seed, j0, k, i, p, 1, &x);
    return x * x;
  }
  /* Marsaglia & Tsang (ACM TOMS 26, 2000): Gamma(alpha) for alpha = m/2 >= 1 by
   * squeezing (1 + c x)^3, x ~ N(0,1), with the exact log acceptance test; an
   * attempt that finds v <= 0 is rejected.  chi^2_m = 2 Gamma(m/2).  After 16
   * rejections (probability below 1e-20 for every m >= 2) the last candidate
   * is returned. */
  double d = 0.5 * (double)m - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double cand = d;
  for (uint32_t a = 0; a < ORC_CHI2_ATTEMPTS; ++a) {
    orc_gaussians(seed, j0 + 2u * a, k, i, p, 1, &x);
    double v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    cand = d * v;
    double U = uniform_at(seed, j0 + 2u * a + 1u, k, i, p);
    if (log(U) < 0.5 * x * x + d - d * v + d * log(v)) return 2.0 * d * v;
  }
  return 2.0 * cand;
}

static void mark_poly(const orc_func* f, int* used) {
  if (f->kind != ORC_POLY) return;
  for (int t = 0; t < f->n_terms; ++t)
    for (int q = f->term_off[t]; q < f->term_off[t + 1]; ++q) used[f->var[q]] = 1;
}

int orc_tracked_set(const orc_manifold* m, const orc_problem* pb, int* T) {
  if (pb->f.kind != ORC_POLY || (!pb->closed && pb->g.kind != ORC_POLY)) return -1;
  int* used = (int*)calloc((size_t)m->n, sizeof(int));
  mark_poly(&pb->f, used);
  if (!pb->closed) {
    mark_poly(&pb->g, used);
    for (int q = 0; q < m->n; ++q)
      if (pb->bnd_normal[q] != 0.0) used[q] = 1;
  }
  int nT = 0;
  for (int q = 0; q < m->n; ++q)
    if (used[q]) {
      if (nT == 32) { free(used); return -1; }
      T[nT++] = q;
    }
  free(used);
  return nT;
}

static int run_walk_reduced(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                            const double* y0, uint32_t p, uint32_t i, work_t* w,
                            double* S_out, int64_t* K_out) {
  int n = m->n;
  int emb = m->kind == ORC_EMBEDDED_SPHERE, sph = m->kind == ORC_SPHERE;
  int D = m->d + 1;
  int T[32], nT, spare = -1;
  if (emb) {
    nT = D;
  } else {
    nT = orc_tracked_set(m, pb, T);
    if (sph)
      for (int q = 0; q < n && spare < 0; ++q) {
        int inT = 0;
        for (int t = 0; t < nT; ++t) inT |= (T[t] == q);
        if (!inT) spare = q;
      }
  }
  int ng = nT + (sph ? 1 : 0);                      /* Gaussians per direction */
  int rest = emb ? n - D : (sph ? n - nT - 1 : n - nT);   /* chi^2 degrees of freedom */
  double sqs = sqrt(pb->sigma);
  double g[33], s[32], th[32], z[32];
  /* state: embedded sphere s = normalize(Q^T (y0 - b)); otherwise Y canonical */
  memset(w->Y, 0, sizeof(double) * (size_t)n);
  if (emb) {
    double ns = 0.0;
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int q = 0; q < n; ++q) acc += m->Q[(size_t)q * D + j] * (y0[q] - m->b[q]);
      s[j] = acc;
      ns += acc * acc;
    }
    for (int j = 0; j < D; ++j) s[j] /= sqrt(ns);
  } else {
    double tt = 0.0;
    for (int t = 0; t < nT; ++t) {
      w->Y[T[t]] = y0[T[t]];
      tt += y0[T[t]] * y0[T[t]];
    }
    if (sph) {
      double yy = dot(y0, y0, n);
      w->Y[spare] = sqrt(yy - tt > 0.0 ? yy - tt : 0.0);
    }
  }
  double W = 1.0, S = 0.0;
  int64_t k = 0;
  int flag = 0;
  for (;;) {
    double dG = INFINITY;
    if (!pb->closed) {
      dG = orc_delta_gamma(m, pb, pr, w->Y, w->yg);
      if (dG < pr->eps) {
        S += W * orc_func_eval(m, &pb->g, pb->sigma, w->yg);
        break;
      }
      if (W == 0.0) break;
    } else if (W < pr->tau_w) {
      break;
    }
    if (k >= pr->max_steps) { flag = 1; break; }
    double rgeo = pr->c_kappa / (1.0 + kappa_of(m));
    double r = pr->theta * (dG < rgeo ? dG : rgeo);
    double a = sqs * r;
    double em1 = orc_em1(n, a);
    double c = 1.0 / (1.0 + em1);
    double omega = ((em1 <= 1.0) ? em1 * c : 1.0 - c) / pb->sigma;
    /* F_k: N_V interior samples Z_l = Y + R_l g_l/|g_l| */
    double F = 0.0;
    for (int l = 0; l < pr->n_v; ++l) {
      uint32_t jv = 64u * (uint32_t)(1 + l);
      double U = uniform_at(pr->seed, 64u * (uint32_t)(1 + pr->n_v) + (uint32_t)l, (uint32_t)k, i, p);
      double t = orc_green_cdf_inv(n, a, U);
      orc_gaussians(pr->seed, jv, (uint32_t)k, i, p, ng, g);
      double X = orc_chi2(pr->seed, jv + 32u, (uint32_t)k, i, p, rest);
      double zs = (r * t) / sqrt(dot(g, g, ng) + X);
      const double* gT = g + (sph ? 1 : 0);   /* sphere: g[0] is the component along Y's rest */
      if (emb) {
        for (int j = 0; j < D; ++j) z[j] = s[j] + zs * gT[j];
        F += quad_at(&pb->f, m->d, pb->sigma, z);
      } else {
        memcpy(w->Z, w->Y, sizeof(double) * (size_t)n);
        for (int q = 0; q < nT; ++q) w->Z[T[q]] += zs * gT[q];
        if (sph) {
          double zr = w->Y[spare] + zs * g[0];
          w->Z[spare] = sqrt(zr * zr + zs * zs * X);
        }
        orc_cp(m, w->Z, w->cZ);
        F += orc_func_eval(m, &pb->f, pb->sigma, w->cZ);
      }
    }
    if (pr->n_v > 1) F /= (double)pr->n_v;
    /* Theta = Y + r g/|g|, Y = cp(Theta) */
    orc_gaussians(pr->seed, 0u, (uint32_t)k, i, p, ng, g);
    double X = orc_chi2(pr->seed, 32u, (uint32_t)k, i, p, rest);
    double sc = r / sqrt(dot(g, g, ng) + X);
    const double* gT = g + (sph ? 1 : 0);
    if (emb) {
      for (int j = 0; j < D; ++j) th[j] = s[j] + sc * gT[j];
      double tn = sqrt(dot(th, th, D));
      for (int j = 0; j < D; ++j) s[j] = th[j] / tn;
    } else {
      memcpy(w->Th, w->Y, sizeof(double) * (size_t)n);
      for (int q = 0; q < nT; ++q) w->Th[T[q]] += sc * gT[q];
      if (sph) {
        double tr_ = w->Y[spare] + sc * g[0];
        w->Th[spare] = sqrt(tr_ * tr_ + sc * sc * X);
      }
    }
    S += (W * omega) * F;
    W *= c;
    if (!emb) orc_cp(m, w->Th, w->Y);
    k++;
  }
  *S_out = S;
  *K_out = k;
  return flag;
}

/* The forms this oracle implements: a torus boundary is a plane through the
 * axis; compensation runs on the torus (TORUS_FOURIER predictor) and the unit
 * sphere of R^3 (SPHERE_QUAD predictor).  Returns -1 for anything else. */
static int check_problem(const orc_manifold* m, const orc_problem* pb) {
  if (m->kind == ORC_REVOLUTION && (!pb->closed || m->n < 4 || pb->f.kind != ORC_REVOLUTION_QUAD || pb->comp))
    return -1;
  if (m->kind == ORC_CURVE_SPHERE && (!pb->closed || m->n != 9 || pb->f.kind != ORC_CURVE_SPHERE_FUNC || pb->comp))
    return -1;
  if (m->kind == ORC_TORUS && !pb->closed && (pb->bnd_normal[2] != 0.0 || pb->bnd_offset != 0.0)) return -1;
  if (pb->comp == ORC_COMP_NONE) return 0;
  if (pb->comp != ORC_COMP_NORMAL2 && pb->comp != ORC_COMP_EXACT) return -1;
  if ((pb->comp == ORC_COMP_NORMAL2 && !(pb->h_eta > 0.0)) || pb->u_star.apply_op) return -1;
  if (m->kind == ORC_TORUS && pb->u_star.kind == ORC_TORUS_FOURIER) return 0;
  if (m->kind == ORC_SPHERE && m->n == 3 && pb->u_star.kind == ORC_SPHERE_QUAD) return 0;
  return -1;
}

int orc_walk_scores(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                    const double* pts, int64_t P, int64_t N, double* S, int64_t* K,
                    int32_t* flags, int n_threads) {
  if (check_problem(m, pb) != 0) return -1;
  int nt = 1;
#ifdef _OPENMP
  nt = n_threads > 0 ? n_threads : omp_get_max_threads();   /* this call only: no process-wide setting */
#endif
  (void)nt;
  int64_t total = P * N;
#pragma omp parallel num_threads(nt)
  {
    work_t w;
    work_alloc(&w, m->n);
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < total; ++q) {
      int64_t p = q / N, i = q % N;
      int64_t nrec = 0;
      const double* y0 = pts + (size_t)p * (size_t)m->n;
      if (pr->sampler == ORC_SAMPLER_REDUCED)
        flags[q] = run_walk_reduced(m, pb, pr, y0, (uint32_t)p, (uint32_t)i, &w, &S[q], &K[q]);
      else
        flags[q] = run_walk(m, pb, pr, y0, (uint32_t)p, (uint32_t)i, &w, &S[q], &K[q], NULL, 0, &nrec);
    }
    work_free(&w);
  }
  return 0;
}

/* Per-point estimator (eq. mc_estimator): the mean of the path scores by a
 * Kahan sum in walk order, and its standard error sqrt(s^2 / N) with the sample
 * variance by its definition, s^2 = sum (S - mean)^2 / (N - 1) (a second Kahan
 * pass in walk order). */
int orc_solve(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
              const double* pts, int64_t P, int64_t N, double* mean, double* stderr_,
              double* mean_steps, int64_t* n_flagged, int n_threads) {
  double* S = (double*)malloc(sizeof(double) * (size_t)(P * N));
  int64_t* K = (int64_t*)malloc(sizeof(int64_t) * (size_t)(P * N));
  int32_t* fl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P * N));
  if (orc_walk_scores(m, pb, pr, pts, P, N, S, K, fl, n_threads) != 0) {
    free(S); free(K); free(fl);
    return -1;
  }
  int64_t nf = 0;
  for (int64_t p = 0; p < P; ++p) {
    double s1 = 0.0, c1 = 0.0, ks = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double v = S[p * N + i];
      double y = v - c1, t = s1 + y; c1 = (t - s1) - y; s1 = t;
      ks += (double)K[p * N + i];
      nf += fl[p * N + i];
    }
    double mu = s1 / (double)N;
    double q = 0.0, cq = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      double dv = S[p * N + i] - mu;
      double y = dv * dv - cq, t = q + y; cq = (t - q) - y; q = t;
    }
    double var = (N > 1) ? q / (double)(N - 1) : 0.0;
    mean[p] = mu;
    stderr_[p] = sqrt(var / (double)N);
    mean_steps[p] = ks / (double)N;
  }
  if (n_flagged) *n_flagged = nf;
  free(S); free(K); free(fl);
  return 0;
}

int64_t orc_trace(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                  const double* y0, int64_t p, int64_t i, orc_trace_rec* rec, int64_t cap,
                  double* S_out, int64_t* K_out) {
  if (check_problem(m, pb) != 0) return -1;
  work_t w;
  work_alloc(&w, m->n);
  int64_t nrec = 0;
  run_walk(m, pb, pr, y0, (uint32_t)p, (uint32_t)i, &w, S_out, K_out, rec, cap, &nrec);
  work_free(&w);
  return nrec;
}
