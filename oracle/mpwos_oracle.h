/*
 * mpwos_oracle.h — FP64 CPU oracle for the modified projected Walk on Spheres
 * (MPWoS) recursion.  TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check
 * and the benchmark's CPU-baseline leg call it; the product library never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Every routine follows the paper's definitions in their plain form:
 *   - problem                 Sec. 2.1, eqs. surface_pde / surface_bc
 *   - c_{sigma,r}             Lemma 2.1 (eq. def_c_sigma_r) via the Bessel-free
 *                             series of Lemma 3.1
 *   - Green density / omega   Remark after Lemma 2.1, eq. omega_of_y, Thm 2.2
 *   - radius rule             eqs. radius_rule_unified, delta_Gamma_general,
 *                             rho_geo_curvature
 *   - projected chain         eq. projected_chain_update
 *   - path score / stopping   eqs. local_average_source, path_score_definition
 *   - estimator               eq. mc_estimator, Algorithm 1
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) at the
 * counter (block j, step k, walk i, point p), key = 64-bit seed.
 */
#ifndef MPWOS_ORACLE_H
#define MPWOS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EUCLID = 0, ORC_SPHERE = 1, ORC_TORUS = 2, ORC_EMBEDDED_SPHERE = 3, ORC_POINT_CLOUD = 4,
       ORC_REVOLUTION = 5, ORC_CURVE_SPHERE = 6 };
enum { ORC_CP_FIT = 0, ORC_CP_NEAREST = 1 };
enum { ORC_POLY = 0, ORC_TORUS_FOURIER = 1, ORC_SPHERE_QUAD = 2, ORC_REVOLUTION_QUAD = 3, ORC_CURVE_SPHERE_FUNC = 4 };

typedef struct {
  int kind, n, d;
  double R, a;            /* torus: centre-circle radius, tube radius; curve x
                             sphere (Example 3, n = 9): curve scale, sphere radius */
  const double* Q;        /* embedded sphere: n x (d+1) row-major, orthonormal */
  const double* b;        /* embedded sphere: shift, length n                  */
  const double* cloud;    /* point cloud: n_cloud x 3                          */
  int64_t n_cloud;
  int k_nn;               /* neighbours for h(y) and the local fit             */
  double c_h;             /* rho_geo = c_h h(y) (eq. rho_geo_spacing)          */
  int cp_mode;            /* ORC_CP_FIT or ORC_CP_NEAREST                      */
  /* hypersurface of revolution about the last axis (Example 2):
   * M = {x = (xh, t) : |xh| = R(t)}, R(t) = sqrt(1 - (t/k)^2) (1 - al + 2 al (t/k)^2) */
  double prof_alpha, prof_kappa;
} orc_manifold;

typedef struct {
  int kind, apply_op, n_terms;
  const double* coef;     /* n_terms                                           */
  const int* term_off;    /* poly: n_terms+1 offsets into var/pw               */
  const int* var;
  const int* pw;
  const int* modes;       /* torus: 4 ints per term (m, q, theta trig, phi trig) */
  double c0;              /* sphere quad: u = c0 + v.s + s^T A s               */
  const double* v;        /* d+1 (revolution quad: n-1)                        */
  const double* A;        /* (d+1)^2 row-major (revolution quad: the n-1 diagonal entries) */
  /* revolution quad: u = c0 + coef[0] t + coef[1] t^2 + v.xh + sum_j A_j xh_j^2, t = x_{n-1} */
  /* curve x sphere: u = sum_t T_t(q_t phi) (coef[t] + v_t.w + w^T A_t w), modes[4t] = q_t,
   * modes[4t+1] = trig (0 cos, 1 sin), v_t = v[3t..], A_t = A[9t..] row-major */
} orc_func;

enum { ORC_COMP_NONE = 0, ORC_COMP_NORMAL2 = 1, ORC_COMP_EXACT = 2 };

typedef struct {
  double sigma;
  int closed;
  const double* bnd_normal;   /* unit normal e of the half-space {e.x > h}  */
  double bnd_offset;          /* h                                          */
  orc_func f, g;
  /* compensation term (Sec. 2.3.3; m of eq. mismatch_definition):
   * ORC_COMP_NONE: m_* = 0; ORC_COMP_NORMAL2: the second-order normal
   * expansion m_* = eta m1 + eta^2 m2 / 2 from central differences of
   * R_*(s; y) at s = -h_eta, 0, h_eta, with predictor u_star (TORUS_FOURIER
   * on the torus, SPHERE_QUAD on the unit sphere of R^3; apply_op = 0);
   * ORC_COMP_EXACT: m_*(x) = R_*(eta(x); y), the mismatch of eq.
   * mismatch_definition with u_star in place of u (exact when u_star = u). */
  int comp;
  orc_func u_star;
  double h_eta;
} orc_problem;

enum { ORC_SAMPLER_FULL = 0, ORC_SAMPLER_REDUCED = 1 };

typedef struct {
  double eps, tau_w, theta, c_kappa;
  int n_v;
  int64_t max_steps;
  uint64_t seed;
  int sampler;            /* ORC_SAMPLER_FULL: n Gaussians per direction;
                             ORC_SAMPLER_REDUCED: the dimension-reduced exact
                             sampler (spheres and R^n with POLY data, embedded
                             spheres); see orc_chi2 */
} orc_params;

/* One trace record per step of one walk (tiny-case pins). */
typedef struct {
  int64_t k;
  double r, c, omega, delta_gamma, W, S, F, U0, t0, theta_norm;
  double y[3];
} orc_trace_rec;

/* primitives */
void   orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u53(uint32_t hi, uint32_t lo);
void   orc_gaussians(uint64_t seed, uint32_t j0, uint32_t k, uint32_t i, uint32_t p, int n, double* g);
double orc_em1(int n, double a);          /* I~_nu(a) - 1 (Lemma 3.1 series)      */
double orc_c_sigma_r(int n, double a);    /* 1 / I~_nu(a)                          */
double orc_green_cdf(int n, double a, double t);
double orc_green_cdf_inv(int n, double a, double U);
double orc_kt_minus_one(double mu, double x);
/* chi^2 with m degrees of freedom from the counter stream at block j0 of step k
 * (Marsaglia-Tsang gamma sampling for m >= 2, attempt a at blocks j0 + 2a and
 * j0 + 2a + 1; x^2 of one Gaussian for m = 1; 0 for m <= 0). */
double orc_chi2(uint64_t seed, uint32_t j0, uint32_t k, uint32_t i, uint32_t p, int m);
/* tracked coordinates of the reduced sampler (ascending; returns their count,
 * -1 if more than 32 or the data are not POLY) */
int    orc_tracked_set(const orc_manifold* m, const orc_problem* pb, int* T);
void   orc_cp(const orc_manifold* m, const double* x, double* out);
double orc_delta_gamma(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                       const double* y, double* y_gamma);
double orc_func_eval(const orc_manifold* m, const orc_func* f, double sigma, const double* x);
/* compensation: eta(x) the signed normal distance of x, R_*(s; y) at the
 * closest point y, and m_*(x) (f evaluated at y = cp(x) inside) */
double orc_normal_coord(const orc_manifold* m, const double* x);
double orc_comp_R(const orc_manifold* m, const orc_problem* pb, const double* y, double s);
double orc_comp_m(const orc_manifold* m, const orc_problem* pb, const double* x);
/* hypersurface of revolution: the profile R(t), R'(t), R''(t); the curvature
 * indicator (largest absolute principal curvature) at a point of M */
void   orc_profile(const orc_manifold* m, double t, double* R, double* R1, double* R2);
double orc_kappa_at(const orc_manifold* m, const double* y);
/* curve x sphere: phi of the nearest point of the Fourier curve to the first six
 * coordinates of x (Newton's method from the angle of (x_1, x_2)) */
double orc_curve_cp_phi(const orc_manifold* m, const double* x);
/* point cloud: k nearest (by distance^2, then index), mean distance h(x) */
double orc_cloud_knn(const orc_manifold* m, const double* x, int64_t* idx, double* d2);

/* the walk: per-walk score S, stopping index K, flag (1 = hit max_steps) */
int orc_walk_scores(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                    const double* pts, int64_t P, int64_t N, double* S, int64_t* K,
                    int32_t* flags, int n_threads);
/* per-point mean / standard error / mean steps (Kahan sums in walk order) */
int orc_solve(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
              const double* pts, int64_t P, int64_t N, double* mean, double* stderr_,
              double* mean_steps, int64_t* n_flagged, int n_threads);
/* one walk with a per-step trace; returns number of records written */
int64_t orc_trace(const orc_manifold* m, const orc_problem* pb, const orc_params* pr,
                  const double* y0, int64_t p, int64_t i, orc_trace_rec* rec, int64_t cap,
                  double* S_out, int64_t* K_out);

#ifdef __cplusplus
}
#endif
#endif
