/*
 * mpwos.h — C ABI of the B300 MPWoS library (libmpwos.so).
 *
 * The library estimates the solution of the screened Poisson equation
 *     -Delta_M u + sigma u = f  on Omega in M,   u = g  on Gamma = boundary of Omega
 * (Sec. 2.1, eqs. surface_pde / surface_bc) at query points y_0 on an embedded
 * manifold M in R^n by the modified projected Walk on Spheres recursion
 * (Algorithm 1; path score eq. path_score_definition; estimator eq.
 * mc_estimator).  Every walk step runs in CUDA kernels on one GPU.
 *
 * Conventions for every entry point:
 *   - the return value is a status code below; the message of the last
 *     failure is kept per context (mpwos_last_error);
 *   - problem data (f, g coefficients, Q, b, the boundary normal) are HOST
 *     pointers, read during the call and copied; the caller keeps ownership;
 *   - query points and result arrays may be host or device pointers; the
 *     library inspects them with cudaPointerGetAttributes.  Host arrays are
 *     copied in/out inside the call; device arrays are read/written in place;
 *   - a call returns after its results are written (synchronous) unless it
 *     is one of the asynchronous request calls (mpwos_submit ...);
 *   - query points must lie on M (the walk starts at y_0 as given).
 */
#ifndef MPWOS_H
#define MPWOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MPWOS_OK 0
#define MPWOS_EINVAL 1      /* invalid argument (message says which)               */
#define MPWOS_ENOMEM 2      /* device allocation failed                            */
#define MPWOS_ECUDA 3       /* a CUDA call failed (message has the CUDA error)     */
#define MPWOS_ETIMEDOUT 4   /* a bounded wait ran out                              */
#define MPWOS_ECANCELED 5   /* request cancelled                                   */
#define MPWOS_EMAXSTEPS 6   /* results written, but some walks reached max_steps   */
#define MPWOS_ENOTFOUND 7   /* unknown request id                                  */
#define MPWOS_EBUSY 8       /* admission refused: no slot or memory free now       */

/* ---- manifold kinds (Sec. 2.1: parametrized manifolds with closed-form cp) */
#define MPWOS_EUCLID 0            /* M = R^n, cp = identity                      */
#define MPWOS_SPHERE 1            /* unit sphere S^{n-1} in R^n, cp(x) = x/|x|    */
#define MPWOS_TORUS 2             /* torus in R^3, centre radius R, tube radius a */
#define MPWOS_EMBEDDED_SPHERE 3   /* Q S^d + b, Q (n x (d+1)) orthonormal columns */
#define MPWOS_POINT_CLOUD 4       /* closed surface in R^3 given by points (Sec. 2.1 (iii)) */
#define MPWOS_REVOLUTION 5        /* implicit hypersurface of revolution about the last axis,
                                     {(xh, t) : |xh| = R(t)}, Example 2's dumbbell profile
                                     R(t) = sqrt(1 - (t/k)^2) (1 - al + 2 al (t/k)^2);
                                     cp by Newton's method in the profile parameter         */
#define MPWOS_CURVE_SPHERE 6      /* Example 3: C(S^1) x S^2(a) in R^9 (n = 9, d = 3),
                                     C(phi) = R (cos phi, sin phi, cos 2phi/2, sin 2phi/2,
                                     cos 3phi/3, sin 3phi/3); R, a from the desc's R, a   */

/* ---- closest point on a point cloud ------------------------------------ */
#define MPWOS_CLOUD_CP_FIT 0      /* k nearest, PCA plane, quadratic height fit, projection */
#define MPWOS_CLOUD_CP_NEAREST 1  /* nearest cloud point                                    */

/* ---- function kinds for f and g (a C ABI cannot pass device code) ------- */
#define MPWOS_FUNC_POLY 0          /* sum_t coef_t prod_j x[var]^pw (ambient coords)  */
#define MPWOS_FUNC_TORUS_FOURIER 1 /* sum_t coef_t T(m theta) P(q phi); T,P in {cos,sin} */
#define MPWOS_FUNC_SPHERE_QUAD 2   /* c0 + v.s + s^T A s, s = intrinsic unit vector   */
#define MPWOS_FUNC_REVOLUTION_QUAD 3 /* c0 + coef[0] t + coef[1] t^2 + v.xh + sum_j A_j xh_j^2 on
                                        MPWOS_REVOLUTION (v, A: n - 1 entries, A diagonal) */
#define MPWOS_FUNC_CURVE_SPHERE 4  /* sum_t T_t(q_t phi) (coef[t] + v_t.w + w^T A_t w) on
                                      MPWOS_CURVE_SPHERE, w the sphere factor's unit vector;
                                      modes: 4 ints per term (q, trig 0 cos / 1 sin, 0, 0);
                                      v: 3, A: 9 (row-major) entries per term           */

/* ---- compensation term m_* (Sec. 2.3.3; m of eq. mismatch_definition) ---- */
#define MPWOS_COMP_NONE 0      /* m_* = 0: the baseline method                              */
#define MPWOS_COMP_NORMAL2 1   /* m_*(x) = eta m1(y) + eta^2 m2(y)/2, y = cp(x), eta the signed
                                  normal distance of x; m1, m2 central differences of
                                  R_*(s; y) = -Delta(E u_*)(y + s n(y)) + sigma u_*(y) - f(y)
                                  at s = -h_eta, 0, h_eta (E u_* = u_* o cp)                 */
#define MPWOS_COMP_EXACT 2     /* m_*(x) = R_*(eta; y): the mismatch itself with u_* for u
                                  (exact when u_* is the solution)                            */

/* ---- precision of the walk --------------------------------------------- */
#define MPWOS_FP64 0   /* FP64 walk; per-walk identical draws to the CPU oracle         */
#define MPWOS_FP32 1   /* FP32 positions/projection/sampling, FP64 weights and sums     */

/* ---- the projection Q^T g of the FP32 embedded-sphere walk --------------- */
#define MPWOS_PROJ_AUTO 0     /* tensor cores for n >= 128, CUDA cores below               */
#define MPWOS_PROJ_TENSOR 1   /* tcgen05 split-BF16 product (hi hi + hi lo + lo hi), FP32
                                 accumulator: ~2^-17 relative per component; FP32 precision
                                 and EMBEDDED_SPHERE only (MPWOS_EINVAL otherwise)           */
#define MPWOS_PROJ_CUDA 2     /* FP32 dot products on the CUDA cores                       */

/* ---- direction sampler (not in the paper; same law of the walk) --------- */
#define MPWOS_SAMPLER_FULL 0     /* n Gaussians per direction (the paper's form)               */
#define MPWOS_SAMPLER_REDUCED 1  /* dimension-reduced exact sampler: the walk reads a direction
                                    only through the coordinates T that f, g and the boundary
                                    normal use (the intrinsic Q^T g on an embedded sphere),
                                    on a sphere the component along Y's part outside T, and
                                    |g|^2; those are drawn directly (normals and a chi^2 of the
                                    remaining dimensions).  SPHERE and EUCLID with n > 3 and
                                    POLY data (|T| <= 32), EMBEDDED_SPHERE; its own Philox
                                    stream layout (the CPU oracle has the same mode).        */

typedef struct mpwos_ctx mpwos_ctx;

/* Manifold M (Sec. 2.1), described for mpwos_manifold_create.  Q, b are host
 * arrays (embedded sphere only), Q row-major n x (d+1) with orthonormal
 * columns.  Point cloud (n = 3, d = 2, closed problems): n_cloud x 3 host
 * array; rho_geo(y) = c_h h(y), h(y) the mean distance from y to its k_nn
 * nearest cloud points (eq. rho_geo_spacing); cp by cp_mode. */
typedef struct {
  int kind;
  int n;            /* ambient dimension                                  */
  int d;            /* manifold dimension                                 */
  double R, a;      /* torus: centre-circle radius, tube radius           */
  const double* Q;  /* embedded sphere                                    */
  const double* b;  /* embedded sphere shift, length n                    */
  const double* cloud;  /* point cloud, n_cloud x 3                       */
  int64_t n_cloud;
  int k_nn;         /* 1 .. 32                                            */
  double c_h;
  int cp_mode;      /* MPWOS_CLOUD_CP_FIT or MPWOS_CLOUD_CP_NEAREST        */
  double prof_alpha, prof_kappa;   /* REVOLUTION: al in (0, 1/2), k > 0   */
} mpwos_manifold_desc;

/* A manifold handle (opaque): owns copies of a description's arrays and the
 * device data the walks read (the embedded sphere's Q^T in FP64 and FP32, b and
 * the tensor-core operand image; the point cloud's search grid; the
 * revolution's curvature range), built once on the context's device. */
typedef struct mpwos_manifold mpwos_manifold;

/* A function on M given as a small closed family of device-evaluable forms.
 * apply_op != 0 (torus Fourier, sphere quad): evaluate (-Delta_M + sigma) of
 * the series in closed form instead of the series itself — the source of a
 * manufactured solution. */
typedef struct {
  int kind;
  int apply_op;
  int n_terms;
  const double* coef;     /* n_terms                                        */
  const int* term_off;    /* POLY: n_terms + 1 offsets into var / pw        */
  const int* var;         /* POLY: coordinate index (0-based)               */
  const int* pw;          /* POLY: power                                    */
  const int* modes;       /* TORUS_FOURIER: 4 ints per term (m, q, Ttrig, Ptrig), trig 0 = cos, 1 = sin */
  double c0;              /* SPHERE_QUAD                                    */
  const double* v;        /* SPHERE_QUAD: d + 1                             */
  const double* A;        /* SPHERE_QUAD: (d + 1)^2 row-major               */
} mpwos_func;

/* The screened Poisson problem (eqs. surface_pde, surface_bc).  Boundary:
 * Omega = M intersected with the half-space {x : e.x > h} (EUCLID, SPHERE;
 * TORUS with a plane through its axis, e_3 = 0 and h = 0, as in Example 1),
 * or closed = 1 (Omega = M).
 * Compensation (comp != MPWOS_COMP_NONE): the step's source becomes
 * f(cp(Z)) + m_*(Z) with the predictor u_star, a TORUS_FOURIER series on the
 * torus (at most 64 terms) or a SPHERE_QUAD on the sphere of R^3, apply_op = 0;
 * walks in R^3 (TORUS, SPHERE with n = 3) with the full sampler only
 * (MPWOS_EINVAL otherwise).  h_eta: the normal difference step (0: 1e-2). */
typedef struct {
  double sigma;               /* screening, > 0                         */
  int closed;
  const double* bnd_normal;   /* unit e, length n (host)                */
  double bnd_offset;          /* h                                      */
  mpwos_func f, g;
  int comp;                   /* MPWOS_COMP_*                           */
  mpwos_func u_star;          /* predictor u_* (comp != NONE)           */
  double h_eta;
} mpwos_problem;

/* Walk parameters (Algorithm 1; radius rule eq. radius_rule_unified). */
typedef struct {
  double eps;        /* boundary layer width epsilon (eq. boundary_layer)      */
  double tau_w;      /* closed-manifold weight cut-off tau_W                   */
  double theta;      /* radius safety factor, 0 < theta < 1                    */
  double c_kappa;    /* rho_geo = c_kappa / (1 + kappa) (eq. rho_geo_curvature) */
  int n_v;           /* interior samples per step N_V (eq. local_average_source) */
  int64_t max_steps; /* per-walk cap; walks reaching it are flagged (EMAXSTEPS) */
  uint64_t seed;     /* Philox key                                              */
  int precision;     /* MPWOS_FP64 or MPWOS_FP32                                */
  int projection;    /* MPWOS_PROJ_*: embedded sphere in FP32 only; ignored elsewhere
                        except that MPWOS_PROJ_TENSOR is rejected there             */
  int sampler;       /* MPWOS_SAMPLER_FULL or MPWOS_SAMPLER_REDUCED               */
} mpwos_params;

/* Fill a params struct with the defaults: eps 1e-3, tau_w 1e-8, theta 0.95,
 * c_kappa 1.2, n_v 1, max_steps 1e7, seed 0, FP64, MPWOS_PROJ_AUTO,
 * MPWOS_SAMPLER_FULL. */
void mpwos_params_default(mpwos_params* p);

/* Create a context on CUDA device `device` (owns device state, tables, a
 * stream).  stream: a cudaStream_t the synchronous calls run on (borrowed, not
 * destroyed with the context), or NULL for the context's own stream.  Returns
 * MPWOS_EINVAL for a bad device, MPWOS_ECUDA otherwise. */
int mpwos_create(int device, void* stream, mpwos_ctx** out);

/* Create a manifold handle (Sec. 2.1: the manifold and its closest-point data)
 * on the context's device from a description; the description's arrays are
 * copied and may be freed afterwards.  The handle serves every later call on
 * contexts of the same device; it must outlive the requests that use it.
 * Returns MPWOS_EINVAL for an invalid description (message in
 * mpwos_last_error), MPWOS_ENOMEM / MPWOS_ECUDA otherwise. */
int mpwos_manifold_create(mpwos_ctx* ctx, const mpwos_manifold_desc* desc, mpwos_manifold** out);

/* Free a manifold handle and its device data.  NULL is a no-op. */
void mpwos_manifold_destroy(mpwos_manifold* m);

/* Destroy a context and free its device memory.  NULL is a no-op. */
void mpwos_destroy(mpwos_ctx* ctx);

/* Message of the last failed call on this context ("" if none). */
const char* mpwos_last_error(const mpwos_ctx* ctx);

/* Use `stream` (a cudaStream_t, borrowed, may be NULL for the context's own
 * stream) for subsequent synchronous calls. */
int mpwos_set_stream(mpwos_ctx* ctx, void* stream);

/* Estimate u at P query points (pts: P x n row-major FP64, host or device)
 * with N walks each (Algorithm 1, estimator eq. mc_estimator).  Outputs (P
 * each, host or device, caller-owned): the mean of the path scores, its
 * standard error, the mean stopping index K.  Returns MPWOS_EMAXSTEPS (with
 * results written) if any walk reached max_steps. */
int mpwos_solve(mpwos_ctx* ctx, const mpwos_manifold* m, const mpwos_problem* prob,
                const mpwos_params* prm, const double* pts, int64_t P, int64_t N,
                double* mean, double* stderr_, double* mean_steps);

/* Per-walk path scores S^i (eq. path_score_definition), stopping indices K^i
 * and max-steps flags, P x N row-major (walk i of point p at p*N + i); host
 * or device.  Walk (p, i) draws its random numbers from Philox4x32-10 at
 * counter (block, step, i, p), so each value depends on (seed, p, i) only. */
int mpwos_walk_scores(mpwos_ctx* ctx, const mpwos_manifold* m, const mpwos_problem* prob,
                      const mpwos_params* prm, const double* pts, int64_t P, int64_t N,
                      double* S, int32_t* K, int32_t* flags);

/* One request split by walk range (the estimator of eq. mc_estimator summed
 * over independent paths, Sec. 2.3 and Algorithm 1; one range per GPU, then a
 * merge on the host).  The walks of a point form blocks of 1024 walk indices;
 * a block's statistic (walk count, mean of S, sum of squared deviations from
 * that mean, sum of K, walks flagged at max_steps) depends only on its own
 * walks, in one fixed summation order, and blocks merge in order with the
 * pairwise update of Chan, Golub and LeVeque.  mpwos_solve runs exactly this
 * order, so merging the ranges [0, i1), [i1, i2), ... of a request gives the
 * bits mpwos_solve gives for the whole request.
 *
 * mpwos_solve_partial: walks i0 <= i < i1 of each of the P points of a request
 * of N walks per point (i0 and i1 multiples of 1024, or i1 = N; walk (p, i)
 * draws the same numbers as in mpwos_solve).  part (host or device,
 * caller-owned): P x nblk x 5 doubles, nblk = ceil((i1 - i0) / 1024), record
 * (p, b) = (count, mean, M2, sum of K, flagged) of block b of the range.
 * MPWOS_EINVAL for a misaligned range; max-steps walks are only counted in the
 * records. */
int mpwos_solve_partial(mpwos_ctx* ctx, const mpwos_manifold* m, const mpwos_problem* prob,
                        const mpwos_params* prm, const double* pts, int64_t P, int64_t N, int64_t i0,
                        int64_t i1, double* part);

/* The block records of per-walk outputs (host arrays, P x N row-major as from
 * mpwos_walk_scores; walk offsets 0..N-1 of a range) computed on the host in
 * the device's summation order: part receives P x ceil(N / 1024) x 5 doubles.
 * Needs no GPU and no context. */
int mpwos_block_partials_host(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                              double* part);

/* The least-squares step of the coarse predictor u_* of the compensation term
 * (Sec. 2.3.3): given estimates u at P points of a torus of centre-circle radius
 * R (pts: P x 3 host), the torus Fourier series sum_t c_t T_t(m theta) P_t(q phi)
 * with T, P in {cos, sin} (no sin of a zero multiple), m <= max_m, q <= max_q,
 * nearest to u in least squares (Householder QR, FP64); theta = atan2(x_3,
 * |(x_1, x_2)| - R), phi = atan2(x_2, x_1).  The estimates come from a
 * baseline solve (comp = NONE) at points of Omega.  Outputs (host): coef and
 * modes (4 per term: m, q, theta trig, phi trig; trig 0 = cos, 1 = sin), in the
 * TORUS_FOURIER layout of u_star, and their number n_terms (at most 64).
 * Returns MPWOS_EINVAL for a basis of more than 64 terms, P smaller than the
 * basis, or a rank-deficient fit.  Needs no GPU and no context. */
int mpwos_fit_torus_series(const double* pts, const double* u, int64_t P, double R, int max_m, int max_q,
                           double* coef, int* modes, int* n_terms);

/* Merge block records on the host: parts[r] (host, P x nblk[r] x 5 doubles)
 * for consecutive walk ranges r = 0 .. nparts-1 of one request, merged per
 * point in range order and block order.  Outputs (P each, host): the mean of
 * the path scores, its standard error sqrt(s^2 / n), s^2 = M2 / (n - 1), and
 * the mean stopping index; n_flagged (nullable) receives the flagged walks.
 * Returns MPWOS_EMAXSTEPS (outputs written) if any walk was flagged, and
 * MPWOS_EINVAL for null or negative arguments.  Needs no GPU and no context. */
int mpwos_merge_partials(const double* const* parts, const int64_t* nblk, int nparts, int64_t P, double* mean,
                         double* stderr_, double* mean_steps, int64_t* n_flagged);

/* Allocation-free variant of mpwos_solve (the paper has no counterpart: this
 * is a deployment convenience).  For callers that cannot call cudaMalloc — an
 * application whose device memory is owned by another allocator, or a
 * latency-critical loop where an allocation (which can synchronize the
 * device) is not allowed.  It runs the same walk and reduction kernels as
 * mpwos_solve, on the same draws, with all scratch (per-walk scores, stopping
 * indices, flags, radius tables, boundary normal, counter) in one fixed 32 MiB
 * device array inside the library, which each GPU holds from its first use
 * until the process exits.
 *   - pts (P x n) and the three outputs must be DEVICE pointers (EINVAL
 *     otherwise); problem data are host pointers as for mpwos_solve;
 *   - P * N must not exceed mpwos_noalloc_max_walks() (EINVAL with the limit
 *     in the message); EMBEDDED_SPHERE, POINT_CLOUD, REVOLUTION and
 *     CURVE_SPHERE manifolds, the reduced sampler, compensation and problems
 *     with two SPHERE_QUAD functions (at most one of f, g) are not supported
 *     (EINVAL); pts and the outputs must be on the context's device;
 *   - the first call on a device looks up the array's device address; make
 *     that first call before any stream capture;
 *   - every call shares the array: calls that overlap on the GPU (other
 *     streams, other contexts on the same device) race and must be serialized
 *     by the caller.  Each call clears and rebuilds what it needs.
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
int mpwos_solve_noalloc(mpwos_ctx* ctx, const mpwos_manifold* m, const mpwos_problem* prob,
                        const mpwos_params* prm, const double* pts, int64_t P, int64_t N,
                        double* mean, double* stderr_, double* mean_steps);

/* Largest P * N accepted by mpwos_solve_noalloc. */
int64_t mpwos_noalloc_max_walks(void);

/* ---- request serving (continuous batching) ------------------------------
 * A request is one solve (same inputs as mpwos_solve; query points on the
 * HOST, copied at submit) with a walk budget per point and an optional target
 * standard error: walks per point start at min(256, budget) and double for the
 * points whose standard error is still above the target, up to the budget
 * (target 0: exactly `walk_budget` walks, as mpwos_solve).  A request (not on
 * a point cloud) whose P x budget walks fill at most a quarter of one resident
 * wave of its walk kernel runs the whole budget in its first round (its
 * latency is its walks' length, which more rounds would only repeat).  Requests are
 * admitted while a stream slot and serving memory are free (16 slots and a
 * quarter of the free device memory by default), run concurrently on their
 * own streams, and are advanced by a scheduler thread of the context.  A
 * round's walks go out in chunks of about 10 ms of GPU time each (the walk
 * cost measured on the request's previous chunks, at its share of the grid;
 * at least one resident wave of walkers, at most chunk_walks walks), two in
 * flight per request, so that a newly admitted request waits at most about one
 * chunk for the SMs.  A walk's draws depend only on (seed, point, walk index), so a
 * request's results do not depend on the other requests in flight; with
 * target 0 they equal mpwos_solve's bit for bit.  Point clouds: the search
 * grid is built at submit. */

/* Serving limits: at most max_active requests in flight (<= 64; change only
 * while idle), mem_bytes of device memory for their scratch, chunk_walks walks
 * per launch.  Values <= 0 keep the current setting. */
int mpwos_serve_config(mpwos_ctx* ctx, int max_active, size_t mem_bytes, int64_t chunk_walks);

/* Queue a request; *request_id identifies it.  Fails with EINVAL on invalid
 * inputs (as mpwos_solve) or device query points. */
int mpwos_submit(mpwos_ctx* ctx, const mpwos_manifold* m, const mpwos_problem* prob,
                 const mpwos_params* prm, const double* pts, int64_t P, int64_t walk_budget,
                 double target_stderr, uint64_t* request_id);

/* *state: 0 queued, 1 running, 2 finished, 3 failed, 4 canceled. */
int mpwos_poll(mpwos_ctx* ctx, uint64_t request_id, int* state);

/* Block until the request leaves the queue/running states or timeout_s
 * seconds pass (MPWOS_ETIMEDOUT; timeout_s < 0 waits without limit). */
int mpwos_wait(mpwos_ctx* ctx, uint64_t request_id, double timeout_s);

/* Cancel a queued or running request (a running one stops after its current
 * round; mpwos_fetch then returns MPWOS_ECANCELED). */
int mpwos_cancel(mpwos_ctx* ctx, uint64_t request_id);

/* Copy a finished request's per-point mean, standard error, mean steps and
 * walks used (host arrays of P; any may be NULL) and its latency (submit to
 * completion, seconds), then release it.  Returns the request's status
 * (MPWOS_OK, MPWOS_EMAXSTEPS, MPWOS_ECANCELED or the failure code);
 * MPWOS_EBUSY if it has not finished. */
int mpwos_fetch(mpwos_ctx* ctx, uint64_t request_id, double* mean, double* stderr_,
                double* mean_steps, int64_t* walks, double* latency_s);

/* ---- primitives exposed for verification ------------------------------ */

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[4q..4q+3] =
 * Philox(ctr[4q..4q+3], key); count blocks; host arrays. */
int mpwos_philox(mpwos_ctx* ctx, const uint32_t* ctr, uint32_t key0, uint32_t key1,
                 uint32_t* out, int64_t count);

/* Radius fraction t = R/r of the interior sample Z ~ rho(y, .) (eq.
 * Z_sampling_density) for uniform U, computed by the device sampler at
 * precision `precision` for ambient dimension n and a = sqrt(sigma) r, through
 * the same tables the walk uses (built for a in [0, a_max]); host arrays. */
int mpwos_green_radius(mpwos_ctx* ctx, int n, double a_max, const double* a, const double* U,
                       double* t, int64_t count, int precision);

/* c_{sigma,r} (Lemma 2.1 via the Lemma 3.1 series) for ambient dimension n at
 * a = sqrt(sigma) r, evaluated by the device code; host arrays. */
int mpwos_c_sigma_r(mpwos_ctx* ctx, int n, const double* a, double* c, int64_t count);

/* The embedded-sphere projection Q^T g (eq. projected_chain_update: the
 * closest point of an embedded sphere needs Q^T (x - b)) on the tensor cores,
 * exactly as the FP32 walk forms it: out[r][j] = sum_i G[r][i] Q[i][j] for the
 * rows of G (rows x n, FP32, row-major), Q n x D row-major (host FP64, rounded
 * to BF16 hi + lo), G rounded to BF16 hi + lo, three BF16 products accumulated
 * in FP32; gg[r] = |G_r|^2 in FP32.  out is rows x D.  1 <= n <= 1024,
 * 1 <= D <= 31.  Host arrays.  MPWOS_ETIMEDOUT if a bounded wait ran out. */
int mpwos_tc_project(mpwos_ctx* ctx, const double* Q, int n, int D, const float* G, int64_t rows,
                     float* out, float* gg);

/* ---- k nearest cloud points --------------------------------------------- */
#define MPWOS_KNN_GRID 0       /* the walk's search: expanding cubes of grid cells, a thread per query */
#define MPWOS_KNN_GRID_WARP 1  /* its warp-cooperative form (FP32 only; the FP32 walk's at k >= 12)   */
#define MPWOS_KNN_SCAN 2       /* every cloud point, staged through shared memory (comparison)         */

/* The k = m->k_nn nearest points of the point cloud m (MPWOS_POINT_CLOUD;
 * Sec. 2.1 representation (iii)) to each of nq query points x (nq x 3,
 * row-major), as the walk's closest-point step finds them (the first step of
 * its cp; h(x), eq. rho_geo_spacing, is their mean distance).  Order: by
 * distance^2, ties by cloud index.  Distances in `precision` (MPWOS_FP32: x
 * and the cloud rounded to FP32 as the FP32 walk holds them; MPWOS_FP64).  All
 * three methods give identical results at one precision.  Outputs
 * (caller-owned): idx (nq x k cloud indices), d2 (nq x k, widened to FP64), h
 * (nq).  x, idx, d2 and h may each be host or device memory.  MPWOS_EINVAL:
 * m not a point cloud, k_nn outside [1, 32], n_cloud outside [k_nn, 2^31),
 * nq < 0, a null array with nq > 0, an unknown method or precision, or
 * MPWOS_KNN_GRID_WARP with MPWOS_FP64. */
int mpwos_cloud_knn(mpwos_ctx* ctx, const mpwos_manifold* m, const double* x, int64_t nq,
                    int precision, int method, int32_t* idx, double* d2, double* h);

/* Number of the library's own kernel launches so far on this context. */
int64_t mpwos_launch_count(const mpwos_ctx* ctx);

/* Launch-shape autotuner (runtime only; the method does not depend on it).
 * enable != 0 turns it on for this context, 0 off (the default).  While on,
 * the first mpwos_solve or mpwos_walk_scores for a walk kernel instance and
 * ambient dimension n with enough walks (at least 2 (candidates + 1) full
 * waves) splits its walks into candidates + 1 equal parts, runs each of the
 * first parts with one candidate block size (32, 64, 128, 256 threads, up to
 * the kernel's limit; each launch fills every SM), times each part with CUDA
 * events, divides by the part's walk-steps, keeps the fastest and runs the last
 * part with it; one host synchronisation.  Later calls for that instance, request serving included,
 * launch the pick.  Smaller calls launch the default shape and record nothing.
 * Results never depend on the shape: each walk's random numbers are a function
 * of (point, walk, step) alone and per-point sums run in a fixed order.  The
 * tensor-core walk keeps its fixed shape; mpwos_solve_noalloc always launches
 * the default shape.  Picks persist until the context is destroyed.
 * MPWOS_EINVAL for a null context. */
int mpwos_set_autotune(mpwos_ctx* ctx, int enable);

/* One autotuned kernel: `kernel` its (mangled) name, owned by the CUDA runtime
 * (NULL if unavailable); n the ambient dimension; block the pick; per
 * candidate block size, the measured GPU time per walk-step in ns. */
typedef struct {
  const char* kernel;
  int n;
  int block;
  int n_candidates;
  int candidates[4];
  double ns_per_walk_step[4];
} mpwos_tune_entry;

/* Copies up to `capacity` picks into `entries` (caller-owned) and their total
 * number into *count.  MPWOS_EINVAL for a null context or count, a negative
 * capacity, or capacity > 0 with null entries. */
int mpwos_autotune_entries(mpwos_ctx* ctx, mpwos_tune_entry* entries, int capacity, int* count);

#ifdef __cplusplus
}
#endif
#endif
