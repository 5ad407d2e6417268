// mpwos_abi.cu — host side of the C ABI declared in include/mpwos.h: argument
// validation, device copies of the problem data, radius-table cache, launch
// configuration and the per-walk / per-point output paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mpwos.h"
#include "launch.h"
#include "estimator.cuh"
#include "revolution.cuh"

using namespace mpwos;

namespace {

constexpr int kTableNS = 1025;   // s-nodes per radius-table row
constexpr int kTableNA = 65;     // rows over z = a^2/4 for variable-radius problems

struct Table {
  double* tab64 = nullptr;
  float4* tabc = nullptr;
  int NA = 0, NS = 0;
  double z_max = 0.0;
};

struct CloudGrid {
  double* pts64 = nullptr;
  float* pts32 = nullptr;
  float4* pts4 = nullptr;
  int* orig = nullptr;
  int* start = nullptr;
  double origin[3] = {0, 0, 0};
  double cell = 0.0;
  int dims[3] = {0, 0, 0};
  double h_max = 0.0;
};

}  // namespace

// A manifold handle: owns copies of the description's arrays and the device
// data the walks read, built once at creation on the context's device.
struct mpwos_manifold {
  int device = 0;
  mpwos_manifold_desc desc{};     // arrays point into the vectors below
  std::vector<double> Q, b, cloud;
  double* qt = nullptr;           // EMBEDDED_SPHERE: Q^T (D x npad, npad = n rounded up to 4), FP64
  float* qtf = nullptr;           //   and FP32
  double* bd = nullptr;           //   the shift b
  uint16_t* tc_img = nullptr;     //   the tensor-core walk's operand image of Q^T
  CloudGrid grid;                 // POINT_CLOUD: the search grid
  bool has_grid = false;
  double rev_kmin = 0.0;          // REVOLUTION: smallest curvature indicator over the profile
};

struct ServeEngine;
void serve_shutdown(mpwos_ctx* ctx);

// One autotuned walk kernel instance: the candidate block sizes, the GPU time
// per walk-step each measured, and the pick.
struct TuneEntry {
  int block = 0;
  std::vector<int> cand;
  std::vector<double> ns_per_step;
};

struct mpwos_ctx {
  std::recursive_mutex mu;           // public calls and the request scheduler
  ServeEngine* serve = nullptr;
  int device = 0;
  int sm_count = 0;
  cudaStream_t own = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  long long launches = 0;
  std::map<std::tuple<int, int, double>, Table> tables;  // (n, NA, z_max or a) -> table
  bool autotune = false;
  std::map<std::pair<const void*, int>, TuneEntry> tune;  // (walk kernel, n) -> measured launch shapes
};

namespace {

int fail(mpwos_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return code;
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(ctx, MPWOS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// A device (or managed) pointer of the given device.
bool is_device_ptr_on(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

double kappa_of(const mpwos_manifold_desc* m) {
  if (m->kind == MPWOS_EUCLID) return 0.0;
  if (m->kind == MPWOS_TORUS) return 1.0 / m->a;
  if (m->kind == MPWOS_CURVE_SPHERE) return std::max(std::sqrt(14.0) / (3.0 * m->R), 1.0 / m->a);
  return 1.0;
}

// Stream-ordered device buffers released at the end of a call (or of a
// served request), on the stream they were allocated on.
struct Scratch {
  mpwos_ctx* ctx;
  cudaStream_t stream;
  std::vector<void*> bufs;
  explicit Scratch(mpwos_ctx* c) : ctx(c), stream(c->stream) {}
  Scratch(mpwos_ctx* c, cudaStream_t s) : ctx(c), stream(s) {}
  ~Scratch() {
    for (void* b : bufs) cudaFreeAsync(b, stream);
  }
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    if (cudaMallocAsync(&p, count * sizeof(T), stream) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return static_cast<T*>(p);
  }
  template <typename T>
  T* upload(const T* host, size_t count) {
    T* d = alloc<T>(count);
    if (d && count) cudaMemcpyAsync(d, host, count * sizeof(T), cudaMemcpyHostToDevice, stream);
    return d;
  }
};

// Coordinates the reduced sampler tracks on SPHERE / EUCLID: the variables of f
// (and g) and the support of the boundary normal, ascending; -1 if more than
// kMaxQuadDim or the data are not POLY.
int tracked_set(const mpwos_manifold_desc* m, const mpwos_problem* pr, int* T) {
  if (pr->f.kind != MPWOS_FUNC_POLY || (!pr->closed && pr->g.kind != MPWOS_FUNC_POLY)) return -1;
  std::vector<char> used(static_cast<size_t>(m->n), 0);
  for (const mpwos_func* f : {&pr->f, &pr->g}) {
    if (f == &pr->g && pr->closed) continue;
    const int nf = f->n_terms ? f->term_off[f->n_terms] : 0;
    for (int q = 0; q < nf; ++q) used[f->var[q]] = 1;
  }
  if (!pr->closed)
    for (int q = 0; q < m->n; ++q)
      if (pr->bnd_normal[q] != 0.0) used[q] = 1;
  int nT = 0;
  for (int q = 0; q < m->n; ++q)
    if (used[q]) {
      if (nT == kMaxQuadDim) return -1;
      T[nT++] = q;
    }
  return nT;
}

// The checks of a manifold description alone (at handle creation).
int validate_manifold(mpwos_ctx* ctx, const mpwos_manifold_desc* m) {
  if (m->n < 3 || m->n > 1024) return fail(ctx, MPWOS_EINVAL, "ambient dimension must lie in [3, 1024] (got %d)", m->n);
  switch (m->kind) {
    case MPWOS_EUCLID:
      if (m->d != m->n) return fail(ctx, MPWOS_EINVAL, "EUCLID needs d == n");
      return MPWOS_OK;
    case MPWOS_SPHERE:
      if (m->d != m->n - 1) return fail(ctx, MPWOS_EINVAL, "SPHERE needs d == n - 1");
      return MPWOS_OK;
    case MPWOS_TORUS:
      if (m->n != 3 || m->d != 2) return fail(ctx, MPWOS_EINVAL, "TORUS lives in R^3 (n = 3, d = 2)");
      if (!(m->R > m->a && m->a > 0.0)) return fail(ctx, MPWOS_EINVAL, "TORUS needs R > a > 0");
      return MPWOS_OK;
    case MPWOS_EMBEDDED_SPHERE:
      if (m->n <= 3) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs n > 3");
      if (m->d < 1 || m->d + 1 > kMaxQuadDim - 1 || m->d + 1 > m->n) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs 1 <= d <= min(n - 1, 30)");
      if (!m->Q || !m->b) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs Q and b");
      return MPWOS_OK;
    case MPWOS_REVOLUTION:
      if (m->n < 4 || m->d != m->n - 1) return fail(ctx, MPWOS_EINVAL, "REVOLUTION needs n >= 4 and d == n - 1");
      if (!(m->prof_alpha > 0.0 && m->prof_alpha < 0.5 && m->prof_kappa > 0.0))
        return fail(ctx, MPWOS_EINVAL, "REVOLUTION needs 0 < prof_alpha < 1/2 and prof_kappa > 0");
      return MPWOS_OK;
    case MPWOS_CURVE_SPHERE:
      if (m->n != 9 || m->d != 3) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE lives in R^9 (n = 9, d = 3)");
      if (!(m->R > 0.0 && m->a > 0.0)) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE needs R > 0 and a > 0");
      return MPWOS_OK;
    case MPWOS_POINT_CLOUD:
      if (m->n != 3 || m->d != 2) return fail(ctx, MPWOS_EINVAL, "POINT_CLOUD lives in R^3 (n = 3, d = 2)");
      if (!m->cloud) return fail(ctx, MPWOS_EINVAL, "POINT_CLOUD needs cloud");
      if (m->k_nn < 1 || m->k_nn > 32) return fail(ctx, MPWOS_EINVAL, "k_nn must lie in [1, 32]");
      if (m->cp_mode == MPWOS_CLOUD_CP_FIT && m->k_nn < 6) return fail(ctx, MPWOS_EINVAL, "the quadratic fit needs k_nn >= 6");
      if (m->n_cloud < m->k_nn || m->n_cloud > 0x7fffffffLL) return fail(ctx, MPWOS_EINVAL, "need k_nn <= n_cloud < 2^31");
      if (!(m->c_h > 0.0)) return fail(ctx, MPWOS_EINVAL, "c_h must be > 0");
      if (m->cp_mode != MPWOS_CLOUD_CP_FIT && m->cp_mode != MPWOS_CLOUD_CP_NEAREST) return fail(ctx, MPWOS_EINVAL, "unknown cp_mode");
      return MPWOS_OK;
    default:
      return fail(ctx, MPWOS_EINVAL, "unknown manifold kind %d", m->kind);
  }
}

// The description of a handle made on this context's device (null: EINVAL).
const mpwos_manifold_desc* handle_desc(mpwos_ctx* ctx, const mpwos_manifold* mh) {
  if (!mh) {
    fail(ctx, MPWOS_EINVAL, "null manifold");
    return nullptr;
  }
  if (mh->device != ctx->device) {
    fail(ctx, MPWOS_EINVAL, "the manifold was created on device %d, the context runs on device %d", mh->device,
         ctx->device);
    return nullptr;
  }
  return &mh->desc;
}

int validate(mpwos_ctx* ctx, const mpwos_manifold_desc* m, const mpwos_problem* pr, const mpwos_params* pa,
             int64_t P, int64_t N) {
  if (!m || !pr || !pa) return fail(ctx, MPWOS_EINVAL, "null manifold, problem or params");
  if (P < 0 || N < 1) return fail(ctx, MPWOS_EINVAL, "need P >= 0 and N >= 1 (got P=%lld N=%lld)", (long long)P, (long long)N);
  if (N > 0x7fffffffLL || P > 0x7fffffffLL) return fail(ctx, MPWOS_EINVAL, "P and N must fit in 32 bits (Philox counter words)");
  if (!(pr->sigma > 0.0)) return fail(ctx, MPWOS_EINVAL, "sigma must be > 0 (got %g)", pr->sigma);
  if (!(pa->theta > 0.0 && pa->theta < 1.0)) return fail(ctx, MPWOS_EINVAL, "theta must lie in (0, 1)");
  if (!(pa->c_kappa > 0.0)) return fail(ctx, MPWOS_EINVAL, "c_kappa must be > 0");
  if (pa->n_v < 1 || pa->n_v > 64) return fail(ctx, MPWOS_EINVAL, "n_v must lie in [1, 64]");
  if (pa->max_steps < 0 || pa->max_steps > 0x7fffffffLL) return fail(ctx, MPWOS_EINVAL, "max_steps must lie in [0, 2^31)");
  if (pa->precision != MPWOS_FP64 && pa->precision != MPWOS_FP32) return fail(ctx, MPWOS_EINVAL, "unknown precision %d", pa->precision);
  if (pa->projection < MPWOS_PROJ_AUTO || pa->projection > MPWOS_PROJ_CUDA) return fail(ctx, MPWOS_EINVAL, "unknown projection %d", pa->projection);
  if (pa->projection == MPWOS_PROJ_TENSOR && (m->kind != MPWOS_EMBEDDED_SPHERE || pa->precision != MPWOS_FP32))
    return fail(ctx, MPWOS_EINVAL, "MPWOS_PROJ_TENSOR needs EMBEDDED_SPHERE and MPWOS_FP32");
  if (m->n < 3 || m->n > 1024) return fail(ctx, MPWOS_EINVAL, "ambient dimension must lie in [3, 1024] (got %d)", m->n);
  switch (m->kind) {
    case MPWOS_EUCLID:
      if (m->d != m->n) return fail(ctx, MPWOS_EINVAL, "EUCLID needs d == n");
      break;
    case MPWOS_SPHERE:
      if (m->d != m->n - 1) return fail(ctx, MPWOS_EINVAL, "SPHERE needs d == n - 1");
      break;
    case MPWOS_TORUS:
      if (m->n != 3 || m->d != 2) return fail(ctx, MPWOS_EINVAL, "TORUS lives in R^3 (n = 3, d = 2)");
      if (!(m->R > m->a && m->a > 0.0)) return fail(ctx, MPWOS_EINVAL, "TORUS needs R > a > 0");
      if (!pr->closed && pr->bnd_normal && (pr->bnd_normal[2] != 0.0 || pr->bnd_offset != 0.0))
        return fail(ctx, MPWOS_EINVAL, "a TORUS boundary must be a plane through the axis (e_3 = 0, h = 0)");
      break;
    case MPWOS_EMBEDDED_SPHERE:
      if (m->n <= 3) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs n > 3");
      if (m->d < 1 || m->d + 1 > kMaxQuadDim - 1 || m->d + 1 > m->n) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs 1 <= d <= min(n - 1, 30)");
      if (!m->Q || !m->b) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE needs Q and b");
      if (!pr->closed) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE supports the closed problem only");
      break;
    case MPWOS_REVOLUTION:
      if (m->n < 4 || m->d != m->n - 1) return fail(ctx, MPWOS_EINVAL, "REVOLUTION needs n >= 4 and d == n - 1");
      if (!(m->prof_alpha > 0.0 && m->prof_alpha < 0.5 && m->prof_kappa > 0.0))
        return fail(ctx, MPWOS_EINVAL, "REVOLUTION needs 0 < prof_alpha < 1/2 and prof_kappa > 0");
      if (!pr->closed) return fail(ctx, MPWOS_EINVAL, "REVOLUTION supports the closed problem only");
      if (pr->f.kind != MPWOS_FUNC_REVOLUTION_QUAD) return fail(ctx, MPWOS_EINVAL, "REVOLUTION source must be REVOLUTION_QUAD");
      if (pa->sampler != MPWOS_SAMPLER_FULL) return fail(ctx, MPWOS_EINVAL, "REVOLUTION needs the full sampler");
      break;
    case MPWOS_CURVE_SPHERE:
      if (m->n != 9 || m->d != 3) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE lives in R^9 (n = 9, d = 3)");
      if (!(m->R > 0.0 && m->a > 0.0)) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE needs R > 0 and a > 0");
      if (!pr->closed) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE supports the closed problem only");
      if (pr->f.kind != MPWOS_FUNC_CURVE_SPHERE) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE source must be CURVE_SPHERE data");
      if (pa->sampler != MPWOS_SAMPLER_FULL) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE needs the full sampler");
      break;
    case MPWOS_POINT_CLOUD:
      if (m->n != 3 || m->d != 2) return fail(ctx, MPWOS_EINVAL, "POINT_CLOUD lives in R^3 (n = 3, d = 2)");
      if (!m->cloud) return fail(ctx, MPWOS_EINVAL, "POINT_CLOUD needs cloud");
      if (m->k_nn < 1 || m->k_nn > 32) return fail(ctx, MPWOS_EINVAL, "k_nn must lie in [1, 32]");
      if (m->cp_mode == MPWOS_CLOUD_CP_FIT && m->k_nn < 6) return fail(ctx, MPWOS_EINVAL, "the quadratic fit needs k_nn >= 6");
      if (m->n_cloud < m->k_nn || m->n_cloud > 0x7fffffffLL) return fail(ctx, MPWOS_EINVAL, "need k_nn <= n_cloud < 2^31");
      if (!(m->c_h > 0.0)) return fail(ctx, MPWOS_EINVAL, "c_h must be > 0");
      if (m->cp_mode != MPWOS_CLOUD_CP_FIT && m->cp_mode != MPWOS_CLOUD_CP_NEAREST) return fail(ctx, MPWOS_EINVAL, "unknown cp_mode");
      if (!pr->closed) return fail(ctx, MPWOS_EINVAL, "POINT_CLOUD supports the closed problem only");
      break;
    default:
      return fail(ctx, MPWOS_EINVAL, "unknown manifold kind %d", m->kind);
  }
  if (!pr->closed) {
    if (m->kind != MPWOS_EUCLID && m->kind != MPWOS_SPHERE && m->kind != MPWOS_TORUS)
      return fail(ctx, MPWOS_EINVAL, "boundary needs EUCLID, SPHERE or TORUS");
    if (!pr->bnd_normal) return fail(ctx, MPWOS_EINVAL, "boundary problem needs bnd_normal");
    double nn = 0.0;
    for (int i = 0; i < m->n; ++i) nn += pr->bnd_normal[i] * pr->bnd_normal[i];
    if (std::fabs(nn - 1.0) > 1e-12) return fail(ctx, MPWOS_EINVAL, "bnd_normal must be a unit vector");
    if (m->kind == MPWOS_SPHERE && !(std::fabs(pr->bnd_offset) < 1.0)) return fail(ctx, MPWOS_EINVAL, "|bnd_offset| < 1 on the unit sphere");
    if (!(pa->eps > 0.0)) return fail(ctx, MPWOS_EINVAL, "eps must be > 0");
  } else if (!(pa->tau_w > 0.0 && pa->tau_w < 1.0)) {
    return fail(ctx, MPWOS_EINVAL, "tau_w must lie in (0, 1)");
  }
  // function kinds each kernel evaluates
  const mpwos_func* fs[2] = {&pr->f, &pr->g};
  for (int q = 0; q < 2; ++q) {
    const mpwos_func* f = fs[q];
    if (q == 1 && pr->closed) continue;
    if (f->n_terms < 0 || f->n_terms > kMaxTerms) return fail(ctx, MPWOS_EINVAL, "at most %d terms per function", kMaxTerms);
    if (f->kind == MPWOS_FUNC_POLY) {
      if (f->n_terms && (!f->coef || !f->term_off)) return fail(ctx, MPWOS_EINVAL, "POLY needs coef and term_off");
      int nf = f->n_terms ? f->term_off[f->n_terms] : 0;
      if (nf > kMaxPolyFactors) return fail(ctx, MPWOS_EINVAL, "at most %d polynomial factors", kMaxPolyFactors);
      for (int t = 0; t < nf; ++t)
        if (f->var[t] < 0 || f->var[t] >= m->n || f->pw[t] < 0 || f->pw[t] > 100)
          return fail(ctx, MPWOS_EINVAL, "POLY factor %d out of range", t);
      if (m->kind == MPWOS_EMBEDDED_SPHERE) return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE data must be SPHERE_QUAD");
    } else if (f->kind == MPWOS_FUNC_TORUS_FOURIER) {
      if (m->kind != MPWOS_TORUS) return fail(ctx, MPWOS_EINVAL, "TORUS_FOURIER needs the TORUS manifold");
      if (f->n_terms && (!f->coef || !f->modes)) return fail(ctx, MPWOS_EINVAL, "TORUS_FOURIER needs coef and modes");
      for (int t = 0; t < f->n_terms; ++t)
        if (f->modes[4 * t] < 0 || f->modes[4 * t] > 64 || f->modes[4 * t + 1] < 0 || f->modes[4 * t + 1] > 64)
          return fail(ctx, MPWOS_EINVAL, "torus mode numbers must lie in [0, 64]");
    } else if (f->kind == MPWOS_FUNC_CURVE_SPHERE) {
      if (m->kind != MPWOS_CURVE_SPHERE) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE data needs the CURVE_SPHERE manifold");
      if (f->n_terms && (!f->coef || !f->modes || !f->v || !f->A)) return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE data needs coef, modes, v, A");
      for (int t = 0; t < f->n_terms; ++t)
        if (f->modes[4 * t] < 0 || f->modes[4 * t] > 64 || (f->modes[4 * t + 1] != 0 && f->modes[4 * t + 1] != 1))
          return fail(ctx, MPWOS_EINVAL, "CURVE_SPHERE modes: q in [0, 64], trig 0 or 1");
    } else if (f->kind == MPWOS_FUNC_REVOLUTION_QUAD) {
      if (m->kind != MPWOS_REVOLUTION) return fail(ctx, MPWOS_EINVAL, "REVOLUTION_QUAD needs the REVOLUTION manifold");
      if (f->n_terms != 2 || !f->coef || !f->v || !f->A) return fail(ctx, MPWOS_EINVAL, "REVOLUTION_QUAD needs 2 coef, v and A");
    } else if (f->kind == MPWOS_FUNC_SPHERE_QUAD) {
      if (!(m->kind == MPWOS_EMBEDDED_SPHERE || (m->kind == MPWOS_SPHERE && m->n == 3)))
        return fail(ctx, MPWOS_EINVAL, "SPHERE_QUAD needs EMBEDDED_SPHERE or the sphere in R^3");
      if (!f->v || !f->A) return fail(ctx, MPWOS_EINVAL, "SPHERE_QUAD needs v and A");
    } else {
      return fail(ctx, MPWOS_EINVAL, "unknown function kind %d", f->kind);
    }
  }
  if (m->kind == MPWOS_EMBEDDED_SPHERE && pr->f.kind != MPWOS_FUNC_SPHERE_QUAD)
    return fail(ctx, MPWOS_EINVAL, "EMBEDDED_SPHERE source must be SPHERE_QUAD");
  if (pa->sampler != MPWOS_SAMPLER_FULL && pa->sampler != MPWOS_SAMPLER_REDUCED)
    return fail(ctx, MPWOS_EINVAL, "unknown sampler %d", pa->sampler);
  if (pr->comp != MPWOS_COMP_NONE) {
    const mpwos_func& u = pr->u_star;
    if (pr->comp != MPWOS_COMP_NORMAL2 && pr->comp != MPWOS_COMP_EXACT) return fail(ctx, MPWOS_EINVAL, "unknown comp %d", pr->comp);
    if (!(m->kind == MPWOS_TORUS || (m->kind == MPWOS_SPHERE && m->n == 3)))
      return fail(ctx, MPWOS_EINVAL, "compensation needs TORUS or the sphere in R^3");
    if (pa->sampler != MPWOS_SAMPLER_FULL) return fail(ctx, MPWOS_EINVAL, "compensation needs the full sampler");
    if (!(pr->h_eta >= 0.0 && pr->h_eta < 0.5)) return fail(ctx, MPWOS_EINVAL, "h_eta must lie in [0, 0.5)");
    if (u.apply_op) return fail(ctx, MPWOS_EINVAL, "the predictor u_star takes apply_op = 0");
    if (m->kind == MPWOS_TORUS) {
      if (u.kind != MPWOS_FUNC_TORUS_FOURIER) return fail(ctx, MPWOS_EINVAL, "on the TORUS u_star must be TORUS_FOURIER");
      if (u.n_terms < 0 || u.n_terms > kMaxPredTerms) return fail(ctx, MPWOS_EINVAL, "u_star takes at most %d terms", kMaxPredTerms);
      if (u.n_terms && (!u.coef || !u.modes)) return fail(ctx, MPWOS_EINVAL, "u_star needs coef and modes");
      for (int t = 0; t < u.n_terms; ++t)
        if (u.modes[4 * t] < 0 || u.modes[4 * t] > 64 || u.modes[4 * t + 1] < 0 || u.modes[4 * t + 1] > 64)
          return fail(ctx, MPWOS_EINVAL, "u_star mode numbers must lie in [0, 64]");
    } else {
      if (u.kind != MPWOS_FUNC_SPHERE_QUAD || !u.v || !u.A) return fail(ctx, MPWOS_EINVAL, "on the sphere u_star must be SPHERE_QUAD with v and A");
    }
  }
  if (pa->sampler == MPWOS_SAMPLER_REDUCED) {
    if (m->kind == MPWOS_EUCLID || m->kind == MPWOS_SPHERE) {
      if (m->n <= 3) return fail(ctx, MPWOS_EINVAL, "the reduced sampler needs n > 3 on SPHERE / EUCLID");
      int T[kMaxQuadDim];
      const int nT = tracked_set(m, pr, T);
      if (nT < 0) return fail(ctx, MPWOS_EINVAL, "the reduced sampler needs POLY data reading at most %d coordinates", kMaxQuadDim);
      if (m->kind == MPWOS_SPHERE && nT >= m->n) return fail(ctx, MPWOS_EINVAL, "the reduced sampler needs a coordinate outside the tracked set");
    } else if (m->kind != MPWOS_EMBEDDED_SPHERE) {
      return fail(ctx, MPWOS_EINVAL, "the reduced sampler supports SPHERE, EUCLID and EMBEDDED_SPHERE");
    }
  }
  return MPWOS_OK;
}

// Coefficients of the FP32 survival-weight polynomial em1(z) = sum_j k_j z^j,
// k_j = 1/(j! (nu+1)_j) (Lemma 3.1), enough terms for 1e-9 relative
// truncation at z_max; otherwise the FP32 walk falls back to the FP64 series.
void fill_em1_poly(DevProblem& pb, int n, double z_max) {
  const double nu = 0.5 * (n - 2);
  double kj = 1.0, zj = 1.0, em = 0.0, last = 1.0;
  int T = 0;
  for (int j = 1; j <= 32; ++j) {
    kj /= static_cast<double>(j) * (nu + j);
    zj *= z_max;
    pb.em1_k[j - 1] = static_cast<float>(kj);
    last = kj * zj;
    em += last;
    T = j;
    if (last <= 1e-9 * em) break;
  }
  pb.em1_terms = T;
  pb.em1_fp64 = (z_max > 0.0 && last > 1e-9 * em) ? 1 : 0;
}

// FP32 copies of the loop-invariant scalars (after the table and cloud are set).
void fill_scalars_f(DevProblem& pb) {
  ScalarsF& f = pb.sf;
  f.eps = static_cast<float>(pb.eps);
  f.theta = static_cast<float>(pb.theta);
  f.rho_geo = static_cast<float>(pb.rho_geo);
  f.sqrt_sigma = static_cast<float>(pb.sqrt_sigma);
  f.sigma = static_cast<float>(pb.sigma);
  f.inv_sigma = static_cast<float>(1.0 / pb.sigma);
  f.R = static_cast<float>(pb.R);
  f.a = static_cast<float>(pb.a_tube);
  f.inv_a = pb.a_tube != 0.0 ? static_cast<float>(1.0 / pb.a_tube) : 0.0f;
  f.h = static_cast<float>(pb.h);
  f.sh = static_cast<float>(std::sqrt(std::max(0.0, 1.0 - pb.h * pb.h)));
  f.c_h = static_cast<float>(pb.cl_c_h);
  f.tab_scale = static_cast<float>((pb.NS - 1) / 0.70710678118654752);
  f.z_scale = (pb.NA > 1 && pb.z_max > 0.0) ? static_cast<float>((pb.NA - 1) / pb.z_max) : 0.0f;
  for (int a = 0; a < 3; ++a) pb.cl_origin_f[a] = static_cast<float>(pb.cl_origin[a]);
  pb.cl_cell_f = static_cast<float>(pb.cl_cell);
}

// The FP32 warp walk's coordinate order (n > 3, full sampler; R^n, the sphere
// and the hypersurface of revolution): walk coordinate c holds ambient
// coordinate perm[c].  The revolution's axis comes first, then the coordinates
// that f and g read, then those of the boundary normal, then the rest in order
// (the walk reads these in slot 0 of the first lanes).  Remaps pb's POLY
// variables and fills e_s0; the host arrays to upload are the order, the whole
// normal in walk order when it reaches past walk coordinate 127, and the
// revolution's v and diag(A) in walk order, each padded to 1024 floats.
struct WalkOrder {
  std::vector<int> perm;
  std::vector<float> ef_w, v32, a32;
};

bool uses_walk_order(const mpwos_manifold_desc* m, const mpwos_params* pa) {
  return pa->precision == MPWOS_FP32 && pa->sampler == MPWOS_SAMPLER_FULL && m->n > 3 &&
         (m->kind == MPWOS_EUCLID || m->kind == MPWOS_SPHERE || m->kind == MPWOS_REVOLUTION);
}

void walk_order(const mpwos_manifold_desc* m, const mpwos_problem* pr, DevProblem& pb, WalkOrder& wo) {
  const int n = m->n;
  std::vector<int> pos(static_cast<size_t>(n), -1);
  wo.perm.clear();
  auto add = [&](int c) {
    if (c >= 0 && c < n && pos[c] < 0) {
      pos[c] = static_cast<int>(wo.perm.size());
      wo.perm.push_back(c);
    }
  };
  if (m->kind == MPWOS_REVOLUTION) add(n - 1);
  for (DevFunc* df : {&pb.f, &pb.g}) {
    if ((df == &pb.g && pr->closed) || df->kind != kPoly) continue;
    for (int q = 0; q < df->term_off[df->n_terms]; ++q) add(df->var[q]);
  }
  if (!pr->closed)
    for (int c = 0; c < n; ++c)
      if (pr->bnd_normal[c] != 0.0) add(c);
  for (int c = 0; c < n; ++c) add(c);
  for (DevFunc* df : {&pb.f, &pb.g}) {
    if ((df == &pb.g && pr->closed) || df->kind != kPoly) continue;
    for (int q = 0; q < df->term_off[df->n_terms]; ++q) df->var[q] = static_cast<int16_t>(pos[df->var[q]]);
  }
  bool past = false;
  for (int c = 0; c < 128; ++c) pb.e_s0[c] = 0.0f;
  if (!pr->closed)
    for (int c = 0; c < n; ++c) {
      const float e = static_cast<float>(pr->bnd_normal[wo.perm[c]]);
      if (c < 128) pb.e_s0[c] = e;
      else if (e != 0.0f) past = true;
    }
  wo.ef_w.clear();
  if (past) {
    wo.ef_w.assign(1024, 0.0f);
    for (int c = 0; c < n; ++c) wo.ef_w[c] = static_cast<float>(pr->bnd_normal[wo.perm[c]]);
  }
  wo.v32.clear();
  wo.a32.clear();
  if (m->kind == MPWOS_REVOLUTION) {
    wo.v32.assign(1024, 0.0f);
    wo.a32.assign(1024, 0.0f);
    for (int c = 1; c < n; ++c) {
      wo.v32[c] = static_cast<float>(pr->f.v[wo.perm[c]]);
      wo.a32[c] = static_cast<float>(pr->f.A[wo.perm[c]]);
    }
  }
}

// Rows of a variable-radius table: the law's dependence on z = a^2/4 enters
// through z/(nu + j); high dimensions need few rows.
int table_rows(int n) { return n <= 8 ? kTableNA : 17; }

void copy_func(const mpwos_func& f, DevFunc& d) {
  std::memset(&d, 0, sizeof d);
  d.single_mq = -1;
  d.kind = f.kind;
  d.apply_op = f.apply_op;
  d.n_terms = f.n_terms;
  d.c0 = f.c0;
  d.c0_f = static_cast<float>(f.c0);
  for (int t = 0; t < f.n_terms; ++t) {
    d.coef[t] = f.coef[t];
    d.coef_f[t] = static_cast<float>(f.coef[t]);
  }
  if (f.kind == MPWOS_FUNC_POLY) {
    for (int t = 0; t <= f.n_terms; ++t) d.term_off[t] = static_cast<int16_t>(f.n_terms ? f.term_off[t] : 0);
    const int nf = f.n_terms ? f.term_off[f.n_terms] : 0;
    for (int q = 0; q < nf; ++q) {
      d.var[q] = static_cast<int16_t>(f.var[q]);
      d.pw[q] = static_cast<int8_t>(f.pw[q]);
    }
  } else if (f.kind == MPWOS_FUNC_TORUS_FOURIER) {
    for (int t = 0; t < f.n_terms; ++t) {
      for (int q = 0; q < 4; ++q) d.modes[t][q] = static_cast<int8_t>(f.modes[4 * t + q]);
      const float m = static_cast<float>(f.modes[4 * t]), qq = static_cast<float>(f.modes[4 * t + 1]);
      d.mode_f[t][0] = m;
      d.mode_f[t][1] = qq;
      d.mode_f[t][2] = m * m;
      d.mode_f[t][3] = qq * qq;
    }
    if (f.n_terms == 1 && f.modes[0] <= 3 && f.modes[1] <= 3)
      d.single_mq = 4 * f.modes[0] + f.modes[1] + (f.modes[2] != 0 ? 16 : 0) + (f.modes[3] != 0 ? 32 : 0);
  } else if (f.kind == MPWOS_FUNC_CURVE_SPHERE) {
    for (int t = 0; t < f.n_terms; ++t)
      for (int q = 0; q < 4; ++q) d.modes[t][q] = static_cast<int8_t>(f.modes[4 * t + q]);
  }
}

// The compensation predictor (validated): coefficients, modes, the step and,
// for the sphere, the central differences of (1 + s)^-2 at 0 with step h.
void copy_pred(const mpwos_problem& pr, DevPredictor& d) {
  std::memset(&d, 0, sizeof d);
  d.comp = pr.comp;
  if (pr.comp == MPWOS_COMP_NONE) return;
  const mpwos_func& u = pr.u_star;
  const double h = pr.h_eta > 0.0 ? pr.h_eta : 1e-2;
  d.kind = u.kind;
  d.h = h;
  d.hf = static_cast<float>(h);
  if (u.kind == MPWOS_FUNC_TORUS_FOURIER) {
    d.n_terms = u.n_terms;
    for (int t = 0; t < u.n_terms; ++t) {
      d.coef[t] = u.coef[t];
      d.coef_f[t] = static_cast<float>(u.coef[t]);
      for (int q = 0; q < 4; ++q) d.modes[t][q] = static_cast<int8_t>(u.modes[4 * t + q]);
      d.mode_f[t][0] = static_cast<float>(u.modes[4 * t]);
      d.mode_f[t][1] = static_cast<float>(u.modes[4 * t + 1]);
    }
  } else {
    d.c0 = u.c0;
    d.c0_f = static_cast<float>(u.c0);
    for (int i = 0; i < 3; ++i) { d.v[i] = u.v[i]; d.v_f[i] = static_cast<float>(u.v[i]); }
    for (int i = 0; i < 9; ++i) { d.A[i] = u.A[i]; d.A_f[i] = static_cast<float>(u.A[i]); }
    const double gp = 1.0 / ((1.0 + h) * (1.0 + h)), gm = 1.0 / ((1.0 - h) * (1.0 - h));
    d.sd1 = static_cast<float>((gp - gm) / (2.0 * h));
    d.sd2 = static_cast<float>((gp - 2.0 + gm) / (h * h));
  }
}

// The radius table for (n, law range): cached per context.
int get_table(mpwos_ctx* ctx, int n, bool fixed, double a_or_zmax, Table** out) {
  const int NA = fixed ? 1 : table_rows(n);
  auto key = std::make_tuple(n, NA, a_or_zmax);
  auto it = ctx->tables.find(key);
  if (it != ctx->tables.end()) {
    *out = &it->second;
    return MPWOS_OK;
  }
  Table t;
  t.NA = NA;
  t.NS = kTableNS;
  t.z_max = fixed ? 0.25 * a_or_zmax * a_or_zmax : a_or_zmax;
  const size_t cnt = static_cast<size_t>(NA) * 2 * (kTableNS + 2);
  CK(cudaMalloc(&t.tab64, cnt * sizeof(double)));
  CK(cudaMalloc(&t.tabc, static_cast<size_t>(NA) * 2 * (kTableNS - 1) * sizeof(float4)));
  CK(launch_build_table(n, NA, kTableNS, t.z_max, fixed ? a_or_zmax : 0.0, t.tab64, t.tabc, ctx->stream));
  ctx->launches += 1;
  auto res = ctx->tables.emplace(key, t);
  *out = &res.first->second;
  return MPWOS_OK;
}

// The search grid of a point cloud (built once, for its manifold handle).
int build_cloud(mpwos_ctx* ctx, const mpwos_manifold_desc* m, CloudGrid& G) {
  const int64_t N = m->n_cloud;
  const double* P = m->cloud;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], P[3 * i + a]);
      hi[a] = std::max(hi[a], P[3 * i + a]);
    }
  // cell size ~ the k-th neighbour distance, estimated on a sample of 32 points
  const int k = m->k_nn;
  double rk = 0.0;
  int ns = 0;
  std::vector<double> best(k);
  for (int64_t sidx = 0; sidx < N && ns < 32; sidx += std::max<int64_t>(1, N / 32), ++ns) {
    std::fill(best.begin(), best.end(), INFINITY);
    for (int64_t i = 0; i < N; ++i) {
      double dd = 0.0;
      for (int a = 0; a < 3; ++a) dd += (P[3 * i + a] - P[3 * sidx + a]) * (P[3 * i + a] - P[3 * sidx + a]);
      if (dd < best[k - 1]) {
        int j = k - 1;
        while (j > 0 && best[j - 1] > dd) { best[j] = best[j - 1]; --j; }
        best[j] = dd;
      }
    }
    rk += std::sqrt(best[k - 1]);
  }
  double cs = 1.25 * rk / ns;
  const double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  if (!(cs > 0.0)) cs = ext > 0.0 ? ext : 1.0;
  for (;;) {
    for (int a = 0; a < 3; ++a) G.dims[a] = static_cast<int>(std::floor((hi[a] - lo[a]) / cs)) + 1;
    if (static_cast<int64_t>(G.dims[0]) * G.dims[1] * G.dims[2] <= (int64_t(1) << 24)) break;
    cs *= 1.25;
  }
  const int ncells = G.dims[0] * G.dims[1] * G.dims[2];
  for (int a = 0; a < 3; ++a) G.origin[a] = lo[a];
  G.cell = cs;
  double* dpts = nullptr;
  int *cell = nullptr, *counts = nullptr, *cursor = nullptr;
  CK(cudaMalloc(&G.pts64, sizeof(double) * 3 * N));
  CK(cudaMalloc(&G.pts32, sizeof(float) * 3 * N));
  CK(cudaMalloc(&G.pts4, sizeof(float4) * N));
  CK(cudaMalloc(&G.orig, sizeof(int) * N));
  CK(cudaMalloc(&G.start, sizeof(int) * (ncells + 1)));
  CK(cudaMalloc(&dpts, sizeof(double) * 3 * N));
  CK(cudaMalloc(&cell, sizeof(int) * N));
  CK(cudaMalloc(&counts, sizeof(int) * ncells));
  CK(cudaMalloc(&cursor, sizeof(int) * ncells));
  CK(cudaMemcpyAsync(dpts, P, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_cloud_grid(dpts, N, G.origin, cs, G.dims, cell, counts, G.start, cursor, G.pts64, G.pts32, G.pts4,
                       G.orig, ctx->stream));
  ctx->launches += 3;
  // largest h(p) over the cloud
  DevProblem tmp;
  std::memset(&tmp, 0, sizeof tmp);
  tmp.cl_pts64 = G.pts64;
  tmp.cl_pts32 = G.pts32;
  tmp.cl_pts4 = G.pts4;
  tmp.cl_orig = G.orig;
  tmp.cl_start = G.start;
  for (int a = 0; a < 3; ++a) { tmp.cl_origin[a] = G.origin[a]; tmp.cl_dims[a] = G.dims[a]; }
  tmp.cl_cell = cs;
  tmp.cl_k = k;
  unsigned long long* hbits = nullptr;
  CK(cudaMalloc(&hbits, sizeof(unsigned long long)));
  CK(cudaMemsetAsync(hbits, 0, sizeof(unsigned long long), ctx->stream));
  CK(launch_cloud_hmax(tmp, N, hbits, ctx->stream));
  ctx->launches++;
  unsigned long long hb = 0;
  CK(cudaMemcpyAsync(&hb, hbits, sizeof hb, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::memcpy(&G.h_max, &hb, sizeof(double));
  cudaFree(dpts);
  cudaFree(cell);
  cudaFree(counts);
  cudaFree(cursor);
  cudaFree(hbits);
  return MPWOS_OK;
}

void free_cloud(CloudGrid& G) {
  cudaFree(G.pts64);
  cudaFree(G.pts32);
  cudaFree(G.pts4);
  cudaFree(G.orig);
  cudaFree(G.start);
  G = CloudGrid{};
}

// BF16 round-to-nearest-even of an FP32 value (finite inputs).
uint16_t bf16_rne(float f) {
  uint32_t x;
  std::memcpy(&x, &f, sizeof x);
  x += 0x7FFFu + ((x >> 16) & 1u);
  return static_cast<uint16_t>(x >> 16);
}
float bf16_value(uint16_t h) {
  const uint32_t x = static_cast<uint32_t>(h) << 16;
  float f;
  std::memcpy(&f, &x, sizeof f);
  return f;
}

// Shared-memory image of Q^T for the tensor-core walk: B operand rows j < 32
// (d + 1 used, rest zero), K-chunks of 64 components, each chunk 32 rows of
// 128 bytes with 16-byte unit u of row j stored at unit u ^ (j mod 8); hi =
// bf16(Q), lo = bf16(Q - hi); hi chunks first, then lo chunks.
void tc_bimage(const double* Q, int n, int D, std::vector<uint16_t>& img) {
  const size_t half = embed_tc_bimg_bytes() / 4;   // uint16 elements in the hi (or lo) part
  img.assign(2 * half, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < D; ++j) {
      const double q = Q[static_cast<size_t>(i) * D + j];
      const uint16_t hi = bf16_rne(static_cast<float>(q));
      const uint16_t lo = bf16_rne(static_cast<float>(q - static_cast<double>(bf16_value(hi))));
      const int c = i / 64, kk = i % 64, u = kk / 8, e = kk % 8;
      const size_t byte = static_cast<size_t>(c) * 4096 + static_cast<size_t>(j) * 128 +
                          static_cast<size_t>(((u ^ (j & 7)) << 4) + 2 * e);
      img[byte / 2] = hi;
      img[half + byte / 2] = lo;
    }
}

// Everything a walk launch needs, built in `sc`.
int prepare(mpwos_ctx* ctx, Scratch& sc, const mpwos_manifold* mh, const mpwos_problem* pr,
            const mpwos_params* pa, const double* pts, int64_t P, int64_t N, DevProblem& pb) {
  const mpwos_manifold_desc* m = &mh->desc;
  std::memset(&pb, 0, sizeof pb);
  pb.mkind = m->kind;
  pb.n = m->n;
  pb.d = m->d;
  pb.R = m->R;
  pb.a_tube = m->a;
  pb.sigma = pr->sigma;
  pb.sqrt_sigma = std::sqrt(pr->sigma);
  pb.closed = pr->closed;
  pb.h = pr->bnd_offset;
  pb.eps = pa->eps;
  pb.tau_w = pa->tau_w;
  pb.theta = pa->theta;
  pb.c_kappa = pa->c_kappa;
  pb.kappa = kappa_of(m);
  pb.rho_geo = pa->c_kappa / (1.0 + pb.kappa);
  pb.n_v = pa->n_v;
  pb.max_steps = pa->max_steps;
  pb.seed = pa->seed;
  pb.keys = philox_keys(static_cast<uint32_t>(pa->seed), static_cast<uint32_t>(pa->seed >> 32));
  pb.P = P;
  pb.N = N;
  pb.wk_points = nullptr;
  pb.wk_np = P;
  pb.wk_i0 = 0;
  pb.wk_i1 = N;
  pb.wk_w0 = 0;
  pb.wk_w1 = P * N;
  pb.out_stride = N;
  copy_func(pr->f, pb.f);
  if (!pr->closed) copy_func(pr->g, pb.g);
  copy_pred(*pr, pb.pred);
  pb.wk_next = sc.alloc<unsigned long long>(1);   // dynamic walk queue (static stride if null)
  const int n = m->n;
  if (!pr->closed) {
    std::vector<float> ef(pr->bnd_normal, pr->bnd_normal + n);
    pb.e = sc.upload(pr->bnd_normal, n);
    pb.ef = sc.upload(ef.data(), n);
    if (!pb.e || !pb.ef) return fail(ctx, MPWOS_ENOMEM, "boundary normal");
  }
  // SPHERE_QUAD coefficient arrays
  const int D = m->d + 1;
  for (DevFunc* df : {&pb.f, &pb.g}) {
    const mpwos_func& hf = (df == &pb.f) ? pr->f : pr->g;
    if (df == &pb.g && pr->closed) continue;
    if (hf.kind == MPWOS_FUNC_SPHERE_QUAD) {
      const int Dq = (m->kind == MPWOS_SPHERE) ? 3 : D;
      std::vector<float> vf(hf.v, hf.v + Dq), Af(hf.A, hf.A + static_cast<size_t>(Dq) * Dq);
      df->v = sc.upload(hf.v, Dq);
      df->A = sc.upload(hf.A, static_cast<size_t>(Dq) * Dq);
      df->vf = sc.upload(vf.data(), vf.size());
      df->Af = sc.upload(Af.data(), Af.size());
      if (!df->v || !df->A || !df->vf || !df->Af) return fail(ctx, MPWOS_ENOMEM, "SPHERE_QUAD data");
    }
  }
  // Fourier curve x sphere: f's v (3 per term) and A (9 per term)
  if (m->kind == MPWOS_CURVE_SPHERE) {
    const int nt = pr->f.n_terms > 0 ? pr->f.n_terms : 1;
    std::vector<double> v(3 * nt, 0.0), A(9 * nt, 0.0);
    if (pr->f.n_terms) {
      std::copy(pr->f.v, pr->f.v + 3 * pr->f.n_terms, v.begin());
      std::copy(pr->f.A, pr->f.A + 9 * pr->f.n_terms, A.begin());
    }
    std::vector<float> vf(v.begin(), v.end()), Af(A.begin(), A.end());
    pb.f.v = sc.upload(v.data(), v.size());
    pb.f.A = sc.upload(A.data(), A.size());
    pb.f.vf = sc.upload(vf.data(), vf.size());
    pb.f.Af = sc.upload(Af.data(), Af.size());
    if (!pb.f.v || !pb.f.A || !pb.f.vf || !pb.f.Af) return fail(ctx, MPWOS_ENOMEM, "CURVE_SPHERE data");
  }
  // hypersurface of revolution: f's v and diag(A) (n - 1 entries), profile, tr(A)/(n-1)
  if (m->kind == MPWOS_REVOLUTION) {
    const int nh = n - 1;
    std::vector<float> vf(pr->f.v, pr->f.v + nh), Af(pr->f.A, pr->f.A + nh);
    pb.f.v = sc.upload(pr->f.v, nh);
    pb.f.A = sc.upload(pr->f.A, nh);
    pb.f.vf = sc.upload(vf.data(), nh);
    pb.f.Af = sc.upload(Af.data(), nh);
    if (!pb.f.v || !pb.f.A || !pb.f.vf || !pb.f.Af) return fail(ctx, MPWOS_ENOMEM, "REVOLUTION_QUAD data");
    double trA = 0.0;
    for (int i = 0; i < nh; ++i) trA += pr->f.A[i];
    pb.rv_alpha = m->prof_alpha;
    pb.rv_kappa = m->prof_kappa;
    pb.rv_mA = trA / nh;
    pb.rv_alpha_f = static_cast<float>(m->prof_alpha);
    pb.rv_kappa_f = static_cast<float>(m->prof_kappa);
    pb.rv_mA_f = static_cast<float>(pb.rv_mA);
    pb.rv_ck_f = static_cast<float>(pa->c_kappa);
  }
  // the FP32 warp walk's coordinate order
  if (uses_walk_order(m, pa)) {
    WalkOrder wo;
    walk_order(m, pr, pb, wo);
    pb.perm = sc.upload(wo.perm.data(), wo.perm.size());
    if (!pb.perm) return fail(ctx, MPWOS_ENOMEM, "walk coordinate order");
    if (!wo.ef_w.empty() && !(pb.ef_w = sc.upload(wo.ef_w.data(), wo.ef_w.size())))
      return fail(ctx, MPWOS_ENOMEM, "boundary normal");
    if (!wo.v32.empty()) {
      pb.rv_v32 = sc.upload(wo.v32.data(), wo.v32.size());
      pb.rv_a32 = sc.upload(wo.a32.data(), wo.a32.size());
      if (!pb.rv_v32 || !pb.rv_a32) return fail(ctx, MPWOS_ENOMEM, "REVOLUTION_QUAD data");
    }
  }
  // query points
  if (is_device_ptr(pts)) {
    pb.pts = pts;
  } else {
    pb.pts = sc.upload(pts, static_cast<size_t>(P) * n);
    if (!pb.pts && P) return fail(ctx, MPWOS_ENOMEM, "query points");
  }
  if (m->kind == MPWOS_EMBEDDED_SPHERE) {
    const int npad = (n + 3) & ~3;
    double* s0 = sc.alloc<double>(static_cast<size_t>(P) * D);
    if (!s0) return fail(ctx, MPWOS_ENOMEM, "intrinsic start points");
    pb.Q = mh->qt;   // Q^T, D x npad
    pb.Qf = mh->qtf;   // group order, rows of 1024
    pb.b = mh->bd;
    pb.s0 = s0;
    if (P) {
      CK(launch_intrinsic_start(pb.pts, mh->qt, mh->bd, n, npad, D, P, s0, sc.stream));
      ctx->launches++;
    }
    const bool tc = pa->precision == MPWOS_FP32 && pa->sampler == MPWOS_SAMPLER_FULL &&
                    (pa->projection == MPWOS_PROJ_TENSOR || (pa->projection == MPWOS_PROJ_AUTO && n >= 128));
    if (tc) {
      pb.tc_bimg = reinterpret_cast<const uint4*>(mh->tc_img);
      pb.dev_status = sc.alloc<unsigned>(1);
      if (!pb.dev_status) return fail(ctx, MPWOS_ENOMEM, "tensor-core walk status");
      CK(cudaMemsetAsync(pb.dev_status, 0, sizeof(unsigned), sc.stream));
    }
  }
  // reduced sampler: tracked coordinates, remapped POLY variables, start states
  if (pa->sampler == MPWOS_SAMPLER_REDUCED) {
    pb.reduced = 1;
    if (m->kind == MPWOS_EMBEDDED_SPHERE) {
      pb.red_nT = D;
      pb.red_rest = n - D;
    } else {
      int T[kMaxQuadDim];
      const int nT = tracked_set(m, pr, T);
      std::vector<int> pos(static_cast<size_t>(n), -1);
      for (int q = 0; q < nT; ++q) pos[T[q]] = q;
      for (DevFunc* df : {&pb.f, &pb.g}) {
        if (df->kind != kPoly) continue;
        const int nf = df->term_off[df->n_terms];
        for (int q = 0; q < nf; ++q) df->var[q] = static_cast<int16_t>(pos[df->var[q]]);
      }
      pb.red_nT = nT;
      pb.red_rest = (m->kind == MPWOS_SPHERE) ? n - nT - 1 : n - nT;
      for (int q = 0; q < nT; ++q) {
        pb.red_e[q] = pr->closed ? 0.0 : pr->bnd_normal[T[q]];
        pb.red_ef[q] = static_cast<float>(pb.red_e[q]);
      }
      int* dT = sc.upload(T, static_cast<size_t>(nT > 0 ? nT : 1));
      double* y0 = sc.alloc<double>(static_cast<size_t>(P > 0 ? P : 1) * (kMaxQuadDim + 1));
      if (!dT || !y0) return fail(ctx, MPWOS_ENOMEM, "reduced start states");
      if (P) {
        CK(launch_reduced_start(pb.pts, n, dT, nT, P, m->kind == MPWOS_SPHERE, y0, sc.stream));
        ctx->launches++;
      }
      pb.red_y0 = y0;
    }
  }
  // point cloud grid; rho_geo varies with h(y)
  double rho_geo_max = pb.rho_geo;
  if (m->kind == MPWOS_POINT_CLOUD) {
    const CloudGrid* G = &mh->grid;
    pb.cl_pts64 = G->pts64;
    pb.cl_pts32 = G->pts32;
    pb.cl_pts4 = G->pts4;
    pb.cl_orig = G->orig;
    pb.cl_start = G->start;
    for (int a = 0; a < 3; ++a) { pb.cl_origin[a] = G->origin[a]; pb.cl_dims[a] = G->dims[a]; }
    pb.cl_cell = G->cell;
    pb.cl_k = m->k_nn;
    pb.cl_c_h = m->c_h;
    pb.cl_mode = m->cp_mode;
    // h at an off-cloud point stays near h at its neighbours; 1.5 x max over the cloud
    rho_geo_max = m->c_h * 1.5 * G->h_max;
  }
  // hypersurface of revolution: rho_geo = c_kappa / (1 + kappa(y)) varies; its
  // largest value from the smallest curvature over a dense scan of the profile
  if (m->kind == MPWOS_REVOLUTION) rho_geo_max = pa->c_kappa / (1.0 + 0.99 * mh->rev_kmin);
  // radius tables
  const bool fixed_radius = pr->closed && m->kind != MPWOS_POINT_CLOUD && m->kind != MPWOS_REVOLUTION;
  const double a_max = pb.sqrt_sigma * pb.theta * rho_geo_max;
  const double nu = 0.5 * (n - 2);
  if (n > 3 && 0.25 * a_max * a_max > 0.5 * nu)
    return fail(ctx, MPWOS_EINVAL,
                "sigma (theta rho_geo)^2 / 4 = %g exceeds (n-2)/4 = %g: outside the series evaluation range", 0.25 * a_max * a_max, 0.5 * nu);
  fill_em1_poly(pb, n, 0.25 * a_max * a_max);
  Table* tab = nullptr;
  int rc = fixed_radius ? get_table(ctx, n, true, a_max, &tab) : get_table(ctx, n, false, 0.25 * a_max * a_max, &tab);
  if (rc) return rc;
  pb.tab64 = tab->tab64;
  pb.tabc = tab->tabc;
  pb.NA = tab->NA;
  pb.NS = tab->NS;
  pb.z_max = tab->z_max;
  fill_scalars_f(pb);
  return MPWOS_OK;
}

int launch_walks(mpwos_ctx* ctx, DevProblem& pb, bool fp64, cudaStream_t st, int64_t max_grid, int block);

int run_walks_on(mpwos_ctx* ctx, DevProblem& pb, bool fp64, cudaStream_t st, int64_t max_grid) {
  return launch_walks(ctx, pb, fp64, st, max_grid, 0);
}

int run_walks(mpwos_ctx* ctx, DevProblem& pb, bool fp64) { return run_walks_on(ctx, pb, fp64, ctx->stream, 0); }

// Launch the walk kernel for pb's work range on st; max_grid > 0 caps the grid,
// max_grid < 0 takes a 1/|max_grid| share of the full grid (served requests
// leave SMs to the other requests in flight).  block > 0 replaces the default
// block size (a multiple of 32 within the kernel's limit; the tensor-core walk
// keeps its own); the grid is then the SM count times the resident blocks of
// that size.
// The launch shape launch_walks uses for pb: block size, walkers per block and
// grid (before the grid is capped to the walks at hand).
struct LaunchShape {
  int block = 0;
  int64_t per_block = 0, grid = 0;
};

LaunchShape launch_shape(mpwos_ctx* ctx, const DevProblem& pb, bool fp64, int64_t max_grid, int block_req) {
  LaunchShape sh;
  if (pb.reduced) {
    sh.block = block_req > 0 ? block_req : 128;
    sh.per_block = sh.block;
    sh.grid = static_cast<int64_t>(ctx->sm_count) * occupancy_walkr(pb, fp64, sh.block);
    if (max_grid < 0) sh.grid = std::max<int64_t>(ctx->sm_count, sh.grid / (-max_grid));
  } else if (pb.tc_bimg && !fp64) {
    // one persistent CTA per SM (or a share of them), 128 walkers per tile
    sh.block = 512;
    sh.per_block = 128;
    sh.grid = ctx->sm_count;
    if (max_grid < 0) sh.grid = std::max<int64_t>(1, sh.grid / (-max_grid));
  } else {
    const bool n3 = pb.n == 3 && pb.mkind != kEmbeddedSphere;
    sh.block = block_req > 0 ? block_req
                             : (n3 ? ((fp64 || pb.mkind == kPointCloud) ? 128 : 256)
                                   : (fp64 ? 128 : walkn32_max_block(pb)));
    const int occ = fp64 ? occupancy_walk_f64(pb, n3, sh.block) : occupancy_walk_f32(pb, n3, sh.block);
    sh.per_block = n3 ? sh.block : sh.block / (fp64 ? 32 : walkn32_lanes_per_walker(pb));
    sh.grid = static_cast<int64_t>(ctx->sm_count) * occ;
    if (max_grid < 0) sh.grid = std::max<int64_t>(ctx->sm_count, sh.grid / (-max_grid));
  }
  if (max_grid > 0 && sh.grid > max_grid) sh.grid = max_grid;
  return sh;
}

int launch_walks(mpwos_ctx* ctx, DevProblem& pb, bool fp64, cudaStream_t st, int64_t max_grid, int block_req) {
  if (pb.wk_w1 <= pb.wk_w0) return MPWOS_OK;
  if (!pb.S_out || !pb.K_out || !pb.flag_out || !pb.pts || !pb.tab64 || !pb.tabc)
    return fail(ctx, MPWOS_EINVAL, "internal: walk launch without its buffers");
  if (pb.wk_next) CK(cudaMemsetAsync(pb.wk_next, 0, sizeof(unsigned long long), st));
  LaunchShape sh = launch_shape(ctx, pb, fp64, max_grid, block_req);
  pb.cl_spread = 1;
  if (!fp64 && pb.mkind == kPointCloud && pb.cl_k >= 12) {
    // the warp-cooperative search runs the warp's walkers' queries one after
    // another: a launch of fewer walks than the grid holds spreads them over
    // more warps (up to one walker per warp), which shortens each step
    const int64_t slots = sh.grid * sh.per_block, walks = pb.wk_w1 - pb.wk_w0;
    while (pb.cl_spread < 32 && walks * 2 * pb.cl_spread <= slots) pb.cl_spread *= 2;
    sh.per_block /= pb.cl_spread;
  }
  const int64_t need = (pb.wk_w1 - pb.wk_w0 + sh.per_block - 1) / sh.per_block;
  const int grid = static_cast<int>(std::min(sh.grid, need));
  cudaError_t e;
  const int64_t walks = pb.wk_w1 - pb.wk_w0;
  if (pb.reduced && !fp64 && walkr_lat_eligible(pb) && walks <= 32 * static_cast<int64_t>(ctx->sm_count)) {
    // few walks on an embedded sphere: one warp per walker shortens each step
    // (the walks are the same bit for bit)
    e = launch_walkr_lat_f32(pb, static_cast<int>((walks + 3) / 4), st);
  } else if (pb.reduced) {
    e = fp64 ? launch_walkr_f64(pb, grid, sh.block, st) : launch_walkr_f32(pb, grid, sh.block, st);
  } else if (pb.tc_bimg && !fp64) {
    e = launch_embed_tc(pb, grid, st);
  } else {
    const bool n3 = pb.n == 3 && pb.mkind != kEmbeddedSphere;
    if (n3) e = fp64 ? launch_walk3_f64(pb, grid, sh.block, st) : launch_walk3_f32(pb, grid, sh.block, st);
    else e = fp64 ? launch_walkn_f64(pb, grid, sh.block, st) : launch_walkn_f32(pb, grid, sh.block, st);
  }
  if (e != cudaSuccess) return fail(ctx, MPWOS_ECUDA, "walk launch: %s", cudaGetErrorString(e));
  ctx->launches++;
  return MPWOS_OK;
}

// The autotuned block size for pb's walk kernel, or 0 (the default shape)
// when tuning is off or nothing was measured for it yet.
int tuned_block(mpwos_ctx* ctx, const DevProblem& pb, bool fp64) {
  if (!ctx->autotune || (pb.tc_bimg && !fp64)) return 0;
  const void* fn = fp64 ? walk_fn_f64(pb) : walk_fn_f32(pb);
  const auto it = ctx->tune.find({fn, pb.n});
  return it == ctx->tune.end() ? 0 : it->second.block;
}

// Walks of pb's range on the context's stream, with the launch-shape
// autotuner when it is on.  The first call for a (kernel, n) with at least two
// waves of walks per part splits its walks into (candidates + 1) equal parts;
// each of the first parts runs with one candidate block size (32 to 256
// threads within the kernel's limit, each launch filling every SM) and is timed
// with CUDA events, divided by its walk-steps (read back from K_out, whose row
// for walk w is w in these calls); the fastest is kept and runs the last part.  Each walk's draws depend only on
// (point, walk, step), so the shape changes no result.
int run_walks_tuned(mpwos_ctx* ctx, DevProblem& pb, bool fp64) {
  cudaStream_t st = ctx->stream;
  if (!ctx->autotune || (pb.tc_bimg && !fp64)) return launch_walks(ctx, pb, fp64, st, 0, 0);
  const void* fn = fp64 ? walk_fn_f64(pb) : walk_fn_f32(pb);
  if (!fn || pb.wk_points || pb.wk_i0 != 0 || pb.out_stride != pb.wk_i1) return launch_walks(ctx, pb, fp64, st, 0, 0);
  const auto key = std::make_pair(fn, pb.n);
  const auto it = ctx->tune.find(key);
  if (it != ctx->tune.end()) return launch_walks(ctx, pb, fp64, st, 0, it->second.block);
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, fn));
  const bool n3 = !pb.reduced && pb.n == 3 && pb.mkind != kEmbeddedSphere;
  const bool warp = !pb.reduced && !n3;
  std::vector<int> cand;
  for (int b : {32, 64, 128, 256})
    if (b <= fa.maxThreadsPerBlock) cand.push_back(b);
  // a chunk is two waves of the largest resident walker set among the candidates
  int64_t wave = 0;
  for (int b : cand) {
    const int occ = pb.reduced ? occupancy_walkr(pb, fp64, b)
                               : (fp64 ? occupancy_walk_f64(pb, n3, b) : occupancy_walk_f32(pb, n3, b));
    const int lpw = fp64 ? 32 : (warp ? walkn32_lanes_per_walker(pb) : 1);
    wave = std::max<int64_t>(wave, static_cast<int64_t>(ctx->sm_count) * occ * (warp ? b / lpw : b));
  }
  const int64_t nc = static_cast<int64_t>(cand.size());
  if (cand.empty() || pb.wk_w1 - pb.wk_w0 < 2 * wave * (nc + 1)) return launch_walks(ctx, pb, fp64, st, 0, 0);
  // every chunk is useful work, so the chunks take most of the call: the more
  // waves a chunk holds, the less its time depends on its longest walk
  const int64_t chunk = (pb.wk_w1 - pb.wk_w0) / (nc + 1);
  std::vector<cudaEvent_t> ev(cand.size() + 1, nullptr);
  int rc = MPWOS_OK;
  for (auto& e : ev)
    if (!rc && cudaEventCreate(&e) != cudaSuccess) rc = fail(ctx, MPWOS_ECUDA, "autotune: event create");
  const int64_t w0 = pb.wk_w0, w1 = pb.wk_w1;
  if (!rc && cudaEventRecord(ev[0], st) != cudaSuccess) rc = fail(ctx, MPWOS_ECUDA, "autotune: event record");
  for (int64_t c = 0; c < nc && !rc; ++c) {
    pb.wk_w0 = w0 + c * chunk;
    pb.wk_w1 = pb.wk_w0 + chunk;
    rc = launch_walks(ctx, pb, fp64, st, 0, cand[c]);
    if (!rc && cudaEventRecord(ev[c + 1], st) != cudaSuccess) rc = fail(ctx, MPWOS_ECUDA, "autotune: event record");
  }
  std::vector<int32_t> ks;
  if (!rc) {
    ks.resize(static_cast<size_t>(nc * chunk));
    if (cudaMemcpyAsync(ks.data(), pb.K_out + w0, ks.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = fail(ctx, MPWOS_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
  }
  TuneEntry te;
  te.cand = cand;
  double best = 0.0;
  for (int64_t c = 0; c < nc && !rc; ++c) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, ev[c], ev[c + 1]) != cudaSuccess) {
      rc = fail(ctx, MPWOS_ECUDA, "autotune: event timing");
      break;
    }
    int64_t steps = 0;
    for (int64_t q = c * chunk; q < (c + 1) * chunk; ++q) steps += ks[static_cast<size_t>(q)];
    const double ns = 1e6 * ms / static_cast<double>(std::max<int64_t>(steps, chunk));
    te.ns_per_step.push_back(ns);
    if (te.block == 0 || ns < best) {
      best = ns;
      te.block = cand[c];
    }
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  pb.wk_w0 = w0 + nc * chunk;
  pb.wk_w1 = w1;
  if (!rc) {
    ctx->tune[key] = te;
    rc = launch_walks(ctx, pb, fp64, st, 0, te.block);
  }
  pb.wk_w0 = w0;
  return rc;
}

}  // namespace

extern "C" {

int mpwos_cloud_knn(mpwos_ctx* ctx, const mpwos_manifold* mh, const double* x, int64_t nq, int precision,
                    int method, int32_t* idx, double* d2, double* h) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  if (m->kind != MPWOS_POINT_CLOUD || !mh->has_grid) return fail(ctx, MPWOS_EINVAL, "not a point cloud");
  if (m->k_nn < 1 || m->k_nn > 32) return fail(ctx, MPWOS_EINVAL, "k_nn must lie in [1, 32]");
  if (m->n_cloud < m->k_nn || m->n_cloud > 0x7fffffffLL) return fail(ctx, MPWOS_EINVAL, "need k_nn <= n_cloud < 2^31");
  if (nq < 0 || (nq > 0 && (!x || !idx || !d2 || !h))) return fail(ctx, MPWOS_EINVAL, "queries or outputs");
  if (precision != MPWOS_FP32 && precision != MPWOS_FP64) return fail(ctx, MPWOS_EINVAL, "precision");
  if (method != MPWOS_KNN_GRID && method != MPWOS_KNN_GRID_WARP && method != MPWOS_KNN_SCAN)
    return fail(ctx, MPWOS_EINVAL, "unknown method %d", method);
  if (method == MPWOS_KNN_GRID_WARP && precision == MPWOS_FP64)
    return fail(ctx, MPWOS_EINVAL, "the warp-cooperative search is FP32 only");
  if (nq == 0) return MPWOS_OK;
  const CloudGrid* G = &mh->grid;
  DevProblem pb;
  std::memset(&pb, 0, sizeof pb);
  pb.cl_pts64 = G->pts64;
  pb.cl_pts32 = G->pts32;
  pb.cl_pts4 = G->pts4;
  pb.cl_orig = G->orig;
  pb.cl_start = G->start;
  for (int a = 0; a < 3; ++a) {
    pb.cl_origin[a] = G->origin[a];
    pb.cl_dims[a] = G->dims[a];
    pb.cl_origin_f[a] = static_cast<float>(G->origin[a]);
  }
  pb.cl_cell = G->cell;
  pb.cl_cell_f = static_cast<float>(G->cell);
  pb.cl_k = m->k_nn;
  const int k = m->k_nn;
  Scratch sc(ctx);
  const bool dx = is_device_ptr(x), di = is_device_ptr(idx), dd = is_device_ptr(d2), dh = is_device_ptr(h);
  const double* xd = x;
  if (!dx) {
    double* t = sc.alloc<double>(static_cast<size_t>(nq) * 3);
    if (!t) return fail(ctx, MPWOS_ENOMEM, "queries");
    CK(cudaMemcpyAsync(t, x, sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, ctx->stream));
    xd = t;
  }
  int32_t* io = di ? idx : sc.alloc<int32_t>(static_cast<size_t>(nq) * k);
  double* d2o = dd ? d2 : sc.alloc<double>(static_cast<size_t>(nq) * k);
  double* ho = dh ? h : sc.alloc<double>(static_cast<size_t>(nq));
  if (!io || !d2o || !ho) return fail(ctx, MPWOS_ENOMEM, "kNN outputs");
  const int max_blocks = ctx->sm_count * 16;
  const cudaError_t e =
      precision == MPWOS_FP32
          ? launch_cloud_knn_f32(pb, xd, nq, method, m->n_cloud, io, d2o, ho, max_blocks, ctx->stream)
          : launch_cloud_knn_f64(pb, xd, nq, method, m->n_cloud, io, d2o, ho, max_blocks, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, MPWOS_ECUDA, "kNN launch: %s", cudaGetErrorString(e));
  ctx->launches++;
  if (!di) CK(cudaMemcpyAsync(idx, io, sizeof(int32_t) * nq * k, cudaMemcpyDeviceToHost, ctx->stream));
  if (!dd) CK(cudaMemcpyAsync(d2, d2o, sizeof(double) * nq * k, cudaMemcpyDeviceToHost, ctx->stream));
  if (!dh) CK(cudaMemcpyAsync(h, ho, sizeof(double) * nq, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MPWOS_OK;
}

int mpwos_set_autotune(mpwos_ctx* ctx, int enable) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  ctx->autotune = enable != 0;
  return MPWOS_OK;
}

int mpwos_autotune_entries(mpwos_ctx* ctx, mpwos_tune_entry* entries, int capacity, int* count) {
  if (!ctx || !count || capacity < 0 || (capacity > 0 && !entries)) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  *count = static_cast<int>(ctx->tune.size());
  int q = 0;
  for (const auto& kv : ctx->tune) {
    if (q >= capacity) break;
    mpwos_tune_entry& e = entries[q++];
    e = mpwos_tune_entry{};
    const char* name = nullptr;
    if (cudaFuncGetName(&name, kv.first.first) != cudaSuccess) {
      cudaGetLastError();
      name = nullptr;
    }
    e.kernel = name;
    e.n = kv.first.second;
    e.block = kv.second.block;
    e.n_candidates = static_cast<int>(std::min<size_t>(kv.second.cand.size(), 4));
    for (int c = 0; c < e.n_candidates; ++c) {
      e.candidates[c] = kv.second.cand[c];
      e.ns_per_walk_step[c] = kv.second.ns_per_step[c];
    }
  }
  return MPWOS_OK;
}

void mpwos_params_default(mpwos_params* p) {
  if (!p) return;
  p->eps = 1e-3;
  p->tau_w = 1e-8;
  p->theta = 0.95;
  p->c_kappa = 1.2;
  p->n_v = 1;
  p->max_steps = 10000000;
  p->seed = 0;
  p->precision = MPWOS_FP64;
  p->projection = MPWOS_PROJ_AUTO;
  p->sampler = MPWOS_SAMPLER_FULL;
}

int mpwos_create(int device, void* stream, mpwos_ctx** out) {
  if (!out) return MPWOS_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return MPWOS_EINVAL;
  }
  mpwos_ctx* ctx = new mpwos_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return MPWOS_ECUDA;
  }
  ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own;
  *out = ctx;
  return MPWOS_OK;
}

int mpwos_manifold_create(mpwos_ctx* ctx, const mpwos_manifold_desc* desc, mpwos_manifold** out) {
  if (!ctx || !out) return MPWOS_EINVAL;
  *out = nullptr;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  if (!desc) return fail(ctx, MPWOS_EINVAL, "null manifold description");
  int rc = validate_manifold(ctx, desc);
  if (rc) return rc;
  std::unique_ptr<mpwos_manifold> mh(new mpwos_manifold());
  mh->device = ctx->device;
  mh->desc = *desc;
  mh->desc.Q = mh->desc.b = mh->desc.cloud = nullptr;
  const int n = desc->n, D = desc->d + 1;
  auto upload = [&](void** dst, const void* src, size_t bytes) -> int {
    if (cudaMalloc(dst, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, MPWOS_ENOMEM, "manifold data (%zu bytes)", bytes);
    }
    CK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return MPWOS_OK;
  };
  if (desc->kind == MPWOS_EMBEDDED_SPHERE) {
    mh->Q.assign(desc->Q, desc->Q + static_cast<size_t>(n) * D);
    mh->b.assign(desc->b, desc->b + n);
    mh->desc.Q = mh->Q.data();
    mh->desc.b = mh->b.data();
    // Q^T, D rows of stride npad = n rounded up to 4 (zero padded: 16-byte row
    // slices); the FP32 copy in the warp walk's group order: rows of 1024, the
    // 16-byte slice c of component group G = lane + 32 s at 512 s + 128 c + 4 lane,
    // so that a warp's loads of one slice are contiguous
    const int npad = (n + 3) & ~3;
    std::vector<double> qt(static_cast<size_t>(D) * npad, 0.0);
    std::vector<float> qtf(static_cast<size_t>(D) * 1024, 0.0f);
    for (int i = 0; i < n; ++i) {
      const int G = i >> 4, lane = G & 31, sg = G >> 5, c = (i >> 2) & 3, e = i & 3;
      const size_t pos = static_cast<size_t>(512 * sg + 128 * c + 4 * lane + e);
      for (int j = 0; j < D; ++j) {
        qt[static_cast<size_t>(j) * npad + i] = mh->Q[static_cast<size_t>(i) * D + j];
        qtf[static_cast<size_t>(j) * 1024 + pos] = static_cast<float>(mh->Q[static_cast<size_t>(i) * D + j]);
      }
    }
    std::vector<uint16_t> img;
    tc_bimage(mh->Q.data(), n, D, img);
    if ((rc = upload(reinterpret_cast<void**>(&mh->qt), qt.data(), qt.size() * sizeof(double))) ||
        (rc = upload(reinterpret_cast<void**>(&mh->qtf), qtf.data(), qtf.size() * sizeof(float))) ||
        (rc = upload(reinterpret_cast<void**>(&mh->bd), mh->b.data(), mh->b.size() * sizeof(double))) ||
        (rc = upload(reinterpret_cast<void**>(&mh->tc_img), img.data(), img.size() * sizeof(uint16_t)))) {
      mpwos_manifold_destroy(mh.release());
      return rc;
    }
  }
  if (desc->kind == MPWOS_POINT_CLOUD) {
    mh->cloud.assign(desc->cloud, desc->cloud + 3 * desc->n_cloud);
    mh->desc.cloud = mh->cloud.data();
    rc = build_cloud(ctx, &mh->desc, mh->grid);
    if (rc) {
      free_cloud(mh->grid);
      mpwos_manifold_destroy(mh.release());
      return rc;
    }
    mh->has_grid = true;
  }
  if (desc->kind == MPWOS_REVOLUTION) {
    // rho_geo = c_kappa / (1 + kappa(y)) varies: its largest value comes from the
    // smallest curvature indicator, found on a dense scan of the profile
    double kmin = INFINITY;
    const double lim = desc->prof_kappa * (1.0 - 1e-6);
    for (int j = 0; j <= 20000; ++j) {
      const double t = -lim + 2.0 * lim * j / 20000.0;
      kmin = std::min(kmin, rev_kappa<double>(rev_profile<double>(t, desc->prof_alpha, desc->prof_kappa)));
    }
    mh->rev_kmin = kmin;
  }
  *out = mh.release();
  return MPWOS_OK;
}

void mpwos_manifold_destroy(mpwos_manifold* mh) {
  if (!mh) return;
  cudaSetDevice(mh->device);
  cudaFree(mh->qt);
  cudaFree(mh->qtf);
  cudaFree(mh->bd);
  cudaFree(mh->tc_img);
  if (mh->has_grid) free_cloud(mh->grid);
  delete mh;
}

void mpwos_destroy(mpwos_ctx* ctx) {
  if (!ctx) return;
  serve_shutdown(ctx);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->tables) {
    cudaFree(kv.second.tab64);
    cudaFree(kv.second.tabc);
  }
  if (ctx->own) cudaStreamDestroy(ctx->own);
  delete ctx;
}

const char* mpwos_last_error(const mpwos_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int mpwos_set_stream(mpwos_ctx* ctx, void* stream) {
  if (!ctx) return MPWOS_EINVAL;
  ctx->stream = stream ? static_cast<cudaStream_t>(stream) : ctx->own;
  return MPWOS_OK;
}

int64_t mpwos_launch_count(const mpwos_ctx* ctx) { return ctx ? ctx->launches : 0; }

int mpwos_walk_scores(mpwos_ctx* ctx, const mpwos_manifold* mh, const mpwos_problem* prob,
                      const mpwos_params* prm, const double* pts, int64_t P, int64_t N, double* S, int32_t* K,
                      int32_t* flags) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  int rc = validate(ctx, m, prob, prm, P, N);
  if (rc) return rc;
  if (!S || !K || !flags) return fail(ctx, MPWOS_EINVAL, "null output");
  Scratch sc(ctx);
  DevProblem pb;
  rc = prepare(ctx, sc, mh, prob, prm, pts, P, N, pb);
  if (rc) return rc;
  const size_t W = static_cast<size_t>(P) * N;
  const bool dS = is_device_ptr(S), dK = is_device_ptr(K), dF = is_device_ptr(flags);
  pb.S_out = dS ? S : sc.alloc<double>(W);
  pb.K_out = dK ? K : sc.alloc<int32_t>(W);
  pb.flag_out = dF ? flags : sc.alloc<int32_t>(W);
  if (!pb.S_out || !pb.K_out || !pb.flag_out) return fail(ctx, MPWOS_ENOMEM, "per-walk outputs (%zu walks)", W);
  rc = run_walks_tuned(ctx, pb, prm->precision == MPWOS_FP64);
  if (rc) return rc;
  if (!dS) CK(cudaMemcpyAsync(S, pb.S_out, W * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (!dK) CK(cudaMemcpyAsync(K, pb.K_out, W * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  if (!dF) CK(cudaMemcpyAsync(flags, pb.flag_out, W * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  unsigned tcst = 0;
  if (pb.dev_status) CK(cudaMemcpyAsync(&tcst, pb.dev_status, sizeof tcst, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (tcst) return fail(ctx, MPWOS_ETIMEDOUT, "tensor-core walk: a bounded mbarrier wait ran out (status %u)", tcst);
  return MPWOS_OK;
}

int mpwos_solve(mpwos_ctx* ctx, const mpwos_manifold* mh, const mpwos_problem* prob, const mpwos_params* prm,
                const double* pts, int64_t P, int64_t N, double* mean, double* stderr_, double* mean_steps) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  int rc = validate(ctx, m, prob, prm, P, N);
  if (rc) return rc;
  if (!mean || !stderr_ || !mean_steps) return fail(ctx, MPWOS_EINVAL, "null output");
  Scratch sc(ctx);
  DevProblem pb;
  rc = prepare(ctx, sc, mh, prob, prm, pts, P, N, pb);
  if (rc) return rc;
  const size_t W = static_cast<size_t>(P) * N;
  pb.S_out = sc.alloc<double>(W);
  pb.K_out = sc.alloc<int32_t>(W);
  pb.flag_out = sc.alloc<int32_t>(W);
  unsigned long long* nflag = sc.alloc<unsigned long long>(1);
  const bool dm = is_device_ptr(mean), ds = is_device_ptr(stderr_), dt = is_device_ptr(mean_steps);
  double* om = dm ? mean : sc.alloc<double>(P);
  double* os = ds ? stderr_ : sc.alloc<double>(P);
  double* ot = dt ? mean_steps : sc.alloc<double>(P);
  if (!pb.S_out || !pb.K_out || !pb.flag_out || !nflag || !om || !os || !ot)
    return fail(ctx, MPWOS_ENOMEM, "scratch for %zu walks", W);
  CK(cudaMemsetAsync(nflag, 0, sizeof(unsigned long long), ctx->stream));
  rc = run_walks_tuned(ctx, pb, prm->precision == MPWOS_FP64);
  if (rc) return rc;
  if (P) {
    CK(launch_reduce(pb.S_out, pb.K_out, pb.flag_out, P, N, om, os, ot, nflag, ctx->stream));
    ctx->launches++;
  }
  unsigned long long hflag = 0;
  CK(cudaMemcpyAsync(&hflag, nflag, sizeof hflag, cudaMemcpyDeviceToHost, ctx->stream));
  if (!dm) CK(cudaMemcpyAsync(mean, om, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (!ds) CK(cudaMemcpyAsync(stderr_, os, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  if (!dt) CK(cudaMemcpyAsync(mean_steps, ot, P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  unsigned tcst = 0;
  if (pb.dev_status) CK(cudaMemcpyAsync(&tcst, pb.dev_status, sizeof tcst, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (tcst) return fail(ctx, MPWOS_ETIMEDOUT, "tensor-core walk: a bounded mbarrier wait ran out (status %u)", tcst);
  if (hflag) return fail(ctx, MPWOS_EMAXSTEPS, "%llu walks reached max_steps", hflag);
  return MPWOS_OK;
}

int mpwos_solve_partial(mpwos_ctx* ctx, const mpwos_manifold* mh, const mpwos_problem* prob,
                        const mpwos_params* prm, const double* pts, int64_t P, int64_t N, int64_t i0, int64_t i1,
                        double* part) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  int rc = validate(ctx, m, prob, prm, P, N);
  if (rc) return rc;
  if (i0 < 0 || i1 > N || i0 > i1 || i0 % kEstBlock != 0 || (i1 % kEstBlock != 0 && i1 != N))
    return fail(ctx, MPWOS_EINVAL, "walk range [%lld, %lld) of %lld: both ends must be multiples of %lld (or the end N)",
                (long long)i0, (long long)i1, (long long)N, (long long)kEstBlock);
  if (!part && P > 0 && i1 > i0) return fail(ctx, MPWOS_EINVAL, "null output");
  const int64_t nr = i1 - i0;
  if (P == 0 || nr == 0) return MPWOS_OK;
  Scratch sc(ctx);
  DevProblem pb;
  rc = prepare(ctx, sc, mh, prob, prm, pts, P, N, pb);
  if (rc) return rc;
  pb.wk_i0 = i0;
  pb.wk_i1 = i1;
  pb.wk_w0 = 0;
  pb.wk_w1 = P * nr;
  pb.out_stride = nr;
  pb.out_i0 = i0;
  const size_t W = static_cast<size_t>(P) * nr;
  const size_t nrec = static_cast<size_t>(P) * ((nr + kEstBlock - 1) / kEstBlock) * kEstFields;
  pb.S_out = sc.alloc<double>(W);
  pb.K_out = sc.alloc<int32_t>(W);
  pb.flag_out = sc.alloc<int32_t>(W);
  const bool dp = is_device_ptr(part);
  double* op = dp ? part : sc.alloc<double>(nrec);
  if (!pb.S_out || !pb.K_out || !pb.flag_out || !op) return fail(ctx, MPWOS_ENOMEM, "scratch for %zu walks", W);
  rc = run_walks(ctx, pb, prm->precision == MPWOS_FP64);
  if (rc) return rc;
  CK(launch_reduce_blocks(pb.S_out, pb.K_out, pb.flag_out, P, nr, op, ctx->stream));
  ctx->launches++;
  if (!dp) CK(cudaMemcpyAsync(part, op, nrec * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  unsigned tcst = 0;
  if (pb.dev_status) CK(cudaMemcpyAsync(&tcst, pb.dev_status, sizeof tcst, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (tcst) return fail(ctx, MPWOS_ETIMEDOUT, "tensor-core walk: a bounded mbarrier wait ran out (status %u)", tcst);
  return MPWOS_OK;
}

int mpwos_fit_torus_series(const double* pts, const double* u, int64_t P, double R, int max_m, int max_q,
                           double* coef, int* modes, int* n_terms) {
  if (!pts || !u || !coef || !modes || !n_terms || max_m < 0 || max_q < 0 || !(R > 0.0)) return MPWOS_EINVAL;
  // the basis T(m theta) P(q phi), T, P in {cos, sin}, without sin(0 .), m outer, q inner
  std::vector<std::array<int, 4>> basis;
  for (int m = 0; m <= max_m; ++m)
    for (int tk = 0; tk < (m == 0 ? 1 : 2); ++tk)
      for (int q = 0; q <= max_q; ++q)
        for (int pk = 0; pk < (q == 0 ? 1 : 2); ++pk) basis.push_back({m, q, tk, pk});
  const int nb = static_cast<int>(basis.size());
  if (nb > kMaxPredTerms || P < nb) return MPWOS_EINVAL;
  // A (P x nb, column-major) at the points' angles: phi the azimuth, theta the
  // angle in the tube's meridian plane (the parametrisation of Example 1)
  std::vector<double> A(static_cast<size_t>(P) * nb), b(u, u + P);
  for (int64_t i = 0; i < P; ++i) {
    const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    const double ph = std::atan2(y, x), th = std::atan2(z, std::hypot(x, y) - R);
    for (int c = 0; c < nb; ++c) {
      const auto& bs = basis[c];
      const double tv = bs[2] ? std::sin(bs[0] * th) : std::cos(bs[0] * th);
      const double pv = bs[3] ? std::sin(bs[1] * ph) : std::cos(bs[1] * ph);
      A[static_cast<size_t>(c) * P + i] = tv * pv;
    }
  }
  // least squares by Householder QR: A = QR, then R c = (Q^T b)[0 .. nb)
  for (int k = 0; k < nb; ++k) {
    double* ak = A.data() + static_cast<size_t>(k) * P;
    double nrm = 0.0;
    for (int64_t i = k; i < P; ++i) nrm += ak[i] * ak[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0)) return MPWOS_EINVAL;   // rank deficient: too few distinct points
    const double alpha = ak[k] > 0.0 ? -nrm : nrm;
    std::vector<double> v(ak + k, ak + P);
    v[0] -= alpha;
    double vv = 0.0;
    for (double t : v) vv += t * t;
    auto reflect = [&](double* col) {
      double d = 0.0;
      for (int64_t i = k; i < P; ++i) d += v[i - k] * col[i];
      const double f = 2.0 * d / vv;
      for (int64_t i = k; i < P; ++i) col[i] -= f * v[i - k];
    };
    for (int c = k; c < nb; ++c) reflect(A.data() + static_cast<size_t>(c) * P);
    reflect(b.data());
  }
  for (int k = nb - 1; k >= 0; --k) {
    double t = b[k];
    for (int c = k + 1; c < nb; ++c) t -= A[static_cast<size_t>(c) * P + k] * coef[c];
    coef[k] = t / A[static_cast<size_t>(k) * P + k];
  }
  for (int c = 0; c < nb; ++c)
    for (int j = 0; j < 4; ++j) modes[4 * c + j] = basis[c][j];
  *n_terms = nb;
  return MPWOS_OK;
}

int mpwos_block_partials_host(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                              double* part) {
  if (P < 0 || N < 0 || ((!S || !K || !flags || !part) && P > 0 && N > 0)) return MPWOS_EINVAL;
  const int64_t nblk = (N + kEstBlock - 1) / kEstBlock;
  for (int64_t p = 0; p < P; ++p)
    for (int64_t b = 0; b < nblk; ++b) {
      const int64_t base = b * kEstBlock;
      const int64_t nb = std::min(kEstBlock, N - base);
      Stat st[32];
      long long ks = 0, nf = 0;
      for (int l = 0; l < 32; ++l) {
        const int cnt = lane_count(nb, l);
        st[l] = stat_lane(S + p * N + base + l, cnt);
        for (int t = 0; t < cnt; ++t) {
          ks += K[p * N + base + l + 32 * t];
          nf += flags[p * N + base + l + 32 * t];
        }
      }
      for (int off = 16; off > 0; off >>= 1)
        for (int l = 0; l < off; ++l) st[l] = stat_merge(st[l], st[l + off]);
      double* rec = part + (p * nblk + b) * kEstFields;
      rec[0] = st[0].n; rec[1] = st[0].m; rec[2] = st[0].M;
      rec[3] = static_cast<double>(ks); rec[4] = static_cast<double>(nf);
    }
  return MPWOS_OK;
}

int mpwos_merge_partials(const double* const* parts, const int64_t* nblk, int nparts, int64_t P, double* mean,
                         double* stderr_, double* mean_steps, int64_t* n_flagged) {
  if (nparts < 0 || P < 0 || (P > 0 && (!mean || !stderr_ || !mean_steps)) || (nparts > 0 && (!parts || !nblk)))
    return MPWOS_EINVAL;
  for (int r = 0; r < nparts; ++r)
    if (nblk[r] < 0 || (nblk[r] > 0 && P > 0 && !parts[r])) return MPWOS_EINVAL;
  long long flagged = 0;
  for (int64_t p = 0; p < P; ++p) {
    Stat acc{0.0, 0.0, 0.0};
    long long ks = 0;
    for (int r = 0; r < nparts; ++r)
      for (int64_t b = 0; b < nblk[r]; ++b) {
        const double* rec = parts[r] + (p * nblk[r] + b) * kEstFields;
        acc = stat_merge(acc, Stat{rec[0], rec[1], rec[2]});
        ks += static_cast<long long>(rec[3]);
        flagged += static_cast<long long>(rec[4]);
      }
    double mu, se;
    stat_finish(acc, mu, se);
    mean[p] = mu;
    stderr_[p] = se;
    mean_steps[p] = acc.n > 0.0 ? static_cast<double>(ks) / acc.n : 0.0;
  }
  if (n_flagged) *n_flagged = flagged;
  return flagged ? MPWOS_EMAXSTEPS : MPWOS_OK;
}

int mpwos_tc_project(mpwos_ctx* ctx, const double* Q, int n, int D, const float* G, int64_t rows, float* out,
                     float* gg) {
  if (!ctx || !Q || !G || !out || !gg || rows < 0 || n < 1 || n > 1024 || D < 1 || D > 31) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Scratch sc(ctx);
  std::vector<uint16_t> img;
  tc_bimage(Q, n, D, img);
  const uint4* dimg = reinterpret_cast<const uint4*>(sc.upload(img.data(), img.size()));
  const float* dG = sc.upload(G, static_cast<size_t>(rows) * n);
  float* dout = sc.alloc<float>(static_cast<size_t>(rows) * 32);
  float* dgg = sc.alloc<float>(static_cast<size_t>(rows));
  unsigned* dst = sc.alloc<unsigned>(1);
  if (!dimg || !dG || !dout || !dgg || !dst) return fail(ctx, MPWOS_ENOMEM, "tc_project buffers");
  CK(cudaMemsetAsync(dst, 0, sizeof(unsigned), ctx->stream));
  if (rows) {
    const int64_t tiles = (rows + 127) / 128;
    const int grid = static_cast<int>(std::min<int64_t>(tiles, ctx->sm_count));
    CK(launch_tc_project(dimg, dG, rows, n, dout, dgg, dst, grid, ctx->stream));
    ctx->launches++;
    CK(cudaMemcpy2DAsync(out, sizeof(float) * D, dout, sizeof(float) * 32, sizeof(float) * D, rows,
                         cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(gg, dgg, sizeof(float) * rows, cudaMemcpyDeviceToHost, ctx->stream));
  }
  unsigned hst = 0;
  CK(cudaMemcpyAsync(&hst, dst, sizeof hst, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hst) return fail(ctx, MPWOS_ETIMEDOUT, "tensor-core projection: a bounded mbarrier wait ran out");
  return MPWOS_OK;
}

int mpwos_philox(mpwos_ctx* ctx, const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out, int64_t count) {
  if (!ctx || !ctr || !out || count < 0) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Scratch sc(ctx);
  uint32_t* dc = sc.upload(ctr, static_cast<size_t>(count) * 4);
  uint32_t* dout = sc.alloc<uint32_t>(static_cast<size_t>(count) * 4);
  if (!dc || !dout) return fail(ctx, MPWOS_ENOMEM, "philox buffers");
  if (count) {
    CK(launch_philox(dc, key0, key1, dout, count, ctx->stream));
    ctx->launches++;
  }
  CK(cudaMemcpyAsync(out, dout, static_cast<size_t>(count) * 16, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MPWOS_OK;
}

int mpwos_green_radius(mpwos_ctx* ctx, int n, double a_max, const double* a, const double* U, double* t,
                       int64_t count, int precision) {
  if (!ctx || !a || !U || !t || count < 0 || n < 3 || n > 1024 || !(a_max > 0.0)) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  if (n > 3 && 0.25 * a_max * a_max > 0.25 * (n - 2)) return fail(ctx, MPWOS_EINVAL, "a_max outside the series range");
  CK(cudaSetDevice(ctx->device));
  Table* tab = nullptr;
  int rc = get_table(ctx, n, false, 0.25 * a_max * a_max, &tab);
  if (rc) return rc;
  Scratch sc(ctx);
  double* da = sc.upload(a, count);
  double* dU = sc.upload(U, count);
  double* dt = sc.alloc<double>(count);
  if (!da || !dU || !dt) return fail(ctx, MPWOS_ENOMEM, "radius buffers");
  if (count) {
    if (precision == MPWOS_FP64)
      CK(launch_green_radius64(n, da, dU, dt, count, tab->tab64, tab->NA, tab->NS, tab->z_max, ctx->stream));
    else
      CK(launch_green_radius32(da, dU, dt, count, tab->tabc, tab->NA, tab->NS, tab->z_max, ctx->stream));
    ctx->launches++;
  }
  CK(cudaMemcpyAsync(t, dt, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MPWOS_OK;
}

int mpwos_c_sigma_r(mpwos_ctx* ctx, int n, const double* a, double* c, int64_t count) {
  if (!ctx || !a || !c || count < 0 || n < 3) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  Scratch sc(ctx);
  double* da = sc.upload(a, count);
  double* dc = sc.alloc<double>(count);
  if (!da || !dc) return fail(ctx, MPWOS_ENOMEM, "c buffers");
  if (count) {
    CK(launch_c_sigma_r(n, da, dc, count, ctx->stream));
    ctx->launches++;
  }
  CK(cudaMemcpyAsync(c, dc, count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return MPWOS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of mpwos_solve.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by another allocator (a framework's caching pool that has
// reserved the free memory), or a latency-critical request loop where an
// allocation — which may synchronize the device — is not allowed.  For them
// mpwos_solve_noalloc runs the same walk and reduction kernels with all of
// their scratch (per-walk scores, stopping indices and flags, the radius
// tables, the boundary normal, the max-steps counter) carved out of one
// file-scope device array of fixed size.  Every GPU that loads the library
// holds this array until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = size_t(32) << 20;   // 32 MiB per device
constexpr size_t kNaHeader = 256;                      // max-steps counter
constexpr size_t kNaNormal = 8192 + 4096;              // boundary normal, n <= 1024 doubles + floats
constexpr size_t kNaQuad = 256;                        // SPHERE_QUAD v, A on S^2 (12 doubles)
constexpr size_t kNaOrder = 8192;                      // FP32 warp walk: coordinate order, dense normal (1024 each)
constexpr size_t kNaTab64 = 1068288;                   // 65 x 2 x 1027 doubles, rounded up to 256
constexpr size_t kNaTabc = 2129920;                    // 65 x 2 x 1024 float4 interval cubics
constexpr size_t kNaFixed = kNaHeader + kNaNormal + kNaQuad + kNaOrder + kNaTab64 + kNaTabc;
constexpr size_t kNaPerWalk = sizeof(double) + 2 * sizeof(int32_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};

// Device address of the scratch array on the current device (looked up once
// per device; host code may not use the symbol itself as a device address).
int noalloc_scratch(mpwos_ctx* ctx, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (ctx->device < 0 || ctx->device >= 256) return fail(ctx, MPWOS_EINVAL, "device index out of range");
  if (!g_noalloc_ptr[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(ctx, MPWOS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    }
    g_noalloc_ptr[ctx->device] = p;
  }
  *out = static_cast<unsigned char*>(g_noalloc_ptr[ctx->device]);
  return MPWOS_OK;
}

}  // namespace

extern "C" int64_t mpwos_noalloc_max_walks(void) {
  return static_cast<int64_t>((kNoAllocBytes - kNaFixed) / kNaPerWalk);
}

extern "C" int mpwos_solve_noalloc(mpwos_ctx* ctx, const mpwos_manifold* mh, const mpwos_problem* prob,
                                   const mpwos_params* prm, const double* pts, int64_t P, int64_t N, double* mean,
                                   double* stderr_, double* mean_steps) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  int rc = validate(ctx, m, prob, prm, P, N);
  if (rc) return rc;
  if (m->kind == MPWOS_EMBEDDED_SPHERE || m->kind == MPWOS_POINT_CLOUD || m->kind == MPWOS_REVOLUTION ||
      m->kind == MPWOS_CURVE_SPHERE)
    return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: EMBEDDED_SPHERE, POINT_CLOUD, REVOLUTION and CURVE_SPHERE are not supported (use mpwos_solve)");
  if (prm->sampler != MPWOS_SAMPLER_FULL)
    return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: the reduced sampler is not supported (use mpwos_solve)");
  if (prob->comp != MPWOS_COMP_NONE)
    return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: compensation is not supported (use mpwos_solve)");
  if (P > 0 && (!is_device_ptr_on(pts, ctx->device) || !is_device_ptr_on(mean, ctx->device) ||
                !is_device_ptr_on(stderr_, ctx->device) || !is_device_ptr_on(mean_steps, ctx->device)))
    return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: pts and the three outputs must be device pointers on device %d",
                ctx->device);
  const int64_t walks = P * N;
  if (walks > mpwos_noalloc_max_walks())
    return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: P*N = %lld walks exceeds the fixed scratch limit of %lld",
                (long long)walks, (long long)mpwos_noalloc_max_walks());
  unsigned char* base = nullptr;
  rc = noalloc_scratch(ctx, &base);
  if (rc) return rc;
  unsigned long long* nflag = reinterpret_cast<unsigned long long*>(base);
  unsigned char* cur = base + kNaHeader;
  double* e_dev = reinterpret_cast<double*>(cur);
  cur += kNaNormal;
  double* quad_dev = reinterpret_cast<double*>(cur);
  cur += kNaQuad;
  int* perm_dev = reinterpret_cast<int*>(cur);
  float* efw_dev = reinterpret_cast<float*>(cur + 4096);
  cur += kNaOrder;
  double* tab64 = reinterpret_cast<double*>(cur);
  cur += kNaTab64;
  float4* tabc = reinterpret_cast<float4*>(cur);
  cur += kNaTabc;
  double* S = reinterpret_cast<double*>(cur);
  int32_t* K = reinterpret_cast<int32_t*>(cur + walks * sizeof(double));
  int32_t* F = K + walks;

  DevProblem pb;
  std::memset(&pb, 0, sizeof pb);
  pb.mkind = m->kind;
  pb.n = m->n;
  pb.d = m->d;
  pb.R = m->R;
  pb.a_tube = m->a;
  pb.sigma = prob->sigma;
  pb.sqrt_sigma = std::sqrt(prob->sigma);
  pb.closed = prob->closed;
  pb.h = prob->bnd_offset;
  pb.eps = prm->eps;
  pb.tau_w = prm->tau_w;
  pb.theta = prm->theta;
  pb.c_kappa = prm->c_kappa;
  pb.kappa = kappa_of(m);
  pb.rho_geo = prm->c_kappa / (1.0 + pb.kappa);
  pb.n_v = prm->n_v;
  pb.max_steps = prm->max_steps;
  pb.seed = prm->seed;
  pb.keys = philox_keys(static_cast<uint32_t>(prm->seed), static_cast<uint32_t>(prm->seed >> 32));
  pb.P = P;
  pb.N = N;
  pb.wk_points = nullptr;
  pb.wk_np = P;
  pb.wk_i0 = 0;
  pb.wk_i1 = N;
  pb.wk_w0 = 0;
  pb.wk_w1 = P * N;
  pb.out_stride = N;
  pb.pts = pts;
  copy_func(prob->f, pb.f);
  if (!prob->closed) {
    copy_func(prob->g, pb.g);
    float ef_host[1024];
    for (int i = 0; i < m->n; ++i) ef_host[i] = static_cast<float>(prob->bnd_normal[i]);
    float* ef_dev = reinterpret_cast<float*>(e_dev + 1024);
    CK(cudaMemcpyAsync(e_dev, prob->bnd_normal, sizeof(double) * m->n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ef_dev, ef_host, sizeof(float) * m->n, cudaMemcpyHostToDevice, ctx->stream));
    pb.e = e_dev;
    pb.ef = ef_dev;
  }
  // SPHERE_QUAD data on S^2: v (3) then A (9)
  for (DevFunc* df : {&pb.f, &pb.g}) {
    const mpwos_func& hf = (df == &pb.f) ? prob->f : prob->g;
    if ((df == &pb.g && prob->closed) || hf.kind != MPWOS_FUNC_SPHERE_QUAD) continue;
    if (df == &pb.g && prob->f.kind == MPWOS_FUNC_SPHERE_QUAD)
      return fail(ctx, MPWOS_EINVAL, "mpwos_solve_noalloc: at most one SPHERE_QUAD function");
    CK(cudaMemcpyAsync(quad_dev, hf.v, 3 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(quad_dev + 3, hf.A, 9 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    df->v = quad_dev;
    df->A = quad_dev + 3;
  }
  // the FP32 warp walk's coordinate order
  if (uses_walk_order(m, prm)) {
    WalkOrder wo;
    walk_order(m, prob, pb, wo);
    CK(cudaMemcpyAsync(perm_dev, wo.perm.data(), sizeof(int) * wo.perm.size(), cudaMemcpyHostToDevice, ctx->stream));
    pb.perm = perm_dev;
    if (!wo.ef_w.empty()) {
      CK(cudaMemcpyAsync(efw_dev, wo.ef_w.data(), sizeof(float) * wo.ef_w.size(), cudaMemcpyHostToDevice, ctx->stream));
      pb.ef_w = efw_dev;
    }
  }
  // the radius table, rebuilt in the shared array on every call
  const double a_max = pb.sqrt_sigma * pb.theta * pb.rho_geo;
  const int n = m->n;
  if (n > 3 && 0.25 * a_max * a_max > 0.25 * (n - 2))
    return fail(ctx, MPWOS_EINVAL, "sigma (theta rho_geo)^2 / 4 = %g exceeds (n-2)/4: outside the series range",
                0.25 * a_max * a_max);
  pb.NS = kTableNS;
  pb.NA = prob->closed ? 1 : table_rows(n);
  pb.z_max = 0.25 * a_max * a_max;
  fill_em1_poly(pb, n, pb.z_max);
  CK(launch_build_table(n, pb.NA, pb.NS, pb.z_max, prob->closed ? a_max : 0.0, tab64, tabc, ctx->stream));
  ctx->launches += 1;
  pb.tab64 = tab64;
  pb.tabc = tabc;
  fill_scalars_f(pb);
  pb.S_out = S;
  pb.K_out = K;
  pb.flag_out = F;
  CK(cudaMemsetAsync(nflag, 0, sizeof(unsigned long long), ctx->stream));
  rc = run_walks(ctx, pb, prm->precision == MPWOS_FP64);
  if (rc) return rc;
  if (P) {
    CK(launch_reduce(S, K, F, P, N, mean, stderr_, mean_steps, nflag, ctx->stream));
    ctx->launches++;
  }
  unsigned long long hflag = 0;
  CK(cudaMemcpyAsync(&hflag, nflag, sizeof hflag, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hflag) return fail(ctx, MPWOS_EMAXSTEPS, "%llu walks reached max_steps", hflag);
  return MPWOS_OK;
}

// ---------------------------------------------------------------------------
// Request serving: continuous batching of solve requests.
//
// Requests are admitted while a stream slot and device memory are free; each
// runs on its own stream in rounds (all points get n0 walks, then points whose
// standard error is still above the target get their walk count doubled, up
// to the budget), and each round's walks are launched in bounded chunks with a
// capped grid so that requests in flight share the SMs.  A walk's result
// depends only on (seed, point, walk index), so a request's results do not
// depend on what else is in flight.  A host scheduler thread advances rounds
// and admits queued requests.
// ---------------------------------------------------------------------------
namespace {

struct OwnedFunc {
  mpwos_func f{};
  std::vector<double> coef, v, A;
  std::vector<int> off, var, pw, modes;
  void take(const mpwos_func& src, int D) {
    f = src;
    coef.assign(src.coef, src.coef + (src.coef ? src.n_terms : 0));
    f.coef = coef.data();
    if (src.kind == MPWOS_FUNC_POLY) {
      const int nf = src.n_terms ? src.term_off[src.n_terms] : 0;
      off.assign(src.term_off, src.term_off + (src.term_off ? src.n_terms + 1 : 0));
      var.assign(src.var, src.var + (src.var ? nf : 0));
      pw.assign(src.pw, src.pw + (src.pw ? nf : 0));
      f.term_off = off.data(); f.var = var.data(); f.pw = pw.data();
    } else if (src.kind == MPWOS_FUNC_TORUS_FOURIER) {
      modes.assign(src.modes, src.modes + (src.modes ? 4 * src.n_terms : 0));
      f.modes = modes.data();
    } else if (src.kind == MPWOS_FUNC_SPHERE_QUAD) {
      v.assign(src.v, src.v + D);
      A.assign(src.A, src.A + static_cast<size_t>(D) * D);
      f.v = v.data(); f.A = A.data();
    } else if (src.kind == MPWOS_FUNC_CURVE_SPHERE) {      // per term: modes, v (3), A (9)
      modes.assign(src.modes, src.modes + (src.modes ? 4 * src.n_terms : 0));
      v.assign(src.v, src.v + (src.v ? 3 * src.n_terms : 0));
      A.assign(src.A, src.A + (src.A ? 9 * src.n_terms : 0));
      f.modes = modes.data(); f.v = v.data(); f.A = A.data();
    } else if (src.kind == MPWOS_FUNC_REVOLUTION_QUAD) {   // D = n - 1: v and diag(A)
      v.assign(src.v, src.v + D);
      A.assign(src.A, src.A + D);
      f.v = v.data(); f.A = A.data();
    }
  }
};

struct Request {
  uint64_t id = 0;
  int state = 0;                 // 0 queued, 1 running, 2 done, 3 failed, 4 canceled
  int status = MPWOS_OK;
  std::string err;
  const mpwos_manifold* mh = nullptr;   // the caller's handle (kept alive by the caller)
  mpwos_problem prob{};
  mpwos_params prm{};
  OwnedFunc f, g, u_star;
  std::vector<double> normal, pts;
  int64_t P = 0, budget = 0;
  double target = 0.0;
  size_t bytes = 0;
  int slot = -1;
  std::unique_ptr<Scratch> sc;
  cudaEvent_t ev = nullptr;
  DevProblem pb{};
  double *S = nullptr, *mean = nullptr, *se = nullptr, *ms = nullptr;
  int32_t *K = nullptr, *F = nullptr;
  int64_t* nper = nullptr;
  int* act = nullptr;
  unsigned long long* nflag = nullptr;
  double *h_mean = nullptr, *h_se = nullptr, *h_ms = nullptr;
  int64_t* h_n = nullptr;
  int* h_act = nullptr;
  unsigned long long* h_flag = nullptr;
  void* hbuf = nullptr;   // the pinned host block the h_ arrays live in
  size_t hcls = 0;        // its size class in the engine's pool
  std::vector<int> active;
  int64_t cur = 0;
  bool cancel = false;
  std::chrono::steady_clock::time_point t_submit, t_done;
  // the round in flight: its walks go out in time-sized chunks, at most two
  // outstanding; the chunk events time them (walk cost per grid block)
  int64_t round_total = 0, round_issued = 0, round_i1 = 0;
  int inflight = 0;
  bool reducing = false;
  cudaEvent_t cev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  int64_t cwalks[2] = {0, 0}, cgrid[2] = {0, 0};
  int chead = 0;
  double block_ns_per_walk = 0.0;   // measured GPU ns per walk times the launch's blocks (0: unknown)
};

}  // namespace

// Pinned host blocks for the requests' results, kept by power-of-two size
// class and reused: cudaFreeHost (and often cudaMallocHost) synchronizes the
// whole device, which would make every finished request wait for the longest
// kernel in flight.
struct PinnedPool {
  std::map<size_t, std::vector<void*>> free_;
  void* get(size_t bytes, size_t* cls) {
    size_t c = 4096;
    while (c < bytes) c <<= 1;
    *cls = c;
    auto& v = free_[c];
    if (!v.empty()) {
      void* p = v.back();
      v.pop_back();
      return p;
    }
    void* p = nullptr;
    if (cudaMallocHost(&p, c) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, size_t cls) {
    if (p) free_[cls].push_back(p);
  }
  void release() {
    for (auto& kv : free_)
      for (void* p : kv.second) cudaFreeHost(p);
    free_.clear();
  }
};

struct ServeEngine {
  PinnedPool pinned;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::deque<uint64_t> queue;
  std::vector<cudaStream_t> streams;
  std::vector<bool> slot_busy;
  int max_active = 16;
  size_t mem_budget = 0, mem_used = 0;
  int64_t chunk_walks = int64_t(1) << 20;   // cap of a chunk
  double chunk_target_ms = 10.0;              // a chunk's aimed GPU time
  uint64_t next_id = 1;
  bool stop = false;
  std::condition_variable_any cv;
  std::thread thr;
};

namespace {

constexpr int64_t kFirstRoundWalks = 256;

void req_free_device(Request& r) {
  r.sc.reset();   // stream-ordered frees on the request's stream
}

void req_finish(mpwos_ctx* ctx, Request& r, int state, int status, const std::string& err) {
  ServeEngine& E = *ctx->serve;
  // a failed request may still have copies into its pinned block in flight:
  // drain its own stream before the block can go back to the pool
  if (state == 3 && r.slot >= 0) cudaStreamSynchronize(E.streams[r.slot]);
  r.state = state;
  r.status = status;
  r.err = err;
  r.t_done = std::chrono::steady_clock::now();
  req_free_device(r);
  if (r.slot >= 0) {
    E.slot_busy[r.slot] = false;
    r.slot = -1;
  }
  E.mem_used -= std::min(E.mem_used, r.bytes);
}

// Launch the next chunk of the round in flight (at most two outstanding).  A
// chunk aims at chunk_target_ms of GPU time at its launch's share of the grid
// (all requests in flight split the SMs), and holds at least one resident wave
// of walkers; the first chunk of a request, with no measurement yet, is one
// wave.
int req_issue(mpwos_ctx* ctx, Request& r) {
  ServeEngine& E = *ctx->serve;
  const cudaStream_t st = E.streams[r.slot];
  const bool fp64 = r.prm.precision == MPWOS_FP64;
  int running = 0;
  for (auto& kv : E.reqs) running += kv.second->state == 1;
  const int64_t max_grid = running > 1 ? -static_cast<int64_t>(running) : 0;
  const int block = tuned_block(ctx, r.pb, fp64);
  const LaunchShape sh = launch_shape(ctx, r.pb, fp64, max_grid, block);
  const int64_t grid = sh.grid;
  // never less than one resident wave: a chunk lasts at least its longest walk,
  // so fewer walks than the grid holds would not end sooner
  const int64_t wave = std::max<int64_t>(1, grid * sh.per_block);
  int64_t n = wave;
  if (r.block_ns_per_walk > 0.0) {
    const double want = E.chunk_target_ms * 1e6 * static_cast<double>(grid) / r.block_ns_per_walk;
    n = want >= static_cast<double>(E.chunk_walks) ? E.chunk_walks : std::max<int64_t>(wave, static_cast<int64_t>(want));
  }
  n = std::min<int64_t>(n, E.chunk_walks);
  n = std::min<int64_t>(n, r.round_total - r.round_issued);
  const int c = (r.chead + r.inflight) & 1;
  r.pb.wk_w0 = r.round_issued;
  r.pb.wk_w1 = r.round_issued + n;
  CK(cudaEventRecord(r.cev[c][0], st));
  int rc = launch_walks(ctx, r.pb, fp64, st, max_grid, block);
  if (rc) return rc;
  CK(cudaEventRecord(r.cev[c][1], st));
  r.cwalks[c] = n;
  r.cgrid[c] = grid;
  r.round_issued += n;
  r.inflight++;
  return MPWOS_OK;
}

// After the round's last chunk: the per-point reduction and its copies to the host.
int req_reduce(mpwos_ctx* ctx, Request& r) {
  ServeEngine& E = *ctx->serve;
  const cudaStream_t st = E.streams[r.slot];
  CK(cudaMemsetAsync(r.nflag, 0, sizeof(unsigned long long), st));
  CK(launch_reduce_strided(r.S, r.K, r.F, r.P, 0, r.budget, r.nper, r.mean, r.se, r.ms, r.nflag, st));
  ctx->launches++;
  CK(cudaMemcpyAsync(r.h_mean, r.mean, sizeof(double) * r.P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(r.h_se, r.se, sizeof(double) * r.P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(r.h_ms, r.ms, sizeof(double) * r.P, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(r.h_flag, r.nflag, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  if (r.pb.dev_status) CK(cudaMemcpyAsync(r.h_flag + 1, r.pb.dev_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaEventRecord(r.ev, st));
  r.reducing = true;
  r.cur = r.round_i1;
  return MPWOS_OK;
}

int req_round(mpwos_ctx* ctx, Request& r, int64_t i1) {
  ServeEngine& E = *ctx->serve;
  const cudaStream_t st = E.streams[r.slot];
  const int64_t i0 = r.cur;
  for (size_t q = 0; q < r.active.size(); ++q) {
    r.h_act[q] = r.active[q];
    r.h_n[r.active[q]] = i1;
  }
  CK(cudaMemcpyAsync(r.act, r.h_act, sizeof(int) * r.active.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(r.nper, r.h_n, sizeof(int64_t) * r.P, cudaMemcpyHostToDevice, st));
  r.pb.wk_points = r.act;
  r.pb.wk_np = static_cast<int64_t>(r.active.size());
  r.pb.wk_i0 = i0;
  r.pb.wk_i1 = i1;
  r.pb.out_stride = r.budget;
  r.round_total = r.pb.wk_np * (i1 - i0);
  r.round_issued = 0;
  r.round_i1 = i1;
  r.reducing = false;
  int rc = req_issue(ctx, r);
  if (!rc && r.round_issued < r.round_total) rc = req_issue(ctx, r);
  return rc;
}

// A chunk of the round in flight has finished: update the walk cost, keep two
// chunks outstanding, and reduce after the last.
int req_chunk_done(mpwos_ctx* ctx, Request& r) {
  const int c = r.chead;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, r.cev[c][0], r.cev[c][1]) == cudaSuccess && r.cwalks[c] > 0) {
    const double cost = 1e6 * static_cast<double>(ms) * static_cast<double>(r.cgrid[c]) / static_cast<double>(r.cwalks[c]);
    r.block_ns_per_walk = r.block_ns_per_walk > 0.0 ? 0.5 * (r.block_ns_per_walk + cost) : cost;
  }
  cudaGetLastError();
  r.chead ^= 1;
  r.inflight--;
  if (!r.cancel && r.round_issued < r.round_total) return req_issue(ctx, r);
  if (r.inflight == 0) return req_reduce(ctx, r);   // a canceled request stops here
  return MPWOS_OK;
}

int req_start(mpwos_ctx* ctx, Request& r) {
  ServeEngine& E = *ctx->serve;
  const cudaStream_t st = E.streams[r.slot];
  r.sc.reset(new Scratch(ctx, st));
  int rc = prepare(ctx, *r.sc, r.mh, &r.prob, &r.prm, r.pts.data(), r.P, r.budget, r.pb);
  if (rc) return rc;
  CK(cudaStreamSynchronize(ctx->stream));   // tables built on the context stream
  const size_t W = static_cast<size_t>(r.P) * r.budget;
  r.S = r.sc->alloc<double>(W);
  r.K = r.sc->alloc<int32_t>(W);
  r.F = r.sc->alloc<int32_t>(W);
  r.mean = r.sc->alloc<double>(r.P);
  r.se = r.sc->alloc<double>(r.P);
  r.ms = r.sc->alloc<double>(r.P);
  r.nper = r.sc->alloc<int64_t>(r.P);
  r.act = r.sc->alloc<int>(r.P);
  r.nflag = r.sc->alloc<unsigned long long>(1);
  if (!r.S || !r.K || !r.F || !r.mean || !r.se || !r.ms || !r.nper || !r.act || !r.nflag)
    return fail(ctx, MPWOS_ENOMEM, "request %llu: device memory", (unsigned long long)r.id);
  r.pb.S_out = r.S;
  r.pb.K_out = r.K;
  r.pb.flag_out = r.F;
  r.active.resize(r.P);
  for (int64_t p = 0; p < r.P; ++p) { r.active[p] = static_cast<int>(p); r.h_n[p] = 0; }
  r.cur = 0;
  for (auto& pair : r.cev)
    for (auto& e : pair)
      if (!e) CK(cudaEventCreate(&e));
  int64_t n0 = r.target > 0.0 ? std::min(r.budget, kFirstRoundWalks) : r.budget;
  if (r.target > 0.0 && r.pb.mkind != kPointCloud) {
    // a request whose whole budget fills at most a quarter of one resident wave
    // is bound by its walks' length, not by the GPU: one round of the full
    // budget ends no later than the first of the doubling rounds (not so on a
    // point cloud, whose cooperative search slows as a warp holds more walkers)
    const LaunchShape sh = launch_shape(ctx, r.pb, r.prm.precision == MPWOS_FP64, 0, 0);
    if (r.P * r.budget * 4 <= sh.grid * sh.per_block) n0 = r.budget;
  }
  return req_round(ctx, r, n0);
}

void req_advance(mpwos_ctx* ctx, Request& r) {
  if (r.cancel) {
    req_finish(ctx, r, 4, MPWOS_ECANCELED, "canceled");
    return;
  }
  if (r.h_flag[1]) {
    req_finish(ctx, r, 3, MPWOS_ETIMEDOUT, "tensor-core walk: a bounded mbarrier wait ran out");
    return;
  }
  std::vector<int> next;
  if (r.target > 0.0)
    for (int p : r.active)
      if (r.h_se[p] > r.target && r.h_n[p] < r.budget) next.push_back(p);
  if (next.empty()) {
    if (*r.h_flag) req_finish(ctx, r, 2, MPWOS_EMAXSTEPS, "some walks reached max_steps");
    else req_finish(ctx, r, 2, MPWOS_OK, "");
    return;
  }
  r.active.swap(next);
  const int rc = req_round(ctx, r, std::min(r.budget, 2 * r.cur));
  if (rc) req_finish(ctx, r, 3, rc, ctx->err);
}

void serve_admit(mpwos_ctx* ctx) {
  ServeEngine& E = *ctx->serve;
  while (!E.queue.empty()) {
    Request& r = *E.reqs[E.queue.front()];
    int active = 0, slot = -1;
    for (int q = 0; q < E.max_active; ++q) {
      if (E.slot_busy[q]) ++active;
      else if (slot < 0) slot = q;
    }
    if (slot < 0) return;
    if (E.mem_used + r.bytes > E.mem_budget) {
      if (active > 0) return;   // wait for memory; a lone oversized request fails below
      E.queue.pop_front();
      req_finish(ctx, r, 3, MPWOS_ENOMEM, "request exceeds the serving memory budget");
      continue;
    }
    E.queue.pop_front();
    E.slot_busy[slot] = true;
    r.slot = slot;
    r.state = 1;
    E.mem_used += r.bytes;
    const int rc = req_start(ctx, r);
    if (rc) req_finish(ctx, r, 3, rc, ctx->err);
  }
}

void serve_loop(mpwos_ctx* ctx) {
  cudaSetDevice(ctx->device);
  ServeEngine& E = *ctx->serve;
  std::unique_lock<std::recursive_mutex> lk(ctx->mu);
  while (!E.stop) {
    for (auto& kv : E.reqs) {
      Request& r = *kv.second;
      if (r.state != 1) continue;
      if (!r.reducing) {
        // chunks finish in order on the request's stream
        while (r.state == 1 && !r.reducing && r.inflight > 0) {
          const cudaError_t q = cudaEventQuery(r.cev[r.chead][1]);
          if (q == cudaErrorNotReady) break;
          if (q != cudaSuccess) {
            req_finish(ctx, r, 3, MPWOS_ECUDA, cudaGetErrorString(q));
            break;
          }
          const int rc = req_chunk_done(ctx, r);
          if (rc) req_finish(ctx, r, 3, rc, ctx->err);
        }
        continue;
      }
      const cudaError_t q = cudaEventQuery(r.ev);
      if (q == cudaSuccess) req_advance(ctx, r);
      else if (q != cudaErrorNotReady) req_finish(ctx, r, 3, MPWOS_ECUDA, cudaGetErrorString(q));
    }
    serve_admit(ctx);
    bool running = false;   // after admission: a request started just now must be polled
    for (auto& kv : E.reqs) running = running || kv.second->state == 1;
    if (!running && E.queue.empty()) {
      E.cv.wait_for(lk, std::chrono::milliseconds(100));
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

int serve_init(mpwos_ctx* ctx) {
  if (ctx->serve) return MPWOS_OK;
  ServeEngine* E = new ServeEngine();
  ctx->serve = E;
  size_t free_b = 0, total_b = 0;
  CK(cudaMemGetInfo(&free_b, &total_b));
  E->mem_budget = free_b / 4;
  E->streams.resize(E->max_active);
  E->slot_busy.assign(E->max_active, false);
  for (auto& st : E->streams) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  E->thr = std::thread(serve_loop, ctx);
  return MPWOS_OK;
}

Request* find_req(mpwos_ctx* ctx, uint64_t id) {
  if (!ctx->serve) return nullptr;
  auto it = ctx->serve->reqs.find(id);
  return it == ctx->serve->reqs.end() ? nullptr : it->second.get();
}

void req_release(mpwos_ctx* ctx, uint64_t id) {
  Request* r = find_req(ctx, id);
  if (!r) return;
  ctx->serve->pinned.put(r->hbuf, r->hcls);
  if (r->ev) cudaEventDestroy(r->ev);
  for (auto& pair : r->cev)
    for (auto& e : pair)
      if (e) cudaEventDestroy(e);
  ctx->serve->reqs.erase(id);
}

}  // namespace

void serve_shutdown(mpwos_ctx* ctx) {
  ServeEngine* E = ctx->serve;
  if (!E) return;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    E->stop = true;
  }
  E->cv.notify_all();
  if (E->thr.joinable()) E->thr.join();
  cudaSetDevice(ctx->device);
  for (auto& st : E->streams) cudaStreamSynchronize(st);
  std::vector<uint64_t> ids;
  for (auto& kv : E->reqs) ids.push_back(kv.first);
  for (uint64_t id : ids) {
    Request* r = find_req(ctx, id);
    if (r) req_free_device(*r);
    req_release(ctx, id);
  }
  for (auto& st : E->streams) cudaStreamDestroy(st);
  E->pinned.release();
  delete E;
  ctx->serve = nullptr;
}

extern "C" {

int mpwos_serve_config(mpwos_ctx* ctx, int max_active, size_t mem_bytes, int64_t chunk_walks) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  int rc = serve_init(ctx);
  if (rc) return rc;
  ServeEngine& E = *ctx->serve;
  bool idle = true;
  for (auto& kv : E.reqs) idle = idle && kv.second->state >= 2;
  if (max_active > 0) {
    if (!idle) return fail(ctx, MPWOS_EBUSY, "change max_active only while no request is queued or running");
    if (max_active > 64) return fail(ctx, MPWOS_EINVAL, "max_active must be <= 64");
    for (auto& st : E.streams) cudaStreamDestroy(st);
    E.max_active = max_active;
    E.streams.resize(max_active);
    E.slot_busy.assign(max_active, false);
    for (auto& st : E.streams) CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  }
  if (mem_bytes > 0) E.mem_budget = mem_bytes;
  if (chunk_walks > 0) E.chunk_walks = chunk_walks;
  return MPWOS_OK;
}

int mpwos_submit(mpwos_ctx* ctx, const mpwos_manifold* mh, const mpwos_problem* prob, const mpwos_params* prm,
                 const double* pts, int64_t P, int64_t walk_budget, double target_stderr, uint64_t* request_id) {
  if (!ctx || !request_id) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  CK(cudaSetDevice(ctx->device));
  const mpwos_manifold_desc* m = handle_desc(ctx, mh);
  if (!m) return MPWOS_EINVAL;
  int rc = validate(ctx, m, prob, prm, P, walk_budget);
  if (rc) return rc;
  if (P > 0 && (!pts || is_device_ptr(pts))) return fail(ctx, MPWOS_EINVAL, "mpwos_submit takes host query points");
  if (!(target_stderr >= 0.0)) return fail(ctx, MPWOS_EINVAL, "target_stderr must be >= 0");
  rc = serve_init(ctx);
  if (rc) return rc;
  ServeEngine& E = *ctx->serve;
  std::unique_ptr<Request> r(new Request());
  r->id = E.next_id++;
  r->P = P;
  r->budget = walk_budget;
  r->target = target_stderr;
  r->mh = mh;
  r->prob = *prob;
  r->prm = *prm;
  const int D = (m->kind == MPWOS_SPHERE && m->n == 3) ? 3 : (m->kind == MPWOS_REVOLUTION ? m->n - 1 : m->d + 1);
  r->f.take(prob->f, D);
  r->prob.f = r->f.f;
  if (!prob->closed) {
    r->g.take(prob->g, D);
    r->prob.g = r->g.f;
    r->normal.assign(prob->bnd_normal, prob->bnd_normal + m->n);
    r->prob.bnd_normal = r->normal.data();
  }
  if (prob->comp != MPWOS_COMP_NONE) {
    r->u_star.take(prob->u_star, D);
    r->prob.u_star = r->u_star.f;
  }
  r->pts.assign(pts, pts + static_cast<size_t>(P) * m->n);
  r->bytes = static_cast<size_t>(P) * walk_budget * 16 + static_cast<size_t>(P) * 48 + (64 << 10);
  CK(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
  {   // one pinned block: mean, se, mean K, walk counts (8 B each per point), two
      // flag words ([0] flagged walks, [1] kernel status), active points (4 B)
    const size_t Pn = static_cast<size_t>(std::max<int64_t>(P, 1));
    r->hbuf = E.pinned.get(Pn * 32 + 16 + Pn * 4, &r->hcls);
    if (!r->hbuf) {
      cudaEventDestroy(r->ev);
      return fail(ctx, MPWOS_ENOMEM, "pinned host memory for the request's results");
    }
    double* h = static_cast<double*>(r->hbuf);
    r->h_mean = h;
    r->h_se = h + Pn;
    r->h_ms = h + 2 * Pn;
    r->h_n = reinterpret_cast<int64_t*>(h + 3 * Pn);
    r->h_flag = reinterpret_cast<unsigned long long*>(h + 4 * Pn);
    r->h_act = reinterpret_cast<int*>(h + 4 * Pn + 2);
  }
  r->h_flag[0] = 0;
  r->h_flag[1] = 0;
  r->t_submit = std::chrono::steady_clock::now();
  const uint64_t id = r->id;
  if (P == 0) {
    r->state = 2;
    r->t_done = r->t_submit;
  } else {
    E.queue.push_back(id);
  }
  E.reqs[id] = std::move(r);
  *request_id = id;
  E.cv.notify_all();
  return MPWOS_OK;
}

int mpwos_poll(mpwos_ctx* ctx, uint64_t id, int* state) {
  if (!ctx || !state) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  Request* r = find_req(ctx, id);
  if (!r) return fail(ctx, MPWOS_ENOTFOUND, "unknown request %llu", (unsigned long long)id);
  *state = r->state;
  return MPWOS_OK;
}

int mpwos_wait(mpwos_ctx* ctx, uint64_t id, double timeout_s) {
  if (!ctx) return MPWOS_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
      Request* r = find_req(ctx, id);
      if (!r) return fail(ctx, MPWOS_ENOTFOUND, "unknown request %llu", (unsigned long long)id);
      if (r->state >= 2) return MPWOS_OK;
    }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_s >= 0.0 && el > timeout_s) {
      std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
      return fail(ctx, MPWOS_ETIMEDOUT, "request %llu not finished after %.3f s", (unsigned long long)id, el);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int mpwos_cancel(mpwos_ctx* ctx, uint64_t id) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  Request* r = find_req(ctx, id);
  if (!r) return fail(ctx, MPWOS_ENOTFOUND, "unknown request %llu", (unsigned long long)id);
  if (r->state == 0) {
    auto& q = ctx->serve->queue;
    for (auto it = q.begin(); it != q.end(); ++it)
      if (*it == id) { q.erase(it); break; }
    r->state = 4;
    r->status = MPWOS_ECANCELED;
    r->t_done = std::chrono::steady_clock::now();
  } else if (r->state == 1) {
    r->cancel = true;
  }
  return MPWOS_OK;
}

int mpwos_fetch(mpwos_ctx* ctx, uint64_t id, double* mean, double* stderr_, double* mean_steps,
                int64_t* walks, double* latency_s) {
  if (!ctx) return MPWOS_EINVAL;
  std::lock_guard<std::recursive_mutex> lock_(ctx->mu);
  Request* r = find_req(ctx, id);
  if (!r) return fail(ctx, MPWOS_ENOTFOUND, "unknown request %llu", (unsigned long long)id);
  if (r->state < 2) return fail(ctx, MPWOS_EBUSY, "request %llu has not finished", (unsigned long long)id);
  const int status = r->status;
  if (status != MPWOS_OK) fail(ctx, status, "request %llu: %s", (unsigned long long)id, r->err.c_str());
  if (r->state == 2) {
    for (int64_t p = 0; p < r->P; ++p) {
      if (mean) mean[p] = r->h_mean[p];
      if (stderr_) stderr_[p] = r->h_se[p];
      if (mean_steps) mean_steps[p] = r->h_ms[p];
      if (walks) walks[p] = r->h_n[p];
    }
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  req_release(ctx, id);
  return status;
}

}  // extern "C"
