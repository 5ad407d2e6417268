// walkr.cuh — the walk with the dimension-reduced exact sampler, one thread
// per walker, on spheres S^{n-1} and R^n (POLY data) and embedded spheres.
//
// A direction's n Gaussians g enter a step only through
//   - the coordinates T that f, g and the boundary normal read (sphere, R^n),
//     or the intrinsic Q^T g (embedded sphere, T = its d + 1 coordinates);
//   - on a sphere, the component h of g along Y's part outside T;
//   - |g|^2.
// For g ~ N(0, I_n) these are independent: N(0, 1) each, and the remainder of
// |g|^2 is chi^2 with n - |T| (R^n, embedded) or n - |T| - 1 (sphere) degrees
// of freedom, so the walk keeps y_T (and rho = |Y_rest| on a sphere) and draws
// |T| (+1) normals and one chi^2 per direction: O(|T|) work per step instead
// of O(n), with the same law of the walk (an exact reformulation; the paper
// draws full directions).
//
// Draws of vector v (0: Theta, 1 + l: Z_l) at step k of walk (p, i), Philox
// counter (j, k, i, p):
//   FP64 (identical to the CPU oracle): normals from blocks 64 v + b, two per
//     block (Box-Muller of u53 pairs), on a sphere the first one being the
//     component along Y's rest, then T's; chi^2 attempt a at blocks 64 v + 32 + 2a
//     (normal) and 64 v + 33 + 2a (U = u53 of words 0, 1); U_l at block
//     64 (1 + N_V) + l, u53 of words 0, 1.
//   FP32: Philox4x32-10 at counter (k, j, i, p) instead (the hoisted form of
//     the other FP32 walks); normals four per block j = 64 v + b (u23 words);
//     chi^2 attempt a at block 64 v + 32 + a (normal from words 0, 1, U from
//     word 2); U_l = word 3 of block 64 (1 + l) + 32 (the first chi^2 block of
//     Z_l, drawn anyway).
// chi^2_m: 0 (m = 0), x^2 (m = 1), else 2 Gamma(m/2) by Marsaglia-Tsang
// (ACM TOMS 26, 2000) with the exact log acceptance test, at most 16 attempts.
#pragma once
#include "dev_common.cuh"
#include "geom3.cuh"
#include "green.cuh"
#include "walkn.cuh"

namespace mpwos {

constexpr int kChi2Attempts = 16;

// ng normals (ng <= NG) of the stream at block j0.
template <int NG>
__device__ __forceinline__ void red_normals(const PhiloxKeys& K, uint32_t j0, uint32_t kk, uint32_t i, uint32_t p,
                                            int ng, double (&g)[NG]) {
#pragma unroll
  for (int b = 0; b < (NG + 1) / 2; ++b) {
    if (2 * b < ng) {
      const U4 r = philox4x32_10(j0 + static_cast<uint32_t>(b), kk, i, p, K);
      double g0, g1;
      box_muller64(u53(r.x, r.y), u53(r.z, r.w), g0, g1);
      g[2 * b] = g0;
      if (2 * b + 1 < NG) g[2 * b + 1] = (2 * b + 1 < ng) ? g1 : 0.0;
    } else {
      g[2 * b] = 0.0;
      if (2 * b + 1 < NG) g[2 * b + 1] = 0.0;
    }
  }
}
// The FP32 walk's blocks: Philox4x32-10 at counter (k, j, i, p) with the
// per-walk and per-step parts of its first rounds computed once (the form of
// the other FP32 walks).
struct RedStream32 {
  uint32_t A0;
  Philox32Step st;
  const PhiloxKeys* K;
  __device__ __forceinline__ U4 operator()(uint32_t j) const { return philox32_block(A0 ^ j, st, *K); }
};

// Block b of a direction's FP32 normals: v[q] = normal 4 b + q (zero past ng).
__device__ __forceinline__ void red_normal_block(const RedStream32& S, uint32_t j0, int b, int ng, float (&v)[4]) {
  const U4 r = S(j0 + static_cast<uint32_t>(b));
  box_muller32(u23(r.x), u23(r.y), v[0], v[1]);
  box_muller32(u23(r.z), u23(r.w), v[2], v[3]);
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = (4 * b + q < ng) ? v[q] : 0.0f;
}

template <int NG>
__device__ __forceinline__ void red_normals(const RedStream32& S, uint32_t j0, int ng, float (&g)[NG]) {
#pragma unroll
  for (int b = 0; b < (NG + 3) / 4; ++b) {
    if (4 * b < ng) {
      const U4 r = S(j0 + static_cast<uint32_t>(b));
      float v[4];
      box_muller32(u23(r.x), u23(r.y), v[0], v[1]);
      box_muller32(u23(r.z), u23(r.w), v[2], v[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * b + q < NG) g[4 * b + q] = (4 * b + q < ng) ? v[q] : 0.0f;
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (4 * b + q < NG) g[4 * b + q] = 0.0f;
    }
  }
}

__device__ __forceinline__ double red_chi2(const PhiloxKeys& K, uint32_t j0, uint32_t kk, uint32_t i, uint32_t p,
                                           int m, double) {
  if (m <= 0) return 0.0;
  if (m == 1) {
    const U4 r = philox4x32_10(j0, kk, i, p, K);
    double x, y;
    box_muller64(u53(r.x, r.y), u53(r.z, r.w), x, y);
    return x * x;
  }
  const double d = 0.5 * static_cast<double>(m) - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double cand = d;
  for (uint32_t a = 0; a < kChi2Attempts; ++a) {
    const U4 r = philox4x32_10(j0 + 2u * a, kk, i, p, K);
    double x, y;
    box_muller64(u53(r.x, r.y), u53(r.z, r.w), x, y);
    double v = 1.0 + c * x;
    if (v <= 0.0) continue;
    v = v * v * v;
    cand = d * v;
    const U4 ru = philox4x32_10(j0 + 2u * a + 1u, kk, i, p, K);
    const double U = u53(ru.x, ru.y);
    if (log(U) < 0.5 * x * x + d - d * v + d * log(v)) return 2.0 * d * v;
  }
  return 2.0 * cand;
}

// 3 log1p(t) - 3t - 3t^2 - t^3: its Taylor series about 0 for |t| < 1/4
// (-9/2 t^2 - 3/4 t^4 + 3/5 t^5 - 1/2 t^6 + 3/7 t^7 - 3/8 t^8 + 1/3 t^9 - 3/10 t^10,
// the t^3 terms cancel; relative error < 3e-7 there), log1pf beyond.
__device__ __forceinline__ float mt_log_term(float t) {
  if (fabsf(t) < 0.25f)
    return t * t *
           (-4.5f + t * t * (-0.75f + t * (0.6f + t * (-0.5f + t * (0.42857143f + t * (-0.375f + t * (0.33333333f +
                                                                                                     t * -0.3f)))))));
  return 3.0f * log1pf(t) - t * (3.0f + t * (3.0f + t));
}

// FP32: the same acceptance test written as d (3 log1p(t) - 3t - 3t^2 - t^3),
// t = c x (identical to d - d v + d log v for v = (1 + t)^3), which avoids the
// cancellation of d - d v in single precision.  `first` is attempt 0's block
// (j0), which the caller also uses for the radius uniform.
// d = m / 2 - 1 / 3 and c = 1 / sqrt(9 d) are the launch's constants.
__device__ __forceinline__ float red_chi2(const RedStream32& S, uint32_t j0, int m, float d, float c,
                                          const U4& first) {
  if (m <= 0) return 0.0f;
  if (m == 1) {
    float x, y;
    box_muller32(u23(first.x), u23(first.y), x, y);
    return x * x;
  }
  float cand = d;
  for (uint32_t a = 0; a < kChi2Attempts; ++a) {
    const U4 r = a == 0 ? first : S(j0 + a);
    float x, y;
    box_muller32(u23(r.x), u23(r.y), x, y);
    const float t = c * x;
    if (t <= -1.0f) continue;
    const float v = (1.0f + t) * (1.0f + t) * (1.0f + t);
    cand = d * v;
    if (__logf(u23(r.z)) < 0.5f * x * x + d * mt_log_term(t)) return 2.0f * d * v;
  }
  return 2.0f * cand;
}

// x[v] for a runtime v < NT without addressing the register array.
template <typename T, int NT>
__device__ __forceinline__ T sel(const T (&x)[NT], int v) {
  T r = x[0];
#pragma unroll
  for (int q = 1; q < NT; ++q) r = (v == q) ? x[q] : r;
  return r;
}

// POLY data at the tracked coordinates x (variables remapped on the host).
template <typename T, int NT>
__device__ __forceinline__ T red_poly(const DevFunc& fn, const T (&x)[NT]) {
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    T prod = pick<T>(fn.coef[t], fn.coef_f[t]);
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const T xv = sel<T, NT>(x, fn.var[q]);
      for (int e = 0; e < fn.pw[q]; ++e) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// SPHERE_QUAD from |z|^2, v.z and z^T A z.
template <typename T>
__device__ __forceinline__ T red_quad_finish(const DevProblem& pb, T trA, T zz, T lin, T quad, int D) {
  const T iz = T(1) / dsqrt<T>(zz);
  lin *= iz;
  quad *= iz * iz;
  const T c0 = pick<T>(pb.f.c0, pb.f.c0_f);
  if (!pb.f.apply_op) return c0 + lin + quad;
  const T dm = T(D - 1), sg = pick<T>(pb.sigma, pb.sf.sigma), mean = trA / T(D);
  return sg * (c0 + mean) + (dm + sg) * lin + (T(2) * (dm + T(1)) + sg) * (quad - mean);
}

// SPHERE_QUAD at the direction of z (NT components, zero padded): A (NT x NT,
// zero padded), v and tr(A) in shared memory; zrow is this thread's shared row
// for the rolled loop over the D rows of A.
template <typename T, int NT>
__device__ __forceinline__ T red_quad(const DevProblem& pb, const T* As, const T* vs, T trA, const T (&z)[NT],
                                      T* zrow, int D) {
  T zz = T(0), lin = T(0);
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    zz += z[j] * z[j];
    lin += vs[j] * z[j];
    zrow[j] = z[j];
  }
  T quad = T(0);
#pragma unroll 1
  for (int a = 0; a < D; ++a) {
    const T* Ar = As + a * NT;
    T Az = T(0);
#pragma unroll
    for (int b = 0; b < NT; ++b) Az += Ar[b] * z[b];
    quad += zrow[a] * Az;
  }
  return red_quad_finish<T>(pb, trA, zz, lin, quad, D);
}

template <typename T, int MK, int NT>
__device__ __forceinline__ void walkr_body(const DevProblem& pb, const T* As, const T* vs, T trA, T* zrow) {
  constexpr bool kF64 = sizeof(T) == 8;
  constexpr bool kSph = MK == kSphere, kEmb = MK == kEmbeddedSphere;
  constexpr int OFF = kSph ? 1 : 0;   // g[0] = h on a sphere, then the T components
  constexpr int NG = NT + OFF;
  const int n = pb.n;
  const int nT = pb.red_nT;
  const int ng = nT + (kSph ? 1 : 0);
  const int rest = pb.red_rest;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const T eps_t = pick<T>(pb.eps, pb.sf.eps), h_t = pick<T>(pb.h, pb.sf.h);
  const T rgeo_t = pick<T>(pb.rho_geo, pb.sf.rho_geo), theta_t = pick<T>(pb.theta, pb.sf.theta);
  const T sqs_t = pick<T>(pb.sqrt_sigma, pb.sf.sqrt_sigma);
  const T sh_t = pick<T>(sqrt(1.0 - pb.h * pb.h), pb.sf.sh);
  const bool bnd = !pb.closed;
  T eT[NT];
#pragma unroll
  for (int q = 0; q < NT; ++q) eT[q] = q < nT ? pick<T>(pb.red_e[q], pb.red_ef[q]) : T(0);

  const int64_t total = pb.wk_w1;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t w = pb.wk_w0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= total) return;
  T y[NT];
  T rho = T(0);
  WalkAcc<T> wa;
  wa.set_tau(pb.tau_w);
  int64_t k = 0, o = 0;
  uint32_t p = 0, wi = 0;
  Philox32Walk pw{0u, 0u};
  // Marsaglia-Tsang constants of chi^2_rest (FP32; rest >= 2)
  const float mt_d = 0.5f * static_cast<float>(rest) - 1.0f / 3.0f;
  const float mt_c = rest >= 2 ? rsqrtf(9.0f * mt_d) : 0.0f;
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; wi = id.i; o = id.o;
    if constexpr (!kF64) pw = philox32_walk(wi, K);
    wa.reset();
    k = 0;
    if constexpr (kEmb) {
#pragma unroll
      for (int q = 0; q < NT; ++q) y[q] = q < nT ? T(pb.s0[static_cast<size_t>(p) * nT + q]) : T(0);
    } else {
      const double* st = pb.red_y0 + static_cast<size_t>(p) * (kMaxQuadDim + 1);
#pragma unroll
      for (int q = 0; q < NT; ++q) y[q] = q < nT ? T(st[q]) : T(0);
      rho = T(st[kMaxQuadDim]);
    }
  };
  init(w);
  T r_prev = T(-1);
  GreenLaw law{};

  for (;;) {
    T dG = T(INFINITY);
    bool done = false;
    int flag = 0;
    if (bnd && !kEmb) {
      T al = T(0), yy = T(0);
#pragma unroll
      for (int q = 0; q < NT; ++q) { al += eT[q] * y[q]; yy += y[q] * y[q]; }
      T ygs, yge;   // y_Gamma = ygs y + yge e
      if constexpr (kSph) {
        yy += rho * rho;
        const T rh = dsqrt<T>(fmax(yy - al * al, T(0)));
        const T rt = rh * h_t - al * sh_t;
        T ex = fabs(T(1) - h_t * al - sh_t * rh) - rgeo_t;
        ex = ex < T(0) ? T(0) : ex;
        dG = (al <= h_t) ? T(0) : dsqrt<T>(rt * rt + ex * ex);
        ygs = sh_t / rh;
        yge = h_t - al * ygs;
      } else {
        dG = (al <= h_t) ? T(0) : fabs(al - h_t);
        ygs = T(1);
        yge = -(al - h_t);
      }
      if (dG < eps_t) {
        T yg[NT];
#pragma unroll
        for (int q = 0; q < NT; ++q) yg[q] = ygs * y[q] + yge * eT[q];
        wa.add_terminal(red_poly<T, NT>(pb.g, yg));
        done = true;
      } else if (wa.zero()) {
        done = true;
      }
    } else if (wa.below()) {
      done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      pb.S_out[o] = wa.score();
      pb.K_out[o] = static_cast<int32_t>(k);
      pb.flag_out[o] = flag;
      w = next_walk(pb, w, stride);
      if (w >= total) break;
      init(w);
      continue;
    }
    const T r = theta_t * (dG < rgeo_t ? dG : rgeo_t);
    const T a = sqs_t * r;
    if (r != r_prev) {
      if constexpr (kF64) {
        law = green_law(n, a);
        wa.set(law.c, law.omc / pb.sigma);
      } else if (!pb.em1_fp64) {
        wa.set_from_em1(em1_poly32(pb, 0.25f * a * a), pb.sf.inv_sigma);
      } else {
        const double ad = static_cast<double>(a);
        const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (ad * ad));
        const double cc = 1.0 / (1.0 + em1);
        wa.set(cc, one_minus_c(em1, cc) / pb.sigma);
      }
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    RedStream32 S32{0u, Philox32Step{0u, 0u, 0u, 0u}, &K};
    if constexpr (!kF64) S32 = RedStream32{pw.A0, philox32_step(pw, kk, p, K), &K};
    T g[NG];
    // ---- interior samples Z_l and F_k ----------------------------------------
    T F = T(0);
    for (int l = 0; l < nv; ++l) {
      const uint32_t jv = 64u * static_cast<uint32_t>(1 + l);
      T t, X;
      if constexpr (kF64) {
        const U4 bu = philox4x32_10(64u * static_cast<uint32_t>(1 + nv) + static_cast<uint32_t>(l), kk, wi, p, K);
        const double U = u53(bu.x, bu.y);
        const double guess = table_lookup<double>(pb.tab64, pb.NA, pb.NS, pb.z_max, a, U);
        t = green_invert64(law, U, guess);
        X = red_chi2(K, jv + 32u, kk, wi, p, rest, 0.0);
      } else {
        const U4 c0 = S32(jv + 32u);
        t = fminf(fmaxf(table_lookup32(pb, a, u23(c0.w)), 0.0f), 1.0f);
        X = red_chi2(S32, jv + 32u, rest, mt_d, mt_c, c0);
      }
      if constexpr (kF64) red_normals<NG>(K, jv, kk, wi, p, ng, g);
      else red_normals<NG>(S32, jv, ng, g);
      T gg = X;
#pragma unroll
      for (int q = 0; q < NG; ++q) gg += g[q] * g[q];
      const T zs = (r * t) / dsqrt<T>(gg);
      T z[NT];
#pragma unroll
      for (int q = 0; q < NT; ++q) z[q] = y[q] + zs * g[q + OFF];
      if constexpr (kEmb) {
        F += red_quad<T, NT>(pb, As, vs, trA, z, zrow, nT);
      } else if constexpr (kSph) {
        const T zr = rho + zs * g[0];
        T zz = zr * zr + zs * zs * X;
#pragma unroll
        for (int q = 0; q < NT; ++q) zz += z[q] * z[q];
        const T iz = T(1) / dsqrt<T>(zz);
#pragma unroll
        for (int q = 0; q < NT; ++q) z[q] *= iz;
        F += red_poly<T, NT>(pb.f, z);
      } else {
        F += red_poly<T, NT>(pb.f, z);
      }
    }
    if (nv > 1) F /= T(nv);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta) ------------------------------------
    T X;
    if constexpr (kF64) {
      red_normals<NG>(K, 0u, kk, wi, p, ng, g);
      X = red_chi2(K, 32u, kk, wi, p, rest, 0.0);
    } else {
      red_normals<NG>(S32, 0u, ng, g);
      X = red_chi2(S32, 32u, rest, mt_d, mt_c, S32(32u));
    }
    T gg = X;
#pragma unroll
    for (int q = 0; q < NG; ++q) gg += g[q] * g[q];
    const T sc = r / dsqrt<T>(gg);
    if constexpr (kEmb) {
      T tt = T(0);
#pragma unroll
      for (int q = 0; q < NT; ++q) { y[q] = y[q] + sc * g[q]; tt += y[q] * y[q]; }
      const T it = T(1) / dsqrt<T>(tt);
#pragma unroll
      for (int q = 0; q < NT; ++q) y[q] *= it;
    } else if constexpr (kSph) {
      const T tr = rho + sc * g[0];
      const T rr = tr * tr + sc * sc * X;
      T tt = rr;
#pragma unroll
      for (int q = 0; q < NT; ++q) { y[q] = y[q] + sc * g[q + OFF]; tt += y[q] * y[q]; }
      const T it = T(1) / dsqrt<T>(tt);
#pragma unroll
      for (int q = 0; q < NT; ++q) y[q] *= it;
      rho = dsqrt<T>(rr) * it;
    } else {
#pragma unroll
      for (int q = 0; q < NT; ++q) y[q] = y[q] + sc * g[q];
    }
    wa.add_step(F);
    ++k;
  }
}

template <typename T, int MK, int NT>
__global__ void __launch_bounds__(128) walkr_kernel(const DevProblem pb) {
  constexpr bool kEmb = MK == kEmbeddedSphere;
  __shared__ T As[kEmb ? NT * NT : 1];
  __shared__ T vs[kEmb ? NT : 1];
  __shared__ T zrows[kEmb ? 128 * (NT + 1) : 1];   // odd row stride: conflict-free
  T trA = T(0);
  if constexpr (kEmb) {
    const int D = pb.red_nT;
    const T* A = reinterpret_cast<const T*>(sizeof(T) == 8 ? static_cast<const void*>(pb.f.A)
                                                              : static_cast<const void*>(pb.f.Af));
    const T* v = reinterpret_cast<const T*>(sizeof(T) == 8 ? static_cast<const void*>(pb.f.v)
                                                              : static_cast<const void*>(pb.f.vf));
    for (int q = threadIdx.x; q < NT * NT; q += blockDim.x) {
      const int a = q / NT, b = q - a * NT;
      As[q] = (a < D && b < D) ? A[a * D + b] : T(0);
    }
    for (int q = threadIdx.x; q < NT; q += blockDim.x) vs[q] = q < D ? v[q] : T(0);
    __syncthreads();
    for (int a = 0; a < D; ++a) trA += As[a * NT + a];
  }
  walkr_body<T, MK, NT>(pb, As, vs, trA, zrows + (kEmb ? threadIdx.x * (NT + 1) : 0));
}

// The reduced walk on an embedded sphere (FP32, N_V = 1) with one warp per
// walker, for launches of few walks, whose time is the walks' length: lanes
// b < NB draw the normals' Philox blocks, lane NB the chi^2 (and Z's radius
// uniform), lanes a < D the rows of A z, in parallel; every sum then runs on
// every lane in walkr_body's order, so the walks are bit-identical to
// walkr_kernel's.  gsh: NT floats, azsh: NT floats of the warp's shared memory.
template <int NT>
__device__ __forceinline__ void walkr_lat_body(const DevProblem& pb, const float* As, const float* vs, float trA,
                                               float* gsh, float* azsh) {
  constexpr int NB = (NT + 3) / 4;   // Philox blocks of a direction's normals
  static_assert(NB < 32, "one lane per block and one for the chi^2");
  const int lane = threadIdx.x & 31;
  const int nT = pb.red_nT, ng = nT, rest = pb.red_rest, D = nT;
  const PhiloxKeys& K = pb.keys;
  const float theta_t = pb.sf.theta, rgeo_t = pb.sf.rho_geo, sqs_t = pb.sf.sqrt_sigma;
  const float mt_d = 0.5f * static_cast<float>(rest) - 1.0f / 3.0f;
  const float mt_c = rest >= 2 ? rsqrtf(9.0f * mt_d) : 0.0f;
  const int64_t total = pb.wk_w1;
  const int64_t stride = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  int64_t w = pb.wk_w0 + ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (w >= total) return;   // warp-uniform
  float y[NT];
  WalkAcc<float> wa;
  wa.set_tau(pb.tau_w);
  int64_t k = 0, o = 0;
  uint32_t p = 0, wi = 0;
  Philox32Walk pw{0u, 0u};
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; wi = id.i; o = id.o;
    pw = philox32_walk(wi, K);
    wa.reset();
    k = 0;
#pragma unroll
    for (int q = 0; q < NT; ++q) y[q] = q < nT ? static_cast<float>(pb.s0[static_cast<size_t>(p) * nT + q]) : 0.0f;
  };
  // a direction's normals into g on every lane, its chi^2 into X (lane NB's
  // draw, broadcast); c0: the first chi^2 block when the caller drew it
  auto direction = [&](const RedStream32& S, uint32_t j0, float (&g)[NT], float& X, float& uz, bool z) {
    float xl = 0.0f, ul = 0.0f;
    if (lane < NB) {
      float v[4];
      red_normal_block(S, j0, lane, ng, v);
      *reinterpret_cast<float4*>(gsh + 4 * lane) = make_float4(v[0], v[1], v[2], v[3]);
    } else if (lane == NB) {
      const U4 c0 = S(j0 + 32u);
      ul = u23(c0.w);
      xl = red_chi2(S, j0 + 32u, rest, mt_d, mt_c, c0);
    }
    X = __shfl_sync(0xffffffffu, xl, NB);
    if (z) uz = __shfl_sync(0xffffffffu, ul, NB);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NT; q += 4) {
      const float4 t4 = *reinterpret_cast<const float4*>(gsh + q);
      g[q] = t4.x; g[q + 1] = t4.y; g[q + 2] = t4.z; g[q + 3] = t4.w;
    }
    __syncwarp();
  };
  init(w);
  float r_prev = -1.0f;
  for (;;) {
    bool done = wa.below();
    int flag = 0;
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      if (lane == 0) {
        pb.S_out[o] = wa.score();
        pb.K_out[o] = static_cast<int32_t>(k);
        pb.flag_out[o] = flag;
      }
      int64_t nxt = 0;
      if (lane == 0) nxt = next_walk(pb, w, stride);
      w = __shfl_sync(0xffffffffu, nxt, 0);
      if (w >= total) break;
      init(w);
      continue;
    }
    const float r = theta_t * rgeo_t;   // closed: delta_Gamma is infinite
    const float a = sqs_t * r;
    if (r != r_prev) {
      if (!pb.em1_fp64) {
        wa.set_from_em1(em1_poly32(pb, 0.25f * a * a), pb.sf.inv_sigma);
      } else {
        const double ad = static_cast<double>(a);
        const double em1 = em1_series(0.5 * static_cast<double>(pb.n - 2), 0.25 * (ad * ad));
        const double cc = 1.0 / (1.0 + em1);
        wa.set(cc, one_minus_c(em1, cc) / pb.sigma);
      }
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    const RedStream32 S32{pw.A0, philox32_step(pw, kk, p, K), &K};
    float g[NT];
    // ---- interior sample Z and F ---------------------------------------------
    float X, U;
    direction(S32, 64u, g, X, U, true);
    const float t = fminf(fmaxf(table_lookup32(pb, a, U), 0.0f), 1.0f);
    float gg = X;
#pragma unroll
    for (int q = 0; q < NT; ++q) gg += g[q] * g[q];
    const float zs = (r * t) / dsqrt<float>(gg);
    float z[NT];
#pragma unroll
    for (int q = 0; q < NT; ++q) z[q] = y[q] + zs * g[q];
    float zz = 0.0f, lin = 0.0f;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      zz += z[j] * z[j];
      lin += vs[j] * z[j];
    }
    if (lane < D) {
      const float* Ar = As + lane * NT;
      float Az = 0.0f;
#pragma unroll
      for (int b = 0; b < NT; ++b) Az += Ar[b] * z[b];
      azsh[lane] = Az;
    }
    __syncwarp();
    float quad = 0.0f;
#pragma unroll
    for (int aa = 0; aa < NT; ++aa)
      if (aa < D) quad += z[aa] * azsh[aa];
    __syncwarp();
    const float F = red_quad_finish<float>(pb, trA, zz, lin, quad, D);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta) ------------------------------------
    direction(S32, 0u, g, X, U, false);
    gg = X;
#pragma unroll
    for (int q = 0; q < NT; ++q) gg += g[q] * g[q];
    const float sc = r / dsqrt<float>(gg);
    float tt = 0.0f;
#pragma unroll
    for (int q = 0; q < NT; ++q) { y[q] = y[q] + sc * g[q]; tt += y[q] * y[q]; }
    const float it = 1.0f / dsqrt<float>(tt);
#pragma unroll
    for (int q = 0; q < NT; ++q) y[q] *= it;
    wa.add_step(F);
    ++k;
  }
}

template <int NT>
__global__ void __launch_bounds__(128) walkr_lat_kernel(const DevProblem pb) {
  __shared__ float As[NT * NT];
  __shared__ float vs[NT];
  __shared__ __align__(16) float gsh[4][NT];
  __shared__ float azsh[4][NT];
  const int D = pb.red_nT;
  for (int q = threadIdx.x; q < NT * NT; q += blockDim.x) {
    const int a = q / NT, b = q - a * NT;
    As[q] = (a < D && b < D) ? pb.f.Af[a * D + b] : 0.0f;
  }
  for (int q = threadIdx.x; q < NT; q += blockDim.x) vs[q] = q < D ? pb.f.vf[q] : 0.0f;
  __syncthreads();
  float trA = 0.0f;
  for (int a = 0; a < D; ++a) trA += As[a * NT + a];
  const int wv = threadIdx.x >> 5;
  walkr_lat_body<NT>(pb, As, vs, trA, gsh[wv], azsh[wv]);
}

inline int walkr_nt(int nT) { return nT <= 4 ? 4 : (nT <= 8 ? 8 : (nT <= 16 ? 16 : (nT <= 24 ? 24 : 32))); }

}  // namespace mpwos
