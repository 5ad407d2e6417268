// walk3.cuh — the MPWoS walk for manifolds in R^3, one thread per walker.
//
// Each thread runs walks to completion and refills itself from a static
// walk queue (walk index w, w + stride, ...): the step loop is one flat loop
// whose body is the same for every lane, so walks of different lengths keep
// the warp converged.  A walk is Algorithm 1 with the path score of eq.
// path_score_definition:
//   stop test (Y_k in Gamma_eps -> S += W g(cp_Gamma(Y)); closed: W < tau_W),
//   r = theta min(delta_Gamma, rho_geo), c, omega,
//   Theta = Y + r g/|g|,  Z_l = Y + R_l g_l/|g_l| (R_l/r ~ radial Green law),
//   S += W omega F_k,  W *= c,  Y = cp(Theta).
#pragma once
#include "dev_common.cuh"
#include "geom3.cuh"
#include "green.cuh"
#include "cloud.cuh"
#include "comp.cuh"

namespace mpwos {

// FP64 walk.  Draws of step k of walk (p, i), Philox counter (j, k, i, p):
//   Theta direction: blocks 0, 1;  Z_l direction: blocks 2(1+l), 2(1+l)+1;
//   U_l: block 2(1+N_V) + l (words x, y);  two Gaussians per block.
// cp(x) for any R^3 manifold (point clouds through their k-nearest fit).
template <int MK, int KM, typename T>
__device__ __forceinline__ void cp_any(const DevProblem& pb, const T* x, T* out) {
  if constexpr (MK == kPointCloud) {
    Knn<T, KM> R;
    const T h = cloud_knn<T, KM>(pb, x, R);
    cloud_project<T, KM>(pb, x, R, h, out);
  } else {
    cp3<MK, T>(pb, x, out);
  }
}

// rho_geo at y: c_kappa/(1 + kappa) (eq. rho_geo_curvature) or c_h h(y) (eq. rho_geo_spacing).
template <int MK, int KM, typename T>
__device__ __forceinline__ T rho_geo_at(const DevProblem& pb, const T* y) {
  if constexpr (MK == kPointCloud) {
    Knn<T, KM> R;
    return pick<T>(pb.cl_c_h, pb.sf.c_h) * cloud_knn<T, KM>(pb, y, R);
  } else {
    return pick<T>(pb.rho_geo, pb.sf.rho_geo);
  }
}

// f constant (a POLY without variables): F needs no projection of Z.
__device__ __forceinline__ bool source_is_constant(const DevFunc& f) {
  return f.kind == kPoly && f.term_off[f.n_terms] == 0;
}

// COMP: the step's source is f(cp(Z)) + m_*(Z) (compensation term, comp.cuh).
template <int MK, int KM, bool COMP>
__device__ __forceinline__ void walk3_f64_body(const DevProblem& pb) {
  const int64_t total = pb.wk_w1;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t w = pb.wk_w0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const uint32_t ub = 2u * static_cast<uint32_t>(1 + nv);

  double Y[3], W = 1.0, S = 0.0;
  int64_t k = 0, o = 0;
  uint32_t p = 0, i = 0;
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; i = id.i; o = id.o;
    const double* y0 = pb.pts + static_cast<size_t>(p) * 3;
    Y[0] = y0[0]; Y[1] = y0[1]; Y[2] = y0[2];
    W = 1.0; S = 0.0; k = 0;
  };
  init(w);
  double r_prev = -1.0, omega = 0.0;
  GreenLaw law{};

  for (;;) {
    double dG = INFINITY;
    bool done = false;
    int flag = 0;
    if (!pb.closed) {
      double yg[3];
      dG = delta_gamma3<MK, double>(pb, Y, yg);
      if (dG < pb.eps) {
        S += W * func3<MK, double>(pb, pb.g, yg);
        done = true;
      } else if (W == 0.0) {
        done = true;
      }
    } else if (W < pb.tau_w) {
      done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      pb.S_out[o] = S;
      pb.K_out[o] = static_cast<int32_t>(k);
      pb.flag_out[o] = flag;
      w = next_walk(pb, w, stride);
      if (w >= total) break;
      init(w);
      continue;
    }
    const double rgeo = rho_geo_at<MK, KM, double>(pb, Y);
    const double r = pb.theta * (dG < rgeo ? dG : rgeo);
    const double a = pb.sqrt_sigma * r;
    if (r != r_prev) {
      law = green_law(3, a);
      omega = law.omc / pb.sigma;
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    // Theta = Y + r g/|g|
    double g[3], gx;
    {
      const U4 b0 = philox4x32_10(0u, kk, i, p, K);
      const U4 b1 = philox4x32_10(1u, kk, i, p, K);
      box_muller64(u53(b0.x, b0.y), u53(b0.z, b0.w), g[0], g[1]);
      box_muller64(u53(b1.x, b1.y), u53(b1.z, b1.w), g[2], gx);
    }
    const double gn = sqrt(dot3(g, g));
    const double sc = r / gn;
    double Th[3];
    for (int q = 0; q < 3; ++q) Th[q] = Y[q] + sc * g[q];
    // F_k over N_V interior samples
    double F = 0.0;
    for (int l = 0; l < nv; ++l) {
      const U4 bu = philox4x32_10(ub + static_cast<uint32_t>(l), kk, i, p, K);
      const double U = u53(bu.x, bu.y);
      const double guess = table_lookup<double>(pb.tab64, pb.NA, pb.NS, pb.z_max, a, U);
      const double t = green_invert64(law, U, guess);
      const uint32_t jb = 2u * static_cast<uint32_t>(1 + l);
      const U4 b0 = philox4x32_10(jb, kk, i, p, K);
      const U4 b1 = philox4x32_10(jb + 1u, kk, i, p, K);
      box_muller64(u53(b0.x, b0.y), u53(b0.z, b0.w), g[0], g[1]);
      box_muller64(u53(b1.x, b1.y), u53(b1.z, b1.w), g[2], gx);
      const double zn = sqrt(dot3(g, g));
      const double zs = (r * t) / zn;
      double Z[3], cZ[3];
      for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * g[q];
      if (MK == kPointCloud && source_is_constant(pb.f)) {
        F += func3<MK, double>(pb, pb.f, Z);
      } else {
        cp_any<MK, KM, double>(pb, Z, cZ);
        double fz = func3<MK, double>(pb, pb.f, cZ);
        if constexpr (COMP) fz = fz + comp_m64<MK>(pb, Z, cZ, fz);
        F += fz;
      }
    }
    if (nv > 1) F /= static_cast<double>(nv);
    S += (W * omega) * F;
    W *= law.c;
    cp_any<MK, KM, double>(pb, Th, Y);
    ++k;
  }
}

// FP32 walk.  Positions, projection and sampling in FP32; c_{sigma,r} and
// omega from the FP64 series (once per radius value); each walk's weight W and
// score S in float pairs (~2^-48 relative), so the step loop issues no FP64
// instruction; per-point sums over walks are FP64 (reduce kernel).
// Draws of a step: N_V = 1 takes one block, block 0 of the step, whose five
// 23-bit uniforms give the directions of Theta and Z (two each, sphere_dir3)
// and U (the fifth, u23_high).  N_V > 1: the step's 3(1+N_V) Gaussians come
// from consecutive uniform pairs (Box-Muller) of the step's uniform stream (four
// 23-bit uniforms per block), U_l follows at uniform index 2 ceil(3(1+N_V)/2) + l.
__device__ __forceinline__ float uniform_at32(uint32_t u, uint32_t kk, uint32_t i, uint32_t p,
                                              const PhiloxKeys& K) {
  const U4 b = philox4x32_10(u >> 2, kk, i, p, K);
  const uint32_t s = u & 3u;
  return u23(s == 0 ? b.x : (s == 1 ? b.y : (s == 2 ? b.z : b.w)));
}

__device__ __forceinline__ float gaussian_at32(uint32_t q, uint32_t kk, uint32_t i, uint32_t p,
                                               const PhiloxKeys& K) {
  const uint32_t pair = q >> 1;
  const U4 b = philox4x32_10(pair >> 1, kk, i, p, K);
  const bool hi = pair & 1u;
  float g0, g1;
  box_muller32(u23(hi ? b.z : b.x), u23(hi ? b.w : b.y), g0, g1);
  return (q & 1u) ? g1 : g0;
}

// Torus angles of cp(x) (same as those of x about the centre circle).
__device__ __forceinline__ void torus_angles32(float R, const float* x, float& ct, float& st, float& cph,
                                               float& sph) {
  const float rho2 = x[0] * x[0] + x[1] * x[1];
  const float irho = rsqrtf(rho2);
  const float dr = rho2 * irho - R;
  const float iw = rsqrtf(dr * dr + x[2] * x[2]);
  ct = dr * iw;
  st = x[2] * iw;
  cph = x[0] * irho;
  sph = x[1] * irho;
}

// (-Delta_M + sigma) u or u itself for a torus Fourier series, from the angles.
__device__ __forceinline__ float torus_series32(const DevProblem& pb, const DevFunc& fn, float ct, float st,
                                               float cph, float sph) {
  const float R = pb.sf.R, a = pb.sf.a;
  const float ia = pb.sf.inv_a;
  const float irr = __fdividef(1.0f, R + a * ct);
  const float sg = pb.sf.sigma;
  float total = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    float cm, sm, cq, sq;
    angle_multiple(fn.modes[t][0], ct, st, cm, sm);
    angle_multiple(fn.modes[t][1], cph, sph, cq, sq);
    const bool tcos = fn.modes[t][2] == 0;
    const float Tv = tcos ? cm : sm;
    const float Pv = fn.modes[t][3] == 0 ? cq : sq;
    float val;
    if (!fn.apply_op) {
      val = Tv * Pv;
    } else {
      const float mf = fn.mode_f[t][0];
      const float Tp = tcos ? -mf * sm : mf * cm;
      const float lap = fn.mode_f[t][2] * Tv * (ia * ia) + st * Tp * (ia * irr) + fn.mode_f[t][3] * Tv * (irr * irr);
      val = Pv * (lap + sg * Tv);
    }
    total += fn.coef_f[t] * val;
  }
  return total;
}

// The single torus Fourier term with compile-time mode numbers M, Q and
// trig choices (TSIN: sin(M theta), else cos; PSIN: sin(Q phi), else cos) --
// the launch picks the instance once, so the angle multiples become
// straight-line code with no per-step selects: the same value as
// torus_series32 for that term.
template <int M, int Q, bool TSIN, bool PSIN>
__device__ __forceinline__ float torus_term32(const DevProblem& pb, const DevFunc& fn, float ct, float st, float cph,
                                              float sph) {
  float cm, sm, cq, sq;
  angle_multiple(M, ct, st, cm, sm);
  angle_multiple(Q, cph, sph, cq, sq);
  const float Tv = TSIN ? sm : cm;
  const float Pv = PSIN ? sq : cq;
  if (!fn.apply_op) return fn.coef_f[0] * (Tv * Pv);
  const float ia = pb.sf.inv_a;
  const float irr = __fdividef(1.0f, pb.sf.R + pb.sf.a * ct);
  const float Tp = TSIN ? static_cast<float>(M) * cm : -static_cast<float>(M) * sm;
  const float lap = static_cast<float>(M * M) * Tv * (ia * ia) + st * Tp * (ia * irr) +
                    static_cast<float>(Q * Q) * Tv * (irr * irr);
  return fn.coef_f[0] * (Pv * (lap + pb.sf.sigma * Tv));
}

// cp(x) in FP32 with reciprocal square roots.
template <int MK>
__device__ __forceinline__ void cp3_f32(const DevProblem& pb, const float* x, float* out) {
  if constexpr (MK == kEuclid) {
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2];
  } else if constexpr (MK == kSphere) {
    const float inv = rsqrtf(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    out[0] = x[0] * inv; out[1] = x[1] * inv; out[2] = x[2] * inv;
  } else {
    // cp = (R + s dr)/rho (x0, x1) + s x2 e_z, dr = rho - R, s = a / sqrt(dr^2 + x2^2)
    const float R = pb.sf.R;
    const float rho2 = x[0] * x[0] + x[1] * x[1];
    const float irho = rsqrtf(rho2);
    const float dr = rho2 * irho - R;
    const float s = pb.sf.a * rsqrtf(dr * dr + x[2] * x[2]);
    const float fac = (R + s * dr) * irho;
    out[0] = x[0] * fac; out[1] = x[1] * fac; out[2] = s * x[2];
  }
}

// f(cp(Z)) in FP32.
template <int MK, int KM>
__device__ __forceinline__ float source_at32(const DevProblem& pb, const float* Z) {
  if constexpr (MK == kPointCloud) {
    if (source_is_constant(pb.f)) return func3<MK, float>(pb, pb.f, Z);
    float cZ[3];
    cp_any<MK, KM, float>(pb, Z, cZ);
    return func3<MK, float>(pb, pb.f, cZ);
  }
  if constexpr (MK == kTorus) {
    if (pb.f.kind == kTorusFourier) {
      float ct, st, cph, sph;
      torus_angles32(pb.sf.R, Z, ct, st, cph, sph);
      return torus_series32(pb, pb.f, ct, st, cph, sph);
    }
  }
  float cZ[3];
  cp3_f32<MK>(pb, Z, cZ);
  return func3<MK, float>(pb, pb.f, cZ);
}

// The FP32 step loop.  FIXED: closed problems on analytic manifolds, where the
// radius, c and omega are constants of the launch; the loop then carries
// V = W omega instead of W (stop at V < tau_W omega), adds V F_k to S with one
// TwoSum whose low parts accumulate unnormalised (renormalised every 64 steps;
// |S.lo| stays below 64 ulp(S.hi)), and updates V *= c without renormalising
// (|V.lo| stays within a few ulp of V.hi).  Otherwise W, S and omega follow the
// radius step by step.
template <int MK, int KM, bool FIXED, bool COMP = false>
__device__ __forceinline__ void walk3_f32_body(const DevProblem& pb) {
  const int64_t total = pb.wk_w1;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t w = pb.wk_w0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const int max_steps = static_cast<int>(pb.max_steps);
  const float eps = pb.sf.eps;
  const float theta = pb.sf.theta;
  const float rgeo = pb.sf.rho_geo;
  const float sqs = pb.sf.sqrt_sigma;
  const F2 tau = f2_from_double(pb.tau_w);
  const float inv_sigma = pb.sf.inv_sigma;

  float Y[3];
  F2 W{1.0f, 0.0f}, S{0.0f, 0.0f};
  int k = 0;
  int64_t o = 0;
  uint32_t p = 0, i = 0;
  PhiloxWalk pw{};
  float r_prev = -1.0f;
  F2 c2{1.0f, 0.0f}, om2{0.0f, 0.0f}, thr{0.0f, 0.0f};
  auto set_weights = [&](float a) {
    if (!pb.em1_fp64) {
      weights_from_em1(em1_poly32(pb, 0.25f * a * a), inv_sigma, c2, om2);
    } else {
      const double ad = static_cast<double>(a);
      const double em1 = em1_series(0.5, 0.25 * (ad * ad));
      const double c = 1.0 / (1.0 + em1);
      c2 = f2_from_double(c);
      om2 = f2_from_double(one_minus_c(em1, c) / pb.sigma);
    }
  };
  int k_stop = max_steps;   // FIXED: the common stopping index of every walk
  bool k_flag = true;       // FIXED: walks end at max_steps (flagged) rather than by V < tau omega
  if constexpr (FIXED) {
    const float r = theta * rgeo;
    set_weights(sqs * r);
    thr = f2_mul(tau, om2);
    // V_k = omega c^k in the same float-pair recurrence as the step loop
    F2 V = om2;
    for (int kq = 0; kq < max_steps; ++kq) {
      if ((V.hi - thr.hi) + (V.lo - thr.lo) < 0.0f) {
        k_stop = kq;
        k_flag = false;
        break;
      }
      const float vh = __fmul_rn(V.hi, c2.hi);
      float ve = __fmaf_rn(V.hi, c2.hi, -vh);
      ve = __fmaf_rn(V.hi, c2.lo, ve);
      ve = __fmaf_rn(V.lo, c2.hi, ve);
      V = F2{vh, ve};
    }
    if (k_flag && (V.hi - thr.hi) + (V.lo - thr.lo) < 0.0f) k_flag = false;   // V falls below at k = max_steps
  }
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; i = id.i; o = id.o;
    const double* y0 = pb.pts + static_cast<size_t>(p) * 3;
    Y[0] = static_cast<float>(y0[0]); Y[1] = static_cast<float>(y0[1]); Y[2] = static_cast<float>(y0[2]);
    W = FIXED ? om2 : F2{1.0f, 0.0f};   // FIXED: W holds V = W omega
    S = F2{0.0f, 0.0f};
    k = 0;
    pw = philox_walk(i, p, K);
  };
  init(w);

  for (;;) {
    float dG = INFINITY;
    bool done = false;
    int flag = 0;
    if constexpr (FIXED) {
      if (k >= k_stop) {
        done = true;
        flag = k_flag ? 1 : 0;
      }
    } else if (!pb.closed) {
      float yg[3];
      dG = delta_gamma3<MK, float>(pb, Y, yg);
      if (dG < eps) {
        S = f2_add(S, f2_mul_f(W, func3<MK, float>(pb, pb.g, yg)));
        done = true;
      } else if (W.hi == 0.0f) {
        done = true;
      }
    } else if (W.hi < tau.hi || (W.hi == tau.hi && W.lo < tau.lo)) {
      done = true;
    }
    if (!FIXED && !done && k >= max_steps) { done = true; flag = 1; }
    if (done) {
      pb.S_out[o] = f2_to_double(S);
      pb.K_out[o] = k;
      pb.flag_out[o] = flag;
      w = next_walk(pb, w, stride);
      if (w >= total) break;
      init(w);
      continue;
    }
    float r, a;
    if constexpr (FIXED) {
      r = theta * rgeo;
      a = sqs * r;
    } else {
      float rg = rgeo;
      if constexpr (MK == kPointCloud) rg = rho_geo_at<MK, KM, float>(pb, Y);
      r = theta * (dG < rg ? dG : rg);
      a = sqs * r;
      if (r != r_prev) {   // constant-radius stretches evaluate the weights once
        set_weights(a);
        r_prev = r;
      }
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    float Th[3], F = 0.0f;
    if (nv == 1) {
      const U4 b = philox_step_one(pw, kk, K);
      float dt[3], dz[3];
      sphere_dir3(u23(b.x), u23(b.y), dt);
      sphere_dir3(u23(b.z), u23(b.w), dz);
      const float U = u23_high(b);
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + r * dt[q];
      float t = table_lookup32(pb, a, U);
      t = fminf(fmaxf(t, 0.0f), 1.0f);
      const float zs = r * t;
      float Z[3];
      for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * dz[q];
      F = source_at32<MK, KM>(pb, Z);
      if constexpr (COMP) F += comp_m32<MK>(pb, Z, F);
    } else {
      float g[3];
      for (int q = 0; q < 3; ++q) g[q] = gaussian_at32(static_cast<uint32_t>(q), kk, i, p, K);
      const float sc = r * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + sc * g[q];
      const uint32_t nu = 2u * ((3u * static_cast<uint32_t>(1 + nv) + 1u) / 2u);
      for (int l = 0; l < nv; ++l) {
        const float U = uniform_at32(nu + static_cast<uint32_t>(l), kk, i, p, K);
        float t = table_lookup32(pb, a, U);
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        for (int q = 0; q < 3; ++q)
          g[q] = gaussian_at32(3u * static_cast<uint32_t>(1 + l) + static_cast<uint32_t>(q), kk, i, p, K);
        const float zs = (r * t) * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
        float Z[3];
        for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * g[q];
        const float fz = source_at32<MK, KM>(pb, Z);
        F += COMP ? fz + comp_m32<MK>(pb, Z, fz) : fz;
      }
      F /= static_cast<float>(nv);
    }
    if constexpr (FIXED) {
      // S += V F: the product's error term and the TwoSum error join S.lo
      const float ph = __fmul_rn(W.hi, F);
      const float pl = __fmaf_rn(W.lo, F, __fmaf_rn(W.hi, F, -ph));
      const float s = __fadd_rn(S.hi, ph);
      const float bb = __fadd_rn(s, -S.hi);
      const float err = __fadd_rn(__fadd_rn(S.hi, -__fadd_rn(s, -bb)), __fadd_rn(ph, -bb));
      S = F2{s, __fadd_rn(S.lo, __fadd_rn(err, pl))};
      if ((k & 63) == 63) S = f2_fast_two_sum(S.hi, S.lo);
      // V *= c
      const float vh = __fmul_rn(W.hi, c2.hi);
      float ve = __fmaf_rn(W.hi, c2.hi, -vh);
      ve = __fmaf_rn(W.hi, c2.lo, ve);
      ve = __fmaf_rn(W.lo, c2.hi, ve);
      W = F2{vh, ve};
    } else {
      S = f2_add(S, f2_mul_f(f2_mul(W, om2), F));
      W = f2_mul(W, c2);
    }
    if constexpr (MK == kPointCloud) cp_any<MK, KM, float>(pb, Th, Y); else cp3_f32<MK>(pb, Th, Y);
    ++k;
  }
}

// The FP32 point-cloud walk: walk3_f32_body's step for a closed cloud problem,
// with every k-nearest search made by the whole warp (cloud_knn_coop; the
// neighbours, and so every result, are those of the per-lane search).  A lane
// whose walks are exhausted stays in the loop inactive -- it offers no query and
// skips its projections -- until every lane of its warp is done, so the warp's
// searches always have all 32 lanes.
template <int KM>
__device__ __forceinline__ void walk3_f32_cloud_body(const DevProblem& pb) {
  // one walker per `spread` lanes (lanes l with l % spread == 0); every lane
  // takes part in the warp's neighbour searches
  const int spread = pb.cl_spread > 1 ? pb.cl_spread : 1;
  const bool holder = (threadIdx.x & (spread - 1)) == 0;
  const int64_t total = pb.wk_w1;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x / spread;
  int64_t w = pb.wk_w0 + (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / spread;
  bool active = holder && w < total;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const int max_steps = static_cast<int>(pb.max_steps);
  const float theta = pb.sf.theta;
  const float sqs = pb.sf.sqrt_sigma;
  const F2 tau = f2_from_double(pb.tau_w);
  const float inv_sigma = pb.sf.inv_sigma;
  const bool f_const = source_is_constant(pb.f);

  float Y[3] = {0.0f, 0.0f, 0.0f};
  F2 W{1.0f, 0.0f}, S{0.0f, 0.0f};
  int k = 0;
  int64_t o = 0;
  uint32_t p = 0, i = 0;
  PhiloxWalk pw{};
  float r_prev = -1.0f;
  F2 c2{1.0f, 0.0f}, om2{0.0f, 0.0f};
  auto set_weights = [&](float a) {
    if (!pb.em1_fp64) {
      weights_from_em1(em1_poly32(pb, 0.25f * a * a), inv_sigma, c2, om2);
    } else {
      const double ad = static_cast<double>(a);
      const double em1 = em1_series(0.5, 0.25 * (ad * ad));
      const double c = 1.0 / (1.0 + em1);
      c2 = f2_from_double(c);
      om2 = f2_from_double(one_minus_c(em1, c) / pb.sigma);
    }
  };
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; i = id.i; o = id.o;
    const double* y0 = pb.pts + static_cast<size_t>(p) * 3;
    Y[0] = static_cast<float>(y0[0]); Y[1] = static_cast<float>(y0[1]); Y[2] = static_cast<float>(y0[2]);
    W = F2{1.0f, 0.0f};
    S = F2{0.0f, 0.0f};
    k = 0;
    pw = philox_walk(i, p, K);
  };
  if (active) init(w);
  // F at Z: f itself when constant, else f at the fitted closest point
  auto source = [&](const float* Z) -> float {
    if (f_const) return func3<kPointCloud, float>(pb, pb.f, Z);
    Knn<float, KM> R;
    const float h = cloud_knn_coop<KM>(pb, Z, active, R);
    float cZ[3] = {Z[0], Z[1], Z[2]};
    if (active) cloud_project<float, KM>(pb, Z, R, h, cZ);
    return func3<kPointCloud, float>(pb, pb.f, cZ);
  };

  for (;;) {
    if (active) {
      bool done = false;
      int flag = 0;
      if (W.hi < tau.hi || (W.hi == tau.hi && W.lo < tau.lo)) done = true;
      if (!done && k >= max_steps) { done = true; flag = 1; }
      if (done) {
        pb.S_out[o] = f2_to_double(S);
        pb.K_out[o] = k;
        pb.flag_out[o] = flag;
        w = next_walk(pb, w, stride);
        active = w < total;
        if (active) init(w);
      }
    }
    if (__all_sync(0xffffffffu, !active)) break;
    float r, a;
    {
      Knn<float, KM> R;
      const float hY = cloud_knn_coop<KM>(pb, Y, active, R);
      r = theta * (pb.sf.c_h * (active ? hY : 0.0f));   // rho_geo = c_h h(Y); closed: no delta_Gamma
      a = sqs * r;
    }
    if (r != r_prev) {
      set_weights(a);
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    float Th[3], F = 0.0f;
    if (nv == 1) {
      const U4 b = philox_step_one(pw, kk, K);
      float dt[3], dz[3];
      sphere_dir3(u23(b.x), u23(b.y), dt);
      sphere_dir3(u23(b.z), u23(b.w), dz);
      const float U = u23_high(b);
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + r * dt[q];
      float t = table_lookup32(pb, a, U);
      t = fminf(fmaxf(t, 0.0f), 1.0f);
      const float zs = r * t;
      float Z[3];
      for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * dz[q];
      F = source(Z);
    } else {
      float g[3];
      for (int q = 0; q < 3; ++q) g[q] = gaussian_at32(static_cast<uint32_t>(q), kk, i, p, K);
      const float sc = r * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + sc * g[q];
      const uint32_t nu = 2u * ((3u * static_cast<uint32_t>(1 + nv) + 1u) / 2u);
      for (int l = 0; l < nv; ++l) {
        const float U = uniform_at32(nu + static_cast<uint32_t>(l), kk, i, p, K);
        float t = table_lookup32(pb, a, U);
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        for (int q = 0; q < 3; ++q)
          g[q] = gaussian_at32(3u * static_cast<uint32_t>(1 + l) + static_cast<uint32_t>(q), kk, i, p, K);
        const float zs = (r * t) * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
        float Z[3];
        for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * g[q];
        F += source(Z);
      }
      F /= static_cast<float>(nv);
    }
    float Yn[3] = {Y[0], Y[1], Y[2]};
    {
      Knn<float, KM> R;
      const float h = cloud_knn_coop<KM>(pb, Th, active, R);
      if (active) cloud_project<float, KM>(pb, Th, R, h, Yn);
    }
    if (active) {
      S = f2_add(S, f2_mul_f(f2_mul(W, om2), F));
      W = f2_mul(W, c2);
      Y[0] = Yn[0]; Y[1] = Yn[1]; Y[2] = Yn[2];
      ++k;
    }
  }
}

// One FP32 step of a constant-radius walk with N_V = 1: the draws of step kk,
// Theta and Z from Y, F = f(cp(Z)) (returned), then Y = cp(Theta).  MQ >= 0:
// the torus source is one Fourier term with modes ((MQ / 4) % 4, MQ % 4),
// sin in theta if bit 4 of MQ is set and sin in phi if bit 5 is (else cos).
template <int MK, int MQ>
__device__ __forceinline__ float fixed_step32(const DevProblem& pb, const PhiloxKeys& K, const PhiloxWalk& pw,
                                              uint32_t kk, float r, float a, float (&Y)[3]) {
  const U4 b = philox_step_one(pw, kk, K);
  float dt[3], dz[3];
  sphere_dir3(u23(b.x), u23(b.y), dt);
  sphere_dir3(u23(b.z), u23(b.w), dz);
  float t = table_lookup32(pb, a, u23_high(b));
  t = fminf(fmaxf(t, 0.0f), 1.0f);
  const float zs = r * t;
  float Z[3], Th[3];
  for (int q = 0; q < 3; ++q) {
    Z[q] = Y[q] + zs * dz[q];
    Th[q] = Y[q] + r * dt[q];
  }
  float F;
  if constexpr (MK == kTorus && MQ >= 0) {
    float ct, st, cph, sph;
    torus_angles32(pb.sf.R, Z, ct, st, cph, sph);
    F = torus_term32<(MQ / 4) % 4, MQ % 4, ((MQ >> 4) & 1) != 0, ((MQ >> 5) & 1) != 0>(pb, pb.f, ct, st, cph, sph);
  } else {
    F = source_at32<MK, 1>(pb, Z);
  }
  cp3_f32<MK>(pb, Th, Y);
  return F;
}

// Closed problems on analytic manifolds with N_V = 1: the radius, c and omega
// are constants of the launch, so every walk has the same weights V_k = W_k
// omega = omega c^k and the same stopping index.  Each thread advances NW walks
// in lockstep (NW independent dependency chains per warp; V and the loop are
// shared), adding V F_k to each walk's S with one TwoSum whose low parts
// accumulate unnormalised (renormalised after every block of 64 steps,
// |S.lo| < 64 ulp(S.hi)).
// V *= c runs without renormalisation (|V.lo| stays within a few ulp of V.hi).
template <int MK, int NW, int MQ>
__device__ __forceinline__ void walk3_fixed_body(const DevProblem& pb) {
  const int64_t total = pb.wk_w1;
  const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const PhiloxKeys& K = pb.keys;
  const int max_steps = static_cast<int>(pb.max_steps);
  const float r = pb.sf.theta * pb.sf.rho_geo;
  const float a = pb.sf.sqrt_sigma * r;
  F2 c2, om2;
  if (!pb.em1_fp64) {
    weights_from_em1(em1_poly32(pb, 0.25f * a * a), pb.sf.inv_sigma, c2, om2);
  } else {
    const double ad = static_cast<double>(a);
    const double em1 = em1_series(0.5, 0.25 * (ad * ad));
    const double c = 1.0 / (1.0 + em1);
    c2 = f2_from_double(c);
    om2 = f2_from_double(one_minus_c(em1, c) / pb.sigma);
  }
  const F2 thr = f2_mul(f2_from_double(pb.tau_w), om2);   // W < tau_W  <=>  V < tau_W omega
  // the common stopping index, in the same float-pair recurrence as the loop
  int k_stop = max_steps;
  int k_flag = 1;
  {
    F2 V = om2;
    int kq = 0;
    for (; kq < max_steps; ++kq) {
      if ((V.hi - thr.hi) + (V.lo - thr.lo) < 0.0f) break;
      const float vh = __fmul_rn(V.hi, c2.hi);
      V = F2{vh, __fmaf_rn(V.lo, c2.hi, __fmaf_rn(V.hi, c2.lo, __fmaf_rn(V.hi, c2.hi, -vh)))};
    }
    if (kq < max_steps || (V.hi - thr.hi) + (V.lo - thr.lo) < 0.0f) {
      k_stop = kq;
      k_flag = 0;
    }
  }
  for (int64_t base = pb.wk_w0 + tid; base < total; base += NW * nthreads) {
    float Y[NW][3];
    F2 S[NW];
    PhiloxWalk pw[NW];
    int64_t o[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const int64_t w = base + j * nthreads;
      const WalkId id = walk_id(pb, w < total ? w : base);   // a missing partner repeats walk `base`
      o[j] = w < total ? id.o : -1;
      const double* y0 = pb.pts + static_cast<size_t>(id.p) * 3;
      Y[j][0] = static_cast<float>(y0[0]); Y[j][1] = static_cast<float>(y0[1]); Y[j][2] = static_cast<float>(y0[2]);
      S[j] = F2{0.0f, 0.0f};
      pw[j] = philox_walk(id.i, id.p, K);
    }
    F2 V = om2;
    for (int k0 = 0; k0 < k_stop; k0 += 64) {   // blocks of 64 steps, S renormalised after each
      const int k1 = k0 + 64 < k_stop ? k0 + 64 : k_stop;
      for (int k = k0; k < k1; ++k) {
#pragma unroll
        for (int j = 0; j < NW; ++j) {
          const float F = fixed_step32<MK, MQ>(pb, K, pw[j], static_cast<uint32_t>(k), r, a, Y[j]);
          // S += V F: the product's error term and the TwoSum error join S.lo
          const float ph = __fmul_rn(V.hi, F);
          const float pl = __fmaf_rn(V.lo, F, __fmaf_rn(V.hi, F, -ph));
          const float sh = __fadd_rn(S[j].hi, ph);
          const float bb = __fadd_rn(sh, -S[j].hi);
          const float err = __fadd_rn(__fadd_rn(S[j].hi, -__fadd_rn(sh, -bb)), __fadd_rn(ph, -bb));
          S[j] = F2{sh, __fadd_rn(S[j].lo, __fadd_rn(err, pl))};
        }
        const float vh = __fmul_rn(V.hi, c2.hi);
        V = F2{vh, __fmaf_rn(V.lo, c2.hi, __fmaf_rn(V.hi, c2.lo, __fmaf_rn(V.hi, c2.hi, -vh)))};
      }
#pragma unroll
      for (int j = 0; j < NW; ++j) S[j] = f2_fast_two_sum(S[j].hi, S[j].lo);
    }
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      if (o[j] < 0) continue;
      pb.S_out[o[j]] = f2_to_double(S[j]);
      pb.K_out[o[j]] = k_stop;
      pb.flag_out[o[j]] = k_flag;
    }
  }
}

// Entry points: the analytic manifolds run 256-thread blocks; the
// fixed-radius loop fits 40 registers (6 blocks, 48 warps per SM: measured
// fastest on B300; 7 blocks spill), the general loop 64 (4 blocks, with some
// spills: measured faster than 3 blocks at 80 registers on the S^2 cap and the
// uncompensated cut torus), the general loop with the compensation term 80
// (3 blocks, spill-free: 4.5 % faster than 4 blocks on Example 1); the
// point-cloud walk uses 128-thread blocks with a larger register budget.
// MQ >= 0 (torus, one Fourier term with modes m = (MQ / 4) % 4, q = MQ % 4 and
// its trig choices in bits 4 and 5, N_V = 1): the host launches the instance
// with those built in.  COMP: with the compensation term (general loop only).
template <int MK, int KM, bool FIXED, int MQ = -1, bool COMP = false>
__global__ void __launch_bounds__(256, FIXED ? 6 : (COMP ? 3 : 4)) walk3_f32_kernel(const DevProblem pb) {
  if constexpr (FIXED) {
    if (pb.n_v == 1) {
      walk3_fixed_body<MK, 1, MQ>(pb);
      return;
    }
  }
  walk3_f32_body<MK, KM, FIXED, COMP>(pb);
}
template <int MK, int KM>
__global__ void __launch_bounds__(128) walk3_f32_cloud_kernel(const DevProblem pb) {
  walk3_f32_body<MK, KM, false>(pb);
}
// The same walk with the warp-cooperative neighbour search: faster where a
// cell holds enough points to fill a warp's scan (k >= 12: +50 % at k = 16),
// slower for small k (-58 % at k = 6), so the host picks by k.
template <int KM>
__global__ void __launch_bounds__(128) walk3_f32_cloud_coop_kernel(const DevProblem pb) {
  walk3_f32_cloud_body<KM>(pb);
}
template <int MK, int KM, bool COMP = false>
__global__ void __launch_bounds__(128) walk3_f64_kernel(const DevProblem pb) { walk3_f64_body<MK, KM, COMP>(pb); }

}  // namespace mpwos
