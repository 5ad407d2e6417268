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

namespace mpwos {

// FP64 walk.  Draws of step k of walk (p, i), Philox counter (j, k, i, p):
//   Theta direction: blocks 0, 1;  Z_l direction: blocks 2(1+l), 2(1+l)+1;
//   U_l: block 2(1+N_V) + l (words x, y);  two Gaussians per block.
template <int MK>
__global__ void __launch_bounds__(128) walk3_f64_kernel(const DevProblem pb) {
  const int64_t total = pb.P * pb.N;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const uint32_t k0 = static_cast<uint32_t>(pb.seed), k1 = static_cast<uint32_t>(pb.seed >> 32);
  const int nv = pb.n_v;
  const uint32_t ub = 2u * static_cast<uint32_t>(1 + nv);

  double Y[3], W = 1.0, S = 0.0;
  int64_t k = 0;
  uint32_t p = 0, i = 0;
  auto init = [&](int64_t ww) {
    p = static_cast<uint32_t>(ww / pb.N);
    i = static_cast<uint32_t>(ww - static_cast<int64_t>(p) * pb.N);
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
      pb.S_out[w] = S;
      pb.K_out[w] = static_cast<int32_t>(k);
      pb.flag_out[w] = flag;
      w += stride;
      if (w >= total) break;
      init(w);
      continue;
    }
    const double rgeo = pb.rho_geo;
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
      const U4 b0 = philox4x32_10(0u, kk, i, p, k0, k1);
      const U4 b1 = philox4x32_10(1u, kk, i, p, k0, k1);
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
      const U4 bu = philox4x32_10(ub + static_cast<uint32_t>(l), kk, i, p, k0, k1);
      const double U = u53(bu.x, bu.y);
      const double guess = table_lookup<double>(pb.tab64, pb.NA, pb.NS, pb.z_max, a, s_of_u64(U));
      const double t = green_invert64(law, U, guess);
      const uint32_t jb = 2u * static_cast<uint32_t>(1 + l);
      const U4 b0 = philox4x32_10(jb, kk, i, p, k0, k1);
      const U4 b1 = philox4x32_10(jb + 1u, kk, i, p, k0, k1);
      box_muller64(u53(b0.x, b0.y), u53(b0.z, b0.w), g[0], g[1]);
      box_muller64(u53(b1.x, b1.y), u53(b1.z, b1.w), g[2], gx);
      const double zn = sqrt(dot3(g, g));
      const double zs = (r * t) / zn;
      double Z[3], cZ[3];
      for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * g[q];
      cp3<MK, double>(pb, Z, cZ);
      F += func3<MK, double>(pb, pb.f, cZ);
    }
    if (nv > 1) F /= static_cast<double>(nv);
    S += (W * omega) * F;
    W *= law.c;
    cp3<MK, double>(pb, Th, Y);
    ++k;
  }
}

// FP32 walk (FP64 weights and score).  Draws of a step are packed: the step's
// 3(1+N_V) Gaussians come from consecutive uniform pairs (Box-Muller) of the
// step's uniform stream (four 24-bit uniforms per block), U_l follows at
// uniform index 2 ceil(3(1+N_V)/2) + l.  N_V = 1 uses two blocks per step.
__device__ __forceinline__ float uniform_at32(uint32_t u, uint32_t kk, uint32_t i, uint32_t p,
                                              uint32_t k0, uint32_t k1) {
  const U4 b = philox4x32_10(u >> 2, kk, i, p, k0, k1);
  const uint32_t s = u & 3u;
  return u24(s == 0 ? b.x : (s == 1 ? b.y : (s == 2 ? b.z : b.w)));
}

__device__ __forceinline__ float gaussian_at32(uint32_t q, uint32_t kk, uint32_t i, uint32_t p,
                                               uint32_t k0, uint32_t k1) {
  const uint32_t pair = q >> 1;
  const U4 b = philox4x32_10(pair >> 1, kk, i, p, k0, k1);
  const bool hi = pair & 1u;
  float g0, g1;
  box_muller32(u24(hi ? b.z : b.x), u24(hi ? b.w : b.y), g0, g1);
  return (q & 1u) ? g1 : g0;
}

template <int MK>
__global__ void __launch_bounds__(256) walk3_f32_kernel(const DevProblem pb) {
  const int64_t total = pb.P * pb.N;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t w = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (w >= total) return;
  const uint32_t k0 = static_cast<uint32_t>(pb.seed), k1 = static_cast<uint32_t>(pb.seed >> 32);
  const int nv = pb.n_v;
  const float eps = static_cast<float>(pb.eps);
  const float theta = static_cast<float>(pb.theta);
  const float rgeo = static_cast<float>(pb.rho_geo);
  const float sqs = static_cast<float>(pb.sqrt_sigma);

  float Y[3];
  double W = 1.0, S = 0.0;
  int64_t k = 0;
  uint32_t p = 0, i = 0;
  auto init = [&](int64_t ww) {
    p = static_cast<uint32_t>(ww / pb.N);
    i = static_cast<uint32_t>(ww - static_cast<int64_t>(p) * pb.N);
    const double* y0 = pb.pts + static_cast<size_t>(p) * 3;
    Y[0] = static_cast<float>(y0[0]); Y[1] = static_cast<float>(y0[1]); Y[2] = static_cast<float>(y0[2]);
    W = 1.0; S = 0.0; k = 0;
  };
  init(w);
  float r_prev = -1.0f;
  double c = 1.0, omega = 0.0;

  for (;;) {
    float dG = INFINITY;
    bool done = false;
    int flag = 0;
    if (!pb.closed) {
      float yg[3];
      dG = delta_gamma3<MK, float>(pb, Y, yg);
      if (dG < eps) {
        S += W * static_cast<double>(func3<MK, float>(pb, pb.g, yg));
        done = true;
      } else if (W == 0.0) {
        done = true;
      }
    } else if (W < pb.tau_w) {
      done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      pb.S_out[w] = S;
      pb.K_out[w] = static_cast<int32_t>(k);
      pb.flag_out[w] = flag;
      w += stride;
      if (w >= total) break;
      init(w);
      continue;
    }
    const float r = theta * (dG < rgeo ? dG : rgeo);
    const float a = sqs * r;
    if (r != r_prev) {   // constant-radius walks compute the weights once
      const double ad = static_cast<double>(a);
      const double em1 = em1_series(0.5, 0.25 * (ad * ad));
      c = 1.0 / (1.0 + em1);
      omega = one_minus_c(em1, c) / pb.sigma;
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    float Th[3], F = 0.0f;
    if (nv == 1) {
      const U4 b0 = philox4x32_10(0u, kk, i, p, k0, k1);
      const U4 b1 = philox4x32_10(1u, kk, i, p, k0, k1);
      float g[3], z[3];
      box_muller32(u24(b0.x), u24(b0.y), g[0], g[1]);
      box_muller32(u24(b0.z), u24(b0.w), g[2], z[0]);
      box_muller32(u24(b1.x), u24(b1.y), z[1], z[2]);
      const float U = u24(b1.z);
      const float sc = r * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + sc * g[q];
      float t = table_lookup<float>(pb.tab32, pb.NA, pb.NS, pb.z_max, a, s_of_u32(U));
      t = fminf(fmaxf(t, 0.0f), 1.0f);
      const float zs = (r * t) * rsqrtf(fmaxf(dot3(z, z), 1e-30f));
      float Z[3], cZ[3];
      for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * z[q];
      cp3<MK, float>(pb, Z, cZ);
      F = func3<MK, float>(pb, pb.f, cZ);
    } else {
      float g[3];
      for (int q = 0; q < 3; ++q) g[q] = gaussian_at32(static_cast<uint32_t>(q), kk, i, p, k0, k1);
      const float sc = r * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
      for (int q = 0; q < 3; ++q) Th[q] = Y[q] + sc * g[q];
      const uint32_t nu = 2u * ((3u * static_cast<uint32_t>(1 + nv) + 1u) / 2u);
      for (int l = 0; l < nv; ++l) {
        const float U = uniform_at32(nu + static_cast<uint32_t>(l), kk, i, p, k0, k1);
        float t = table_lookup<float>(pb.tab32, pb.NA, pb.NS, pb.z_max, a, s_of_u32(U));
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        for (int q = 0; q < 3; ++q)
          g[q] = gaussian_at32(3u * static_cast<uint32_t>(1 + l) + static_cast<uint32_t>(q), kk, i, p, k0, k1);
        const float zs = (r * t) * rsqrtf(fmaxf(dot3(g, g), 1e-30f));
        float Z[3], cZ[3];
        for (int q = 0; q < 3; ++q) Z[q] = Y[q] + zs * g[q];
        cp3<MK, float>(pb, Z, cZ);
        F += func3<MK, float>(pb, pb.f, cZ);
      }
      F /= static_cast<float>(nv);
    }
    S += (W * omega) * static_cast<double>(F);
    W *= c;
    cp3<MK, float>(pb, Th, Y);
    ++k;
  }
}

}  // namespace mpwos
