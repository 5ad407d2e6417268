// dev_common.cuh — device-side problem description, Philox4x32-10 and the
// uniform / Gaussian transforms shared by every walk kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpwos {

constexpr int kMaxTerms = 32;       // terms of a POLY / TORUS function
constexpr int kMaxPolyFactors = 64; // total (var, pow) factors of a POLY
constexpr int kMaxQuadDim = 32;     // d + 1 of a SPHERE_QUAD / embedded sphere

enum ManifoldKind : int { kEuclid = 0, kSphere = 1, kTorus = 2, kEmbeddedSphere = 3 };
enum FuncKind : int { kPoly = 0, kTorusFourier = 1, kSphereQuad = 2 };

// A function on M (f or g), copied by value into the kernel parameters.
struct DevFunc {
  int kind, apply_op, n_terms;
  double coef[kMaxTerms];
  int16_t term_off[kMaxTerms + 1];
  int16_t var[kMaxPolyFactors];
  int8_t pw[kMaxPolyFactors];
  int8_t modes[kMaxTerms][4];          // m, q, theta trig, phi trig
  double c0;
  const double* v;                     // device, d + 1
  const double* A;                     // device, (d + 1)^2
  const float* vf;                     // float copies
  const float* Af;
};

// Everything a walk kernel reads, passed by value (kernel parameter space).
struct DevProblem {
  // manifold
  int mkind, n, d;
  double R, a_tube;
  const double* Q;    // n x (d+1) row-major (embedded sphere), device
  const double* b;
  const float* Qf;
  const float* bf;
  // problem
  double sigma, sqrt_sigma;
  int closed;
  const double* e;    // boundary normal, device (n)
  const float* ef;
  double h;
  DevFunc f, g;
  // parameters
  double eps, tau_w, theta, c_kappa, kappa, rho_geo;
  int n_v;
  int64_t max_steps;
  uint64_t seed;
  // radius tables (inverse CDF of the Green density in s = (2/pi) asin(sqrt U))
  const double* tab64;
  const float* tab32;
  int NA, NS;         // a-rows (uniform in z = a^2/4), s-nodes (+2 ghosts per row)
  double z_max;
  // queries and outputs
  int64_t P, N;
  const double* pts;  // P x n
  const double* s0;   // embedded sphere: P x (d+1) intrinsic start points (or null)
  double* S_out;
  int32_t* K_out;
  int32_t* flag_out;
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                             uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// 53-bit uniform in (0, 1] from two words (top 53 bits of hi:lo, plus one).
__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((static_cast<uint64_t>(hi) << 32) | lo) >> 11;
  return static_cast<double>(m + 1ull) * 0x1p-53;
}

// 24-bit uniform in (0, 1] from one word.
__device__ __forceinline__ float u24(uint32_t x) {
  return static_cast<float>((x >> 8) + 1u) * 0x1p-24f;
}

constexpr double kTwoPi = 6.283185307179586;
constexpr float kTwoPiF = 6.28318530717958648f;

// FP64 Box-Muller pair from two 53-bit uniforms.
__device__ __forceinline__ void box_muller64(double ua, double ub, double& g0, double& g1) {
  const double rad = sqrt(-2.0 * log(ua));
  const double ang = kTwoPi * ub;
  double s, c;
  sincos(ang, &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

// FP32 Box-Muller pair (hardware approximations: MUFU lg2 / sin / cos).
__device__ __forceinline__ void box_muller32(float ua, float ub, float& g0, float& g1) {
  const float rad = sqrtf(-2.0f * __logf(ua));
  float s, c;
  __sincosf(kTwoPiF * ub, &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

}  // namespace mpwos
