// dev_common.cuh — device-side problem description, Philox4x32-10 and the
// uniform / Gaussian transforms shared by every walk kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpwos {

constexpr int kMaxTerms = 32;       // terms of a POLY / TORUS function
constexpr int kMaxPolyFactors = 64; // total (var, pow) factors of a POLY
constexpr int kMaxQuadDim = 32;     // d + 1 of a SPHERE_QUAD / embedded sphere

enum ManifoldKind : int { kEuclid = 0, kSphere = 1, kTorus = 2, kEmbeddedSphere = 3, kPointCloud = 4, kRevolution = 5,
                          kCurveSphere = 6 };
enum FuncKind : int { kPoly = 0, kTorusFourier = 1, kSphereQuad = 2, kRevolutionQuad = 3, kCurveSphereFunc = 4 };

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
  float coef_f[kMaxTerms];             // FP32 copies of coef, c0 (the FP32 walks read no double)
  float c0_f;
  float mode_f[kMaxTerms][4];          // TORUS_FOURIER: m, q, m^2, q^2 as floats
  int single_mq;                       // TORUS_FOURIER with one term, m, q <= 3: 4 m + q + 16 [sin in theta]
                                       // + 32 [sin in phi]; else -1
};

// Compensation term m_* (Sec. 2.3.3): the predictor u_* and the difference
// step.  Torus: a Fourier series (m, q, theta trig, phi trig per term); unit
// sphere of R^3: u_* = c0 + v.y + y^T A y.  FP32 walks read the float copies
// and the launch constants sd1, sd2 (sphere: the central differences of
// (1 + s)^-2 at s = 0 with step h, from FP64 on the host).
constexpr int kMaxPredTerms = 64;
constexpr int kCompNone = 0, kCompNormal2 = 1, kCompExact = 2;
struct DevPredictor {
  int comp, kind, n_terms;
  double h;
  double coef[kMaxPredTerms];
  int8_t modes[kMaxPredTerms][4];
  double c0, v[3], A[9];
  float coef_f[kMaxPredTerms];
  float mode_f[kMaxPredTerms][2];   // m, q
  float c0_f, v_f[3], A_f[9];
  float hf, sd1, sd2;
};

// FP32 copies of the loop-invariant scalars, filled on the host: a double read
// in an FP32 walk costs a conversion on B300's narrow FP64 pipe every step.
struct ScalarsF {
  float eps, theta, rho_geo, sqrt_sigma, sigma, inv_sigma, R, a, inv_a, h, sh, c_h;
  float tab_scale;   // (NS - 1) / sqrt(1/2): table abscissa per sqrt(U)
  float z_scale;     // (NA - 1) / z_max (0 when NA == 1)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

// Round keys of one seed: k_r = (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85), r = 0..9.
struct PhiloxKeys { uint32_t a[10], b[10]; };

// Everything a walk kernel reads, passed by value (kernel parameter space).
struct DevProblem {
  // manifold
  int mkind, n, d;
  double R, a_tube;
  const double* Q;    // embedded sphere: Q^T, (d+1) rows of npad = n rounded up to 4, device
  const double* b;
  const float* Qf;    // FP32 Q^T in the warp walk's group order: (d+1) rows of 1024
  const float* bf;
  // point cloud: points sorted by grid cell (xyz interleaved), original
  // indices, cell start offsets (cells + 1), grid origin / cell size / dims
  const double* cl_pts64;
  const float* cl_pts32;
  const int* cl_orig;
  const int* cl_start;
  double cl_origin[3];
  double cl_cell;
  float cl_origin_f[3];
  float cl_cell_f;
  int cl_dims[3];
  int cl_k;          // neighbours (k_nn)
  double cl_c_h;     // rho_geo = c_h h(y)
  int cl_mode;       // 0: quadratic fit projection, 1: nearest point
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
  PhiloxKeys keys;   // round keys of seed (host-made; read as constant operands)
  ScalarsF sf;
  // FP32 survival weight: em1(z) = I~_nu(a) - 1 = sum_{j=1..T} k_j z^j (Lemma 3.1
  // series, coefficients k_j = 1/(j! (nu+1)_j) from FP64 on the host, T chosen
  // so the truncation is below 1e-9 relative at z_max); em1_fp64 = 1 when T
  // terms do not suffice (the FP32 walk then uses the FP64 series).
  float em1_k[32];
  int em1_terms;
  int em1_fp64;
  // radius tables (inverse CDF of the Green law; layout in green.cuh)
  const double* tab64;
  const float4* tabc;  // FP32 walks: per interval the cubic c0 + c1 f + c2 f^2 + c3 f^3 (NS - 1 per side)
  int NA, NS;         // a-rows (uniform in z = a^2/4), s-nodes (+2 ghosts per row)
  double z_max;
  // work map: walk (p, i) for p in wk_points (all points 0..P-1 when null),
  // i in [wk_i0, wk_i1); this launch covers enumeration indices [wk_w0, wk_w1)
  // of the wk_np * (wk_i1 - wk_i0) walks; outputs at p * out_stride + i - out_i0
  const int* wk_points;
  int64_t wk_np, wk_i0, wk_i1, wk_w0, wk_w1, out_stride;
  // queries and outputs
  int64_t P, N;
  const double* pts;  // P x n
  const double* s0;   // embedded sphere: P x (d+1) intrinsic start points (or null)
  double* S_out;
  int32_t* K_out;
  int32_t* flag_out;
  // tensor-core embedded walk: Q^T as BF16 hi + lo in the kernel's swizzled
  // shared-memory image (128 KB), and a status word (bit 0: a wait ran out)
  const uint4* tc_bimg;
  unsigned* dev_status;
  // dimension-reduced exact sampler: tracked coordinates (count, normal on
  // them), chi^2 degrees of freedom of the rest, per-point start states
  // (row p: y_T in kMaxQuadDim slots, then |y_rest|; host-made from the points)
  int reduced;
  int red_nT, red_rest;
  double red_e[kMaxQuadDim];
  float red_ef[kMaxQuadDim];
  const double* red_y0;
  // compensation term (last, so the fields above keep their offsets)
  DevPredictor pred;
  // hypersurface of revolution: profile parameters, c_kappa, tr(A)/(n-1) of f
  double rv_alpha, rv_kappa, rv_mA;
  float rv_alpha_f, rv_kappa_f, rv_mA_f, rv_ck_f;
  // dynamic walk queue (zeroed before each launch; null: static stride)
  unsigned long long* wk_next;
  // point cloud in cell order as FP32 (x, y, z, original index as int bits):
  // one 16-byte load per candidate in the FP32 searches
  const float4* cl_pts4;
  // FP32 warp walk in R^n (n > 3): the walk's coordinate order, perm[c] = the
  // ambient index of walk coordinate c (null: identity), chosen so that the
  // coordinates f, g and the boundary normal read come first; the normal's
  // first 128 walk coordinates, and the whole normal in walk order when it has
  // others (ef_w, zero padded to 1024; null otherwise); the hypersurface of
  // revolution's v and diag(A) in walk order (the axis is walk coordinate 0,
  // zero there), zero padded to 1024
  const int* perm;
  const float* ef_w;
  const float* rv_v32;
  const float* rv_a32;
  float e_s0[128];
  // output slot of walk (p, i): p * out_stride + i - out_i0 (a walk range's own buffer)
  int64_t out_i0;
  // the warp-cooperative point-cloud walk: one walker per cl_spread lanes (1 ..
  // 32, a power of two), so that a launch of few walks spreads over more warps
  int cl_spread;
};

__host__ __device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    K.a[r] = k0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
    K.b[r] = k1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
  }
  return K;
}

__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                      const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c0;
    const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c1 ^ K.a[r];
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c3 ^ K.b[r];
    c0 = n0; c1 = static_cast<uint32_t>(p1); c2 = n2; c3 = static_cast<uint32_t>(p0);
  }
  return U4{c0, c1, c2, c3};
}

// The two blocks j = 0, 1 of counter (j, k, i, p) for every step k of one walk
// (i, p), with the work that depends on (i, p) only done once per walk and
// the work both blocks share done once per step.  Writing one Philox round as
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ a_r, lo(M1 c2), hi(M0 c0) ^ c3 ^ b_r, lo(M0 c0)),
// round 0 of block j gives (hi(M1 i) ^ k ^ a_0, lo(M1 i), p ^ b_0, j M0) since
// M0 j < 2^32; round 1 then has a per-walk c0, c1 and a per-step c3, and the
// blocks differ only in c2 (by M0); round 2 shares c2, c3; rounds 3..9 run in
// full.  Output is identical to philox4x32_10(j, k, i, p, K).
struct PhiloxWalk {
  uint32_t x0;    // hi(M1 i) ^ a_0 (round 0 c0 before the step index)
  uint32_t A, L;  // round 1 c0, c1
  uint32_t HA;    // hi(M0 A) ^ b_2
  uint32_t LA;    // lo(M0 A)
};

__host__ __device__ __forceinline__ PhiloxWalk philox_walk(uint32_t i, uint32_t p, const PhiloxKeys& K) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  PhiloxWalk w;
  const uint64_t pi = static_cast<uint64_t>(M1) * i;
  w.x0 = static_cast<uint32_t>(pi >> 32) ^ K.a[0];
  const uint64_t pp = static_cast<uint64_t>(M1) * (p ^ K.b[0]);
  w.A = static_cast<uint32_t>(pp >> 32) ^ static_cast<uint32_t>(pi) ^ K.a[1];
  w.L = static_cast<uint32_t>(pp);
  const uint64_t pa = static_cast<uint64_t>(M0) * w.A;
  w.HA = static_cast<uint32_t>(pa >> 32) ^ K.b[2];
  w.LA = static_cast<uint32_t>(pa);
  return w;
}

__host__ __device__ __forceinline__ void philox_step_pair(const PhiloxWalk& w, uint32_t k, const PhiloxKeys& K,
                                                          U4& out0, U4& out1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  // round 1 (shared product of the step)
  const uint64_t P = static_cast<uint64_t>(M0) * (w.x0 ^ k);
  const uint32_t c2_0 = static_cast<uint32_t>(P >> 32) ^ K.b[1];
  const uint32_t c2_1 = c2_0 ^ M0;
  // round 2
  const uint64_t q0 = static_cast<uint64_t>(M1) * c2_0;
  const uint64_t q1 = static_cast<uint64_t>(M1) * c2_1;
  uint32_t a0 = static_cast<uint32_t>(q0 >> 32) ^ w.L ^ K.a[2], a1 = static_cast<uint32_t>(q0);
  uint32_t b0 = static_cast<uint32_t>(q1 >> 32) ^ w.L ^ K.a[2], b1 = static_cast<uint32_t>(q1);
  uint32_t a2 = w.HA ^ static_cast<uint32_t>(P), a3 = w.LA;
  uint32_t b2 = a2, b3 = a3;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t pa0 = static_cast<uint64_t>(M0) * a0, pa1 = static_cast<uint64_t>(M1) * a2;
    const uint64_t pb0 = static_cast<uint64_t>(M0) * b0, pb1 = static_cast<uint64_t>(M1) * b2;
    const uint32_t na0 = static_cast<uint32_t>(pa1 >> 32) ^ a1 ^ K.a[r];
    const uint32_t na2 = static_cast<uint32_t>(pa0 >> 32) ^ a3 ^ K.b[r];
    const uint32_t nb0 = static_cast<uint32_t>(pb1 >> 32) ^ b1 ^ K.a[r];
    const uint32_t nb2 = static_cast<uint32_t>(pb0 >> 32) ^ b3 ^ K.b[r];
    a0 = na0; a1 = static_cast<uint32_t>(pa1); a2 = na2; a3 = static_cast<uint32_t>(pa0);
    b0 = nb0; b1 = static_cast<uint32_t>(pb1); b2 = nb2; b3 = static_cast<uint32_t>(pb0);
  }
  out0 = U4{a0, a1, a2, a3};
  out1 = U4{b0, b1, b2, b3};
}

// Block j = 0 of step k alone, with the same hoisting as philox_step_pair.
__host__ __device__ __forceinline__ U4 philox_step_one(const PhiloxWalk& w, uint32_t k, const PhiloxKeys& K) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint64_t P = static_cast<uint64_t>(M0) * (w.x0 ^ k);
  const uint32_t c2 = static_cast<uint32_t>(P >> 32) ^ K.b[1];
  const uint64_t q = static_cast<uint64_t>(M1) * c2;
  uint32_t a0 = static_cast<uint32_t>(q >> 32) ^ w.L ^ K.a[2], a1 = static_cast<uint32_t>(q);
  uint32_t a2 = w.HA ^ static_cast<uint32_t>(P), a3 = w.LA;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t pa0 = static_cast<uint64_t>(M0) * a0, pa1 = static_cast<uint64_t>(M1) * a2;
    const uint32_t na0 = static_cast<uint32_t>(pa1 >> 32) ^ a1 ^ K.a[r];
    const uint32_t na2 = static_cast<uint32_t>(pa0 >> 32) ^ a3 ^ K.b[r];
    a0 = na0; a1 = static_cast<uint32_t>(pa1); a2 = na2; a3 = static_cast<uint32_t>(pa0);
  }
  return U4{a0, a1, a2, a3};
}

// FP32 walks in R^n (n > 3): block j of step k of walk (p, i) is Philox4x32-10
// at counter (k, j, i, p).  With j in the XOR slot of round 0, every block of a
// step shares the rest of rounds 0..2:
//   round 0: (H1(i) ^ a_0 ^ j, L1(i), H0(k) ^ p ^ b_0, L0(k))      [H, L: hi, lo of M1 x or M0 x]
//   round 1: (A1, B1, H0(A0 ^ j) ^ L0(k) ^ b_1, L0(A0 ^ j)),  A1 = H1(C0) ^ L1(i) ^ a_1, B1 = L1(C0)
//   round 2: (H1(t2) ^ B1 ^ a_2, L1(t2), H0(A1) ^ b_2 ^ L0(A0 ^ j), L0(A1))
// so a block costs two wide multiplies and four XORs before rounds 3..9 (34
// operations instead of 40).  A walk's blocks j = 256 v + b (v: the vector,
// b < 256: its 4-component block) keep j's low byte free, so A0 ^ j =
// (A0 ^ 256 v ^ lane) ^ 32 m for the lane-interleaved blocks b = lane + 32 m.
struct Philox32Walk { uint32_t A0, B0; };
struct Philox32Step { uint32_t D1x, B2x, E2, La; };

__host__ __device__ __forceinline__ Philox32Walk philox32_walk(uint32_t i, const PhiloxKeys& K) {
  const uint64_t q = static_cast<uint64_t>(0xCD9E8D57u) * i;
  return Philox32Walk{static_cast<uint32_t>(q >> 32) ^ K.a[0], static_cast<uint32_t>(q)};
}

__host__ __device__ __forceinline__ Philox32Step philox32_step(const Philox32Walk& w, uint32_t k, uint32_t p,
                                                              const PhiloxKeys& K) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint64_t pk = static_cast<uint64_t>(M0) * k;
  const uint32_t C0 = static_cast<uint32_t>(pk >> 32) ^ p ^ K.b[0];
  const uint64_t pc = static_cast<uint64_t>(M1) * C0;
  const uint32_t A1 = static_cast<uint32_t>(pc >> 32) ^ w.B0 ^ K.a[1];
  const uint64_t pa = static_cast<uint64_t>(M0) * A1;
  Philox32Step s;
  s.D1x = static_cast<uint32_t>(pk) ^ K.b[1];
  s.B2x = static_cast<uint32_t>(pc) ^ K.a[2];
  s.E2 = static_cast<uint32_t>(pa >> 32) ^ K.b[2];
  s.La = static_cast<uint32_t>(pa);
  return s;
}

// The block whose round-0 first word is s0 = A0 ^ j.
__host__ __device__ __forceinline__ U4 philox32_block(uint32_t s0, const Philox32Step& s, const PhiloxKeys& K) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint64_t pj = static_cast<uint64_t>(M0) * s0;
  const uint32_t t2 = static_cast<uint32_t>(pj >> 32) ^ s.D1x;
  const uint64_t pq = static_cast<uint64_t>(M1) * t2;
  uint32_t x0 = static_cast<uint32_t>(pq >> 32) ^ s.B2x, x1 = static_cast<uint32_t>(pq);
  uint32_t x2 = s.E2 ^ static_cast<uint32_t>(pj), x3 = s.La;
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t p0 = static_cast<uint64_t>(M0) * x0, p1 = static_cast<uint64_t>(M1) * x2;
    const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ x1 ^ K.a[r];
    const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ x3 ^ K.b[r];
    x0 = n0; x1 = static_cast<uint32_t>(p1); x2 = n2; x3 = static_cast<uint32_t>(p0);
  }
  return U4{x0, x1, x2, x3};
}

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

// 23-bit uniform in (0, 1] from one word without an int->float conversion:
// 2 - [1, 2) built from the low 23 bits as a float mantissa (one logic op).
__device__ __forceinline__ float u23(uint32_t x) {
  return 2.0f - __uint_as_float(0x3f800000u | (x & 0x7FFFFFu));
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
// The fifth 23-bit uniform of a block whose four words' low 23 bits are already
// used: bits 24..31 of x and y and bits 24..30 of z (disjoint from those), the
// top bytes gathered by two byte permutes.
__device__ __forceinline__ float u23_high(const U4& b) {
  const uint32_t xy = __byte_perm(b.x, b.y, 0x0073u);   // bytes: x.b3, y.b3, x.b0, x.b0
  return u23(__byte_perm(xy, b.z, 0x0710u));            // bytes: x.b3, y.b3, z.b3, x.b3
}

// A uniform direction on S^2 from two uniforms in (0, 1] (Archimedes: the height
// of a uniform point of the unit sphere is uniform on [-1, 1] and independent of
// its azimuth): z = 2 uz - 1, sqrt(1 - z^2) = 2 sqrt(uz (1 - uz)), azimuth 2 pi uphi.
// The same law as a normalised Gaussian 3-vector, from two uniforms instead of
// three Gaussians and a norm.
__device__ __forceinline__ void sphere_dir3(float uz, float uphi, float (&d)[3]) {
  const float s = 2.0f * sqrtf(fmaf(-uz, uz, uz));
  float sn, cs;
  __sincosf(kTwoPiF * uphi, &sn, &cs);
  d[0] = s * cs;
  d[1] = s * sn;
  d[2] = fmaf(2.0f, uz, -1.0f);
}

__device__ __forceinline__ void box_muller32(float ua, float ub, float& g0, float& g1) {
  const float rad = sqrtf(-1.38629436111989061f * __log2f(ua));   // -2 ln(ua) = -2 ln2 log2(ua)
  float s, c;
  __sincosf(kTwoPiF * ub, &s, &c);
  g0 = rad * c;
  g1 = rad * s;
}

// Box-Muller for a direction (FP32 walks in R^n): two components of the
// Gaussian vector up to the common factor sqrt(2 ln 2), which the normalised
// direction g/|g| does not see: sqrt(-log2 u) (cos 2 pi v, sin 2 pi v), u in
// (0, 1] from the low 23 bits of x and v in [1, 2) from the low 23 bits of y
// (sine and cosine have period 1 in v).  Returns -log2 u, the pair's part of
// |g|^2 (cos^2 + sin^2 = 1), so a norm needs no squares.
__device__ __forceinline__ float gauss_pair32(uint32_t x, uint32_t y, float& g0, float& g1) {
  const float u = 2.0f - __uint_as_float(0x3f800000u | (x & 0x7FFFFFu));
  const float l = __log2f(u);
  const float R = sqrtf(-l);
  float s, c;
  __sincosf(kTwoPiF * __uint_as_float(0x3f800000u | (y & 0x7FFFFFu)), &s, &c);
  g0 = R * c;
  g1 = R * s;
  return -l;
}

// Radial half of one block: R = sqrt(-log2 u) of four pairs; returns the sum
// of -log2 u.
__device__ __forceinline__ float radial4(const U4& r, float* R) {
  const uint32_t w[4] = {r.x, r.y, r.z, r.w};
  float sl = 0.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float u = 2.0f - __uint_as_float(0x3f800000u | (w[k] & 0x7FFFFFu));
    const float l = __log2f(u);
    R[k] = sqrtf(-l);
    sl -= l;
  }
  return sl;
}

// Angle halves: the group's 16 components g[2q] = R_q cos, g[2q+1] = R_q sin,
// angle of pair 2k from the low and of pair 2k + 1 from the high 16 bits of
// word k (as the fraction bits of a float in [1, 2): sine and cosine have
// period 1 there).
__device__ __forceinline__ void angle8(const U4& a, const float (&R)[8], float (&g)[16]) {
  const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float s, c;
    __sincosf(kTwoPiF * __uint_as_float(0x3f800000u | ((w[k] << 7) & 0x7FFF80u)), &s, &c);
    g[4 * k] = R[2 * k] * c;
    g[4 * k + 1] = R[2 * k] * s;
    __sincosf(kTwoPiF * __uint_as_float(0x3f800000u | ((w[k] >> 9) & 0x7FFF80u)), &s, &c);
    g[4 * k + 2] = R[2 * k + 1] * c;
    g[4 * k + 3] = R[2 * k + 1] * s;
  }
}

// One group of 16 direction components, 16 G .. 16 G + 15, of the FP32 walks in
// R^n (n > 3): radial words from blocks j = 4 G and 4 G + 1 (pairs 8 G + 0..7),
// angle halves from block 4 G + 2, each pair sqrt(-log2 u) (cos 2 pi a, sin
// 2 pi a) with a 16-bit angle a; X = A0 ^ 256 v selects the vector (philox32_block
// then runs at counter (k, 256 v + 4 G + c, i, p)).  Components past n are zero;
// returns the sum of squares of the group's components.
__device__ __forceinline__ float gauss_group16(uint32_t X, int G, const Philox32Step& st, const PhiloxKeys& K,
                                               int n, float (&g)[16]) {
  float R[8];
  const uint32_t j = static_cast<uint32_t>(4 * G);
  const float sl = radial4(philox32_block(X ^ j, st, K), R) + radial4(philox32_block(X ^ (j + 1u), st, K), R + 4);
  angle8(philox32_block(X ^ (j + 2u), st, K), R, g);
  const int valid = n - 16 * G;
  if (valid >= 16) return sl;
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    g[q] = q < valid ? g[q] : 0.0f;
    s += g[q] * g[q];
  }
  return s;
}

// ---------------------------------------------------------------------------
// Pairs of floats (hi + lo, |lo| <= ulp(hi)/2) with error-free transformations
// (Knuth TwoSum, FMA TwoProd): about 46-48 bits of significand (~2^-46
// relative per operation, less than FP64's 2^-53) on the FP32 pipes.
// Used for each walk's running weight W and score S in the FP32 walk, where
// B300's FP64 pipe (about 1/64 of the FP32 rate) would otherwise co-limit the
// step; per-point sums over walks stay in FP64.
// ---------------------------------------------------------------------------
// The double or the host-made float copy of a scalar, by walk precision.
template <typename T> __device__ __forceinline__ T pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// The walk a thread (or warp) takes after walk w.  With a queue counter the
// first walk of each of the `stride` threads is static and every later one is
// taken from the counter, so threads whose walks end early take more walks and
// walks of uneven length keep the lanes busy; without one, the static stride.
// Either way each enumeration index is walked once, and a walk's draws depend
// on (seed, point, walk index) only.
__device__ __forceinline__ int64_t next_walk(const DevProblem& pb, int64_t w, int64_t stride) {
  if (pb.wk_next) return pb.wk_w0 + stride + static_cast<int64_t>(atomicAdd(pb.wk_next, 1ull));
  return w + stride;
}

// Walk enumeration index -> (point, walk index, output slot).
struct WalkId {
  uint32_t p, i;
  int64_t o;
};

__device__ __forceinline__ WalkId walk_id(const DevProblem& pb, int64_t w) {
  const int64_t nw = pb.wk_i1 - pb.wk_i0;
  const int64_t r = w / nw;
  WalkId id;
  id.p = static_cast<uint32_t>(pb.wk_points ? pb.wk_points[r] : r);
  id.i = static_cast<uint32_t>(pb.wk_i0 + (w - r * nw));
  id.o = static_cast<int64_t>(id.p) * pb.out_stride + id.i - pb.out_i0;
  return id;
}

struct F2 { float hi, lo; };

// c = 1 / (1 + em1) as a float pair and omega = (1 - c)/sigma, from an FP32
// em1.  For em1 <= 1, c = 1 - delta with delta = em1/(1 + em1) held exactly
// as (hi, lo); otherwise c = 1/(1 + em1) directly.
__device__ __forceinline__ void weights_from_em1(float em1, float inv_sigma, F2& c, F2& om) {
  if (em1 <= 1.0f) {
    const float delta = __fdividef(em1, 1.0f + em1);
    const float hi = __fadd_rn(1.0f, -delta);
    c = F2{hi, __fadd_rn(__fadd_rn(1.0f, -hi), -delta)};
    om = F2{delta * inv_sigma, 0.0f};
  } else {
    const float cc = __fdividef(1.0f, 1.0f + em1);
    c = F2{cc, 0.0f};
    om = F2{(1.0f - cc) * inv_sigma, 0.0f};
  }
}

__device__ __forceinline__ F2 f2_from_double(double x) {
  const float hi = static_cast<float>(x);
  return F2{hi, static_cast<float>(x - static_cast<double>(hi))};
}
__device__ __forceinline__ double f2_to_double(F2 x) {
  return static_cast<double>(x.hi) + static_cast<double>(x.lo);
}
__device__ __forceinline__ F2 f2_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return F2{s, __fadd_rn(b, -__fadd_rn(s, -a))};
}
__device__ __forceinline__ F2 f2_mul(F2 x, F2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return f2_fast_two_sum(p, e);
}
__device__ __forceinline__ F2 f2_mul_f(F2 x, float f) {
  const float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return f2_fast_two_sum(p, e);
}
__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fadd_rn(s, -x.hi);
  const float err = __fadd_rn(__fadd_rn(x.hi, -__fadd_rn(s, -bb)), __fadd_rn(y.hi, -bb));
  return f2_fast_two_sum(s, __fadd_rn(err, __fadd_rn(x.lo, y.lo)));
}

}  // namespace mpwos
