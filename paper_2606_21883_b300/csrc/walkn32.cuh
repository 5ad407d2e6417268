// walkn32.cuh — the FP32 MPWoS walk in R^n (3 < n <= 1024), one warp per walker.
//
// Layout.  The walker's n-vectors live in registers, spread over the 32 lanes
// in 4-component blocks: block b (components 4b .. 4b + 3) belongs to lane
// b mod 32, register slot b / 32 (MB slots, n <= 128 MB).  A lane generates
// exactly the Gaussians of the components it owns; norms and dot products are
// per-lane partial sums and one butterfly reduction.
//
// Draws of step k of walk (p, i): Philox4x32-10 at counter (k, j, i, p),
//   Theta direction: j = b;  Z_l direction: j = 256 (1 + l) + b (the embedded
//   sphere instead draws in 16-component groups, gen_groups, the layout of the
//   tensor-core walk and of walkn32s.cuh);
//   U_l = u23(word l mod 4) of block j = 256 (1 + N_V) + l / 4,
// the per-walk and per-step parts of rounds 0..2 computed once (dev_common.cuh,
// Philox32Step), each word pair giving two components sqrt(-log2 u)(cos, sin)
// of the Gaussian vector up to one common factor (gauss_pair32) and its share of
// |g|^2.  The tensor-core walk (embed_tc.cuh) draws the same numbers.
//
// Coordinates.  The walk runs in a coordinate order chosen by the host (perm):
// the coordinates that f, g and the boundary normal e read come first, so they
// all sit in slot 0 of the first lanes, which publish slot 0 of Y and of the
// last Gaussian vector to shared memory; the hypersurface of revolution puts
// its axis first.  The walk law is invariant under a permutation of the
// ambient coordinates (the Gaussian components are i.i.d.).
//
// State.  Y = lambda Yh with lambda warp-uniform: the sphere step
// Y' = (Y + sc g)/|Y + sc g| becomes Yh += (sc/lambda) g (one FMA per
// component) and lambda' = 1/|Yh'|, with |Yh|^2 and e.Yh carried from the
// step's reductions and recomputed exactly every 64 steps (when Yh is also
// rescaled to lambda = 1).  The hypersurface of revolution scales the
// non-axis part the same way, to the profile radius R(t).
#pragma once
#include "dev_common.cuh"
#include "green.cuh"
#include "revolution.cuh"
#include "curve_sphere.cuh"
#include "walkn.cuh"

namespace mpwos {
namespace w32 {

constexpr int kThreads = 128;   // block size bound: 4 warps, each with its shared row

struct WarpRow {
  float y[128];   // slot 0 of Yh (all lanes)
  float g[128];   // slot 0 of the last Gaussian vector
};

// The lane's components of one Gaussian vector (blocks b = lane + 32 m with
// X = A0 ^ 256 v ^ lane) into g; returns the lane's part of |g|^2.  nbf: full
// blocks (n / 4); rem = n mod 4 components of block nbf.
template <int MB>
__device__ __forceinline__ float gen_vec(float (&g)[4 * MB], uint32_t X, const Philox32Step& st,
                                         const PhiloxKeys& K, int lane, int nbf, int rem) {
  float sl = 0.0f;
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = lane + 32 * m;
    if (b < nbf || (b == nbf && rem)) {
      const U4 r = philox32_block(X ^ static_cast<uint32_t>(32 * m), st, K);
      const float l0 = gauss_pair32(r.x, r.y, g[4 * m], g[4 * m + 1]);
      const float l1 = gauss_pair32(r.z, r.w, g[4 * m + 2], g[4 * m + 3]);
      if (b < nbf) {
        sl += l0 + l1;
      } else {   // the partial last block: components past n are zero
        g[4 * m + 3] = 0.0f;
        if (rem < 3) g[4 * m + 2] = 0.0f;
        if (rem < 2) g[4 * m + 1] = 0.0f;
        sl += g[4 * m] * g[4 * m] + g[4 * m + 1] * g[4 * m + 1] + g[4 * m + 2] * g[4 * m + 2];
      }
    } else {
      g[4 * m] = g[4 * m + 1] = g[4 * m + 2] = g[4 * m + 3] = 0.0f;
    }
  }
  return sl;
}

// POLY at x_v = (ya ys[v] + gb gs[v]) inv (walk coordinates v < 128).
__device__ __forceinline__ float poly_rows(const DevFunc& fn, const float* ys, const float* gs, float ya, float gb,
                                           float inv) {
  float total = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    float prod = fn.coef_f[t];
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const float xv = (ya * ys[v] + gb * gs[v]) * inv;
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// POLY at y_Gamma = ya ys + ye e (walk coordinates v < 128).
__device__ __forceinline__ float poly_bnd(const DevFunc& fn, const float* ys, const float* es, float ya, float ye) {
  float total = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    float prod = fn.coef_f[t];
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const float xv = ya * ys[v] + ye * es[v];
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

template <int NV>
__device__ __forceinline__ void wsum(float (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
}

// The embedded sphere's draws in 16-component groups (the layout of the FP32
// walk in R^n, gauss_group16): lane owns groups G = lane + 32 s, s < MB / 4,
// components 16 G + q in g[16 s + q].  X = A0 ^ 256 v.  Returns the lane's part
// of |g|^2.
template <int MB>
__device__ __forceinline__ float gen_groups(float (&g)[4 * MB], uint32_t X, const Philox32Step& st,
                                            const PhiloxKeys& K, int lane, int n) {
  static_assert(MB % 4 == 0, "groups of 16 components");
  float sl = 0.0f;
#pragma unroll
  for (int s = 0; s < MB / 4; ++s) {
    const int G = lane + 32 * s;
    float gq[16];
    if (16 * G < n) {
      sl += gauss_group16(X, G, st, K, n, gq);
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) gq[q] = 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) g[16 * s + q] = gq[q];
  }
  return sl;
}

// (Q^T g)_lane for the group layout.  The FP32 Q^T is stored in group order
// (rows of 1024 floats, zero past n): the 16-byte slice c of group
// G = lane + 32 s sits at 512 s + 128 c + 4 lane, so each load of a slice is
// contiguous across the warp.
template <int DQ, int MB>
__device__ __forceinline__ float qt_groups(const float* QT, const float (&g)[4 * MB], int lane, int D, int n) {
  float acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = 0.0f;
#pragma unroll
  for (int s = 0; s < MB / 4; ++s) {
    if (16 * 32 * s < n) {   // warp-uniform: some lane holds a group of this slot
#pragma unroll
      for (int c = 0; c < 4; ++c) {
#pragma unroll
        for (int j = 0; j < DQ; ++j) {
          if (j < D) {
            const float4 q4 =
                *reinterpret_cast<const float4*>(QT + static_cast<size_t>(j) * 1024 + 512 * s + 128 * c + 4 * lane);
            const float* gg = g + 16 * s + 4 * c;
            acc[j] += q4.x * gg[0] + q4.y * gg[1] + q4.z * gg[2] + q4.w * gg[3];
          }
        }
      }
    }
  }
  return reduce_scatter32(acc, lane);
}

template <int MK, int MB, int DQ>
__device__ __forceinline__ void walk_body(const DevProblem& pb, WarpRow& row) {
  constexpr int L = 4 * MB;
  const int lane = threadIdx.x & 31;
  const int64_t total = pb.wk_w1;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  int64_t w = pb.wk_w0 + ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (w >= total) return;
  const int n = pb.n;
  const int nbf = n >> 2, rem = n & 3;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const float eps = pb.sf.eps, h = pb.sf.h, rgeo = pb.sf.rho_geo, theta = pb.sf.theta;
  const float sqs = pb.sf.sqrt_sigma, sh = pb.sf.sh, inv_sigma = pb.sf.inv_sigma, sig = pb.sf.sigma;
  const bool bnd = !pb.closed;
  const bool dense_e = pb.ef_w != nullptr;
  // the lane's slot-0 entries of the boundary normal (walk order)
  float e0[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) e0[q] = bnd ? pb.e_s0[4 * lane + q] : 0.0f;
  // embedded sphere: D = d + 1 intrinsic coordinates
  const int D = pb.d + 1;
  // hypersurface of revolution: profile, c_kappa, f's scalars
  const float rv_al = pb.rv_alpha_f, rv_k = pb.rv_kappa_f, rv_mA = pb.rv_mA_f, ck = pb.rv_ck_f;
  const float c0f = pb.f.c0_f, c1f = pb.f.coef_f[0], c2f = pb.f.coef_f[1];

  float Y[L];            // Yh (ambient kinds) in walk coordinates
  float sj = 0.0f;       // embedded sphere: intrinsic coordinate s_lane (lane < D)
  float lam = 1.0f;      // Y = lam Yh
  float yy = 1.0f;       // |Yh|^2 (revolution: of the non-axis part)
  float ae = 0.0f;       // e.Yh
  float ty = 0.0f;       // revolution: the axis coordinate
  WalkAcc<float> wa;
  wa.set_tau(pb.tau_w);
  int64_t k = 0, o = 0;
  uint32_t p = 0;
  Philox32Walk pw{0u, 0u};

  // exact |Yh|^2 and e.Yh, Yh rescaled to lam = 1, slot 0 published
  auto resync = [&]() {
    if constexpr (MK != kEmbeddedSphere) {
      float acc[2] = {0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < L; ++q) {
        Y[q] *= lam;
        acc[0] += Y[q] * Y[q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[1] += e0[q] * Y[q];
      if (bnd && dense_e) {
        acc[1] = 0.0f;
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          const float4 ev = reinterpret_cast<const float4*>(pb.ef_w)[lane + 32 * m];
          acc[1] += ev.x * Y[4 * m] + ev.y * Y[4 * m + 1] + ev.z * Y[4 * m + 2] + ev.w * Y[4 * m + 3];
        }
      }
      wsum<2>(acc);
      yy = acc[0];
      ae = acc[1];
      lam = (MK == kSphere) ? rsqrtf(yy) : 1.0f;
      if (MK == kRevolution) lam = 1.0f;
      __syncwarp();
      *reinterpret_cast<float4*>(&row.y[4 * lane]) = make_float4(Y[0], Y[1], Y[2], Y[3]);
      __syncwarp();
    }
  };
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p;
    o = id.o;
    pw = philox32_walk(id.i, K);
    wa.reset();
    k = 0;
    lam = 1.0f;
    if constexpr (MK == kEmbeddedSphere) {
      sj = lane < D ? static_cast<float>(pb.s0[static_cast<size_t>(p) * D + lane]) : 0.0f;
    } else {
      const double* y0 = pb.pts + static_cast<size_t>(p) * n;
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = 4 * (lane + 32 * m) + q;
          Y[4 * m + q] = c < n ? static_cast<float>(y0[pb.perm ? pb.perm[c] : c]) : 0.0f;
        }
      if constexpr (MK == kRevolution) {   // the axis is walk coordinate 0 (lane 0, slot 0)
        ty = __shfl_sync(0xffffffffu, Y[0], 0);
        if (lane == 0) Y[0] = 0.0f;
      }
      resync();
    }
  };
  init(w);
  float r_prev = -1.0f;
  float g[L];

  for (;;) {
    // ---- stop test --------------------------------------------------------
    float dG = INFINITY;
    bool done = false;
    int flag = 0;
    if ((MK == kEuclid || MK == kSphere) && bnd) {
      const float al = lam * ae;
      float yg_scale, yg_e;   // y_Gamma = yg_e e + yg_scale Y
      if constexpr (MK == kEuclid) {
        dG = (al <= h) ? 0.0f : fabsf(al - h);
        yg_scale = 1.0f;
        yg_e = -(al - h);
      } else {
        // unit sphere, Omega = {e.x > h}: alpha = e.Y, rho = |Y - alpha e|,
        // y_G = h e + sh (Y - alpha e)/rho, |P_T r_G| = |rho h - alpha sh|,
        // |P_N r_G| = |1 - h alpha - sh rho|
        const float rho = sqrtf(fmaxf(lam * lam * yy - al * al, 0.0f));
        const float rt = rho * h - al * sh;
        float ex = fabsf(1.0f - h * al - sh * rho) - rgeo;
        ex = ex < 0.0f ? 0.0f : ex;
        dG = (al <= h) ? 0.0f : sqrtf(rt * rt + ex * ex);
        yg_scale = sh / rho;
        yg_e = h - al * yg_scale;
      }
      if (dG < eps) {
        float gv = 0.0f;
        if (pb.g.kind == kPoly) gv = poly_bnd(pb.g, row.y, pb.e_s0, yg_scale * lam, yg_e);
        wa.add_terminal(gv);
        done = true;
      } else if (wa.zero()) {
        done = true;
      }
    } else if (wa.below()) {
      done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      if (lane == 0) {
        pb.S_out[o] = wa.score();
        pb.K_out[o] = static_cast<int32_t>(k);
        pb.flag_out[o] = flag;
      }
      int64_t nxt = 0;
      if (lane == 0) nxt = next_walk(pb, w, nwarps);
      w = __shfl_sync(0xffffffffu, nxt, 0);
      if (w >= total) break;
      init(w);
      r_prev = -1.0f;
      continue;
    }
    // ---- radius and weights -------------------------------------------------
    float rg = rgeo;   // rho_geo = c_kappa / (1 + kappa(Y)) (eq. rho_geo_curvature)
    if constexpr (MK == kRevolution) rg = ck / (1.0f + rev_kappa<float>(rev_profile<float>(ty, rv_al, rv_k)));
    const float r = theta * (dG < rg ? dG : rg);
    const float a = sqs * r;
    if (r != r_prev) {
      if (!pb.em1_fp64) {
        wa.set_from_em1(em1_poly32(pb, 0.25f * a * a), inv_sigma);
      } else {
        const double ad = static_cast<double>(a);
        const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (ad * ad));
        const double cc = 1.0 / (1.0 + em1);
        wa.set(cc, one_minus_c(em1, cc) / pb.sigma);
      }
      r_prev = r;
    }
    const Philox32Step st = philox32_step(pw, static_cast<uint32_t>(k), p, K);
    const uint32_t xl = pw.A0 ^ static_cast<uint32_t>(lane);
    // ---- interior samples Z_l and F_k ----------------------------------------
    float F = 0.0f;
    for (int l = 0; l < nv; ++l) {
      const U4 bu = philox32_block(pw.A0 ^ static_cast<uint32_t>(256 * (1 + nv) + (l >> 2)), st, K);
      const int s4 = l & 3;
      const float U = u23(s4 == 0 ? bu.x : (s4 == 1 ? bu.y : (s4 == 2 ? bu.z : bu.w)));
      const float t = fminf(fmaxf(table_lookup32(pb, a, U), 0.0f), 1.0f);
      float sl;
      if constexpr (MK == kEmbeddedSphere)
        sl = gen_groups<MB>(g, pw.A0 ^ static_cast<uint32_t>(256 * (1 + l)), st, K, lane, n);
      else
        sl = gen_vec<MB>(g, xl ^ static_cast<uint32_t>(256 * (1 + l)), st, K, lane, nbf, rem);
      if constexpr (MK == kEmbeddedSphere) {
        const float qgj = qt_groups<DQ, MB>(pb.Qf, g, lane, D, n);
        float acc[1] = {sl};
        wsum<1>(acc);
        const float zs = (r * t) * rsqrtf(fmaxf(acc[0], 1e-30f));
        const float zj = lane < D ? sj + zs * qgj : 0.0f;
        float zz[1] = {zj * zj};
        wsum<1>(zz);
        F += sphere_quad_at<float>(pb, pb.f, pb.f.vf, pb.f.Af, zj * rsqrtf(zz[0]), lane, D);
      } else if constexpr (MK == kCurveSphere) {
        float acc[1] = {sl};
        wsum<1>(acc);
        const float zs = (r * t) * rsqrtf(fmaxf(acc[0], 1e-30f));
        *reinterpret_cast<float4*>(&row.g[4 * lane]) = make_float4(g[0], g[1], g[2], g[3]);
        __syncwarp();
        float X[9], y9[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) X[c] = row.y[c] + zs * row.g[c];
        __syncwarp();
        curve_sphere_cp<float>(pb.sf.R, pb.sf.a, X, y9);
        F += curve_sphere_value<float>(pb.f, pb.f.vf, pb.f.Af, pb.sf.R, pb.sf.a, sig, y9);
      } else if constexpr (MK == kRevolution) {
        // Z = Y + zs g: Zh / lam = Yh + (zs / lam) g_h, Z_axis = ty + zs g_axis
        float acc[1] = {sl};
        wsum<1>(acc);
        const float zs = (r * t) * rsqrtf(fmaxf(acc[0], 1e-30f));
        const float gax = __shfl_sync(0xffffffffu, g[0], 0);
        const float s2 = zs / lam;
        float za[3] = {0.0f, 0.0f, 0.0f};
        const float4* v4 = reinterpret_cast<const float4*>(pb.rv_v32);
        const float4* a4 = reinterpret_cast<const float4*>(pb.rv_a32);
#pragma unroll
        for (int m = 0; m < MB; ++m) {
          const float4 vv = v4[lane + 32 * m], aa = a4[lane + 32 * m];
          const float z0 = Y[4 * m] + s2 * g[4 * m], z1 = Y[4 * m + 1] + s2 * g[4 * m + 1];
          const float z2 = Y[4 * m + 2] + s2 * g[4 * m + 2], z3 = Y[4 * m + 3] + s2 * g[4 * m + 3];
          za[0] += z0 * z0 + z1 * z1 + z2 * z2 + z3 * z3;
          za[1] += vv.x * z0 + vv.y * z1 + vv.z * z2 + vv.w * z3;
          za[2] += (aa.x * z0) * z0 + (aa.y * z1) * z1 + (aa.z * z2) * z2 + (aa.w * z3) * z3;
        }
        wsum<3>(za);
        const float zax = s2 * gax;
        const float rho0 = lam * sqrtf(fmaxf(za[0] - zax * zax, 0.0f));
        Profile<float> P;
        const float tz = rev_cp_t<float>(rho0, ty + zs * gax, rv_al, rv_k, P);
        // on the axis cp takes the direction of walk coordinate 1
        const float vw = rho0 > 0.0f ? lam * za[1] / rho0 : pb.rv_v32[1];
        const float aw = rho0 > 0.0f ? lam * lam * za[2] / (rho0 * rho0) : pb.rv_a32[1];
        F += rev_quad_value<float>(P, tz, vw, aw, rv_mA, c0f, c1f, c2f, sig, n, pb.f.apply_op != 0);
      } else {
        // sphere / R^n: |g|^2 and Yh.g in one reduction; f at the coordinates of slot 0
        float acc[2] = {sl, 0.0f};
#pragma unroll
        for (int q = 0; q < L; ++q) acc[1] += Y[q] * g[q];
        wsum<2>(acc);
        const float zs = (r * t) * rsqrtf(fmaxf(acc[0], 1e-30f));
        float inv = 1.0f;
        if (MK == kSphere) inv = rsqrtf(lam * lam * yy + zs * (2.0f * lam * acc[1] + zs * acc[0]));
        *reinterpret_cast<float4*>(&row.g[4 * lane]) = make_float4(g[0], g[1], g[2], g[3]);
        __syncwarp();
        if (pb.f.kind == kPoly) F += poly_rows(pb.f, row.y, row.g, lam, zs, inv);
        __syncwarp();
      }
    }
    if (nv > 1) F /= static_cast<float>(nv);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta) --------------------------------------
    float sl;
    if constexpr (MK == kEmbeddedSphere)
      sl = gen_groups<MB>(g, pw.A0, st, K, lane, n);
    else
      sl = gen_vec<MB>(g, xl, st, K, lane, nbf, rem);
    if constexpr (MK == kEmbeddedSphere) {
      const float qgj = qt_groups<DQ, MB>(pb.Qf, g, lane, D, n);
      float acc[1] = {sl};
      wsum<1>(acc);
      const float sc = r * rsqrtf(fmaxf(acc[0], 1e-30f));
      const float tj = lane < D ? sj + sc * qgj : 0.0f;
      float tt[1] = {tj * tj};
      wsum<1>(tt);
      sj = tj * rsqrtf(tt[0]);
    } else if constexpr (MK == kCurveSphere) {
      float acc[1] = {sl};
      wsum<1>(acc);
      const float sc = r * rsqrtf(fmaxf(acc[0], 1e-30f));
      *reinterpret_cast<float4*>(&row.g[4 * lane]) = make_float4(g[0], g[1], g[2], g[3]);
      __syncwarp();
      float X[9], y9[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) X[c] = row.y[c] + sc * row.g[c];
      curve_sphere_cp<float>(pb.sf.R, pb.sf.a, X, y9);
      __syncwarp();
      if (lane == 0)
#pragma unroll
        for (int c = 0; c < 9; ++c) row.y[c] = y9[c];
      __syncwarp();
      const float4 y4 = *reinterpret_cast<const float4*>(&row.y[4 * lane]);
      Y[0] = y4.x; Y[1] = y4.y; Y[2] = y4.z; Y[3] = y4.w;
    } else if constexpr (MK == kRevolution) {
      float acc[2] = {sl, 0.0f};
#pragma unroll
      for (int q = 0; q < L; ++q) acc[1] += Y[q] * g[q];
      wsum<2>(acc);
      const float gax = __shfl_sync(0xffffffffu, g[0], 0);
      const float sc = r * rsqrtf(fmaxf(acc[0], 1e-30f));
      const float s2 = sc / lam;
      const float gh2 = fmaxf(acc[0] - gax * gax, 0.0f);
#pragma unroll
      for (int q = 0; q < L; ++q) Y[q] += s2 * g[q];
      if (lane == 0) Y[0] = 0.0f;
      yy = fmaxf(yy + s2 * (2.0f * acc[1] + s2 * gh2), 0.0f);
      const float rho0 = lam * sqrtf(yy);
      Profile<float> P;
      ty = rev_cp_t<float>(rho0, ty + sc * gax, rv_al, rv_k, P);
      lam = rho0 > 0.0f ? P.R * rsqrtf(yy) : 1.0f;
      if (!(rho0 > 0.0f)) {   // on the axis: cp takes the direction of walk coordinate 1
#pragma unroll
        for (int q = 0; q < L; ++q) Y[q] = 0.0f;
        if (lane == 0) Y[1] = P.R;
        yy = P.R * P.R;
      }
      if ((k & 63) == 63) resync();
    } else {
      // sphere / R^n: |g|^2, Yh.g and e.g in one reduction; the new |Yh|^2 and
      // e.Yh follow without another pass
      float acc[3] = {sl, 0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < L; ++q) acc[1] += Y[q] * g[q];
      if (bnd) {
        if (!dense_e) {
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[2] += e0[q] * g[q];
        } else {
#pragma unroll
          for (int m = 0; m < MB; ++m) {
            const float4 ev = reinterpret_cast<const float4*>(pb.ef_w)[lane + 32 * m];
            acc[2] += ev.x * g[4 * m] + ev.y * g[4 * m + 1] + ev.z * g[4 * m + 2] + ev.w * g[4 * m + 3];
          }
        }
      }
      wsum<3>(acc);
      const float sc = r * rsqrtf(fmaxf(acc[0], 1e-30f));
      const float s2 = sc / lam;
#pragma unroll
      for (int q = 0; q < L; ++q) Y[q] += s2 * g[q];
      yy = yy + s2 * (2.0f * acc[1] + s2 * acc[0]);
      ae = ae + s2 * acc[2];
      if (MK == kSphere) lam = rsqrtf(yy);
      if ((k & 63) == 63) {
        resync();
      } else {
        __syncwarp();
        *reinterpret_cast<float4*>(&row.y[4 * lane]) = make_float4(Y[0], Y[1], Y[2], Y[3]);
        __syncwarp();
      }
    }
    wa.add_step(F);
    ++k;
  }
}

template <int MK, int MB, int DQ>
__global__ void __launch_bounds__(kThreads, 4) walkn32_kernel(const DevProblem pb) {
  __shared__ WarpRow rows[kThreads / 32];
  walk_body<MK, MB, DQ>(pb, rows[threadIdx.x >> 5]);
}

// Slots per lane for n: n <= 128 MB.
inline int walkn32_mb(int n) { return n <= 128 ? 1 : (n <= 256 ? 2 : (n <= 512 ? 4 : 8)); }

}  // namespace w32
}  // namespace mpwos
