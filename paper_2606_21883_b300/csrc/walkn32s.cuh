// walkn32s.cuh — the FP32 MPWoS walk in R^n (3 < n <= 1024) for R^n, the unit
// sphere S^{n-1} and the hypersurface of revolution: LPW lanes per walker (16:
// two walkers per warp, so the step's scalar work — stop test, radius,
// weights, the radial sample, the source — is shared by two walks), with each
// walker's position in shared memory.
//
// Components come in groups of 16 (group G: components 16G .. 16G + 15, pairs
// 8G .. 8G + 7 of the Gaussian vector); lane h of a walker owns groups
// G = h + LPW m.  Draws of step k of walk (p, i), Philox4x32-10 at counter
// (k, j, i, p):
//   vector v (0: Theta, 1 + l: Z_l), group G: radial words from blocks
//   j = 256 v + 4 G and 256 v + 4 G + 1 (words 0..3 each: pairs 8G + 0..7),
//   angle halves from block j = 256 v + 4 G + 2 (word w: pair 8G + 2w from
//   its low 16 bits, pair 8G + 2w + 1 from its high 16 bits); pair q is
//   sqrt(-log2 u) (cos 2 pi a, sin 2 pi a), u in (0, 1] from its radial word's
//   low 23 bits, a = b / 65536 from its 16-bit angle b (the direction's
//   Gaussian vector up to one common factor, which g/|g| does not see; on the
//   grid of 65536 equally spaced angles every trigonometric moment of degree
//   below 65536 is that of the uniform angle);
//   U_l = u23(word l mod 4) of block j = 256 (1 + N_V) + l / 4.
// The draws depend on (seed, p, i, k, j) only, not on LPW.
// The radial halves come first: the sum over pairs of -log2 u is |g|^2, so a
// step's scale r/|g| is known before any component is formed, and the second
// pass (the angles) updates the position directly: no Gaussian vector is
// stored, only the radii (shared memory).  Z on the sphere and in R^n needs
// only |g|^2, Y.g and the components f reads, so it takes one pass.
//
// State: Y = lambda Yh (lambda per walker; Yh in shared memory, component
// 16G + q at 16 LPW m + 4 LPW (q / 4) + 4 h + q mod 4: conflict-free 16-byte
// accesses), |Yh|^2 and e.Yh carried, recomputed exactly every 64 steps.  The
// coordinate order (perm) puts the coordinates f, g and the boundary normal
// read first (groups 0..7, m = 0), the revolution's axis at coordinate 0.
#pragma once
#include "dev_common.cuh"
#include "green.cuh"
#include "revolution.cuh"
#include "walkn.cuh"

namespace mpwos {
namespace w32s {

constexpr int kThreads = 64;   // 2 warps, 4 walkers: 26 KB of static shared memory at n <= 1024

// Shared-memory position of walk coordinate c.
template <int LPW>
__device__ __forceinline__ int ypos(int c) {
  const int G = c >> 4, q = c & 15;
  return (G / LPW) * (16 * LPW) + (q >> 2) * (4 * LPW) + (G % LPW) * 4 + (q & 3);
}

// Sum over the LPW lanes of a walker (a butterfly within the lane group).
template <int LPW, int NV>
__device__ __forceinline__ void wsum(float (&v)[NV], unsigned mask) {
#pragma unroll
  for (int off = LPW / 2; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(mask, v[q], off);
}

// POLY at x_v = (ya Yh_v + gb g_v) inv (walk coordinates v < 128; g_v in gs).
template <int LPW>
__device__ __forceinline__ float poly_z(const DevFunc& fn, const float* ys, const float* gs, float ya, float gb,
                                        float inv) {
  float total = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    float prod = fn.coef_f[t];
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const float xv = (ya * ys[ypos<LPW>(v)] + gb * gs[v]) * inv;
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// POLY at y_Gamma = ya Yh + ye e (walk coordinates v < 128).
template <int LPW>
__device__ __forceinline__ float poly_b(const DevFunc& fn, const float* ys, const float* es, float ya, float ye) {
  float total = 0.0f;
  for (int t = 0; t < fn.n_terms; ++t) {
    float prod = fn.coef_f[t];
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const float xv = ya * ys[ypos<LPW>(v)] + ye * es[v];
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

template <int MK, int LPW, int MG>
__device__ __forceinline__ void walk_body(const DevProblem& pb, float* ys, float* gs, float* rs, const float* es) {
  const int lane = threadIdx.x & 31;
  const int hl = lane & (LPW - 1);                                   // lane within the walker
  const int hb = lane & ~(LPW - 1);                                  // the walker's first lane
  const unsigned hmask = LPW == 32 ? 0xffffffffu : (((1u << LPW) - 1u) << hb);
  const int64_t total = pb.wk_w1;
  const int64_t nslots = (static_cast<int64_t>(gridDim.x) * blockDim.x) / LPW;
  int64_t w = pb.wk_w0 + (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / LPW;
  if (w >= total) return;
  const int n = pb.n;
  const int nGf = n >> 4, rem = n & 15;   // full groups; components of the partial group
  // the lane's full groups are m < nfull; m == mpart (if >= 0) is the partial one
  const int nfull = nGf > hl ? (nGf - hl + LPW - 1) / LPW : 0;
  const int mpart = (rem && hl + LPW * nfull == nGf) ? nfull : -1;
  const int mend = mpart >= 0 ? mpart + 1 : nfull;   // groups the lane owns
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const float eps = pb.sf.eps, h = pb.sf.h, rgeo = pb.sf.rho_geo, theta = pb.sf.theta;
  const float sqs = pb.sf.sqrt_sigma, sh = pb.sf.sh, inv_sigma = pb.sf.inv_sigma, sig = pb.sf.sigma;
  const bool bnd = (MK != kRevolution) && !pb.closed;
  const bool dense_e = pb.ef_w != nullptr;
  const float rv_al = pb.rv_alpha_f, rv_k = pb.rv_kappa_f, rv_mA = pb.rv_mA_f, ck = pb.rv_ck_f;
  const float c0f = pb.f.c0_f, c1f = pb.f.coef_f[0], c2f = pb.f.coef_f[1];
  constexpr int YM = 16 * LPW, YQ = 4 * LPW;   // Yh: stride of m, of a group's quarters
  constexpr int RM = 8 * LPW;                  // radii: stride of m

  float lam = 1.0f;   // Y = lam Yh
  float yy = 1.0f;    // |Yh|^2 (revolution: of the non-axis part)
  float ae = 0.0f;    // e.Yh
  float ty = 0.0f;    // revolution: the axis coordinate
  WalkAcc<float> wa;
  wa.set_tau(pb.tau_w);
  int64_t k = 0, o = 0;
  uint32_t p = 0;
  Philox32Walk pw{0u, 0u};
  Philox32Step st{0u, 0u, 0u, 0u};

  auto load16 = [&](const float* base, int m, float (&y)[16]) {
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const float4 a = *reinterpret_cast<const float4*>(base + YM * m + YQ * qq + 4 * hl);
      y[4 * qq] = a.x; y[4 * qq + 1] = a.y; y[4 * qq + 2] = a.z; y[4 * qq + 3] = a.w;
    }
  };
  auto store16 = [&](int m, const float (&y)[16]) {
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
      *reinterpret_cast<float4*>(ys + YM * m + YQ * qq + 4 * hl) =
          make_float4(y[4 * qq], y[4 * qq + 1], y[4 * qq + 2], y[4 * qq + 3]);
  };
  // 16 consecutive floats of a walk-order array at group G (global, L1-resident)
  auto gload16 = [&](const float* a, int m, float (&v)[16]) {
    const float4* a4 = reinterpret_cast<const float4*>(a) + 4 * (hl + LPW * m);
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const float4 t = a4[qq];
      v[4 * qq] = t.x; v[4 * qq + 1] = t.y; v[4 * qq + 2] = t.z; v[4 * qq + 3] = t.w;
    }
  };
  // e (walk order) on the lane's group m
  auto e_group = [&](int m, float (&e16)[16]) {
    if (dense_e) {
      gload16(pb.ef_w, m, e16);
    } else if (m == 0 && 16 * hl < 128) {
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const float4 t = *reinterpret_cast<const float4*>(es + 16 * hl + 4 * qq);
        e16[4 * qq] = t.x; e16[4 * qq + 1] = t.y; e16[4 * qq + 2] = t.z; e16[4 * qq + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 16; ++q) e16[q] = 0.0f;
    }
  };
  // blocks of group m of a vector: A0 ^ x ^ (4 LPW m + c), x = 256 v ^ 4 h, c = 0, 1
  // (radial words), 2 (angle halves)
  auto blk = [&](uint32_t x, int m, int c) {
    return philox32_block(x ^ static_cast<uint32_t>(4 * LPW * m + c), st, K);
  };
  // the group's 8 radii and their sum of -log2 u
  auto radii = [&](uint32_t x, int m, float (&R)[8]) -> float {
    return radial4(blk(x, m, 0), R) + radial4(blk(x, m, 1), R + 4);
  };
  // pass 1 of a vector: the radii of the lane's pairs into shared memory; returns
  // the lane's part of |g|^2 (of the partial last group: the squares of its
  // valid components)
  // (the partial group runs in the same iteration as the other lanes' last full
  // group; with an even number of valid components its pairs are whole and need
  // no angles)
  auto radial_pass = [&](uint32_t x) -> float {
    float sl = 0.0f;
    for (int m = 0; m < mend; ++m) {
      float R[8];
      const float s_all = radii(x, m, R);
      *reinterpret_cast<float4*>(rs + RM * m + 4 * hl) = make_float4(R[0], R[1], R[2], R[3]);
      *reinterpret_cast<float4*>(rs + RM * m + YQ + 4 * hl) = make_float4(R[4], R[5], R[6], R[7]);
      if (m != mpart) {
        sl += s_all;
      } else if ((rem & 1) == 0) {
#pragma unroll
        for (int q = 0; q < 8; ++q) sl += 2 * q < rem ? R[q] * R[q] : 0.0f;
      } else {
        float gq[16];
        angle8(blk(x, m, 2), R, gq);
#pragma unroll
        for (int q = 0; q < 16; ++q) sl += q < rem ? gq[q] * gq[q] : 0.0f;
      }
    }
    return sl;
  };
  // the components of group m of a vector whose radii are in shared memory
  auto angle_group = [&](uint32_t x, int m, float (&gq)[16]) {
    const float4 r0 = *reinterpret_cast<const float4*>(rs + RM * m + 4 * hl);
    const float4 r1 = *reinterpret_cast<const float4*>(rs + RM * m + YQ + 4 * hl);
    const float R[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    angle8(blk(x, m, 2), R, gq);
    if (m == mpart)
#pragma unroll
      for (int q = 0; q < 16; ++q) gq[q] = q < rem ? gq[q] : 0.0f;
  };
  // exact |Yh|^2 and e.Yh with Yh rescaled to lam = 1
  auto resync = [&]() {
    float acc[2] = {0.0f, 0.0f};
    for (int m = 0; m < mend; ++m) {
      float y[16], e16[16];
      load16(ys, m, y);
      e_group(m, e16);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        y[q] *= lam;
        acc[0] += y[q] * y[q];
        acc[1] += e16[q] * y[q];
      }
      store16(m, y);
    }
    wsum<LPW, 2>(acc, hmask);
    yy = acc[0];
    ae = acc[1];
    lam = (MK == kSphere) ? rsqrtf(yy) : 1.0f;
    __syncwarp(hmask);
  };
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p;
    o = id.o;
    pw = philox32_walk(id.i, K);
    wa.reset();
    k = 0;
    lam = 1.0f;
    const double* y0 = pb.pts + static_cast<size_t>(p) * n;
    __syncwarp(hmask);
    for (int m = 0; m < MG; ++m) {
      float y[16];
      const int base = 16 * (hl + LPW * m);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int c = base + q;
        y[q] = c < n ? static_cast<float>(y0[pb.perm ? pb.perm[c] : c]) : 0.0f;
      }
      if (MK == kRevolution && m == 0 && hl == 0) {   // the axis is walk coordinate 0
        ty = y[0];
        y[0] = 0.0f;
      }
      store16(m, y);
    }
    if constexpr (MK == kRevolution) ty = __shfl_sync(hmask, ty, hb);
    __syncwarp(hmask);
    resync();
  };
  init(w);
  float r_prev = -1.0f;

  for (;;) {
    // ---- stop test --------------------------------------------------------
    float dG = INFINITY;
    bool done = false;
    int flag = 0;
    if (bnd) {
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
        if (pb.g.kind == kPoly) gv = poly_b<LPW>(pb.g, ys, es, yg_scale * lam, yg_e);
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
      if (hl == 0) {
        pb.S_out[o] = wa.score();
        pb.K_out[o] = static_cast<int32_t>(k);
        pb.flag_out[o] = flag;
      }
      int64_t nxt = 0;
      if (hl == 0) nxt = next_walk(pb, w, nslots);
      w = __shfl_sync(hmask, nxt, hb);
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
    st = philox32_step(pw, static_cast<uint32_t>(k), p, K);
    const uint32_t xl = pw.A0 ^ static_cast<uint32_t>(4 * hl);
    // ---- interior samples Z_l and F_k ----------------------------------------
    float F = 0.0f;
    for (int l = 0; l < nv; ++l) {
      const U4 bu = philox32_block(pw.A0 ^ static_cast<uint32_t>(256 * (1 + nv) + (l >> 2)), st, K);
      const int s4 = l & 3;
      const float U = u23(s4 == 0 ? bu.x : (s4 == 1 ? bu.y : (s4 == 2 ? bu.z : bu.w)));
      const float t = fminf(fmaxf(table_lookup32(pb, a, U), 0.0f), 1.0f);
      const uint32_t xv = xl ^ static_cast<uint32_t>(256 * (1 + l));
      if constexpr (MK == kRevolution) {
        // pass 1: |g|^2 and the radii; pass 2: Zh / lam = Yh + (zs / lam) g_h
        float acc1[1] = {radial_pass(xv)};
        wsum<LPW, 1>(acc1, hmask);
        const float zs = (r * t) * rsqrtf(fmaxf(acc1[0], 1e-30f));
        const float s2 = zs / lam;
        float za[3] = {0.0f, 0.0f, 0.0f};
        float g0 = 0.0f;
        for (int m = 0; m < mend; ++m) {
          float gq[16], y[16], vv[16], av[16];
          angle_group(xv, m, gq);
          load16(ys, m, y);
          gload16(pb.rv_v32, m, vv);
          gload16(pb.rv_a32, m, av);
          if (m == 0) g0 = gq[0];
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const float z = y[q] + s2 * gq[q];
            za[0] += z * z;
            za[1] += vv[q] * z;
            za[2] += (av[q] * z) * z;
          }
        }
        wsum<LPW, 3>(za, hmask);
        const float gax = __shfl_sync(hmask, g0, hb);
        const float zax = s2 * gax;   // walk coordinate 0 (the axis) is not part of Zh
        const float rho0 = lam * sqrtf(fmaxf(za[0] - zax * zax, 0.0f));
        Profile<float> P;
        const float tz = rev_cp_t<float>(rho0, ty + zs * gax, rv_al, rv_k, P);
        const float vw = rho0 > 0.0f ? lam * za[1] / rho0 : pb.rv_v32[1];
        const float aw = rho0 > 0.0f ? lam * lam * za[2] / (rho0 * rho0) : pb.rv_a32[1];
        F += rev_quad_value<float>(P, tz, vw, aw, rv_mA, c0f, c1f, c2f, sig, n, pb.f.apply_op != 0);
      } else {
        // sphere / R^n, one pass: |g|^2 and Yh.g; the lanes holding groups 0..7
        // (the walk coordinates f reads, < 128) write their components to gs
        float acc[2] = {0.0f, 0.0f};
        for (int m = 0; m < mend; ++m) {
          float R[8], gq[16], y[16];
          const float sl = radii(xv, m, R);
          angle8(blk(xv, m, 2), R, gq);
          load16(ys, m, y);
          if (m != mpart) {
            acc[0] += sl;
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
              gq[q] = q < rem ? gq[q] : 0.0f;
              acc[0] += gq[q] * gq[q];
            }
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[1] += y[q] * gq[q];
          if (m == 0 && 16 * hl < 128)
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
              *reinterpret_cast<float4*>(gs + 16 * hl + 4 * qq) =
                  make_float4(gq[4 * qq], gq[4 * qq + 1], gq[4 * qq + 2], gq[4 * qq + 3]);
        }
        wsum<LPW, 2>(acc, hmask);
        __syncwarp(hmask);
        const float zs = (r * t) * rsqrtf(fmaxf(acc[0], 1e-30f));
        float inv = 1.0f;
        if (MK == kSphere) inv = rsqrtf(lam * lam * yy + zs * (2.0f * lam * acc[1] + zs * acc[0]));
        if (pb.f.kind == kPoly) F += poly_z<LPW>(pb.f, ys, gs, lam, zs, inv);
        __syncwarp(hmask);
      }
    }
    if (nv > 1) F /= static_cast<float>(nv);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta): pass 1 radii and |g|^2 --------------
    float acc1[1] = {radial_pass(xl)};
    wsum<LPW, 1>(acc1, hmask);
    const float sc = r * rsqrtf(fmaxf(acc1[0], 1e-30f));
    const float s2 = sc / lam;
    // pass 2: Yh += (sc / lam) g, with the new |Yh|^2 and e.Yh
    float acc[2] = {0.0f, 0.0f};
    float g0 = 0.0f;
    for (int m = 0; m < mend; ++m) {
      float gq[16], y[16];
      angle_group(xl, m, gq);
      load16(ys, m, y);
      if (MK == kRevolution && m == 0) {
        g0 = gq[0];
        if (hl == 0) gq[0] = 0.0f;   // the axis coordinate follows the closest point, not Yh
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        y[q] += s2 * gq[q];
        acc[0] += y[q] * y[q];
      }
      if (bnd && (dense_e || m == 0)) {
        float e16[16];
        e_group(m, e16);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[1] += e16[q] * y[q];
      }
      store16(m, y);
    }
    wsum<LPW, 2>(acc, hmask);
    if constexpr (MK == kRevolution) {
      const float gax = __shfl_sync(hmask, g0, hb);
      yy = acc[0];
      const float rho0 = lam * sqrtf(yy);
      Profile<float> P;
      ty = rev_cp_t<float>(rho0, ty + sc * gax, rv_al, rv_k, P);
      if (rho0 > 0.0f) {
        lam = P.R * rsqrtf(yy);
      } else {   // on the axis: cp takes the direction of walk coordinate 1
        __syncwarp(hmask);
        if (hl == 0) ys[ypos<LPW>(1)] = 1.0f;
        yy = 1.0f;
        lam = P.R;
      }
    } else {
      yy = acc[0];
      ae = acc[1];
      if (MK == kSphere) lam = rsqrtf(yy);
    }
    __syncwarp(hmask);
    if ((k & 63) == 63) resync();
    wa.add_step(F);
    ++k;
  }
}

// Walkers per block: kThreads / LPW; shared memory per walker: Yh (16 LPW MG
// floats), radii (8 LPW MG), the components f reads (128); the normal's first
// 128 walk coordinates once per block.
template <int MK, int LPW, int MG>
__global__ void __launch_bounds__(kThreads, 8) walkn32s_kernel(const DevProblem pb) {
  constexpr int W = kThreads / LPW;
  __shared__ __align__(16) float ys_all[W][16 * LPW * MG];
  __shared__ __align__(16) float rs_all[W][8 * LPW * MG];
  __shared__ __align__(16) float gs_all[W][128];
  __shared__ __align__(16) float es[128];
  for (int i = threadIdx.x; i < 128; i += blockDim.x) es[i] = pb.closed ? 0.0f : pb.e_s0[i];
  __syncthreads();
  const int ws = threadIdx.x / LPW;
  walk_body<MK, LPW, MG>(pb, ys_all[ws], gs_all[ws], rs_all[ws], es);
}

// Lanes per walker, and groups per lane for n (n <= 16 LPW MG).
constexpr int kLPW = 16;
inline int walkn32s_mg(int n) { return n <= 256 ? 1 : (n <= 512 ? 2 : 4); }

}  // namespace w32s
}  // namespace mpwos
