// walkn.cuh — the FP64 MPWoS walk in R^n (n up to 1024), one warp per walker,
// and the precision-generic pieces (WalkAcc, the source evaluators) that the
// FP32 walks in walkn32s.cuh and walkn32.cuh reuse.
//
// Layout: the walker's n-vectors live in registers, distributed over the 32
// lanes in Philox-block order: block b (components 2b, 2b + 1) belongs to lane
// b mod 32, register slot b / 32.  A lane therefore generates exactly the
// Gaussians of the components it owns, and every norm or dot product is a
// per-lane partial sum followed by a butterfly shuffle reduction.  The
// embedded sphere Q S^d + b is walked in its intrinsic coordinate s (lane j
// holds s_j, j <= d): cp(Y + v) = Q normalize(s + Q^T v) + b, so only Q^T g of
// each Gaussian vector is needed; Q^T is stored transposed (D x n) so that a
// lane's 16-byte slice of a row is one coalesced load.
//
// Draws of step k of walk (p, i), Philox counter (j, k, i, p), nb = ceil(n/2):
//   Theta direction: blocks [0, nb);  Z_l direction: blocks [nb(1+l), nb(2+l));
//   U_l = u53(x, y) of block nb(1+N_V) + l  (identical to the CPU oracle).
// The hypersurface of revolution (revolution.cuh) keeps Y in the ambient layout;
// its closest point needs |Yh|^2 and Y_{n-1} (one reduction), then the same
// Newton iteration in every lane.
#pragma once
#include "dev_common.cuh"
#include "green.cuh"
#include "revolution.cuh"
#include "curve_sphere.cuh"

namespace mpwos {

template <typename T> struct Prec;
template <> struct Prec<double> {
  static constexpr int G = 2;
  static constexpr int MB = 16;   // blocks per lane: n <= 32 * 2 * 16 = 1024
};
template <> struct Prec<float> {
  static constexpr int G = 4;
  static constexpr int MB = 8;    // n <= 32 * 4 * 8 = 1024
};

// Running weight W and score S of one walk: FP64 in the FP64 walk, float
// pairs in the FP32 walk (no FP64 instruction in the FP32 step loop).
template <typename T> struct WalkAcc;
template <> struct WalkAcc<double> {
  double W = 1.0, S = 0.0, c = 1.0, om = 0.0, tau = 0.0;
  __device__ void set_tau(double t) { tau = t; }
  __device__ void reset() { W = 1.0; S = 0.0; }
  __device__ void set(double cc, double omega) { c = cc; om = omega; }
  __device__ void set_from_em1(float, float) {}
  __device__ void add_terminal(double g) { S += W * g; }
  __device__ void add_step(double F) { S += (W * om) * F; W *= c; }
  __device__ bool below() const { return W < tau; }
  __device__ bool zero() const { return W == 0.0; }
  __device__ double score() const { return S; }
};
template <> struct WalkAcc<float> {
  F2 W{1.0f, 0.0f}, S{0.0f, 0.0f}, c{1.0f, 0.0f}, om{0.0f, 0.0f}, tau{0.0f, 0.0f};
  __device__ void set_tau(double t) { tau = f2_from_double(t); }
  __device__ void reset() { W = F2{1.0f, 0.0f}; S = F2{0.0f, 0.0f}; }
  __device__ void set(double cc, double omega) { c = f2_from_double(cc); om = f2_from_double(omega); }
  __device__ void set_from_em1(float em1, float inv_sigma) { weights_from_em1(em1, inv_sigma, c, om); }
  __device__ void add_terminal(float g) { S = f2_add(S, f2_mul_f(W, g)); }
  __device__ void add_step(float F) { S = f2_add(S, f2_mul_f(f2_mul(W, om), F)); W = f2_mul(W, c); }
  __device__ bool below() const { return W.hi < tau.hi || (W.hi == tau.hi && W.lo < tau.lo); }
  __device__ bool zero() const { return W.hi == 0.0f; }
  __device__ double score() const { return f2_to_double(S); }
};

template <int NV, typename T>
__device__ __forceinline__ void warp_sum(T (&v)[NV]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], off);
}

template <typename T>
__device__ __forceinline__ T warp_sum1(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// The n-vector of Gaussians for blocks jb + b (b = lane + 32 m) of step kk.
template <typename T>
__device__ __forceinline__ void gen_vector(T (&g)[Prec<T>::G * Prec<T>::MB], int n, int lane, uint32_t jb,
                                           uint32_t kk, uint32_t wi, uint32_t p, const PhiloxKeys& K) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB;
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = lane + 32 * m;
    if (G * b < n) {
      const U4 r = philox4x32_10(jb + static_cast<uint32_t>(b), kk, wi, p, K);
      if constexpr (G == 2) {
        double g0, g1;
        box_muller64(u53(r.x, r.y), u53(r.z, r.w), g0, g1);
        g[2 * m] = g0;
        g[2 * m + 1] = (2 * b + 1 < n) ? g1 : 0.0;
      } else {
        float g0, g1, g2, g3;
        box_muller32(u23(r.x), u23(r.y), g0, g1);
        box_muller32(u23(r.z), u23(r.w), g2, g3);
        g[4 * m] = g0;
        g[4 * m + 1] = (4 * b + 1 < n) ? g1 : 0.0f;
        g[4 * m + 2] = (4 * b + 2 < n) ? g2 : 0.0f;
        g[4 * m + 3] = (4 * b + 3 < n) ? g3 : 0.0f;
      }
    } else {
#pragma unroll
      for (int q = 0; q < G; ++q) g[G * m + q] = T(0);
    }
  }
}

// Component v of a distributed vector, broadcast to all lanes (v is warp-
// uniform).  Components v < 32 G live in register slot v mod G of lane v/G.
template <typename T, int L, int G>
__device__ __forceinline__ T gather(const T (&x)[L], int v) {
  const int blk = v / G;
  const int owner = blk & 31;
  T val = x[0];
  if (blk < 32) {
    const int slot = v - blk * G;
#pragma unroll
    for (int t = 1; t < G; ++t)
      if (t == slot) val = x[t];
  } else {
    const int slot = (blk >> 5) * G + (v - blk * G);
#pragma unroll
    for (int t = 1; t < L; ++t)
      if (t == slot) val = x[t];
  }
  return __shfl_sync(0xffffffffu, val, owner);
}

// POLY at the point X_v = (base_v + sc dir_v) inv.
template <typename T, int L, int G>
__device__ __forceinline__ T poly_at(const DevFunc& fn, const T (&base)[L], const T (&dir)[L], T sc, T inv) {
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    T prod = pick<T>(fn.coef[t], fn.coef_f[t]);
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const T xv = (gather<T, L, G>(base, v) + sc * gather<T, L, G>(dir, v)) * inv;
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// POLY at y_Gamma = yg_scale Y + yg_e e.
template <typename T, int L, int G>
__device__ __forceinline__ T poly_at_boundary(const DevFunc& fn, const T (&Y)[L], const T* e, T yg_scale, T yg_e) {
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    T prod = pick<T>(fn.coef[t], fn.coef_f[t]);
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const T xv = yg_scale * gather<T, L, G>(Y, v) + yg_e * e[v];
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// Lane l receives the warp-wide sum of v[l] (recursive halving: 31 shuffles
// for 32 values instead of 5 per value).
template <typename T>
__device__ __forceinline__ T reduce_scatter32(T (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const T send = up ? v[i] : v[i + o];
      const T keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// SPHERE_QUAD at the unit vector s (lane j holds s_j, j < D; others 0).
template <typename T>
__device__ __forceinline__ T sphere_quad_at(const DevProblem& pb, const DevFunc& fn, const T* vT, const T* AT,
                                            T sj, int lane, int D) {
  const bool on = lane < D;
  T As = T(0);
  for (int q = 0; q < D; ++q) {
    const T sq = __shfl_sync(0xffffffffu, sj, q);
    if (on) As += AT[lane * D + q] * sq;
  }
  T acc[3] = {on ? vT[lane] * sj : T(0), sj * As, on ? AT[lane * D + lane] : T(0)};
  warp_sum<3>(acc);
  const T lin = acc[0], quad = acc[1], tr = acc[2];
  const T c0 = pick<T>(fn.c0, fn.c0_f);
  if (!fn.apply_op) return c0 + lin + quad;
  const T d = T(D - 1), sg = pick<T>(pb.sigma, pb.sf.sigma), mean = tr / T(D);
  return sg * (c0 + mean) + (d + sg) * lin + (T(2) * (d + T(1)) + sg) * (quad - mean);
}

// (Q^T g)_lane and |g|^2 for one Gaussian vector: per-lane partial products
// with 16-byte loads of the transposed, zero-padded Q^T (row stride npad),
// then one reduce-scatter; |g|^2 rides in slot 31 (D <= 31).
template <typename T, int DQ>
__device__ __forceinline__ T qt_times(const T* QT, int npad, const T (&g)[Prec<T>::G * Prec<T>::MB], int n,
                                      int lane, int D, T& gg) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB;
  T acc[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] = T(0);
  T g2 = T(0);
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = lane + 32 * m;
    if (G * b < n) {
#pragma unroll
      for (int q = 0; q < G; ++q) g2 += g[G * m + q] * g[G * m + q];
#pragma unroll
      for (int j = 0; j < DQ; ++j) {
        if (j < D) {
          const T* row = QT + static_cast<size_t>(j) * npad + G * b;
          if constexpr (G == 4) {
            const float4 q4 = *reinterpret_cast<const float4*>(row);
            acc[j] += q4.x * g[4 * m] + q4.y * g[4 * m + 1] + q4.z * g[4 * m + 2] + q4.w * g[4 * m + 3];
          } else {
            const double2 q2 = *reinterpret_cast<const double2*>(row);
            acc[j] += q2.x * g[2 * m] + q2.y * g[2 * m + 1];
          }
        }
      }
    }
  }
  acc[31] = g2;
  const T mine = reduce_scatter32(acc, lane);
  gg = __shfl_sync(0xffffffffu, mine, 31);
  return mine;
}

// ---------------------------------------------------------------------------
// The warp walk.  T = double: the FP64 walk (per-walk identical draws to the
// CPU oracle, explicit norms); T = float: the FP32 walk (norms of the updated
// state from the reductions already done, float-pair W and S).
// ---------------------------------------------------------------------------
template <typename T, int MK, int DQ>
__device__ __forceinline__ void walkn_body(const DevProblem& pb) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB, L = G * MB;
  constexpr bool kF64 = sizeof(T) == 8;
  const int lane = threadIdx.x & 31;
  const int64_t total = pb.wk_w1;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  int64_t w = pb.wk_w0 + ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (w >= total) return;
  const int n = pb.n;
  const int D = pb.d + 1;
  const int npad = (n + 3) & ~3;
  const PhiloxKeys& K = pb.keys;
  const int nv = pb.n_v;
  const uint32_t nb = static_cast<uint32_t>((n + G - 1) / G);
  // loop-invariant parameters in the walk's precision
  const T eps_t = pick<T>(pb.eps, pb.sf.eps), h_t = pick<T>(pb.h, pb.sf.h);
  const T rgeo_t = pick<T>(pb.rho_geo, pb.sf.rho_geo), theta_t = pick<T>(pb.theta, pb.sf.theta);
  const T sqs_t = pick<T>(pb.sqrt_sigma, pb.sf.sqrt_sigma);
  const T sh_t = pick<T>(sqrt(1.0 - pb.h * pb.h), pb.sf.sh);
  const float inv_sigma_f = pb.sf.inv_sigma;
  const bool bnd = !pb.closed;
  const T* eT = kF64 ? reinterpret_cast<const T*>(pb.e) : reinterpret_cast<const T*>(pb.ef);
  const T* QT = nullptr;
  const T* vT = nullptr;
  const T* AT = nullptr;
  if constexpr (MK == kEmbeddedSphere) {
    QT = kF64 ? reinterpret_cast<const T*>(pb.Q) : reinterpret_cast<const T*>(pb.Qf);
    vT = kF64 ? reinterpret_cast<const T*>(pb.f.v) : reinterpret_cast<const T*>(pb.f.vf);
    AT = kF64 ? reinterpret_cast<const T*>(pb.f.A) : reinterpret_cast<const T*>(pb.f.Af);
  }
  // hypersurface of revolution: v and diag(A) of f (n - 1 entries), profile, c_kappa
  const T* vR = nullptr;
  const T* aR = nullptr;
  T rv_al = T(0), rv_k = T(1), rv_mA = T(0), ck_t = T(0), c0_t = T(0), c1_t = T(0), c2_t = T(0);
  const T sig_t = pick<T>(pb.sigma, pb.sf.sigma);
  if constexpr (MK == kRevolution) {
    vR = kF64 ? reinterpret_cast<const T*>(pb.f.v) : reinterpret_cast<const T*>(pb.f.vf);
    aR = kF64 ? reinterpret_cast<const T*>(pb.f.A) : reinterpret_cast<const T*>(pb.f.Af);
    rv_al = pick<T>(pb.rv_alpha, pb.rv_alpha_f);
    rv_k = pick<T>(pb.rv_kappa, pb.rv_kappa_f);
    rv_mA = pick<T>(pb.rv_mA, pb.rv_mA_f);
    ck_t = pick<T>(pb.c_kappa, pb.rv_ck_f);
    c0_t = pick<T>(pb.f.c0, pb.f.c0_f);
    c1_t = pick<T>(pb.f.coef[0], pb.f.coef_f[0]);
    c2_t = pick<T>(pb.f.coef[1], pb.f.coef_f[1]);
  }
  T ty = T(0);   // revolution: the axis coordinate Y_{n-1}
  // Fourier curve x sphere (n = 9): v, A of f (3 and 9 per term), R, a
  const T* vC = nullptr;
  const T* aC = nullptr;
  const T cs_R = pick<T>(pb.R, pb.sf.R), cs_a = pick<T>(pb.a_tube, pb.sf.a);
  if constexpr (MK == kCurveSphere) {
    vC = kF64 ? reinterpret_cast<const T*>(pb.f.v) : reinterpret_cast<const T*>(pb.f.vf);
    aC = kF64 ? reinterpret_cast<const T*>(pb.f.A) : reinterpret_cast<const T*>(pb.f.Af);
  }

  T Y[L];          // ambient state (sphere, R^n)
  T sj = T(0);     // intrinsic state (embedded sphere), lane j < D
  T al = T(0), yy = T(1);   // e.Y and |Y|^2 (boundary problems)
  WalkAcc<T> wa;
  wa.set_tau(pb.tau_w);
  int64_t k = 0, o = 0;
  uint32_t p = 0, wi = 0;

  auto state_dots = [&]() {
    T acc[2] = {T(0), T(0)};
#pragma unroll
    for (int m = 0; m < MB; ++m)
#pragma unroll
      for (int q = 0; q < G; ++q) {
        const int cc = G * (lane + 32 * m) + q;
        const T ev = cc < n ? eT[cc] : T(0);
        acc[0] += Y[G * m + q] * ev;
        acc[1] += Y[G * m + q] * Y[G * m + q];
      }
    warp_sum<2>(acc);
    al = acc[0];
    yy = acc[1];
  };
  auto init = [&](int64_t ww) {
    const WalkId id = walk_id(pb, ww);
    p = id.p; wi = id.i; o = id.o;
    wa.reset();
    k = 0;
    if constexpr (MK == kEmbeddedSphere) {
      sj = lane < D ? T(pb.s0[static_cast<size_t>(p) * D + lane]) : T(0);
    } else {
      const double* y0 = pb.pts + static_cast<size_t>(p) * n;
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int c = G * (lane + 32 * m) + q;
          Y[G * m + q] = c < n ? T(y0[c]) : T(0);
        }
      if constexpr (MK == kRevolution) ty = T(y0[n - 1]);
      if (bnd) state_dots();
    }
  };
  init(w);
  T r_prev = T(-1);
  GreenLaw law{};
  T g[L];

  for (;;) {
    // ---- stop test --------------------------------------------------------
    T dG = T(INFINITY);
    bool done = false;
    int flag = 0;
    if constexpr (MK != kEmbeddedSphere) {
      if (bnd) {
        // FP64 recomputes e.Y and |Y|^2 every step; FP32 carries them from the
        // last update and resynchronises every 64 steps (bounded rounding drift)
        if (kF64 || (k & 63) == 0) state_dots();
        T yg_scale, yg_e;   // y_Gamma = yg_e e + yg_scale Y
        if constexpr (MK == kEuclid) {
          dG = (al <= h_t) ? T(0) : fabs(al - h_t);
          yg_scale = T(1);
          yg_e = -(al - h_t);
        } else {
          // unit sphere, Omega = {e.x > h}: with alpha = e.Y, rho = |Y - alpha e|,
          // sh = sqrt(1 - h^2):  y_G = h e + sh (Y - alpha e)/rho,
          // |P_T r_G| = |rho h - alpha sh|,  |P_N r_G| = |1 - h alpha - sh rho|.
          const T rho = sqrt(fmax(yy - al * al, T(0)));
          const T rt = rho * h_t - al * sh_t;
          T ex = fabs(T(1) - h_t * al - sh_t * rho) - rgeo_t;
          ex = ex < T(0) ? T(0) : ex;
          dG = (al <= h_t) ? T(0) : sqrt(rt * rt + ex * ex);
          yg_scale = sh_t / rho;
          yg_e = h_t - al * yg_scale;
        }
        if (dG < eps_t) {
          T gv = T(0);
          if (pb.g.kind == kPoly) gv = poly_at_boundary<T, L, G>(pb.g, Y, eT, yg_scale, yg_e);
          wa.add_terminal(gv);
          done = true;
        } else if (wa.zero()) {
          done = true;
        }
      } else if (wa.below()) {
        done = true;
      }
    } else {
      if (wa.below()) done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      if (lane == 0) {
        pb.S_out[o] = wa.score();
        pb.K_out[o] = static_cast<int32_t>(k);
        pb.flag_out[o] = flag;
      }
      {
        int64_t nxt = 0;
        if (lane == 0) nxt = next_walk(pb, w, nwarps);
        w = __shfl_sync(0xffffffffu, nxt, 0);
      }
      if (w >= total) break;
      init(w);
      continue;
    }
    // ---- radius and weights -------------------------------------------------
    T rg = rgeo_t;   // rho_geo = c_kappa / (1 + kappa(Y)) (eq. rho_geo_curvature)
    if constexpr (MK == kRevolution) rg = ck_t / (T(1) + rev_kappa<T>(rev_profile<T>(ty, rv_al, rv_k)));
    const T r = theta_t * (dG < rg ? dG : rg);
    const T a = sqs_t * r;
    if (r != r_prev) {
      if constexpr (kF64) {
        law = green_law(n, a);
        wa.set(law.c, law.omc / pb.sigma);
      } else if (!pb.em1_fp64) {
        wa.set_from_em1(em1_poly32(pb, 0.25f * a * a), inv_sigma_f);
      } else {
        const double ad = static_cast<double>(a);
        const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (ad * ad));
        const double cc = 1.0 / (1.0 + em1);
        wa.set(cc, one_minus_c(em1, cc) / pb.sigma);
      }
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    // ---- interior samples Z_l and F_k ----------------------------------------
    T F = T(0);
    for (int l = 0; l < nv; ++l) {
      T t;
      if constexpr (kF64) {
        const U4 bu = philox4x32_10(nb * static_cast<uint32_t>(1 + nv) + static_cast<uint32_t>(l), kk, wi, p, K);
        const double U = u53(bu.x, bu.y);
        const double guess = table_lookup<double>(pb.tab64, pb.NA, pb.NS, pb.z_max, a, U);
        t = green_invert64(law, U, guess);
      } else {
        const U4 bu = philox4x32_10(nb * static_cast<uint32_t>(1 + nv) + static_cast<uint32_t>(l >> 2), kk, wi, p, K);
        const int s4 = l & 3;
        const float U = u23(s4 == 0 ? bu.x : (s4 == 1 ? bu.y : (s4 == 2 ? bu.z : bu.w)));
        t = table_lookup32(pb, a, U);
        t = fminf(fmaxf(t, 0.0f), 1.0f);
      }
      gen_vector<T>(g, n, lane, nb * static_cast<uint32_t>(1 + l), kk, wi, p, K);
      if constexpr (MK == kEmbeddedSphere) {
        T gg;
        const T qgj = qt_times<T, DQ>(QT, npad, g, n, lane, D, gg);
        const T zs = (r * t) / sqrt(fmax(gg, T(1e-30)));
        const T zj = lane < D ? sj + zs * qgj : T(0);
        const T zn = sqrt(warp_sum1(zj * zj));
        F += sphere_quad_at<T>(pb, pb.f, vT, AT, zj / zn, lane, D);
      } else {
        T acc[2] = {T(0), T(0)};
#pragma unroll
        for (int q = 0; q < L; ++q) { acc[0] += g[q] * g[q]; acc[1] += Y[q] * g[q]; }
        warp_sum<2>(acc);
        const T zs = (r * t) / sqrt(fmax(acc[0], T(1e-30)));
        if constexpr (MK == kCurveSphere) {
          // n = 9: every lane takes the whole Z and its closest point
          T X[9], y9[9];
#pragma unroll
          for (int c = 0; c < 9; ++c) X[c] = gather<T, L, G>(Y, c) + zs * gather<T, L, G>(g, c);
          curve_sphere_cp<T>(cs_R, cs_a, X, y9);
          F += curve_sphere_value<T>(pb.f, vC, aC, cs_R, cs_a, sig_t, y9);
          continue;
        }
        if constexpr (MK == kRevolution) {
          // Z = Y + zs g; |Zh|^2, v.Zh, Zh^T diag(A) Zh and Z_{n-1} in one reduction
          T za[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
          for (int m = 0; m < MB; ++m)
#pragma unroll
            for (int q = 0; q < G; ++q) {
              const int cc = G * (lane + 32 * m) + q;
              const T zc = Y[G * m + q] + zs * g[G * m + q];
              if (cc < n - 1) {
                za[0] += zc * zc;
                za[1] += vR[cc] * zc;
                za[2] += aR[cc] * zc * zc;
              } else if (cc == n - 1) {
                za[3] = zc;
              }
            }
          warp_sum<4>(za);
          const T rho0 = sqrt(za[0]);
          Profile<T> P;
          const T tz = rev_cp_t<T>(rho0, za[3], rv_al, rv_k, P);
          // on the axis cp takes the direction e_1 (w = e_1)
          const T vw = rho0 > T(0) ? za[1] / rho0 : vR[0];
          const T aw = rho0 > T(0) ? za[2] / (rho0 * rho0) : aR[0];
          F += rev_quad_value<T>(P, tz, vw, aw, rv_mA, c0_t, c1_t, c2_t, sig_t, n, pb.f.apply_op != 0);
          continue;
        }
        T inv = T(1);
        if constexpr (MK == kSphere) {
          if constexpr (kF64) {
            T zz = T(0);
#pragma unroll
            for (int q = 0; q < L; ++q) { const T zq = Y[q] + zs * g[q]; zz += zq * zq; }
            inv = T(1) / sqrt(warp_sum1(zz));
          } else {
            inv = rsqrtf(yy + zs * (T(2) * acc[1] + zs * acc[0]));
          }
        }
        if (pb.f.kind == kPoly) F += poly_at<T, L, G>(pb.f, Y, g, zs, inv);
      }
    }
    if (nv > 1) F /= T(nv);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta) --------------------------------------
    gen_vector<T>(g, n, lane, 0u, kk, wi, p, K);
    if constexpr (MK == kEmbeddedSphere) {
      T gg;
      const T qgj = qt_times<T, DQ>(QT, npad, g, n, lane, D, gg);
      const T sc = r / sqrt(fmax(gg, T(1e-30)));
      const T tj = lane < D ? sj + sc * qgj : T(0);
      const T tn = sqrt(warp_sum1(tj * tj));
      sj = tj / tn;
    } else if constexpr (MK == kCurveSphere) {
      T gg = T(0);
#pragma unroll
      for (int q = 0; q < L; ++q) gg += g[q] * g[q];
      gg = fmax(warp_sum1(gg), T(1e-30));
      const T sc = r / sqrt(gg);
      T X[9], y9[9];
#pragma unroll
      for (int c = 0; c < 9; ++c) X[c] = gather<T, L, G>(Y, c) + sc * gather<T, L, G>(g, c);
      curve_sphere_cp<T>(cs_R, cs_a, X, y9);
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int cc = G * (lane + 32 * m) + q;
#pragma unroll
          for (int c = 0; c < 9; ++c)
            if (c == cc) Y[G * m + q] = y9[c];
        }
    } else if constexpr (MK == kRevolution) {
      // Theta = Y + r g/|g|; Y = cp(Theta): scale Theta_h to R(t)/|Theta_h|, Y_{n-1} = t
      T gg = T(0);
#pragma unroll
      for (int q = 0; q < L; ++q) gg += g[q] * g[q];
      gg = fmax(warp_sum1(gg), T(1e-30));
      const T sc = r / sqrt(gg);
      T ta[2] = {T(0), T(0)};
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int cc = G * (lane + 32 * m) + q;
          const T th = Y[G * m + q] + sc * g[G * m + q];
          Y[G * m + q] = th;
          if (cc < n - 1) ta[0] += th * th;
          else if (cc == n - 1) ta[1] = th;
        }
      warp_sum<2>(ta);
      const T rho0 = sqrt(ta[0]);
      Profile<T> P;
      ty = rev_cp_t<T>(rho0, ta[1], rv_al, rv_k, P);
      const T sR = rho0 > T(0) ? P.R / rho0 : T(0);
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const int cc = G * (lane + 32 * m) + q;
          T& yc = Y[G * m + q];
          if (cc < n - 1) yc = rho0 > T(0) ? yc * sR : (cc == 0 ? P.R : T(0));
          else if (cc == n - 1) yc = ty;
        }
    } else if constexpr (kF64) {
      T gg = T(0);
#pragma unroll
      for (int q = 0; q < L; ++q) gg += g[q] * g[q];
      gg = fmax(warp_sum1(gg), T(1e-30));
      const T sc = r / sqrt(gg);
#pragma unroll
      for (int q = 0; q < L; ++q) Y[q] = Y[q] + sc * g[q];
      if (MK == kSphere) {
        T ys = T(0);
#pragma unroll
        for (int q = 0; q < L; ++q) ys += Y[q] * Y[q];
        const T yn = sqrt(warp_sum1(ys));
#pragma unroll
        for (int q = 0; q < L; ++q) Y[q] = Y[q] / yn;
      }
    } else {
      // FP32: one reduction gives |g|^2, Y.g and e.g; the updated e.Y and |Y|^2
      // follow without another pass.
      T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
      for (int m = 0; m < MB; ++m)
#pragma unroll
        for (int q = 0; q < G; ++q) {
          const T gq = g[G * m + q];
          acc[0] += gq * gq;
          acc[1] += Y[G * m + q] * gq;
          if (bnd) {
            const int cc = G * (lane + 32 * m) + q;
            acc[2] += gq * (cc < n ? eT[cc] : T(0));
          }
        }
      warp_sum<3>(acc);
      const T sc = r * rsqrtf(fmaxf(acc[0], 1e-30f));
      T inv = T(1);
      const T tt = yy + sc * (T(2) * acc[1] + sc * acc[0]);
      if (MK == kSphere) inv = rsqrtf(tt);
#pragma unroll
      for (int q = 0; q < L; ++q) Y[q] = (Y[q] + sc * g[q]) * inv;
      al = (al + sc * acc[2]) * inv;
      yy = tt * inv * inv;
    }
    wa.add_step(F);
    ++k;
  }
}

template <int MK, int DQ>
__global__ void __launch_bounds__(128) walkn_f64_kernel(const DevProblem pb) { walkn_body<double, MK, DQ>(pb); }

// Embedded-sphere dimension bucket (d + 1 <= DQ).
inline int walkn_dq(int D) { return D <= 8 ? 8 : (D <= 16 ? 16 : (D <= 24 ? 24 : 32)); }

}  // namespace mpwos
