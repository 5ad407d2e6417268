// walkn.cuh — the MPWoS walk in R^n (n up to 1024), one warp per walker.
//
// Layout: the walker's n-vectors live in registers, distributed over the 32
// lanes in Philox-block order: block b (G consecutive components G b .. G b +
// G - 1; G = 4 in FP32, 2 in FP64) belongs to lane b mod 32, register slot
// b / 32.  A lane therefore generates exactly the Gaussians of the components
// it owns, and every norm or dot product is a per-lane partial sum followed by
// a butterfly shuffle reduction.  The embedded sphere Q S^d + b is walked in
// its intrinsic coordinate s (lane j holds s_j, j <= d): cp(Y + v) = Q
// normalize(s + Q^T v) + b, so only Q^T g of each Gaussian vector is needed;
// Q^T is stored transposed (D x n) so that a lane's 16-byte slice of a row is
// one coalesced load.
//
// Draws of step k of walk (p, i), Philox counter (j, k, i, p), nb = ceil(n/G):
//   Theta direction: blocks [0, nb);  Z_l direction: blocks [nb(1+l), nb(2+l));
//   FP64: U_l = u53(x, y) of block nb(1+N_V) + l  (identical to the CPU oracle);
//   FP32: U_l = u24(word l mod 4) of block nb(1+N_V) + l/4.
#pragma once
#include "dev_common.cuh"
#include "green.cuh"

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
                                           uint32_t kk, uint32_t wi, uint32_t p, uint32_t k0, uint32_t k1) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB;
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = lane + 32 * m;
    if (G * b < n) {
      const U4 r = philox4x32_10(jb + static_cast<uint32_t>(b), kk, wi, p, k0, k1);
      if constexpr (G == 2) {
        double g0, g1;
        box_muller64(u53(r.x, r.y), u53(r.z, r.w), g0, g1);
        g[2 * m] = g0;
        g[2 * m + 1] = (2 * b + 1 < n) ? g1 : 0.0;
      } else {
        float g0, g1, g2, g3;
        box_muller32(u24(r.x), u24(r.y), g0, g1);
        box_muller32(u24(r.z), u24(r.w), g2, g3);
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

// Value of component v of a distributed vector, broadcast to all lanes.
template <typename T, int L>
__device__ __forceinline__ T gather(const T (&x)[L], int v, int G) {
  const int blk = v / G;
  const int owner = blk & 31;
  const int slot = (blk >> 5) * G + (v - blk * G);
  T val = T(0);
#pragma unroll
  for (int t = 0; t < L; ++t)
    if (t == slot) val = x[t];
  return __shfl_sync(0xffffffffu, val, owner);
}

// POLY at the point whose component v is base_v + sc * dir_v, divided by den.
template <typename T, int L>
__device__ __forceinline__ T poly_at(const DevFunc& fn, const T (&base)[L], const T (&dir)[L], T sc, T inv_den,
                                     bool use_dir, int G) {
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    T prod = T(fn.coef[t]);
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      T xv = gather(base, v, G);
      if (use_dir) xv += sc * gather(dir, v, G);
      xv *= inv_den;
      for (int e = 0; e < fn.pw[q]; ++e) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// POLY at y_Gamma = yg_scale Y + yg_e e (e a host-copied device array).
template <typename T, int L>
__device__ __forceinline__ T poly_at_boundary(const DevFunc& fn, const T (&Y)[L], const double* e, T yg_scale,
                                              T yg_e, int G) {
  T total = T(0);
  for (int t = 0; t < fn.n_terms; ++t) {
    T prod = T(fn.coef[t]);
    for (int q = fn.term_off[t]; q < fn.term_off[t + 1]; ++q) {
      const int v = fn.var[q];
      const T xv = yg_scale * gather(Y, v, G) + yg_e * T(e[v]);
      for (int ee = 0; ee < fn.pw[q]; ++ee) prod *= xv;
    }
    total += prod;
  }
  return total;
}

// SPHERE_QUAD at the unit vector s (lane j holds s_j, j < D; others 0).
template <typename T>
__device__ __forceinline__ T sphere_quad_at(const DevProblem& pb, const DevFunc& fn, T sj, int lane, int D) {
  const bool on = lane < D;
  const T vj = on ? T(fn.v[lane]) : T(0);
  T As = T(0);
  for (int q = 0; q < D; ++q) {
    const T sq = __shfl_sync(0xffffffffu, sj, q);
    if (on) As += T(fn.A[lane * D + q]) * sq;
  }
  T acc[3] = {vj * sj, sj * As, on ? T(fn.A[lane * D + lane]) : T(0)};
  warp_sum<3>(acc);
  const T lin = acc[0], quad = acc[1], tr = acc[2];
  if (!fn.apply_op) return T(fn.c0) + lin + quad;
  const T d = T(D - 1), sg = T(pb.sigma), mean = tr / T(D);
  return sg * (T(fn.c0) + mean) + (d + sg) * lin + (T(2) * (d + T(1)) + sg) * (quad - mean);
}

// Per-lane partial of Q^T g (acc[j], j < D), reduced over the warp.
template <typename T, int D_MAX>
__device__ __forceinline__ void qt_times(const DevProblem& pb, const T* QT, const T (&g)[Prec<T>::G * Prec<T>::MB],
                                         int lane, int D, T (&acc)[D_MAX]) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB;
  const int n = pb.n;
#pragma unroll
  for (int j = 0; j < D_MAX; ++j) acc[j] = T(0);
#pragma unroll
  for (int m = 0; m < MB; ++m) {
    const int b = lane + 32 * m;
    if (G * b < n) {
#pragma unroll
      for (int j = 0; j < D_MAX; ++j) {
        if (j < D) {
          const T* row = QT + static_cast<size_t>(j) * n + G * b;
#pragma unroll
          for (int q = 0; q < G; ++q)
            if (G * b + q < n) acc[j] += row[q] * g[G * m + q];
        }
      }
    }
  }
  warp_sum<D_MAX>(acc);
}

// ---------------------------------------------------------------------------
// The warp walk.  T = double: the FP64 walk (per-walk identical draws to the
// CPU oracle); T = float: the FP32 walk with FP64 weights and score.
// ---------------------------------------------------------------------------
template <typename T, int MK>
__device__ __forceinline__ void walkn_body(const DevProblem& pb) {
  constexpr int G = Prec<T>::G, MB = Prec<T>::MB, L = G * MB;
  constexpr int DQ = 32;
  const int lane = threadIdx.x & 31;
  const int64_t total = pb.P * pb.N;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (w >= total) return;
  const int n = pb.n;
  const int D = pb.d + 1;
  const uint32_t k0 = static_cast<uint32_t>(pb.seed), k1 = static_cast<uint32_t>(pb.seed >> 32);
  const int nv = pb.n_v;
  const uint32_t nb = static_cast<uint32_t>((n + G - 1) / G);
  const T* QT = nullptr;
  if constexpr (MK == kEmbeddedSphere) {
    if constexpr (sizeof(T) == 8) QT = reinterpret_cast<const T*>(pb.Q); else QT = reinterpret_cast<const T*>(pb.Qf);
  }

  T Y[L];        // ambient state (sphere, R^n)
  T sj = T(0);   // intrinsic state (embedded sphere), lane j < D
  double W = 1.0, S = 0.0;
  int64_t k = 0;
  uint32_t p = 0, wi = 0;

  auto init = [&](int64_t ww) {
    p = static_cast<uint32_t>(ww / pb.N);
    wi = static_cast<uint32_t>(ww - static_cast<int64_t>(p) * pb.N);
    W = 1.0; S = 0.0; k = 0;
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
    }
  };
  init(w);
  T r_prev = T(-1);
  double c = 1.0, omega = 0.0;
  GreenLaw law{};
  T g[L];

  for (;;) {
    // ---- stop test --------------------------------------------------------
    T dG = T(INFINITY);
    bool done = false;
    int flag = 0;
    if constexpr (MK != kEmbeddedSphere) {
      if (!pb.closed) {
        T acc[2] = {T(0), T(0)};
#pragma unroll
        for (int m = 0; m < MB; ++m)
#pragma unroll
          for (int q = 0; q < G; ++q) {
            const int cc = G * (lane + 32 * m) + q;
            const T ev = cc < n ? T(pb.e[cc]) : T(0);
            acc[0] += Y[G * m + q] * ev;
            acc[1] += Y[G * m + q] * Y[G * m + q];
          }
        warp_sum<2>(acc);
        const T al = acc[0], h = T(pb.h);
        T yg_scale, yg_e;   // y_Gamma = yg_e e + yg_scale Y
        if (MK == kEuclid) {
          dG = (al <= h) ? T(0) : fabs(al - h);
          yg_scale = T(1);
          yg_e = -(al - h);
        } else {
          // unit sphere, Omega = {e.x > h}: with alpha = e.Y, rho = |Y - alpha e|,
          // sh = sqrt(1 - h^2):  y_G = h e + sh (Y - alpha e)/rho,
          // |P_T r_G| = |rho h - alpha sh|,  |P_N r_G| = |1 - h alpha - sh rho|.
          const T rho = sqrt(fmax(acc[1] - al * al, T(0)));
          const T sh = sqrt(T(1) - h * h);
          const T rt = rho * h - al * sh;
          T ex = fabs(T(1) - h * al - sh * rho) - T(pb.rho_geo);
          ex = ex < T(0) ? T(0) : ex;
          dG = (al <= h) ? T(0) : sqrt(rt * rt + ex * ex);
          yg_scale = sh / rho;
          yg_e = h - al * yg_scale;
        }
        if (dG < T(pb.eps)) {
          // g at y_Gamma = yg_e e + yg_scale Y
          T gv = T(0);
          if (pb.g.kind == kPoly) gv = poly_at_boundary<T, L>(pb.g, Y, pb.e, yg_scale, yg_e, G);
          S += W * static_cast<double>(gv);
          done = true;
        } else if (W == 0.0) {
          done = true;
        }
      } else if (W < pb.tau_w) {
        done = true;
      }
    } else {
      if (W < pb.tau_w) done = true;
    }
    if (!done && k >= pb.max_steps) { done = true; flag = 1; }
    if (done) {
      if (lane == 0) {
        pb.S_out[w] = S;
        pb.K_out[w] = static_cast<int32_t>(k);
        pb.flag_out[w] = flag;
      }
      w += nwarps;
      if (w >= total) break;
      init(w);
      continue;
    }
    // ---- radius and weights -------------------------------------------------
    const T rgeo = T(pb.rho_geo);
    const T r = T(pb.theta) * (dG < rgeo ? dG : rgeo);
    const T a = T(pb.sqrt_sigma) * r;
    if (r != r_prev) {
      if constexpr (sizeof(T) == 8) {
        law = green_law(n, a);
        c = law.c;
        omega = law.omc / pb.sigma;
      } else {
        const double ad = static_cast<double>(a);
        const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (ad * ad));
        c = 1.0 / (1.0 + em1);
        omega = one_minus_c(em1, c) / pb.sigma;
      }
      r_prev = r;
    }
    const uint32_t kk = static_cast<uint32_t>(k);
    // ---- interior samples Z_l and F_k ----------------------------------------
    T F = T(0);
    for (int l = 0; l < nv; ++l) {
      T t;
      {
        T U;
        if constexpr (G == 2) {
          const U4 bu = philox4x32_10(nb * static_cast<uint32_t>(1 + nv) + static_cast<uint32_t>(l), kk, wi, p, k0, k1);
          U = u53(bu.x, bu.y);
          const double guess = table_lookup<double>(pb.tab64, pb.NA, pb.NS, pb.z_max, a, s_of_u64(U));
          t = green_invert64(law, U, guess);
        } else {
          const U4 bu = philox4x32_10(nb * static_cast<uint32_t>(1 + nv) + static_cast<uint32_t>(l >> 2), kk, wi,
                                      p, k0, k1);
          const int s4 = l & 3;
          U = u24(s4 == 0 ? bu.x : (s4 == 1 ? bu.y : (s4 == 2 ? bu.z : bu.w)));
          t = table_lookup<float>(pb.tab32, pb.NA, pb.NS, pb.z_max, a, s_of_u32(U));
          t = fminf(fmaxf(t, 0.0f), 1.0f);
        }
      }
      gen_vector<T>(g, n, lane, nb * static_cast<uint32_t>(1 + l), kk, wi, p, k0, k1);
      if constexpr (MK == kEmbeddedSphere) {
        T qg[DQ];
        qt_times<T, DQ>(pb, QT, g, lane, D, qg);
        T gg = T(0);
#pragma unroll
        for (int q = 0; q < L; ++q) gg += g[q] * g[q];
        gg = fmax(warp_sum1(gg), T(1e-30));
        const T zs = (r * t) / sqrt(gg);
        T qgj = T(0);
#pragma unroll
        for (int j = 0; j < DQ; ++j)
          if (j == lane) qgj = qg[j];
        T zj = lane < D ? sj + zs * qgj : T(0);
        const T zn = sqrt(warp_sum1(zj * zj));
        F += sphere_quad_at<T>(pb, pb.f, zj / zn, lane, D);
      } else {
        T gg = T(0);
#pragma unroll
        for (int q = 0; q < L; ++q) gg += g[q] * g[q];
        gg = fmax(warp_sum1(gg), T(1e-30));
        const T zs = (r * t) / sqrt(gg);
        T inv = T(1);
        if (MK == kSphere) {
          T zz = T(0);
#pragma unroll
          for (int q = 0; q < L; ++q) { const T zq = Y[q] + zs * g[q]; zz += zq * zq; }
          inv = T(1) / sqrt(warp_sum1(zz));
        }
        if (pb.f.kind == kPoly) F += poly_at<T, L>(pb.f, Y, g, zs, inv, true, G);
      }
    }
    if (nv > 1) F /= T(nv);
    // ---- Theta = Y + r g/|g|, Y = cp(Theta) --------------------------------------
    gen_vector<T>(g, n, lane, 0u, kk, wi, p, k0, k1);
    if constexpr (MK == kEmbeddedSphere) {
      T qg[DQ];
      qt_times<T, DQ>(pb, QT, g, lane, D, qg);
      T gg = T(0);
#pragma unroll
      for (int q = 0; q < L; ++q) gg += g[q] * g[q];
      gg = fmax(warp_sum1(gg), T(1e-30));
      const T sc = r / sqrt(gg);
      T qgj = T(0);
#pragma unroll
      for (int j = 0; j < DQ; ++j)
        if (j == lane) qgj = qg[j];
      T tj = lane < D ? sj + sc * qgj : T(0);
      const T tn = sqrt(warp_sum1(tj * tj));
      sj = tj / tn;
    } else {
      T gg = T(0);
#pragma unroll
      for (int q = 0; q < L; ++q) gg += g[q] * g[q];
      gg = fmax(warp_sum1(gg), T(1e-30));
      const T sc = r / sqrt(gg);
#pragma unroll
      for (int q = 0; q < L; ++q) Y[q] = Y[q] + sc * g[q];
      if (MK == kSphere) {
        T yy = T(0);
#pragma unroll
        for (int q = 0; q < L; ++q) yy += Y[q] * Y[q];
        const T yn = sqrt(warp_sum1(yy));
#pragma unroll
        for (int q = 0; q < L; ++q) Y[q] = Y[q] / yn;
      }
    }
    S += (W * omega) * static_cast<double>(F);
    W *= c;
    ++k;
  }
}

template <int MK>
__global__ void __launch_bounds__(128) walkn_f64_kernel(const DevProblem pb) { walkn_body<double, MK>(pb); }

template <int MK>
__global__ void __launch_bounds__(128) walkn_f32_kernel(const DevProblem pb) { walkn_body<float, MK>(pb); }

}  // namespace mpwos
