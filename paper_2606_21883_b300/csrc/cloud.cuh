// cloud.cuh — closest point on a point-cloud surface (Sec. 2.1, representation
// (iii); the radius uses rho_geo = c_h h(y), eq. rho_geo_spacing).
//
// Search: a uniform cell grid over the cloud (points sorted by cell, original
// index kept for tie-breaks).  k nearest by expanding cubes of cells: after the
// cube of radius R around x's cell, the k-th distance is final once it does
// not exceed the distance from x to the cube's nearest open face.  Ordering by
// (distance^2, original index), distances in the scalar type T.
// Fit: centroid and covariance of the k neighbours, normal = eigenvector of the
// smallest eigenvalue (cyclic Jacobi), least-squares quadratic height
// z = a0 + a1 u + a2 v + a3 u^2 + a4 uv + a5 v^2 in plane coordinates scaled
// by h(x) (6x6 normal equations, Cholesky), projection of x onto the graph by
// its vertical foot point plus one Newton step on the squared distance.
#pragma once
#include "dev_common.cuh"

namespace mpwos {

template <typename T, int KM>
struct Knn {
  T d2[KM];
  int idx[KM];   // sorted-array positions
  int gid[KM];   // original indices
};

template <typename T>
__device__ __forceinline__ const T* cloud_pts(const DevProblem& pb);
template <>
__device__ __forceinline__ const double* cloud_pts<double>(const DevProblem& pb) { return pb.cl_pts64; }
template <>
__device__ __forceinline__ const float* cloud_pts<float>(const DevProblem& pb) { return pb.cl_pts32; }

template <typename T, int KM>
__device__ __forceinline__ void knn_insert(Knn<T, KM>& R, int k, T dd, int pos, int g) {
  // candidate goes before entry j when (dd, g) < (d2[j], gid[j])
  if (!(dd < R.d2[k - 1] || (dd == R.d2[k - 1] && g < R.gid[k - 1]))) return;
#pragma unroll
  for (int j = KM - 1; j >= 0; --j) {
    if (j >= k) continue;
    const bool before_prev = j > 0 && (dd < R.d2[j - 1] || (dd == R.d2[j - 1] && g < R.gid[j - 1]));
    if (before_prev) {
      R.d2[j] = R.d2[j - 1]; R.idx[j] = R.idx[j - 1]; R.gid[j] = R.gid[j - 1];
    } else {
      R.d2[j] = dd; R.idx[j] = pos; R.gid[j] = g;
      break;
    }
  }
}

// The k nearest cloud points of x; returns h(x) = their mean distance.
template <typename T, int KM>
__device__ __forceinline__ T cloud_knn(const DevProblem& pb, const T* x, Knn<T, KM>& R) {
  const int k = pb.cl_k;
  const T* P = cloud_pts<T>(pb);
#pragma unroll
  for (int j = 0; j < KM; ++j) { R.d2[j] = T(INFINITY); R.idx[j] = -1; R.gid[j] = 0x7fffffff; }
  const T cs = pick<T>(pb.cl_cell, pb.cl_cell_f);
  int c[3];
  T lo[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = pick<T>(pb.cl_origin[a], pb.cl_origin_f[a]);
    int ci = static_cast<int>(floor((x[a] - lo[a]) / cs));
    c[a] = ci < 0 ? 0 : (ci >= pb.cl_dims[a] ? pb.cl_dims[a] - 1 : ci);
  }
  const int gx = pb.cl_dims[0], gy = pb.cl_dims[1], gz = pb.cl_dims[2];
  const int rmax = max(gx, max(gy, gz));
  for (int Rr = 0; Rr <= rmax; ++Rr) {
    // the shell of cells at Chebyshev distance Rr from c
    for (int dz = -Rr; dz <= Rr; ++dz) {
      const int zz = c[2] + dz;
      if (zz < 0 || zz >= gz) continue;
      for (int dy = -Rr; dy <= Rr; ++dy) {
        const int yy = c[1] + dy;
        if (yy < 0 || yy >= gy) continue;
        const bool face = (dz == -Rr || dz == Rr || dy == -Rr || dy == Rr);
        const int step = face ? 1 : 2 * Rr;   // inner rows: only the two end cells lie on the shell
        for (int dx = -Rr; dx <= Rr; dx += step) {
          const int xx = c[0] + dx;
          if (xx >= 0 && xx < gx) {
            const int cell = (zz * gy + yy) * gx + xx;
            const int b = pb.cl_start[cell], e = pb.cl_start[cell + 1];
            for (int q = b; q < e; ++q) {
              T px, py, pz;
              int g;
              if constexpr (sizeof(T) == 4) {   // one 16-byte load: x, y, z, original index
                const float4 c4 = pb.cl_pts4[q];
                px = c4.x; py = c4.y; pz = c4.z;
                g = __float_as_int(c4.w);
              } else {
                px = P[3 * q]; py = P[3 * q + 1]; pz = P[3 * q + 2];
                g = pb.cl_orig[q];
              }
              const T ddx = px - x[0], ddy = py - x[1], ddz = pz - x[2];
              const T dd = ddx * ddx + ddy * ddy + ddz * ddz;
              knn_insert<T, KM>(R, k, dd, q, g);
            }
          }
        }
      }
    }
    // distance from x to the nearest face of the searched cube that has cells beyond it
    T guard = T(INFINITY);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (c[a] - Rr > 0) guard = fmin(guard, x[a] - (lo[a] + T(c[a] - Rr) * cs));
      if (c[a] + Rr < pb.cl_dims[a] - 1) guard = fmin(guard, (lo[a] + T(c[a] + Rr + 1) * cs) - x[a]);
    }
    if (R.d2[k - 1] <= guard * guard || guard == T(INFINITY)) break;
  }
  T h = T(0);
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < k) h += sqrt(R.d2[j]);
  return h / T(k);
}

// cloud_knn for the FP32 walk, made by a whole warp (all 32 lanes call it
// together, each with its own query x and a flag saying whether it has one).
// The warp takes the queries one at a time: for each it visits the same cells
// as cloud_knn, scans each cell's points one per lane, and keeps the sorted list
// of the nearest so far spread one entry per lane (entry j in lane j), a
// candidate being inserted by shifting the entries after it one lane up.
// Candidates are inserted in the order cloud_knn inserts them (cells, then
// points ascending), so the k nearest -- and everything computed from them --
// are identical to cloud_knn's; the query's lane then receives them.  A
// candidate that passed the filter but no longer beats the k-th entry lands
// beyond entry k - 1 and never moves back (entries only move up).
template <int KM>
__device__ __forceinline__ float cloud_knn_coop(const DevProblem& pb, const float* x, bool valid, Knn<float, KM>& R) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int k = pb.cl_k;
#pragma unroll
  for (int j = 0; j < KM; ++j) { R.d2[j] = INFINITY; R.idx[j] = -1; R.gid[j] = 0x7fffffff; }
  const float cs = pb.cl_cell_f;
  const int gx = pb.cl_dims[0], gy = pb.cl_dims[1], gz = pb.cl_dims[2];
  const int rmax = max(gx, max(gy, gz));
  unsigned qm = __ballot_sync(kAll, valid);
  while (qm) {
    const int src = __ffs(qm) - 1;
    qm &= qm - 1;
    const float q[3] = {__shfl_sync(kAll, x[0], src), __shfl_sync(kAll, x[1], src), __shfl_sync(kAll, x[2], src)};
    int c[3];
    float lo[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = pb.cl_origin_f[a];
      int ci = static_cast<int>(floorf((q[a] - lo[a]) / cs));
      c[a] = ci < 0 ? 0 : (ci >= pb.cl_dims[a] ? pb.cl_dims[a] - 1 : ci);
    }
    float ld = INFINITY;
    int lg = 0x7fffffff, lp = -1;
    for (int Rr = 0; Rr <= rmax; ++Rr) {
      for (int dz = -Rr; dz <= Rr; ++dz) {
        const int zz = c[2] + dz;
        if (zz < 0 || zz >= gz) continue;
        for (int dy = -Rr; dy <= Rr; ++dy) {
          const int yy = c[1] + dy;
          if (yy < 0 || yy >= gy) continue;
          const bool face = (dz == -Rr || dz == Rr || dy == -Rr || dy == Rr);
          const int step = face ? 1 : 2 * Rr;
          for (int dx = -Rr; dx <= Rr; dx += step) {
            const int xx = c[0] + dx;
            if (xx < 0 || xx >= gx) continue;
            const int cell = (zz * gy + yy) * gx + xx;
            const int b = pb.cl_start[cell], e = pb.cl_start[cell + 1];
            for (int base = b; base < e; base += 32) {
              const int qq = base + lane;
              const bool ok = qq < e;
              float cd = INFINITY;
              int cg = 0x7fffffff;
              if (ok) {
                const float4 c4 = pb.cl_pts4[qq];   // x, y, z, original index
                const float ddx = c4.x - q[0], ddy = c4.y - q[1], ddz = c4.z - q[2];
                cd = ddx * ddx + ddy * ddy + ddz * ddz;
                cg = __float_as_int(c4.w);
              }
              const float kd = __shfl_sync(kAll, ld, k - 1);
              const int kg = __shfl_sync(kAll, lg, k - 1);
              unsigned bm = __ballot_sync(kAll, ok && (cd < kd || (cd == kd && cg < kg)));
              while (bm) {
                const int s = __ffs(bm) - 1;
                bm &= bm - 1;
                const float nd = __shfl_sync(kAll, cd, s);
                const int ng = __shfl_sync(kAll, cg, s);
                const int np = base + s;
                const float pd = __shfl_up_sync(kAll, ld, 1);
                const int pg = __shfl_up_sync(kAll, lg, 1), pp = __shfl_up_sync(kAll, lp, 1);
                const bool lt_here = nd < ld || (nd == ld && ng < lg);
                const bool lt_prev = lane > 0 && (nd < pd || (nd == pd && ng < pg));
                if (lt_here) {
                  if (lt_prev) { ld = pd; lg = pg; lp = pp; } else { ld = nd; lg = ng; lp = np; }
                }
              }
            }
          }
        }
      }
      float guard = INFINITY;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (c[a] - Rr > 0) guard = fminf(guard, q[a] - (lo[a] + static_cast<float>(c[a] - Rr) * cs));
        if (c[a] + Rr < pb.cl_dims[a] - 1) guard = fminf(guard, (lo[a] + static_cast<float>(c[a] + Rr + 1) * cs) - q[a]);
      }
      const float kd = __shfl_sync(kAll, ld, k - 1);
      if (kd <= guard * guard || guard == INFINITY) break;
    }
#pragma unroll
    for (int j = 0; j < KM; ++j) {
      if (j < k) {
        const float dj = __shfl_sync(kAll, ld, j);
        const int pj = __shfl_sync(kAll, lp, j), gj = __shfl_sync(kAll, lg, j);
        if (lane == src) { R.d2[j] = dj; R.idx[j] = pj; R.gid[j] = gj; }
      }
    }
  }
  float h = 0.0f;
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < k) h += sqrtf(R.d2[j]);
  return h / static_cast<float>(k);
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi (columns of V).
template <typename T>
__device__ __forceinline__ void jacobi3_dev(T A[3][3], T lam[3], T V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? T(1) : T(0);
  for (int sweep = 0; sweep < 12; ++sweep) {
    const T off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    const T scale = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= T(1e-30) * scale || off == T(0)) break;
#pragma unroll
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      if (A[p][q] == T(0)) continue;
      const T th = (A[q][q] - A[p][p]) / (T(2) * A[p][q]);
      const T t = (th >= T(0) ? T(1) : T(-1)) / (fabs(th) + sqrt(th * th + T(1)));
      const T cc = T(1) / sqrt(t * t + T(1)), ss = t * cc;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const T arp = A[r][p], arq = A[r][q];
        A[r][p] = cc * arp - ss * arq;
        A[r][q] = ss * arp + cc * arq;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const T apr = A[p][r], aqr = A[q][r];
        A[p][r] = cc * apr - ss * aqr;
        A[q][r] = ss * apr + cc * aqr;
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const T vrp = V[r][p], vrq = V[r][q];
        V[r][p] = cc * vrp - ss * vrq;
        V[r][q] = ss * vrp + cc * vrq;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) lam[i] = A[i][i];
}

// cp(x) on the cloud from the neighbours R of x (h = their mean distance).
template <typename T, int KM>
__device__ __forceinline__ void cloud_project(const DevProblem& pb, const T* x, const Knn<T, KM>& R, T h, T* out) {
  const T* P = cloud_pts<T>(pb);
  const int k = pb.cl_k;
  if (pb.cl_mode == 1) {   // nearest cloud point
    const int q = R.idx[0];
    out[0] = P[3 * q]; out[1] = P[3 * q + 1]; out[2] = P[3 * q + 2];
    return;
  }
  T c[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < k) {
      const int q = R.idx[j];
      c[0] += P[3 * q]; c[1] += P[3 * q + 1]; c[2] += P[3 * q + 2];
    }
  c[0] /= T(k); c[1] /= T(k); c[2] /= T(k);
  T C[3][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < k) {
      const int q = R.idx[j];
      const T d[3] = {P[3 * q] - c[0], P[3 * q + 1] - c[1], P[3 * q + 2] - c[2]};
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) C[a][b] += d[a] * d[b];
    }
  T lam[3], V[3][3];
  jacobi3_dev<T>(C, lam, V);
  int imin = 0, imax = 0;
#pragma unroll
  for (int i = 1; i < 3; ++i) {
    if (lam[i] < lam[imin]) imin = i;
    if (lam[i] > lam[imax]) imax = i;
  }
  const T nr[3] = {V[0][imin], V[1][imin], V[2][imin]};
  const T u[3] = {V[0][imax], V[1][imax], V[2][imax]};
  const T v[3] = {nr[1] * u[2] - nr[2] * u[1], nr[2] * u[0] - nr[0] * u[2], nr[0] * u[1] - nr[1] * u[0]};
  const T s = h > T(0) ? h : T(1);
  // normal equations of the 6-coefficient height fit (upper triangle)
  T M[21], rhs[6];
#pragma unroll
  for (int i = 0; i < 21; ++i) M[i] = T(0);
#pragma unroll
  for (int i = 0; i < 6; ++i) rhs[i] = T(0);
#pragma unroll
  for (int j = 0; j < KM; ++j)
    if (j < k) {
      const int q = R.idx[j];
      const T d[3] = {(P[3 * q] - c[0]) / s, (P[3 * q + 1] - c[1]) / s, (P[3 * q + 2] - c[2]) / s};
      const T xi = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
      const T et = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
      const T ze = d[0] * nr[0] + d[1] * nr[1] + d[2] * nr[2];
      const T row[6] = {T(1), xi, et, xi * xi, xi * et, et * et};
      int t = 0;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        rhs[a] += row[a] * ze;
#pragma unroll
        for (int b = a; b < 6; ++b) M[t++] += row[a] * row[b];
      }
    }
  // Cholesky M = L L^T (packed), then two triangular solves
  T L[6][6];
  {
    int t = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int b = a; b < 6; ++b) { L[b][a] = M[t]; L[a][b] = M[t]; ++t; }
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    T dsum = L[j][j];
#pragma unroll
    for (int p = 0; p < j; ++p) dsum -= L[j][p] * L[j][p];
    // floor against a singular fit (collinear or repeated neighbours): a tiny
    // positive pivot representable in T (1e-300 underflows to 0 in FP32)
    const T djj = sqrt(fmax(dsum, sizeof(T) == 4 ? T(1e-30f) : T(1e-300)));
    L[j][j] = djj;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      T sum = L[i][j];
#pragma unroll
      for (int p = 0; p < j; ++p) sum -= L[i][p] * L[j][p];
      L[i][j] = sum / djj;
    }
  }
  T y6[6], a6[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    T sum = rhs[i];
#pragma unroll
    for (int p = 0; p < i; ++p) sum -= L[i][p] * y6[p];
    y6[i] = sum / L[i][i];
  }
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    T sum = y6[i];
#pragma unroll
    for (int p = i + 1; p < 6; ++p) sum -= L[p][i] * a6[p];
    a6[i] = sum / L[i][i];
  }
  const T d[3] = {(x[0] - c[0]) / s, (x[1] - c[1]) / s, (x[2] - c[2]) / s};
  const T xi0 = d[0] * u[0] + d[1] * u[1] + d[2] * u[2];
  const T et0 = d[0] * v[0] + d[1] * v[1] + d[2] * v[2];
  const T ze0 = d[0] * nr[0] + d[1] * nr[1] + d[2] * nr[2];
  const T hz = a6[0] + a6[1] * xi0 + a6[2] * et0 + a6[3] * xi0 * xi0 + a6[4] * xi0 * et0 + a6[5] * et0 * et0;
  const T hx = a6[1] + T(2) * a6[3] * xi0 + a6[4] * et0;
  const T hy = a6[2] + a6[4] * xi0 + T(2) * a6[5] * et0;
  const T e = hz - ze0;
  const T g0 = e * hx, g1 = e * hy;
  const T H00 = T(1) + hx * hx + e * T(2) * a6[3], H01 = hx * hy + e * a6[4], H11 = T(1) + hy * hy + e * T(2) * a6[5];
  const T det = H00 * H11 - H01 * H01;
  const T xi1 = xi0 - (H11 * g0 - H01 * g1) / det;
  const T et1 = et0 - (H00 * g1 - H01 * g0) / det;
  const T z1 = a6[0] + a6[1] * xi1 + a6[2] * et1 + a6[3] * xi1 * xi1 + a6[4] * xi1 * et1 + a6[5] * et1 * et1;
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = c[i] + s * (xi1 * u[i] + et1 * v[i] + z1 * nr[i]);
}

// ---------------------------------------------------------------------------
// k-nearest queries outside the walk (verification and the search comparison)
// ---------------------------------------------------------------------------
template <typename T, int KM>
__device__ __forceinline__ void knn_store(const Knn<T, KM>& R, int k, T hq, int64_t q, int32_t* idx, double* d2,
                                          double* h) {
#pragma unroll
  for (int j = 0; j < KM; ++j) {
    if (j < k) {
      idx[q * k + j] = R.gid[j];
      d2[q * k + j] = static_cast<double>(R.d2[j]);
    }
  }
  h[q] = static_cast<double>(hq);
}

// The walk's own grid search for nq query points (x: nq x 3, FP64, converted
// to T as the walk holds them).  COOP (FP32 only): the warp-cooperative search,
// all 32 lanes of a warp passing through it together.
template <typename T, int KM, bool COOP>
__global__ void __launch_bounds__(128) cloud_knn_query_kernel(const DevProblem pb, const double* xq, int64_t nq,
                                                              int32_t* idx, double* d2, double* h) {
  const int64_t nthreads = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x - lane); base < nq;
       base += nthreads) {   // warp-uniform trip count
    const int64_t q = base + lane;
    const bool has = q < nq;
    T x[3] = {T(0), T(0), T(0)};
    if (has)
      for (int a = 0; a < 3; ++a) x[a] = static_cast<T>(xq[3 * q + a]);
    Knn<T, KM> R;
    T hq;
    if constexpr (COOP) {
      hq = cloud_knn_coop<KM>(pb, x, has, R);
    } else {
      if (!has) continue;
      hq = cloud_knn<T, KM>(pb, x, R);
    }
    if (has) knn_store<T, KM>(R, pb.cl_k, hq, q, idx, d2, h);
  }
}

// The all-pairs search: every cloud point against each query, the cloud
// staged through shared memory kScanTile points at a time as (x, y, z,
// original index) quadruples (one 16-byte load per point in FP32).  Tile t
// holds the sorted positions t, t + T, t + 2T, ... (T tiles): a sample of the
// whole cloud, so the first tile already bounds the k-th distance closely and
// later insertions are rare (in cell order a query's bound would shrink only
// as the sweep approached it, inserting thousands of times).  Each thread
// serves kScanQ queries (q0 + m blockDim.x), so that one pass of the cloud
// through L2 serves kScanQ x 128 queries, and keeps each query's current k-th
// distance in a register so that most pairs end after one comparison.  Same
// distances and the same (distance^2, original index) order as the grid
// search, so the same k nearest; kept as the measured comparison for it.
constexpr int kScanTile = 512;
constexpr int kScanQ = 4;

// knn_insert out of line: the scan's rare insertions stay off the per-pair path.
template <typename T, int KM>
__device__ __noinline__ void knn_insert_outlined(Knn<T, KM>& R, int k, T dd, int pos, int g) {
  knn_insert<T, KM>(R, k, dd, pos, g);
}

template <typename T>
struct ScanPt { T x, y, z; int g; };
template <>
struct __align__(16) ScanPt<float> { float x, y, z; int g; };

template <typename T, int KM>
__global__ void __launch_bounds__(128) cloud_knn_scan_kernel(const DevProblem pb, const double* xq, int64_t nq,
                                                             int64_t ncl, int32_t* idx, double* d2, double* h) {
  __shared__ ScanPt<T> sp[kScanTile];
  const int64_t q0 = static_cast<int64_t>(blockIdx.x) * blockDim.x * kScanQ + threadIdx.x;
  const int k = pb.cl_k;
  T x[kScanQ][3];
  bool has[kScanQ];
  T kth[kScanQ];
  Knn<T, KM> R[kScanQ];
#pragma unroll
  for (int m = 0; m < kScanQ; ++m) {
    const int64_t q = q0 + static_cast<int64_t>(m) * blockDim.x;
    has[m] = q < nq;
    for (int a = 0; a < 3; ++a) x[m][a] = has[m] ? static_cast<T>(xq[3 * q + a]) : T(0);
    kth[m] = T(INFINITY);
#pragma unroll
    for (int j = 0; j < KM; ++j) { R[m].d2[j] = T(INFINITY); R[m].idx[j] = -1; R[m].gid[j] = 0x7fffffff; }
  }
  const T* P = cloud_pts<T>(pb);
  const int64_t ntiles = (ncl + kScanTile - 1) / kScanTile;
  for (int64_t t = 0; t < ntiles; ++t) {
    const int nt = static_cast<int>((ncl - t + ntiles - 1) / ntiles);   // positions t + i ntiles < ncl
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      const int64_t pi = t + static_cast<int64_t>(i) * ntiles;
      if constexpr (sizeof(T) == 4) {
        const float4 c4 = pb.cl_pts4[pi];
        sp[i] = ScanPt<T>{c4.x, c4.y, c4.z, __float_as_int(c4.w)};
      } else {
        sp[i] = ScanPt<T>{P[3 * pi], P[3 * pi + 1], P[3 * pi + 2], pb.cl_orig[pi]};
      }
    }
    __syncthreads();
    for (int i = 0; i < nt; ++i) {
      const ScanPt<T> c = sp[i];
      const int pos = static_cast<int>(t + static_cast<int64_t>(i) * ntiles);
#pragma unroll
      for (int m = 0; m < kScanQ; ++m) {
        const T ddx = c.x - x[m][0], ddy = c.y - x[m][1], ddz = c.z - x[m][2];
        const T dd = ddx * ddx + ddy * ddy + ddz * ddz;
        if (has[m] && dd <= kth[m]) {   // otherwise knn_insert would reject it too
          knn_insert_outlined<T, KM>(R[m], k, dd, pos, c.g);
          kth[m] = R[m].d2[k - 1];
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < kScanQ; ++m) {
    if (!has[m]) continue;
    T hq = T(0);
#pragma unroll
    for (int j = 0; j < KM; ++j)
      if (j < k) hq += sqrt(R[m].d2[j]);
    knn_store<T, KM>(R[m], k, hq / T(k), q0 + static_cast<int64_t>(m) * blockDim.x, idx, d2, h);
  }
}

}  // namespace mpwos
