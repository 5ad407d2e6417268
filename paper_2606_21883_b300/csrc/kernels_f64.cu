// kernels_f64.cu — FP64 kernels: the FP64 walks, the radius tables, the
// per-point reduction and the verification primitives.  Compiled with
// --fmad=false so that every FP64 + and * is one IEEE operation.
#include "launch.h"
#include "estimator.cuh"
#include "walk3.cuh"
#include "walkn.cuh"
#include "cloud.cuh"
#include "walkr.cuh"

namespace mpwos {

// ---------------------------------------------------------------------------
// Radius tables (layout in green.cuh): one thread per node; bisection to a
// bracket, then the safeguarded Newton polish, in FP64.
// ---------------------------------------------------------------------------
__global__ void build_table_kernel(int n, int NA, int NS, double z_max, double a_fixed, double* tab64) {
  const int side_len = NS + 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NA * 2 * side_len) return;
  const int ia = idx / (2 * side_len);
  const int rem = idx - ia * 2 * side_len;
  const int side = rem / side_len;
  const int j = rem - side * side_len - 1;            // node index -1 .. NS
  const double a = (NA == 1) ? a_fixed : 2.0 * sqrt(z_max * static_cast<double>(ia) / static_cast<double>(NA - 1));
  const double v = static_cast<double>(j < 0 ? -j : j) * (kTableVmax / static_cast<double>(NS - 1));
  const double U = side == 0 ? v * v : 1.0 - v * v;
  const GreenLaw L = green_law(n, a);
  double t;
  if (U <= 0.0) {
    t = 0.0;
  } else if (U >= 1.0) {
    t = 1.0;
  } else {
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 12; ++it) {   // bracket to 2^-12, then Newton converges in a few steps
      const double mid = 0.5 * (lo + hi);
      double F, dF;
      green_cdf_pdf(L, mid, F, dF);
      if (F < U) lo = mid; else hi = mid;
    }
    t = green_invert64(L, U, 0.5 * (lo + hi));
  }
  if (j < 0) t = side == 0 ? -t : 2.0 - t;
  tab64[idx] = t;
}

// Monomial coefficients of each interval's Catmull-Rom cubic, in FP64 from the
// FP64 nodes p0..p3 (nodes j-1 .. j+2):
//   t(f) = p1 + f (p2 - p0)/2 + f^2 (2 p0 - 5 p1 + 4 p2 - p3)/2 + f^3 (3 (p1 - p2) + p3 - p0)/2.
__global__ void build_coef_kernel(int NA, int NS, const double* tab64, float4* tabc) {
  const int NI = NS - 1, side_len = NS + 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NA * 2 * NI) return;
  const int row = idx / NI, j = idx - row * NI;   // row = 2 ia + side
  const double* nd = tab64 + static_cast<size_t>(row) * side_len + j;
  const double p0 = nd[0], p1 = nd[1], p2 = nd[2], p3 = nd[3];
  tabc[idx] = make_float4(static_cast<float>(p1), static_cast<float>(0.5 * (p2 - p0)),
                          static_cast<float>(0.5 * (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3)),
                          static_cast<float>(0.5 * (3.0 * (p1 - p2) + p3 - p0)));
}

cudaError_t launch_build_table(int n, int NA, int NS, double z_max, double a_fixed, double* tab64,
                               float4* tabc, cudaStream_t st) {
  const int total = NA * 2 * (NS + 2);
  build_table_kernel<<<(total + 127) / 128, 128, 0, st>>>(n, NA, NS, z_max, a_fixed, tab64);
  const int nint = NA * 2 * (NS - 1);
  build_coef_kernel<<<(nint + 127) / 128, 128, 0, st>>>(NA, NS, tab64, tabc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-point estimator (eq. mc_estimator) in the block order of estimator.cuh:
// one warp per point.  part == null: the blocks merge in order into the mean,
// its standard error and the mean stopping index; otherwise each block's
// record (count, mean, M2, sum of K, flagged walks) goes to
// part[((p nblk_part) + b) kEstFields ...].
__global__ void reduce_kernel(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t Nu,
                              int64_t stride, const int64_t* n_per_point, double* mean, double* se, double* msteps,
                              unsigned long long* n_flagged, double* part, int64_t nblk_part) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (p >= P) return;
  const int64_t N = n_per_point ? n_per_point[p] : Nu;
  const double* Sp = S + p * stride;
  const int32_t* Kp = K + p * stride;
  const int32_t* Fp = flags + p * stride;
  Stat acc{0.0, 0.0, 0.0};
  long long ks_all = 0, nf_all = 0;
  const int64_t nblk = (N + kEstBlock - 1) / kEstBlock;
  for (int64_t b = 0; b < nblk; ++b) {
    const int64_t base = b * kEstBlock;
    const int64_t nb = (N - base < kEstBlock) ? N - base : kEstBlock;
    const int cnt = lane_count(nb, lane);
    Stat st = stat_lane(Sp + base + lane, cnt);
    long long ks = 0, nf = 0;
    for (int t = 0; t < cnt; ++t) {
      ks += Kp[base + lane + 32 * t];
      nf += Fp[base + lane + 32 * t];
    }
    for (int off = 16; off > 0; off >>= 1) {
      const Stat o{__shfl_down_sync(0xffffffffu, st.n, off), __shfl_down_sync(0xffffffffu, st.m, off),
                   __shfl_down_sync(0xffffffffu, st.M, off)};
      ks += __shfl_down_sync(0xffffffffu, ks, off);
      nf += __shfl_down_sync(0xffffffffu, nf, off);
      if (lane < off) st = stat_merge(st, o);
    }
    if (lane == 0) {
      if (part) {
        if (b < nblk_part) {
          double* rec = part + (p * nblk_part + b) * kEstFields;
          rec[0] = st.n; rec[1] = st.m; rec[2] = st.M;
          rec[3] = static_cast<double>(ks); rec[4] = static_cast<double>(nf);
        }
      } else {
        acc = stat_merge(acc, st);
        ks_all += ks;
        nf_all += nf;
      }
    }
  }
  if (!part && lane == 0) {
    double mu, s;
    stat_finish(acc, mu, s);
    mean[p] = mu;
    se[p] = s;
    msteps[p] = N > 0 ? static_cast<double>(ks_all) / static_cast<double>(N) : 0.0;
    if (nf_all) atomicAdd(n_flagged, static_cast<unsigned long long>(nf_all));
  }
}

cudaError_t launch_reduce(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                          double* mean, double* se, double* msteps, unsigned long long* n_flagged,
                          cudaStream_t st) {
  return launch_reduce_strided(S, K, flags, P, N, N, nullptr, mean, se, msteps, n_flagged, st);
}

cudaError_t launch_reduce_strided(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                                  int64_t stride, const int64_t* n_per_point, double* mean, double* se,
                                  double* msteps, unsigned long long* n_flagged, cudaStream_t st) {
  const int block = 256;
  const int64_t grid = (P * 32 + block - 1) / block;
  reduce_kernel<<<static_cast<unsigned>(grid), block, 0, st>>>(S, K, flags, P, N, stride, n_per_point, mean, se,
                                                               msteps, n_flagged, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_reduce_blocks(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                                 double* part, cudaStream_t st) {
  if (P <= 0) return cudaSuccess;
  const int block = 256;
  const int64_t grid = (P * 32 + block - 1) / block;
  const int64_t nblk = (N + kEstBlock - 1) / kEstBlock;
  reduce_kernel<<<static_cast<unsigned>(grid), block, 0, st>>>(S, K, flags, P, N, N, nullptr, nullptr, nullptr,
                                                               nullptr, nullptr, part, nblk);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 walks
// ---------------------------------------------------------------------------
static const void* walk3_f64_fn(const DevProblem& pb) {
  switch (pb.mkind) {
    case kEuclid: return reinterpret_cast<const void*>(walk3_f64_kernel<kEuclid, 1>);
    case kSphere:
      return pb.pred.comp != kCompNone ? reinterpret_cast<const void*>(walk3_f64_kernel<kSphere, 1, true>)
                                       : reinterpret_cast<const void*>(walk3_f64_kernel<kSphere, 1>);
    case kTorus:
      return pb.pred.comp != kCompNone ? reinterpret_cast<const void*>(walk3_f64_kernel<kTorus, 1, true>)
                                       : reinterpret_cast<const void*>(walk3_f64_kernel<kTorus, 1>);
    case kPointCloud:
      return pb.cl_k <= 8 ? reinterpret_cast<const void*>(walk3_f64_kernel<kPointCloud, 8>)
           : pb.cl_k <= 16 ? reinterpret_cast<const void*>(walk3_f64_kernel<kPointCloud, 16>)
                           : reinterpret_cast<const void*>(walk3_f64_kernel<kPointCloud, 32>);
    default: return nullptr;
  }
}

cudaError_t launch_walk3_f64(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  const void* fn = walk3_f64_fn(pb);
  if (!fn) return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

static const void* walkn_f64_fn(const DevProblem& pb) {
  if (pb.mkind == kEuclid) return reinterpret_cast<const void*>(walkn_f64_kernel<kEuclid, 8>);
  if (pb.mkind == kSphere) return reinterpret_cast<const void*>(walkn_f64_kernel<kSphere, 8>);
  if (pb.mkind == kRevolution) return reinterpret_cast<const void*>(walkn_f64_kernel<kRevolution, 8>);
  if (pb.mkind == kCurveSphere) return reinterpret_cast<const void*>(walkn_f64_kernel<kCurveSphere, 8>);
  switch (walkn_dq(pb.d + 1)) {
    case 8: return reinterpret_cast<const void*>(walkn_f64_kernel<kEmbeddedSphere, 8>);
    case 16: return reinterpret_cast<const void*>(walkn_f64_kernel<kEmbeddedSphere, 16>);
    case 24: return reinterpret_cast<const void*>(walkn_f64_kernel<kEmbeddedSphere, 24>);
    default: return reinterpret_cast<const void*>(walkn_f64_kernel<kEmbeddedSphere, 32>);
  }
}

cudaError_t launch_walkn_f64(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  if (pb.mkind != kEuclid && pb.mkind != kSphere && pb.mkind != kEmbeddedSphere && pb.mkind != kRevolution &&
      pb.mkind != kCurveSphere)
    return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(walkn_f64_fn(pb), dim3(grid), dim3(block), args, 0, st);
}

template <typename T>
static const void* walkr_fn(const DevProblem& pb) {
  const int nt = walkr_nt(pb.red_nT);
#define MPWOS_WALKR(MK)                                                              \
  switch (nt) {                                                                      \
    case 4: return reinterpret_cast<const void*>(walkr_kernel<T, MK, 4>);            \
    case 8: return reinterpret_cast<const void*>(walkr_kernel<T, MK, 8>);            \
    case 16: return reinterpret_cast<const void*>(walkr_kernel<T, MK, 16>);          \
    case 24: return reinterpret_cast<const void*>(walkr_kernel<T, MK, 24>);          \
    default: return reinterpret_cast<const void*>(walkr_kernel<T, MK, 32>);          \
  }
  if (pb.mkind == kEuclid) { MPWOS_WALKR(kEuclid) }
  if (pb.mkind == kSphere) { MPWOS_WALKR(kSphere) }
  MPWOS_WALKR(kEmbeddedSphere)
#undef MPWOS_WALKR
}

cudaError_t launch_walkr_f64(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  if (pb.mkind != kEuclid && pb.mkind != kSphere && pb.mkind != kEmbeddedSphere) return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(walkr_fn<double>(pb), dim3(grid), dim3(block), args, 0, st);
}

// Per point: y_T and rho = sqrt(|y|^2 - |y_T|^2) (sphere) of the reduced state,
// row p of red_y0 = [y_T (kMaxQuadDim slots), rho].
__global__ void reduced_start_kernel(const double* pts, int n, const int* T, int nT, int64_t P, int sphere,
                                     double* out) {
  const int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double* y = pts + static_cast<size_t>(p) * n;
  double* o = out + static_cast<size_t>(p) * (kMaxQuadDim + 1);
  double tt = 0.0;
  for (int q = 0; q < kMaxQuadDim; ++q) {
    const double v = q < nT ? y[T[q]] : 0.0;
    o[q] = v;
    tt += v * v;
  }
  double rho = 0.0;
  if (sphere) {
    double yy = 0.0;
    for (int q = 0; q < n; ++q) yy += y[q] * y[q];
    rho = sqrt(yy - tt > 0.0 ? yy - tt : 0.0);
  }
  o[kMaxQuadDim] = rho;
}

cudaError_t launch_reduced_start(const double* pts, int n, const int* T, int nT, int64_t P, int sphere, double* out,
                                 cudaStream_t st) {
  reduced_start_kernel<<<static_cast<unsigned>((P + 127) / 128), 128, 0, st>>>(pts, n, T, nT, P, sphere, out);
  return cudaGetLastError();
}

cudaError_t launch_cloud_knn_f64(const DevProblem& pb, const double* x, int64_t nq, int method, int64_t ncl,
                                 int32_t* idx, double* d2, double* h, int max_blocks, cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  const int64_t need = (nq + 127) / 128;
  const unsigned grid = static_cast<unsigned>(need < max_blocks ? need : max_blocks);
  const bool small = pb.cl_k <= 8, mid = pb.cl_k <= 16;
  if (method == 0) {
    if (small) cloud_knn_query_kernel<double, 8, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
    else if (mid) cloud_knn_query_kernel<double, 16, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
    else cloud_knn_query_kernel<double, 32, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
  } else if (method == 2) {
    const unsigned g = static_cast<unsigned>((nq + 128 * kScanQ - 1) / (128 * kScanQ));
    if (small) cloud_knn_scan_kernel<double, 8><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
    else if (mid) cloud_knn_scan_kernel<double, 16><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
    else cloud_knn_scan_kernel<double, 32><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

const void* walk_fn_f64(const DevProblem& pb) {
  if (pb.reduced)
    return (pb.mkind == kEuclid || pb.mkind == kSphere || pb.mkind == kEmbeddedSphere) ? walkr_fn<double>(pb)
                                                                                       : nullptr;
  if (pb.n == 3 && pb.mkind != kEmbeddedSphere) return walk3_f64_fn(pb);
  if (pb.mkind != kEuclid && pb.mkind != kSphere && pb.mkind != kEmbeddedSphere && pb.mkind != kRevolution &&
      pb.mkind != kCurveSphere)
    return nullptr;
  return walkn_f64_fn(pb);
}

int occupancy_walkr_f64(const DevProblem& pb, int block) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walkr_fn<double>(pb), block, 0);
  return nb < 1 ? 1 : nb;
}

int occupancy_walk_f64(const DevProblem& pb, bool n3, int block) {
  int nb = 0;
  const void* fn = nullptr;
  if (n3) {
    fn = walk3_f64_fn(pb);
  } else {
    fn = walkn_f64_fn(pb);
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0);
  return nb < 1 ? 1 : nb;
}

// ---------------------------------------------------------------------------
// Verification primitives
// ---------------------------------------------------------------------------
__global__ void philox_kernel(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int64_t count) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const U4 r = philox4x32_10(ctr[4 * q], ctr[4 * q + 1], ctr[4 * q + 2], ctr[4 * q + 3], k0, k1);
  out[4 * q] = r.x; out[4 * q + 1] = r.y; out[4 * q + 2] = r.z; out[4 * q + 3] = r.w;
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int64_t count,
                          cudaStream_t st) {
  philox_kernel<<<static_cast<unsigned>((count + 127) / 128), 128, 0, st>>>(ctr, k0, k1, out, count);
  return cudaGetLastError();
}

__global__ void green_radius64_kernel(int n, const double* a, const double* U, double* t, int64_t count,
                                      const double* tab64, int NA, int NS, double z_max) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const GreenLaw L = green_law(n, a[q]);
  const double guess = table_lookup<double>(tab64, NA, NS, z_max, a[q], U[q]);
  t[q] = green_invert64(L, U[q], guess);
}

cudaError_t launch_green_radius64(int n, const double* a, const double* U, double* t, int64_t count,
                                  const double* tab64, int NA, int NS, double z_max, cudaStream_t st) {
  green_radius64_kernel<<<static_cast<unsigned>((count + 127) / 128), 128, 0, st>>>(n, a, U, t, count, tab64,
                                                                                   NA, NS, z_max);
  return cudaGetLastError();
}

__global__ void c_sigma_r_kernel(int n, const double* a, double* c, int64_t count) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const double em1 = em1_series(0.5 * static_cast<double>(n - 2), 0.25 * (a[q] * a[q]));
  c[q] = 1.0 / (1.0 + em1);
}

cudaError_t launch_c_sigma_r(int n, const double* a, double* c, int64_t count, cudaStream_t st) {
  c_sigma_r_kernel<<<static_cast<unsigned>((count + 127) / 128), 128, 0, st>>>(n, a, c, count);
  return cudaGetLastError();
}

}  // namespace mpwos

namespace mpwos {

// s0 = normalize(Q^T (y0 - b)) for each query point (embedded sphere start state).
__global__ void intrinsic_start_kernel(const double* pts, const double* QT, const double* b, int n, int npad,
                                       int D, int64_t P, double* s0) {
  const int lane = threadIdx.x & 31;
  const int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (p >= P) return;
  double sj = 0.0;
  if (lane < D) {
    const double* y = pts + p * n;
    const double* row = QT + static_cast<size_t>(lane) * npad;
    for (int i = 0; i < n; ++i) sj += row[i] * (y[i] - b[i]);
  }
  const double nn = sqrt(warp_sum1(sj * sj));
  if (lane < D) s0[p * D + lane] = sj / nn;
}

cudaError_t launch_intrinsic_start(const double* pts, const double* QT, const double* b, int n, int npad, int D, int64_t P,
                                   double* s0, cudaStream_t st) {
  const int block = 128;
  intrinsic_start_kernel<<<static_cast<unsigned>((P * 32 + block - 1) / block), block, 0, st>>>(pts, QT, b, n, npad,
                                                                                               D, P, s0);
  return cudaGetLastError();
}

}  // namespace mpwos

// ---------------------------------------------------------------------------
// Point-cloud grid: cell of each point, counts, exclusive scan, scatter into
// cell order (original index kept), and h(p) at every cloud point (its max
// sets the radius-table range).
// ---------------------------------------------------------------------------
namespace mpwos {

__global__ void cloud_cell_kernel(const double* pts, int64_t N, double ox, double oy, double oz, double cs, int gx,
                                  int gy, int gz, int* cell, int* counts) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int c[3];
  const double o[3] = {ox, oy, oz};
  const int g[3] = {gx, gy, gz};
  for (int a = 0; a < 3; ++a) {
    int ci = static_cast<int>(floor((pts[3 * i + a] - o[a]) / cs));
    c[a] = ci < 0 ? 0 : (ci >= g[a] ? g[a] - 1 : ci);
  }
  const int id = (c[2] * gy + c[1]) * gx + c[0];
  cell[i] = id;
  atomicAdd(&counts[id], 1);
}

// Exclusive scan of counts (ncells) into start (ncells + 1), one block.
__global__ void cloud_scan_kernel(const int* counts, int ncells, int* start) {
  __shared__ int partial[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (ncells + T - 1) / T;
  const int b = t * per, e = min(ncells, b + per);
  int s = 0;
  for (int q = b; q < e; ++q) s += counts[q];
  partial[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int q = 0; q < T; ++q) { const int v = partial[q]; partial[q] = run; run += v; }
    start[ncells] = run;
  }
  __syncthreads();
  int run = partial[t];
  for (int q = b; q < e; ++q) { start[q] = run; run += counts[q]; }
}

__global__ void cloud_scatter_kernel(const double* pts, int64_t N, const int* cell, const int* start, int* cursor,
                                     double* spts64, float* spts32, float4* spts4, int* orig) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int id = cell[i];
  const int pos = start[id] + atomicAdd(&cursor[id], 1);
  for (int a = 0; a < 3; ++a) {
    spts64[3 * pos + a] = pts[3 * i + a];
    spts32[3 * pos + a] = static_cast<float>(pts[3 * i + a]);
  }
  spts4[pos] = make_float4(static_cast<float>(pts[3 * i]), static_cast<float>(pts[3 * i + 1]),
                           static_cast<float>(pts[3 * i + 2]), __int_as_float(static_cast<int>(i)));
  orig[pos] = static_cast<int>(i);
}

template <int KM>
__global__ void cloud_hmax_kernel(const DevProblem pb, int64_t N, unsigned long long* hmax_bits) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const double x[3] = {pb.cl_pts64[3 * q], pb.cl_pts64[3 * q + 1], pb.cl_pts64[3 * q + 2]};
  Knn<double, KM> R;
  const double h = cloud_knn<double, KM>(pb, x, R);
  atomicMax(hmax_bits, static_cast<unsigned long long>(__double_as_longlong(h)));
}

cudaError_t launch_cloud_grid(const double* pts, int64_t N, const double origin[3], double cs, const int dims[3],
                              int* cell, int* counts, int* start, int* cursor, double* spts64, float* spts32,
                              float4* spts4, int* orig, cudaStream_t st) {
  const int ncells = dims[0] * dims[1] * dims[2];
  cudaMemsetAsync(counts, 0, sizeof(int) * ncells, st);
  cudaMemsetAsync(cursor, 0, sizeof(int) * ncells, st);
  const unsigned grid = static_cast<unsigned>((N + 255) / 256);
  cloud_cell_kernel<<<grid, 256, 0, st>>>(pts, N, origin[0], origin[1], origin[2], cs, dims[0], dims[1], dims[2], cell,
                                          counts);
  cloud_scan_kernel<<<1, 1024, 0, st>>>(counts, ncells, start);
  cloud_scatter_kernel<<<grid, 256, 0, st>>>(pts, N, cell, start, cursor, spts64, spts32, spts4, orig);
  return cudaGetLastError();
}

cudaError_t launch_cloud_hmax(const DevProblem& pb, int64_t N, unsigned long long* hmax_bits, cudaStream_t st) {
  const unsigned grid = static_cast<unsigned>((N + 127) / 128);
  if (pb.cl_k <= 8) cloud_hmax_kernel<8><<<grid, 128, 0, st>>>(pb, N, hmax_bits);
  else if (pb.cl_k <= 16) cloud_hmax_kernel<16><<<grid, 128, 0, st>>>(pb, N, hmax_bits);
  else cloud_hmax_kernel<32><<<grid, 128, 0, st>>>(pb, N, hmax_bits);
  return cudaGetLastError();
}

}  // namespace mpwos
