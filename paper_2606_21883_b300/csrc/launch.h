// launch.h — host-side launchers of the library's kernels (internal C++ API).
#pragma once
#include <cuda_runtime.h>
#include "dev_common.cuh"

namespace mpwos {

// Walks for R^3 manifolds, one thread per walker (kernels_f64.cu / kernels_f32.cu).
cudaError_t launch_walk3_f64(const DevProblem& pb, int grid, int block, cudaStream_t st);
cudaError_t launch_walk3_f32(const DevProblem& pb, int grid, int block, cudaStream_t st);
// Walks for R^n manifolds (n > 3), one warp per walker.
cudaError_t launch_walkn_f64(const DevProblem& pb, int grid, int block, cudaStream_t st);
cudaError_t launch_walkn_f32(const DevProblem& pb, int grid, int block, cudaStream_t st);
// The FP32 warp walk's kernel for pb (kernels_n32.cu; null if none applies) and
// its resident blocks per SM.
const void* walkn32_fn(const DevProblem& pb);
int occupancy_walkn32(const DevProblem& pb, int block);
// Lanes per walker of that kernel (16 or 32) and its largest block (also its
// default block size).
int walkn32_lanes_per_walker(const DevProblem& pb);
int walkn32_max_block(const DevProblem& pb);
// FP32 embedded-sphere walk with the projection on the tensor cores (one
// persistent 512-thread CTA per SM, 128 walkers per tile; pb.tc_bimg set).
cudaError_t launch_embed_tc(const DevProblem& pb, int grid, cudaStream_t st);
// Size in bytes of the tensor-core kernel's shared-memory image of Q^T.
size_t embed_tc_bimg_bytes();
// out (rows x 32) = G Q through the walk's tensor-core contraction, gg = |G_row|^2.
cudaError_t launch_tc_project(const uint4* bimg, const float* G, int64_t rows, int n, float* out, float* gg,
                              unsigned* status, int grid, cudaStream_t st);
// Walks with the dimension-reduced sampler, one thread per walker.
cudaError_t launch_walkr_f64(const DevProblem& pb, int grid, int block, cudaStream_t st);
cudaError_t launch_walkr_f32(const DevProblem& pb, int grid, int block, cudaStream_t st);
int occupancy_walkr(const DevProblem& pb, bool fp64, int block);
// The reduced embedded-sphere walk with one warp per walker (FP32, N_V = 1): for
// launches of few walks; bit-identical walks to launch_walkr_f32's.  128-thread
// blocks, 4 walkers each.
bool walkr_lat_eligible(const DevProblem& pb);
cudaError_t launch_walkr_lat_f32(const DevProblem& pb, int grid, cudaStream_t st);
// Reduced start states (y_T, |y_rest|) of the query points.
cudaError_t launch_reduced_start(const double* pts, int n, const int* T, int nT, int64_t P, int sphere, double* out,
                                 cudaStream_t st);
// Resident blocks per SM of the walk kernel chosen for pb.
int occupancy_walk_f64(const DevProblem& pb, bool n3, int block);
int occupancy_walk_f32(const DevProblem& pb, bool n3, int block);
// The kernel that launch_walkr_*, launch_walk3_* or launch_walkn_* runs for pb
// (reduced sampler, n = 3 thread walk or warp walk, in that order); nullptr if
// none applies.  The launch-shape autotuner keys its picks by it.
const void* walk_fn_f64(const DevProblem& pb);
const void* walk_fn_f32(const DevProblem& pb);

// Intrinsic start points s0 = normalize(Q^T (y0 - b)) of an embedded sphere
// (QT: D x n device array), one warp per point.
cudaError_t launch_intrinsic_start(const double* pts, const double* QT, const double* b, int n, int npad, int D, int64_t P,
                                   double* s0, cudaStream_t st);

// Per-point mean, standard error and mean steps from per-walk scores.
cudaError_t launch_reduce(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                          double* mean, double* se, double* msteps, unsigned long long* n_flagged,
                          cudaStream_t st);

// Per-point, per-block estimator records (estimator.cuh) of P x N per-walk
// outputs: part holds P x ceil(N / kEstBlock) x kEstFields doubles.
cudaError_t launch_reduce_blocks(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                                 double* part, cudaStream_t st);

// Same over a strided per-walk layout (row p at p * stride), each point with
// n_per_point[p] walks (N walks for every point when n_per_point is null).
cudaError_t launch_reduce_strided(const double* S, const int32_t* K, const int32_t* flags, int64_t P, int64_t N,
                                  int64_t stride, const int64_t* n_per_point, double* mean, double* se,
                                  double* msteps, unsigned long long* n_flagged, cudaStream_t st);

// Inverse-CDF tables of the radial Green law: NA rows over z = a^2/4 in
// [0, z_max] (NA == 1: the single law at a = a_fixed); two sides of NS + 2
// FP64 nodes per row, and NS - 1 float4 interval cubics per side for FP32.
cudaError_t launch_build_table(int n, int NA, int NS, double z_max, double a_fixed, double* tab64,
                               float4* tabc, cudaStream_t st);

// Point-cloud grid (counting sort by cell) and the largest h(p) over the cloud.
cudaError_t launch_cloud_grid(const double* pts, int64_t N, const double origin[3], double cs, const int dims[3],
                              int* cell, int* counts, int* start, int* cursor, double* spts64, float* spts32,
                              float4* spts4, int* orig, cudaStream_t st);
cudaError_t launch_cloud_hmax(const DevProblem& pb, int64_t N, unsigned long long* hmax_bits, cudaStream_t st);

// k nearest cloud points of nq queries (x: nq x 3 FP64, device) by method
// (0: the walk's grid search, 1: its warp-cooperative form, FP32 only, 2: the
// all-pairs scan); idx and d2 nq x k, h nq, all device arrays.
cudaError_t launch_cloud_knn_f32(const DevProblem& pb, const double* x, int64_t nq, int method, int64_t ncl,
                                 int32_t* idx, double* d2, double* h, int max_blocks, cudaStream_t st);
cudaError_t launch_cloud_knn_f64(const DevProblem& pb, const double* x, int64_t nq, int method, int64_t ncl,
                                 int32_t* idx, double* d2, double* h, int max_blocks, cudaStream_t st);

// Verification primitives.
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int64_t count,
                          cudaStream_t st);
cudaError_t launch_green_radius64(int n, const double* a, const double* U, double* t, int64_t count,
                                  const double* tab64, int NA, int NS, double z_max, cudaStream_t st);
cudaError_t launch_green_radius32(const double* a, const double* U, double* t, int64_t count, const float4* tabc,
                                  int NA, int NS, double z_max, cudaStream_t st);
cudaError_t launch_c_sigma_r(int n, const double* a, double* c, int64_t count, cudaStream_t st);

}  // namespace mpwos
