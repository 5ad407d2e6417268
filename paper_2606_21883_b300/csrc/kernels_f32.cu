// kernels_f32.cu — FP32 walks (FP64 weights and score) and the FP32 radius
// sampler.  Compiled with fast single-precision math (MUFU transcendentals,
// FMA contraction); the FP64 parts keep IEEE double arithmetic.
#include "launch.h"
#include "walk3.cuh"
#include "embed_tc.cuh"
#include "walkr.cuh"

namespace mpwos {

static const void* walk3_f32_fn(const DevProblem& pb) {
  switch (pb.mkind) {
    case kEuclid:
      return pb.closed ? reinterpret_cast<const void*>(walk3_f32_kernel<kEuclid, 1, true>)
                       : reinterpret_cast<const void*>(walk3_f32_kernel<kEuclid, 1, false>);
    case kSphere:
      if (pb.pred.comp != kCompNone) return reinterpret_cast<const void*>(walk3_f32_kernel<kSphere, 1, false, -1, true>);
      return pb.closed ? reinterpret_cast<const void*>(walk3_f32_kernel<kSphere, 1, true>)
                       : reinterpret_cast<const void*>(walk3_f32_kernel<kSphere, 1, false>);
    case kTorus: {
      if (pb.pred.comp != kCompNone) return reinterpret_cast<const void*>(walk3_f32_kernel<kTorus, 1, false, -1, true>);
      if (!pb.closed) return reinterpret_cast<const void*>(walk3_f32_kernel<kTorus, 1, false>);
      const int mq = (pb.n_v == 1 && pb.f.kind == kTorusFourier) ? pb.f.single_mq : -1;
      switch (mq) {
#define MPWOS_MQ(c) case c: return reinterpret_cast<const void*>(walk3_f32_kernel<kTorus, 1, true, c>);
#define MPWOS_MQ16(b) MPWOS_MQ(b + 0) MPWOS_MQ(b + 1) MPWOS_MQ(b + 2) MPWOS_MQ(b + 3) MPWOS_MQ(b + 4) \
  MPWOS_MQ(b + 5) MPWOS_MQ(b + 6) MPWOS_MQ(b + 7) MPWOS_MQ(b + 8) MPWOS_MQ(b + 9) MPWOS_MQ(b + 10)           \
  MPWOS_MQ(b + 11) MPWOS_MQ(b + 12) MPWOS_MQ(b + 13) MPWOS_MQ(b + 14) MPWOS_MQ(b + 15)
        MPWOS_MQ16(0) MPWOS_MQ16(16) MPWOS_MQ16(32) MPWOS_MQ16(48)
#undef MPWOS_MQ16
#undef MPWOS_MQ
        default: return reinterpret_cast<const void*>(walk3_f32_kernel<kTorus, 1, true>);
      }
    }
    case kPointCloud:   // k >= 12: the warp-cooperative neighbour search (same results, faster there)
      if (pb.cl_k >= 12)
        return pb.cl_k <= 16 ? reinterpret_cast<const void*>(walk3_f32_cloud_coop_kernel<16>)
                             : reinterpret_cast<const void*>(walk3_f32_cloud_coop_kernel<32>);
      return pb.cl_k <= 8 ? reinterpret_cast<const void*>(walk3_f32_cloud_kernel<kPointCloud, 8>)
                          : reinterpret_cast<const void*>(walk3_f32_cloud_kernel<kPointCloud, 16>);
    default: return nullptr;
  }
}

cudaError_t launch_walk3_f32(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  const void* fn = walk3_f32_fn(pb);
  if (!fn) return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

static const void* embed_tc_fn(int D) {
  switch (walkn_dq(D)) {
    case 8: return reinterpret_cast<const void*>(tc::embed_tc_kernel<8>);
    case 16: return reinterpret_cast<const void*>(tc::embed_tc_kernel<16>);
    case 24: return reinterpret_cast<const void*>(tc::embed_tc_kernel<24>);
    default: return reinterpret_cast<const void*>(tc::embed_tc_kernel<32>);
  }
}

size_t embed_tc_bimg_bytes() { return static_cast<size_t>(tc::kBBytes); }

cudaError_t launch_embed_tc(const DevProblem& pb, int grid, cudaStream_t st) {
  if (pb.mkind != kEmbeddedSphere || !pb.tc_bimg || !pb.dev_status || pb.n > 64 * tc::kMaxChunks || pb.d + 1 > 31)
    return cudaErrorInvalidValue;
  const void* fn = embed_tc_fn(pb.d + 1);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
  if (e != cudaSuccess) return e;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(tc::kThreads), args, tc::kSmemBytes, st);
}

cudaError_t launch_tc_project(const uint4* bimg, const float* G, int64_t rows, int n, float* out, float* gg,
                              unsigned* status, int grid, cudaStream_t st) {
  if (n < 1 || n > 64 * tc::kMaxChunks || grid < 1) return cudaErrorInvalidValue;
  const void* fn = reinterpret_cast<const void*>(tc::tc_project_kernel);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
  if (e != cudaSuccess) return e;
  void* args[] = {&bimg, &G, &rows, &n, &out, &gg, &status};
  return cudaLaunchKernel(fn, dim3(grid), dim3(tc::kThreads), args, tc::kSmemBytes, st);
}

static const void* walkr32_fn(const DevProblem& pb) {
  const int nt = walkr_nt(pb.red_nT);
#define MPWOS_WALKR(MK)                                                              \
  switch (nt) {                                                                      \
    case 4: return reinterpret_cast<const void*>(walkr_kernel<float, MK, 4>);        \
    case 8: return reinterpret_cast<const void*>(walkr_kernel<float, MK, 8>);        \
    case 16: return reinterpret_cast<const void*>(walkr_kernel<float, MK, 16>);      \
    case 24: return reinterpret_cast<const void*>(walkr_kernel<float, MK, 24>);      \
    default: return reinterpret_cast<const void*>(walkr_kernel<float, MK, 32>);      \
  }
  if (pb.mkind == kEuclid) { MPWOS_WALKR(kEuclid) }
  if (pb.mkind == kSphere) { MPWOS_WALKR(kSphere) }
  MPWOS_WALKR(kEmbeddedSphere)
#undef MPWOS_WALKR
}

cudaError_t launch_walkr_f32(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  if (pb.mkind != kEuclid && pb.mkind != kSphere && pb.mkind != kEmbeddedSphere) return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(walkr32_fn(pb), dim3(grid), dim3(block), args, 0, st);
}

bool walkr_lat_eligible(const DevProblem& pb) {
  return pb.reduced && pb.mkind == kEmbeddedSphere && pb.n_v == 1 && pb.red_nT <= 32;
}

cudaError_t launch_walkr_lat_f32(const DevProblem& pb, int grid, cudaStream_t st) {
  if (!walkr_lat_eligible(pb)) return cudaErrorInvalidValue;
  const void* fn;
  switch (walkr_nt(pb.red_nT)) {
    case 4: fn = reinterpret_cast<const void*>(walkr_lat_kernel<4>); break;
    case 8: fn = reinterpret_cast<const void*>(walkr_lat_kernel<8>); break;
    case 16: fn = reinterpret_cast<const void*>(walkr_lat_kernel<16>); break;
    case 24: fn = reinterpret_cast<const void*>(walkr_lat_kernel<24>); break;
    default: fn = reinterpret_cast<const void*>(walkr_lat_kernel<32>); break;
  }
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(128), args, 0, st);
}

int occupancy_walkr_f64(const DevProblem& pb, int block);

const void* walk_fn_f32(const DevProblem& pb) {
  if (pb.reduced)
    return (pb.mkind == kEuclid || pb.mkind == kSphere || pb.mkind == kEmbeddedSphere) ? walkr32_fn(pb) : nullptr;
  if (pb.n == 3 && pb.mkind != kEmbeddedSphere) return walk3_f32_fn(pb);
  return walkn32_fn(pb);
}

int occupancy_walkr(const DevProblem& pb, bool fp64, int block) {
  if (fp64) return occupancy_walkr_f64(pb, block);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walkr32_fn(pb), block, 0);
  return nb < 1 ? 1 : nb;
}

int occupancy_walk_f32(const DevProblem& pb, bool n3, int block) {
  if (!n3) return occupancy_walkn32(pb, block);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk3_f32_fn(pb), block, 0);
  return nb < 1 ? 1 : nb;
}

cudaError_t launch_cloud_knn_f32(const DevProblem& pb, const double* x, int64_t nq, int method, int64_t ncl,
                                 int32_t* idx, double* d2, double* h, int max_blocks, cudaStream_t st) {
  if (nq <= 0) return cudaSuccess;
  const int64_t need = (nq + 127) / 128;
  const unsigned grid = static_cast<unsigned>(need < max_blocks ? need : max_blocks);
  const bool small = pb.cl_k <= 8, mid = pb.cl_k <= 16;
  if (method == 0) {
    if (small) cloud_knn_query_kernel<float, 8, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
    else if (mid) cloud_knn_query_kernel<float, 16, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
    else cloud_knn_query_kernel<float, 32, false><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
  } else if (method == 1) {
    if (mid) cloud_knn_query_kernel<float, 16, true><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
    else cloud_knn_query_kernel<float, 32, true><<<grid, 128, 0, st>>>(pb, x, nq, idx, d2, h);
  } else if (method == 2) {
    const unsigned g = static_cast<unsigned>((nq + 128 * kScanQ - 1) / (128 * kScanQ));
    if (small) cloud_knn_scan_kernel<float, 8><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
    else if (mid) cloud_knn_scan_kernel<float, 16><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
    else cloud_knn_scan_kernel<float, 32><<<g, 128, 0, st>>>(pb, x, nq, ncl, idx, d2, h);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

__global__ void green_radius32_kernel(const double* a, const double* U, double* t, int64_t count,
                                      const float4* tabc, int NA, int NS, float tab_scale, float z_scale) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const float v = table_lookup32(tabc, NA, NS, tab_scale, z_scale, static_cast<float>(a[q]), static_cast<float>(U[q]));
  t[q] = static_cast<double>(fminf(fmaxf(v, 0.0f), 1.0f));
}

cudaError_t launch_green_radius32(const double* a, const double* U, double* t, int64_t count, const float4* tabc,
                                  int NA, int NS, double z_max, cudaStream_t st) {
  const float tab_scale = static_cast<float>((NS - 1) / 0.70710678118654752);
  const float z_scale = (NA > 1 && z_max > 0.0) ? static_cast<float>((NA - 1) / z_max) : 0.0f;
  green_radius32_kernel<<<static_cast<unsigned>((count + 127) / 128), 128, 0, st>>>(a, U, t, count, tabc, NA, NS,
                                                                                   tab_scale, z_scale);
  return cudaGetLastError();
}

}  // namespace mpwos
