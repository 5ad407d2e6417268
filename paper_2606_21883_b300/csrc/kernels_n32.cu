// kernels_n32.cu — the FP32 warp walk in R^n (walkn32.cuh): kernel instances
// by manifold kind and slots per lane, launcher and occupancy.  Compiled with
// fast single-precision math (MUFU transcendentals, contraction).
#include "launch.h"
#include "walkn32.cuh"
#include "walkn32s.cuh"

namespace mpwos {

template <int MK>
static const void* by_mg(int mg) {
  using w32s::kLPW;
  switch (mg) {
    case 1: return reinterpret_cast<const void*>(w32s::walkn32s_kernel<MK, kLPW, 1>);
    case 2: return reinterpret_cast<const void*>(w32s::walkn32s_kernel<MK, kLPW, 2>);
    default: return reinterpret_cast<const void*>(w32s::walkn32s_kernel<MK, kLPW, 4>);
  }
}

// R^n, the sphere and the hypersurface of revolution run the shared-memory walk
// (walkn32s.cuh, kLPW lanes per walker); the others the register walk (a warp).
static bool shared_walk(const DevProblem& pb) {
  return pb.mkind == kEuclid || pb.mkind == kSphere || pb.mkind == kRevolution;
}

int walkn32_lanes_per_walker(const DevProblem& pb) { return shared_walk(pb) ? w32s::kLPW : 32; }

int walkn32_max_block(const DevProblem& pb) { return shared_walk(pb) ? w32s::kThreads : w32::kThreads; }

template <int MK>
static const void* by_mb(int mb) {
  switch (mb) {
    case 1: return reinterpret_cast<const void*>(w32::walkn32_kernel<MK, 1, 8>);
    case 2: return reinterpret_cast<const void*>(w32::walkn32_kernel<MK, 2, 8>);
    case 4: return reinterpret_cast<const void*>(w32::walkn32_kernel<MK, 4, 8>);
    default: return reinterpret_cast<const void*>(w32::walkn32_kernel<MK, 8, 8>);
  }
}

const void* walkn32_fn(const DevProblem& pb) {
  if (pb.n <= 3 || pb.n > 1024) return nullptr;
  const int mg = w32s::walkn32s_mg(pb.n);
  switch (pb.mkind) {
    case kEuclid: return by_mg<kEuclid>(mg);
    case kSphere: return by_mg<kSphere>(mg);
    case kRevolution: return by_mg<kRevolution>(mg);
    case kCurveSphere: return pb.n == 9 ? reinterpret_cast<const void*>(w32::walkn32_kernel<kCurveSphere, 1, 8>) : nullptr;
    case kEmbeddedSphere:
      switch (walkn_dq(pb.d + 1)) {
        case 8: return reinterpret_cast<const void*>(w32::walkn32_kernel<kEmbeddedSphere, 8, 8>);
        case 16: return reinterpret_cast<const void*>(w32::walkn32_kernel<kEmbeddedSphere, 8, 16>);
        case 24: return reinterpret_cast<const void*>(w32::walkn32_kernel<kEmbeddedSphere, 8, 24>);
        default: return reinterpret_cast<const void*>(w32::walkn32_kernel<kEmbeddedSphere, 8, 32>);
      }
    default: return nullptr;
  }
}

cudaError_t launch_walkn_f32(const DevProblem& pb, int grid, int block, cudaStream_t st) {
  const void* fn = walkn32_fn(pb);
  if (!fn || block > walkn32_max_block(pb) || block % 32 != 0) return cudaErrorInvalidValue;
  if (pb.mkind == kRevolution && (!pb.rv_v32 || !pb.rv_a32)) return cudaErrorInvalidValue;
  if (pb.mkind == kEmbeddedSphere && (!pb.Qf || !pb.s0)) return cudaErrorInvalidValue;
  DevProblem arg = pb;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, st);
}

int occupancy_walkn32(const DevProblem& pb, int block) {
  int nb = 0;
  const void* fn = walkn32_fn(pb);
  if (fn) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0);
  return nb < 1 ? 1 : nb;
}

}  // namespace mpwos
