// estimator.cuh — the per-point Monte Carlo estimator (eq. mc_estimator) and
// its standard error, in one fixed summation order shared by the device
// reduction and the host merge of walk ranges.
//
// The walks of a point are cut into blocks of kEstBlock walk indices (block b:
// walks kEstBlock b .. kEstBlock (b + 1) - 1).  Within a block, lane l
// (0..31) takes walks b kEstBlock + l + 32 t, t = 0..31, in t order, forming
// (count, mean, sum of squared deviations) by two passes (mean first); the 32
// lanes merge by a fixed tree (at offset 16, 8, 4, 2, 1 lane l < offset merges
// lane l + offset into itself); the blocks merge in block order.  Merges use
// the pairwise update of Chan, Golub and LeVeque (1979).  A block's statistic
// depends only on its own walks, so a request split into walk ranges that
// start at block boundaries (one range per GPU) merges to the same bits as the
// whole request (the device kernel and the host merge run the same IEEE
// operations: no FMA contraction in either).
#pragma once
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace mpwos {

constexpr int64_t kEstBlock = 1024;   // walks per estimator block
constexpr int kEstFields = 5;         // block record: count, mean, M2, sum of K, flagged walks

struct Stat {
  double n, m, M;   // count, mean, sum of squared deviations from the mean
};

__host__ __device__ inline Stat stat_merge(Stat a, Stat b) {
  if (b.n == 0.0) return a;
  if (a.n == 0.0) return b;
  const double n = a.n + b.n;
  const double d = b.m - a.m;
  Stat r;
  r.n = n;
  r.m = a.m + d * (b.n / n);
  r.M = (a.M + b.M) + (d * d) * ((a.n * b.n) / n);
  return r;
}

// One lane's walks of a block: values x[t * 32] for t < cnt, two passes.
__host__ __device__ inline Stat stat_lane(const double* x, int cnt) {
  if (cnt <= 0) return Stat{0.0, 0.0, 0.0};
  double s = 0.0;
  for (int t = 0; t < cnt; ++t) s += x[static_cast<int64_t>(t) * 32];
  const double m = s / static_cast<double>(cnt);
  double M = 0.0;
  for (int t = 0; t < cnt; ++t) {
    const double d = x[static_cast<int64_t>(t) * 32] - m;
    M += d * d;
  }
  return Stat{static_cast<double>(cnt), m, M};
}

// Walks of lane l in a block of nb walks (nb <= kEstBlock).
__host__ __device__ inline int lane_count(int64_t nb, int l) {
  return nb > l ? static_cast<int>((nb - l + 31) / 32) : 0;
}

// mean, standard error sqrt(s^2 / n) with s^2 = M / (n - 1).
__host__ __device__ inline void stat_finish(Stat s, double& mean, double& se) {
  mean = s.m;
  const double var = (s.n > 1.0) ? s.M / (s.n - 1.0) : 0.0;
  se = (s.n > 0.0) ? sqrt(var / s.n) : 0.0;
}

}  // namespace mpwos
