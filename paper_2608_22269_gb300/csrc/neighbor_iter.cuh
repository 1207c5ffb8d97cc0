// neighbor_iter.cuh -- the exact FP64 neighbour test d <= 2h of Algorithm 1
// (candidates are enumerated by warp_scan_candidates in warp_scan.cuh).
#pragma once
#include "common.cuh"

namespace wbsph {

// Exact neighbour criterion: r^2 = (dx*dx + dy*dy) + dz*dz, left to right,
// every operation IEEE round-to-nearest without contraction, against
// (2h)*(2h); j != i and r > 0.
__device__ __forceinline__ bool exact_neighbor(const Params& p, const double* __restrict__ x, int64_t n,
                                               uint32_t i, uint32_t j) {
  double d0 = __dsub_rn(x[j], x[i]);
  double r2 = __dmul_rn(d0, d0);
  double d1 = __dsub_rn(x[n + j], x[n + i]);
  r2 = __dadd_rn(r2, __dmul_rn(d1, d1));
  if (p.dim == 3) {
    double d2 = __dsub_rn(x[2 * n + j], x[2 * n + i]);
    r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
  }
  return r2 <= p.four_h2 && r2 > 0.0;
}

}  // namespace wbsph
