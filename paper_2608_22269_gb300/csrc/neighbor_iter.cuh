// neighbor_iter.cuh -- enumeration of neighbour candidates of one particle
// over the 3^d cells around its own (Algorithm 1), with the exact FP64
// distance test d <= 2h.
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

// Iterates over the sorted indices of all particles j != i whose FP32
// distance passes the conservative prefilter r_f^2 <= prefilter_r2 (a bound
// chosen on the host so that every exact neighbour passes). For each (z, y)
// row of the 3^d neighbourhood the three x-adjacent cells are contiguous in
// key order, so a row is one sorted index range [lb[a], lb[b + 1]).
struct CandidateIter {
  int ix, iy, iz, row;
  uint32_t cur, end, self;
  float xi, yi, zi;

  __device__ __forceinline__ void init(const Params& p, const Work& w, int64_t, uint32_t i) {
    uint32_t key = w.key[i];
    uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
    ix = (int)(key % nx);
    iy = (int)((key / nx) % ny);
    iz = (int)(key / (nx * ny));
    float4 f = w.xf[i];
    xi = f.x; yi = f.y; zi = f.z;
    self = i;
    row = -1;
    cur = end = 0;
    advance_row(p, w);
  }

  __device__ __forceinline__ bool advance_row(const Params& p, const Work& w) {
    const int nrows = p.dim == 3 ? 9 : 3;
    while (++row < nrows) {
      int oy = row % 3 - 1;
      int oz = p.dim == 3 ? row / 3 - 1 : 0;
      int cy = iy + oy, cz = iz + oz;
      if (cy < 0 || cy >= p.nc[1] || cz < 0 || cz >= p.nc[2]) continue;
      int x0 = ix > 0 ? ix - 1 : 0;
      int x1 = ix + 1 < p.nc[0] ? ix + 1 : p.nc[0] - 1;
      int64_t base = (int64_t)cy * p.nc[0] + (int64_t)cz * p.nc[0] * p.nc[1];
      cur = w.cell_lb[base + x0];
      end = w.cell_lb[base + x1 + 1];
      if (cur < end) return true;
    }
    cur = end = 0;
    return false;
  }

  // Next candidate j and its FP32 squared distance r2f.
  __device__ __forceinline__ bool next(const Params& p, const Work& w, uint32_t& j, float& r2f) {
    for (;;) {
      while (cur < end) {
        uint32_t c = cur++;
        if (c == self) continue;
        float4 f = __ldg(&w.xf[c]);
        float dx = f.x - xi, dy = f.y - yi, dz = f.z - zi;
        float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 <= p.prefilter_r2) {
          j = c;
          r2f = r2;
          return true;
        }
      }
      if (!advance_row(p, w)) return false;
    }
  }

  __device__ __forceinline__ bool next(const Params& p, const Work& w, uint32_t& j) {
    float r2f;
    return next(p, w, j, r2f);
  }
};

}  // namespace wbsph
