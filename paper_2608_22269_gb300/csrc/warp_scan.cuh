// warp_scan.cuh -- warp-cooperative enumeration of neighbour candidates with
// shared-memory staging of candidate positions (the cell-tile staging of the
// neighbour loop of Algorithm 1).
//
// The 32 lanes of a warp hold particles that are consecutive in cell-key
// order, so they sit in one or a few x-runs of cells. Lanes are grouped by
// (y, z) cell row and contiguous x cells; for each group the union of the
// lanes' 3^d neighbourhoods is 3^(d-1) rows times one x-run [min ix - 1, max ix + 1],
// each a contiguous sorted index range. The warp stages 32 candidate
// positions at a time into shared memory and every lane of the group tests
// all of them (uniform loop, broadcast reads), instead of each lane walking
// its own cells with divergent loops. Candidates come out per lane in
// Algorithm 1 order (z row, y row, then sorted index); extra x-cells of the
// union contribute only particles beyond 2h, which the distance test drops.
#pragma once
#include <climits>

#include "common.cuh"

namespace wbsph {

struct LaneCell {
  int ix, iy, iz;
  int row;  // iy + iz * ny: lanes of one group share it
};

__device__ __forceinline__ LaneCell lane_cell(const Params& p, uint32_t key) {
  uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
  LaneCell c;
  c.ix = (int)(key % nx);
  c.row = (int)(key / nx);
  c.iy = c.row % (int)ny;
  c.iz = c.row / (int)ny;
  return c;
}

// f(j, r2f, type_j) is called for every candidate j != self of the lane's
// particle with FP32 squared distance r2f <= prefilter_r2 (type_j from the .w
// component of the FP32 position copy). `stage` holds 32 float4 of
// this warp. All 32 lanes must call this function together.
template <class F>
__device__ __forceinline__ void warp_scan_candidates(const Params& p, const Work& w, bool active,
                                                     uint32_t self, uint32_t key, float4 xs,
                                                     float4* stage, F&& f) {
  const int lane = threadIdx.x & 31;
  LaneCell c = lane_cell(p, active ? key : 0u);
  // groups: consecutive active lanes of one cell row whose x cells are no
  // more than 2 apart (a row of wall particles can hold both ends of a row)
  int prev_row = __shfl_up_sync(0xffffffffu, c.row, 1);
  int prev_ix = __shfl_up_sync(0xffffffffu, c.ix, 1);
  bool prev_active = __shfl_up_sync(0xffffffffu, (int)active, 1) != 0;
  bool starts = active && (lane == 0 || !prev_active || prev_row != c.row || c.ix > prev_ix + 2);
  unsigned starts_mask = __ballot_sync(0xffffffffu, starts);
  int gid = __popc(starts_mask & ((2u << lane) - 1u));  // group number (1-based) of this lane
  unsigned pending = __ballot_sync(0xffffffffu, active);
  while (pending) {
    int leader = __ffs(pending) - 1;
    int ggid = __shfl_sync(0xffffffffu, gid, leader);
    int grow = __shfl_sync(0xffffffffu, c.row, leader);
    bool in_g = active && gid == ggid;
    unsigned gmask = __ballot_sync(0xffffffffu, in_g);
    pending &= ~gmask;
    int xlo = __reduce_min_sync(0xffffffffu, in_g ? c.ix : INT_MAX);
    int xhi = __reduce_max_sync(0xffffffffu, in_g ? c.ix : -1);
    int gy = grow % p.nc[1], gz = grow / p.nc[1];
    int x0 = xlo > 0 ? xlo - 1 : 0;
    int x1 = xhi + 1 < p.nc[0] ? xhi + 1 : p.nc[0] - 1;
    int z0 = p.dim == 3 ? gz - 1 : 0, z1 = p.dim == 3 ? gz + 1 : 0;
    for (int cz = z0; cz <= z1; ++cz) {
      if (cz < 0 || cz >= p.nc[2]) continue;
      for (int cy = gy - 1; cy <= gy + 1; ++cy) {
        if (cy < 0 || cy >= p.nc[1]) continue;
        int64_t base = (int64_t)cy * p.nc[0] + (int64_t)cz * p.nc[0] * p.nc[1];
        uint32_t beg = w.cell_lb[base + x0], end = w.cell_lb[base + x1 + 1];
        for (uint32_t c0 = beg; c0 < end; c0 += 32) {
          uint32_t idx = c0 + lane;
          // slots past the run hold a point at infinity, which no test passes
          stage[lane] = idx < end ? __ldg(&w.xf[idx]) : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
          __syncwarp();
          if (in_g) {
            // independent tests of all 32 staged candidates, then the hits in order
            unsigned hits = 0u;
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
              float4 q = stage[k];
              float dx = q.x - xs.x, dy = q.y - xs.y, dz = q.z - xs.z;
              float r2 = dx * dx + dy * dy + dz * dz;
              hits |= (r2 <= p.prefilter_r2 ? 1u : 0u) << k;
            }
            if (self - c0 < 32u) hits &= ~(1u << (self - c0));
            while (hits) {
              int k = __ffs(hits) - 1;
              hits &= hits - 1u;
              float4 q = stage[k];
              float dx = q.x - xs.x, dy = q.y - xs.y, dz = q.z - xs.z;
              f(c0 + k, dx * dx + dy * dy + dz * dz, q.w);
            }
          }
          __syncwarp();
        }
      }
    }
  }
}

}  // namespace wbsph
