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

// Paired FP32 arithmetic (two lanes of a 64-bit register, round to nearest):
// the candidate tests run two candidates per instruction.
__device__ __forceinline__ unsigned long long f32x2_pack(float lo, float hi) {
  unsigned long long d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f32x2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f32x2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f32x2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long f32x2_fma(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// Sorted index of position q of the group's flattened candidate stream:
// rows r = 0..nrows-1 hold [beg_r, beg_r + len_r), incl_r = len_0 + ... + len_r.
template <int NR>
__device__ __forceinline__ uint32_t flat_candidate(uint32_t q, const uint32_t (&beg)[NR],
                                                   const uint32_t (&incl)[NR]) {
  uint32_t idx = 0, lo = 0;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (q >= lo && q < incl[r]) idx = beg[r] + (q - lo);
    lo = incl[r];
  }
  return idx;
}

// Where candidates come from: cell lower bounds `lb` (ncells + 1 entries,
// the first position with key >= c) over an array of candidates in key
// order, their FP32 positions `xf` (.w = type) and, when `map` is not null,
// the sorted particle index of each position (candidates = a compacted
// subset such as the fluid particles); otherwise the position is the index.
struct CandSource {
  const uint32_t* lb;
  const float4* xf;
  const uint32_t* map;
};

// f(j, r2f, type_j) is called for every candidate j != self of the lane's
// particle with FP32 squared distance r2f <= pre_r2 (type_j from the .w
// component of the FP32 position copy). `stage` holds 32 float4 and `sidx`
// 32 indices of this warp; the positions are staged as four arrays of 32
// (x, y, z, type) so that pairs of candidates load as one 64-bit word. All
// 32 lanes must call this function together.
//
// Per group the 3^(d-1) row ranges are fetched by one lane each, scanned
// into one flattened candidate stream (rows in (z, y) order, each in key
// order), and the stream is staged 32 at a time with the next 32 loaded
// into registers while the current ones are tested: no partially filled
// batches at row ends, and the gather latency overlaps the tests.
template <int DIM, class F>
__device__ __forceinline__ void warp_scan_candidates_r(const Params& p, const CandSource& src, bool active,
                                                       uint32_t self, uint32_t key, float4 xs, float pre_r2,
                                                       float4* stage, uint32_t* sidx, F&& f) {
  constexpr int NR = DIM == 3 ? 9 : 3;
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
  const float4 far = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
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
    // lane r < NR: row r = (cz, cy) = (gz - 1 + r / 3, gy - 1 + r % 3) in 3D
    uint32_t rb = 0, rl = 0;
    if (lane < NR) {
      int cy = gy - 1 + lane % 3;
      int cz = DIM == 3 ? gz - 1 + lane / 3 : 0;
      if (cy >= 0 && cy < p.nc[1] && cz >= 0 && cz < p.nc[2]) {
        int64_t base = (int64_t)cy * p.nc[0] + (int64_t)cz * p.nc[0] * p.nc[1];
        rb = src.lb[base + x0];
        rl = src.lb[base + x1 + 1] - rb;
      }
    }
    uint32_t inc = rl;
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    uint32_t beg[NR], incl[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      beg[r] = __shfl_sync(0xffffffffu, rb, r);
      incl[r] = __shfl_sync(0xffffffffu, inc, r);
    }
    const uint32_t total = incl[NR - 1];
    uint32_t nidx = flat_candidate<NR>((uint32_t)lane, beg, incl);
    const bool has0 = (uint32_t)lane < total;
    float4 nxt = has0 ? __ldg(&src.xf[nidx]) : far;
    uint32_t nj = (src.map && has0) ? __ldg(&src.map[nidx]) : nidx;
    float* sx = reinterpret_cast<float*>(stage);  // [x 32][y 32][z 32][type 32]
    // a lane whose own position is not finite tests against -inf: every
    // candidate then fails, as it would fail an ordered comparison with NaN
    const bool fin = isfinite(xs.x) && isfinite(xs.y) && isfinite(xs.z);
    const float qx = fin ? xs.x : -INFINITY, qy = fin ? xs.y : -INFINITY, qz = fin ? xs.z : -INFINITY;
    const unsigned long long px = f32x2_pack(qx, qx), py = f32x2_pack(qy, qy), pz = f32x2_pack(qz, qz);
    const unsigned long long pre2 = f32x2_pack(pre_r2, pre_r2);
    for (uint32_t c0 = 0; c0 < total; c0 += 32) {
      // slots past the stream hold a point at infinity, which no test passes
      sx[lane] = nxt.x;
      sx[32 + lane] = nxt.y;
      sx[64 + lane] = nxt.z;
      sx[96 + lane] = nxt.w;
      sidx[lane] = nj;
      __syncwarp();
      const uint32_t q = c0 + 32 + (uint32_t)lane;
      if (c0 + 32 < total) {
        nidx = flat_candidate<NR>(q, beg, incl);
        const bool has = q < total;
        nxt = has ? __ldg(&src.xf[nidx]) : far;
        nj = (src.map && has) ? __ldg(&src.map[nidx]) : nidx;
      }
      if (in_g) {
        // independent tests of all 32 staged candidates, then the hits in
        // order. Four candidates per 16-byte broadcast load, two per paired
        // instruction; candidate k fails r2 <= pre_r2 exactly when the
        // difference pre_r2 - r2 is negative (it is never rounded to
        // zero), so its sign bit is shifted into bit k of the miss mask.
        unsigned miss = 0u;
        const ulonglong2* s4 = reinterpret_cast<const ulonglong2*>(sx);
#pragma unroll
        for (int g = 7; g >= 0; --g) {
          const ulonglong2 X = s4[g], Y = s4[8 + g], Z = s4[16 + g];
          unsigned long long d[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // h = 0: candidates 4g, 4g + 1; h = 1: 4g + 2, 4g + 3
            unsigned long long dx = f32x2_sub(h ? X.y : X.x, px);
            unsigned long long dy = f32x2_sub(h ? Y.y : Y.x, py);
            unsigned long long dz = f32x2_sub(h ? Z.y : Z.x, pz);
            unsigned long long r2 = f32x2_fma(dz, dz, f32x2_fma(dy, dy, f32x2_mul(dx, dx)));
            d[h] = f32x2_sub(pre2, r2);
          }
          miss = __funnelshift_l((unsigned)(d[1] >> 32), miss, 1);
          miss = __funnelshift_l((unsigned)d[1], miss, 1);
          miss = __funnelshift_l((unsigned)(d[0] >> 32), miss, 1);
          miss = __funnelshift_l((unsigned)d[0], miss, 1);
        }
        unsigned hits = ~miss;
        while (hits) {
          int k = __ffs(hits) - 1;
          hits &= hits - 1u;
          uint32_t j = sidx[k];
          if (j == self) continue;
          float dx = sx[k] - xs.x, dy = sx[32 + k] - xs.y, dz = sx[64 + k] - xs.z;
          f(j, fmaf(dz, dz, fmaf(dy, dy, dx * dx)), sx[96 + k]);
        }
      }
      __syncwarp();
    }
  }
}

// The scan with the candidate threshold of Algorithm 1's test (prefilter_r2).
template <int DIM, class F>
__device__ __forceinline__ void warp_scan_candidates(const Params& p, const CandSource& src, bool active,
                                                     uint32_t self, uint32_t key, float4 xs,
                                                     float4* stage, uint32_t* sidx, F&& f) {
  warp_scan_candidates_r<DIM>(p, src, active, self, key, xs, p.prefilter_r2, stage, sidx, static_cast<F&&>(f));
}

// Candidates = all particles in sorted order.
__device__ __forceinline__ CandSource all_particles(const Work& w) { return CandSource{w.cell_lb, w.xf, nullptr}; }

// Candidates = the fluid particles (compacted in sorted order).
__device__ __forceinline__ CandSource fluid_particles(const Work& w) {
  return CandSource{w.fcell_lb, w.xff, w.fluid_list};
}

}  // namespace wbsph
