// lists.cu -- per-stage neighbour lists of the fluid particles (Algorithm 1),
// built from the warp-cooperative candidate scan of warp_scan.cuh.
#include "common.cuh"
#include "neighbor_iter.cuh"
#include "warp_scan.cuh"

namespace wbsph {
// ---------------------------------------------------------------------------
// Neighbour lists: for fluid particle gi (sorted index fluid_list[gi]), in
// Algorithm 1 order, stored k-major: nbr[k * nf + gi].
//  EXACT (FP64 path, surrogate graph): every j != i with exact r <= 2h
//    (Algorithm 1's test). The FP32 distance of the warp scan decides for
//    candidates inside the inner bound; the rest of the candidates that pass
//    the conservative prefilter (a thin band near 2h) take the exact FP64 test.
//  otherwise (mixed path): every candidate that passes the FP32 prefilter;
//    the mixed pair pass applies its own FP32 test. With `skin` the
//    prefilter radius is 2h + delta (device scalar of the time step), and
//    the same lists serve both stages of the step.
// Lists are staged per warp in shared memory so the global stores are
// coalesced rows.
// ---------------------------------------------------------------------------
constexpr int LIST_THREADS = 64;

template <int DIM, bool EXACT>
__global__ void __launch_bounds__(LIST_THREADS) k_nbr_list(Params p, State s, Work w, int64_t n, int64_t nf,
                                                         int kmax, int ks, int skin) {
  extern __shared__ float4 smem_f4[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4* stage = smem_f4 + warp * 32;
  uint32_t* sidx = reinterpret_cast<uint32_t*>(smem_f4 + (LIST_THREADS / 32) * 32) + warp * 32;
  uint32_t* my = reinterpret_cast<uint32_t*>(smem_f4 + (LIST_THREADS / 32) * 32) + LIST_THREADS +
                 warp * ks * 32;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;
  const uint32_t key = active ? w.key[i] : 0u;
  const float4 xs = active ? w.xf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  int cnt = 0, nband = 0;
  constexpr uint32_t kBand = 0x80000000u;  // entry still needs the exact test
  // kept lists (mixed path, stage 1): every candidate within 2h + delta
  const float pre_r2 = (!EXACT && skin) ? __double2float_ru(w.scalars[3]) : p.prefilter_r2;
  warp_scan_candidates_r<DIM>(p, all_particles(w), active, i, key, xs, pre_r2, stage, sidx, [&](uint32_t j, float r2f, float) {
    // neighbour test of Algorithm 1: FP32 decides inside the inner bound;
    // candidates in the rounding band near 2h (and at r_f = 0) are flagged
    // for the exact FP64 test below
    const bool band = EXACT && !(r2f > 0.f && r2f <= p.inner_r2);
    nband += band ? 1 : 0;
    const uint32_t v = j | (band ? kBand : 0u);
    // the first ks entries are staged; the rare ones beyond go straight out
    if (cnt < ks) my[cnt * 32 + lane] = v;
    else if (cnt < kmax) w.nbr[(int64_t)cnt * nf + gi] = v;
    ++cnt;
  });
  if (EXACT && nband > 0) {  // rare: exact test of the flagged entries, compacting in order
    const int m = cnt < kmax ? cnt : kmax;
    int kept = 0;
    for (int k = 0; k < m; ++k) {
      uint32_t v = k < ks ? my[k * 32 + lane] : w.nbr[(int64_t)k * nf + gi];
      if (v & kBand) {
        v &= ~kBand;
        if (!exact_neighbor(p, s.x, n, i, v)) continue;
      }
      if (kept < ks) my[kept * 32 + lane] = v;
      else w.nbr[(int64_t)kept * nf + gi] = v;
      ++kept;
    }
    if (cnt > kmax) atomicOr(w.status, kStatOverflow);
    cnt = kept;
  }
  if (active) {
    if (cnt > kmax) {
      atomicOr(w.status, kStatOverflow);
      cnt = kmax;
    }
    w.nbr_cnt[gi] = (uint32_t)cnt;
  }
  __syncwarp();
  const int staged = cnt < ks ? cnt : ks;
  int maxc = __reduce_max_sync(0xffffffffu, staged);
  for (int k = 0; k < maxc; ++k)
    if (k < staged) w.nbr[(int64_t)k * nf + gi] = my[k * 32 + lane];
}


int pair_list_kmax(int dim) { return dim == 3 ? 128 : 48; }

// List entries per lane staged in shared memory (the rest are stored
// directly, uncoalesced). A 3D list holds about 75 exact neighbours (h =
// 1.3 dx) or 90 kept candidates; staging 48 of them leaves room for about
// 34 resident warps per SM, and this latency-bound kernel gains more from
// those warps than it loses on the uncoalesced stores of the entries beyond
// (against 80 staged entries and 18 warps: mixed step 2.96 -> 2.86 ms, FP64
// step 23.66 -> 23.54 ms on the 1.21M-particle dam break).
#ifndef WBSPH_LIST_STAGE_3D
#define WBSPH_LIST_STAGE_3D 48
#endif
static int pair_list_stage(int dim) { return dim == 3 ? WBSPH_LIST_STAGE_3D : 48; }

void launch_nbr_list(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, cudaStream_t st,
                     bool exact, bool skin) {
  if (nf == 0) return;
  int kmax = pair_list_kmax(p.dim);
  int ks = pair_list_stage(p.dim);
  if (ks > kmax) ks = kmax;
  size_t sm = (size_t)ks * 32 * (LIST_THREADS / 32) * sizeof(uint32_t) +
              (LIST_THREADS / 32) * 32 * (sizeof(float4) + sizeof(uint32_t));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_nbr_list<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_nbr_list<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_nbr_list<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_nbr_list<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    attr = true;
  }
  unsigned blocks = (unsigned)div_up(nf, LIST_THREADS);
  if (p.dim == 3) {
    if (exact) k_nbr_list<3, true><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks, 0);
    else k_nbr_list<3, false><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks, skin ? 1 : 0);
  } else {
    if (exact) k_nbr_list<2, true><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks, 0);
    else k_nbr_list<2, false><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks, skin ? 1 : 0);
  }
}

}  // namespace wbsph
