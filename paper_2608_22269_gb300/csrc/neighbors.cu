// neighbors.cu -- cell-linked-list neighbour build (Sec. 3, Eqs. hashid and
// ixyz, Algorithm 1): cell key per particle, stable LSD radix sort of
// (key, particle index), gather of all particle data into key order, and a
// lower-bound table giving the sorted index range of any run of cells.
#include "common.cuh"
#include "neighbor_iter.cuh"
#include "warp_scan.cuh"

namespace wbsph {

// ---------------------------------------------------------------------------
// Cell key (Eqs. hashid, ixyz): i_k = floor((x_k - x_min,k) / R), R = 2h;
// key = i_x + i_y N_x + i_z N_x N_y, with the subtraction and the division
// IEEE round-to-nearest in FP64 as the CPU definition has them. Almost every
// particle gets floor of an FP32 estimate of the quotient: its error bound
// (derived with the margin on the host) keeps the FP64 quotient on the same
// side of every integer when the estimate's fractional part is more than
// the margin from 0 and 1; the rest take the FP64 subtraction and division.
// Either way the key equals the definition bit for bit.
// ---------------------------------------------------------------------------
// FP32 value of a double with its mantissa truncated (relative error below
// 2^-23), on the IEEE fields with integer instructions; magnitudes below
// 2^-126 give zero. The input is finite.
__device__ __forceinline__ float key_d2f_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e <= 1023u - 127u) return 0.f;
  return __uint_as_float((hi & 0x80000000u) | ((e - (1023u - 127u)) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

__global__ void k_cell_keys(Params p, const double* __restrict__ x, int64_t n,
                            uint32_t* __restrict__ key, unsigned* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t ic[3] = {0, 0, 0};
  bool bad = false;
  for (int k = 0; k < p.dim; ++k) {
    double xk = x[k * n + i];
    // min <= x <= max, compared on order-preserving integer images (-0 as
    // +0; NaN falls outside), which keeps the FP64 pipe free
    long long b = __double_as_longlong(xk);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    b = b < 0 ? b ^ 0x7FFFFFFFFFFFFFFFLL : b;
    if (!(b >= p.key_lo[k] && b <= p.key_hi[k])) {
      bad = true;
      continue;
    }
    const float qf = (key_d2f_trunc(xk) - p.key_min_f[k]) * p.key_inv_R_f;
    const float fl = floorf(qf), fr = qf - fl;
    if (fr > p.key_margin[k] && fr < 1.f - p.key_margin[k])
      ic[k] = (int64_t)fl;
    else
      ic[k] = (int64_t)floor(__ddiv_rn(__dsub_rn(xk, p.domain_min[k]), p.R));
    if (ic[k] >= p.nc[k]) ic[k] = p.nc[k] - 1;  // unreachable for in-domain x; guards indexing
  }
  if (bad) {
    atomicOr(status, kStatDomain);
    key[i] = 0;
    return;
  }
  key[i] = (uint32_t)(ic[0] + ic[1] * (int64_t)p.nc[0] + ic[2] * (int64_t)p.nc[0] * p.nc[1]);
}

void launch_cell_keys(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  k_cell_keys<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p, s.x, n, w.key, w.status);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of 32-bit keys with 32-bit values, 8-bit digits.
// Per pass: tile histograms (digit-major table: row d holds digit d's count
// in every tile), an exclusive scan of every row by its own block plus the
// row totals, then a scatter that adds the exclusive scan of the 256 row
// totals (done in shared memory by every scatter block) and ranks equal
// digits inside a tile in index order (warp match + per-warp counts), which
// keeps the sort stable.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int SCAN_THREADS = 1024;

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                          int shift, uint32_t mask,
                                                          uint32_t* __restrict__ hist, int64_t nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = blockIdx.x * (int64_t)RS_TILE;
#pragma unroll 4
  for (int r = 0; r < RS_ITEMS; ++r) {
    int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` 32-bit counts in place, one block.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_exclusive(uint32_t* data, int64_t total) {
  __shared__ uint32_t part[SCAN_THREADS];
  int t = threadIdx.x;
  int64_t chunk = div_up(total, SCAN_THREADS);
  int64_t beg = t * chunk, end = beg + chunk < total ? beg + chunk : total;
  uint32_t s = 0;
  for (int64_t i = beg; i < end; ++i) s += data[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = part[t] - s;  // exclusive prefix of this chunk
  for (int64_t i = beg; i < end; ++i) {
    uint32_t v = data[i];
    data[i] = run;
    run += v;
  }
}

// Exclusive scan of each digit row of the histogram table in place (block
// d scans row d, RS_THREADS entries per round, coalesced); totals[d] gets the
// row's sum. Rows of digits above `mask` are all zero and are skipped.
__global__ void __launch_bounds__(RS_THREADS) k_radix_scan_rows(uint32_t* __restrict__ hist, int64_t nblocks,
                                                               uint32_t* __restrict__ totals) {
  __shared__ uint32_t wsum[RS_WARPS];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint32_t* row = hist + (int64_t)blockIdx.x * nblocks;
  uint32_t carry = 0;
  for (int64_t c0 = 0; c0 < nblocks; c0 += RS_THREADS) {
    int64_t i = c0 + t;
    uint32_t v = i < nblocks ? row[i] : 0u;
    uint32_t inc = v;  // inclusive warp scan
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, all = 0;
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) {
      uint32_t x = wsum[k];
      wpre += k < warp ? x : 0u;
      all += x;
    }
    if (i < nblocks) row[i] = carry + wpre + inc - v;
    carry += all;
    __syncthreads();
  }
  if (t == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n, int shift,
    uint32_t mask, const uint32_t* __restrict__ hist, int64_t nblocks,
    const uint32_t* __restrict__ totals) {
  __shared__ uint32_t offs[256];
  __shared__ uint32_t wcnt[RS_WARPS][256];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  {
    // digit base = exclusive scan of the row totals (digits above mask: 0)
    uint32_t v = t <= (int)mask ? totals[t] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += o;
    }
    if (lane == 31) wcnt[0][warp] = inc;
    __syncthreads();
    uint32_t wpre = 0;
    for (int k = 0; k < warp; ++k) wpre += wcnt[0][k];
    offs[t] = wpre + inc - v + (t <= (int)mask ? hist[(int64_t)t * nblocks + blockIdx.x] : 0u);
    __syncthreads();
  }
  int64_t base = blockIdx.x * (int64_t)RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) wcnt[w][t] = 0;
    __syncthreads();
    int64_t i = base + r * RS_THREADS + t;
    bool valid = i < n;
    uint32_t key = valid ? keys_in[i] : 0u;
    uint32_t digit = valid ? ((key >> shift) & mask) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    uint32_t rank = __popc(peers & lt_mask);
    if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pos = offs[digit] + rank;
      for (int w = 0; w < warp; ++w) pos += wcnt[w][digit];
      keys_out[pos] = key;
      vals_out[pos] = vals_in ? vals_in[i] : (uint32_t)i;
    }
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) add += wcnt[w][t];
    offs[t] += add;
    __syncthreads();
  }
}

void launch_scan_exclusive(uint32_t* data, int64_t total, cudaStream_t st) {
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(data, total);
}

// ---------------------------------------------------------------------------
// Exclusive scan of a long array by chunks of SCAN_CHUNK: chunk sums, one
// scan of the sums, then each chunk scanned in place from its offset.
// ---------------------------------------------------------------------------
constexpr int SCAN_PER = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_PER;

// inclusive scan of one value per thread over the block; *total = block sum
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += o;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < SCAN_THREADS / 32 ? wsum[lane] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, w, off);
      if (lane >= off) w += o;
    }
    wsum[lane] = w;  // inclusive warp-total prefix
  }
  __syncthreads();
  if (total) *total = wsum[SCAN_THREADS / 32 - 1];
  return v + (warp > 0 ? wsum[warp - 1] : 0u);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_chunk_sums(const uint32_t* __restrict__ data, int64_t total,
                                                            uint32_t* __restrict__ sums) {
  __shared__ uint32_t wsum[32];
  const int64_t b0 = blockIdx.x * (int64_t)SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER;
  uint32_t v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) v += b0 + k < total ? data[b0 + k] : 0u;
  uint32_t tot;
  block_inclusive_scan(v, wsum, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_chunk_scan(uint32_t* __restrict__ data, int64_t total,
                                                            const uint32_t* __restrict__ offs) {
  __shared__ uint32_t wsum[32];
  const int64_t b0 = blockIdx.x * (int64_t)SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_PER;
  uint32_t x[SCAN_PER], v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    x[k] = b0 + k < total ? data[b0 + k] : 0u;
    v += x[k];
  }
  uint32_t run = block_inclusive_scan(v, wsum, nullptr) - v + offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_PER; ++k) {
    if (b0 + k < total) data[b0 + k] = run;
    run += x[k];
  }
}

int scan_scratch_words(int64_t total) { return (int)div_up(total > 0 ? total : 1, SCAN_CHUNK); }

// In-place exclusive scan of `total` counts; scratch holds scan_scratch_words(total) words.
void launch_scan_exclusive_chunked(uint32_t* data, int64_t total, uint32_t* scratch, cudaStream_t st) {
  if (total <= 0) return;
  const int64_t nb = div_up(total, SCAN_CHUNK);
  k_chunk_sums<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, total, scratch);
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(scratch, nb);
  k_chunk_scan<<<(unsigned)nb, SCAN_THREADS, 0, st>>>(data, total, scratch);
}

// histogram table (256 rows x tiles) followed by the 256 row totals
int radix_sort_scratch_words(int64_t n) { return (int)(256 * div_up(n > 0 ? n : 1, RS_TILE) + 256); }

static int bits_for(int64_t ncells) {
  int b = 1;
  while (b < 32 && (int64_t(1) << b) < ncells) ++b;
  return b;
}

void launch_radix_sort(const Params& p, Work& w, int64_t n, cudaStream_t st, int* launches) {
  if (n == 0) return;
  int64_t nblocks = div_up(n, RS_TILE);
  int bits = bits_for(p.ncells);
  const uint32_t* vin = nullptr;
  for (int shift = 0; shift < bits; shift += 8) {
    int b = bits - shift < 8 ? bits - shift : 8;
    uint32_t mask = (1u << b) - 1u;
    uint32_t* totals = w.hist + 256 * nblocks;
    k_radix_hist<<<(unsigned)nblocks, RS_THREADS, 0, st>>>(w.key, n, shift, mask, w.hist, nblocks);
    k_radix_scan_rows<<<mask + 1u, RS_THREADS, 0, st>>>(w.hist, nblocks, totals);
    k_radix_scatter<<<(unsigned)nblocks, RS_THREADS, 0, st>>>(w.key, vin, w.key_alt, w.perm_alt, n,
                                                             shift, mask, w.hist, nblocks, totals);
    *launches += 3;
    uint32_t* tk = w.key; w.key = w.key_alt; w.key_alt = tk;
    uint32_t* tp = w.perm; w.perm = w.perm_alt; w.perm_alt = tp;
    vin = w.perm;
  }
}

// ---------------------------------------------------------------------------
// Reorder (Sec. 3: particles of one cell stored contiguously): gather every
// per-particle array by the sort permutation; also writes the FP32 position
// copy used by the candidate prefilter (.w = particle type).
// ---------------------------------------------------------------------------
__global__ void k_gather(int dim, State src, State dst, const uint32_t* __restrict__ perm, int64_t n,
                         int with_base, float4* __restrict__ xf) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t j = perm[i];
  const uint8_t ty = src.type[j];
  float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < dim; ++k) {
    double xv = src.x[k * n + j];
    dst.x[k * n + i] = xv;
    dst.u[k * n + i] = src.u[k * n + j];
    // wall normals are read for dummy particles only (the dummy update);
    // fluid entries of the normal array are left as they are
    if (ty != kFluid) dst.normal[k * n + i] = src.normal[k * n + j];
    if (with_base) {
      dst.x0[k * n + i] = src.x0[k * n + j];
      dst.u0[k * n + i] = src.u0[k * n + j];
    }
    float fv = (float)xv;
    if (k == 0) f.x = fv; else if (k == 1) f.y = fv; else f.z = fv;
  }
  dst.phi[i] = src.phi[j];
  if (with_base) dst.phi0[i] = src.phi0[j];
  dst.mass[i] = src.mass[j];
  dst.type[i] = ty;
  f.w = (float)ty;
  dst.oid[i] = src.oid[j];
  xf[i] = f;
}

void launch_gather(const Params& p, const State& src, const State& dst, const Work& w, int64_t n,
                   bool with_base, cudaStream_t st) {
  if (n == 0) return;
  k_gather<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p.dim, src, dst, w.perm, n, with_base ? 1 : 0,
                                                     w.xf);
}

// lb[c] = number of sorted keys < c, for c in [0, ncells]: the particles of
// cells [a, b] occupy sorted positions [lb[a], lb[b + 1]).
__global__ void k_cell_lower_bounds(const uint32_t* __restrict__ key, int64_t n, int64_t ncells,
                                    uint32_t* __restrict__ lb) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c > ncells) return;
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)key[mid] < c) lo = mid + 1; else hi = mid;
  }
  lb[c] = (uint32_t)lo;
}

void launch_cell_bounds(const Params& p, const Work& w, int64_t n, cudaStream_t st) {
  k_cell_lower_bounds<<<(unsigned)div_up(p.ncells + 1, 256), 256, 0, st>>>(w.key, n, p.ncells,
                                                                           w.cell_lb);
}

// ---------------------------------------------------------------------------
// Ordered compaction of the sorted indices of fluid particles (the pair
// pass runs over fluid particles only).
// ---------------------------------------------------------------------------
constexpr int CMP_THREADS = 1024;
constexpr uint8_t kAnyWall = 255;  // `want` of the compaction: every non-fluid particle

__global__ void __launch_bounds__(CMP_THREADS) k_count_type(const uint8_t* __restrict__ type, int64_t n,
                                                           uint8_t want, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t wsum[CMP_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)CMP_THREADS + threadIdx.x;
  bool f = i < n && (want == kAnyWall ? type[i] != kFluid : type[i] == want);
  unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < CMP_THREADS / 32; ++k) s += wsum[k];
    cnt[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(CMP_THREADS) k_write_type(const uint8_t* __restrict__ type, int64_t n,
                                                           uint8_t want, const uint32_t* __restrict__ off,
                                                           uint32_t* __restrict__ list,
                                                           const float4* __restrict__ xf, float4* xf_out,
                                                           const uint32_t* __restrict__ key,
                                                           uint32_t* key_out) {
  __shared__ uint32_t wsum[CMP_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)CMP_THREADS + threadIdx.x;
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool f = i < n && (want == kAnyWall ? type[i] != kFluid : type[i] == want);
  unsigned b = __ballot_sync(0xffffffffu, f);
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  uint32_t pos = off[blockIdx.x];
  for (int k = 0; k < warp; ++k) pos += wsum[k];
  pos += __popc(b & ((1u << lane) - 1u));
  if (f) {
    list[pos] = (uint32_t)i;
    if (xf_out) {  // compacted copies for scans over this type only
      xf_out[pos] = xf[i];
      key_out[pos] = key[i];
    }
  }
}

// Ordered lists of the sorted indices of fluid and of dummy particles. With
// dummies present, the fluid particles also get compacted positions and keys
// and their own cell lower bounds: the dummy update scans fluid candidates
// only (the nearest fluid particle is all it looks for).
void launch_fluid_list(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int64_t nd,
                       cudaStream_t st, int* launches) {
  if (n == 0) return;
  int64_t nb = div_up(n, CMP_THREADS);
  const bool compact = nd > 0 && w.dummy_list;
  k_count_type<<<(unsigned)nb, CMP_THREADS, 0, st>>>(s.type, n, (uint8_t)kFluid, w.block_cnt);
  k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(w.block_cnt, nb);
  k_write_type<<<(unsigned)nb, CMP_THREADS, 0, st>>>(s.type, n, (uint8_t)kFluid, w.block_cnt, w.fluid_list,
                                                      w.xf, compact ? w.xff : nullptr, w.key, w.fkey);
  *launches += 3;
  if (compact) {
    k_cell_lower_bounds<<<(unsigned)div_up(p.ncells + 1, 256), 256, 0, st>>>(w.fkey, nf, p.ncells, w.fcell_lb);
    k_count_type<<<(unsigned)nb, CMP_THREADS, 0, st>>>(s.type, n, kAnyWall, w.block_cnt);
    k_scan_exclusive<<<1, SCAN_THREADS, 0, st>>>(w.block_cnt, nb);
    k_write_type<<<(unsigned)nb, CMP_THREADS, 0, st>>>(s.type, n, kAnyWall, w.block_cnt, w.dummy_list,
                                                        nullptr, nullptr, nullptr, nullptr);
    *launches += 4;
  }
}

// ---------------------------------------------------------------------------
// Test hook: the neighbour lists themselves (all particle types), with the
// same warp-cooperative candidate enumeration (warp_scan_candidates) as the
// pair pass and the exact FP64 test of Algorithm 1.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(128) k_count_neighbors(Params p, State s, Work w, int64_t n,
                                                        uint32_t* counts) {
  __shared__ float4 stage[4][32];
  __shared__ uint32_t sidx[4][32];
  const int warp = threadIdx.x >> 5;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < n;
  const uint32_t i = active ? (uint32_t)gi : 0u;
  const uint32_t key = active ? w.key[i] : 0u;
  const float4 xs = active ? w.xf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t c = 0;
  warp_scan_candidates<DIM>(p, all_particles(w), active, i, key, xs, stage[warp], sidx[warp], [&](uint32_t j, float, float) {
    if (exact_neighbor(p, s.x, n, i, j)) ++c;
  });
  if (active) counts[s.oid[i]] = c;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_fill_neighbors(Params p, State s, Work w, int64_t n,
                                                       const int64_t* row_ptr, int32_t* cols) {
  __shared__ float4 stage[4][32];
  __shared__ uint32_t sidx[4][32];
  const int warp = threadIdx.x >> 5;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < n;
  const uint32_t i = active ? (uint32_t)gi : 0u;
  const uint32_t key = active ? w.key[i] : 0u;
  const float4 xs = active ? w.xf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  int64_t o = active ? row_ptr[s.oid[i]] : 0;
  warp_scan_candidates<DIM>(p, all_particles(w), active, i, key, xs, stage[warp], sidx[warp], [&](uint32_t j, float, float) {
    if (exact_neighbor(p, s.x, n, i, j)) cols[o++] = (int32_t)s.oid[j];
  });
}

void launch_count_neighbors(const Params& p, const State& s, const Work& w, int64_t n,
                            uint32_t* counts, cudaStream_t st) {
  if (n == 0) return;
  unsigned blocks = (unsigned)div_up(n, 128);
  if (p.dim == 3) k_count_neighbors<3><<<blocks, 128, 0, st>>>(p, s, w, n, counts);
  else k_count_neighbors<2><<<blocks, 128, 0, st>>>(p, s, w, n, counts);
}

void launch_fill_neighbors(const Params& p, const State& s, const Work& w, int64_t n,
                           const int64_t* row_ptr_by_oid, int32_t* cols, cudaStream_t st) {
  if (n == 0) return;
  unsigned blocks = (unsigned)div_up(n, 128);
  if (p.dim == 3) k_fill_neighbors<3><<<blocks, 128, 0, st>>>(p, s, w, n, row_ptr_by_oid, cols);
  else k_fill_neighbors<2><<<blocks, 128, 0, st>>>(p, s, w, n, row_ptr_by_oid, cols);
}

}  // namespace wbsph
