// prepass.cu -- per-stage work before the pair pass: the dummy wall update
// (Sec. 2.4), particle volumes and U_max, the time step (Sec. 2.3), the
// packed FP32 copies of the mixed path and the hi/lo copies of the
// double-float path.
#include "../../include/wbsph.h"
#include "common.cuh"
#include "neighbor_iter.cuh"
#include "physics.cuh"
#include "warp_scan.cuh"

namespace wbsph {
// ---------------------------------------------------------------------------
// Prepass. (1) Dummy particles (Sec. 2.4), one lane per dummy: nearest fluid
// particle f within 2h (exact FP64 squared distance; ties to the smaller
// original id), phi_d = phi_f + G(t).(x_d - x_f) (Eq. phiBn), slip velocity
// U_d = U_f - (U_f.n_d) n_d. A warp-staged FP32 scan evaluates the exact
// FP64 distance only for candidates within a proven rounding band of the
// running FP32 minimum. (2) V = m / rho(phi) for
// every particle and max |U|^2 over fluid particles.
// ---------------------------------------------------------------------------
constexpr int DUM_THREADS = 128;

template <int DIM>
__global__ void __launch_bounds__(DUM_THREADS) k_dummy_update(Params p, State s, Work w, int64_t n,
                                                             int64_t nd, int stage2) {
  __shared__ float4 stage[DUM_THREADS / 32][32];
  __shared__ uint32_t sidx[DUM_THREADS / 32][32];
  const int warp = threadIdx.x >> 5;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nd;
  const uint32_t i = active ? w.dummy_list[gi] : 0u;
  const uint32_t key = active ? w.key[i] : 0u;
  const float4 xs = active ? w.xf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  // One FP32 scan keeps the (at most 4) fluid candidates whose FP32 distance
  // lies within the rounding band of the running FP32 minimum; the exact
  // FP64 distances decide among those left within the band of the final
  // minimum. A candidate dropped at any point lies outside the band of the
  // final minimum too, so it cannot be the exact nearest. If more than 4
  // candidates share the band, a second scan evaluates all of them exactly.
  constexpr int KEEP = 4;
  float best_f = INFINITY;
  uint32_t kj[KEEP] = {0u, 0u, 0u, 0u};
  float kr[KEEP] = {INFINITY, INFINITY, INFINITY, INFINITY};  // slot free when > band limit
  bool spill = false;
  warp_scan_candidates<DIM>(p, fluid_particles(w), active, i, key, xs, stage[warp], sidx[warp],
                            [&](uint32_t j, float r2f, float jtype) {
    if (jtype != 0.f) return;  // fluid neighbours only
    if (r2f > best_f + p.nearest_band_r2) return;
    best_f = fminf(best_f, r2f);
    const float lim_now = best_f + p.nearest_band_r2;
    bool placed = false;
#pragma unroll
    for (int q = 0; q < KEEP; ++q)
      if (!placed && kr[q] > lim_now) { kr[q] = r2f; kj[q] = j; placed = true; }
    spill |= !placed;
  });
  uint32_t best = kEmpty, best_oid = kEmpty;
  double best_r2 = 0.0;
  auto consider = [&](uint32_t j) {
    double d0 = __dsub_rn(s.x[j], s.x[i]);
    double r2 = __dmul_rn(d0, d0);
    double d1 = __dsub_rn(s.x[n + j], s.x[n + i]);
    r2 = __dadd_rn(r2, __dmul_rn(d1, d1));
    if (p.dim == 3) {
      double d2 = __dsub_rn(s.x[2 * n + j], s.x[2 * n + i]);
      r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
    }
    if (!(r2 <= p.four_h2 && r2 > 0.0)) return;
    uint32_t o = s.oid[j];
    if (best == kEmpty || r2 < best_r2 || (r2 == best_r2 && o < best_oid)) {
      best = j; best_r2 = r2; best_oid = o;
    }
  };
  const float lim = best_f + p.nearest_band_r2;
  if (!spill && best_f < INFINITY) {  // empty slots hold r = inf and no index
#pragma unroll
    for (int q = 0; q < KEEP; ++q)
      if (kr[q] <= lim) consider(kj[q]);
  }
  if (__any_sync(0xffffffffu, spill)) {
    warp_scan_candidates<DIM>(p, fluid_particles(w), active && spill, i, key, xs, stage[warp], sidx[warp],
                              [&](uint32_t j, float r2f, float jtype) {
      if (jtype == 0.f && r2f <= lim) consider(j);
    });
  }
  if (!active || best == kEmpty) return;
  double fs = forcing_factor(p, stage_time(w, stage2));
  // wall velocity U_w: zero for fixed walls, body_u for body particles; slip
  // U_d = U_f - ((U_f - U_w).n) n, or no-slip U_d = 2 U_w - U_f (Eq. velBn)
  const bool body = s.type[i] == kBody;
  double gdot = 0.0, un = 0.0;
  for (int k = 0; k < p.dim; ++k) {
    const double uw = body ? p.body_u[k] : 0.0;
    gdot += (p.g[k] + p.force_amp[k] * fs) * (s.x[k * n + i] - s.x[k * n + best]);
    un += (s.u[k * n + best] - uw) * s.normal[k * n + i];
  }
  s.phi[i] = s.phi[best] + gdot;
  for (int k = 0; k < p.dim; ++k) {
    const double uw = body ? p.body_u[k] : 0.0;
    s.u[k * n + i] = p.wall_bc == 1 ? 2.0 * uw - s.u[k * n + best] : s.u[k * n + best] - un * s.normal[k * n + i];
  }
}

constexpr int PRE_THREADS = 256;

__global__ void __launch_bounds__(PRE_THREADS) k_volumes_umax(Params p, State s, Work w, int64_t n) {
  __shared__ unsigned long long red[PRE_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double umax2 = 0.0;
  if (i < n) {
    if (s.type[i] == kFluid)
      for (int k = 0; k < p.dim; ++k) umax2 += s.u[k * n + i] * s.u[k * n + i];
    const double rho = eos_density(p, s.phi[i]);
    double v = s.mass[i] / rho;
    w.vol[i] = v;
    if (p.scheme == 1) {  // the conventional scheme's density and pressure (EOS)
      w.rho[i] = rho;
      w.pres[i] = p.eos == 0 ? p.c0sq * (rho - p.rho0)
                             : p.rho0 * p.c0sq / p.gamma * (pow(rho / p.rho0, p.gamma) - 1.0);
    }
    w.volc[i] = p.neg_dwdr_over_r_coef * v;  // -W'(r)/r V = volc (1 - q/2)^3
    if (!isfinite(v)) atomicOr(w.status, kStatNaN);
  }
  // block max of |U|^2, then one atomic per block on the bit pattern
  // (non-negative doubles order like their unsigned 64-bit patterns)
  unsigned long long b = __double_as_longlong(umax2);
  for (int off = 16; off; off >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
    b = o > b ? o : b;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int k = 0; k < PRE_THREADS / 32; ++k) m = red[k] > m ? red[k] : m;
    if (m) atomicMax(w.umax_bits, m);
  }
}

// U_max^2 over fluid particles alone (surrogate stages, which need no
// volumes); the block max and one atomic per block as in k_volumes_umax.
__global__ void __launch_bounds__(PRE_THREADS) k_umax(Params p, State s, Work w, int64_t n) {
  __shared__ unsigned long long red[PRE_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double umax2 = 0.0;
  if (i < n && s.type[i] == kFluid)
    for (int k = 0; k < p.dim; ++k) umax2 += s.u[k * n + i] * s.u[k * n + i];
  unsigned long long b = __double_as_longlong(umax2);
  for (int off = 16; off; off >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, b, off);
    b = o > b ? o : b;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int k = 0; k < PRE_THREADS / 32; ++k) m = red[k] > m ? red[k] : m;
    if (m) atomicMax(w.umax_bits, m);
  }
}

void launch_umax(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st) {
  if (n > 0) k_umax<<<(unsigned)div_up(n, PRE_THREADS), PRE_THREADS, 0, st>>>(p, s, w, n);
}

void launch_prepass(const Params& p, const State& s, const Work& w, int64_t n, int64_t nd,
                    int stage2, cudaStream_t st, bool volumes) {
  cudaMemsetAsync(w.umax_bits, 0, sizeof(unsigned long long), st);
  if (n == 0) return;
  if (nd > 0) {
    unsigned blocks = (unsigned)div_up(nd, DUM_THREADS);
    if (p.dim == 3) k_dummy_update<3><<<blocks, DUM_THREADS, 0, st>>>(p, s, w, n, nd, stage2);
    else k_dummy_update<2><<<blocks, DUM_THREADS, 0, st>>>(p, s, w, n, nd, stage2);
  }
  if (volumes) k_volumes_umax<<<(unsigned)div_up(n, PRE_THREADS), PRE_THREADS, 0, st>>>(p, s, w, n);
}

// Time step (Sec. 2.3): CFL * min(dx/(C0 + U_max), dx^2/(2 nu), sqrt(2 dx/|G|)).
__global__ void k_time_step(Params p, Work w, int keep_lists) {
  double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
  if (p.body_speed > umax) umax = p.body_speed;  // a prescribed body also bounds the step
  double dt;
  if (p.fixed_dt > 0) {
    dt = p.fixed_dt;
  } else {
    double t = p.dx / (p.c0 + umax);
    if (p.nu > 0) {
      double td = p.dx * p.dx / (2.0 * p.nu);
      if (td < t) t = td;
    }
    double g2 = 0.0;
    for (int k = 0; k < p.dim; ++k) g2 += p.g[k] * p.g[k];
    if (g2 > 0) {
      double tg = sqrt(2.0 * p.dx / sqrt(g2));
      if (tg < t) t = tg;
    }
    dt = p.cfl * t;
  }
  w.scalars[1] = dt;
  if (p.skin && keep_lists) {
    // lists kept for stage 2: a particle moves at most dt (U_max + U_max/2)
    // (or dt |body_u|) in stage 1, so pairs within 2h at stage 2 lie within
    // 2h + delta at stage 1; the margin covers the rounding of the move
    const double delta = 3.0 * dt * umax * (1.0 + 1e-6);
    if (delta > p.skin_max) atomicOr(w.status, kStatSkin);
    const double rl = p.two_h + delta + p.skin_e;
    w.scalars[3] = rl * rl * (1.0 + 16.0 * 5.9604644775390625e-08);
  }
}

void launch_time_step(const Params& p, const Work& w, cudaStream_t st, bool keep_lists) {
  k_time_step<<<1, 1, 0, st>>>(p, w, keep_lists ? 1 : 0);
}

// FP32 value of a finite double, rounded to nearest (ties away from zero) on
// its IEEE fields with integer instructions, so that the FP64 pipe only
// does the arithmetic that needs it; magnitudes below 2^-126 give zero.
__device__ __forceinline__ float mx_d2f(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  b = (b & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);  // half of the 29 dropped bits; a carry renormalises
  const unsigned e = (unsigned)(b >> 52);
  if (e <= 1023u - 127u) return 0.f;
  return __uint_as_float(sign | ((e - (1023u - 127u)) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu));
}

// FP64 value of a positive normal float (V), widened exactly on the IEEE
// fields; zero and anything else non-normal gives zero.
__device__ __forceinline__ double mx_f2d(float v) {
  const unsigned b = __float_as_uint(v), e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return 0.0;
  return __hiloint2double((int)((b & 0x80000000u) | ((e + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3)),
                          (int)(b << 29));
}

// exponent field of a double is all ones: infinity or NaN
__device__ __forceinline__ bool mx_nonfinite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7FF00000u) == 0x7FF00000u;
}

// ---- prepass of the mixed path, per particle (after the dummy update) ----
// U_max^2 over fluid particles (FP64, for the time step and shifting); the
// volume V = m / rho(phi) in FP32 (it only enters the FP32 pair sums); and the
// packed FP32 copies read by the pair pass:
//   A[i] = (x - cell origin, phi - phi_hs(x)), B[i] = (U, V) with V < 0 marking
//   wall particles (with slip walls the Laplacian operator takes fluid neighbours only),
//   C[i] = cell coordinates packed 11/11/10 bits.
// w.vol receives V widened to FP64.
constexpr int MXP_THREADS = 256;

__global__ void __launch_bounds__(MXP_THREADS) k_prepass_mixed(Params p, State s, Work w, int64_t n, float4* A,
                                                               float4* B, uint32_t* Cc) {
  __shared__ unsigned long long red[MXP_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double umax2 = 0.0;
  if (i < n) {
    const bool fluid = s.type[i] == kFluid;
    const uint32_t key = w.key[i];
    const uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
    const uint32_t ic[3] = {key % nx, (key / nx) % ny, key / (nx * ny)};
    float o[3] = {0.f, 0.f, 0.f};
    float u[3] = {0.f, 0.f, 0.f};
    double phs = p.phs0;
    bool bad = false;
    const double* org = w.cell_origin;  // origins of axis 0, then 1, then 2
    for (int k = 0; k < p.dim; ++k) {
      const double xk = s.x[k * n + i], uk = s.u[k * n + i];
      bad |= mx_nonfinite(xk) | mx_nonfinite(uk);
      o[k] = mx_d2f(xk - __ldg(org + ic[k]));  // x - (domain_min + i R)
      org += p.nc[k];
      u[k] = mx_d2f(uk);
      if (fluid) umax2 = fma(uk, uk, umax2);
      if (p.g[k] != 0.0) phs = fma(p.g[k], xk, phs);
    }
    const double phi = s.phi[i];
    bad |= mx_nonfinite(phi);
    const float phif = mx_d2f(phi);
    // rho / rho0 = exp(phi / C0^2) (linear EOS) or (1 + (gamma-1) phi / c0^2)^(1/(gamma-1)) (Tait)
    const float inv_c0sq = p.inv_c0sq_f;
    float inv_rel;
    if (p.eos == 0) {
      inv_rel = expf(-phif * inv_c0sq);
    } else {
      const float gm1 = (float)(p.gamma - 1.0);
      inv_rel = powf(fmaf(gm1 * phif, inv_c0sq, 1.f), -1.f / gm1);
    }
    float v = mx_d2f(s.mass[i]) * p.inv_rho0_f * inv_rel;
    bad |= !isfinite(v);
    if (bad) atomicOr(w.status, kStatNaN);
    w.vol[i] = mx_f2d(v);
    A[i] = make_float4(o[0], o[1], o[2], mx_d2f(phi - phs));
    B[i] = make_float4(u[0], u[1], u[2], fluid ? v : -v);
    Cc[i] = ic[0] | (ic[1] << 11) | (ic[2] << 22);
  }
  // block max of |U|^2, one atomic per block on the bit pattern
  unsigned long long b = (unsigned long long)__double_as_longlong(umax2);
  for (int off = 16; off; off >>= 1) {
    unsigned long long q = __shfl_xor_sync(0xffffffffu, b, off);
    b = q > b ? q : b;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int k = 0; k < MXP_THREADS / 32; ++k) m = red[k] > m ? red[k] : m;
    if (m) atomicMax(w.umax_bits, m);
  }
}

// Mixed prepass (after the dummy update, which resets U_max); fails when the
// grid is too large for the packed cell coordinates (11/11/10 bits).
int launch_prepass_mixed(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st) {
  if (n == 0) return 0;
  if (p.nc[0] > 2048 || p.nc[1] > 2048 || p.nc[2] > 1024) return WBSPH_E_INVAL;
  k_prepass_mixed<<<(unsigned)div_up(n, MXP_THREADS), MXP_THREADS, 0, st>>>(p, s, w, n, w.packA, w.packB,
                                                                            w.packC);
  return 0;
}

// ---- pack of the double-float path, per particle (after the FP64 prepass:
// dummy walls, V, volc, U_max) ----
//   A  = (o_hi, phi'_hi)   Al = (o_lo, phi'_lo)
//   B  = (U_hi, volc_hi)   Bl = (U_lo, volc_lo)   volc negated (both parts) for wall particles
//   C  = cell coordinates packed 11/11/10 bits
// o = (x - cell origin) / R in cell units. o_hi is o rounded to a multiple of
// 2^-23 by adding and subtracting 1.5 * 2^29 (its ulp is 2^-23, exact for
// |o| < 2^28), an FP32 number for |o| < 2; |o| < 1.5 is required (a
// particle may drift half a cell out of the cell of its last neighbour
// build), else the domain bit is set. The other hi parts are the nearest
// FP32 numbers; each lo part is the FP64 remainder (exact: Sterbenz's
// lemma) rounded to FP32. The moves between FP64 and FP32 are integer
// instructions, so the FP64 pipe only does the additions.
constexpr int DFP_THREADS = 256;

__device__ __forceinline__ void df_split(double v, float& hi, float& lo) {
  hi = mx_d2f(v);
  lo = mx_d2f(v - mx_f2d(hi));
}

__global__ void __launch_bounds__(DFP_THREADS) k_pack_df(Params p, State s, Work w, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t key = w.key[i];
  const uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
  const uint32_t ic[3] = {key % nx, (key / nx) % ny, key / (nx * ny)};
  float ah[4] = {0.f, 0.f, 0.f, 0.f}, al[4] = {0.f, 0.f, 0.f, 0.f};
  float bh[4] = {0.f, 0.f, 0.f, 0.f}, bl[4] = {0.f, 0.f, 0.f, 0.f};
  constexpr double kRound23 = 805306368.0;  // 1.5 * 2^29
  double phs = p.phs0;
  bool bad = false, off = false;
  const double* org = w.cell_origin;  // origins of axis 0, then 1, then 2
  for (int k = 0; k < p.dim; ++k) {
    const double xk = s.x[k * n + i], uk = s.u[k * n + i];
    bad |= mx_nonfinite(xk) | mx_nonfinite(uk);
    const double o = (xk - __ldg(org + ic[k])) * p.inv_R;
    org += p.nc[k];
    off |= !(fabs(o) < 1.5);
    const double q = __dsub_rn(__dadd_rn(o, kRound23), kRound23);  // multiple of 2^-23
    ah[k] = mx_d2f(q);                            // exact
    al[k] = mx_d2f(o - q);
    df_split(uk, bh[k], bl[k]);
    if (p.g[k] != 0.0) phs = fma(p.g[k], xk, phs);
  }
  const double phi = s.phi[i];
  bad |= mx_nonfinite(phi);
  df_split(phi - phs, ah[3], al[3]);
  df_split(w.volc[i], bh[3], bl[3]);
  if (s.type[i] != kFluid) {
    bh[3] = -bh[3];
    bl[3] = -bl[3];
  }
  if (bad) atomicOr(w.status, kStatNaN);
  if (off) atomicOr(w.status, kStatDomain);
  w.packA[i] = make_float4(ah[0], ah[1], ah[2], ah[3]);
  w.packAl[i] = make_float4(al[0], al[1], al[2], al[3]);
  w.packB[i] = make_float4(bh[0], bh[1], bh[2], bh[3]);
  w.packBl[i] = make_float4(bl[0], bl[1], bl[2], bl[3]);
  w.packC[i] = ic[0] | (ic[1] << 11) | (ic[2] << 22);
}

// Double-float pack (after the FP64 prepass); fails when the grid is too
// large for the packed cell coordinates (11/11/10 bits).
int launch_pack_df(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st) {
  if (n == 0) return 0;
  if (p.nc[0] > 2048 || p.nc[1] > 2048 || p.nc[2] > 1024) return WBSPH_E_INVAL;
  k_pack_df<<<(unsigned)div_up(n, DFP_THREADS), DFP_THREADS, 0, st>>>(p, s, w, n);
  return 0;
}

}  // namespace wbsph
