// pair_fp64.cu -- FP64 stage kernels of the well-balanced WCSPH step:
// prepass (dummy wall update, volumes, U_max), time step, neighbour-list
// build, the fused FP64 pair pass with its epilogue (Eq. sph with TIC,
// viscosity, delta-SPH and shifting), the SSP-RK2 stage updates, and field
// output in the caller's order.
//
// On GB300 the FP64 pipe (2 DFMA per clock per SM, 1/61 of FP32) bounds this
// path. Candidate enumeration of the 3^d cells is therefore done by a
// separate FP32/integer kernel that writes each fluid particle's candidate
// list (k-major, coalesced); the FP64 kernel then walks these lists with
// every lane busy and no shared memory, so more warps per SM cover the
// latency of the gathers and of the FP64 pipe itself.
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
  double gdot = 0.0, un = 0.0;
  for (int k = 0; k < p.dim; ++k) {
    gdot += (p.g[k] + p.force_amp[k] * fs) * (s.x[k * n + i] - s.x[k * n + best]);
    un += s.u[k * n + best] * s.normal[k * n + i];
  }
  s.phi[i] = s.phi[best] + gdot;
  for (int k = 0; k < p.dim; ++k) s.u[k * n + i] = s.u[k * n + best] - un * s.normal[k * n + i];
}

constexpr int PRE_THREADS = 256;

__global__ void __launch_bounds__(PRE_THREADS) k_volumes_umax(Params p, State s, Work w, int64_t n) {
  __shared__ unsigned long long red[PRE_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double umax2 = 0.0;
  if (i < n) {
    if (s.type[i] == kFluid)
      for (int k = 0; k < p.dim; ++k) umax2 += s.u[k * n + i] * s.u[k * n + i];
    double v = s.mass[i] / eos_density(p, s.phi[i]);
    w.vol[i] = v;
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
__global__ void k_time_step(Params p, Work w) {
  double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
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
}

void launch_time_step(const Params& p, const Work& w, cudaStream_t st) {
  k_time_step<<<1, 1, 0, st>>>(p, w);
}

// ---------------------------------------------------------------------------
// Neighbour lists: for fluid particle gi (sorted index fluid_list[gi]), in
// Algorithm 1 order, stored k-major: nbr[k * nf + gi].
//  EXACT (FP64 path, surrogate graph): every j != i with exact r <= 2h
//    (Algorithm 1's test). The FP32 distance of the warp scan decides for
//    candidates inside the inner bound; the rest of the candidates that pass
//    the conservative prefilter (a thin band near 2h) take the exact FP64 test.
//  otherwise (mixed path): every candidate that passes the FP32 prefilter;
//    the mixed pair pass applies its own FP32 test.
// Lists are staged per warp in shared memory so the global stores are
// coalesced rows.
// ---------------------------------------------------------------------------
constexpr int LIST_THREADS = 64;

template <int DIM, bool EXACT>
__global__ void __launch_bounds__(LIST_THREADS) k_nbr_list(Params p, State s, Work w, int64_t n, int64_t nf,
                                                         int kmax, int ks) {
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
  warp_scan_candidates<DIM>(p, all_particles(w), active, i, key, xs, stage, sidx, [&](uint32_t j, float r2f, float) {
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

// ---------------------------------------------------------------------------
// Fused FP64 pair pass over fluid particles (one lane per particle i).
// Accumulated with g = -W'(r)/r V_j >= 0, so grad_i W_ij V_j = g r (r = x_j - x_i):
//   L  += r (x) g r                       (Eq. renorm; symmetric)
//   S  += [phi_j - phi_i - C0 (U_j - U_i).r/|r|] g r      (2(phi* - phi_i), Eq. lfsover)
//   M  += (U_j - U_i) (x) g r             (continuity, corrected in the epilogue)
//   C  += (phi_i + phi_j) g r             (conservative gradient, TIC branch)
//   D  += (phi_j - phi_i) g               (delta-SPH: (x_j-x_i).grad W/|r|^2 V_j = g)
//   Lam+= (U_j - U_i) g, fluid j only     (Laplacian operator, Sec. 2.1/2.4)
//   P  += [1 + R (W_ij / W(dx))^n] g r    (shifting)
// ---------------------------------------------------------------------------
constexpr int PAIR_THREADS = 128;

// Reciprocal square root: FP32 estimate refined by one Newton-Raphson step
// y <- y + (y/2)(1 - r2 y^2) in FP64, relative error about 1e-13 (the step
// squares the ~2e-7 error of the estimate). The FP64 <-> FP32 moves are done
// on the IEEE fields with integer instructions, keeping the FP64 pipe for
// the pair sums: r2 (positive, FP32 normal range) is truncated to FP32 by
// rebiasing the exponent (1023 -> 127) and keeping the top 23 mantissa bits;
// y and y/2 are widened exactly the other way.
__device__ __forceinline__ double rsqrt_nr1(double r2) {
  constexpr unsigned kRebias = (1023u - 127u) << 20;
  const unsigned hi = (unsigned)__double2hiint(r2), lo = (unsigned)__double2loint(r2);
  const unsigned fb = ((hi - kRebias) << 3) | (lo >> 29);
  const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const double y = __hiloint2double((int)((yb >> 3) + kRebias), (int)(yb << 29));
  const double hy = __hiloint2double((int)((yb >> 3) + kRebias - (1u << 20)), (int)(yb << 29));
  return fma(hy, fma(-r2 * y, y, 1.0), y);
}

template <int DIM>
__global__ void __launch_bounds__(PAIR_THREADS, 4)
    k_pair_fp64(Params p, State s, Work w, int64_t n, int64_t nf, int stage2) {
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;
  const int cnt = active ? (int)w.nbr_cnt[gi] : 0;

  double xi[DIM], ui[DIM], phii = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    xi[k] = active ? s.x[k * n + i] : 0.0;
    ui[k] = active ? s.u[k * n + i] : 0.0;
  }
  if (active) phii = s.phi[i];

  double L[6] = {0, 0, 0, 0, 0, 0}, S[DIM], M[DIM * DIM], C[DIM], Lam[DIM], P[DIM], D = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) { S[k] = C[k] = Lam[k] = P[k] = 0.0; }
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) M[k] = 0.0;

  const bool pst4 = p.use_pst && p.pst_n == 4.0;
  unsigned npairs = 0;
  const int maxc = __reduce_max_sync(0xffffffffu, cnt);
  const uint32_t* lst = w.nbr + gi;
  for (int k = 0; k < maxc; ++k) {
    if (k >= cnt) continue;
    uint32_t j = __ldg(lst + (int64_t)k * nf);
    // every list entry is an exact neighbour (k_nbr_list applies the test)
    double r[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) r[c] = __dsub_rn(s.x[c * n + j], xi[c]);
    double r2 = r[0] * r[0];
#pragma unroll
    for (int c = 1; c < DIM; ++c) r2 = fma(r[c], r[c], r2);
    ++npairs;
    double inv_r = rsqrt_nr1(r2);
    double rr = r2 * inv_r;
    double t = fma(-rr, p.inv_two_h, 1.0);
    double t2 = t * t;
    double g = t2 * (t * w.volc[j]);
    double gr[DIM], du[DIM];
    double dun = 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      gr[c] = g * r[c];
      du[c] = s.u[c * n + j] - ui[c];
      dun = fma(du[c], r[c], dun);
    }
    dun *= inv_r;
    double phij = s.phi[j];
    double dphi = phij - phii;
    double sphi = phij + phii;
    double rs = fma(-p.c0, dun, dphi);
    if (DIM == 2) {
      L[0] = fma(r[0], gr[0], L[0]);
      L[1] = fma(r[0], gr[1], L[1]);
      L[2] = fma(r[1], gr[1], L[2]);
    } else {
      L[0] = fma(r[0], gr[0], L[0]);
      L[1] = fma(r[0], gr[1], L[1]);
      L[2] = fma(r[0], gr[DIM - 1], L[2]);
      L[3] = fma(r[1], gr[1], L[3]);
      L[4] = fma(r[1], gr[DIM - 1], L[4]);
      L[5] = fma(r[DIM - 1], gr[DIM - 1], L[5]);
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      S[c] = fma(rs, gr[c], S[c]);
      C[c] = fma(sphi, gr[c], C[c]);
#pragma unroll
      for (int e = 0; e < DIM; ++e) M[c * DIM + e] = fma(du[c], gr[e], M[c * DIM + e]);
    }
    D = fma(dphi, g, D);
    if (s.type[j] == kFluid) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) Lam[c] = fma(du[c], g, Lam[c]);
    }
    if (p.use_pst) {
      double q21 = fma(rr, p.two_over_h, 1.0);  // 2q + 1
      double v = (t2 * t2) * q21;               // W_ij / W(dx) = pst_alpha_over_wdx * v
      double f;
      if (pst4) {
        double v2 = v * v;
        f = fma(p.pst_R_a4, v2 * v2, 1.0);      // 1 + R (W_ij / W(dx))^4
      } else {
        f = fma(p.pst_R, pow(p.pst_alpha_over_wdx * v, p.pst_n), 1.0);
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) P[c] = fma(f, gr[c], P[c]);
    }
  }
  const int lane = threadIdx.x & 31;
  unsigned wp = __reduce_add_sync(0xffffffffu, npairs);
  if (lane == 0 && wp) atomicAdd(w.pairs, (unsigned long long)wp);
  if (!active) return;

  // ---- epilogue (Eq. sph with the TIC switch; Sec. 3: correction outside the sum) ----
  // The switch needs only lambda_min < threshold: the FP32 closed form
  // decides unless it lies within 0.05 of the threshold (its error is below
  // 1e-2 even where two eigenvalues meet), where the FP64 closed form decides.
  // The lambda_min field itself is formed in FP64 from the stored L when it
  // is read (k_lambda_fp64).
  bool tic_branch = false;
  if (p.use_tic) {
    const float lf = DIM == 2 ? lambda_min_2f((float)L[0], (float)L[1], (float)L[2])
                              : lambda_min_3f((float)L[0], (float)L[1], (float)L[2], (float)L[3], (float)L[4],
                                              (float)L[5]);
    const float tl = (float)p.tic_lambda;
    if (fabsf(lf - tl) > 0.05f) {
      tic_branch = lf < tl;
    } else {
      const double lam = DIM == 2 ? lambda_min_2(L[0], L[1], L[2])
                                  : lambda_min_3(L[0], L[1], L[2], L[3], L[4], L[5]);
      tic_branch = lam < p.tic_lambda;
    }
  }
#pragma unroll
  for (int k = 0; k < (DIM == 2 ? 3 : 6); ++k) w.Lmat[k * n + i] = L[k];
  double gradphi[DIM], divu = 0.0;
  if (tic_branch) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      gradphi[c] = C[c];
      divu += M[c * DIM + c];
    }
  } else {
    double inv[DIM][DIM];
    if (!sym_inverse<DIM>(L, inv)) atomicOr(w.status, kStatSingular);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double gsum = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        gsum = fma(inv[c][e], S[e], gsum);
        divu = fma(inv[c][e], M[c * DIM + e], divu);
      }
      gradphi[c] = gsum;
    }
  }
  double fs = forcing_factor(p, stage_time(w, stage2));
  double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
  bool bad = false;
  double dstar[DIM], dn2 = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double visc = p.use_visc ? 2.0 * p.nu * Lam[c] : 0.0;
    double acc = -gradphi[c] + visc + (p.g[c] + p.force_amp[c] * fs);
    w.dudt[c * n + i] = acc;
    bad |= !isfinite(acc);
    dstar[c] = -2.0 * p.h * umax * P[c];
    dn2 += dstar[c] * dstar[c];
  }
  double diff = p.use_delta ? p.delta_h_c0 * (2.0 * D) : 0.0;
  double dphidt = -eos_c2(p, phii) * divu + diff;
  w.dphidt[i] = dphidt;
  bad |= !isfinite(dphidt);
  double dn = sqrt(dn2);
  double scale = 0.0;
  if (p.use_pst && dn > 0.0) scale = fmin(dn, 0.5 * umax) / dn;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double v = dstar[c] * scale;
    w.dushift[c * n + i] = v;
    bad |= !isfinite(v);
  }
  if (bad) atomicOr(w.status, kStatNaN);
}

// lambda_min(L) of the last FP64 pair pass, from the stored L (fluid rows;
// dummies keep zero).
__global__ void k_lambda_fp64(Params p, Work w, int64_t n, int64_t nf) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= nf) return;
  const uint32_t i = w.fluid_list[gi];
  const double* L = w.Lmat;
  w.lambda[i] = p.dim == 2 ? lambda_min_2(L[i], L[n + i], L[2 * n + i])
                           : lambda_min_3(L[i], L[n + i], L[2 * n + i], L[3 * n + i], L[4 * n + i], L[5 * n + i]);
}

void launch_lambda_fp64(const Params& p, const Work& w, int64_t n, int64_t nf, cudaStream_t st) {
  if (nf == 0) return;
  k_lambda_fp64<<<(unsigned)div_up(nf, 256), 256, 0, st>>>(p, w, n, nf);
}

int pair_list_kmax(int dim) { return dim == 3 ? 128 : 48; }

// List entries per lane staged in shared memory (the rest are stored
// directly, uncoalesced): 80 holds the candidates of most particles of 3D
// lattices at h = 1.3 dx (about 75) and leaves room for 20 resident warps
// per SM, which this latency-bound kernel needs more than coalesced stores
// of the few entries beyond.
#ifndef WBSPH_LIST_STAGE_3D
#define WBSPH_LIST_STAGE_3D 80
#endif
static int pair_list_stage(int dim) { return dim == 3 ? WBSPH_LIST_STAGE_3D : 48; }

void launch_nbr_list(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, cudaStream_t st,
                     bool exact) {
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
    if (exact) k_nbr_list<3, true><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks);
    else k_nbr_list<3, false><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks);
  } else {
    if (exact) k_nbr_list<2, true><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks);
    else k_nbr_list<2, false><<<blocks, LIST_THREADS, sm, st>>>(p, s, w, n, nf, kmax, ks);
  }
}

void launch_pair_fp64(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                      int stage2, cudaStream_t st) {
  if (nf == 0) return;
  unsigned blocks = (unsigned)div_up(nf, PAIR_THREADS);
  if (p.dim == 2) k_pair_fp64<2><<<blocks, PAIR_THREADS, 0, st>>>(p, s, w, n, nf, stage2);
  else k_pair_fp64<3><<<blocks, PAIR_THREADS, 0, st>>>(p, s, w, n, nf, stage2);
}

// ---------------------------------------------------------------------------
// SSP-RK2 stages (Sec. 2.3), fluid particles; dummies stay fixed.
//   stage 1: y0 = y;  y = y0 + dt F(y0);  x = x0 + dt (U0 + dU0)
//   stage 2: y = y0/2 + (y1 + dt F(y1))/2; x = x0/2 + (x1 + dt (U1 + dU1))/2
// Stage 2 also advances t by dt (one thread, after every reader of t).
// ---------------------------------------------------------------------------
__global__ void k_rk_stage(Params p, State s, Work w, int64_t n, int stage) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dt = w.scalars[1];
  if (stage == 2 && i == 0) w.scalars[0] = w.scalars[0] + dt;
  if (i >= n) return;
  bool fluid = s.type[i] == kFluid;
  if (stage == 1) {
    for (int k = 0; k < p.dim; ++k) {
      double x0 = s.x[k * n + i], u0 = s.u[k * n + i];
      s.x0[k * n + i] = x0;
      s.u0[k * n + i] = u0;
      if (fluid) {
        s.x[k * n + i] = x0 + dt * (u0 + w.dushift[k * n + i]);
        s.u[k * n + i] = u0 + dt * w.dudt[k * n + i];
      }
    }
    double ph0 = s.phi[i];
    s.phi0[i] = ph0;
    if (fluid) s.phi[i] = ph0 + dt * w.dphidt[i];
  } else if (fluid) {
    for (int k = 0; k < p.dim; ++k) {
      double x1 = s.x[k * n + i], u1 = s.u[k * n + i];
      s.x[k * n + i] = 0.5 * s.x0[k * n + i] + 0.5 * (x1 + dt * (u1 + w.dushift[k * n + i]));
      s.u[k * n + i] = 0.5 * s.u0[k * n + i] + 0.5 * (u1 + dt * w.dudt[k * n + i]);
    }
    s.phi[i] = 0.5 * s.phi0[i] + 0.5 * (s.phi[i] + dt * w.dphidt[i]);
  }
}

void launch_rk_stage(const Params& p, const State& s, const Work& w, int64_t n, int stage,
                     cudaStream_t st) {
  k_rk_stage<<<(unsigned)div_up(n > 0 ? n : 1, 256), 256, 0, st>>>(p, s, w, n, stage);
}

// ---------------------------------------------------------------------------
// Field output in original order: out[k n + oid[i]] = field[k n + i].
// ---------------------------------------------------------------------------
__global__ void k_field(Params p, State s, Work w, int64_t n, int field, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = s.oid[i];
  const double* src = nullptr;
  int comps = 1;
  switch (field) {
    case 0: src = s.x; comps = p.dim; break;
    case 1: src = s.u; comps = p.dim; break;
    case 2: src = s.phi; break;
    case 5: src = w.dudt; comps = p.dim; break;
    case 6: src = w.dphidt; break;
    case 7: src = w.dushift; comps = p.dim; break;
    case 8: src = w.lambda; break;
    case 9: src = s.mass; break;
    case 10: src = w.vol; break;
    default: break;
  }
  if (field == 3 || field == 4) {
    double rho = eos_density(p, s.phi[i]);
    double v = rho;
    if (field == 4) {
      v = p.eos == 0 ? p.c0sq * (rho - p.rho0)
                     : p.rho0 * p.c0sq / p.gamma * (pow(rho / p.rho0, p.gamma) - 1.0);
    }
    out[o] = v;
    return;
  }
  if (!src) return;
  for (int k = 0; k < comps; ++k) out[k * n + o] = src[k * n + i];
}

void launch_field(const Params& p, const State& s, const Work& w, int64_t n, int field,
                  double* out, cudaStream_t st) {
  if (n == 0) return;
  k_field<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p, s, w, n, field, out);
}

}  // namespace wbsph
