// pair_fp64.cu -- FP64 stage kernels of the well-balanced WCSPH step:
// prepass (dummy wall update, volumes, U_max), time step, the fused pair pass
// with its epilogue (Eq. sph with TIC, viscosity, delta-SPH and shifting),
// the SSP-RK2 stage updates, and field output in the caller's order.
//
// On GB300 the FP64 pipe (about 2 DFMA per clock per SM) bounds this path,
// so the pair pass is split per warp into (A) an FP32/integer phase that
// enumerates candidates of the 3^d cells and writes compact per-lane
// neighbour lists to shared memory, and (B) an FP64 phase that walks those
// lists with every lane busy. Lanes that would otherwise idle in FP64
// instructions cost pipe cycles, so (B) never runs on candidate tests.
#include <cstdio>
#include "common.cuh"
#include "neighbor_iter.cuh"

namespace wbsph {

__device__ __forceinline__ double eos_density(const Params& p, double phi) {
  if (p.eos == 0) return p.rho0 * exp(phi / p.c0sq);
  double gm1 = p.gamma - 1.0;
  return p.rho0 * pow(1.0 + gm1 * phi / p.c0sq, 1.0 / gm1);
}

// D(phi)/Dt = -c^2 div U: c^2 = C0^2 (linear EOS), c0^2 + (gamma - 1) phi (Tait).
__device__ __forceinline__ double eos_c2(const Params& p, double phi) {
  return p.eos == 0 ? p.c0sq : p.c0sq + (p.gamma - 1.0) * phi;
}

__device__ __forceinline__ void body_force(const Params& p, double t, double g[3]) {
  double s = 0.0;
  if (p.omega > 0.0) s = p.omega * p.omega * sin(p.omega * t);
  for (int k = 0; k < 3; ++k) g[k] = p.g[k] + p.force_amp[k] * s;
}

__device__ __forceinline__ double stage_time(const Work& w, int stage2) {
  return stage2 ? w.scalars[0] + w.scalars[1] : w.scalars[0];
}

// ---------------------------------------------------------------------------
// Prepass, all particles. Dummy particles (Sec. 2.4): nearest fluid particle
// f within 2h (exact FP64 squared distance; ties to the smaller original id),
// phi_d = phi_f + G(t).(x_d - x_f) (Eq. phiBn), slip velocity
// U_d = U_f - (U_f.n_d) n_d. Then V = m / rho(phi) for every particle and the
// maximum |U|^2 over fluid particles (for the shifting velocity scale).
// ---------------------------------------------------------------------------
constexpr int PRE_THREADS = 256;

__global__ void __launch_bounds__(PRE_THREADS) k_prepass(Params p, State s, Work w, int64_t n, int stage2) {
  __shared__ unsigned long long red[PRE_THREADS / 32];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double umax2 = 0.0;
  if (i < n) {
    int ty = s.type[i];
    if (ty == kDummy) {
      CandidateIter it;
      it.init(p, w, n, (uint32_t)i);
      uint32_t j, best = kEmpty, best_oid = kEmpty;
      double best_r2 = 0.0;
      while (it.next(p, w, j)) {
        if (s.type[j] != kFluid) continue;
        double d0 = __dsub_rn(s.x[j], s.x[i]);
        double r2 = __dmul_rn(d0, d0);
        double d1 = __dsub_rn(s.x[n + j], s.x[n + i]);
        r2 = __dadd_rn(r2, __dmul_rn(d1, d1));
        if (p.dim == 3) {
          double d2 = __dsub_rn(s.x[2 * n + j], s.x[2 * n + i]);
          r2 = __dadd_rn(r2, __dmul_rn(d2, d2));
        }
        if (!(r2 <= p.four_h2 && r2 > 0.0)) continue;
        uint32_t o = s.oid[j];
        if (best == kEmpty || r2 < best_r2 || (r2 == best_r2 && o < best_oid)) {
          best = j; best_r2 = r2; best_oid = o;
        }
      }
      if (best != kEmpty) {
        double G[3];
        body_force(p, stage_time(w, stage2), G);
        double gdot = 0.0, un = 0.0;
        for (int k = 0; k < p.dim; ++k) {
          gdot += G[k] * (s.x[k * n + i] - s.x[k * n + best]);
          un += s.u[k * n + best] * s.normal[k * n + i];
        }
        s.phi[i] = s.phi[best] + gdot;
        for (int k = 0; k < p.dim; ++k)
          s.u[k * n + i] = s.u[k * n + best] - un * s.normal[k * n + i];
      }
    } else {
      for (int k = 0; k < p.dim; ++k) umax2 += s.u[k * n + i] * s.u[k * n + i];
    }
    double v = s.mass[i] / eos_density(p, s.phi[i]);
    w.vol[i] = v;
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

void launch_prepass(const Params& p, const State& s, const Work& w, int64_t n, int stage2,
                    cudaStream_t st) {
  cudaMemsetAsync(w.umax_bits, 0, sizeof(unsigned long long), st);
  if (n == 0) return;
  k_prepass<<<(unsigned)div_up(n, PRE_THREADS), PRE_THREADS, 0, st>>>(p, s, w, n, stage2);
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
// Closed-form smallest eigenvalue of the symmetric renormalisation matrix
// (Sec. 3). 2D: mean - sqrt(half-difference^2 + off^2). 3D: trigonometric
// root of the characteristic cubic (Smith, CACM 1961).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double lambda_min_2(double a, double b, double c) {
  double m = 0.5 * (a + c), d = 0.5 * (a - c);
  return m - sqrt(d * d + b * b);
}

__device__ __forceinline__ double lambda_min_3(double a00, double a01, double a02, double a11,
                                               double a12, double a22) {
  double off = a01 * a01 + a02 * a02 + a12 * a12;
  if (off == 0.0) return fmin(fmin(a00, a11), a22);
  double mean = (a00 + a11 + a22) * (1.0 / 3.0);
  double b00 = a00 - mean, b11 = a11 - mean, b22 = a22 - mean;
  double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * off;
  double pp = sqrt(p2 * (1.0 / 6.0));
  double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
               a02 * (a01 * a12 - b11 * a02);
  double r = det / (2.0 * pp * pp * pp);
  r = fmin(1.0, fmax(-1.0, r));
  double ang = acos(r) * (1.0 / 3.0);
  return mean + 2.0 * pp * cos(ang + 2.0943951023931954923);  // 2 pi / 3
}

// Reciprocal square root: FP32 estimate refined by two Newton-Raphson steps
// y <- y (3 - r2 y^2) / 2 in FP64 (each step roughly doubles the correct
// bits: ~23 -> ~46 -> full double precision).
__device__ __forceinline__ double rsqrt_nr(double r2) {
  double y = (double)rsqrtf((float)r2);
  double hy = 0.5 * y;
  y = fma(hy, fma(-r2 * y, y, 1.0), y);
  hy = 0.5 * y;
  y = fma(hy, fma(-r2 * y, y, 1.0), y);
  return y;
}

// ---------------------------------------------------------------------------
// Fused pair pass over fluid particles (one lane per particle i).
// Accumulated with g = -W'(r)/r V_j >= 0, so grad_i W_ij V_j = g r (r = x_j - x_i):
//   L  += r (x) g r                       (Eq. renorm; symmetric)
//   S  += [phi_j - phi_i - C0 (U_j - U_i).r/|r|] g r      (2(phi* - phi_i), Eq. lfsover)
//   M  += (U_j - U_i) (x) g r             (continuity, corrected in the epilogue)
//   C  += (phi_i + phi_j) g r             (conservative gradient, TIC branch)
//   D  += (phi_j - phi_i) g               (delta-SPH: (x_j-x_i).grad W/|r|^2 V_j = g)
//   Lam+= (U_j - U_i) g, fluid j only     (Laplacian operator, Sec. 2.1/2.4)
//   P  += [1 + R (W_ij / W(dx))^n] g r    (shifting)
// ---------------------------------------------------------------------------
template <int DIM>
struct PairAcc {
  double L[6], S[DIM], M[DIM * DIM], C[DIM], D, Lam[DIM], P[DIM];
};

constexpr int PAIR_THREADS = 128;

template <int DIM>
__host__ __device__ constexpr int pair_kcap() { return DIM == 3 ? 96 : 40; }

template <int DIM>
__global__ void __launch_bounds__(PAIR_THREADS, 3)
    k_pair_fp64(Params p, State s, Work w, int64_t n, int64_t nf, int stage2) {
  constexpr int KCAP = pair_kcap<DIM>();
  extern __shared__ uint32_t lists[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* my = lists + warp * KCAP * 32;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;

  double xi[DIM], ui[DIM], phii = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    xi[k] = active ? s.x[k * n + i] : 0.0;
    ui[k] = active ? s.u[k * n + i] : 0.0;
  }
  if (active) phii = s.phi[i];

  PairAcc<DIM> a;
#pragma unroll
  for (int k = 0; k < 6; ++k) a.L[k] = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) { a.S[k] = a.C[k] = a.Lam[k] = a.P[k] = 0.0; }
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) a.M[k] = 0.0;
  a.D = 0.0;

  const bool pst4 = p.use_pst && p.pst_n == 4.0;
  unsigned npairs = 0;
  CandidateIter it;
  bool done = !active;
  if (active) it.init(p, w, n, i);

  while (__any_sync(0xffffffffu, !done)) {
    // (A) candidate enumeration, FP32 prefilter, compact list
    int cnt = 0;
    while (!done && cnt < KCAP) {
      uint32_t j;
      if (it.next(p, w, j)) my[cnt++ * 32 + lane] = j;
      else done = true;
    }
    __syncwarp();
    int maxc = __reduce_max_sync(0xffffffffu, cnt);
    // (B) FP64 pair terms
    for (int k = 0; k < maxc; ++k) {
      if (k >= cnt) continue;
      uint32_t j = my[k * 32 + lane];
      double r[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) r[c] = __dsub_rn(s.x[c * n + j], xi[c]);
      double r2 = __dmul_rn(r[0], r[0]);
#pragma unroll
      for (int c = 1; c < DIM; ++c) r2 = __dadd_rn(r2, __dmul_rn(r[c], r[c]));
      if (!(r2 <= p.four_h2 && r2 > 0.0)) continue;
      ++npairs;
      double inv_r = rsqrt_nr(r2);
      double rr = r2 * inv_r;
      double t = fma(-rr, p.inv_two_h, 1.0);
      double t3 = t * t * t;
      double g = p.neg_dwdr_over_r_coef * t3 * w.vol[j];
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
      // L (upper triangle, row-major order 00 01 [02] 11 [12 22])
      if (DIM == 2) {
        a.L[0] = fma(r[0], gr[0], a.L[0]);
        a.L[1] = fma(r[0], gr[1], a.L[1]);
        a.L[2] = fma(r[1], gr[1], a.L[2]);
      } else {
        a.L[0] = fma(r[0], gr[0], a.L[0]);
        a.L[1] = fma(r[0], gr[1], a.L[1]);
        a.L[2] = fma(r[0], gr[2], a.L[2]);
        a.L[3] = fma(r[1], gr[1], a.L[3]);
        a.L[4] = fma(r[1], gr[2], a.L[4]);
        a.L[5] = fma(r[2], gr[2], a.L[5]);
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        a.S[c] = fma(rs, gr[c], a.S[c]);
        a.C[c] = fma(sphi, gr[c], a.C[c]);
#pragma unroll
        for (int e = 0; e < DIM; ++e) a.M[c * DIM + e] = fma(du[c], gr[e], a.M[c * DIM + e]);
      }
      a.D = fma(dphi, g, a.D);
      if (s.type[j] == kFluid) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) a.Lam[c] = fma(du[c], g, a.Lam[c]);
      }
      if (p.use_pst) {
        double q21 = fma(rr, p.two_over_h, 1.0);           // 2q + 1
        double ratio = p.pst_alpha_over_wdx * (t3 * t) * q21;  // W_ij / W(dx)
        double rn = pst4 ? (ratio * ratio) * (ratio * ratio) : pow(ratio, p.pst_n);
        double f = fma(p.pst_R, rn, 1.0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) a.P[c] = fma(f, gr[c], a.P[c]);
      }
    }
    __syncwarp();
  }
  unsigned wp = __reduce_add_sync(0xffffffffu, npairs);
  if (lane == 0 && wp) atomicAdd(w.pairs, (unsigned long long)wp);
  if (!active) return;

  // ---- epilogue (Eq. sph with the TIC switch, K8/K9 of Sec. 3) ----
  double Lf[3][3];
  if (DIM == 2) {
    Lf[0][0] = a.L[0]; Lf[0][1] = Lf[1][0] = a.L[1]; Lf[1][1] = a.L[2];
  } else {
    Lf[0][0] = a.L[0]; Lf[0][1] = Lf[1][0] = a.L[1]; Lf[0][2] = Lf[2][0] = a.L[2];
    Lf[1][1] = a.L[3]; Lf[1][2] = Lf[2][1] = a.L[4]; Lf[2][2] = a.L[5];
  }
  double lam = DIM == 2 ? lambda_min_2(Lf[0][0], Lf[0][1], Lf[1][1])
                        : lambda_min_3(Lf[0][0], Lf[0][1], Lf[0][2], Lf[1][1], Lf[1][2], Lf[2][2]);
  double gradphi[DIM], divu = 0.0;
  if (p.use_tic && lam < p.tic_lambda) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      gradphi[c] = a.C[c];
      divu += a.M[c * DIM + c];
    }
  } else {
    double inv[DIM][DIM], det, amax = 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int e = 0; e < DIM; ++e) amax = fmax(amax, fabs(Lf[c][e]));
    if (DIM == 2) {
      det = Lf[0][0] * Lf[1][1] - Lf[0][1] * Lf[1][0];
      double id = 1.0 / det;
      inv[0][0] = Lf[1][1] * id; inv[1][1] = Lf[0][0] * id;
      inv[0][1] = -Lf[0][1] * id; inv[1][0] = -Lf[1][0] * id;
    } else {
      double c00 = Lf[1][1] * Lf[2][2] - Lf[1][2] * Lf[2][1];
      double c01 = Lf[1][2] * Lf[2][0] - Lf[1][0] * Lf[2][2];
      double c02 = Lf[1][0] * Lf[2][1] - Lf[1][1] * Lf[2][0];
      det = Lf[0][0] * c00 + Lf[0][1] * c01 + Lf[0][2] * c02;
      double id = 1.0 / det;
      double m[3][3];
      m[0][0] = c00; m[1][0] = c01; m[2][0] = c02;
      m[0][1] = Lf[0][2] * Lf[2][1] - Lf[0][1] * Lf[2][2];
      m[1][1] = Lf[0][0] * Lf[2][2] - Lf[0][2] * Lf[2][0];
      m[2][1] = Lf[0][1] * Lf[2][0] - Lf[0][0] * Lf[2][1];
      m[0][2] = Lf[0][1] * Lf[1][2] - Lf[0][2] * Lf[1][1];
      m[1][2] = Lf[0][2] * Lf[1][0] - Lf[0][0] * Lf[1][2];
      m[2][2] = Lf[0][0] * Lf[1][1] - Lf[0][1] * Lf[1][0];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int e = 0; e < 3; ++e) inv[c][e] = m[c][e] * id;
    }
    double amd = DIM == 2 ? amax * amax : amax * amax * amax;
    if (!(fabs(det) > 1e-12 * amd)) {
      atomicOr(w.status, kStatSingular);
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int e = 0; e < DIM; ++e) inv[c][e] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double gsum = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        gsum = fma(inv[c][e], a.S[e], gsum);
        divu = fma(inv[c][e], a.M[c * DIM + e], divu);
      }
      gradphi[c] = gsum;
    }
  }
  double G[3];
  body_force(p, stage_time(w, stage2), G);
  double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
  bool bad = false;
  double dstar[DIM], dn2 = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double visc = p.use_visc ? 2.0 * p.nu * a.Lam[c] : 0.0;
    double acc = -gradphi[c] + visc + G[c];
    w.dudt[c * n + i] = acc;
    bad |= !isfinite(acc);
    dstar[c] = -2.0 * p.h * umax * a.P[c];
    dn2 += dstar[c] * dstar[c];
  }
  double diff = p.use_delta ? p.delta_h_c0 * (2.0 * a.D) : 0.0;
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
  w.lambda[i] = lam;
  if (bad) atomicOr(w.status, kStatNaN);
}

void launch_pair_fp64(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                      int stage2, cudaStream_t st) {
  if (nf == 0) return;
  unsigned blocks = (unsigned)div_up(nf, PAIR_THREADS);
  if (p.dim == 2) {
    size_t sm = (size_t)pair_kcap<2>() * 32 * (PAIR_THREADS / 32) * sizeof(uint32_t);
    k_pair_fp64<2><<<blocks, PAIR_THREADS, sm, st>>>(p, s, w, n, nf, stage2);
  } else {
    size_t sm = (size_t)pair_kcap<3>() * 32 * (PAIR_THREADS / 32) * sizeof(uint32_t);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_pair_fp64<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    k_pair_fp64<3><<<blocks, PAIR_THREADS, sm, st>>>(p, s, w, n, nf, stage2);
  }
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
