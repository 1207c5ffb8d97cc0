// pair_fp64.cu -- the fused FP64 pair pass of the well-balanced WCSPH step
// and its epilogue (Eq. sph with TIC, viscosity, delta-SPH and shifting),
// and lambda_min of the stored renormalisation matrices.
//
// On GB300 the FP64 pipe (2 DFMA per clock per SM, 1/61 of FP32) bounds this
// path. Candidate enumeration of the 3^d cells is therefore done by a
// separate FP32/integer kernel that writes each fluid particle's neighbour
// list (k-major, coalesced; lists.cu); the FP64 kernel then walks these
// lists with every lane busy and no shared memory, so more warps per SM
// cover the latency of the gathers and of the FP64 pipe itself.
#include "common.cuh"
#include "physics.cuh"

namespace wbsph {
// ---------------------------------------------------------------------------
// Fused FP64 pair pass over fluid particles (one lane per particle i).
// Accumulated with g = -W'(r)/r V_j >= 0, so grad_i W_ij V_j = g r (r = x_j - x_i):
//   L  += r (x) g r                       (Eq. renorm; symmetric)
//   S  += [phi_j - phi_i - C0 (U_j - U_i).r/|r|] g r      (2(phi* - phi_i), Eq. lfsover)
//   M  += (U_j - U_i) (x) g r             (continuity, corrected in the epilogue)
//   C  += (phi_i + phi_j) g r             (conservative gradient, TIC branch)
//   D  += (phi_j - phi_i) g               (delta-SPH: (x_j-x_i).grad W/|r|^2 V_j = g)
//   Lam+= (U_j - U_i) g, fluid j only     (Laplacian operator, Sec. 2.1/2.4;
//                                          every j with no-slip walls)
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
    if (p.wall_bc || s.type[j] == kFluid) {
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

void launch_pair_fp64(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                      int stage2, cudaStream_t st) {
  if (nf == 0) return;
  unsigned blocks = (unsigned)div_up(nf, PAIR_THREADS);
  if (p.dim == 2) k_pair_fp64<2><<<blocks, PAIR_THREADS, 0, st>>>(p, s, w, n, nf, stage2);
  else k_pair_fp64<3><<<blocks, PAIR_THREADS, 0, st>>>(p, s, w, n, nf, stage2);
}

}  // namespace wbsph
