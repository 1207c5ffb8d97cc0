// pair_conventional.cu -- conventional WCSPH (Sec. 2.1: Eq. nslag with the
// printed operators <div U>, <grad p>, <lap U>, and the EOS), with
// artificial viscosity: the foil of the hydrostatic comparison (Sec. 4.1),
// which unlike the well-balanced scheme does not hold a tank at rest.
//
// The state stays (x, U, phi) with rho and p from the EOS (written per
// particle by the prepass); since d(phi) = c^2 d(rho)/rho, the conventional
// continuity equation Drho/Dt = -rho div U is Dphi/Dt = -c^2 div U. Per
// fluid particle i over its exact neighbour list, with
// g = -W'(r)/r V_j >= 0 so that grad_i W_ij V_j = g r (r = x_j - x_i):
//   DU/Dt   = -(1/rho_i) sum (p_i + p_j) g r + 2 nu Lambda + G(t) - sum rho_j Pi_ij g r
//   Dphi/Dt = -c^2 sum (U_j - U_i).r g
//   Pi_ij   = -alpha h C0 (U_ij.x_ij) / (rho_ij (r^2 + 0.01 h^2)) when U_ij.x_ij < 0,
//             else 0; U_ij.x_ij = (U_j - U_i).r, rho_ij = (rho_i + rho_j)/2
//   Lambda  = sum over fluid j of (U_j - U_i) g
// It runs only on small validation scenes, so it is written for clarity
// (IEEE square root and division), not for the FP64 pipe.
#include "common.cuh"
#include "physics.cuh"

namespace wbsph {

template <int DIM>
__global__ void __launch_bounds__(128) k_pair_conventional(Params p, State s, Work w, int64_t n, int64_t nf,
                                                           int stage2) {
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= nf) return;
  const uint32_t i = w.fluid_list[gi];
  const int cnt = (int)w.nbr_cnt[gi];
  double xi[DIM], ui[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    xi[c] = s.x[c * n + i];
    ui[c] = s.u[c * n + i];
  }
  const double rho_i = w.rho[i], p_i = w.pres[i];
  double gp[DIM], lam[DIM], av[DIM], divu = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) gp[c] = lam[c] = av[c] = 0.0;
  for (int k = 0; k < cnt; ++k) {
    const uint32_t j = w.nbr[(int64_t)k * nf + gi];  // exact neighbours (k_nbr_list)
    double r[DIM], du[DIM], r2 = 0.0, dun = 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      r[c] = s.x[c * n + j] - xi[c];
      du[c] = s.u[c * n + j] - ui[c];
      r2 += r[c] * r[c];
      dun += du[c] * r[c];
    }
    const double rr = sqrt(r2);
    const double t = 1.0 - rr * p.inv_two_h;
    const double g = t * t * t * w.volc[j];
    const double pp = p_i + w.pres[j];
    double pij = 0.0;
    if (dun < 0.0) pij = -p.art_ahc0 * dun / (0.5 * (rho_i + w.rho[j]) * (r2 + p.avis_eps2));
    const double rho_j = w.rho[j];
    const bool fluid_j = p.wall_bc || s.type[j] == kFluid;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      gp[c] += pp * g * r[c];
      av[c] += rho_j * pij * g * r[c];
      if (fluid_j) lam[c] += du[c] * g;
    }
    divu += g * dun;
  }
  const double fs = forcing_factor(p, stage_time(w, stage2));
  bool bad = false;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const double visc = p.use_visc ? 2.0 * p.nu * lam[c] : 0.0;
    const double acc = -gp[c] / rho_i + visc + (p.g[c] + p.force_amp[c] * fs) - av[c];
    w.dudt[c * n + i] = acc;
    w.dushift[c * n + i] = 0.0;
    bad |= !isfinite(acc);
  }
  const double dphidt = -eos_c2(p, s.phi[i]) * divu;
  w.dphidt[i] = dphidt;
  bad |= !isfinite(dphidt);
#pragma unroll
  for (int k = 0; k < (DIM == 2 ? 3 : 6); ++k) w.Lmat[k * n + i] = 0.0;  // no renormalisation matrix
  if (bad) atomicOr(w.status, kStatNaN);
}

void launch_pair_conventional(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                              int stage2, cudaStream_t st) {
  if (nf == 0) return;
  const unsigned blocks = (unsigned)div_up(nf, 128);
  if (p.dim == 2) k_pair_conventional<2><<<blocks, 128, 0, st>>>(p, s, w, n, nf, stage2);
  else k_pair_conventional<3><<<blocks, 128, 0, st>>>(p, s, w, n, nf, stage2);
}

}  // namespace wbsph
