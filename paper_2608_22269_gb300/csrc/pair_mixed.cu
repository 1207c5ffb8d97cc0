// pair_mixed.cu -- mixed-precision pair pass: cell-relative FP32 coordinates,
// FP32 pair sums with Kahan-compensated accumulation, FP64 epilogue.
//
// Hydrostatic split (well-balance by construction): with
// phi = phi_hs(x) + phi', phi_hs(x) = G.x + |G| H (Eq. eqSol with the free
// surface at phi = 0), every pair difference is phi_j - phi_i =
// (phi'_j - phi'_i) + G.(x_j - x_i), and because L is symmetric,
//   L^-1 sum (G.r) grad W V = L^-1 L G = G   exactly.
// So the corrected gradient is grad phi = L^-1 S' + G, where S' is the
// Riemann sum (Eqs. parGrad, lfsover) of phi' alone, and
//   DU/Dt = -L^-1 S' + 2 nu Lambda + (G(t) - G),
// with the -G + G cancellation taken analytically in FP64. At rest phi' = 0
// up to the rounding of phi_hs, so no FP32 rounding of the large hydrostatic
// differences enters the momentum balance. The conservative (TIC) and
// delta-SPH sums are rebuilt from phi' sums in FP64:
//   C = C' + 2 phi_hs,i K + L G,   D = D' + G.K,   K = sum grad W V.
// The state (x, U, phi) stays FP64; only the pair sums run in FP32.
#include "../../include/wbsph.h"
#include "common.cuh"

namespace wbsph {

// ---- helpers (FP64 epilogue) ----
__device__ __forceinline__ double mx_lambda_min_2(double a, double b, double c) {
  double m = 0.5 * (a + c), d = 0.5 * (a - c);
  return m - sqrt(d * d + b * b);
}

__device__ __forceinline__ double mx_lambda_min_3(double a00, double a01, double a02, double a11,
                                                  double a12, double a22) {
  double off = a01 * a01 + a02 * a02 + a12 * a12;
  if (off == 0.0) return fmin(fmin(a00, a11), a22);
  double mean = (a00 + a11 + a22) * (1.0 / 3.0);
  double b00 = a00 - mean, b11 = a11 - mean, b22 = a22 - mean;
  double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * off;
  double pp = sqrt(p2 * (1.0 / 6.0));
  double det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
               a02 * (a01 * a12 - b11 * a02);
  double r = fmin(1.0, fmax(-1.0, det / (2.0 * pp * pp * pp)));
  return mean + 2.0 * pp * cos(acos(r) * (1.0 / 3.0) + 2.0943951023931954923);
}

// Kahan-compensated FP32 accumulator: s + (-c) carries the running sum.
struct Kahan {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ---- pack: cell-relative FP32 offsets, phi', U, signed V ----
// A[i] = (x - cell origin, phi - phi_hs(x)), B[i] = (U, V) with V < 0 marking
// dummy particles (the Laplacian operator takes fluid neighbours only).
__global__ void k_pack_mixed(Params p, State s, Work w, int64_t n, float4* A, float4* B) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t key = w.key[i];
  uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
  uint32_t ic[3] = {key % nx, (key / nx) % ny, key / (nx * ny)};
  float o[3] = {0.f, 0.f, 0.f};
  float u[3] = {0.f, 0.f, 0.f};
  double phs = 0.0, gn2 = 0.0;
  for (int k = 0; k < p.dim; ++k) {
    double xk = s.x[k * n + i];
    o[k] = (float)(xk - (p.domain_min[k] + (double)ic[k] * p.R));
    u[k] = (float)s.u[k * n + i];
    phs += p.g[k] * xk;
    gn2 += p.g[k] * p.g[k];
  }
  phs += sqrt(gn2) * p.water_height;
  float phip = (float)(s.phi[i] - phs);
  float v = (float)w.vol[i];
  if (s.type[i] != kFluid) v = -v;
  A[i] = make_float4(o[0], o[1], o[2], phip);
  B[i] = make_float4(u[0], u[1], u[2], v);
}

constexpr int MX_THREADS = 128;

template <int DIM>
__host__ __device__ constexpr int mx_kcap() { return DIM == 3 ? 96 : 40; }

template <int DIM>
__global__ void __launch_bounds__(MX_THREADS, 3)
    k_pair_mixed(Params p, State s, Work w, int64_t n, int64_t nf, int stage2, const float4* __restrict__ A,
                 const float4* __restrict__ B) {
  constexpr int KCAP = mx_kcap<DIM>();
  extern __shared__ uint32_t lists[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* my = lists + warp * KCAP * 32;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;
  const float R = (float)p.R;
  const float four_h2 = (float)p.four_h2;
  const float inv_two_h = (float)p.inv_two_h;
  const float two_over_h = (float)p.two_over_h;
  const float coef = (float)p.neg_dwdr_over_r_coef;
  const float c0 = (float)p.c0;
  const float pst_a = (float)p.pst_alpha_over_wdx;
  const float pst_R = (float)p.pst_R;

  float4 Ai = make_float4(0.f, 0.f, 0.f, 0.f), Bi = Ai;
  int ix = 0, iy = 0, iz = 0;
  if (active) {
    Ai = A[i];
    Bi = B[i];
    uint32_t key = w.key[i];
    uint32_t nx = (uint32_t)p.nc[0], ny = (uint32_t)p.nc[1];
    ix = (int)(key % nx);
    iy = (int)((key / nx) % ny);
    iz = (int)(key / (nx * ny));
  }
  Kahan L[6], S[DIM], M[DIM * DIM], Cc[DIM], K[DIM], D, Lam[DIM], P[DIM];
#pragma unroll
  for (int k = 0; k < 6; ++k) L[k].zero();
#pragma unroll
  for (int k = 0; k < DIM; ++k) { S[k].zero(); Cc[k].zero(); K[k].zero(); Lam[k].zero(); P[k].zero(); }
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) M[k].zero();
  D.zero();

  // row iterator state (phase A)
  const int nrows = DIM == 3 ? 9 : 3;
  int row = active ? 0 : nrows;
  uint32_t cur = 0, end = 0, b0 = 0, b1 = 0;
  int oy = 0, oz = 0;
  bool have_row = false;
  unsigned npairs = 0;

  while (__any_sync(0xffffffffu, row < nrows || have_row)) {
    int cnt = 0;
    // (A) candidates of the 3^d cells: FP32 cell-relative distance test
    while (cnt < KCAP && (row < nrows || have_row)) {
      if (!have_row) {
        oy = row % 3 - 1;
        oz = DIM == 3 ? row / 3 - 1 : 0;
        ++row;
        int cy = iy + oy, cz = iz + oz;
        if (cy < 0 || cy >= p.nc[1] || cz < 0 || cz >= p.nc[2]) continue;
        int x0 = ix > 0 ? ix - 1 : 0;
        int x1 = ix + 1 < p.nc[0] ? ix + 1 : p.nc[0] - 1;
        int64_t base = (int64_t)cy * p.nc[0] + (int64_t)cz * p.nc[0] * p.nc[1];
        cur = w.cell_lb[base + x0];
        end = w.cell_lb[base + x1 + 1];
        b0 = w.cell_lb[base + ix];
        b1 = w.cell_lb[base + ix + 1];
        have_row = cur < end;
        continue;
      }
      uint32_t j = cur++;
      if (cur >= end) have_row = false;
      if (j == i) continue;
      int dcx = (j >= b0) + (j >= b1) - 1;
      float4 Aj = A[j];
      float rx = fmaf((float)dcx, R, Aj.x - Ai.x);
      float ry = fmaf((float)oy, R, Aj.y - Ai.y);
      float r2 = rx * rx + ry * ry;
      if (DIM == 3) {
        float rz = fmaf((float)oz, R, Aj.z - Ai.z);
        r2 += rz * rz;
      }
      if (r2 <= four_h2 && r2 > 0.f) {
        uint32_t code = (uint32_t)((dcx + 1) + 3 * (oy + 1) + 9 * (oz + 1));
        my[cnt++ * 32 + lane] = (j << 5) | code;
      }
    }
    __syncwarp();
    int maxc = __reduce_max_sync(0xffffffffu, cnt);
    // (B) FP32 pair terms with compensated sums
    for (int k = 0; k < maxc; ++k) {
      if (k >= cnt) continue;
      uint32_t e = my[k * 32 + lane];
      uint32_t j = e >> 5, code = e & 31u;
      int dc[3] = {(int)(code % 3) - 1, (int)((code / 3) % 3) - 1, (int)(code / 9) - 1};
      float4 Aj = A[j], Bj = B[j];
      float r[DIM], du[DIM];
      r[0] = fmaf((float)dc[0], R, Aj.x - Ai.x);
      r[1] = fmaf((float)dc[1], R, Aj.y - Ai.y);
      if (DIM == 3) r[DIM - 1] = fmaf((float)dc[2], R, Aj.z - Ai.z);
      du[0] = Bj.x - Bi.x;
      du[1] = Bj.y - Bi.y;
      if (DIM == 3) du[DIM - 1] = Bj.z - Bi.z;
      float r2 = 0.f, dun = 0.f;
#pragma unroll
      for (int c = 0; c < DIM; ++c) { r2 = fmaf(r[c], r[c], r2); dun = fmaf(du[c], r[c], dun); }
      ++npairs;
      float inv_r = rsqrtf(r2);
      float rr = r2 * inv_r;
      float t = fmaf(-rr, inv_two_h, 1.f);
      float t3 = t * t * t;
      float vj = fabsf(Bj.w);
      float g = coef * t3 * vj;
      dun *= inv_r;
      float dphi = Aj.w - Ai.w, sphi = Aj.w + Ai.w;
      float rs = fmaf(-c0, dun, dphi);
      float gr[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) gr[c] = g * r[c];
      if (DIM == 2) {
        L[0].add(r[0] * gr[0]); L[1].add(r[0] * gr[1]); L[2].add(r[1] * gr[1]);
      } else {
        L[0].add(r[0] * gr[0]); L[1].add(r[0] * gr[1]); L[2].add(r[0] * gr[DIM - 1]);
        L[3].add(r[1] * gr[1]); L[4].add(r[1] * gr[DIM - 1]); L[5].add(r[DIM - 1] * gr[DIM - 1]);
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        S[c].add(rs * gr[c]);
        Cc[c].add(sphi * gr[c]);
        K[c].add(gr[c]);
#pragma unroll
        for (int d2 = 0; d2 < DIM; ++d2) M[c * DIM + d2].add(du[c] * gr[d2]);
      }
      D.add(dphi * g);
      if (Bj.w > 0.f) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) Lam[c].add(du[c] * g);
      }
      if (p.use_pst) {
        float q21 = fmaf(rr, two_over_h, 1.f);
        float ratio = pst_a * (t3 * t) * q21;
        float r4 = (ratio * ratio) * (ratio * ratio);
        float f = fmaf(pst_R, r4, 1.f);
#pragma unroll
        for (int c = 0; c < DIM; ++c) P[c].add(f * gr[c]);
      }
    }
    __syncwarp();
  }
  unsigned wp = __reduce_add_sync(0xffffffffu, npairs);
  if (lane == 0 && wp) atomicAdd(w.pairs, (unsigned long long)wp);
  if (!active) return;

  // ---- FP64 epilogue ----
  double Lf[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (DIM == 2) {
    Lf[0][0] = L[0].value(); Lf[0][1] = Lf[1][0] = L[1].value(); Lf[1][1] = L[2].value();
  } else {
    Lf[0][0] = L[0].value(); Lf[0][1] = Lf[1][0] = L[1].value(); Lf[0][2] = Lf[2][0] = L[2].value();
    Lf[1][1] = L[3].value(); Lf[1][2] = Lf[2][1] = L[4].value(); Lf[2][2] = L[5].value();
  }
  double Sd[DIM], Md[DIM * DIM], Cd[DIM], Kd[DIM], Ld[DIM], Pd[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    Sd[c] = S[c].value(); Cd[c] = Cc[c].value(); Kd[c] = K[c].value();
    Ld[c] = Lam[c].value(); Pd[c] = P[c].value();
  }
#pragma unroll
  for (int c = 0; c < DIM * DIM; ++c) Md[c] = M[c].value();
  double lam = DIM == 2 ? mx_lambda_min_2(Lf[0][0], Lf[0][1], Lf[1][1])
                        : mx_lambda_min_3(Lf[0][0], Lf[0][1], Lf[0][2], Lf[1][1], Lf[1][2], Lf[2][2]);
  double t_stage = stage2 ? w.scalars[0] + w.scalars[1] : w.scalars[0];
  double fs = p.omega > 0.0 ? p.omega * p.omega * sin(p.omega * t_stage) : 0.0;
  double xi[DIM], phs = 0.0, gn2 = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    xi[c] = s.x[c * n + i];
    phs += p.g[c] * xi[c];
    gn2 += p.g[c] * p.g[c];
  }
  phs += sqrt(gn2) * p.water_height;
  double acc[DIM], divu = 0.0;
  if (p.use_tic && lam < p.tic_lambda) {
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double lg = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) lg += Lf[c][e] * p.g[e];
      double gradphi = Cd[c] + 2.0 * phs * Kd[c] + lg;
      acc[c] = -gradphi + p.g[c] + p.force_amp[c] * fs;
      divu += Md[c * DIM + c];
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
      inv[0][0] = Lf[1][1] * id; inv[DIM - 1][DIM - 1] = Lf[0][0] * id;
      inv[0][DIM - 1] = -Lf[0][1] * id; inv[DIM - 1][0] = -Lf[1][0] * id;
    } else {
      double m[3][3];
      m[0][0] = Lf[1][1] * Lf[2][2] - Lf[1][2] * Lf[2][1];
      m[1][0] = Lf[1][2] * Lf[2][0] - Lf[1][0] * Lf[2][2];
      m[2][0] = Lf[1][0] * Lf[2][1] - Lf[1][1] * Lf[2][0];
      det = Lf[0][0] * m[0][0] + Lf[0][1] * m[1][0] + Lf[0][2] * m[2][0];
      m[0][1] = Lf[0][2] * Lf[2][1] - Lf[0][1] * Lf[2][2];
      m[1][1] = Lf[0][0] * Lf[2][2] - Lf[0][2] * Lf[2][0];
      m[2][1] = Lf[0][1] * Lf[2][0] - Lf[0][0] * Lf[2][1];
      m[0][2] = Lf[0][1] * Lf[1][2] - Lf[0][2] * Lf[1][1];
      m[1][2] = Lf[0][2] * Lf[1][0] - Lf[0][0] * Lf[1][2];
      m[2][2] = Lf[0][0] * Lf[1][1] - Lf[0][1] * Lf[1][0];
      double id = 1.0 / det;
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int e = 0; e < DIM; ++e) inv[c][e] = m[c][e] * id;
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
      double gs = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        gs = fma(inv[c][e], Sd[e], gs);
        divu = fma(inv[c][e], Md[c * DIM + e], divu);
      }
      acc[c] = -gs + p.force_amp[c] * fs;   // -(L^-1 S' + G) + G(t)
    }
  }
  double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
  double phii = s.phi[i];
  bool bad = false;
  double dstar[DIM], dn2 = 0.0, gk = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double a = acc[c] + (p.use_visc ? 2.0 * p.nu * Ld[c] : 0.0);
    w.dudt[c * n + i] = a;
    bad |= !isfinite(a);
    dstar[c] = -2.0 * p.h * umax * Pd[c];
    dn2 += dstar[c] * dstar[c];
    gk += p.g[c] * Kd[c];
  }
  double c2 = p.eos == 0 ? p.c0sq : p.c0sq + (p.gamma - 1.0) * phii;
  double diff = p.use_delta ? p.delta_h_c0 * 2.0 * (D.value() + gk) : 0.0;
  double dphidt = -c2 * divu + diff;
  w.dphidt[i] = dphidt;
  bad |= !isfinite(dphidt);
  double dn = sqrt(dn2);
  double scale = (p.use_pst && dn > 0.0) ? fmin(dn, 0.5 * umax) / dn : 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double v = dstar[c] * scale;
    w.dushift[c * n + i] = v;
    bad |= !isfinite(v);
  }
  w.lambda[i] = lam;
  if (bad) atomicOr(w.status, kStatNaN);
}

int launch_mixed_stage(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                       int stage2, cudaStream_t st) {
  if (n == 0) return 0;
  if (n >= ((int64_t)1 << 27)) return WBSPH_E_INVAL;  // list entries pack the index in 27 bits
  k_pack_mixed<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p, s, w, n, w.packA, w.packB);
  if (nf == 0) return 0;
  unsigned blocks = (unsigned)div_up(nf, MX_THREADS);
  if (p.dim == 2) {
    size_t sm = (size_t)mx_kcap<2>() * 32 * (MX_THREADS / 32) * sizeof(uint32_t);
    k_pair_mixed<2><<<blocks, MX_THREADS, sm, st>>>(p, s, w, n, nf, stage2, w.packA, w.packB);
  } else {
    size_t sm = (size_t)mx_kcap<3>() * 32 * (MX_THREADS / 32) * sizeof(uint32_t);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_pair_mixed<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      attr = true;
    }
    k_pair_mixed<3><<<blocks, MX_THREADS, sm, st>>>(p, s, w, n, nf, stage2, w.packA, w.packB);
  }
  return 0;
}

}  // namespace wbsph
