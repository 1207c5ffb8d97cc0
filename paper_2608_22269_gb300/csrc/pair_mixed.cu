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
#include <type_traits>

#include "../../include/wbsph.h"
#include "common.cuh"
#include "physics.cuh"

namespace wbsph {

// Kahan-compensated FP32 accumulator: s + (-c) carries the running sum.
// The terms of list entries 2m and 2m + 1 enter as one compensated step:
// defer() parks the first in the compensation (one subtraction), add()
// folds it in with the second (y = v - c takes both), so the compensated
// update costs 2.5 operations per term instead of 4. The parked term adds
// one FP32 rounding of its own magnitude per pair of terms, where plain
// Kahan has none; the compensation of the running sum is unchanged.
struct Kahan {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ void defer(float v) { c -= v; }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <bool FULL>
__device__ __forceinline__ void kacc(Kahan& a, float v) {
  if constexpr (FULL) a.add(v);
  else a.defer(v);
}

constexpr int MX_THREADS = 128;
#ifndef WBSPH_MX_MIN_BLOCKS
#define WBSPH_MX_MIN_BLOCKS 4  // resident blocks per SM the register budget is sized for
#endif
#ifndef WBSPH_MX_RING
#define WBSPH_MX_RING 4  // list entries of each lane in flight (shared-memory ring)
#endif
constexpr int MX_RING = WBSPH_MX_RING;

// Asynchronous global -> shared copies (cp.async, cached in L1), one group
// per list entry; a thread waits only for its own groups.
__device__ __forceinline__ void mx_cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void mx_cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void mx_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void mx_wait_ring() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(MX_RING - 1) : "memory");
}

// Pair sums over the candidate lists built by k_nbr_list (the same lists as
// the FP64 pass); the neighbour test is the FP32 cell-relative distance.
template <int DIM>
__global__ void __launch_bounds__(MX_THREADS, WBSPH_MX_MIN_BLOCKS)
    k_pair_mixed(Params p, State s, Work w, int64_t n, int64_t nf, int stage2, const float4* __restrict__ A,
                 const float4* __restrict__ B, const uint32_t* __restrict__ Cc) {
  const int lane = threadIdx.x & 31;
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;
  const int cnt = active ? (int)w.nbr_cnt[gi] : 0;
  const float R = (float)p.R;
  const float four_h2 = (float)p.four_h2;
  const float inv_two_h = (float)p.inv_two_h;
  const float two_over_h = (float)p.two_over_h;
  const float coef = (float)p.neg_dwdr_over_r_coef;
  const float c0 = (float)p.c0;
  const float pst_a = (float)p.pst_alpha_over_wdx;
  const float pst_R = (float)p.pst_R;

  float4 Ai = make_float4(0.f, 0.f, 0.f, 0.f), Bi = Ai;
  uint32_t ci = 0;
  if (active) { Ai = A[i]; Bi = B[i]; ci = Cc[i]; }
  const int cix = (int)(ci & 2047u), ciy = (int)((ci >> 11) & 2047u), ciz = (int)(ci >> 22);
  Kahan L[6], S[DIM], M[DIM * DIM], Cs[DIM], K[DIM], D, Lam[DIM], P[DIM];
#pragma unroll
  for (int k = 0; k < 6; ++k) L[k].zero();
#pragma unroll
  for (int k = 0; k < DIM; ++k) { S[k].zero(); Cs[k].zero(); K[k].zero(); Lam[k].zero(); P[k].zero(); }
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) M[k].zero();
  D.zero();
  unsigned npairs = 0;
  const int maxc = __reduce_max_sync(0xffffffffu, cnt);
  const uint32_t* lst = w.nbr + gi;
  // The packed data of list entries k + 1 .. k + MX_RING - 1 is gathered
  // (cp.async into this lane's slots of a shared-memory ring) while entry k
  // is summed: the loop is latency bound on these dependent gathers, and the
  // ring holds them without registers, which leaves room for four resident
  // blocks per SM.
  __shared__ float4 ringA[MX_RING * MX_THREADS];
  __shared__ float4 ringB[MX_RING * MX_THREADS];
  __shared__ uint32_t ringC[MX_RING * MX_THREADS];
  const int t = threadIdx.x;
  auto fetch = [&](int k, uint32_t j) {  // entry k (< cnt), neighbour j, into slot k % MX_RING
    const int q = (k % MX_RING) * MX_THREADS + t;
    mx_cp16(&ringA[q], A + j);
    mx_cp16(&ringB[q], B + j);
    mx_cp4(&ringC[q], Cc + j);
  };
#pragma unroll
  for (int k = 0; k < MX_RING; ++k) {  // one group per entry (empty past the list)
    if (k < cnt) fetch(k, __ldg(lst + (int64_t)k * nf));
    mx_commit();
  }
  uint32_t jn = MX_RING < cnt ? __ldg(lst + (int64_t)MX_RING * nf) : 0u;  // next entry to fetch
  // entry k of the lists; terms of even k are parked (defer), odd k
  // completes the compensated step of the pair (add)
  auto entry = [&](int k, auto odd) {
    constexpr bool FULL = decltype(odd)::value;
    if (k >= cnt) return;
    mx_wait_ring();  // entry k's group has landed; the later ones may still be in flight
    const int q = (k % MX_RING) * MX_THREADS + t;
    const float4 Aj = ringA[q], Bj = ringB[q];
    const uint32_t cj = ringC[q];
    float r[DIM], du[DIM];
    r[0] = fmaf((float)((int)(cj & 2047u) - cix), R, Aj.x - Ai.x);
    r[1] = fmaf((float)((int)((cj >> 11) & 2047u) - ciy), R, Aj.y - Ai.y);
    if (DIM == 3) r[DIM - 1] = fmaf((float)((int)(cj >> 22) - ciz), R, Aj.z - Ai.z);
    float r2 = 0.f, dun = 0.f;
    du[0] = Bj.x - Bi.x;
    du[1] = Bj.y - Bi.y;
    if (DIM == 3) du[DIM - 1] = Bj.z - Bi.z;
#pragma unroll
    for (int c = 0; c < DIM; ++c) { r2 = fmaf(r[c], r[c], r2); dun = fmaf(du[c], r[c], dun); }
    const float Bjw = Bj.w, Ajw = Aj.w;
    // the slot is refilled with entry k + MX_RING only after the values read
    // from it (two 16-byte and one 4-byte shared load) have been used above
    if (k + MX_RING < cnt) {
      fetch(k + MX_RING, jn);
      if (k + MX_RING + 1 < cnt) jn = __ldg(lst + (int64_t)(k + MX_RING + 1) * nf);
    }
    mx_commit();
    if (!(r2 <= four_h2 && r2 > 0.f)) return;  // the neighbour test in FP32
    ++npairs;
    float inv_r = rsqrtf(r2);
    float rr = r2 * inv_r;
    float t = fmaf(-rr, inv_two_h, 1.f);
    float t3 = t * t * t;
    float g = coef * t3 * fabsf(Bjw);
    dun *= inv_r;
    float dphi = Ajw - Ai.w, sphi = Ajw + Ai.w;
    float rs = fmaf(-c0, dun, dphi);
    float gr[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) gr[c] = g * r[c];
    if (DIM == 2) {
      kacc<FULL>(L[0], r[0] * gr[0]); kacc<FULL>(L[1], r[0] * gr[1]); kacc<FULL>(L[2], r[1] * gr[1]);
    } else {
      kacc<FULL>(L[0], r[0] * gr[0]); kacc<FULL>(L[1], r[0] * gr[1]); kacc<FULL>(L[2], r[0] * gr[DIM - 1]);
      kacc<FULL>(L[3], r[1] * gr[1]); kacc<FULL>(L[4], r[1] * gr[DIM - 1]); kacc<FULL>(L[5], r[DIM - 1] * gr[DIM - 1]);
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      kacc<FULL>(S[c], rs * gr[c]);
      kacc<FULL>(Cs[c], sphi * gr[c]);
      kacc<FULL>(K[c], gr[c]);
#pragma unroll
      for (int d2 = 0; d2 < DIM; ++d2) kacc<FULL>(M[c * DIM + d2], du[c] * gr[d2]);
    }
    kacc<FULL>(D, dphi * g);
    if (Bjw > 0.f || p.wall_bc) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) kacc<FULL>(Lam[c], du[c] * g);
    }
    if (p.use_pst) {
      float q21 = fmaf(rr, two_over_h, 1.f);
      float ratio = pst_a * (t3 * t) * q21;
      float r4 = (ratio * ratio) * (ratio * ratio);
      float f = fmaf(pst_R, r4, 1.f);
#pragma unroll
      for (int c = 0; c < DIM; ++c) kacc<FULL>(P[c], f * gr[c]);
    }
  };
  for (int k = 0; k < maxc; k += 2) {
    entry(k, std::false_type{});
    if (k + 1 < maxc) entry(k + 1, std::true_type{});
  }
  unsigned wp = __reduce_add_sync(0xffffffffu, npairs);
  if (lane == 0 && wp) atomicAdd(w.pairs, (unsigned long long)wp);
  if (!active) return;

  // ---- epilogue. FP64: L^-1 (adjugate) and its contractions with S' and M,
  // the hydrostatic rebuild of the TIC branch and the continuity terms.
  // FP32: lambda_min (selects the branch), the viscous and shifting parts
  // (their pair sums are FP32-accurate, so FP64 arithmetic would add nothing).
  float lf[6];
  const int nl = DIM == 2 ? 3 : 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) lf[k] = k < nl ? L[k].s - L[k].c : 0.f;
  float lamf;
  if (DIM == 2) {
    float m = 0.5f * (lf[0] + lf[2]), d = 0.5f * (lf[0] - lf[2]);
    lamf = m - sqrtf(d * d + lf[1] * lf[1]);
  } else {
    lamf = lambda_min_3f(lf[0], lf[1], lf[2], lf[3], lf[4], lf[5]);
  }
  double fs = 0.0;
  if (p.omega > 0.0) fs = forcing_factor(p, stage2 ? w.scalars[0] + w.scalars[1] : w.scalars[0]);
  double acc[DIM], divu = 0.0;
  if (p.use_tic && lamf < (float)p.tic_lambda) {
    // conservative gradient of the full phi rebuilt from the phi' sums:
    // C = C' + 2 phi_hs,i K + L G, phi_hs,i = G.x_i + |G| H
    double phs = p.phs0;
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (p.g[c] != 0.0) phs = fma(p.g[c], s.x[c * n + i], phs);
    const double l00 = lf[0], l01 = lf[1], l11 = DIM == 3 ? lf[3] : lf[2];
    const double l02 = DIM == 3 ? lf[2] : 0.0, l12 = DIM == 3 ? lf[4] : 0.0, l22 = DIM == 3 ? lf[5] : 0.0;
    const double Lm[3][3] = {{l00, l01, l02}, {l01, l11, l12}, {l02, l12, l22}};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double lg = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) lg += Lm[c][e] * p.g[e];
      double gradphi = (double)(Cs[c].s - Cs[c].c) + 2.0 * phs * (double)(K[c].s - K[c].c) + lg;
      acc[c] = -gradphi + p.g[c] + p.force_amp[c] * fs;
      divu += (double)(M[c * DIM + c].s - M[c * DIM + c].c);
    }
  } else {
    // L^-1 = adj(L) / det(L); the FP32 sums are exact in FP64, and so is
    // max |L_ab| taken in FP32 for the singularity test |det| <= 1e-12 max^d
    float amax = 0.f;
#pragma unroll
    for (int k = 0; k < nl; ++k) amax = fmaxf(amax, fabsf(lf[k]));
    double adj[DIM][DIM], det;
    if (DIM == 2) {
      const double a = lf[0], b = lf[1], c = lf[2];
      det = a * c - b * b;
      adj[0][0] = c;
      adj[DIM - 1][DIM - 1] = a;
      adj[0][DIM - 1] = adj[DIM - 1][0] = -b;
    } else {
      const double a00 = lf[0], a01 = lf[1], a02 = lf[2], a11 = lf[3], a12 = lf[4], a22 = lf[5];
      double m[3][3];
      m[0][0] = a11 * a22 - a12 * a12;
      m[0][1] = a12 * a02 - a01 * a22;
      m[0][2] = a01 * a12 - a11 * a02;
      m[1][1] = a00 * a22 - a02 * a02;
      m[1][2] = a02 * a01 - a00 * a12;
      m[2][2] = a00 * a11 - a01 * a01;
      m[1][0] = m[0][1]; m[2][0] = m[0][2]; m[2][1] = m[1][2];
      det = a00 * m[0][0] + a01 * m[0][1] + a02 * m[0][2];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) adj[r % DIM][c % DIM] = m[r][c];
    }
    const double am = (double)amax;
    const double lim = DIM == 2 ? 1e-12 * am * am : 1e-12 * am * am * am;
    const bool ok = fabs(det) > lim;
    if (!ok) atomicOr(w.status, kStatSingular);
    const double id = ok ? 1.0 / det : 0.0;
    double Sd[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) Sd[c] = (double)(S[c].s - S[c].c);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double gs = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        gs = fma(adj[c][e], Sd[e], gs);
        divu = fma(adj[c][e], (double)(M[c * DIM + e].s - M[c * DIM + e].c), divu);
      }
      acc[c] = -gs * id + p.force_amp[c] * fs;   // -(L^-1 S' + G) + G(t)
    }
    divu *= id;
  }
  const float umax = sqrtf((float)__longlong_as_double((long long)*w.umax_bits));
  const double phii = s.phi[i];
  const float two_nu = (float)(2.0 * p.nu), m2h = (float)(-2.0 * p.h);
  unsigned bad = 0u;
  float dstar[DIM], dn2 = 0.f;
  double gk = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    double a = acc[c];
    if (p.use_visc) a += (double)(two_nu * (Lam[c].s - Lam[c].c));
    w.dudt[c * n + i] = a;
    bad |= ((unsigned)__double2hiint(a) & 0x7ff00000u) == 0x7ff00000u ? 1u : 0u;
    dstar[c] = m2h * umax * (P[c].s - P[c].c);
    dn2 = fmaf(dstar[c], dstar[c], dn2);
    gk += p.g[c] * (double)(K[c].s - K[c].c);
  }
  double diff = p.use_delta ? p.delta_h_c0 * 2.0 * ((double)(D.s - D.c) + gk) : 0.0;
  double dphidt = -eos_c2(p, phii) * divu + diff;
  w.dphidt[i] = dphidt;
  bad |= ((unsigned)__double2hiint(dphidt) & 0x7ff00000u) == 0x7ff00000u ? 1u : 0u;
  const float dn = sqrtf(dn2);
  const float scale = (p.use_pst && dn > 0.f) ? fminf(dn, 0.5f * umax) / dn : 0.f;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    float v = dstar[c] * scale;
    w.dushift[c * n + i] = (double)v;
    bad |= isfinite(v) ? 0u : 1u;
  }
  w.lambda[i] = (double)lamf;
  if (bad) atomicOr(w.status, kStatNaN);
}


// Pair sums over the candidate lists of k_nbr_list (built before this).
void launch_pair_mixed(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int stage2,
                       cudaStream_t st) {
  if (n == 0 || nf == 0) return;
  unsigned blocks = (unsigned)div_up(nf, MX_THREADS);
  if (p.dim == 2) k_pair_mixed<2><<<blocks, MX_THREADS, 0, st>>>(p, s, w, n, nf, stage2, w.packA, w.packB, w.packC);
  else k_pair_mixed<3><<<blocks, MX_THREADS, 0, st>>>(p, s, w, n, nf, stage2, w.packA, w.packB, w.packC);
}

}  // namespace wbsph
