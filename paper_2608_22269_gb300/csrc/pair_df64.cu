// pair_df64.cu -- the well-balanced pair pass at FP64-level accuracy on the
// FP32 pipe: double-float (df64) pair sums and an FP64 epilogue.
//
// On GB300 the FP64 pipe runs at 1/61 of the FP32 rate and bounds the FP64
// pass. Here every pair term is a double-float (about 48 significand bits,
// df64.cuh), so one FP64 multiply-add becomes 4 to 15 FP32 instructions and
// the pass moves to a pipe 61 times wider. Three choices keep the
// double-float work small and the accuracy at the FP64 level:
//  * Offsets in cell units: o = (x - cell origin) / R with the high part a
//    multiple of 2^-23. For a pair closer than R, (o_j,hi - o_i,hi) plus the
//    cell offset (-1, 0 or 1) is exact in FP32, so r / R costs one rounding
//    (of the low parts, about 2^-48 R). The sums are formed in these units
//    and rescaled by R or R^2 in FP64 at the end.
//  * Hydrostatic split, as in the mixed pass: phi = phi_hs(x) + phi' with
//    phi_hs = G.x + |G| H. The Riemann sum S' of phi' alone gives
//    grad phi = L^-1 S' + G, so the hydrostatic part never enters a pair sum
//    and the scheme is well balanced by construction. The TIC and delta-SPH
//    sums are rebuilt in FP64: C = C' + 2 phi_hs,i K + L G, D = D' + G.K,
//    K = sum grad W V.
//  * The same exact FP64 neighbour lists as the FP64 pass, so both passes
//    sum over the same pairs.
// The shifting sum is split as P = K + P', P' = sum (f - 1) grad W V, so only
// the shifting correction needs a separate accumulator. The packed hi/lo
// copies it reads are written per particle by k_pack_df (prepass.cu).
#include "../../include/wbsph.h"
#include "common.cuh"
#include "neighbor_iter.cuh"
#include "df64.cuh"
#include "physics.cuh"

namespace wbsph {

// ---------------------------------------------------------------------------
// Double-float pair pass over fluid particles (one lane per particle i), in
// cell units (rhat = r / R, R = 2h): with g = -W'(r)/r V_j = t^3 volc_j,
// t = 1 - |rhat|,
//   Lh += rhat (x) g rhat            L = R^2 Lh     (Eq. renorm)
//   Sh += [phi'_j - phi'_i - C0 (U_j - U_i).rhat/|rhat|] g rhat    S' = R Sh
//   Mh += (U_j - U_i) (x) g rhat     M = R Mh       (continuity)
//   Ch += (phi'_i + phi'_j) g rhat   C' = R Ch      (TIC branch)
//   Kh += g rhat                     K = R Kh
//   D' += (phi'_j - phi'_i) g                       (delta-SPH)
//   Lam+= (U_j - U_i) g, fluid j only (every j with no-slip walls)
//   Ph += (f - 1) g rhat             P = R (Kh + Ph), f = 1 + R_pst (W_ij / W(dx))^n
// ---------------------------------------------------------------------------
constexpr int DF_THREADS = 128;
#ifndef WBSPH_DF_MIN_BLOCKS
#define WBSPH_DF_MIN_BLOCKS 3  // resident blocks per SM the register budget is sized for
#endif
#ifndef WBSPH_DF_RING
#define WBSPH_DF_RING 2  // list entries of each lane in flight (shared-memory ring)
#endif
constexpr int DF_RING = WBSPH_DF_RING;

// Asynchronous global -> shared copies (cp.async, cached in L1), one group
// per list entry; a thread waits only for its own groups.
__device__ __forceinline__ void df_cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void df_cp4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void df_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void df_wait_ring() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(DF_RING - 1) : "memory");
}

// FP64 value of a float, widened exactly on the IEEE fields with integer
// instructions (the FP64 pipe keeps only the additions of the epilogue);
// zero and subnormal floats give zero (below 2^-126, far under the
// accuracy of any sum here), infinities and NaN stay non-finite.
__device__ __forceinline__ double df_f2d(float v) {
  const unsigned b = __float_as_uint(v), e = (b >> 23) & 0xFFu;
  if (e == 0u) return 0.0;
  const unsigned ed = e == 0xFFu ? 0x7FFu : e + (1023u - 127u);
  return __hiloint2double((int)((b & 0x80000000u) | (ed << 20) | ((b & 0x7FFFFFu) >> 3)), (int)(b << 29));
}

// hi + lo of a double-float in FP64: one rounding of the exact sum
__device__ __forceinline__ double df_val(df a) { return df_f2d(a.hi) + df_f2d(a.lo); }

template <int DIM>
__global__ void __launch_bounds__(DF_THREADS, WBSPH_DF_MIN_BLOCKS)
    k_pair_df(Params p, State s, Work w, int64_t n, int64_t nf, int stage2, int kept) {
  const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool active = gi < nf;
  const uint32_t i = active ? w.fluid_list[gi] : 0u;
  const int cnt = active ? (int)w.nbr_cnt[gi] : 0;
  const float4* __restrict__ A = w.packA;
  const float4* __restrict__ Al = w.packAl;
  const float4* __restrict__ B = w.packB;
  const float4* __restrict__ Bl = w.packBl;
  const uint32_t* __restrict__ Cc = w.packC;

  float4 Ai = make_float4(0.f, 0.f, 0.f, 0.f), Ali = Ai, Bi = Ai, Bli = Ai;
  uint32_t ci = 0;
  if (active) {
    Ai = A[i];
    Ali = Al[i];
    Bi = B[i];
    Bli = Bl[i];
    ci = Cc[i];
  }
  const int cix = (int)(ci & 2047u), ciy = (int)((ci >> 11) & 2047u), ciz = (int)(ci >> 22);
  const df phii = {Ai.w, Ali.w};
  const df ui[3] = {{Bi.x, Bli.x}, {Bi.y, Bli.y}, {Bi.z, Bli.z}};
  const df c0 = {p.df_c0[0], p.df_c0[1]};
  const df pra4 = {p.df_pst_Ra4[0], p.df_pst_Ra4[1]};
  const bool pst4 = p.use_pst && p.pst_n == 4.0;
  const bool needK = p.use_tic || p.use_delta || p.use_pst;

  constexpr int NL = DIM == 2 ? 3 : 6;
  const df z = {0.f, 0.f};
  df L[NL], S[DIM], M[DIM * DIM], Cs[DIM], K[DIM], Pp[DIM], Lam[DIM], D = z;
#pragma unroll
  for (int k = 0; k < NL; ++k) L[k] = z;
#pragma unroll
  for (int c = 0; c < DIM; ++c) S[c] = Cs[c] = K[c] = Pp[c] = Lam[c] = z;
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) M[k] = z;

  unsigned npairs = 0;
  const int maxc = __reduce_max_sync(0xffffffffu, cnt);
  const uint32_t* lst = w.nbr + gi;
  // The packed data of list entries k + 1 .. k + DF_RING - 1 is gathered
  // (cp.async into this lane's slots of a shared-memory ring) while entry k
  // is summed, so the gathers do not hold registers and their latency is
  // covered by the arithmetic of the entries before them.
  __shared__ float4 ringA[DF_RING * DF_THREADS], ringAl[DF_RING * DF_THREADS];
  __shared__ float4 ringB[DF_RING * DF_THREADS], ringBl[DF_RING * DF_THREADS];
  __shared__ uint32_t ringC[DF_RING * DF_THREADS];
  __shared__ uint32_t ringJ[DF_RING * DF_THREADS];  // the entry itself, for the exact test of kept lists
  const int tid = threadIdx.x;
  auto fetch = [&](int k, uint32_t j) {  // entry k (< cnt), neighbour j, into slot k % DF_RING
    const int q = (k % DF_RING) * DF_THREADS + tid;
    df_cp16(&ringA[q], A + j);
    df_cp16(&ringAl[q], Al + j);
    df_cp16(&ringB[q], B + j);
    df_cp16(&ringBl[q], Bl + j);
    df_cp4(&ringC[q], Cc + j);
    ringJ[q] = j;
  };
#pragma unroll
  for (int k = 0; k < DF_RING; ++k) {  // one group per entry (empty past the list)
    if (k < cnt) fetch(k, __ldg(lst + (int64_t)k * nf));
    df_commit();
  }
  uint32_t jn = DF_RING < cnt ? __ldg(lst + (int64_t)DF_RING * nf) : 0u;  // next entry to fetch
  for (int k = 0; k < maxc; ++k) {
    if (k >= cnt) continue;
    df_wait_ring();  // entry k's group has landed; the later ones may still be in flight
    const int q = (k % DF_RING) * DF_THREADS + tid;
    const float4 Aj = ringA[q], Alj = ringAl[q], Bj = ringB[q], Blj = ringBl[q];
    const uint32_t cj = ringC[q];
    const uint32_t jj = ringJ[q];
    // r / R: the high part (cell offset plus a difference of multiples of
    // 2^-23, below 2 in magnitude) is exact; the low parts round once
    df r[DIM];
    r[0] = {__fadd_rn((float)((int)(cj & 2047u) - cix), __fsub_rn(Aj.x, Ai.x)), __fsub_rn(Alj.x, Ali.x)};
    r[1] = {__fadd_rn((float)((int)((cj >> 11) & 2047u) - ciy), __fsub_rn(Aj.y, Ai.y)), __fsub_rn(Alj.y, Ali.y)};
    if (DIM == 3)
      r[DIM - 1] = {__fadd_rn((float)((int)(cj >> 22) - ciz), __fsub_rn(Aj.z, Ai.z)), __fsub_rn(Alj.z, Ali.z)};
    // |r/R|^2: squares of the high parts exact, cross terms 2 hi lo added in FP32
    df r2;
    {
      const df q0 = df_two_prod(r[0].hi, r[0].hi), q1 = df_two_prod(r[1].hi, r[1].hi);
      const df s01 = df_two_sum(q0.hi, q1.hi);
      float hi = s01.hi;
      float lo = __fadd_rn(s01.lo, __fadd_rn(q0.lo, q1.lo));
      lo = __fmaf_rn(__fmul_rn(2.f, r[0].hi), r[0].lo, lo);
      lo = __fmaf_rn(__fmul_rn(2.f, r[1].hi), r[1].lo, lo);
      if (DIM == 3) {
        const df q2 = df_two_prod(r[DIM - 1].hi, r[DIM - 1].hi);
        const df s2 = df_two_sum(hi, q2.hi);
        hi = s2.hi;
        lo = __fadd_rn(lo, __fadd_rn(s2.lo, q2.lo));
        lo = __fmaf_rn(__fmul_rn(2.f, r[DIM - 1].hi), r[DIM - 1].lo, lo);
      }
      r2 = df_fast_two_sum(hi, lo);
    }
    // R / |r|: FP32 estimate, a Newton-Raphson step y <- y (3 - r2 y^2) / 2 in
    // FP32 and one in double-float, y <- y + (y/2)(1 - r2 y^2), with the
    // residual 1 - r2 y^2 (near 2^-23) formed from exact products
    df inv;
    {
      float y = rsqrtf(r2.hi);
      y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f, r2.hi), __fmul_rn(y, y), 1.5f));
      const df yy = df_two_prod(y, y);
      const df a = df_two_prod(r2.hi, yy.hi);
      float e = __fsub_rn(1.f, a.hi);  // exact: a.hi is within a few ulp of 1
      e = __fsub_rn(e, a.lo);
      e = __fmaf_rn(-r2.hi, yy.lo, e);
      e = __fmaf_rn(-r2.lo, yy.hi, e);
      inv = df_fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), e));
    }
    // q / 2 = |r| / (2h) = (|r| / R) (R / 2h); R / 2h = 1 unless the cells
    // are widened for kept lists (then the product rounds once more)
    const df rr = df_mul(df_mul(r2, inv), df{p.df_R_2h[0], p.df_R_2h[1]});
    df t = df_fast_two_sum(1.f, -rr.hi);
    t = df_fast_two_sum(t.hi, __fsub_rn(t.lo, rr.lo));  // 1 - q/2
    // products that only feed other products or running sums stay
    // unrenormalised (df_mul_raw: the exact product of the high parts and the
    // cross terms; the next product or sum absorbs the unnormalised low part)
    const df t2 = df_mul_raw(t, t);
    const df t3 = df_mul_raw(t2, t);
    df vj = {Bj.w, Blj.w};
    const bool jfluid = vj.hi > 0.f;
    if (!jfluid) vj = df_neg(vj);
    const df g = df_mul_raw(t3, vj);
    df gr[DIM], du[DIM];
    du[0] = df_sub_raw({Bj.x, Blj.x}, ui[0]);
    du[1] = df_sub_raw({Bj.y, Blj.y}, ui[1]);
    if (DIM == 3) du[DIM - 1] = df_sub_raw({Bj.z, Blj.z}, ui[DIM - 1]);
    const df phij = {Aj.w, Alj.w};
    const df dphi = df_sub_raw(phij, phii);
    // the slot is refilled with entry k + DF_RING only after every value
    // read from it has been used above
    if (k + DF_RING < cnt) {
      fetch(k + DF_RING, jn);
      if (k + DF_RING + 1 < cnt) jn = __ldg(lst + (int64_t)(k + DF_RING + 1) * nf);
    }
    df_commit();
    if (kept) {
      // kept lists (radius 2h + delta): Algorithm 1's test. The double-float
      // |r/R|^2 is within ~1e-13 of the FP64 one, so outside a band of 1e-12
      // around (2h/R)^2 it decides as the FP64 test would; inside the band,
      // and near r = 0, the FP64 test itself decides
      const float dd = __fadd_rn(__fsub_rn(r2.hi, p.df_4h2_R2[0]), __fsub_rn(r2.lo, p.df_4h2_R2[1]));
      bool nb;
      if (dd < -1e-12f && r2.hi > 1e-6f) nb = true;
      else if (dd > 1e-12f) nb = false;
      else nb = exact_neighbor(p, s.x, n, i, jj);
      if (!nb) continue;
    } else if (!(r2.hi > 0.f)) {
      continue;
    }
    ++npairs;  // an exact neighbour (exact lists: k_nbr_list applied the FP64 test)
#pragma unroll
    for (int c = 0; c < DIM; ++c) gr[c] = df_mul_raw(g, r[c]);
    // (U_j - U_i).r / |r|
    df dun;
    {
      df pd = df_mul_raw(du[0], r[0]);
#pragma unroll
      for (int c = 1; c < DIM; ++c) {
        const df q = df_mul_raw(du[c], r[c]);
        const df sq = df_two_sum(pd.hi, q.hi);
        pd = {sq.hi, __fadd_rn(sq.lo, __fadd_rn(pd.lo, q.lo))};
      }
      dun = df_mul(df_norm(pd), inv);
    }
    df rs = dphi;  // phi'_j - phi'_i - C0 (U_j - U_i).r/|r|: 2 (phi* - phi_i) of Eq. lfsover
    df_acc(rs, df_neg(df_mul_raw(c0, dun)));
    if (DIM == 2) {
      df_acc(L[0], df_mul_raw(r[0], gr[0]));
      df_acc(L[1], df_mul_raw(r[0], gr[1]));
      df_acc(L[2], df_mul_raw(r[1], gr[1]));
    } else {
      df_acc(L[0], df_mul_raw(r[0], gr[0]));
      df_acc(L[1], df_mul_raw(r[0], gr[1]));
      df_acc(L[2 % NL], df_mul_raw(r[0], gr[DIM - 1]));
      df_acc(L[3 % NL], df_mul_raw(r[1], gr[1]));
      df_acc(L[4 % NL], df_mul_raw(r[1], gr[DIM - 1]));
      df_acc(L[5 % NL], df_mul_raw(r[DIM - 1], gr[DIM - 1]));
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      df_acc(S[c], df_mul_raw(rs, gr[c]));
#pragma unroll
      for (int e = 0; e < DIM; ++e) df_acc(M[c * DIM + e], df_mul_raw(du[c], gr[e]));
    }
    if (needK) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) df_acc(K[c], gr[c]);
    }
    if (p.use_tic) {
      const df s2 = df_two_sum(Aj.w, Ai.w);
      const df sphi = {s2.hi, __fadd_rn(s2.lo, __fadd_rn(Alj.w, Ali.w))};
#pragma unroll
      for (int c = 0; c < DIM; ++c) df_acc(Cs[c], df_mul_raw(sphi, gr[c]));
    }
    if (p.use_delta) df_acc(D, df_mul_raw(dphi, g));
    if (p.use_visc && (jfluid || p.wall_bc)) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) df_acc(Lam[c], df_mul_raw(du[c], g));
    }
    if (p.use_pst) {
      // W_ij / W(dx) = (alpha / W(dx)) v, v = t^4 (2q + 1), 2q + 1 = 4 |r|/R + 1
      const df q4 = df_two_sum(1.f, __fmul_rn(4.f, rr.hi));
      const df q21 = df_fast_two_sum(q4.hi, __fmaf_rn(4.f, rr.lo, q4.lo));
      const df v = df_mul_raw(df_mul_raw(t2, t2), q21);
      df fm1;  // f - 1 = R_pst (W_ij / W(dx))^n
      if (pst4) {
        const df v2 = df_mul_raw(v, v);
        fm1 = df_mul_raw(df_mul_raw(v2, v2), pra4);
      } else {
        fm1 = df_from_double(p.pst_R * pow(p.pst_alpha_over_wdx * df_to_double(v), p.pst_n));
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) df_acc(Pp[c], df_mul_raw(fm1, gr[c]));
    }
  }
  const int lane = threadIdx.x & 31;
  unsigned wp = __reduce_add_sync(0xffffffffu, npairs);
  if (lane == 0 && wp) atomicAdd(w.pairs, (unsigned long long)wp);
  if (!active) return;

  // ---- epilogue in FP64 (Eq. sph with the TIC switch; the correction
  // outside the sum, Sec. 3). The branch test is the one of the FP64 pass:
  // the FP32 closed form of lambda_min decides unless it lies within 0.05
  // of the threshold, where the FP64 closed form decides.
  const double R = p.R, R2 = R * R;
  double Ld[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < NL; ++k) Ld[k] = R2 * df_val(L[k]);
  bool tic_branch = false;
  if (p.use_tic) {
    const float lf = DIM == 2 ? lambda_min_2f((float)Ld[0], (float)Ld[1], (float)Ld[2])
                              : lambda_min_3f((float)Ld[0], (float)Ld[1], (float)Ld[2], (float)Ld[3],
                                              (float)Ld[4], (float)Ld[5]);
    const float tl = (float)p.tic_lambda;
    if (fabsf(lf - tl) > 0.05f) {
      tic_branch = lf < tl;
    } else {
      const double lam = DIM == 2 ? lambda_min_2(Ld[0], Ld[1], Ld[2])
                                  : lambda_min_3(Ld[0], Ld[1], Ld[2], Ld[3], Ld[4], Ld[5]);
      tic_branch = lam < p.tic_lambda;
    }
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) w.Lmat[k * n + i] = Ld[k];
  double Kd[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) Kd[c] = R * df_val(K[c]);
  const double fs = forcing_factor(p, stage_time(w, stage2));
  double acc[DIM], divu = 0.0;
  if (tic_branch) {
    // conservative gradient of the full phi: C = C' + 2 phi_hs,i K + L G
    double phs = p.phs0;
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (p.g[c] != 0.0) phs = fma(p.g[c], s.x[c * n + i], phs);
    const double l00 = Ld[0], l01 = Ld[1], l11 = DIM == 3 ? Ld[3] : Ld[2];
    const double l02 = DIM == 3 ? Ld[2] : 0.0, l12 = DIM == 3 ? Ld[4] : 0.0, l22 = DIM == 3 ? Ld[5] : 0.0;
    const double Lm[3][3] = {{l00, l01, l02}, {l01, l11, l12}, {l02, l12, l22}};
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double lg = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) lg = fma(Lm[c][e], p.g[e], lg);
      const double gradphi = R * df_val(Cs[c]) + 2.0 * phs * Kd[c] + lg;
      acc[c] = -gradphi + p.g[c] + p.force_amp[c] * fs;
      divu += R * df_val(M[c * DIM + c]);
    }
  } else {
    // grad phi = L^-1 S' + G, so -grad phi + G(t) = -L^-1 S' + A omega^2 sin(omega t)
    double inv[DIM][DIM];
    const bool ok = sym_inverse<DIM>(Ld, inv);
    if (!ok) atomicOr(w.status, kStatSingular);
    // the factor R of S' = R Sh and M = R Mh is applied to the contractions
    double Sd[DIM];
#pragma unroll
    for (int e = 0; e < DIM; ++e) Sd[e] = df_val(S[e]);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double gs = 0.0;
#pragma unroll
      for (int e = 0; e < DIM; ++e) {
        gs = fma(inv[c][e], Sd[e], gs);
        divu = fma(inv[c][e], df_val(M[c * DIM + e]), divu);
      }
      // a singular L zeroes the inverse: grad phi = 0, as in the FP64 pass
      acc[c] = -R * gs + (ok ? 0.0 : p.g[c]) + p.force_amp[c] * fs;
    }
    divu *= R;
  }
  const double umax = sqrt(__longlong_as_double((long long)*w.umax_bits));
  bool bad = false;
  double dstar[DIM], dn2 = 0.0, gk = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const double visc = p.use_visc ? 2.0 * p.nu * df_val(Lam[c]) : 0.0;
    const double a = acc[c] + visc;
    w.dudt[c * n + i] = a;
    bad |= !isfinite(a);
    const double P = p.use_pst ? Kd[c] + R * df_val(Pp[c]) : 0.0;
    dstar[c] = -2.0 * p.h * umax * P;
    dn2 += dstar[c] * dstar[c];
    gk = fma(p.g[c], Kd[c], gk);
  }
  const double diff = p.use_delta ? p.delta_h_c0 * (2.0 * (df_val(D) + gk)) : 0.0;
  const double dphidt = -eos_c2(p, s.phi[i]) * divu + diff;
  w.dphidt[i] = dphidt;
  bad |= !isfinite(dphidt);
  const double dn = sqrt(dn2);
  double scale = 0.0;
  if (p.use_pst && dn > 0.0) scale = fmin(dn, 0.5 * umax) / dn;
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const double v = dstar[c] * scale;
    w.dushift[c * n + i] = v;
    bad |= !isfinite(v);
  }
  if (bad) atomicOr(w.status, kStatNaN);
}

void launch_pair_df(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int stage2,
                    cudaStream_t st, bool kept) {
  if (nf == 0) return;
  const unsigned blocks = (unsigned)div_up(nf, DF_THREADS);
  if (p.dim == 2) k_pair_df<2><<<blocks, DF_THREADS, 0, st>>>(p, s, w, n, nf, stage2, kept ? 1 : 0);
  else k_pair_df<3><<<blocks, DF_THREADS, 0, st>>>(p, s, w, n, nf, stage2, kept ? 1 : 0);
}

}  // namespace wbsph
