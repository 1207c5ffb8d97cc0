// physics.cuh -- per-particle closed forms shared by the pair-pass epilogues:
// equation of state in potential form (Sec. 2.2.1), body force with the
// optional harmonic tank forcing, closed-form lambda_min of the symmetric
// renormalisation matrix (Sec. 3), and the adjugate inverse of L.
#pragma once
#include "common.cuh"

namespace wbsph {

// rho = rho0 exp(phi / C0^2) (linear EOS); rho0 (1 + (gamma-1) phi / c0^2)^(1/(gamma-1)) (Tait).
__device__ __forceinline__ double eos_density(const Params& p, double phi) {
  if (p.eos == 0) return p.rho0 * exp(phi / p.c0sq);
  double gm1 = p.gamma - 1.0;
  return p.rho0 * pow(1.0 + gm1 * phi / p.c0sq, 1.0 / gm1);
}

// D(phi)/Dt = -c^2 div U: c^2 = C0^2 (linear EOS), c0^2 + (gamma - 1) phi (Tait).
__device__ __forceinline__ double eos_c2(const Params& p, double phi) {
  return p.eos == 0 ? p.c0sq : p.c0sq + (p.gamma - 1.0) * phi;
}

// Frame acceleration of a harmonically forced tank, A w^2 sin(w t) per unit A.
__device__ __forceinline__ double forcing_factor(const Params& p, double t) {
  return p.omega > 0.0 ? p.omega * p.omega * sin(p.omega * t) : 0.0;
}

__device__ __forceinline__ double stage_time(const Work& w, int stage2) {
  return stage2 ? w.scalars[0] + w.scalars[1] : w.scalars[0];
}

// Smallest eigenvalue of a symmetric matrix in closed form. 2D:
// mean - sqrt(half-difference^2 + off^2). 3D: trigonometric root of the
// characteristic cubic (Smith, CACM 1961).
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
  double r = fmin(1.0, fmax(-1.0, det / (2.0 * pp * pp * pp)));
  return mean + 2.0 * pp * cos(acos(r) * (1.0 / 3.0) + 2.0943951023931954923);  // + 2 pi / 3
}

// FP32 forms of the same closed forms (branch selection and the mixed path).
__device__ __forceinline__ float lambda_min_2f(float a, float b, float c) {
  float m = 0.5f * (a + c), d = 0.5f * (a - c);
  return m - sqrtf(d * d + b * b);
}

__device__ __forceinline__ float lambda_min_3f(float a00, float a01, float a02, float a11, float a12,
                                               float a22) {
  float off = a01 * a01 + a02 * a02 + a12 * a12;
  if (off == 0.f) return fminf(fminf(a00, a11), a22);
  float mean = (a00 + a11 + a22) * (1.f / 3.f);
  float b00 = a00 - mean, b11 = a11 - mean, b22 = a22 - mean;
  float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.f * off;
  float pp = sqrtf(p2 * (1.f / 6.f));
  float det = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) + a02 * (a01 * a12 - b11 * a02);
  float r = fminf(1.f, fmaxf(-1.f, det / (2.f * pp * pp * pp)));
  return mean + 2.f * pp * cosf(acosf(r) * (1.f / 3.f) + 2.09439510f);
}

// Inverse of the symmetric L (upper triangle l[]: 2D 00 01 11; 3D 00 01 02
// 11 12 22) by the adjugate. Returns false (inverse zeroed) when
// |det| <= 1e-12 max|L_ab|^d, the singularity test of the corrected branch.
template <int DIM>
__device__ __forceinline__ bool sym_inverse(const double* l, double inv[DIM][DIM]) {
  double amax = 0.0;
  bool ok;
  if (DIM == 2) {
    double a = l[0], b = l[1], c = l[2];
    amax = fmax(fabs(a), fmax(fabs(b), fabs(c)));
    double det = a * c - b * b;
    ok = fabs(det) > 1e-12 * amax * amax;
    double id = ok ? 1.0 / det : 0.0;
    inv[0][0] = c * id;
    inv[DIM - 1][DIM - 1] = a * id;
    inv[0][DIM - 1] = inv[DIM - 1][0] = -b * id;
  } else {
    double a00 = l[0], a01 = l[1], a02 = l[2], a11 = l[3], a12 = l[4], a22 = l[5];
    amax = fmax(fmax(fabs(a00), fabs(a01)), fmax(fmax(fabs(a02), fabs(a11)), fmax(fabs(a12), fabs(a22))));
    double c00 = a11 * a22 - a12 * a12;
    double c01 = a12 * a02 - a01 * a22;
    double c02 = a01 * a12 - a11 * a02;
    double det = a00 * c00 + a01 * c01 + a02 * c02;
    ok = fabs(det) > 1e-12 * amax * amax * amax;
    double id = ok ? 1.0 / det : 0.0;
    double m[3][3];
    m[0][0] = c00; m[0][1] = c01; m[0][2] = c02;
    m[1][1] = a00 * a22 - a02 * a02;
    m[1][2] = a02 * a01 - a00 * a12;
    m[2][2] = a00 * a11 - a01 * a01;
    m[1][0] = c01; m[2][0] = c02; m[2][1] = m[1][2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) inv[r % DIM][c % DIM] = m[r][c] * id;
  }
  return ok;
}

}  // namespace wbsph
