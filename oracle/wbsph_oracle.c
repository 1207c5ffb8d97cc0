/*
 * wbsph_oracle.c -- plain FP64 CPU oracle of the well-balanced WCSPH step.
 *
 * TEST INFRASTRUCTURE ONLY (see wbsph_oracle.h): the tests, the smoke check
 * and the benchmark's CPU-baseline leg are its only callers. It follows the
 * paper's definitions in their order, sums every neighbour list in ascending
 * particle index, keeps the caller's particle order (it never reorders) and
 * must be compiled without floating-point contraction (-ffp-contract=off) so
 * that the neighbour distance test is the plain IEEE expression.
 *
 * The OpenMP loops run over independent particles only; each particle's sum
 * has a fixed order, so results do not depend on the thread count.
 */
#include "wbsph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FLUID 0
#define DUMMY 1
#define BODY 2

static const double PI = 3.14159265358979323846;

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int valid_config(const orc_config* c) {
  if (!c) return 0;
  if (c->dim != 2 && c->dim != 3) return 0;
  if (!(c->dx > 0) || !(c->h_over_dx > 0) || !(c->rho0 > 0) || !(c->c0 > 0)) return 0;
  if (c->nu < 0 || c->cfl <= 0) return 0;
  if (c->eos != 0 && c->eos != 1) return 0;
  if (c->eos == 1 && !(c->tait_gamma > 1)) return 0;
  for (int k = 0; k < c->dim; ++k)
    if (!(c->domain_max[k] > c->domain_min[k])) return 0;
  if (c->scheme != 0 && c->scheme != 1) return 0;
  if (c->scheme == 1 && (c->use_delta || c->use_pst || c->use_tic || c->art_alpha < 0)) return 0;
  if (c->wall_bc != 0 && c->wall_bc != 1) return 0;
  return 1;
}

/* ---------------------------------------------------------------------------
 * Kernel, Eq. (c2kernel): W(q) = alpha (1 - q/2)^4 (2q + 1) for q = r/h <= 2.
 * alpha = 7/(4 pi h^2) in 2D (printed); 21/(16 pi h^3) in 3D (normalised so
 * that the kernel integrates to one over its support of radius 2h).
 * ------------------------------------------------------------------------- */
static double kernel_alpha(int dim, double h) {
  if (dim == 2) return 7.0 / (4.0 * PI * h * h);
  return 21.0 / (16.0 * PI * h * h * h);
}

static double kernel_w(int dim, double h, double r) {
  double q = r / h;
  if (q > 2.0) return 0.0;
  double t = 1.0 - 0.5 * q;
  return kernel_alpha(dim, h) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr, from differentiating the kernel in q: d/dq[(1-q/2)^4 (2q+1)] = -5 q (1-q/2)^3. */
static double kernel_dwdr(int dim, double h, double r) {
  double q = r / h;
  if (q > 2.0) return 0.0;
  double t = 1.0 - 0.5 * q;
  return -5.0 * kernel_alpha(dim, h) * q * t * t * t / h;
}

int orc_kernel_eval(const orc_config* c, int64_t m, const double* r, double* w, double* dwdr) {
  if (!valid_config(c) || m < 0) return ORC_E_INVAL;
  double h = c->h_over_dx * c->dx;
  for (int64_t i = 0; i < m; ++i) {
    if (w) w[i] = kernel_w(c->dim, h, r[i]);
    if (dwdr) dwdr[i] = kernel_dwdr(c->dim, h, r[i]);
  }
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Equation of state in potential form (Sec. 2.2.1).
 * Linear EOS p = C0^2 (rho - rho0) gives phi = C0^2 ln(rho/rho0), i.e.
 * rho = rho0 exp(phi / C0^2), and D(phi)/Dt = -C0^2 div U.
 * Tait EOS p = rho0 c0^2/gamma ((rho/rho0)^gamma - 1) gives, with
 * phi = integral of dp/rho from rho0, phi = c0^2/(gamma-1) ((rho/rho0)^(gamma-1) - 1)
 * and D(phi)/Dt = -(c0^2 + (gamma-1) phi) div U.
 * ------------------------------------------------------------------------- */
static double eos_density(const orc_config* c, double phi) {
  if (c->eos == 0) return c->rho0 * exp(phi / (c->c0 * c->c0));
  double gm1 = c->tait_gamma - 1.0;
  return c->rho0 * pow(1.0 + gm1 * phi / (c->c0 * c->c0), 1.0 / gm1);
}

static double eos_pressure(const orc_config* c, double phi) {
  double rho = eos_density(c, phi);
  if (c->eos == 0) return c->c0 * c->c0 * (rho - c->rho0);
  double gam = c->tait_gamma;
  return c->rho0 * c->c0 * c->c0 / gam * (pow(rho / c->rho0, gam) - 1.0);
}

static double eos_c2(const orc_config* c, double phi) {
  if (c->eos == 0) return c->c0 * c->c0;
  return c->c0 * c->c0 + (c->tait_gamma - 1.0) * phi;
}

int orc_density(const orc_config* c, int64_t n, const double* phi, double* rho) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  for (int64_t i = 0; i < n; ++i) rho[i] = eos_density(c, phi[i]);
  return ORC_OK;
}

int orc_pressure(const orc_config* c, int64_t n, const double* phi, double* p) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  for (int64_t i = 0; i < n; ++i) p[i] = eos_pressure(c, phi[i]);
  return ORC_OK;
}

/* Particle mass: the initial density times the particle volume dx^d. */
int orc_mass(const orc_config* c, int64_t n, const double* phi, double* mass) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  double vol = c->dim == 2 ? c->dx * c->dx : c->dx * c->dx * c->dx;
  for (int64_t i = 0; i < n; ++i) mass[i] = eos_density(c, phi[i]) * vol;
  return ORC_OK;
}

/* Body force at time t: constant G plus, for a harmonically forced tank
 * x_tank(t) = A sin(w t), the frame acceleration A w^2 sin(w t). */
static void body_force(const orc_config* c, double t, double* g) {
  for (int k = 0; k < 3; ++k) g[k] = c->g[k];
  if (c->force_period > 0) {
    double w = 2.0 * PI / c->force_period;
    double s = w * w * sin(w * t);
    for (int k = 0; k < 3; ++k) g[k] += c->force_amp[k] * s;
  }
}

/* ---------------------------------------------------------------------------
 * Cell keys, Eqs. (hashid) and (ixyz). R = 2h. The grid extent per axis is
 * floor((max - min)/R) + 1 cells so that x = max falls in the last cell.
 * ------------------------------------------------------------------------- */
static void grid_dims(const orc_config* c, int64_t* nc) {
  double R = 2.0 * (c->h_over_dx * c->dx);
  for (int k = 0; k < 3; ++k) nc[k] = 1;
  for (int k = 0; k < c->dim; ++k)
    nc[k] = (int64_t)floor((c->domain_max[k] - c->domain_min[k]) / R) + 1;
}

static int cell_coords(const orc_config* c, int64_t n, const double* x, int64_t i, int64_t* ic) {
  double R = 2.0 * (c->h_over_dx * c->dx);
  ic[0] = ic[1] = ic[2] = 0;
  for (int k = 0; k < c->dim; ++k) {
    double xk = x[k * n + i];
    if (!(xk >= c->domain_min[k] && xk <= c->domain_max[k])) return ORC_E_DOMAIN;
    ic[k] = (int64_t)floor((xk - c->domain_min[k]) / R);
  }
  return ORC_OK;
}

int orc_cell_keys(const orc_config* c, int64_t n, const double* x, uint32_t* key) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  int64_t nc[3];
  grid_dims(c, nc);
  if (nc[0] * nc[1] * nc[2] > 0xFFFFFFFFLL) return ORC_E_INVAL;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ic[3];
    int rc = cell_coords(c, n, x, i, ic);
    if (rc) return rc;
    key[i] = (uint32_t)(ic[0] + ic[1] * nc[0] + ic[2] * nc[0] * nc[1]);
  }
  return ORC_OK;
}

/* Stable ascending sort of particle indices by key (counting sort on the
 * full key range would be too large; a stable merge sort is used). */
int orc_sort_by_key(int64_t n, const uint32_t* key, uint32_t* perm) {
  if (n < 0) return ORC_E_INVAL;
  uint32_t* tmp = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  if (!tmp) return ORC_E_NOMEM;
  for (int64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
  for (int64_t width = 1; width < n; width *= 2) {
    for (int64_t lo = 0; lo < n; lo += 2 * width) {
      int64_t mid = lo + width < n ? lo + width : n;
      int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
      int64_t a = lo, b = mid, o = lo;
      while (a < mid && b < hi) {
        if (key[perm[b]] < key[perm[a]]) tmp[o++] = perm[b++];
        else tmp[o++] = perm[a++]; /* equal keys keep their order: stable */
      }
      while (a < mid) tmp[o++] = perm[a++];
      while (b < hi) tmp[o++] = perm[b++];
    }
    memcpy(perm, tmp, sizeof(uint32_t) * (size_t)n);
  }
  free(tmp);
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Neighbour criterion (Algorithm 1): j is a neighbour of i when j != i and
 * the distance d <= 2h. Evaluated as r^2 = (dx*dx + dy*dy) + dz*dz, left to
 * right without contraction, against (2h)*(2h). Coincident pairs (r^2 = 0)
 * are excluded: the kernel gradient has no direction there.
 * ------------------------------------------------------------------------- */
static int is_neighbor(const orc_config* c, int64_t n, const double* x, int64_t i, int64_t j,
                       double four_h2) {
  if (i == j) return 0;
  double d0 = x[j] - x[i];
  double r2 = d0 * d0;
  double d1 = x[n + j] - x[n + i];
  r2 = r2 + d1 * d1;
  if (c->dim == 3) {
    double d2 = x[2 * n + j] - x[2 * n + i];
    r2 = r2 + d2 * d2;
  }
  return r2 <= four_h2 && r2 > 0.0;
}

typedef struct {
  int64_t* row;
  int32_t* col;
  int64_t nnz;
} csr_t;

static void csr_free(csr_t* a) {
  free(a->row);
  free(a->col);
  a->row = NULL;
  a->col = NULL;
}

/* Cell-list build of the neighbour lists; every row ascending in j. */
static int build_neighbors(const orc_config* c, int64_t n, const double* x, int brute,
                           csr_t* out) {
  double two_h = 2.0 * (c->h_over_dx * c->dx);
  double four_h2 = two_h * two_h;
  out->row = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  out->col = NULL;
  out->nnz = 0;
  if (!out->row) return ORC_E_NOMEM;
  int64_t nc[3];
  grid_dims(c, nc);
  int64_t ncell = nc[0] * nc[1] * nc[2];
  uint32_t* key = NULL;
  uint32_t* perm = NULL;
  int64_t* start = NULL;
  int rc = ORC_OK;
  if (!brute) {
    key = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
    if (!key || !perm || !start) { rc = ORC_E_NOMEM; goto done; }
    rc = orc_cell_keys(c, n, x, key);
    if (rc) goto done;
    rc = orc_sort_by_key(n, key, perm);
    if (rc) goto done;
    /* start[k] .. start[k+1]: sorted positions of the particles in cell k */
    for (int64_t k = 0; k <= ncell; ++k) start[k] = 0;
    for (int64_t i = 0; i < n; ++i) start[key[i] + 1] += 1;
    for (int64_t k = 0; k < ncell; ++k) start[k + 1] += start[k];
  } else {
    for (int64_t i = 0; i < n; ++i) {
      int64_t ic[3];
      rc = cell_coords(c, n, x, i, ic);
      if (rc) goto done;
    }
  }
  for (int pass = 0; pass < 2; ++pass) {
    int err = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : err)
    for (int64_t i = 0; i < n; ++i) {
      int64_t cnt = 0;
      int64_t base = pass ? out->row[i] : 0;
      if (brute) {
        for (int64_t j = 0; j < n; ++j)
          if (is_neighbor(c, n, x, i, j, four_h2)) {
            if (pass) out->col[base + cnt] = (int32_t)j;
            ++cnt;
          }
      } else {
        int64_t ic[3];
        if (cell_coords(c, n, x, i, ic)) { err = 1; continue; }
        int64_t lo2 = c->dim == 3 ? -1 : 0, hi2 = c->dim == 3 ? 1 : 0;
        for (int64_t oz = lo2; oz <= hi2; ++oz)
          for (int64_t oy = -1; oy <= 1; ++oy)
            for (int64_t ox = -1; ox <= 1; ++ox) {
              int64_t cx = ic[0] + ox, cy = ic[1] + oy, cz = ic[2] + oz;
              if (cx < 0 || cy < 0 || cz < 0 || cx >= nc[0] || cy >= nc[1] || cz >= nc[2])
                continue;
              int64_t cell = cx + cy * nc[0] + cz * nc[0] * nc[1];
              for (int64_t s = start[cell]; s < start[cell + 1]; ++s) {
                int64_t j = perm[s];
                if (is_neighbor(c, n, x, i, j, four_h2)) {
                  if (pass) out->col[base + cnt] = (int32_t)j;
                  ++cnt;
                }
              }
            }
        if (pass) {
          /* ascending j within the row (insertion sort of a short list) */
          int32_t* r = out->col + base;
          for (int64_t a = 1; a < cnt; ++a) {
            int32_t v = r[a];
            int64_t b = a - 1;
            while (b >= 0 && r[b] > v) { r[b + 1] = r[b]; --b; }
            r[b + 1] = v;
          }
        }
      }
      if (!pass) out->row[i + 1] = cnt;
    }
    if (err) { rc = ORC_E_DOMAIN; goto done; }
    if (!pass) {
      for (int64_t i = 0; i < n; ++i) out->row[i + 1] += out->row[i];
      out->nnz = out->row[n];
      out->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(out->nnz > 0 ? out->nnz : 1));
      if (!out->col) { rc = ORC_E_NOMEM; goto done; }
    }
  }
done:
  free(key);
  free(perm);
  free(start);
  if (rc) csr_free(out);
  return rc;
}

int64_t orc_neighbors(const orc_config* c, int64_t n, const double* x, int brute,
                      int64_t* row_ptr, int32_t* cols, int64_t cap) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  csr_t a;
  int rc = build_neighbors(c, n, x, brute, &a);
  if (rc) return rc;
  int64_t nnz = a.nnz;
  if (row_ptr) memcpy(row_ptr, a.row, sizeof(int64_t) * (size_t)(n + 1));
  if (cols) {
    if (nnz > cap) { csr_free(&a); return ORC_E_CAP; }
    memcpy(cols, a.col, sizeof(int32_t) * (size_t)nnz);
  }
  csr_free(&a);
  return nnz;
}

/* ---------------------------------------------------------------------------
 * Smallest eigenvalue of the symmetric renormalisation matrix in closed form
 * (Sec. 3: L is symmetric for a radial kernel, so no iteration is needed).
 * 2D: (a+c)/2 - sqrt(((a-c)/2)^2 + b^2).
 * 3D: the trigonometric solution of the characteristic cubic (O. K. Smith,
 * "Eigenvalues of a symmetric 3x3 matrix", CACM 4(4), 1961).
 * ------------------------------------------------------------------------- */
int orc_eig_min_sym(int dim, const double* a, double* lam) {
  if (dim == 2) {
    double p = a[0], b = a[1], q = a[4];
    double m = 0.5 * (p + q), d = 0.5 * (p - q);
    *lam = m - sqrt(d * d + b * b);
    return ORC_OK;
  }
  if (dim != 3) return ORC_E_INVAL;
  double a00 = a[0], a11 = a[4], a22 = a[8];
  double a01 = a[1], a02 = a[2], a12 = a[5];
  double off = a01 * a01 + a02 * a02 + a12 * a12;
  if (off == 0.0) {
    double m = a00 < a11 ? a00 : a11;
    *lam = m < a22 ? m : a22;
    return ORC_OK;
  }
  double mean = (a00 + a11 + a22) / 3.0;
  double b00 = a00 - mean, b11 = a11 - mean, b22 = a22 - mean;
  double p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.0 * off;
  double p = sqrt(p2 / 6.0);
  /* det of B = (A - mean I) / p, halved */
  double detb = b00 * (b11 * b22 - a12 * a12) - a01 * (a01 * b22 - a12 * a02) +
                a02 * (a01 * a12 - b11 * a02);
  double r = detb / (2.0 * p * p * p);
  if (r < -1.0) r = -1.0;
  if (r > 1.0) r = 1.0;
  double ang = acos(r) / 3.0;
  *lam = mean + 2.0 * p * cos(ang + 2.0 * PI / 3.0);
  return ORC_OK;
}

/* Inverse of a small matrix by Gauss-Jordan elimination with partial
 * pivoting. Returns the determinant through *det (0 when a pivot vanishes). */
static void small_inverse(int d, const double* a, double* inv, double* det) {
  double m[3][6];
  for (int r = 0; r < d; ++r)
    for (int k = 0; k < 2 * d; ++k)
      m[r][k] = k < d ? a[r * 3 + k] : (k - d == r ? 1.0 : 0.0);
  double dt = 1.0;
  for (int col = 0; col < d; ++col) {
    int piv = col;
    for (int r = col + 1; r < d; ++r)
      if (fabs(m[r][col]) > fabs(m[piv][col])) piv = r;
    if (m[piv][col] == 0.0) { *det = 0.0; return; }
    if (piv != col) {
      for (int k = 0; k < 2 * d; ++k) { double t = m[col][k]; m[col][k] = m[piv][k]; m[piv][k] = t; }
      dt = -dt;
    }
    double pv = m[col][col];
    dt *= pv;
    for (int k = 0; k < 2 * d; ++k) m[col][k] /= pv;
    for (int r = 0; r < d; ++r) {
      if (r == col) continue;
      double f = m[r][col];
      for (int k = 0; k < 2 * d; ++k) m[r][k] -= f * m[col][k];
    }
  }
  for (int r = 0; r < d; ++r)
    for (int k = 0; k < d; ++k) inv[r * 3 + k] = m[r][d + k];
  *det = dt;
}

/* ---------------------------------------------------------------------------
 * Wall particles (Sec. 2.4): each dummy (and body) particle takes the
 * potential of its nearest fluid particle f within 2h shifted by the body
 * force, Eq. (phiBn), phi_d = phi_f + G . (x_d - x_f), and with the wall
 * velocity U_w (zero for fixed walls, body_u for body particles) the slip
 * velocity U_d = U_f - ((U_f - U_w) . n_d) n_d (the paper's choice, stated
 * there for a fixed wall) or the no-slip velocity of Eq. (velBn),
 * U_d = 2 U_w - U_f. Ties in distance go to the smallest index; a wall
 * particle with no fluid particle within 2h keeps its values (it then lies
 * in no fluid particle's support).
 * ------------------------------------------------------------------------- */
static int dummy_update_csr(const orc_config* c, int64_t n, const double* x, double* u,
                            double* phi, const uint8_t* type, const double* normal, double t,
                            const csr_t* nb) {
  int d = c->dim;
  double G[3];
  body_force(c, t, G);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    if (type[i] == FLUID) continue;
    int64_t best = -1;
    double best_r2 = 0.0;
    for (int64_t e = nb->row[i]; e < nb->row[i + 1]; ++e) {
      int64_t j = nb->col[e];
      if (type[j] != FLUID) continue;
      double r2 = 0.0;
      for (int k = 0; k < d; ++k) {
        double dk = x[k * n + j] - x[k * n + i];
        r2 = r2 + dk * dk;
      }
      if (best < 0 || r2 < best_r2) { best = j; best_r2 = r2; }
    }
    if (best < 0) continue;
    double uw[3] = {0.0, 0.0, 0.0};
    if (type[i] == BODY)
      for (int k = 0; k < d; ++k) uw[k] = c->body_u[k];
    double gdot = 0.0, un = 0.0;
    for (int k = 0; k < d; ++k) {
      gdot += G[k] * (x[k * n + i] - x[k * n + best]);
      un += (u[k * n + best] - uw[k]) * normal[k * n + i];
    }
    phi[i] = phi[best] + gdot;
    for (int k = 0; k < d; ++k) {
      if (c->wall_bc == 1) u[k * n + i] = 2.0 * uw[k] - u[k * n + best];
      else u[k * n + i] = u[k * n + best] - un * normal[k * n + i];
    }
  }
  return ORC_OK;
}

int orc_dummy_update(const orc_config* c, int64_t n, const double* x, double* u, double* phi,
                     const uint8_t* type, const double* normal, double t) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  csr_t nb;
  int rc = build_neighbors(c, n, x, 0, &nb);
  if (rc) return rc;
  rc = dummy_update_csr(c, n, x, u, phi, type, normal, t, &nb);
  csr_free(&nb);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Pair sums of one particle i over its neighbour list (Eqs. renorm, lfsover,
 * parGrad, the conservative formula, delta-SPH, particle shifting and the
 * Laplacian operator of Sec. 2.1), with grad_i W_ij = dW/dr (x_i - x_j)/r:
 *   L      = sum (x_j - x_i) (x) grad_i W_ij V_j
 *   S      = sum 2 (phi*_ij - phi_i) grad_i W_ij V_j
 *   M      = sum (U_j - U_i) (x) grad_i W_ij V_j
 *   C      = sum (phi_j + phi_i) grad_i W_ij V_j
 *   D      = sum 2 (phi_j - phi_i) (x_j - x_i).grad_i W_ij / r^2 V_j
 *   P      = sum [1 + R (W_ij / W(dx))^n] grad_i W_ij V_j
 *   Lambda = sum over fluid j of (U_j - U_i) (x_j - x_i).grad_i W_ij / r^2 V_j
 * with phi*_ij = (phi_i + phi_j)/2 - C0/2 (U_j.e - U_i.e), e = (x_j - x_i)/r.
 * D carries no delta h C0 factor here; it is applied in the rates.
 * ------------------------------------------------------------------------- */
static void pair_sums_one(const orc_config* c, int64_t n, const double* x, const double* u,
                          const double* phi, const double* vol, const uint8_t* type,
                          const csr_t* nb, int64_t i, double* out) {
  int d = c->dim;
  double h = c->h_over_dx * c->dx;
  double w_dx = kernel_w(d, h, c->dx);
  double L[9] = {0}, S[3] = {0}, M[9] = {0}, C[3] = {0}, D = 0, P[3] = {0}, Lam[3] = {0};
  for (int64_t e = nb->row[i]; e < nb->row[i + 1]; ++e) {
    int64_t j = nb->col[e];
    double rij[3] = {0, 0, 0};
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
      rij[k] = x[k * n + j] - x[k * n + i];
      r2 += rij[k] * rij[k];
    }
    double r = sqrt(r2);
    double dwdr = kernel_dwdr(d, h, r);
    double gw[3] = {0, 0, 0}; /* grad_i W_ij = dW/dr (x_i - x_j) / r */
    for (int k = 0; k < d; ++k) gw[k] = dwdr * (-rij[k]) / r;
    double vj = vol[j];
    /* Lax-Friedrichs interface potential, Eq. (lfsover) */
    double uni = 0.0, unj = 0.0;
    for (int k = 0; k < d; ++k) {
      uni += u[k * n + i] * rij[k] / r;
      unj += u[k * n + j] * rij[k] / r;
    }
    double phistar = 0.5 * (phi[i] + phi[j]) - 0.5 * c->c0 * (unj - uni);
    double rgw = 0.0; /* (x_j - x_i) . grad_i W_ij */
    for (int k = 0; k < d; ++k) rgw += rij[k] * gw[k];
    double wij = kernel_w(d, h, r);
    double ratio = wij / w_dx;
    double shift = 1.0 + c->pst_R * pow(ratio, c->pst_n);
    for (int a = 0; a < d; ++a) {
      for (int b = 0; b < d; ++b) {
        L[a * 3 + b] += rij[a] * gw[b] * vj;
        M[a * 3 + b] += (u[a * n + j] - u[a * n + i]) * gw[b] * vj;
      }
      S[a] += 2.0 * (phistar - phi[i]) * gw[a] * vj;
      C[a] += (phi[j] + phi[i]) * gw[a] * vj;
      P[a] += shift * gw[a] * vj;
      if (type[j] == FLUID || c->wall_bc == 1) Lam[a] += (u[a * n + j] - u[a * n + i]) * rgw / r2 * vj;
    }
    D += 2.0 * (phi[j] - phi[i]) * rgw / r2 * vj;
  }
  memcpy(out, L, sizeof L);
  memcpy(out + 9, S, sizeof S);
  memcpy(out + 12, M, sizeof M);
  memcpy(out + 21, C, sizeof C);
  out[24] = D;
  memcpy(out + 25, P, sizeof P);
  memcpy(out + 28, Lam, sizeof Lam);
}

/* ---------------------------------------------------------------------------
 * Conventional WCSPH rates of fluid particle i (Sec. 2.1: Eq. nslag, the
 * linear EOS of Eq. eos-water, the printed operators <div U>, <grad p> and
 * <lap U>), the foil of the hydrostatic comparison. The state stays
 * (x, U, phi) with rho = rho(phi) and p = p(phi) by the EOS; since
 * d(phi) = c^2 d(rho)/rho, Drho/Dt = -rho div U is Dphi/Dt = -c^2 div U:
 *   DU/Dt   = -(1/rho_i) sum (p_i + p_j) grad_i W_ij V_j + 2 nu Lambda + Pi + G(t)
 *   Dphi/Dt = -c^2 sum (U_j - U_i).grad_i W_ij V_j
 *   Pi      = -sum m_j Pi_ij grad_i W_ij, m_j = rho_j V_j,
 *   Pi_ij   = -alpha h C0 (U_ij.x_ij) / (rho_ij (|x_ij|^2 + 0.01 h^2)) when
 *             U_ij.x_ij < 0, else 0; U_ij = U_i - U_j, x_ij = x_i - x_j,
 *             rho_ij = (rho_i + rho_j)/2 (artificial viscosity, Monaghan's form)
 * with Lambda the Laplacian sum of pair_sums_one (fluid neighbours).
 * ------------------------------------------------------------------------- */
static void conventional_rates_one(const orc_config* c, int64_t n, const double* x, const double* u,
                                   const double* phi, const double* vol, const uint8_t* type,
                                   const csr_t* nb, int64_t i, const double* G, double* dudt,
                                   double* dphidt) {
  int d = c->dim;
  double h = c->h_over_dx * c->dx;
  double rho_i = eos_density(c, phi[i]), p_i = eos_pressure(c, phi[i]);
  double gp[3] = {0, 0, 0}, lam[3] = {0, 0, 0}, av[3] = {0, 0, 0}, divu = 0.0;
  for (int64_t e = nb->row[i]; e < nb->row[i + 1]; ++e) {
    int64_t j = nb->col[e];
    double rij[3] = {0, 0, 0}, r2 = 0.0;
    for (int k = 0; k < d; ++k) {
      rij[k] = x[k * n + j] - x[k * n + i];
      r2 += rij[k] * rij[k];
    }
    double r = sqrt(r2);
    double dwdr = kernel_dwdr(d, h, r);
    double gw[3] = {0, 0, 0}; /* grad_i W_ij = dW/dr (x_i - x_j) / r */
    for (int k = 0; k < d; ++k) gw[k] = dwdr * (-rij[k]) / r;
    double vj = vol[j];
    double rho_j = eos_density(c, phi[j]), p_j = eos_pressure(c, phi[j]);
    double rgw = 0.0, uijxij = 0.0;
    for (int k = 0; k < d; ++k) {
      rgw += rij[k] * gw[k];
      /* (U_i - U_j).(x_i - x_j) */
      uijxij += (u[k * n + i] - u[k * n + j]) * (-rij[k]);
    }
    double pi_ij = 0.0;
    if (uijxij < 0.0) {
      double rho_bar = 0.5 * (rho_i + rho_j);
      pi_ij = -c->art_alpha * h * c->c0 * uijxij / (rho_bar * (r2 + 0.01 * h * h));
    }
    for (int k = 0; k < d; ++k) {
      double duk = u[k * n + j] - u[k * n + i];
      gp[k] += (p_i + p_j) * gw[k] * vj;
      divu += duk * gw[k] * vj;
      if (type[j] == FLUID || c->wall_bc == 1) lam[k] += duk * rgw / r2 * vj;
      av[k] += rho_j * vj * pi_ij * gw[k];
    }
  }
  for (int k = 0; k < d; ++k) {
    double visc = c->use_visc ? 2.0 * c->nu * lam[k] : 0.0;
    dudt[k] = -gp[k] / rho_i + visc - av[k] + G[k];
  }
  *dphidt = -eos_c2(c, phi[i]) * divu;
}

static int volumes(const orc_config* c, int64_t n, const double* phi, const double* mass,
                   double* vol) {
  for (int64_t i = 0; i < n; ++i) {
    double rho = eos_density(c, phi[i]);
    vol[i] = mass[i] / rho;
    if (!isfinite(vol[i])) return ORC_E_NAN;
  }
  return ORC_OK;
}

int orc_pair_sums(const orc_config* c, int64_t n, const double* x, const double* u,
                  const double* phi, const double* mass, const uint8_t* type, int all_types,
                  double* sums) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  double* vol = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!vol) return ORC_E_NOMEM;
  int rc = volumes(c, n, phi, mass, vol);
  csr_t nb = {0};
  if (!rc) rc = build_neighbors(c, n, x, 0, &nb);
  if (!rc) {
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
      if (!all_types && type[i] != FLUID) {
        memset(sums + i * ORC_NSUMS, 0, sizeof(double) * ORC_NSUMS);
        continue;
      }
      pair_sums_one(c, n, x, u, phi, vol, type, &nb, i, sums + i * ORC_NSUMS);
    }
  }
  csr_free(&nb);
  free(vol);
  return rc;
}

/* ---------------------------------------------------------------------------
 * Rates of one stage (Eq. sph with the TIC switch, viscosity and shifting):
 *   lambda_min(L) < tic_lambda with TIC on:  grad phi = C,     div U = tr M
 *   otherwise:                               grad phi = L^-1 S, div U = sum_ab (L^-1)_ab M_ab
 *   DU/Dt   = -grad phi + 2 nu Lambda + G(t)
 *   Dphi/Dt = -c^2 div U + delta h C0 D
 *   dUs     = -2 h U_max P,  dU = min(|dUs|, U_max/2) dUs / |dUs|
 * The corrected kernel gradient is L^-1 grad W (Eq. sph), so the corrected
 * divergence contracts L^-1 with M over both indices.
 * ------------------------------------------------------------------------- */
static int rates_from_sums(const orc_config* c, double phi_i, const double* s, double umax,
                           const double* G, double* dudt, double* dphidt, double* dushift,
                           double* lambda) {
  int d = c->dim;
  double h = c->h_over_dx * c->dx;
  const double *L = s, *S = s + 9, *M = s + 12, *C = s + 21, *P = s + 25, *Lam = s + 28;
  double D = s[24];
  double lam;
  orc_eig_min_sym(d, L, &lam);
  *lambda = lam;
  double gradphi[3] = {0, 0, 0}, divu = 0.0;
  if (c->use_tic && lam < c->tic_lambda) {
    for (int a = 0; a < d; ++a) {
      gradphi[a] = C[a];
      divu += M[a * 3 + a];
    }
  } else {
    double inv[9], det, amax = 0.0;
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b)
        if (fabs(L[a * 3 + b]) > amax) amax = fabs(L[a * 3 + b]);
    small_inverse(d, L, inv, &det);
    if (!(fabs(det) > 1e-12 * pow(amax, d))) return ORC_E_SINGULAR;
    for (int a = 0; a < d; ++a) {
      for (int b = 0; b < d; ++b) {
        gradphi[a] += inv[a * 3 + b] * S[b];
        divu += inv[a * 3 + b] * M[a * 3 + b];
      }
    }
  }
  for (int a = 0; a < d; ++a) {
    double visc = c->use_visc ? 2.0 * c->nu * Lam[a] : 0.0;
    dudt[a] = -gradphi[a] + visc + G[a];
  }
  double diff = c->use_delta ? c->delta * h * c->c0 * D : 0.0;
  *dphidt = -eos_c2(c, phi_i) * divu + diff;
  for (int a = 0; a < d; ++a) dushift[a] = 0.0;
  if (c->use_pst) {
    double du[3], nrm2 = 0.0;
    for (int a = 0; a < d; ++a) {
      du[a] = -2.0 * h * umax * P[a];
      nrm2 += du[a] * du[a];
    }
    double nrm = sqrt(nrm2);
    if (nrm > 0.0) {
      double mag = nrm < 0.5 * umax ? nrm : 0.5 * umax;
      for (int a = 0; a < d; ++a) dushift[a] = mag * du[a] / nrm;
    }
  }
  for (int a = 0; a < d; ++a)
    if (!isfinite(dudt[a]) || !isfinite(dushift[a])) return ORC_E_NAN;
  if (!isfinite(*dphidt)) return ORC_E_NAN;
  return ORC_OK;
}

static double fluid_umax(const orc_config* c, int64_t n, const double* u, const uint8_t* type) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (type[i] != FLUID) continue;
    double s = 0.0;
    for (int k = 0; k < c->dim; ++k) s += u[k * n + i] * u[k * n + i];
    double v = sqrt(s);
    if (v > m) m = v;
  }
  return m;
}

/* One stage: neighbours, dummy update, volumes, U_max, pair sums, rates.
 * Rates are written for fluid particles; dummy entries are zero. */
int orc_stage_rates(const orc_config* c, int64_t n, const double* x, double* u, double* phi,
                    const double* mass, const uint8_t* type, const double* normal, double t,
                    double* dudt, double* dphidt, double* dushift, double* lambda,
                    double* umax_out) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  int d = c->dim;
  csr_t nb = {0};
  int rc = build_neighbors(c, n, x, 0, &nb);
  if (rc) return rc;
  dummy_update_csr(c, n, x, u, phi, type, normal, t, &nb);
  double* vol = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!vol) { csr_free(&nb); return ORC_E_NOMEM; }
  rc = volumes(c, n, phi, mass, vol);
  double umax = c->umax_override >= 0 ? c->umax_override : fluid_umax(c, n, u, type);
  if (umax_out) *umax_out = umax;
  double G[3];
  body_force(c, t, G);
  if (!rc) {
    int err = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(min : err)
    for (int64_t i = 0; i < n; ++i) {
      double a[3], sh[3], dp = 0.0, lam = 0.0;
      if (type[i] != FLUID) {
        for (int k = 0; k < d; ++k) { dudt[k * n + i] = 0.0; dushift[k * n + i] = 0.0; }
        dphidt[i] = 0.0;
        lambda[i] = 0.0;
        continue;
      }
      int e = ORC_OK;
      if (c->scheme == 1) {
        conventional_rates_one(c, n, x, u, phi, vol, type, &nb, i, G, a, &dp);
        for (int k = 0; k < d; ++k) sh[k] = 0.0;
        for (int k = 0; k < d; ++k)
          if (!isfinite(a[k])) e = ORC_E_NAN;
        if (!isfinite(dp)) e = ORC_E_NAN;
      } else {
        double s[ORC_NSUMS];
        pair_sums_one(c, n, x, u, phi, vol, type, &nb, i, s);
        e = rates_from_sums(c, phi[i], s, umax, G, a, &dp, sh, &lam);
      }
      if (e < err) err = e;
      for (int k = 0; k < d; ++k) { dudt[k * n + i] = a[k]; dushift[k * n + i] = sh[k]; }
      dphidt[i] = dp;
      lambda[i] = lam;
    }
    rc = err;
  }
  free(vol);
  csr_free(&nb);
  return rc;
}

/* Time step: CFL * min(dx/(C0 + U_max), dx^2/(2 nu), sqrt(2 dx/|G|)); the
 * viscous (gravity) limit is skipped when nu (|G|) is zero. */
int orc_time_step(const orc_config* c, int64_t n, const double* u, const uint8_t* type,
                  double* dt) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  if (c->fixed_dt > 0) { *dt = c->fixed_dt; return ORC_OK; }
  double umax = fluid_umax(c, n, u, type);
  double ub = 0.0; /* the prescribed body speed also bounds the step */
  for (int k = 0; k < c->dim; ++k) ub += c->body_u[k] * c->body_u[k];
  ub = sqrt(ub);
  if (ub > umax) umax = ub;
  double t = c->dx / (c->c0 + umax);
  if (c->nu > 0) {
    double td = c->dx * c->dx / (2.0 * c->nu);
    if (td < t) t = td;
  }
  double g2 = 0.0;
  for (int k = 0; k < c->dim; ++k) g2 += c->g[k] * c->g[k];
  if (g2 > 0) {
    double tg = sqrt(2.0 * c->dx / sqrt(g2));
    if (tg < t) t = tg;
  }
  *dt = c->cfl * t;
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * SSP-RK2 (Sec. 2.3), fluid particles only; dummies stay fixed in space and
 * receive their potential and velocity from the dummy update of each stage.
 *   stage 1: y1 = yn + dt F(yn),       x1 = xn + dt (Un + dUn)
 *   stage 2: yn+1 = yn/2 + (y1 + dt F(y1))/2,
 *            xn+1 = xn/2 + (x1 + dt (U1 + dU1))/2
 * ------------------------------------------------------------------------- */
int orc_step(const orc_config* c, int64_t n, double* x, double* u, double* phi,
             const double* mass, const uint8_t* type, const double* normal, double* t,
             int64_t nsteps, double* dt_last, double* dudt, double* dphidt, double* dushift,
             double* lambda) {
  if (!valid_config(c) || n < 0 || nsteps < 0 || !t) return ORC_E_INVAL;
  if (c->umax_override >= 0) return ORC_E_INVAL; /* a full step computes U_max itself */
  int d = c->dim;
  size_t nd = (size_t)(n > 0 ? n : 1);
  double* x0 = (double*)malloc(sizeof(double) * nd * d);
  double* u0 = (double*)malloc(sizeof(double) * nd * d);
  double* p0 = (double*)malloc(sizeof(double) * nd);
  double* ra = (double*)malloc(sizeof(double) * nd * d);
  double* rp = (double*)malloc(sizeof(double) * nd);
  double* rs = (double*)malloc(sizeof(double) * nd * d);
  double* rl = (double*)malloc(sizeof(double) * nd);
  int rc = ORC_OK;
  if (!x0 || !u0 || !p0 || !ra || !rp || !rs || !rl) { rc = ORC_E_NOMEM; goto done; }
  for (int64_t step = 0; step < nsteps; ++step) {
    double dt;
    rc = orc_time_step(c, n, u, type, &dt);
    if (rc) goto done;
    memcpy(x0, x, sizeof(double) * (size_t)n * d);
    memcpy(u0, u, sizeof(double) * (size_t)n * d);
    memcpy(p0, phi, sizeof(double) * (size_t)n);
    /* stage 1 at time t */
    rc = orc_stage_rates(c, n, x, u, phi, mass, type, normal, *t, ra, rp, rs, rl, NULL);
    if (rc) goto done;
    for (int64_t i = 0; i < n; ++i) {
      if (type[i] == BODY) /* prescribed rigid translation, the same SSP-RK2 update */
        for (int k = 0; k < d; ++k) x[k * n + i] = x0[k * n + i] + dt * c->body_u[k];
      if (type[i] != FLUID) continue;
      for (int k = 0; k < d; ++k) {
        x[k * n + i] = x0[k * n + i] + dt * (u0[k * n + i] + rs[k * n + i]);
        u[k * n + i] = u0[k * n + i] + dt * ra[k * n + i];
      }
      phi[i] = p0[i] + dt * rp[i];
    }
    /* stage 2 at time t + dt */
    rc = orc_stage_rates(c, n, x, u, phi, mass, type, normal, *t + dt, ra, rp, rs, rl, NULL);
    if (rc) goto done;
    for (int64_t i = 0; i < n; ++i) {
      if (type[i] == BODY)
        for (int k = 0; k < d; ++k) x[k * n + i] = 0.5 * x0[k * n + i] + 0.5 * (x[k * n + i] + dt * c->body_u[k]);
      if (type[i] != FLUID) continue;
      for (int k = 0; k < d; ++k) {
        double x1 = x[k * n + i], u1 = u[k * n + i];
        x[k * n + i] = 0.5 * x0[k * n + i] + 0.5 * (x1 + dt * (u1 + rs[k * n + i]));
        u[k * n + i] = 0.5 * u0[k * n + i] + 0.5 * (u1 + dt * ra[k * n + i]);
      }
      phi[i] = 0.5 * p0[i] + 0.5 * (phi[i] + dt * rp[i]);
    }
    *t += dt;
    if (dt_last) *dt_last = dt;
  }
  if (dudt) memcpy(dudt, ra, sizeof(double) * (size_t)n * d);
  if (dphidt) memcpy(dphidt, rp, sizeof(double) * (size_t)n);
  if (dushift) memcpy(dushift, rs, sizeof(double) * (size_t)n * d);
  if (lambda) memcpy(lambda, rl, sizeof(double) * (size_t)n);
done:
  free(x0); free(u0); free(p0); free(ra); free(rp); free(rs); free(rl);
  return rc;
}

/* L2 spurious-velocity measure of Sec. 4.1 over fluid particles:
 * sqrt(sum |U_j|^2 V_j / sum V_j); also returns max |U|. */
int orc_l2_velocity(const orc_config* c, int64_t n, const double* u, const double* phi,
                    const double* mass, const uint8_t* type, double* l2, double* umax) {
  if (!valid_config(c) || n < 0) return ORC_E_INVAL;
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (type[i] != FLUID) continue;
    double v = mass[i] / eos_density(c, phi[i]);
    double s = 0.0;
    for (int k = 0; k < c->dim; ++k) s += u[k * n + i] * u[k * n + i];
    num += s * v;
    den += v;
  }
  *l2 = den > 0 ? sqrt(num / den) : 0.0;
  *umax = fluid_umax(c, n, u, type);
  return ORC_OK;
}
