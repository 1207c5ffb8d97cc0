/*
 * wbsph_oracle.h -- plain FP64 CPU oracle of the well-balanced WCSPH step.
 *
 * TEST INFRASTRUCTURE ONLY. This library states, slowly and literally, what
 * the per-timestep particle-interaction path of the well-balanced weakly
 * compressible SPH method (Zhang, Zhao, Gan, Xu) computes. Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may call it. It
 * shares no code, header, helper or constant with the CUDA library.
 *
 * Passages followed (section / equation of the paper):
 *   kernel ............ Sec. 2.1, Eq. (c2kernel); 3D normalisation 21/(16 pi h^3)
 *   potential form .... Sec. 2.2.1, Eq. (newEqns); rho = rho0 exp(phi/C0^2)
 *   Riemann gradient .. Sec. 2.2.2, Eqs. (parGrad), (renorm), (lfsover)
 *   stabilisers ....... Sec. 2.3: delta-SPH diffusion, particle shifting, TIC
 *   final system ...... Eq. (sph)
 *   time integration .. SSP-RK2 stages and the three-condition time step
 *   walls ............. Sec. 2.4, Eq. (phiBn) and the slip velocity condition
 *   neighbours ........ Sec. 3, Eqs. (hashid), (ixyz), Algorithm 1 (d <= 2h)
 *   conventional foil . Sec. 2.1, Eq. (nslag), Eq. (eos-water), the printed operators
 *                        <div U>, <grad p>, <lap U>; artificial viscosity (Monaghan form)
 *
 * Layouts: positions, velocities and normals are structure-of-arrays,
 * component k of particle i at [k*n + i]. Types: 0 fluid, 1 dummy (fixed wall),
 * 2 body (a wall particle translating with the prescribed velocity body_u).
 * Every function returns 0 on success or a negative ORC_E_* code.
 */
#ifndef WBSPH_ORACLE_H
#define WBSPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_E_INVAL = -1,
  ORC_E_NOMEM = -2,
  ORC_E_DOMAIN = -4,
  ORC_E_SINGULAR = -5,
  ORC_E_NAN = -6,
  ORC_E_CAP = -9
};

typedef struct {
  int dim;                 /* 2 or 3 */
  double dx;               /* initial particle spacing */
  double h_over_dx;        /* h = h_over_dx * dx */
  double rho0;             /* reference density */
  double c0;               /* artificial sound speed C0 */
  double nu;               /* kinematic viscosity */
  double g[3];             /* constant body force G */
  double cfl;              /* CFL number of the time step */
  double delta;            /* delta-SPH coefficient */
  double pst_R, pst_n;     /* particle-shifting constants R and n */
  double tic_lambda;       /* surface / TIC threshold on lambda_min(L) */
  int use_delta, use_pst, use_tic, use_visc;
  int eos;                 /* 0: linear p = C0^2 (rho - rho0); 1: Tait */
  double tait_gamma;
  double domain_min[3], domain_max[3];
  double force_amp[3];     /* tank displacement amplitude A (harmonic forcing) */
  double force_period;     /* forcing period T; <= 0 disables the forcing */
  double fixed_dt;         /* > 0 replaces the adaptive time step */
  double umax_override;    /* >= 0: U_max used by shifting in orc_stage_rates (an input
                              when rates are evaluated on a patch of a larger scene);
                              < 0: computed from the particles */
  int scheme;              /* 0: well-balanced WCSPH (Eq. sph); 1: conventional WCSPH
                              (Eq. nslag with the printed operators and artificial
                              viscosity), the foil of the hydrostatic comparison; it
                              takes no delta-SPH, shifting or TIC */
  double art_alpha;        /* artificial-viscosity coefficient of the conventional scheme */
  int wall_bc;             /* 0: slip walls (Sec. 2.4, the paper's choice); 1: no-slip walls,
                              Eq. (velBn) U_d = 2 U_w - U_f, with the viscous interaction of
                              fluid particles with wall particles included */
  double body_u[3];        /* velocity of the moving wall particles (type 2): they translate
                              rigidly with it, and it is their wall velocity U_w */
} orc_config;

/* Number of doubles per particle written by orc_pair_sums:
 * L (9, row-major 3x3), S (3), M (9), C (3), D (1), P (3), Lambda (3). */
#define ORC_NSUMS 31

int orc_kernel_eval(const orc_config* c, int64_t m, const double* r, double* w, double* dwdr);
int orc_cell_keys(const orc_config* c, int64_t n, const double* x, uint32_t* key);
int orc_sort_by_key(int64_t n, const uint32_t* key, uint32_t* perm);
int64_t orc_neighbors(const orc_config* c, int64_t n, const double* x, int brute,
                      int64_t* row_ptr, int32_t* cols, int64_t cap);
int orc_mass(const orc_config* c, int64_t n, const double* phi, double* mass);
int orc_density(const orc_config* c, int64_t n, const double* phi, double* rho);
int orc_pressure(const orc_config* c, int64_t n, const double* phi, double* p);
int orc_eig_min_sym(int dim, const double* a, double* lam);
int orc_dummy_update(const orc_config* c, int64_t n, const double* x, double* u, double* phi,
                     const uint8_t* type, const double* normal, double t);
int orc_pair_sums(const orc_config* c, int64_t n, const double* x, const double* u,
                  const double* phi, const double* mass, const uint8_t* type,
                  int all_types, double* sums);
int orc_stage_rates(const orc_config* c, int64_t n, const double* x, double* u, double* phi,
                    const double* mass, const uint8_t* type, const double* normal, double t,
                    double* dudt, double* dphidt, double* dushift, double* lambda,
                    double* umax_out);
int orc_time_step(const orc_config* c, int64_t n, const double* u, const uint8_t* type,
                  double* dt);
int orc_step(const orc_config* c, int64_t n, double* x, double* u, double* phi,
             const double* mass, const uint8_t* type, const double* normal, double* t,
             int64_t nsteps, double* dt_last, double* dudt, double* dphidt, double* dushift,
             double* lambda);
int orc_l2_velocity(const orc_config* c, int64_t n, const double* u, const double* phi,
                    const double* mass, const uint8_t* type, double* l2, double* umax);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
