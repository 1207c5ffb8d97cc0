// common.cuh -- shared definitions of the sm_103a well-balanced WCSPH kernels.
//
// Layout in HBM: structure-of-arrays, one array per component, particles in
// the order of the last neighbour build (cell-key order). Every per-particle
// array of the state is double-buffered so that the reorder of Sec. 3 is a
// gather into the second buffer followed by a pointer swap.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wbsph {

constexpr int kFluid = 0;
constexpr int kDummy = 1;
constexpr int kBody = 2;  // wall particle of the rigid body translating with Params::body_u
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// Device status word bits (read by the host at synchronising calls).
enum : unsigned {
  kStatDomain = 1u,     // particle outside the grid
  kStatSingular = 2u,   // singular renormalisation matrix on the corrected branch
  kStatNaN = 4u,        // non-finite rate or state
  kStatOverflow = 8u,   // a neighbour list had more entries than it holds
  kStatTimeout = 16u,   // bounded device wait gave up
  kStatSkin = 32u       // a particle may move further in a stage than the reused lists allow
};

// Numerical parameters, derived once on the host from the configuration and
// passed to kernels by value.
struct Params {
  int dim;
  int eos;              // 0 linear, 1 Tait
  int use_delta, use_pst, use_tic, use_visc;
  double dx, h, two_h, four_h2;   // four_h2 = (2h)*(2h), the Algorithm 1 test
  float prefilter_r2;             // FP32 candidate threshold, >= (2h)^2 plus a rounding margin
  double alpha;                   // kernel normalisation (Eq. c2kernel)
  double neg_dwdr_over_r_coef;    // -W'(r)/r = coef * (1 - q/2)^3, coef = 5 alpha / h^2
  double inv_two_h;               // 1/(2h): (1 - q/2) = 1 - r/(2h)
  double two_over_h;              // 2q + 1 = 1 + r * 2/h
  double pst_alpha_over_wdx;      // alpha / W(dx), for W_ij / W(dx)
  double pst_R, pst_n;
  double pst_R_a4;                // pst_R * pst_alpha_over_wdx^4
  double rho0, c0, c0sq, nu, gamma;
  float inv_c0sq_f, inv_rho0_f;   // 1/C0^2 and 1/rho0 rounded to FP32 (the mixed prepass)
  double delta_h_c0;              // delta * h * C0
  double tic_lambda;
  double g[3];
  double force_amp[3];
  double omega;                   // 2 pi / period, 0 = no forcing
  double cfl, fixed_dt;
  float nearest_band_r2;          // FP32 band around the FP32 minimum that holds the exact nearest
  float inner_r2;                 // FP32 r^2 at or below it (and > 0): an exact neighbour, no FP64 test
  double domain_min[3], domain_max[3];
  double R;                       // cell size: 2h, plus skin_max on the mixed and double-float paths
  double inv_R;                   // 1 / R
  // Mixed and double-float paths: the candidate lists of stage 1 are kept for stage 2. They
  // hold every pair within 2h + delta, delta = 3 dt U* (U* = max(U_max,
  // |body_u|)), twice the largest move of a particle in stage 1 (U0 plus a
  // shift clamped to U_max/2, times dt), so that every pair within 2h at the
  // stage-2 positions is listed; cells are widened by skin_max >= delta so
  // that the listed pairs and the wall update's nearest fluid particle stay
  // in adjacent cells without a new sort.
  int skin;                       // 1: lists kept for stage 2 (mixed and double-float paths)
  double skin_max;                // largest delta the cells allow
  double skin_e;                  // FP32 rounding margin of a list distance
  // cell keys: FP32 estimate of (x - min)/R, trusted where its fractional
  // part is more than key_margin from a cell boundary (exact FP64 otherwise)
  float key_min_f[3];             // domain_min rounded to FP32
  float key_inv_R_f;              // 1/R rounded to FP32
  float key_margin[3];            // twice the bound on |estimate - FP64 quotient|, per axis
  long long key_lo[3], key_hi[3]; // order-preserving integer images of domain_min, domain_max
  int nc[3];                      // grid cells per axis
  int64_t ncells;
  double water_height;
  double phs0;  // |G| H: hydrostatic potential at height zero (phi_hs = G.x + |G| H)
  int scheme;          // 0 well-balanced, 1 conventional WCSPH (the hydrostatic foil)
  double art_ahc0;     // conventional scheme: alpha h C0 of the artificial viscosity
  double avis_eps2;    // 0.01 h^2
  int wall_bc;         // 0 slip walls, 1 no-slip walls (Eq. velBn)
  double body_u[3];    // velocity of the body particles
  double body_speed;   // |body_u|: bounds the time step
  float df_c0[2];      // double-float path: C0 and R_pst (alpha / W(dx))^4 as hi + lo
  float df_pst_Ra4[2];
  float df_4h2_R2[2];  // double-float path: (2h / R)^2 as hi + lo (kept lists' exact test)
  float df_R_2h[2];    // double-float path: R / 2h as hi + lo (1 when the cells are 2h wide)
};

// Device arrays of one particle-state buffer.
struct State {
  double* x;        // dim * n
  double* u;        // dim * n
  double* phi;      // n
  double* x0;       // dim * n: stage-start state y^n (SSP-RK2)
  double* u0;       // dim * n
  double* phi0;     // n
  double* mass;     // n
  double* normal;   // dim * n
  uint8_t* type;    // n
  uint32_t* oid;    // n: original particle id
};

// Rates and per-stage scratch (not reordered: recomputed every stage).
struct Work {
  double* dudt;      // dim * n
  double* dphidt;    // n
  double* dushift;   // dim * n
  double* lambda;    // n
  double* Lmat;      // 3n (2D) or 6n (3D): L of the last FP64 pair pass (upper triangle, SoA)
  double* vol;       // n
  double* rho;       // n: densities of the stage (conventional scheme only)
  double* pres;      // n: pressures of the stage (conventional scheme only)
  double* volc;      // n: 5 alpha / h^2 * V, so that -W'(r)/r V = volc (1 - q/2)^3
  float4* xf;        // n: FP32 copy of positions (.w = type) for the candidate prefilter
  uint32_t* key;     // n: sorted cell keys
  uint32_t* key_alt; // n
  uint32_t* perm;    // n: source index of each sorted position
  uint32_t* perm_alt;
  uint32_t* cell_lb; // ncells + 1: first sorted index with key >= c
  uint32_t* fluid_list;  // n_fluid: sorted indices of fluid particles
  float4* xff;           // n_fluid: xf of the fluid particles, in fluid_list order
  uint32_t* fkey;        // n_fluid: their cell keys
  uint32_t* fcell_lb;    // ncells + 1: first fluid_list position with key >= c
  uint32_t* dummy_list;  // n_dummy: sorted indices of dummy particles
  uint32_t* block_cnt;   // scratch for scans
  uint32_t* hist;        // radix histograms
  unsigned long long* umax_bits;  // [0]: max |U|^2 over fluid (bits of a non-negative double)
  double* scalars;   // [0] t, [1] dt, [2] unused, [3] FP32 candidate threshold of the kept lists
  unsigned* status;  // device status word
  unsigned long long* pairs;  // [0]: neighbour pairs summed by pair passes (units of work)
  uint32_t* nbr;     // kmax * n_fluid: candidate lists, k-major (nbr[k * nf + gi])
  uint32_t* nbr_cnt; // n_fluid: candidates per fluid particle
  float4* packA;     // n: mixed path, (cell-relative offset, phi - phi_hs) in FP32;
                     //    double-float path, high parts of (offset / R, phi - phi_hs)
  float4* packB;     // n: mixed path, (U, +-V) in FP32; double-float path, high parts of (U, +-volc)
  uint32_t* packC;   // n: mixed and double-float paths, cell coordinates packed 11/11/10 bits
  float4* packAl;    // n: double-float path, low parts of packA (packA/packB hold the high parts)
  float4* packBl;    // n: double-float path, low parts of packB
  double* cell_origin;  // mixed and double-float paths: domain_min[k] + i R for the cells of axis k, axes one after
                        // another (nc[0] + nc[1] + nc[2] entries)
};

__host__ __device__ inline int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- launchers (neighbors.cu) ----
int radix_sort_scratch_words(int64_t n);
void launch_cell_keys(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st);
void launch_radix_sort(const Params& p, Work& w, int64_t n, cudaStream_t st, int* launches);
void launch_gather(const Params& p, const State& src, const State& dst, const Work& w, int64_t n,
                   bool with_base, cudaStream_t st);
void launch_cell_bounds(const Params& p, const Work& w, int64_t n, cudaStream_t st);
void launch_fluid_list(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int64_t nd,
                       cudaStream_t st, int* launches);
void launch_count_neighbors(const Params& p, const State& s, const Work& w, int64_t n,
                            uint32_t* counts, cudaStream_t st);
void launch_fill_neighbors(const Params& p, const State& s, const Work& w, int64_t n,
                           const int64_t* row_ptr_by_oid, int32_t* cols, cudaStream_t st);

// ---- prepass.cu ----
// U_max^2 of the fluid particles alone (after launch_prepass without volumes)
void launch_umax(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st);
// Dummy walls, then (volumes = true) V = m / rho and U_max of the stage.
void launch_prepass(const Params& p, const State& s, const Work& w, int64_t n, int64_t nd,
                    int stage2, cudaStream_t st, bool volumes = true);
// keep_lists: also the radius of the mixed path's kept lists (and the check
// that the widened cells hold it)
void launch_time_step(const Params& p, const Work& w, cudaStream_t st, bool keep_lists = false);
// Mixed path: V, U_max and the packed FP32 copies; WBSPH_E_INVAL when the
// grid exceeds the packed cell word (2048 x 2048 x 1024 cells).
int launch_prepass_mixed(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st);
// Double-float path: the hi/lo copies (after launch_prepass); the same grid limit.
int launch_pack_df(const Params& p, const State& s, const Work& w, int64_t n, cudaStream_t st);

// ---- lists.cu ----
int pair_list_kmax(int dim);
// exact: FP64 neighbour sets (FP64 path, surrogate graph); skin: the mixed
// path's lists of stage 1, kept for stage 2 (radius 2h + delta)
void launch_nbr_list(const Params& p, const State& s, const Work& w, int64_t n, int64_t n_fluid, cudaStream_t st,
                     bool exact, bool skin = false);

// ---- pair passes: pair_fp64.cu, pair_mixed.cu, pair_df64.cu, pair_conventional.cu ----
void launch_pair_fp64(const Params& p, const State& s, const Work& w, int64_t n, int64_t n_fluid,
                      int stage2, cudaStream_t st);
void launch_lambda_fp64(const Params& p, const Work& w, int64_t n, int64_t nf, cudaStream_t st);
void launch_pair_mixed(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int stage2,
                       cudaStream_t st);
// kept: the lists are the kept lists of radius 2h + delta (the pass applies
// the exact test); otherwise every entry is an exact neighbour
void launch_pair_df(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int stage2,
                    cudaStream_t st, bool kept = false);
void launch_pair_conventional(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf,
                              int stage2, cudaStream_t st);

// ---- update.cu ----
void launch_rk_stage(const Params& p, const State& s, const Work& w, int64_t n, int stage,
                     cudaStream_t st);
void launch_field(const Params& p, const State& s, const Work& w, int64_t n, int field,
                  double* out, cudaStream_t st);
// FP32 position copies (xf, and xff of the fluid particles) brought to the
// current positions of the fluid and body particles, in the order of the
// last neighbour build (mixed path, stage 2 without a new build)
void launch_refresh_xf(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int64_t nd,
                       cudaStream_t st);

}  // namespace wbsph
