/*
 * wbsph.h -- C-ABI of the GB300 (sm_103a) well-balanced WCSPH hot path.
 *
 * The library advances a set of SPH particles (fluid and fixed dummy wall
 * particles) with the well-balanced weakly compressible SPH method of Zhang,
 * Zhao, Gan and Xu: auxiliary potential phi with rho = rho0 exp(phi/C0^2)
 * (Sec. 2.2.1, Eq. newEqns), Riemann-based corrected gradient (Eqs. parGrad,
 * renorm, lfsover), delta-SPH diffusion, particle shifting and tensile
 * instability control (Sec. 2.3), the final semi-discrete system (Eq. sph),
 * SSP-RK2 with the three-condition time step (Sec. 2.3), and dummy-particle
 * slip walls (Sec. 2.4, Eq. phiBn). The neighbour build follows Sec. 3
 * (Eqs. hashid, ixyz; Algorithm 1): cell key, stable radix sort, reorder.
 *
 * Conventions (every function):
 *  - Return value: WBSPH_OK (0) or a negative wbsph_status. A message for
 *    the last failure of a handle is available from wbsph_last_error().
 *  - Arrays are structure-of-arrays: component k of particle i at [k*n + i],
 *    k < dim. Types: 0 fluid, 1 dummy.
 *  - Pointers are borrowed for the duration of the call. Host or device
 *    memory is selected by the `where` argument (WBSPH_HOST / WBSPH_DEVICE);
 *    device pointers must be on the handle's device.
 *  - Work is enqueued on the caller's CUDA stream (wbsph_config.cuda_stream,
 *    NULL = legacy default stream). Only wbsph_sync, the wbsph_get_* calls
 *    and wbsph_set_particles with host input synchronise that stream.
 *  - The handle owns its device memory, obtained from the caller's allocator
 *    callbacks when given, otherwise from cudaMallocAsync on the stream.
 *  - Device-side failures (particle outside the domain, singular
 *    renormalisation matrix with TIC off, non-finite value, neighbour list
 *    overflow) set a status word that is read at the next synchronising call.
 */
#ifndef WBSPH_H
#define WBSPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wbsph_s* wbsph_handle;

typedef enum {
  WBSPH_OK = 0,
  WBSPH_E_INVAL = -1,     /* bad argument or configuration */
  WBSPH_E_NOMEM = -2,     /* device allocation failed */
  WBSPH_E_CUDA = -3,      /* CUDA runtime error (message in wbsph_last_error) */
  WBSPH_E_DOMAIN = -4,    /* a particle left [domain_min, domain_max] */
  WBSPH_E_SINGULAR = -5,  /* renormalisation matrix singular and TIC off */
  WBSPH_E_NAN = -6,       /* a non-finite rate or state value */
  WBSPH_E_TIMEOUT = -7,   /* a bounded device-side wait gave up */
  WBSPH_E_STATE = -8,     /* call out of order (e.g. step before set_particles) */
  WBSPH_E_CAPACITY = -9,  /* output capacity too small / neighbour list overflow / list skin exceeded */
  WBSPH_E_NOSYM = -10     /* feature not built into this library */
} wbsph_status;
/* Conditions found on the device during a step are returned by the next
 * synchronising call. When several were flagged, the neighbour-list ones
 * come first (WBSPH_E_CAPACITY: a move beyond the skin of kept lists, or a
 * list overflow, more than 48 entries for a particle in 2D or 128 in 3D),
 * because every sum after them left pairs out; then WBSPH_E_NAN,
 * WBSPH_E_SINGULAR, WBSPH_E_DOMAIN and WBSPH_E_TIMEOUT. set_particles
 * clears them. */

/* Arithmetic of the pair pass (the state x, U, phi is FP64 in every mode):
 *  WBSPH_FP64  FP64 pair sums, the full potential (the reference arithmetic).
 *  WBSPH_MIXED FP32 pair sums with Kahan compensation on cell-relative
 *              offsets and the hydrostatic split phi - phi_hs (Eq. eqSol),
 *              FP64 epilogue: about 1e-5 of the field scale.
 *  WBSPH_DF64  double-float pair sums (pairs of FP32, about 48 bits) on
 *              offsets in cell units and the same hydrostatic split, FP64
 *              epilogue, Algorithm 1's exact FP64 neighbour test: FP64-level
 *              results on the FP32 pipe.
 * MIXED and DF64 sort once per step: stage 1 lists every pair within
 * 2h + 3 dt U* (U* = max(U_max, |body_u|), twice the largest move of a
 * particle in stage 1) and stage 2 reuses those lists with its own
 * neighbour test. Their cells are 2h + 3 CFL dx 0.3 / 1.3 wide (the skin of
 * a flow at Mach 0.3); a step whose skin would be wider (a faster flow, or
 * a fixed time step too long) returns WBSPH_E_CAPACITY at the next
 * synchronising call. They need grids of at most 2048 x 2048 x 1024 cells
 * (WBSPH_E_INVAL at the first stage otherwise), and DF64 sets the domain
 * status when a particle has moved more than half a cell since the last
 * neighbour build. */
typedef enum { WBSPH_FP64 = 0, WBSPH_MIXED = 1, WBSPH_DF64 = 2 } wbsph_precision;
typedef enum { WBSPH_HOST = 0, WBSPH_DEVICE = 1 } wbsph_where;

typedef enum {
  WBSPH_FIELD_X = 0,       /* dim*n positions */
  WBSPH_FIELD_U = 1,       /* dim*n velocities */
  WBSPH_FIELD_PHI = 2,     /* n potentials */
  WBSPH_FIELD_RHO = 3,     /* n densities from the EOS */
  WBSPH_FIELD_P = 4,       /* n pressures from the EOS */
  WBSPH_FIELD_DUDT = 5,    /* dim*n: DU/Dt of the last evaluated stage (fluid; 0 for dummies) */
  WBSPH_FIELD_DPHIDT = 6,  /* n: Dphi/Dt of the last evaluated stage */
  WBSPH_FIELD_DUSHIFT = 7, /* dim*n: shifting velocity dU of the last evaluated stage */
  WBSPH_FIELD_LAMBDA = 8,  /* n: lambda_min(L) of the last evaluated stage */
  WBSPH_FIELD_MASS = 9,    /* n masses */
  WBSPH_FIELD_VOL = 10     /* n volumes m/rho of the last evaluated stage */
} wbsph_field;

/* Optional allocator hooks (e.g. a framework's caching allocator). */
typedef void* (*wbsph_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*wbsph_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
  int dim;                  /* 2 or 3 */
  double dx;                /* initial particle spacing */
  double h_over_dx;         /* smoothing length h = h_over_dx * dx (paper: 1.5, Sec. 2.1) */
  double rho0;              /* reference density (paper: 1000, Sec. 4) */
  double c0;                /* artificial sound speed C0 (paper: 30, Sec. 4) */
  double nu;                /* kinematic viscosity (paper: 1e-4, Sec. 4) */
  double g[3];              /* body force G */
  double cfl;               /* CFL number (paper: 0.2, Sec. 2.3) */
  double delta;             /* delta-SPH coefficient (paper: 0.1, Sec. 2.3) */
  double pst_R, pst_n;      /* shifting constants R, n (paper: 0.2, 4, Sec. 2.3) */
  double tic_lambda;        /* surface / TIC threshold on lambda_min (paper: 0.75) */
  int use_delta, use_pst, use_tic, use_visc;
  int eos;                  /* 0: linear p = C0^2 (rho - rho0) (Eq. eos-water); 1: Tait */
  double tait_gamma;        /* Tait exponent (7) */
  double domain_min[3], domain_max[3]; /* grid extent; particles must stay inside */
  double force_amp[3];      /* harmonic tank displacement amplitude A: G(t) = G + A w^2 sin(w t) */
  double force_period;      /* forcing period; <= 0 disables */
  double fixed_dt;          /* > 0 replaces the adaptive time step */
  int precision;            /* wbsph_precision */
  int device;               /* CUDA device ordinal */
  void* cuda_stream;        /* cudaStream_t owned by the caller; NULL = default stream */
  wbsph_alloc_fn alloc;     /* NULL: cudaMallocAsync on cuda_stream */
  wbsph_free_fn free;
  void* alloc_ctx;
  double water_height;      /* free-surface height H of the hydrostatic split (mixed, df64) */
  int scheme;               /* WBSPH_SCHEME_WB (default): the well-balanced scheme, Eq. (sph);
                               WBSPH_SCHEME_CONVENTIONAL: conventional WCSPH (Sec. 2.1, Eq. nslag
                               with the printed operators, Eq. eos-water) plus artificial
                               viscosity, the foil of the hydrostatic comparison (Sec. 4.1).
                               The conventional scheme runs in FP64 with delta-SPH, shifting
                               and TIC off; anything else is WBSPH_E_INVAL. */
  double art_alpha;         /* conventional scheme: artificial-viscosity coefficient alpha of
                               Pi_ij = -alpha h C0 (U_ij.x_ij) / (rho_ij (r^2 + 0.01 h^2)) for
                               approaching pairs (default 0.02) */
  int wall_bc;              /* 0 (default): slip walls, U_d = U_f - ((U_f - U_w).n_d) n_d, viscous
                               interaction with fluid neighbours only (the paper's choice,
                               Sec. 2.4); 1: no-slip walls, U_d = 2 U_w - U_f (Eq. velBn), wall
                               particles included in the viscous sum */
  double body_u[3];         /* velocity of the body particles (type 2): they translate rigidly
                               with it and it is their wall velocity U_w (fixed walls: U_w = 0);
                               its magnitude also bounds the time step */
} wbsph_config;

typedef enum { WBSPH_SCHEME_WB = 0, WBSPH_SCHEME_CONVENTIONAL = 1 } wbsph_scheme;

typedef struct {
  int64_t n, n_fluid, n_dummy;
  int64_t ncells;           /* background grid cells (R = 2h) */
  int64_t grid[3];
  int64_t steps;            /* steps taken */
  int64_t launches;         /* kernels launched by this handle so far */
  int64_t device_bytes;     /* device memory held by the handle */
  double t, dt;             /* simulated time and last time step (after a sync) */
  int64_t pairs;            /* neighbour pairs summed by pair passes since set_particles */
} wbsph_stats;

/* Kernel classes timed when profiling is on (CUDA events on the stream). */
typedef enum {
  WBSPH_K_KEYS = 0, WBSPH_K_SORT = 1, WBSPH_K_REORDER = 2, WBSPH_K_CELLS = 3,
  WBSPH_K_PREPASS = 4, WBSPH_K_PAIR = 5, WBSPH_K_UPDATE = 6, WBSPH_K_OTHER = 7,
  WBSPH_K_NLIST = 8, /* candidate lists of the pair pass (k_nbr_list) */
  WBSPH_K_COUNT = 9
} wbsph_kernel_class;

/* Fill *cfg with the paper's constants (Sec. 4) for dimension dim. */
int wbsph_config_default(wbsph_config* cfg, int dim);

/* Create a handle; validates cfg and copies it. */
int wbsph_create(const wbsph_config* cfg, wbsph_handle* out);

/* Load n particles (Sec. 2.4: fluid and dummy). x, u, normal: dim*n SoA;
 * phi: n; mass: n or NULL (then m = rho(phi) dx^dim, the initial density
 * times the particle volume); type: n bytes (0 fluid, 1 dummy wall, 2 body wall); normal may
 * be NULL when there are no dummies. Sets t = 0. */
int wbsph_set_particles(wbsph_handle h, int64_t n, const double* x, const double* u,
                        const double* phi, const double* mass, const uint8_t* type,
                        const double* normal, int where);

/* Cell key, stable radix sort by key and reorder of all particle data, then
 * the per-cell index bounds (Sec. 3, Eqs. hashid/ixyz). */
int wbsph_build_neighbors(wbsph_handle h);

/* One rate evaluation at the current state and time: neighbour build, dummy
 * update, volumes, pair pass (Eq. sph). State is not advanced. */
int wbsph_eval_rates(wbsph_handle h);

/* Advance nsteps SSP-RK2 steps (two stages each; FP64 rebuilds the
 * neighbours per stage, MIXED and DF64 once per step, see wbsph_precision).
 * Asynchronous: errors surface at the next synchronising call. */
int wbsph_step(wbsph_handle h, int64_t nsteps);

/* One SSP-RK2 stage (Sec. 2.3) of a subdomain of a domain decomposition:
 * neighbour build, dummy walls at the stage's time, volumes, pair pass and
 * the stage's update, for every particle of the handle (the caller keeps
 * the results of the particles it owns and discards its ghosts'). The caller
 * gives the values that span subdomains: t, the time at the start of the
 * step (stage 2 runs at t + dt); umax, the stage's maximum fluid speed over
 * the whole domain (shifting; for stage 1 also the time step); dt > 0 the
 * step's time step, or dt <= 0 to compute it from umax in stage 1 (the
 * three-condition step) and to keep stage 1's in stage 2. Stage 2 must follow
 * stage 1 with no set_particles between (wbsph_update_particles may refresh
 * the ghosts). Asynchronous; WBSPH_E_STATE out of order. */
int wbsph_stage(wbsph_handle h, int stage, double t, double dt, double umax);

/* Overwrite x, U and phi of `count` particles identified by their index in
 * the last wbsph_set_particles input (host arrays; x and u SoA dim*count).
 * Between the stages of a domain decomposition this brings the ghosts to the
 * stage-1 state their owners computed. The ids must be distinct: for an id
 * given twice, which of its two rows is written is unspecified. An id not
 * below the particle count returns WBSPH_E_INVAL before anything is
 * written. Synchronises the stream. */
int wbsph_update_particles(wbsph_handle h, int64_t count, const uint32_t* ids, const double* x,
                           const double* u, const double* phi);

/* Wait for the handle's stream and read the device status word. */
int wbsph_sync(wbsph_handle h);

/* Copy one field out in the caller's original particle order: out holds
 * dim*n (x, U, DU/Dt, shift velocity; SoA) or n doubles, on the host
 * (where = WBSPH_HOST, pageable or pinned) or the device (WBSPH_DEVICE).
 * Synchronises the handle's stream once and reads the status word in the
 * same synchronisation: if a step since the last check set an error (NaN,
 * domain, singular, overflow, timeout) that code is returned and the
 * contents of out are unspecified. */
int wbsph_get_fields(wbsph_handle h, int field, double* out, int where);

/* Test hook: cell keys in sorted order and the original particle id at each
 * sorted position, from the last neighbour build (host arrays of n). */
int wbsph_get_cell_keys(wbsph_handle h, uint32_t* keys_sorted, uint32_t* ids_sorted);

/* Test hook: neighbour lists of every particle (d <= 2h, j != i, r > 0) in
 * CSR form over original ids, each row ascending. Returns the number of
 * entries (>= 0) or a negative status; row_ptr has n+1 entries; when cols is
 * NULL or cap is too small only row_ptr is written (then
 * WBSPH_E_CAPACITY is returned if cols was given). */
int64_t wbsph_get_neighbors(wbsph_handle h, int64_t* row_ptr, int32_t* cols, int64_t cap);

int wbsph_get_stats(wbsph_handle h, wbsph_stats* out);

/* Profiling: when on, CUDA events bracket each kernel class on the stream;
 * wbsph_get_profile returns total milliseconds and launch counts per class
 * (arrays of WBSPH_K_COUNT) accumulated since the last reset, and
 * synchronises the stream. */
int wbsph_set_profiling(wbsph_handle h, int on);
int wbsph_get_profile(wbsph_handle h, double* ms, int64_t* launches, int reset);

/* ---- learned surrogate (the paper has no learned part) ----------------
 * A message-passing network over the same neighbour lists predicts the
 * stage rates (DU/Dt, Dphi/Dt) of fluid particles. Node inputs: (U,
 * rho/rho0 - 1, phi') normalised, and a dummy flag, with the hydrostatic
 * split phi' = phi - phi_hs(x), phi_hs = G.x + |G| H (H the handle's water
 * height, as the mixed path); edge inputs: ((x_j - x_i)/h, |x_j - x_i|/h,
 * (U_j - U_i)/s_U, (phi'_j - phi'_i)/s_phi). Per layer the message of
 * receiver i is m_i = sum_j MLP_e([g_ij, h_i, h_j[:32]]) (a sender
 * contributes the first 32 of its 64 state features) and h_i += MLP_n([h_i,
 * m_i]); nothing is kept per edge, so inference allocates per node only.
 * Three layers, hidden width 64, BF16 weights and activations, FP32
 * accumulation on the tensor cores (tcgen05); trained on the GPU against
 * the plain FP64 rates of the states it is shown. Parameters are a flat
 * FP32 vector: blocks node encoder, (edge MLP, node MLP) per layer,
 * decoder; each W1 [in][64], b1 [64], W2 [64][out], b2 [out], row-major;
 * the edge MLP's W1 rows are the 2 dim + 2 edge inputs, then h_i (64), then
 * h_j[:32].
 * This interface departs from a load-from-file / train-from-a-directory
 * pair: parameters and normalisation are set from host arrays, and
 * training is one step at a time on a state the caller loads, so that the
 * caller owns files, datasets and schedules. */
enum { WBSPH_SURROGATE_NETWORK = 0, WBSPH_SURROGATE_FROZEN = 1 };
typedef struct wbsph_surrogate_s* wbsph_surrogate;
typedef struct {
  int dim;            /* 2 or 3 */
  int hidden;         /* 64 */
  int layers;         /* message-passing layers (3) */
  float beta1, beta2, eps;  /* Adam */
  int device;
} wbsph_surrogate_config;

typedef struct {
  int64_t surrogate_steps, plain_steps, anchors, fallbacks;
  double last_rel_err;   /* relative L2 of surrogate vs plain DU/Dt at the last anchor */
  double max_rel_err;
} wbsph_anchor_stats;

int wbsph_surrogate_config_default(wbsph_surrogate_config* cfg, int dim);
int wbsph_surrogate_create(const wbsph_surrogate_config* cfg, wbsph_surrogate* out);
int64_t wbsph_surrogate_num_params(wbsph_surrogate s);
/* host FP32 arrays of wbsph_surrogate_num_params() values */
int wbsph_surrogate_set_params(wbsph_surrogate s, const float* params);
int wbsph_surrogate_get_params(wbsph_surrogate s, float* params);
/* node mean/std: dim+2 values (U, rho/rho0-1, phi'); edge_std: 2 values
 * (s_U, s_phi) of the edge inputs; output mean/std: dim+1. Host arrays. */
int wbsph_surrogate_set_normalization(wbsph_surrogate s, const float* node_mean, const float* node_std,
                                      const float* edge_std, const float* out_mean, const float* out_std);
/* WBSPH_SURROGATE_NETWORK (default): the network predicts the rates.
 * WBSPH_SURROGATE_FROZEN: a control for measuring what the network gains:
 * surrogate stages reuse, per particle, the rates of the last plain stage of
 * the rollout (wbsph_step_surrogate only; train, eval and debug need the
 * network mode and return WBSPH_E_STATE otherwise). */
int wbsph_surrogate_set_mode(wbsph_surrogate s, int mode);
/* One training step on the sim's current state: plain FP64 rates as targets,
 * forward, MSE loss on normalised outputs, backward, Adam with rate lr.
 * Synchronises; *loss (nullable) receives the loss before the update. */
int wbsph_surrogate_train_step(wbsph_surrogate s, wbsph_handle h, float lr, double* loss);
/* Loss on the sim's current state without an update. */
int wbsph_surrogate_eval(wbsph_surrogate s, wbsph_handle h, double* loss);
/* Surrogate stage rates at the sim's current state into its rate fields
 * (WBSPH_FIELD_DUDT / DPHIDT; DUSHIFT set to zero). */
int wbsph_surrogate_predict(wbsph_surrogate s, wbsph_handle h);
/* Test hook: graph, features, outputs and loss gradient of the sim's
 * current state, all host arrays; ids are original particle ids. Call with
 * null arrays first to get *n_edges. out: n_fluid*(dim+1) normalised outputs
 * in the order of fluid_ids; grad: num_params; node_feat: n*8; edge_feat:
 * n_edges*8 (BF16 values as float). */
int wbsph_surrogate_debug(wbsph_surrogate s, wbsph_handle h, int64_t* n_edges, uint32_t* recv_ids,
                          uint32_t* send_ids, float* edge_feat, float* node_feat, uint32_t* fluid_ids,
                          float* out, float* grad, double* loss);
/* Advance nsteps SSP-RK2 steps with surrogate rates; every anchor_every-th
 * step, starting with the first, is a plain FP64 step (an anchor), and at
 * each anchor the surrogate's DU/Dt is compared with the plain one on the
 * same state (relative L2 over fluid). If it exceeds tau the next window
 * runs plain (fallback). anchor_every = 0: no anchors. Synchronises. */
int wbsph_step_surrogate(wbsph_handle h, wbsph_surrogate s, int64_t nsteps, int anchor_every, double tau,
                         wbsph_anchor_stats* stats);
void wbsph_surrogate_destroy(wbsph_surrogate s);
const char* wbsph_surrogate_last_error(wbsph_surrogate s);

/* Cell keys and stable sort without any device allocation. The paper has no
 * counterpart: this is a variant of the neighbour build's key and radix-sort
 * kernels for callers that cannot let a library allocate device memory (a
 * framework that owns the device memory pool, or a loop that cannot afford
 * the implicit synchronisation of cudaMalloc/cudaFree).
 * x: device pointer, dim*n SoA positions; keys_sorted, ids_sorted: device
 * arrays of n, written with the sorted cell keys and, for each sorted
 * position, the input index (the same result as wbsph_build_neighbors +
 * wbsph_get_cell_keys on particles loaded in that order). The grid comes
 * from h's configuration; h needs no wbsph_set_particles, and the handle's
 * stream is used and synchronised before returning. The call runs on h's
 * device and restores the caller's current device before it returns.
 * The pointers are not checked beyond NULL: x must hold dim*n doubles and
 * each output n 32-bit words, all on h's device (the Python binding checks
 * this on the tensors before calling).
 * Scratch lives in a file-scope device array sized for WBSPH_NOALLOC_MAX_N
 * particles (4.3 MB, held by every GPU that loads the library until
 * the process exits); larger n returns WBSPH_E_CAPACITY. The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) for
 * that device and keeps it until the process exits, so a device reset
 * (cudaDeviceReset) after that first call is not supported. The call
 * synchronises its stream and reads the status word back to the host, so it
 * must not be called while that stream is being captured into a CUDA graph.
 * All calls share the array: calls that overlap on the GPU (other threads or
 * streams) race and must be serialised by the caller. Returns WBSPH_E_DOMAIN
 * if a particle lies outside the domain. */
#define WBSPH_NOALLOC_MAX_N 524288
int wbsph_sort_cells_noalloc(wbsph_handle h, const double* x, int64_t n, uint32_t* keys_sorted,
                             uint32_t* ids_sorted);

/* Check of the bounded device waits (failure detection without a GPU fault):
 * launches two warps that use the waits of the surrogate's fused layer. The
 * first waits, with at most `limit` polls (1 .. 2^20), on an mbarrier that
 * nothing arrives on, and raises the block's abort flag when the limit runs
 * out. The second waits on another such mbarrier with a 64 times longer
 * limit and must leave as soon as it sees the flag, as the layer's roles
 * do when one of them times out. Only when both happen does the probe set
 * the status word; the call then synchronises and returns WBSPH_E_TIMEOUT
 * (the status stays set until the next wbsph_set_particles), else
 * WBSPH_OK. The context stays usable. Requires loaded particles; a limit
 * out of range returns WBSPH_E_INVAL. */
int wbsph_test_bounded_wait(wbsph_handle h, int64_t limit);

void wbsph_destroy(wbsph_handle h);
const char* wbsph_last_error(wbsph_handle h);
const char* wbsph_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
