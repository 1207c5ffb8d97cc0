// engine.cu -- the C-ABI of include/wbsph.h: handle, device buffers, stage
// sequencing on the caller's stream, status word, profiling events.
//
// One SSP-RK2 step (Sec. 2.3) is enqueued as, per stage s = 1, 2:
//   keys -> radix sort -> gather (reorder) -> cell bounds -> fluid list   (Sec. 3)
//   prepass: dummy walls (Sec. 2.4), volumes, U_max
//   [s = 1] time step from U_max of y^n
//   neighbour lists, fused pair pass + epilogue (Eq. sph)
//   RK stage update
// with no host synchronisation inside a step. The mixed and double-float
// paths sort once per step: stage 2 keeps stage 1's order, cells and lists
// (built with radius 2h + 3 dt U*, on cells widened for that skin).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wbsph.h"
#include "common.cuh"

using namespace wbsph;

namespace wbsph {
void launch_mass(const Params& p, const double* phi, double* mass, int64_t n, cudaStream_t st);
void launch_wait_probe(unsigned* status, uint32_t limit, cudaStream_t st);
}

struct ProfEvent {
  int cls;
  cudaEvent_t a, b;
};

struct wbsph_s {
  wbsph_config cfg;
  Params P;
  cudaStream_t stream = nullptr;
  int64_t n = 0, nf = 0, nd = 0;
  State A{}, B{};
  Work W{};
  std::vector<void*> blocks;
  int64_t device_bytes = 0;
  int64_t launches = 0, steps = 0;
  bool loaded = false;
  bool alloc_failed = false;
  bool use_graphs = true;            // replay captured steps (caller stream only)
  // Captured steps, each with the buffer pointers it starts from and leaves
  // behind. A step of the FP64 and double-float paths sorts twice and
  // leaves every pointer where it found it, so one graph serves every step;
  // a mixed-path step sorts once, so its pointers alternate between two
  // states and a graph is kept for each.
  struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    State a0{}, b0{}, a1{}, b1{};
    Work w0{}, w1{};
    int64_t launches = 0;              // kernels in the captured step
  } graphs[2];
  int64_t steps_since_load = 0;
  bool capturing = false;
  int64_t n_alloc = -1;  // particle count the buffers were sized for
  std::string err;
  bool prof = false;
  std::vector<ProfEvent> events, pool;
  double prof_ms[WBSPH_K_COUNT] = {0};
  int64_t prof_cnt[WBSPH_K_COUNT] = {0};
  double* field_tmp = nullptr;       // device: a field in the caller's order, on its way to the host
  unsigned* status_host = nullptr;   // pinned host copy of the status word
  // distributed stages (wbsph_stage): host values copied to the device, the
  // last stage run since set_particles, and whether a time step is in place
  double dist_host[3] = {0.0, 0.0, 0.0};
  int dist_stage = 0;
  double dist_dt = 0.0;
};

static const char* kStatusNames[] = {"ok", "invalid argument", "out of device memory",
                                     "CUDA error", "particle outside the domain",
                                     "singular renormalisation matrix", "non-finite value",
                                     "device wait timed out", "call out of order",
                                     "capacity too small", "feature not built"};

extern "C" const char* wbsph_status_string(int s) {
  if (s > 0 || s < -10) return "unknown status";
  return kStatusNames[-s];
}

static int fail(wbsph_s* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  return code;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, WBSPH_E_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));      \
  } while (0)

static int check_launch(wbsph_s* h, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, WBSPH_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return WBSPH_OK;
}

// ---- profiling: CUDA events around each kernel class on the stream ----
static void prof_begin(wbsph_s* h, int cls, ProfEvent* out) {
  if (!h->prof) return;
  ProfEvent e;
  if (!h->pool.empty()) {
    e = h->pool.back();
    h->pool.pop_back();
  } else {
    cudaEventCreate(&e.a);
    cudaEventCreate(&e.b);
  }
  e.cls = cls;
  cudaEventRecord(e.a, h->stream);
  *out = e;
}

static void prof_end(wbsph_s* h, ProfEvent* e) {
  if (!h->prof) return;
  cudaEventRecord(e->b, h->stream);
  h->events.push_back(*e);
}

struct ProfScope {
  wbsph_s* h;
  ProfEvent e;
  ProfScope(wbsph_s* h_, int cls) : h(h_) { prof_begin(h, cls, &e); }
  ~ProfScope() { prof_end(h, &e); }
};

// ---- allocation ----
static void* dev_alloc(wbsph_s* h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (h->cfg.alloc) {
    p = h->cfg.alloc(bytes, (void*)h->stream, h->cfg.alloc_ctx);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    p = nullptr;
  }
  if (p) {
    h->blocks.push_back(p);
    h->device_bytes += (int64_t)bytes;
  } else {
    cudaGetLastError();
    h->alloc_failed = true;
  }
  return p;
}

static void free_all(wbsph_s* h) {
  for (void* p : h->blocks) {
    if (h->cfg.free) h->cfg.free(p, (void*)h->stream, h->cfg.alloc_ctx);
    else cudaFreeAsync(p, h->stream);
  }
  h->blocks.clear();
  h->device_bytes = 0;
  h->alloc_failed = false;
  h->n_alloc = -1;
  h->A = State{};
  h->B = State{};
  h->W = Work{};
}

// ---- parameters ----
static const double kPi = 3.14159265358979323846;

// Integer image of a double that orders like the value (-0 maps to +0, NaN
// outside the images of all numbers); the same map as the cell-key kernel's.
static long long ordered_bits(double v) {
  long long b;
  memcpy(&b, &v, 8);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return b < 0 ? b ^ 0x7FFFFFFFFFFFFFFFLL : b;
}

static int derive_params(wbsph_s* h) {
  const wbsph_config& c = h->cfg;
  Params& p = h->P;
  memset(&p, 0, sizeof p);
  p.dim = c.dim;
  p.eos = c.eos;
  p.use_delta = c.use_delta;
  p.use_pst = c.use_pst;
  p.use_tic = c.use_tic;
  p.use_visc = c.use_visc;
  p.dx = c.dx;
  p.h = c.h_over_dx * c.dx;
  p.two_h = 2.0 * p.h;
  p.four_h2 = p.two_h * p.two_h;
  p.R = p.two_h;
  // Mixed and double-float paths: lists kept for stage 2 (see
  // Params::skin). The cells are widened by the largest skin that a flow at
  // Mach 0.3 needs at this CFL number: a particle moves at most 1.5 dt U_max
  // in stage 1 and dt <= CFL dx / (C0 + U_max).
  p.skin = (c.precision == WBSPH_MIXED || c.precision == WBSPH_DF64) ? 1 : 0;
  if (p.skin) {
    const double mach = 0.3;
    p.skin_max = 3.0 * c.cfl * c.dx * mach / (1.0 + mach);
    p.R = p.two_h + p.skin_max;
  }
  p.inv_R = 1.0 / p.R;
  p.alpha = c.dim == 2 ? 7.0 / (4.0 * kPi * p.h * p.h) : 21.0 / (16.0 * kPi * p.h * p.h * p.h);
  p.neg_dwdr_over_r_coef = 5.0 * p.alpha / (p.h * p.h);
  p.inv_two_h = 1.0 / p.two_h;
  p.two_over_h = 2.0 / p.h;
  double q = c.dx / p.h, tq = 1.0 - 0.5 * q;
  p.pst_alpha_over_wdx = 1.0 / (tq * tq * tq * tq * (2.0 * q + 1.0));
  p.pst_R = c.pst_R;
  {
    double a2 = p.pst_alpha_over_wdx * p.pst_alpha_over_wdx;
    p.pst_R_a4 = c.pst_R * a2 * a2;
  }
  p.pst_n = c.pst_n;
  {
    // double-float constants: hi = the nearest float, lo = the nearest float to the rest
    const float c0h = (float)c.c0, pah = (float)p.pst_R_a4;
    p.df_c0[0] = c0h;
    p.df_c0[1] = (float)(c.c0 - (double)c0h);
    p.df_pst_Ra4[0] = pah;
    p.df_pst_Ra4[1] = (float)(p.pst_R_a4 - (double)pah);
    const double t4 = p.four_h2 / (p.R * p.R);
    const float t4h = (float)t4;
    p.df_4h2_R2[0] = t4h;
    p.df_4h2_R2[1] = (float)(t4 - (double)t4h);
    const double rs = p.R / p.two_h;
    const float rsh = (float)rs;
    p.df_R_2h[0] = rsh;
    p.df_R_2h[1] = (float)(rs - (double)rsh);
  }
  p.rho0 = c.rho0;
  p.c0 = c.c0;
  p.c0sq = c.c0 * c.c0;
  p.inv_c0sq_f = (float)(1.0 / p.c0sq);
  p.inv_rho0_f = (float)(1.0 / c.rho0);
  p.nu = c.nu;
  p.gamma = c.tait_gamma;
  p.delta_h_c0 = c.delta * p.h * c.c0;
  p.tic_lambda = c.tic_lambda;
  for (int k = 0; k < 3; ++k) {
    p.g[k] = k < c.dim ? c.g[k] : 0.0;
    p.force_amp[k] = k < c.dim ? c.force_amp[k] : 0.0;
    p.domain_min[k] = c.domain_min[k];
    p.domain_max[k] = c.domain_max[k];
  }
  p.omega = c.force_period > 0 ? 2.0 * kPi / c.force_period : 0.0;
  p.cfl = c.cfl;
  p.fixed_dt = c.fixed_dt;
  p.water_height = c.water_height;
  p.phs0 = std::sqrt(c.g[0] * c.g[0] + c.g[1] * c.g[1] + c.g[2] * c.g[2]) * c.water_height;
  p.scheme = c.scheme;
  p.wall_bc = c.wall_bc;
  p.body_speed = 0.0;
  for (int k = 0; k < 3; ++k) {
    p.body_u[k] = k < c.dim ? c.body_u[k] : 0.0;
    p.body_speed += p.body_u[k] * p.body_u[k];
  }
  p.body_speed = std::sqrt(p.body_speed);
  p.art_ahc0 = c.art_alpha * p.h * c.c0;
  p.avis_eps2 = 0.01 * p.h * p.h;
  int64_t ncells = 1;
  for (int k = 0; k < 3; ++k) {
    int64_t m = 1;
    if (k < c.dim) m = (int64_t)std::floor((c.domain_max[k] - c.domain_min[k]) / p.R) + 1;
    if (m < 1 || m > (int64_t)1 << 30) return fail(h, WBSPH_E_INVAL, "grid extent out of range on axis %d", k);
    p.nc[k] = (int)m;
    ncells *= m;
  }
  if (ncells >= (int64_t)0xFFFFFFFFLL) return fail(h, WBSPH_E_INVAL, "too many grid cells (%lld)", (long long)ncells);
  p.ncells = ncells;
  // Cell keys. With x in [min, max] on axis k, A = max(|min|, |max|), the
  // FP32 estimate qf = (fl32(x) - fl32(min)) * fl32(1/R), with fl32(x) the
  // truncation of x (relative error below 2^-23) and every FP32 operation
  // rounded to nearest, differs from the FP64 quotient fl64(fl64(x - min)/R)
  // by less than 1.6 A 2^-23 / R + 3.1 N 2^-24 + N 2^-50 (N = cells on the
  // axis, the largest quotient); twice that is the margin. An estimate whose
  // fractional part lies within the margin of 0 or 1 takes the exact path.
  p.key_inv_R_f = (float)(1.0 / p.R);
  for (int k = 0; k < 3; ++k) {
    p.key_lo[k] = ordered_bits(c.domain_min[k]);
    p.key_hi[k] = ordered_bits(c.domain_max[k]);
    p.key_min_f[k] = (float)c.domain_min[k];
    double A = std::max(std::fabs(c.domain_min[k]), std::fabs(c.domain_max[k]));
    double N = (double)p.nc[k];
    double E = 1.6 * A * std::ldexp(1.0, -23) / p.R + 3.1 * N * std::ldexp(1.0, -24) + N * std::ldexp(1.0, -50);
    double m = 2.0 * E;
    p.key_margin[k] = m < 0.25 ? (float)m * 1.001f : 0.5f;  // 0.5: always exact
  }
  // FP32 prefilter bound: every pair with exact r <= 2h has FP32 distance
  // below (2h + e)^2 (1 + 16 ulp), e twice the worst coordinate rounding.
  double X = 0.0;
  for (int k = 0; k < c.dim; ++k) X = std::max(X, std::max(std::fabs(c.domain_min[k]), std::fabs(c.domain_max[k])));
  const double u24 = std::ldexp(1.0, -24);
  double e = 2.0 * std::sqrt((double)c.dim) * (2.0 * X + 2.0 * p.two_h) * u24;
  double thr = (p.two_h + e) * (p.two_h + e) * (1.0 + 16.0 * u24);
  // the same margin for distances up to 2h + skin_max (kept lists)
  p.skin_e = 2.0 * std::sqrt((double)c.dim) * (2.0 * X + 2.0 * (p.two_h + p.skin_max)) * u24;
  float tf = (float)thr;
  if ((double)tf < thr) tf = std::nextafter(tf, INFINITY);
  p.prefilter_r2 = tf;
  // Nearest-fluid band: |r_f^2 - r^2| <= B for every candidate (r <= 2h), so
  // the exact nearest lies within 2B of the FP32 minimum.
  double eps = std::sqrt((double)c.dim) * (2.0 * X + 2.0 * p.two_h) * u24;
  double B = 2.0 * (2.0 * p.two_h * eps + eps * eps + 4.0 * u24 * p.four_h2);
  float bf = (float)(2.0 * B);
  if ((double)bf < 2.0 * B) bf = std::nextafter(bf, INFINITY);
  p.nearest_band_r2 = bf;
  // Inner bound: FP32 r^2 <= (2h)^2 - 2B implies exact r^2 <= (2h)^2, so only
  // candidates above it (a relative band of ~1e-4 in r^2) need the FP64 test.
  double inner = p.four_h2 - 2.0 * B;
  float inf32 = (float)inner;
  if ((double)inf32 > inner) inf32 = std::nextafter(inf32, -INFINITY);
  p.inner_r2 = inf32 > 0.f ? inf32 : 0.f;
  return WBSPH_OK;
}

static int validate(const wbsph_config* c, wbsph_s* h) {
  if (!c) return fail(h, WBSPH_E_INVAL, "null config");
  if (c->dim != 2 && c->dim != 3) return fail(h, WBSPH_E_INVAL, "dim must be 2 or 3");
  if (!(c->dx > 0) || !(c->h_over_dx > 0) || !(c->rho0 > 0) || !(c->c0 > 0))
    return fail(h, WBSPH_E_INVAL, "dx, h_over_dx, rho0 and c0 must be positive");
  if (c->nu < 0 || !(c->cfl > 0)) return fail(h, WBSPH_E_INVAL, "nu >= 0 and cfl > 0 required");
  if (c->eos != 0 && c->eos != 1) return fail(h, WBSPH_E_INVAL, "eos must be 0 or 1");
  if (c->eos == 1 && !(c->tait_gamma > 1)) return fail(h, WBSPH_E_INVAL, "tait_gamma must exceed 1");
  if (c->precision != WBSPH_FP64 && c->precision != WBSPH_MIXED && c->precision != WBSPH_DF64)
    return fail(h, WBSPH_E_INVAL, "unknown precision");
  for (int k = 0; k < c->dim; ++k)
    if (!(c->domain_max[k] > c->domain_min[k])) return fail(h, WBSPH_E_INVAL, "empty domain on axis %d", k);
  if ((c->alloc == nullptr) != (c->free == nullptr))
    return fail(h, WBSPH_E_INVAL, "alloc and free hooks must be given together");
  if (c->scheme != WBSPH_SCHEME_WB && c->scheme != WBSPH_SCHEME_CONVENTIONAL)
    return fail(h, WBSPH_E_INVAL, "unknown scheme");
  if (c->wall_bc != 0 && c->wall_bc != 1) return fail(h, WBSPH_E_INVAL, "wall_bc must be 0 (slip) or 1 (no-slip)");
  if (c->scheme == WBSPH_SCHEME_CONVENTIONAL &&
      (c->precision != WBSPH_FP64 || c->use_delta || c->use_pst || c->use_tic || !(c->art_alpha >= 0)))
    return fail(h, WBSPH_E_INVAL, "the conventional scheme runs in FP64 without delta-SPH, shifting or TIC");
  return WBSPH_OK;
}

extern "C" int wbsph_config_default(wbsph_config* cfg, int dim) {
  if (!cfg || (dim != 2 && dim != 3)) return WBSPH_E_INVAL;
  memset(cfg, 0, sizeof *cfg);
  cfg->dim = dim;
  cfg->dx = 0.01;
  cfg->h_over_dx = 1.5;
  cfg->rho0 = 1000.0;
  cfg->c0 = 30.0;
  cfg->nu = 1e-4;
  cfg->g[dim - 1] = -9.81;
  cfg->cfl = 0.2;
  cfg->delta = 0.1;
  cfg->pst_R = 0.2;
  cfg->pst_n = 4.0;
  cfg->tic_lambda = 0.75;
  cfg->use_delta = cfg->use_pst = cfg->use_tic = cfg->use_visc = 1;
  cfg->eos = 0;
  cfg->tait_gamma = 7.0;
  for (int k = 0; k < 3; ++k) cfg->domain_max[k] = 1.0;
  cfg->precision = WBSPH_FP64;
  cfg->scheme = WBSPH_SCHEME_WB;
  cfg->art_alpha = 0.02;
  return WBSPH_OK;
}

extern "C" int wbsph_create(const wbsph_config* cfg, wbsph_handle* out) {
  if (!out) return WBSPH_E_INVAL;
  *out = nullptr;
  wbsph_s* h = new wbsph_s();
  int rc = validate(cfg, h);
  if (rc) { delete h; return rc; }
  h->cfg = *cfg;
  h->stream = (cudaStream_t)cfg->cuda_stream;
  rc = derive_params(h);
  if (rc) { delete h; return rc; }
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return WBSPH_E_CUDA;
  }
  *out = h;
  return WBSPH_OK;
}

static void drop_graph(wbsph_s* h);

extern "C" void wbsph_destroy(wbsph_handle h) {
  if (!h) return;
  cudaSetDevice(h->cfg.device);
  drop_graph(h);
  free_all(h);
  cudaStreamSynchronize(h->stream);
  if (h->status_host) cudaFreeHost(h->status_host);
  for (auto& e : h->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto& e : h->pool) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  delete h;
}

extern "C" const char* wbsph_last_error(wbsph_handle h) { return h ? h->err.c_str() : "null handle"; }

static int allocate(wbsph_s* h, int64_t n) {
  free_all(h);
  const int d = h->cfg.dim;
  size_t nn = (size_t)(n > 0 ? n : 1);
  auto D = [&](size_t cnt) { return (double*)dev_alloc(h, cnt * sizeof(double)); };
  auto U32 = [&](size_t cnt) { return (uint32_t*)dev_alloc(h, cnt * sizeof(uint32_t)); };
  for (State* s : {&h->A, &h->B}) {
    s->x = D(d * nn); s->u = D(d * nn); s->phi = D(nn);
    s->x0 = D(d * nn); s->u0 = D(d * nn); s->phi0 = D(nn);
    s->mass = D(nn); s->normal = D(d * nn);
    s->type = (uint8_t*)dev_alloc(h, nn);
    s->oid = U32(nn);
  }
  Work& w = h->W;
  w.dudt = D(d * nn); w.dushift = D(d * nn); w.dphidt = D(nn); w.lambda = D(nn); w.vol = D(nn);
  w.volc = D(nn);
  if (h->cfg.scheme == WBSPH_SCHEME_CONVENTIONAL) { w.rho = D(nn); w.pres = D(nn); }
  w.Lmat = D((size_t)(d == 3 ? 6 : 3) * nn);
  w.xf = (float4*)dev_alloc(h, nn * sizeof(float4));
  w.key = U32(nn); w.key_alt = U32(nn); w.perm = U32(nn); w.perm_alt = U32(nn);
  w.cell_lb = U32((size_t)h->P.ncells + 1);
  w.fluid_list = U32(nn);
  w.dummy_list = U32((size_t)(h->nd > 0 ? h->nd : 1));
  if (h->nd > 0) {
    const size_t nfl = (size_t)(h->nf > 0 ? h->nf : 1);
    w.xff = (float4*)dev_alloc(h, nfl * sizeof(float4));
    w.fkey = U32(nfl);
    w.fcell_lb = U32((size_t)h->P.ncells + 1);
  }
  w.block_cnt = U32((size_t)div_up((int64_t)nn, 1024) + 1);
  w.hist = U32((size_t)radix_sort_scratch_words((int64_t)nn));
  w.umax_bits = (unsigned long long*)dev_alloc(h, 8);
  w.scalars = D(4);
  w.status = (unsigned*)dev_alloc(h, sizeof(unsigned));
  w.pairs = (unsigned long long*)dev_alloc(h, 8);
  {
    size_t nfl = (size_t)(h->nf > 0 ? h->nf : 1);
    w.nbr = U32(nfl * (size_t)pair_list_kmax(d));
    w.nbr_cnt = U32(nfl);
  }
  h->field_tmp = D(d * nn);
  if (h->cfg.precision == WBSPH_MIXED || h->cfg.precision == WBSPH_DF64) {
    w.packA = (float4*)dev_alloc(h, nn * sizeof(float4));
    w.packB = (float4*)dev_alloc(h, nn * sizeof(float4));
    if (h->cfg.precision == WBSPH_DF64) {
      w.packAl = (float4*)dev_alloc(h, nn * sizeof(float4));
      w.packBl = (float4*)dev_alloc(h, nn * sizeof(float4));
    }
    w.packC = U32(nn);
    const size_t no = (size_t)h->P.nc[0] + h->P.nc[1] + h->P.nc[2];
    w.cell_origin = D(no);
    if (w.cell_origin) {
      std::vector<double> org;
      org.reserve(no);
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < h->P.nc[k]; ++i) org.push_back(h->P.domain_min[k] + (double)i * h->P.R);
      CK(cudaMemcpyAsync(w.cell_origin, org.data(), no * sizeof(double), cudaMemcpyHostToDevice, h->stream));
      CK(cudaStreamSynchronize(h->stream));  // the host vector goes out of scope
    }
  }
  if (h->alloc_failed) return fail(h, WBSPH_E_NOMEM, "device allocation failed");
  h->n_alloc = n;
  return WBSPH_OK;
}

__global__ void k_iota(uint32_t* a, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) a[i] = (uint32_t)i;
}

extern "C" int wbsph_set_particles(wbsph_handle h, int64_t n, const double* x, const double* u,
                                   const double* phi, const double* mass, const uint8_t* type,
                                   const double* normal, int where) {
  if (!h) return WBSPH_E_INVAL;
  if (n < 0 || n > (int64_t)0x7FFFFFFF) return fail(h, WBSPH_E_INVAL, "particle count out of range");
  if (n > 0 && (!x || !u || !phi || !type)) return fail(h, WBSPH_E_INVAL, "x, u, phi and type are required");
  if (where != WBSPH_HOST && where != WBSPH_DEVICE) return fail(h, WBSPH_E_INVAL, "bad 'where'");
  CK(cudaSetDevice(h->cfg.device));
  const int d = h->cfg.dim;
  cudaMemcpyKind kind = where == WBSPH_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  // types are counted on the host (branch-free, vectorisable); device input
  // is read back first
  std::vector<uint8_t> ty_copy;
  const uint8_t* ty = type;
  if (where == WBSPH_DEVICE && n) {
    ty_copy.resize((size_t)n);
    CK(cudaMemcpyAsync(ty_copy.data(), type, (size_t)n, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    ty = ty_copy.data();
  }
  // fluid (0), wall (1 fixed dummy, 2 body) and invalid counts; 16-bit sums
  // over blocks of 4096 let the compiler vectorise the byte compares
  int64_t nf = 0, nd = 0, bad = 0;
  for (int64_t s = 0; s < n; s += 4096) {
    const int64_t m = n - s < 4096 ? n - s : 4096;
    const uint8_t* q = ty + s;
    uint16_t f16 = 0, d16 = 0, b16 = 0;
    for (int64_t i = 0; i < m; ++i) {
      const uint8_t v = q[i];
      f16 += (uint16_t)(v == 0);
      d16 += (uint16_t)((uint8_t)(v - 1) < 2);
      b16 += (uint16_t)(v > 2);
    }
    nf += f16;
    nd += d16;
    bad += b16;
  }
  if (bad) {
    int64_t i = 0;
    while (ty[i] <= 2) ++i;
    return fail(h, WBSPH_E_INVAL, "particle %lld has type %d (0 fluid, 1 dummy, 2 body)", (long long)i, ty[i]);
  }
  if (nd > 0 && !normal) return fail(h, WBSPH_E_INVAL, "dummy particles need normals");
  h->loaded = false;
  int rc = WBSPH_OK;
  bool same = n == h->n_alloc && nf == h->nf && nd == h->nd && !h->blocks.empty();
  h->n = n; h->nf = nf; h->nd = nd;
  if (!same) {
    drop_graph(h);           // buffers move: a captured step is stale
    rc = allocate(h, n);     // same counts: reuse the buffers and the captured step
  }
  if (rc) return rc;
  size_t vb = (size_t)n * sizeof(double);
  if (n) {
    CK(cudaMemcpyAsync(h->A.x, x, d * vb, kind, h->stream));
    CK(cudaMemcpyAsync(h->A.u, u, d * vb, kind, h->stream));
    CK(cudaMemcpyAsync(h->A.phi, phi, vb, kind, h->stream));
    CK(cudaMemcpyAsync(h->A.type, type, (size_t)n, kind, h->stream));
    if (normal) CK(cudaMemcpyAsync(h->A.normal, normal, d * vb, kind, h->stream));
    else CK(cudaMemsetAsync(h->A.normal, 0, d * vb, h->stream));
    if (mass) CK(cudaMemcpyAsync(h->A.mass, mass, vb, kind, h->stream));
    else launch_mass(h->P, h->A.phi, h->A.mass, n, h->stream);
    k_iota<<<(unsigned)div_up(n, 256), 256, 0, h->stream>>>(h->A.oid, n);
    h->launches += mass ? 1 : 2;
  }
  CK(cudaMemsetAsync(h->W.scalars, 0, 4 * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->W.status, 0, sizeof(unsigned), h->stream));
  CK(cudaMemsetAsync(h->W.umax_bits, 0, 8, h->stream));
  CK(cudaMemsetAsync(h->W.pairs, 0, 8, h->stream));
  if (n) {
    CK(cudaMemsetAsync(h->W.dudt, 0, d * vb, h->stream));
    CK(cudaMemsetAsync(h->W.dushift, 0, d * vb, h->stream));
    CK(cudaMemsetAsync(h->W.dphidt, 0, vb, h->stream));
    CK(cudaMemsetAsync(h->W.lambda, 0, vb, h->stream));
    CK(cudaMemsetAsync(h->W.Lmat, 0, (d == 3 ? 6 : 3) * vb, h->stream));
    CK(cudaMemsetAsync(h->W.vol, 0, vb, h->stream));
  }
  rc = check_launch(h, "set_particles");
  if (rc) return rc;
  if (where == WBSPH_HOST) CK(cudaStreamSynchronize(h->stream));
  h->steps = 0;
  h->steps_since_load = 0;
  h->dist_stage = 0;
  h->dist_dt = 0.0;
  h->loaded = true;
  return WBSPH_OK;
}

// Neighbour build for the current positions (stage 2 also carries y^n).
static int build(wbsph_s* h, bool with_base) {
  const int64_t n = h->n;
  if (n == 0) return WBSPH_OK;
  cudaStream_t st = h->stream;
  {
    ProfScope ps(h, WBSPH_K_KEYS);
    launch_cell_keys(h->P, h->A, h->W, n, st);
  }
  int l = 0;
  {
    ProfScope ps(h, WBSPH_K_SORT);
    launch_radix_sort(h->P, h->W, n, st, &l);
  }
  {
    ProfScope ps(h, WBSPH_K_REORDER);
    launch_gather(h->P, h->A, h->B, h->W, n, with_base, st);
  }
  std::swap(h->A, h->B);
  {
    ProfScope ps(h, WBSPH_K_CELLS);
    launch_cell_bounds(h->P, h->W, n, st);
    launch_fluid_list(h->P, h->A, h->W, n, h->nf, h->nd, st, &l);
  }
  h->launches += 3 + l;
  return check_launch(h, "neighbour build");
}

// dummy walls, then V and U_max (FP64 path) or V, U_max and the packed FP32
// copies in one kernel (mixed path); the double-float path packs its hi/lo
// copies after the FP64 volumes
static int prepass(wbsph_s* h, int stage2) {
  const int64_t n = h->n;
  cudaStream_t st = h->stream;
  const bool mixed = h->cfg.precision == WBSPH_MIXED;
  const bool dfp = h->cfg.precision == WBSPH_DF64;
  ProfScope ps(h, WBSPH_K_PREPASS);
  launch_prepass(h->P, h->A, h->W, n, h->nd, stage2, st, !mixed);
  if (mixed) {
    int rc = launch_prepass_mixed(h->P, h->A, h->W, n, st);
    if (rc) return fail(h, rc, "mixed path: grid too large for packed cell coordinates");
  }
  if (dfp) {
    int rc = launch_pack_df(h->P, h->A, h->W, n, st);
    if (rc) return fail(h, rc, "df64 path: grid too large for packed cell coordinates");
  }
  h->launches += (n ? 1 : 0) + (h->nd ? 1 : 0) + (dfp && n ? 1 : 0);
  return WBSPH_OK;
}

// neighbour lists and the pair pass of the configured precision and scheme;
// lists: LISTS_STAGE builds them for this stage, LISTS_KEEP builds the
// mixed path's kept lists (radius 2h + delta), LISTS_REUSE uses those of
// stage 1
enum { LISTS_STAGE = 0, LISTS_KEEP = 1, LISTS_REUSE = 2 };
static void pair_pass(wbsph_s* h, int stage2, int lists = LISTS_STAGE) {
  const int64_t n = h->n;
  cudaStream_t st = h->stream;
  const bool mixed = h->cfg.precision == WBSPH_MIXED;
  const bool dfp = h->cfg.precision == WBSPH_DF64;
  if (lists != LISTS_REUSE) {
    // exact lists for the FP64 path, and for the double-float path unless
    // they are kept lists (then its pass applies the exact test)
    ProfScope ps(h, WBSPH_K_NLIST);
    launch_nbr_list(h->P, h->A, h->W, n, h->nf, st, !mixed && lists == LISTS_STAGE, lists == LISTS_KEEP);
    h->launches += h->nf ? 1 : 0;
  }
  {
    ProfScope ps(h, WBSPH_K_PAIR);
    if (mixed) launch_pair_mixed(h->P, h->A, h->W, n, h->nf, stage2, st);
    else if (dfp) launch_pair_df(h->P, h->A, h->W, n, h->nf, stage2, st, lists != LISTS_STAGE);
    else if (h->P.scheme == WBSPH_SCHEME_CONVENTIONAL) launch_pair_conventional(h->P, h->A, h->W, n, h->nf, stage2, st);
    else launch_pair_fp64(h->P, h->A, h->W, n, h->nf, stage2, st);
  }
  h->launches += h->nf ? 1 : 0;
}

static int rates(wbsph_s* h, int stage2) {
  int rc = prepass(h, stage2);
  if (rc) return rc;
  if (!stage2) {
    ProfScope ps(h, WBSPH_K_OTHER);
    launch_time_step(h->P, h->W, h->stream);
    h->launches += 1;
  }
  pair_pass(h, stage2);
  return check_launch(h, "stage rates");
}

extern "C" int wbsph_build_neighbors(wbsph_handle h) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  CK(cudaSetDevice(h->cfg.device));
  return build(h, false);
}

extern "C" int wbsph_eval_rates(wbsph_handle h) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  CK(cudaSetDevice(h->cfg.device));
  int rc = build(h, false);
  if (rc) return rc;
  return rates(h, 0);
}

// ---------------------------------------------------------------------------
// Stages of a domain decomposition: one SSP-RK2 stage with the step's start
// time, its time step and the stage's U_max (over all fluid particles of all
// subdomains) given by the caller, and an update of selected particles (the
// ghosts a neighbouring subdomain owns) between the stages.
// ---------------------------------------------------------------------------
__global__ void k_inverse_oid(const uint32_t* oid, int64_t n, uint32_t* inv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) inv[oid[i]] = (uint32_t)i;
}

__global__ void k_scatter_state(int dim, State s, int64_t n, const uint32_t* inv, const uint32_t* ids, int64_t count,
                                const double* xs, const double* us, const double* phis) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t i = inv[ids[k]];
  for (int d = 0; d < dim; ++d) {
    s.x[d * n + i] = xs[d * count + k];
    s.u[d * n + i] = us[d * count + k];
  }
  s.phi[i] = phis[k];
}

extern "C" int wbsph_stage(wbsph_handle h, int stage, double t, double dt, double umax) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (stage != 1 && stage != 2) return fail(h, WBSPH_E_INVAL, "stage must be 1 or 2");
  if (!std::isfinite(t) || !std::isfinite(dt) || !(umax >= 0.0) || !std::isfinite(umax))
    return fail(h, WBSPH_E_INVAL, "bad time, time step or U_max");
  if (stage == 2 && h->dist_stage != 1) return fail(h, WBSPH_E_STATE, "stage 2 needs a stage 1 first");
  CK(cudaSetDevice(h->cfg.device));
  drop_graph(h);  // builds outside a captured step
  cudaStream_t st = h->stream;
  const int stage2 = stage == 2;
  h->dist_host[0] = t;
  h->dist_host[1] = dt;
  const double u2 = umax * umax;
  memcpy(&h->dist_host[2], &u2, sizeof u2);
  CK(cudaMemcpyAsync(h->W.scalars, h->dist_host, (dt > 0.0 ? 2 : 1) * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = build(h, stage2);
  if (rc) return rc;
  if ((rc = prepass(h, stage2))) return rc;
  // the stage's U_max of the whole domain (shifting, and the time step below)
  CK(cudaMemcpyAsync(h->W.umax_bits, &h->dist_host[2], 8, cudaMemcpyHostToDevice, st));
  if (!stage2 && !(dt > 0.0)) {
    ProfScope ps(h, WBSPH_K_OTHER);
    launch_time_step(h->P, h->W, st);
    h->launches += 1;
  } else if (stage2 && !(dt > 0.0) && h->dist_dt <= 0.0) {
    return fail(h, WBSPH_E_STATE, "no time step for stage 2");
  }
  pair_pass(h, stage2);
  {
    ProfScope ps(h, WBSPH_K_UPDATE);
    launch_rk_stage(h->P, h->A, h->W, h->n, stage, st);
    h->launches += 1;
  }
  h->dist_stage = stage;
  h->dist_dt = 1.0;  // a time step is in place on the device
  if (stage2) ++h->steps;
  return check_launch(h, "distributed stage");
}

extern "C" int wbsph_update_particles(wbsph_handle h, int64_t count, const uint32_t* ids, const double* x,
                                      const double* u, const double* phi) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (count < 0 || count > h->n) return fail(h, WBSPH_E_INVAL, "bad particle count");
  if (count == 0) return WBSPH_OK;
  if (!ids || !x || !u || !phi) return fail(h, WBSPH_E_INVAL, "null array");
  for (int64_t k = 0; k < count; ++k)
    if ((int64_t)ids[k] >= h->n) return fail(h, WBSPH_E_INVAL, "particle id %lld out of range", (long long)ids[k]);
  CK(cudaSetDevice(h->cfg.device));
  cudaStream_t st = h->stream;
  const int d = h->cfg.dim;
  const int64_t n = h->n;
  uint32_t *inv = nullptr, *dids = nullptr;
  double* vals = nullptr;
  CK(cudaMallocAsync((void**)&inv, (size_t)n * 4, st));
  CK(cudaMallocAsync((void**)&dids, (size_t)count * 4, st));
  CK(cudaMallocAsync((void**)&vals, (size_t)count * (2 * d + 1) * sizeof(double), st));
  CK(cudaMemcpyAsync(dids, ids, (size_t)count * 4, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(vals, x, (size_t)count * d * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(vals + (size_t)count * d, u, (size_t)count * d * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(vals + (size_t)count * 2 * d, phi, (size_t)count * sizeof(double), cudaMemcpyHostToDevice, st));
  k_inverse_oid<<<(unsigned)div_up(n, 256), 256, 0, st>>>(h->A.oid, n, inv);
  k_scatter_state<<<(unsigned)div_up(count, 256), 256, 0, st>>>(d, h->A, n, inv, dids, count, vals,
                                                               vals + (size_t)count * d, vals + (size_t)count * 2 * d);
  h->launches += 2;
  CK(cudaStreamSynchronize(st));  // the host arrays may be reused when this returns
  cudaFreeAsync(inv, st);
  cudaFreeAsync(dids, st);
  cudaFreeAsync(vals, st);
  return check_launch(h, "update_particles");
}

// One SSP-RK2 step as a launch sequence (no host synchronisation).
static int enqueue_step(wbsph_s* h) {
  int rc = build(h, false);
  if (rc) return rc;
  if (h->P.skin) {
    // mixed and double-float paths: one build per step; stage 2 keeps the
    // sorted order, the cells and the lists of stage 1 (2h + delta), with
    // the FP32 position copies brought to the stage-1 positions for the wall
    // update's scan
    if ((rc = prepass(h, 0))) return rc;
    {
      ProfScope ps(h, WBSPH_K_OTHER);
      launch_time_step(h->P, h->W, h->stream, true);
      h->launches += 1;
    }
    pair_pass(h, 0, LISTS_KEEP);
    {
      ProfScope ps(h, WBSPH_K_UPDATE);
      launch_rk_stage(h->P, h->A, h->W, h->n, 1, h->stream);
      launch_refresh_xf(h->P, h->A, h->W, h->n, h->nf, h->nd, h->stream);
    }
    if ((rc = prepass(h, 1))) return rc;
    pair_pass(h, 1, LISTS_REUSE);
    {
      ProfScope ps(h, WBSPH_K_UPDATE);
      launch_rk_stage(h->P, h->A, h->W, h->n, 2, h->stream);
    }
    h->launches += 3;
    return check_launch(h, "step");
  }
  rc = rates(h, 0);
  if (rc) return rc;
  {
    ProfScope ps(h, WBSPH_K_UPDATE);
    launch_rk_stage(h->P, h->A, h->W, h->n, 1, h->stream);
  }
  rc = build(h, true);
  if (rc) return rc;
  rc = rates(h, 1);
  if (rc) return rc;
  {
    ProfScope ps(h, WBSPH_K_UPDATE);
    launch_rk_stage(h->P, h->A, h->W, h->n, 2, h->stream);
  }
  h->launches += 2;
  return check_launch(h, "step");
}

static void drop_graph(wbsph_s* h) {
  for (auto& g : h->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = wbsph_s::StepGraph{};
  }
}

// the captured step that starts from the current buffer pointers, if any
static wbsph_s::StepGraph* find_graph(wbsph_s* h) {
  for (auto& g : h->graphs)
    if (g.exec && !memcmp(&g.a0, &h->A, sizeof(State)) && !memcmp(&g.b0, &h->B, sizeof(State)) &&
        !memcmp(&g.w0, &h->W, sizeof(Work)))
      return &g;
  return nullptr;
}

// Capture one step from the current buffer pointers into a free graph slot
// (both slots in use: both dropped first). The enqueue leaves the host's
// pointers where the step leaves them; the graph is launched next.
static int capture_step(wbsph_s* h, wbsph_s::StepGraph** out) {
  wbsph_s::StepGraph* g = !h->graphs[0].exec ? &h->graphs[0] : !h->graphs[1].exec ? &h->graphs[1] : nullptr;
  if (!g) {
    drop_graph(h);
    g = &h->graphs[0];
  }
  int64_t l0 = h->launches;
  g->a0 = h->A; g->b0 = h->B; g->w0 = h->W;
  cudaGraph_t cg = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  h->capturing = true;
  int rc = enqueue_step(h);
  h->capturing = false;
  cudaError_t e = cudaStreamEndCapture(h->stream, &cg);
  if (rc || e != cudaSuccess) {
    if (cg) cudaGraphDestroy(cg);
    cudaGetLastError();
    h->A = g->a0; h->B = g->b0; h->W = g->w0;  // nothing ran
    *g = wbsph_s::StepGraph{};
    return rc ? rc : fail(h, WBSPH_E_CUDA, "step capture: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&g->exec, cg, 0);
  cudaGraphDestroy(cg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->A = g->a0; h->B = g->b0; h->W = g->w0;
    *g = wbsph_s::StepGraph{};
    return fail(h, WBSPH_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  g->a1 = h->A; g->b1 = h->B; g->w1 = h->W;
  g->launches = h->launches - l0;
  h->launches = l0;
  *out = g;
  return WBSPH_OK;
}

extern "C" int wbsph_step(wbsph_handle h, int64_t nsteps) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (nsteps < 0) return fail(h, WBSPH_E_INVAL, "nsteps < 0");
  CK(cudaSetDevice(h->cfg.device));
  // Graph replay on a caller stream (not the legacy default stream) when
  // profiling is off. The first step of a handle runs eagerly, so that
  // one-time kernel attributes are set outside the capture; the captured step
  // survives set_particles with unchanged counts (same buffers; whole steps
  // leave the double-buffer pointers where the capture found them).
  bool graphs = h->use_graphs && h->stream != nullptr && !h->prof && h->n > 0;
  for (int64_t s = 0; s < nsteps; ++s) {
    int rc;
    wbsph_s::StepGraph* g = graphs ? find_graph(h) : nullptr;
    if (graphs && (g || h->steps_since_load > 0)) {
      if (!g && capture_step(h, &g) != WBSPH_OK) {
        h->use_graphs = false;
        graphs = false;
        rc = enqueue_step(h);
      } else {
        CK(cudaGraphLaunch(g->exec, h->stream));
        h->A = g->a1; h->B = g->b1; h->W = g->w1;
        h->launches += g->launches;
        rc = check_launch(h, "graph step");
      }
    } else {
      rc = enqueue_step(h);
    }
    if (rc) return rc;
    ++h->steps;
    ++h->steps_since_load;
  }
  return WBSPH_OK;
}

// Status bits -> status code (the copy of the word must have landed).
static int decode_status(wbsph_s* h, unsigned s);

static int read_status(wbsph_s* h) {
  if (!h->status_host) CK(cudaMallocHost((void**)&h->status_host, sizeof(unsigned)));
  CK(cudaMemcpyAsync(h->status_host, h->W.status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return decode_status(h, *h->status_host);
}

static int decode_status(wbsph_s* h, unsigned s) {
  if (!s) return WBSPH_OK;
  // the kept lists no longer covered every pair: what
  // followed is not the method, whatever else went wrong after it
  if (s & kStatSkin)
    return fail(h, WBSPH_E_CAPACITY,
                "a particle can move more than the neighbour-list skin in one stage (mixed and double-float "
                "paths: flow above Mach 0.3 at this CFL number, or a fixed time step that is too long)");
  // so did a list that overflowed: its particle's sums left pairs out
  if (s & kStatOverflow)
    return fail(h, WBSPH_E_CAPACITY,
                "neighbour list overflow: a particle has more neighbours (or kept candidates) than a list "
                "holds (48 in 2D, 128 in 3D); the particle spacing is far below dx");
  // a non-finite value also sends positions out of the domain: report it first
  if (s & kStatNaN) return fail(h, WBSPH_E_NAN, "non-finite rate or state value");
  if (s & kStatSingular) return fail(h, WBSPH_E_SINGULAR, "singular renormalisation matrix (TIC off)");
  if (s & kStatDomain) return fail(h, WBSPH_E_DOMAIN, "a particle left the domain");
  if (s & kStatTimeout) return fail(h, WBSPH_E_TIMEOUT, "a bounded device wait gave up");
  return fail(h, WBSPH_E_CUDA, "unexpected device status word 0x%x", s);
}

extern "C" int wbsph_test_bounded_wait(wbsph_handle h, int64_t limit) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (limit < 1 || limit > ((int64_t)1 << 20)) return fail(h, WBSPH_E_INVAL, "limit out of range (1 .. 2^20)");
  CK(cudaSetDevice(h->cfg.device));
  launch_wait_probe(h->W.status, (uint32_t)limit, h->stream);
  int rc = check_launch(h, "wait probe");
  if (rc) return rc;
  return read_status(h);
}

extern "C" int wbsph_sync(wbsph_handle h) {
  if (!h) return WBSPH_E_INVAL;
  CK(cudaSetDevice(h->cfg.device));
  CK(cudaStreamSynchronize(h->stream));
  if (!h->loaded) return WBSPH_OK;
  return read_status(h);
}

extern "C" int wbsph_get_fields(wbsph_handle h, int field, double* out, int where) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (field < 0 || field > WBSPH_FIELD_VOL || !out) return fail(h, WBSPH_E_INVAL, "bad field or output");
  if (where != WBSPH_HOST && where != WBSPH_DEVICE) return fail(h, WBSPH_E_INVAL, "bad 'where'");
  CK(cudaSetDevice(h->cfg.device));
  const int64_t n = h->n;
  if (n == 0) return read_status(h);
  if (!h->status_host) CK(cudaMallocHost((void**)&h->status_host, sizeof(unsigned)));
  bool vec = field == WBSPH_FIELD_X || field == WBSPH_FIELD_U || field == WBSPH_FIELD_DUDT ||
             field == WBSPH_FIELD_DUSHIFT;
  size_t bytes = (size_t)n * (vec ? h->cfg.dim : 1) * sizeof(double);
  // field in the caller's order, copy out and the status word, then one
  // synchronisation: the output is valid only when the status is clean
  double* tmp = where == WBSPH_HOST ? h->field_tmp : out;
  if (field == WBSPH_FIELD_LAMBDA && h->cfg.precision != WBSPH_MIXED) {
    // the FP64 pass stores L; lambda_min is formed here, in FP64
    launch_lambda_fp64(h->P, h->W, n, h->nf, h->stream);
    h->launches += 1;
  }
  launch_field(h->P, h->A, h->W, n, field, tmp, h->stream);
  h->launches += 1;
  int rc = check_launch(h, "get_fields");
  if (rc) return rc;
  if (where == WBSPH_HOST) CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->status_host, h->W.status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return decode_status(h, *h->status_host);
}

extern "C" int wbsph_get_cell_keys(wbsph_handle h, uint32_t* keys_sorted, uint32_t* ids_sorted) {
  if (!h) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  CK(cudaSetDevice(h->cfg.device));
  int rc = read_status(h);
  if (rc) return rc;
  if (h->n == 0) return WBSPH_OK;
  if (keys_sorted) CK(cudaMemcpyAsync(keys_sorted, h->W.key, h->n * 4, cudaMemcpyDeviceToHost, h->stream));
  if (ids_sorted) CK(cudaMemcpyAsync(ids_sorted, h->A.oid, h->n * 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return WBSPH_OK;
}

extern "C" int64_t wbsph_get_neighbors(wbsph_handle h, int64_t* row_ptr, int32_t* cols, int64_t cap) {
  if (!h || !row_ptr) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  CK(cudaSetDevice(h->cfg.device));
  const int64_t n = h->n;
  int rc = build(h, false);
  if (rc) return rc;
  rc = read_status(h);
  if (rc) return rc;
  row_ptr[0] = 0;
  if (n == 0) return 0;
  uint32_t* counts = nullptr;
  CK(cudaMallocAsync((void**)&counts, n * 4, h->stream));
  launch_count_neighbors(h->P, h->A, h->W, n, counts, h->stream);
  std::vector<uint32_t> hc((size_t)n);
  CK(cudaMemcpyAsync(hc.data(), counts, n * 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  cudaFreeAsync(counts, h->stream);
  for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + hc[i];
  int64_t nnz = row_ptr[n];
  h->launches += 1;
  if (!cols) return nnz;
  if (nnz > cap) return fail(h, WBSPH_E_CAPACITY, "need %lld entries", (long long)nnz);
  int64_t* drow = nullptr;
  int32_t* dcol = nullptr;
  CK(cudaMallocAsync((void**)&drow, (n + 1) * 8, h->stream));
  CK(cudaMallocAsync((void**)&dcol, (nnz > 0 ? nnz : 1) * 4, h->stream));
  CK(cudaMemcpyAsync(drow, row_ptr, (n + 1) * 8, cudaMemcpyHostToDevice, h->stream));
  launch_fill_neighbors(h->P, h->A, h->W, n, drow, dcol, h->stream);
  h->launches += 1;
  if (nnz) CK(cudaMemcpyAsync(cols, dcol, nnz * 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  cudaFreeAsync(drow, h->stream);
  cudaFreeAsync(dcol, h->stream);
  CK(cudaStreamSynchronize(h->stream));
  for (int64_t i = 0; i < n; ++i) std::sort(cols + row_ptr[i], cols + row_ptr[i + 1]);
  return nnz;
}

extern "C" int wbsph_get_stats(wbsph_handle h, wbsph_stats* out) {
  if (!h || !out) return WBSPH_E_INVAL;
  memset(out, 0, sizeof *out);
  out->n = h->n; out->n_fluid = h->nf; out->n_dummy = h->nd;
  out->ncells = h->P.ncells;
  for (int k = 0; k < 3; ++k) out->grid[k] = h->P.nc[k];
  out->steps = h->steps;
  out->launches = h->launches;
  out->device_bytes = h->device_bytes;
  if (h->loaded) {
    double sc[2] = {0, 0};
    unsigned long long pairs = 0;
    CK(cudaSetDevice(h->cfg.device));
    CK(cudaMemcpyAsync(sc, h->W.scalars, sizeof sc, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&pairs, h->W.pairs, 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out->t = sc[0];
    out->dt = sc[1];
    out->pairs = (int64_t)pairs;
  }
  return WBSPH_OK;
}

extern "C" int wbsph_set_profiling(wbsph_handle h, int on) {
  if (!h) return WBSPH_E_INVAL;
  h->prof = on != 0;
  return WBSPH_OK;
}

extern "C" int wbsph_get_profile(wbsph_handle h, double* ms, int64_t* launches, int reset) {
  if (!h) return WBSPH_E_INVAL;
  CK(cudaSetDevice(h->cfg.device));
  CK(cudaStreamSynchronize(h->stream));
  for (auto& e : h->events) {
    float t = 0.f;
    cudaEventElapsedTime(&t, e.a, e.b);
    h->prof_ms[e.cls] += t;
    h->prof_cnt[e.cls] += 1;
    h->pool.push_back(e);
  }
  h->events.clear();
  for (int k = 0; k < WBSPH_K_COUNT; ++k) {
    if (ms) ms[k] = h->prof_ms[k];
    if (launches) launches[k] = h->prof_cnt[k];
    if (reset) { h->prof_ms[k] = 0; h->prof_cnt[k] = 0; }
  }
  return WBSPH_OK;
}

// ---- small kernels owned by the engine ----
namespace wbsph {
__global__ void k_mass(Params p, const double* phi, double* mass, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double rho = p.eos == 0 ? p.rho0 * exp(phi[i] / p.c0sq)
                          : p.rho0 * pow(1.0 + (p.gamma - 1.0) * phi[i] / p.c0sq, 1.0 / (p.gamma - 1.0));
  double vol = p.dim == 2 ? p.dx * p.dx : p.dx * p.dx * p.dx;
  mass[i] = rho * vol;
}

void launch_mass(const Params& p, const double* phi, double* mass, int64_t n, cudaStream_t st) {
  k_mass<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p, phi, mass, n);
}
}  // namespace wbsph

// ---- read-only accessors for other translation units of the library ----
namespace wbsph {
const Params* handle_params(wbsph_handle h) { return h ? &h->P : nullptr; }
cudaStream_t handle_stream(wbsph_handle h) { return h ? h->stream : nullptr; }
int handle_device(wbsph_handle h) { return h ? h->cfg.device : 0; }
int handle_fail(wbsph_handle h, int code, const char* msg) { return fail(h, code, "%s", msg); }
}  // namespace wbsph

// ---------------------------------------------------------------------------
// Learned surrogate: training, prediction and anchored rollouts
// ---------------------------------------------------------------------------
#include <cuda_bf16.h>
namespace wbsph {
int surrogate_stage_rates(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n,
                          int64_t nf, cudaStream_t cs);
int surrogate_loss(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n, int64_t nf,
                   cudaStream_t cs, int train, float lr, double* loss_out, const float* dout_override,
                   float* grad_out);
int64_t surrogate_edges(wbsph_surrogate s);
int surrogate_stage_launches(wbsph_surrogate s, int64_t nf);
int surrogate_mode(wbsph_surrogate s);
int surrogate_plain_rates(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n, int64_t nf,
                          int64_t n_ids, cudaStream_t cs);
const float* surrogate_out(wbsph_surrogate s);
const uint32_t* surrogate_recv(wbsph_surrogate s);
const uint32_t* surrogate_send(wbsph_surrogate s);
const __nv_bfloat16* surrogate_efeat(wbsph_surrogate s);
const __nv_bfloat16* surrogate_nfeat(wbsph_surrogate s);
void launch_rel_err(const Params& p, const Work& w, int64_t n, int64_t nf, const double* a_ref_copy,
                    double* sums, cudaStream_t st);
}  // namespace wbsph

static int check_pair(wbsph_s* h, wbsph_surrogate s) {
  if (!h || !s) return WBSPH_E_INVAL;
  if (!h->loaded) return fail(h, WBSPH_E_STATE, "set_particles first");
  if (h->cfg.precision != WBSPH_FP64) return fail(h, WBSPH_E_INVAL, "the surrogate needs an FP64 handle");
  return WBSPH_OK;
}

// Surrogate stage: dummy walls, U_max, [time step], surrogate rates. The
// network reads no volumes, so none are formed.
static int surrogate_stage(wbsph_s* h, wbsph_surrogate s, int stage2) {
  cudaStream_t st = h->stream;
  {
    ProfScope ps(h, WBSPH_K_PREPASS);
    launch_prepass(h->P, h->A, h->W, h->n, h->nd, stage2, st, false);
    launch_umax(h->P, h->A, h->W, h->n, st);
  }
  if (!stage2) {
    ProfScope ps(h, WBSPH_K_OTHER);
    launch_time_step(h->P, h->W, st);
  }
  int rc;
  {
    ProfScope ps(h, WBSPH_K_PAIR);
    rc = surrogate_stage_rates(s, h->P, h->A, h->W, h->n, h->nf, st);
  }
  // prepass (dummy update, U_max), time step, and the surrogate stage's
  // kernels (network: neighbour lists, node inputs, encoder, one fused
  // kernel per layer, decoder, rates; frozen-rates control: one)
  h->launches += (h->n ? (h->nd ? 2 : 1) : 0) + (stage2 ? 0 : 1) + surrogate_stage_launches(s, h->nf);
  if (rc) return fail(h, rc, "surrogate stage failed");
  return check_launch(h, "surrogate stage");
}

extern "C" int wbsph_surrogate_train_step(wbsph_surrogate s, wbsph_handle h, float lr, double* loss) {
  int rc = check_pair(h, s);
  if (rc) return rc;
  CK(cudaSetDevice(h->cfg.device));
  if ((rc = build(h, false)) || (rc = rates(h, 0))) return rc;
  rc = surrogate_loss(s, h->P, h->A, h->W, h->n, h->nf, h->stream, 1, lr, loss, nullptr, nullptr);
  if (rc) return fail(h, rc, "surrogate training step failed");
  return read_status(h);
}

extern "C" int wbsph_surrogate_eval(wbsph_surrogate s, wbsph_handle h, double* loss) {
  int rc = check_pair(h, s);
  if (rc) return rc;
  CK(cudaSetDevice(h->cfg.device));
  if ((rc = build(h, false)) || (rc = rates(h, 0))) return rc;
  rc = surrogate_loss(s, h->P, h->A, h->W, h->n, h->nf, h->stream, 0, 0.f, loss, nullptr, nullptr);
  if (rc) return fail(h, rc, "surrogate evaluation failed");
  return read_status(h);
}

extern "C" int wbsph_surrogate_predict(wbsph_surrogate s, wbsph_handle h) {
  int rc = check_pair(h, s);
  if (rc) return rc;
  CK(cudaSetDevice(h->cfg.device));
  if ((rc = build(h, false))) return rc;
  return surrogate_stage(h, s, 0);
}

static void bf16_to_host(const __nv_bfloat16* d, int64_t count, float* out, cudaStream_t st) {
  std::vector<uint16_t> tmp((size_t)count);
  if (count) cudaMemcpyAsync(tmp.data(), d, count * 2, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  for (int64_t k = 0; k < count; ++k) {
    uint32_t b = (uint32_t)tmp[k] << 16;
    memcpy(&out[k], &b, 4);
  }
}

extern "C" int wbsph_surrogate_debug(wbsph_surrogate s, wbsph_handle h, int64_t* n_edges, uint32_t* recv_ids,
                                     uint32_t* send_ids, float* edge_feat, float* node_feat,
                                     uint32_t* fluid_ids, float* out, float* grad, double* loss) {
  int rc = check_pair(h, s);
  if (rc) return rc;
  if (!n_edges) return fail(h, WBSPH_E_INVAL, "n_edges required");
  CK(cudaSetDevice(h->cfg.device));
  if ((rc = build(h, false)) || (rc = rates(h, 0))) return rc;
  rc = surrogate_loss(s, h->P, h->A, h->W, h->n, h->nf, h->stream, 0, 0.f, loss, nullptr, grad);
  if (rc) return fail(h, rc, "surrogate evaluation failed");
  int64_t E = surrogate_edges(s);
  *n_edges = E;
  const int64_t n = h->n, nf = h->nf;
  const int fo = h->cfg.dim + 1;
  cudaStream_t st = h->stream;
  std::vector<uint32_t> oid((size_t)n), fl((size_t)nf), tmp((size_t)E);
  CK(cudaMemcpyAsync(oid.data(), h->A.oid, n * 4, cudaMemcpyDeviceToHost, st));
  if (nf) CK(cudaMemcpyAsync(fl.data(), h->W.fluid_list, nf * 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (fluid_ids)
    for (int64_t g = 0; g < nf; ++g) fluid_ids[g] = oid[fl[g]];
  if (recv_ids && E) {
    CK(cudaMemcpyAsync(tmp.data(), surrogate_recv(s), E * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int64_t e = 0; e < E; ++e) recv_ids[e] = oid[tmp[e]];
  }
  if (send_ids && E) {
    CK(cudaMemcpyAsync(tmp.data(), surrogate_send(s), E * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int64_t e = 0; e < E; ++e) send_ids[e] = oid[tmp[e]];
  }
  if (edge_feat) bf16_to_host(surrogate_efeat(s), E * 8, edge_feat, st);
  if (node_feat) {
    std::vector<float> nfe((size_t)n * 8);
    bf16_to_host(surrogate_nfeat(s), n * 8, nfe.data(), st);
    for (int64_t i = 0; i < n; ++i) memcpy(node_feat + (int64_t)oid[i] * 8, &nfe[(size_t)i * 8], 32);
  }
  if (out && nf) {
    CK(cudaMemcpyAsync(out, surrogate_out(s), nf * fo * 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return read_status(h);
}

extern "C" int wbsph_step_surrogate(wbsph_handle h, wbsph_surrogate s, int64_t nsteps, int anchor_every,
                                    double tau, wbsph_anchor_stats* stats) {
  int rc = check_pair(h, s);
  if (rc) return rc;
  if (nsteps < 0 || anchor_every < 0) return fail(h, WBSPH_E_INVAL, "bad step counts");
  CK(cudaSetDevice(h->cfg.device));
  wbsph_anchor_stats local;
  memset(&local, 0, sizeof local);
  const int d = h->cfg.dim;
  double* ref = nullptr;  // copy of the surrogate DU/Dt at an anchor, then error sums
  CK(cudaMallocAsync((void**)&ref, ((size_t)d * (h->n > 0 ? h->n : 1) + 2) * sizeof(double), h->stream));
  int64_t plain_until = -1;
  bool have_plain = false;  // a plain stage has run (the frozen-rates control needs one)
  for (int64_t k = 0; k < nsteps && !rc; ++k) {
    bool anchor = anchor_every > 0 && k % anchor_every == 0;
    bool plain = anchor || k < plain_until;
    // the frozen-rates control has nothing to compare before its first plain stage
    bool compare = anchor && (have_plain || surrogate_mode(s) != WBSPH_SURROGATE_FROZEN);
    if ((rc = build(h, false))) break;
    if (compare) {
      // surrogate rates at this state, kept for the comparison with the plain ones
      if ((rc = surrogate_stage(h, s, 0))) break;
      CK(cudaMemcpyAsync(ref, h->W.dudt, (size_t)d * h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    if (plain) {
      if ((rc = rates(h, 0))) break;
      if ((rc = surrogate_plain_rates(s, h->P, h->A, h->W, h->n, h->nf, h->n, h->stream))) {
        rc = fail(h, rc, "surrogate: keeping the plain rates failed");
        break;
      }
      have_plain = true;
    } else {
      if ((rc = surrogate_stage(h, s, 0))) break;
    }
    if (compare) {
      double sums[2] = {0, 0};
      launch_rel_err(h->P, h->W, h->n, h->nf, ref, ref + (size_t)d * h->n, h->stream);
      CK(cudaMemcpyAsync(sums, ref + (size_t)d * h->n, 16, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      double e = sums[1] > 0 ? std::sqrt(sums[0] / sums[1]) : 0.0;
      local.anchors += 1;
      local.last_rel_err = e;
      local.max_rel_err = std::max(local.max_rel_err, e);
      if (e > tau) {
        local.fallbacks += 1;
        plain_until = k + 1 + anchor_every;
      }
    }
    launch_rk_stage(h->P, h->A, h->W, h->n, 1, h->stream);
    if ((rc = build(h, true))) break;
    if (plain) rc = rates(h, 1);
    else rc = surrogate_stage(h, s, 1);
    if (rc) break;
    launch_rk_stage(h->P, h->A, h->W, h->n, 2, h->stream);
    h->launches += 2;
    if (plain) local.plain_steps += 1; else local.surrogate_steps += 1;
    ++h->steps;
  }
  cudaFreeAsync(ref, h->stream);
  if (stats) *stats = local;
  if (rc) return rc;
  return read_status(h);
}
