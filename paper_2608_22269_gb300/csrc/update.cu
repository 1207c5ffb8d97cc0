// update.cu -- the SSP-RK2 stage updates (Sec. 2.3) and field output in the
// caller's order.
#include "common.cuh"
#include "physics.cuh"

namespace wbsph {
// ---------------------------------------------------------------------------
// SSP-RK2 stages (Sec. 2.3), fluid particles; dummies stay fixed.
//   stage 1: y0 = y;  y = y0 + dt F(y0);  x = x0 + dt (U0 + dU0)
//   stage 2: y = y0/2 + (y1 + dt F(y1))/2; x = x0/2 + (x1 + dt (U1 + dU1))/2
// Stage 2 also advances t by dt (one thread, after every reader of t).
// ---------------------------------------------------------------------------
__global__ void k_rk_stage(Params p, State s, Work w, int64_t n, int stage) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double dt = w.scalars[1];
  if (stage == 2 && i == 0) w.scalars[0] = w.scalars[0] + dt;
  if (i >= n) return;
  bool fluid = s.type[i] == kFluid;
  const bool body = s.type[i] == kBody;  // prescribed rigid translation, the same SSP-RK2 update
  if (!fluid && !body) return;  // fixed wall particles: nothing moves, no stage-start copy is read
  if (stage == 1) {
    for (int k = 0; k < p.dim; ++k) {
      double x0 = s.x[k * n + i], u0 = s.u[k * n + i];
      s.x0[k * n + i] = x0;
      s.u0[k * n + i] = u0;
      if (fluid) {
        s.x[k * n + i] = x0 + dt * (u0 + w.dushift[k * n + i]);
        s.u[k * n + i] = u0 + dt * w.dudt[k * n + i];
      } else if (body) {
        s.x[k * n + i] = x0 + dt * p.body_u[k];
      }
    }
    double ph0 = s.phi[i];
    s.phi0[i] = ph0;
    if (fluid) s.phi[i] = ph0 + dt * w.dphidt[i];
  } else if (body) {
    for (int k = 0; k < p.dim; ++k)
      s.x[k * n + i] = 0.5 * s.x0[k * n + i] + 0.5 * (s.x[k * n + i] + dt * p.body_u[k]);
  } else if (fluid) {
    for (int k = 0; k < p.dim; ++k) {
      double x1 = s.x[k * n + i], u1 = s.u[k * n + i];
      s.x[k * n + i] = 0.5 * s.x0[k * n + i] + 0.5 * (x1 + dt * (u1 + w.dushift[k * n + i]));
      s.u[k * n + i] = 0.5 * s.u0[k * n + i] + 0.5 * (u1 + dt * w.dudt[k * n + i]);
    }
    s.phi[i] = 0.5 * s.phi0[i] + 0.5 * (s.phi[i] + dt * w.dphidt[i]);
  }
}

void launch_rk_stage(const Params& p, const State& s, const Work& w, int64_t n, int stage,
                     cudaStream_t st) {
  k_rk_stage<<<(unsigned)div_up(n > 0 ? n : 1, 256), 256, 0, st>>>(p, s, w, n, stage);
}

// FP32 position copies of the moved particles (fluid and body) at their
// current positions, in the sorted order of the last neighbour build: xf for
// the candidate tests, xff for the wall update's scan over fluid particles.
__global__ void k_refresh_xf(int dim, State s, Work w, int64_t n, int64_t nf, int64_t nd, int compact) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  auto pos = [&](uint32_t i) {
    float4 f = make_float4(0.f, 0.f, 0.f, (float)s.type[i]);
    f.x = (float)s.x[i];
    f.y = (float)s.x[n + i];
    if (dim == 3) f.z = (float)s.x[2 * n + i];
    return f;
  };
  if (t < nf) {
    const uint32_t i = w.fluid_list[t];
    const float4 f = pos(i);
    w.xf[i] = f;
    if (compact) w.xff[t] = f;
  }
  if (t < nd) {
    const uint32_t i = w.dummy_list[t];
    if (s.type[i] == kBody) w.xf[i] = pos(i);
  }
}

void launch_refresh_xf(const Params& p, const State& s, const Work& w, int64_t n, int64_t nf, int64_t nd,
                       cudaStream_t st) {
  const int64_t m = nf > nd ? nf : nd;
  if (m == 0) return;
  k_refresh_xf<<<(unsigned)div_up(m, 256), 256, 0, st>>>(p.dim, s, w, n, nf, nd, nd > 0 && w.dummy_list ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Field output in original order: out[k n + oid[i]] = field[k n + i].
// ---------------------------------------------------------------------------
__global__ void k_field(Params p, State s, Work w, int64_t n, int field, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = s.oid[i];
  const double* src = nullptr;
  int comps = 1;
  switch (field) {
    case 0: src = s.x; comps = p.dim; break;
    case 1: src = s.u; comps = p.dim; break;
    case 2: src = s.phi; break;
    case 5: src = w.dudt; comps = p.dim; break;
    case 6: src = w.dphidt; break;
    case 7: src = w.dushift; comps = p.dim; break;
    case 8: src = w.lambda; break;
    case 9: src = s.mass; break;
    case 10: src = w.vol; break;
    default: break;
  }
  if (field == 3 || field == 4) {
    double rho = eos_density(p, s.phi[i]);
    double v = rho;
    if (field == 4) {
      v = p.eos == 0 ? p.c0sq * (rho - p.rho0)
                     : p.rho0 * p.c0sq / p.gamma * (pow(rho / p.rho0, p.gamma) - 1.0);
    }
    out[o] = v;
    return;
  }
  if (!src) return;
  for (int k = 0; k < comps; ++k) out[k * n + o] = src[k * n + i];
}

void launch_field(const Params& p, const State& s, const Work& w, int64_t n, int field,
                  double* out, cudaStream_t st) {
  if (n == 0) return;
  k_field<<<(unsigned)div_up(n, 256), 256, 0, st>>>(p, s, w, n, field, out);
}

}  // namespace wbsph
