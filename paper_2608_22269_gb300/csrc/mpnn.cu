// mpnn.cu -- BF16 message-passing surrogate of the pair pass: the network
// over the same neighbour lists, one fused tcgen05 kernel per message-passing
// layer (inference and training forward), mma.sync MLP kernels for the node
// encoder, the decoder and every backward pass, loss, Adam, and the
// surrogate stage rates.
//
// Network (the paper has no learned part): node input f_i = normalised
// (U_i, rho_i/rho0 - 1, phi'_i) plus a dummy flag, phi' = phi - phi_hs(x);
// edge input g_ij = ((x_j - x_i)/h, |x_j - x_i|/h, (U_j - U_i)/s_U,
// (phi'_j - phi'_i)/s_phi) for every fluid receiver i and every particle j
// within 2h; MLP(x) = W2 silu(W1 x + b1) + b2; a node encoder, three layers
// of m_i = sum_j MLP_e([g_ij, h_i, h_j[:32]]), h <- h + MLP_n([h, m]), and a
// decoder to normalised (DU/Dt, Dphi/Dt). Flat parameter layout: blocks node
// encoder, (edge MLP, node MLP) per layer, decoder; each block W1 [in][64],
// b1, W2 [64][out], b2.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/wbsph.h"
#include "common.cuh"
#include "physics.cuh"

namespace wbsph {
const Params* handle_params(wbsph_handle h);
cudaStream_t handle_stream(wbsph_handle h);
int handle_device(wbsph_handle h);
int handle_fail(wbsph_handle h, int code, const char* msg);
void launch_scan_exclusive(uint32_t* data, int64_t total, cudaStream_t st);
void launch_scan_exclusive_chunked(uint32_t* data, int64_t total, uint32_t* scratch, cudaStream_t st);
int scan_scratch_words(int64_t total);
}  // namespace wbsph

using namespace wbsph;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int HID = 64;
constexpr int FEAT = 8;   // padded width of node and edge input features
constexpr int MLP_THREADS = 128;
constexpr int TILE = 64;  // rows per tile (4 warps x 16)

enum { MODE_DIRECT = 0, MODE_LIST = 1, MODE_EDGE = 2, MODE_NODE = 3 };

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragments of m16n8k16 (PTX ISA fragment layouts): lane = 4 g + t.
// A (16x16 at m0,k0): {(g,2t),(g,2t+1)}, {(g+8,2t),..}, {(g,2t+8),..}, {(g+8,2t+8),..}
// B (16x8 at k0,n0):  {(2t,g),(2t+1,g)}, {(2t+8,g),(2t+9,g)}
// C (16x8):           (g,2t),(g,2t+1),(g+8,2t),(g+8,2t+1)
// Row-major smem [m][k] with even k gives 32-bit pair loads.
__device__ __forceinline__ void frag_a_rm(uint32_t r[4], const bf16* s, int ld, int m0, int k0) {
  int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* p0 = reinterpret_cast<const uint32_t*>(s + (m0 + g) * ld + k0 + 2 * t);
  const uint32_t* p1 = reinterpret_cast<const uint32_t*>(s + (m0 + g + 8) * ld + k0 + 2 * t);
  r[0] = p0[0]; r[1] = p1[0]; r[2] = p0[4]; r[3] = p1[4];
}
// B from smem stored [n][k] (k contiguous).
__device__ __forceinline__ void frag_b_nk(uint32_t r[2], const bf16* s, int ld, int k0, int n0) {
  int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t* p = reinterpret_cast<const uint32_t*>(s + (n0 + g) * ld + k0 + 2 * t);
  r[0] = p[0]; r[1] = p[4];
}
// A from smem stored [k][m] (transposed access, 16-bit loads).
__device__ __forceinline__ void frag_a_t(uint32_t r[4], const bf16* s, int ld, int m0, int k0) {
  int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto e = [&](int m, int k) { return s[k * ld + m]; };
  r[0] = pack2(e(m0 + g, k0 + 2 * t), e(m0 + g, k0 + 2 * t + 1));
  r[1] = pack2(e(m0 + g + 8, k0 + 2 * t), e(m0 + g + 8, k0 + 2 * t + 1));
  r[2] = pack2(e(m0 + g, k0 + 2 * t + 8), e(m0 + g, k0 + 2 * t + 9));
  r[3] = pack2(e(m0 + g + 8, k0 + 2 * t + 8), e(m0 + g + 8, k0 + 2 * t + 9));
}
// B from smem stored [k][n] (n contiguous, 16-bit loads).
__device__ __forceinline__ void frag_b_kn(uint32_t r[2], const bf16* s, int ld, int k0, int n0) {
  int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  r[0] = pack2(s[(k0 + 2 * t) * ld + n0 + g], s[(k0 + 2 * t + 1) * ld + n0 + g]);
  r[1] = pack2(s[(k0 + 2 * t + 8) * ld + n0 + g], s[(k0 + 2 * t + 9) * ld + n0 + g]);
}

// ldmatrix: four 8x8 b16 matrices, one row address per lane (16-byte aligned rows).
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const bf16* p) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
// A fragment (16x16 at m0,k0) of row-major [m][k] smem.
__device__ __forceinline__ void ldsm_a(uint32_t r[4], const bf16* s, int ld, int m0, int k0) {
  int lane = threadIdx.x & 31;
  ldsm_x4(r, s + (m0 + (lane & 15)) * ld + k0 + ((lane >> 4) << 3));
}
// B fragments of n-tiles n0 and n0+8 (16 k at k0) of [n][k] smem: b0 = {r0,r1}, b1 = {r2,r3}.
__device__ __forceinline__ void ldsm_b2(uint32_t r[4], const bf16* s, int ld, int k0, int n0) {
  int lane = threadIdx.x & 31;
  ldsm_x4(r, s + (n0 + (lane & 7) + ((lane >> 4) << 3)) * ld + k0 + (((lane >> 3) & 1) << 3));
}

// silu(z) = z sigmoid(z) = h + h tanh(h), h = z / 2, with the hardware tanh
// approximation (one special-function operation instead of an exponential
// and a division; absolute error ~1e-3 |z|, below the BF16 rounding of the
// result)
__device__ __forceinline__ float silu(float z) {
  const float h = 0.5f * z;
  float th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(h));
  return fmaf(h, th, h);
}
__device__ __forceinline__ float silu_grad(float z) {
  float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Inputs and outputs of one fused MLP launch over `rows` rows.
struct MlpArgs {
  const uint32_t* rows_dev;  // row count in device memory (edges), or null
  int64_t rows;              // row count when rows_dev is null
  // gather sources
  const bf16* in;            // DIRECT: [rows][FEAT]; LIST: node table [n][64]
  const uint32_t* list;      // LIST: row -> node
  const bf16* e;             // EDGE: edge inputs [E][8]
  const bf16* h;             // EDGE, NODE: [n][64]
  const uint32_t* recv;      // EDGE
  const uint32_t* send;      // EDGE
  const bf16* agg;           // NODE: [n][64]
  int kin, nout;             // true widths
  int kg;                    // EDGE: edge inputs (2d + 2) at the head of the padded row [g | h_i | h_j[:32]]
  const bf16* w1; const float* b1; const bf16* w2; const float* b2;  // block parameters
  // forward outputs
  bf16* out_bf;              // [rows][64] (+ residual for EDGE/NODE)
  float* out_f;              // [rows][nout] (decoder)
  // decoder of a stage: the de-normalised rates straight into the work arrays
  // (row = fluid index, list[row] = sorted index), with out_f left unwritten
  double* r_dudt; double* r_dphidt; double* r_shift;  // [dim][n], [n], [dim][n]
  const float* r_mean; const float* r_std;            // target mean and std
  int64_t r_n;                                        // particles (array stride)
  // backward
  const float* dout;         // [rows][nout] incoming gradient (EDGE/NODE/DIRECT: [rows][64])
  float* din_row;            // NODE: dh_in ([rows][64], = dout + dX[0:64])
  float* dh;                 // EDGE: atomics into [n][64] (h_i and h_j[:32]); LIST: writes dh[list[row]]
  float* dagg;               // NODE: [rows][64]
  float* gw1; float* gb1; float* gw2; float* gb2;  // FP32 parameter gradients
};

__device__ __forceinline__ int64_t arg_rows(const MlpArgs& a) {
  return a.rows_dev ? (int64_t)*a.rows_dev : a.rows;
}

// Padded input width of the edge MLP: the edge inputs padded to 16, h_i and
// the sender's first 32 features (the message's sender part).
constexpr int EDGE_SEND = 32;
constexpr int EDGE_KP = 16 + HID + EDGE_SEND;

// Row of the block's W1 (flat parameters) that multiplies padded input
// column k, or -1 for a padding column. The edge MLP's W1 rows are the kg
// edge inputs, then h_i (64) and h_j[:32]; its padded input puts the edge
// inputs in columns 0 .. 15.
template <int MODE>
__device__ __forceinline__ int param_row(const MlpArgs& a, int k) {
  if (MODE == MODE_EDGE) return k < 16 ? (k < a.kg ? k : -1) : a.kg + (k - 16);
  return k < a.kin ? k : -1;
}

// Gather of input element pair (k, k+1) of row `row` (KP padded width).
template <int MODE, int KP>
__device__ __forceinline__ uint32_t gather_pair(const MlpArgs& a, int64_t row, int k) {
  if (MODE == MODE_DIRECT) {
    if (k >= FEAT) return 0u;
    return *reinterpret_cast<const uint32_t*>(a.in + row * FEAT + k);
  } else if (MODE == MODE_LIST) {
    return *reinterpret_cast<const uint32_t*>(a.in + (int64_t)a.list[row] * HID + k);
  } else if (MODE == MODE_EDGE) {
    if (k < 16) return k < FEAT ? *reinterpret_cast<const uint32_t*>(a.e + row * FEAT + k) : 0u;
    if (k < 16 + HID) return *reinterpret_cast<const uint32_t*>(a.h + (int64_t)a.recv[row] * HID + k - 16);
    return *reinterpret_cast<const uint32_t*>(a.h + (int64_t)a.send[row] * HID + k - 16 - HID);
  } else {
    if (k < HID) return *reinterpret_cast<const uint32_t*>(a.h + row * HID + k);
    return *reinterpret_cast<const uint32_t*>(a.agg + row * HID + k - HID);
  }
}

template <int MODE, int KP>
__device__ __forceinline__ void load_tile(const MlpArgs& a, int64_t row0, int64_t rows, bf16* X, int ldx) {
  for (int idx = threadIdx.x; idx < TILE * (KP / 2); idx += MLP_THREADS) {
    int r = idx / (KP / 2), k = (idx % (KP / 2)) * 2;
    int64_t row = row0 + r;
    uint32_t v = row < rows ? gather_pair<MODE, KP>(a, row, k) : 0u;
    *reinterpret_cast<uint32_t*>(X + r * ldx + k) = v;
  }
}

// smem layout sizes (elements) with +8 padding per row against bank conflicts
template <int KP, int NP>
struct Smem {
  static constexpr int LDX = KP + 8, LDH = HID + 8, LDO = NP + 8;
  static constexpr size_t fwd_bytes =
      (size_t)(HID * LDX + NP * LDH + TILE * LDX + TILE * LDH) * 2 + (HID + NP) * 4;
};

// ---------------------------------------------------------------------------
// Forward: out = MLP([gathered row]) (+ residual). Weights are staged once per
// CTA (transposed to [n][k]); the CTA then walks row tiles of 64 with the
// gather of the next tile (cp.async, 16-byte chunks, zero fill past the last
// row) in flight while the current tile runs through both GEMMs. The
// residual comes from the staged tile; outputs are staged per warp and
// written as whole 128-byte rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n));
}
// the same copy, cached in L1 as well (rows that neighbouring receivers read again)
__device__ __forceinline__ void cp_async16_ca(void* smem_dst, const void* gsrc, bool valid) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  int n = valid ? 16 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Row indices a tile's gather needs (EDGE: receiver and sender; LIST: node),
// copied asynchronously two tiles ahead into a small ring in shared memory.
template <int MODE>
__device__ __forceinline__ void issue_idx(const MlpArgs& a, int64_t row0, int64_t rows, uint32_t* I) {
  if (MODE == MODE_EDGE || MODE == MODE_LIST) {
    const int per = TILE / 4;  // 16-byte chunks per index array
    const int narr = MODE == MODE_LIST ? 1 : 2;
    if (threadIdx.x < per * narr) {
      int arr = threadIdx.x / per, c = threadIdx.x % per;
      const uint32_t* src = MODE == MODE_LIST ? a.list : (arr == 0 ? a.recv : a.send);
      int64_t r = row0 + c * 4;
      bool valid = r + 3 < rows;  // a partial last chunk is gathered below with plain loads
      cp_async16(I + arr * TILE + c * 4, valid ? (const void*)(src + r) : (const void*)a.w1, valid);
      if (!valid)
        for (int q = 0; q < 4; ++q) I[arr * TILE + c * 4 + q] = (r + q < rows) ? src[r + q] : 0u;
    }
  }
  cp_async_commit();
}

// Source of 16-byte chunk c8 (8 elements) of tile row r (row < rows).
template <int MODE>
__device__ __forceinline__ const bf16* chunk_src(const MlpArgs& a, int64_t row, int r, int c8,
                                                 const uint32_t* I) {
  if (MODE == MODE_DIRECT) return a.in + row * FEAT;  // only chunk 0 carries data
  if (MODE == MODE_LIST) return a.in + (int64_t)I[r] * HID + c8 * 8;
  static_assert(MODE != MODE_EDGE, "the edge MLP runs forward in the fused layer kernel");
  if (c8 < 8) return a.h + row * HID + c8 * 8;
  return a.agg + row * HID + (c8 - 8) * 8;
}

template <int MODE, int KP>
__device__ __forceinline__ void issue_tile(const MlpArgs& a, int64_t row0, int64_t rows, bf16* X, int ldx,
                                           const uint32_t* I) {
  constexpr int C8 = KP / 8;
  for (int idx = threadIdx.x; idx < TILE * C8; idx += MLP_THREADS) {
    int r = idx / C8, c8 = idx % C8;
    int64_t row = row0 + r;
    bool valid = row < rows && (MODE != MODE_DIRECT || c8 == 0);
    const bf16* src = valid ? chunk_src<MODE>(a, row, r, c8, I) : a.w1;  // any address when zero-filling
    cp_async16(X + r * ldx + c8 * 8, src, valid);
  }
  cp_async_commit();
}

template <int MODE, int KP, int NP>
struct FwdSmem {
  static constexpr int LDX = KP + 8, LDH = HID + 8;
  static constexpr size_t bytes = (size_t)(HID * LDX + NP * LDH + 2 * TILE * LDX + TILE * LDH) * 2 +
                                  (HID + NP) * 4 + 3 * 2 * TILE * 4;
};

template <int MODE, int KP, int NP>
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_fwd(MlpArgs a) {
  using S = FwdSmem<MODE, KP, NP>;
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* W1t = reinterpret_cast<bf16*>(smem);      // [64][LDX]  W1t[n][k] = W1[k][n]
  bf16* W2t = W1t + HID * S::LDX;                  // [NP][LDH]  W2t[o][c] = W2[c][o]
  bf16* Xb = W2t + NP * S::LDH;                    // 2 x [64][LDX]
  bf16* A1 = Xb + 2 * TILE * S::LDX;               // [64][LDH]
  float* B1 = reinterpret_cast<float*>(A1 + TILE * S::LDH);
  float* B2 = B1 + HID;
  uint32_t* Ib = reinterpret_cast<uint32_t*>(B2 + NP);  // 3 x [2][64] row indices
  const int64_t rows = arg_rows(a);
  const int64_t stride = gridDim.x;
  int64_t tile = blockIdx.x;
  // pipeline: indices two tiles ahead, rows one tile ahead. Commit order per
  // tile t: idx(t+2), data(t+1); so waiting for all but the newest group
  // leaves data(t) and idx(t+1) complete.
  issue_idx<MODE>(a, tile * TILE, rows, Ib);
  issue_idx<MODE>(a, (tile + stride) * TILE, rows, Ib + 2 * TILE);
  cp_async_wait<1>();
  __syncthreads();
  if (tile * TILE < rows) issue_tile<MODE, KP>(a, tile * TILE, rows, Xb, S::LDX, Ib);
  else cp_async_commit();
  const bf16 zero = __float2bfloat16(0.f);
  for (int idx = threadIdx.x; idx < HID * KP; idx += MLP_THREADS) {
    int n = idx / KP, k = idx % KP;
    W1t[n * S::LDX + k] = k < a.kin ? a.w1[k * HID + n] : zero;
  }
  for (int idx = threadIdx.x; idx < NP * HID; idx += MLP_THREADS) {
    int o = idx / HID, c = idx % HID;
    W2t[o * S::LDH + c] = o < a.nout ? a.w2[c * a.nout + o] : zero;
  }
  for (int idx = threadIdx.x; idx < HID; idx += MLP_THREADS) B1[idx] = a.b1[idx];
  for (int idx = threadIdx.x; idx < NP; idx += MLP_THREADS) B2[idx] = idx < a.nout ? a.b2[idx] : 0.f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int m0 = warp * 16;
  for (int buf = 0, ring = 0; tile * TILE < rows; tile += stride, buf ^= 1, ring = (ring + 1) % 3) {
    const int64_t row0 = tile * TILE;
    bf16* X = Xb + buf * TILE * S::LDX;
    issue_idx<MODE>(a, (tile + 2 * stride) * TILE, rows, Ib + ((ring + 2) % 3) * 2 * TILE);
    cp_async_wait<1>();
    __syncthreads();  // data(t) and idx(t+1) visible to all threads
    if ((tile + stride) * TILE < rows)
      issue_tile<MODE, KP>(a, (tile + stride) * TILE, rows, Xb + (buf ^ 1) * TILE * S::LDX, S::LDX,
                           Ib + ((ring + 1) % 3) * 2 * TILE);
    else
      cp_async_commit();
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KP / 16; ++kt) {
      uint32_t af[4];
      ldsm_a(af, X, S::LDX, m0, kt * 16);
#pragma unroll
      for (int nt = 0; nt < 8; nt += 2) {
        uint32_t bq[4];
        ldsm_b2(bq, W1t, S::LDX, kt * 16, nt * 8);
        mma16816(acc[nt], af, bq);
        mma16816(acc[nt + 1], af, bq + 2);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      int c = nt * 8 + 2 * t;
      *reinterpret_cast<__nv_bfloat162*>(A1 + (m0 + g) * S::LDH + c) =
          __floats2bfloat162_rn(silu(acc[nt][0] + B1[c]), silu(acc[nt][1] + B1[c + 1]));
      *reinterpret_cast<__nv_bfloat162*>(A1 + (m0 + g + 8) * S::LDH + c) =
          __floats2bfloat162_rn(silu(acc[nt][2] + B1[c]), silu(acc[nt][3] + B1[c + 1]));
    }
    __syncwarp();
    float acc2[NP / 8][4];
#pragma unroll
    for (int nt = 0; nt < NP / 8; ++nt) acc2[nt][0] = acc2[nt][1] = acc2[nt][2] = acc2[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < HID / 16; ++kt) {
      uint32_t af[4];
      ldsm_a(af, A1, S::LDH, m0, kt * 16);
#pragma unroll
      for (int nt = 0; nt < NP / 8; nt += 2) {
        uint32_t bq[4];
        ldsm_b2(bq, W2t, S::LDH, kt * 16, nt * 8);
        mma16816(acc2[nt], af, bq);
        mma16816(acc2[nt + 1], af, bq + 2);
      }
    }
    __syncwarp();
    if (a.r_dudt) {  // decoder of a stage: rates (shifting velocity zero), few columns
      const int dim = a.nout - 1;
#pragma unroll
      for (int nt = 0; nt < NP / 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = m0 + g + (q >> 1) * 8, o = nt * 8 + 2 * t + (q & 1);
          int64_t row = row0 + r;
          if (row < rows && o < a.nout) {
            const int64_t i = a.list[row];
            const double v = (double)(acc2[nt][q] + B2[o]) * a.r_std[o] + a.r_mean[o];
            if (o < dim) {
              a.r_dudt[o * a.r_n + i] = v;
              a.r_shift[o * a.r_n + i] = 0.0;
            } else {
              a.r_dphidt[i] = v;
            }
          }
        }
    } else if (a.out_f) {  // decoder: FP32 outputs, few columns
#pragma unroll
      for (int nt = 0; nt < NP / 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = m0 + g + (q >> 1) * 8, o = nt * 8 + 2 * t + (q & 1);
          int64_t row = row0 + r;
          if (row < rows && o < a.nout) a.out_f[row * a.nout + o] = acc2[nt][q] + B2[o];
        }
    } else {
      // bias and residual (first 64 staged columns are e for EDGE, h for NODE)
#pragma unroll
      for (int nt = 0; nt < NP / 8; ++nt)
#pragma unroll
        for (int hq = 0; hq < 2; ++hq) {
          int r = m0 + g + hq * 8, o = nt * 8 + 2 * t;
          float v0 = acc2[nt][2 * hq] + B2[o], v1 = acc2[nt][2 * hq + 1] + B2[o + 1];
          if (MODE == MODE_NODE) {
            __nv_bfloat162 res = *reinterpret_cast<const __nv_bfloat162*>(X + r * S::LDX + o);
            v0 += __bfloat162float(res.x);
            v1 += __bfloat162float(res.y);
          }
          *reinterpret_cast<__nv_bfloat162*>(A1 + r * S::LDH + o) = __floats2bfloat162_rn(v0, v1);
        }
      __syncwarp();
      // the warp's 16 output rows, 8 chunks of 16 bytes each
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int idx = q * 32 + lane, r = m0 + (idx >> 3), c8 = idx & 7;
        int64_t row = row0 + r;
        if (row < rows)
          *reinterpret_cast<uint4*>(a.out_bf + row * HID + c8 * 8) =
              *reinterpret_cast<const uint4*>(A1 + r * S::LDH + c8 * 8);
      }
    }
    __syncthreads();  // X[buf] is refilled by the next-but-one prefetch
  }
}

// ---------------------------------------------------------------------------
// tcgen05 helpers. Operands sit in shared memory in the K-major
// 128-byte-swizzled layout the tensor core reads through matrix descriptors
// (row r of 64 BF16 = 128 B at r * 128, 16-byte chunk c stored at chunk
// c ^ (r % 8); 8-row groups 1024 B apart); FP32 accumulators live in tensor
// memory (TMEM: lane = operand row) and are read back by the warp that owns
// those 32 lanes. One thread issues the MMAs and their commit to an
// mbarrier; every wait on an mbarrier is bounded.
// ---------------------------------------------------------------------------
constexpr int TC_ROWS = 128;
constexpr uint32_t TC_TILE_BYTES = TC_ROWS * 128;        // 128 rows x 64 BF16
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16,
// both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (the leading-dimension offset is unused in this layout)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// byte offset of 16-byte chunk c of row r in the swizzled layout
__device__ __forceinline__ uint32_t sw128(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// bounded wait for the mbarrier phase `parity`; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit = TC_WAIT_LIMIT) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}



// ---------------------------------------------------------------------------
// Edge inputs of the network for receiver i and sender j, from the per-node
// FP32 packs A = (x, y, z, phi') and B = (U, 0) (phi' = phi - phi_hs):
// ((x_j - x_i)/h, |x_j - x_i|/h, (U_j - U_i)/s_U, (phi'_j - phi'_i)/s_phi),
// 2d + 2 values rounded to BF16 and zero padded to 8 (one 16-byte row). The
// fused layer kernel and the training graph both form them here, so that
// the backward sees exactly the inputs of the forward. |x_j - x_i| takes the
// hardware's approximate square root: its error of a few FP32 units in the
// last place changes the BF16 feature only next to a BF16 rounding boundary.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 edge_features(int dim, float4 ai, float4 bi, float4 aj, float4 bj,
                                               float inv_h, float inv_su, float inv_sphi) {
  const float rx = aj.x - ai.x, ry = aj.y - ai.y, rz = aj.z - ai.z;  // z = 0 in 2D
  float rn;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(rn) : "f"(fmaf(rx, rx, fmaf(ry, ry, rz * rz))));
  float f[8];
  if (dim == 3) {
    f[0] = rx * inv_h; f[1] = ry * inv_h; f[2] = rz * inv_h; f[3] = rn * inv_h;
    f[4] = (bj.x - bi.x) * inv_su; f[5] = (bj.y - bi.y) * inv_su; f[6] = (bj.z - bi.z) * inv_su;
    f[7] = (aj.w - ai.w) * inv_sphi;
  } else {
    f[0] = rx * inv_h; f[1] = ry * inv_h; f[2] = rn * inv_h;
    f[3] = (bj.x - bi.x) * inv_su; f[4] = (bj.y - bi.y) * inv_su; f[5] = (aj.w - ai.w) * inv_sphi;
    f[6] = 0.f; f[7] = 0.f;
  }
  uint4 v;
  v.x = pack2(__float2bfloat16(f[0]), __float2bfloat16(f[1]));
  v.y = pack2(__float2bfloat16(f[2]), __float2bfloat16(f[3]));
  v.z = pack2(__float2bfloat16(f[4]), __float2bfloat16(f[5]));
  v.w = pack2(__float2bfloat16(f[6]), __float2bfloat16(f[7]));
  return v;
}

// 16 FP32 columns of this thread's TMEM lane (32x32b shape), one wait
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t bf2_u32(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ __nv_bfloat162 u32_bf2(uint32_t v) { return *reinterpret_cast<__nv_bfloat162*>(&v); }

// ---------------------------------------------------------------------------
// One message-passing layer, fused, on tcgen05:
//   m_i = sum_j MLP_e([g_ij, h_i, h_j[:SEND]]) = (sum_j silu(z_ij)) W2 + n_i b2,
//   z_ij = g_ij W_g + h_i W_r + h_j[:SEND] W_s + b1,   h'_i = h_i + MLP_n([h_i, m_i]).
// The second layer of the message MLP is linear, so it is applied once per
// receiver, to the sum of the receiver's SiLU rows, rather than once per
// edge. Nothing per edge is ever written to memory. A sender contributes
// the first SEND = 32 of its 64 state features, so a gathered row is 64 B,
// plus a 32-byte pack per edge, from L2.
//
// A tile is 128 receivers (fluid particles in sorted order, one TMEM lane and
// one shared-memory operand row each; then tiles of wall particles, which
// receive no messages). Step k of a tile takes the k-th entry of every
// receiver's k-major neighbour list. One CTA per SM, split into roles that
// hand off through mbarriers (no CTA-wide barrier inside the loop):
//   - gather: two groups of four warps, for the even and the odd steps;
//     thread r fills row r. Per step, the 16-wide edge-input row goes into a
//     slot of an 8-deep operand ring. It is formed from the FP32 packs of
//     receiver and sender, prefetched two of the group's steps ahead (the
//     neighbour index three). The sender's first SEND features go into the
//     slot by cp.async, through L1 (neighbouring receivers read the same rows
//     over a tile's steps). A slot is announced on its "full" barrier once the
//     thread's copies into it have landed. A thread announces its slots
//     three at a time, under one proxy fence, once a fourth copy group is in
//     flight: the fence is the costly part, and no thread blocks on a fresh
//     copy. Group 0 also writes the tile record (counts, node ids, longest
//     list, tile index), group 1 the tile's h_i rows.
//   - MMA: one thread. Per tile it issues P_r / 2 = h_i W_r / 2. Per step it
//     issues D = G W_g/2 + H W_s/2 into a ring of four TMEM accumulators:
//     three K = 16 MMAs, M = 128, N = 64, BF16 in, FP32 out. Per tile it
//     then issues the W2 product of the summed SiLU rows and the node MLP's
//     two GEMMs.
//   - epilogue: eight warps; thread (r, ch) holds TMEM lane r and the
//     accumulator column half ch.
//       Per step: u = D + (P_r + b1)/2 in BF16, then silu(2u) = u + u tanh(u)
//       with the packed BF16 hardware tanh (the first-layer weights were
//       halved on staging, exactly, in BF16). The result is added in FP32
//       to 32 running sums; receivers without a k-th neighbour add nothing.
//       At the end of the tile: the sums go to shared memory as BF16 high
//       and low parts (s = hi + lo to about 2^-17 relative), and the tensor
//       core forms (hi + lo) W2. m_i = that + n_i b2 is rounded to BF16.
//       Then z = [h_i, m_i] W1 + b1, the hidden layer silu(z), and
//       h'_i = h_i + silu(z) W2 + b2.
// The terms of a receiver's message sum are its BF16-rounded SiLU rows; the
// sum is rounded once, at the end. A CTA's first tile is fixed by its index;
// the following ones come from a counter shared by all CTAs, so that CTAs
// that drew long fluid tiles take fewer. Every mbarrier wait is bounded. A
// timeout in any role ends all roles and is reported through the status
// word.
// ---------------------------------------------------------------------------
constexpr int SEND = 32;               // sender features in a message (the first SEND of h_j)
constexpr uint32_t MS_W_BYTES = 8192;  // [64][64] BF16 weight tile, K-major swizzled
constexpr int MS_NW = 7;

struct MsgArgs {
  int64_t nf, nd;
  const uint32_t* fluid_list;
  const uint32_t* dummy_list;
  const uint32_t* nbr;      // k-major exact neighbour lists of the fluid particles
  const uint32_t* nbr_cnt;
  const float4* pack;       // per node: (x, y, z, phi'), (U, 0)
  const bf16* h_in;         // [n][64]
  bf16* h_out;              // [n][64]
  bf16* m_out;              // [n][64] message sums (training), or null
  const bf16* we_w1; const float* we_b1; const bf16* we_w2; const float* we_b2;  // edge MLP
  const bf16* wn_w1; const float* wn_b1; const bf16* wn_w2; const float* wn_b2;  // node MLP
  int dim, kg;              // kg = 2d + 2 edge inputs
  float inv_h, inv_su, inv_sphi;
  unsigned* status;
  int* tile_ctr;            // tiles handed out beyond each CTA's first (zeroed per launch)
};

constexpr int MS_NS = 8;                       // operand ring slots
constexpr int MS_ND = 4;                       // step accumulators in TMEM
constexpr int MS_GATHER = 128, MS_EPI = 256;   // threads of one gather group, of the epilogue
constexpr int MS_THREADS = 2 * MS_GATHER + MS_EPI + 32;
constexpr int MS_NTILES = 2 + 4 + 2 + 2;       // edge inputs, sender rows, h_i (x2), sum hi / m_i / hidden, sum lo
constexpr int MS_INFO = 128 * 2 + 4;           // ints per tile record: cnt[128], node[128], kmax, tile
// mbarriers (full: the producer is done with it; free: the consumer is)
enum {
  WB_SFULL = 0, WB_SFREE = WB_SFULL + MS_NS,                   // operand ring slots: gather -> MMA
  WB_DFULL = WB_SFREE + MS_NS, WB_DFREE = WB_DFULL + MS_ND,    // step accumulators: MMA -> epilogue
  WB_HFULL = WB_DFREE + MS_ND, WB_HFREE = WB_HFULL + 2,         // h_i tiles, by tile parity
  WB_IFULL = WB_HFREE + 2, WB_IFREE = WB_IFULL + 2,             // tile records, by tile parity
  WB_PR = WB_IFREE + 2, WB_HL = WB_PR + 1, WB_DM = WB_HL + 1,   // P_r; summed SiLU rows; their W2 product
  WB_M = WB_DM + 1, WB_Z = WB_M + 1, WB_ZT = WB_Z + 1, WB_O = WB_ZT + 1,  // node MLP operands and products
  WB_TILE = WB_O + 1,                                           // the tile index, within gather group 0
  WB_FIN = WB_TILE + 2, WB_COUNT = WB_FIN + 1                   // the last MMA, before TMEM is released
};
constexpr size_t MS_SMEM_BYTES = 1024 + MS_NW * MS_W_BYTES + 256 * 4 + (size_t)MS_NTILES * TC_TILE_BYTES +
                                 2 * MS_INFO * 4 + WB_COUNT * 8 + 16;

__device__ __forceinline__ void ms_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}
// bounded wait on the phase `parity`; gives up early once another role has aborted
// (`polls`, when given, receives the number of polls made)
__device__ __forceinline__ bool ms_wait(uint32_t mbar, uint32_t parity, volatile int* abort_flag,
                                        uint32_t limit = TC_WAIT_LIMIT, uint32_t* polls = nullptr) {
  bool ok = false;
  uint32_t it = 0;
  for (; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) {
      ok = true;
      break;
    }
    if ((it & 1023u) == 1023u && *abort_flag) break;
  }
  if (polls) *polls = it;
  if (!ok && it == limit) *abort_flag = 1;
  return ok;
}

// the same wait, decided for the whole warp (the roles that use it run
// warp-collective instructions after it, so a warp never splits on a timeout)
__device__ __forceinline__ bool ms_wait_warp(uint32_t mbar, uint32_t parity, volatile int* abort_flag,
                                             uint32_t limit = TC_WAIT_LIMIT, uint32_t* polls = nullptr) {
  return __all_sync(0xffffffffu, ms_wait(mbar, parity, abort_flag, limit, polls));
}

// Check of the fused layer's bounded waits (failure detection without a GPU
// fault). Warp 0 waits, for at most `limit` polls, on an mbarrier that
// nothing arrives on; when the limit runs out it raises the CTA's abort
// flag. Warp 1 waits on a second such mbarrier with a limit 64 times as long
// (at most 2^26 polls) and must leave as soon as it sees the flag, as every
// role of the layer leaves when another role times out. The timeout is
// reported through the status word only when both happened: warp 0 timed
// out, and warp 1 left on the flag before its own limit. The kernel ends
// normally either way.
__global__ void k_wait_probe(unsigned* status, uint32_t limit) {
  __shared__ uint64_t bar[2];
  __shared__ int abort_flag;
  __shared__ uint32_t polls1;
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    for (int i = 0; i < 2; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
    polls1 = 0;
  }
  __syncthreads();
  const uint64_t l1 = (uint64_t)limit * 64u;
  const uint32_t limit1 = l1 < (1u << 26) ? (uint32_t)l1 : (1u << 26);
  uint32_t polls = 0;
  ms_wait_warp(smem_u32(bar + warp), 0u, &abort_flag, warp == 0 ? limit : limit1, &polls);
  if (warp == 1 && (t & 31) == 0) polls1 = polls;
  __syncthreads();
  if (t == 0 && abort_flag && polls1 < limit1) atomicOr(status, (unsigned)kStatTimeout);
}

// (a0, a1) += the two BF16 halves of w (low, high), FP32 adds with BF16 operands
__device__ __forceinline__ void add_bf16x2_f32(float& a0, float& a1, uint32_t w) {
  asm("{\n.reg .b16 lo, hi;\nmov.b32 {lo, hi}, %2;\nadd.rn.f32.bf16 %0, lo, %0;\nadd.rn.f32.bf16 %1, hi, %1;\n}\n"
      : "+f"(a0), "+f"(a1)
      : "r"(w));
}

__global__ void __launch_bounds__(MS_THREADS, 1) k_message_tc(const MsgArgs a) {
  extern __shared__ unsigned char ms_raw[];
  unsigned char* base = ms_raw + ((1024u - (smem_u32(ms_raw) & 1023u)) & 1023u);  // 1024-byte aligned
  enum { WG = 0, WS = 1, WR = 2, WE2 = 3, WH = 4, WM = 5, WN2 = 6 };
  unsigned char* W = base;
  float* bias = reinterpret_cast<float*>(W + MS_NW * MS_W_BYTES);  // b1/2 | b2 (edge) | b1 | b2 (node)
  unsigned char* TG = reinterpret_cast<unsigned char*>(bias + 256);  // edge inputs: slots 0-3, 4-7
  unsigned char* TH = TG + 2 * TC_TILE_BYTES;    // sender rows, two slots per tile
  unsigned char* THI = TH + 4 * TC_TILE_BYTES;   // h_i rows, by tile parity
  unsigned char* TM = THI + 2 * TC_TILE_BYTES;   // sum_j silu (high part), m_i, the node MLP's hidden layer
  unsigned char* TL = TM + TC_TILE_BYTES;        // sum_j silu (low part)
  int* info = reinterpret_cast<int*>(TL + TC_TILE_BYTES);
  uint64_t* bar = reinterpret_cast<uint64_t*>(info + 2 * MS_INFO);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + WB_COUNT);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

  // weights (K-major, 128-byte swizzle, [n][k] = W[k][n]); the first layer
  // of the edge MLP halved; its input rows: kg edge inputs, h_i, h_j
  const bf16 zero = __float2bfloat16(0.f);
  auto half = [](bf16 v) { return __float2bfloat16(0.5f * __bfloat162float(v)); };
  for (int idx = t; idx < 64 * 64; idx += MS_THREADS) {
    const int n = idx >> 6, k = idx & 63;
    const uint32_t off = sw128(n, k >> 3) + (k & 7) * 2;
    auto put = [&](int w, bf16 v) { *reinterpret_cast<bf16*>(W + w * MS_W_BYTES + off) = v; };
    put(WG, k < a.kg ? half(a.we_w1[k * HID + n]) : zero);
    put(WR, half(a.we_w1[(a.kg + k) * HID + n]));
    put(WS, k < SEND ? half(a.we_w1[(a.kg + HID + k) * HID + n]) : zero);
    put(WE2, a.we_w2[k * HID + n]);
    put(WH, a.wn_w1[k * HID + n]);
    put(WM, a.wn_w1[(HID + k) * HID + n]);
    put(WN2, a.wn_w2[k * HID + n]);
  }
  if (t < 64) {
    bias[t] = 0.5f * a.we_b1[t];
    bias[64 + t] = a.we_b2[t];
    bias[128 + t] = a.wn_b1[t];
    bias[192 + t] = a.wn_b2[t];
  }
  // the K padding chunk of every edge-input slot stays zero
  for (int idx = t; idx < 128 * MS_NS; idx += MS_THREADS) {
    const int r = idx / MS_NS, s = idx % MS_NS;
    *reinterpret_cast<uint4*>(TG + (s >> 2) * TC_TILE_BYTES + sw128(r, 2 * (s & 3) + 1)) =
        make_uint4(0u, 0u, 0u, 0u);
  }
  if (t == 0) {
    *abort_flag = 0;
    auto init = [&](int i, uint32_t count) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar + i)), "r"(count) : "memory");
    };
    for (int s = 0; s < MS_NS; ++s) { init(WB_SFULL + s, MS_GATHER); init(WB_SFREE + s, 1); }
    for (int d = 0; d < MS_ND; ++d) { init(WB_DFULL + d, 1); init(WB_DFREE + d, MS_EPI / 32); }
    for (int i = 0; i < 2; ++i) {
      init(WB_HFULL + i, MS_GATHER); init(WB_HFREE + i, MS_EPI);
      init(WB_IFULL + i, MS_GATHER); init(WB_IFREE + i, MS_EPI);
    }
    init(WB_PR, 1); init(WB_HL, MS_EPI); init(WB_DM, 1);
    init(WB_M, MS_EPI); init(WB_Z, 1); init(WB_ZT, MS_EPI); init(WB_O, 1);
    init(WB_TILE, 1); init(WB_TILE + 1, 1); init(WB_FIN, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 16) {  // the MMA warp owns the TMEM allocation
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "n"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // TMEM columns: step accumulators 0-255, (sum_j silu) W2 256, P_r 320, node MLP z 384 and output 448
  const uint32_t TD = tmem, TDM = tmem + 256u, TPR = tmem + 320u, TZ = tmem + 384u, TO = tmem + 448u;
  auto B = [&](int i) { return smem_u32(bar + i); };
  const int64_t ntf = div_up(a.nf, 128), ntd = div_up(a.nd, 128), ntiles = ntf + ntd;

  if (warp < 8) {
    // ---- gather: two groups of four warps, even and odd steps; thread r of
    // a group fills row r of its steps' operand slots. Group 0 also writes
    // the tile record, group 1 the h_i rows. A slot (or h_i tile) is
    // announced once this thread's copies into it have landed. When a copy
    // group is committed with QD unannounced ones before it, those QD are
    // announced together: one wait for all but the newest group, one proxy
    // fence, QD arrivals. A thread waits for a free slot with at most QD
    // unannounced groups, spanning fewer than 2 QD < MS_NS steps, so the MMA
    // never waits for a slot whose announcement waits for a slot to free.
    constexpr int QD = 3;
    const int grp = warp >> 2, r = t & 127;
    uint32_t q0 = 0, q1 = 0, q2 = 0;  // barriers of the copy groups in flight, oldest first
    int nq = 0;
    auto announce_oldest = [&]() {
      ms_arrive(q0);
      q0 = q1;
      q1 = q2;
      --nq;
    };
    auto push = [&](uint32_t mb) {  // after the commit of the group that fills mb
      if (nq == QD) {
        cp_async_wait<1>();
        fence_async_smem();
        announce_oldest();
        announce_oldest();
        announce_oldest();
      }
      (nq == 0 ? q0 : nq == 1 ? q1 : q2) = mb;
      ++nq;
    };
    auto flush_to = [&](int keep) {  // announce all but the newest `keep` groups
      if (nq <= keep) return;
      if (keep <= 0) cp_async_wait<0>();
      else if (keep == 1) cp_async_wait<1>();
      else cp_async_wait<2>();
      fence_async_smem();
      while (nq > keep) announce_oldest();
    };
    uint32_t gs0 = 0;      // index of the tile's first step in this CTA
    int prev_groups = QD;  // copy groups of this thread in the previous tile
    int64_t next = blockIdx.x;  // thread 0: this CTA's next tile (the first by the CTA's index,
                                // then from a counter shared by all CTAs)
    bool ok = true;
    for (int it = 0;; ++it) {
      const int tb = it & 1;
      int* inf = info + tb * MS_INFO;
      // this thread's groups of tile it - 2 are announced before waiting for its end
      flush_to(min(prev_groups, QD));
      int groups = 0;
      int64_t tile, gi;
      int cnt, kmax;
      uint32_t node;
      bool valid;
      if (grp == 0) {
        if (!(ok = ms_wait_warp(B(WB_IFREE + tb), ((it >> 1) & 1) ^ 1, abort_flag))) break;
        if (t == 0) {
          inf[257] = (int)(next < ntiles ? next : ntiles);
          ms_arrive(B(WB_TILE + tb));
          if (next < ntiles) next = (int64_t)gridDim.x + atomicAdd(a.tile_ctr, 1);
        }
        if (!(ok = ms_wait_warp(B(WB_TILE + tb), (it >> 1) & 1, abort_flag))) break;
        tile = inf[257];
        if (tile >= ntiles) {  // the end, for every role
          ms_arrive(B(WB_IFULL + tb));
          break;
        }
        const bool fluid = tile < ntf;
        const int64_t row0 = (fluid ? tile : tile - ntf) * 128, rows = fluid ? a.nf : a.nd;
        gi = row0 + r;
        valid = gi < rows;
        node = valid ? __ldg((fluid ? a.fluid_list : a.dummy_list) + gi) : 0u;
        cnt = (valid && fluid) ? (int)__ldg(a.nbr_cnt + gi) : 0;
        // the tile's longest list
        int km = 0;
        if (fluid) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int64_t g2 = row0 + 32 * c + lane;
            if (g2 < rows) km = max(km, (int)__ldg(a.nbr_cnt + g2));
          }
        }
        kmax = __reduce_max_sync(0xffffffffu, km);
        inf[r] = cnt;
        inf[128 + r] = (int)node;
        if (r == 0) inf[256] = kmax;
        ms_arrive(B(WB_IFULL + tb));
      } else {
        if (!(ok = ms_wait_warp(B(WB_IFULL + tb), (it >> 1) & 1, abort_flag))) break;
        tile = inf[257];
        if (tile >= ntiles) break;
        cnt = inf[r];
        node = (uint32_t)inf[128 + r];
        kmax = inf[256];
        const bool fluid = tile < ntf;
        gi = (fluid ? tile : tile - ntf) * 128 + r;
        valid = gi < (fluid ? a.nf : a.nd);
        if (!(ok = ms_wait_warp(B(WB_HFREE + tb), ((it >> 1) & 1) ^ 1, abort_flag))) break;
        unsigned char* T = THI + tb * TC_TILE_BYTES;
        const bf16* src = a.h_in + (int64_t)node * HID;
#pragma unroll
        for (int c = 0; c < 8; ++c) cp_async16(T + sw128(r, c), src + c * 8, valid);
        cp_async_commit();
        push(B(WB_HFULL + tb));
        groups = 1;
      }
      // this group's tile steps k0, k0 + 2, ...
      const int k0 = (int)((gs0 ^ (uint32_t)grp) & 1u);
      if (k0 < kmax) {
        const float4 ai = __ldg(a.pack + 2 * node), bi = __ldg(a.pack + 2 * node + 1);
        // neighbour indices three of the group's steps ahead, packs two
        uint32_t j0 = k0 < cnt ? __ldg(a.nbr + (int64_t)k0 * a.nf + gi) : 0u;
        uint32_t j1 = k0 + 2 < cnt ? __ldg(a.nbr + (int64_t)(k0 + 2) * a.nf + gi) : 0u;
        uint32_t j2 = k0 + 4 < cnt ? __ldg(a.nbr + (int64_t)(k0 + 4) * a.nf + gi) : 0u;
        int64_t o6 = (int64_t)(k0 + 6) * a.nf + gi;  // offset of this row's entry k + 6
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 aj0 = z4, bj0 = z4, aj1 = z4, bj1 = z4;
        if (k0 < cnt) { aj0 = __ldg(a.pack + 2 * j0); bj0 = __ldg(a.pack + 2 * j0 + 1); }
        if (k0 + 2 < cnt) { aj1 = __ldg(a.pack + 2 * j1); bj1 = __ldg(a.pack + 2 * j1 + 1); }
        for (int k = k0; k < kmax; k += 2) {
          const uint32_t gs = gs0 + (uint32_t)k;
          const int s = (int)(gs % MS_NS);
          const uint32_t j3 = k + 6 < cnt ? __ldg(a.nbr + o6) : 0u;
          o6 += 2 * a.nf;
          float4 aj2 = z4, bj2 = z4;
          if (k + 4 < cnt) { aj2 = __ldg(a.pack + 2 * j2); bj2 = __ldg(a.pack + 2 * j2 + 1); }
          const bool act = k < cnt;
          uint4 f = make_uint4(0u, 0u, 0u, 0u);
          if (act) f = edge_features(a.dim, ai, bi, aj0, bj0, a.inv_h, a.inv_su, a.inv_sphi);
          if (!(ok = ms_wait_warp(B(WB_SFREE + s), (uint32_t)((gs / MS_NS) & 1) ^ 1u, abort_flag))) break;
          *reinterpret_cast<uint4*>(TG + (s >> 2) * TC_TILE_BYTES + sw128(r, 2 * (s & 3))) = f;
          {
            unsigned char* T = TH + (s >> 1) * TC_TILE_BYTES;
            const bf16* src = a.h_in + (int64_t)j0 * HID;
#pragma unroll
            for (int c = 0; c < 4; ++c) cp_async16_ca(T + sw128(r, 4 * (s & 1) + c), src + c * 8, act);
          }
          cp_async_commit();
          push(B(WB_SFULL + s));
          ++groups;
          j0 = j1; j1 = j2; j2 = j3;
          aj0 = aj1; bj0 = bj1; aj1 = aj2; bj1 = bj2;
        }
        if (!ok) break;
      }
      gs0 += (uint32_t)kmax;
      prev_groups = groups;
    }
    if (ok) flush_to(0);
    cp_async_wait<0>();
  } else if (warp < 16) {
    // ---- epilogue: row r (TMEM lane), column half ch ----
    const int ew = warp - 8;
    const int q = ew & 3, ch = ew >> 2, r = q * 32 + lane;
    const uint32_t lane_off = ((uint32_t)(q * 32) << 16) + 32u * ch;
    const float* b1h = bias;
    const float* b2e = bias + 64;
    const float* b1n = bias + 128;
    const float* b2n = bias + 192;
    uint32_t gs = 0;
    int nmsg = 0;
    bool ok = true;
    for (int it = 0;; ++it) {
      const int tb = it & 1;
      if (!(ok = ms_wait_warp(B(WB_IFULL + tb), (it >> 1) & 1, abort_flag))) break;
      const int* inf = info + tb * MS_INFO;
      const int64_t tile = inf[257];
      if (tile >= ntiles) break;
      const int cnt = inf[r];
      const uint32_t node = (uint32_t)inf[128 + r];
      const int kmax = inf[256];
      const bool fluid = tile < ntf;
      const bool valid = (fluid ? tile : tile - ntf) * 128 + r < (fluid ? a.nf : a.nd);
      if (kmax > 0) {
        if (!(ok = ms_wait_warp(B(WB_PR), nmsg & 1, abort_flag))) break;
        tc_fence_after();
        uint32_t pr[16];  // (P_r + b1) / 2 of this thread's 32 columns, BF16 pairs
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16];
          tc_ld16(TPR + lane_off + 16 * hh, v);
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const int col = 32 * ch + 16 * hh + 2 * p;
            pr[8 * hh + p] = bf2_u32(__floats2bfloat162_rn(v[2 * p] + b1h[col], v[2 * p + 1] + b1h[col + 1]));
          }
        }
        float acc[32];  // sum_j silu(z_ij) of this thread's 32 columns
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = 0.f;
        for (int k = 0; k < kmax; ++k, ++gs) {
          const int d = (int)(gs % MS_ND);
          if (!(ok = ms_wait_warp(B(WB_DFULL + d), (uint32_t)((gs / MS_ND) & 1), abort_flag))) break;
          tc_fence_after();
          const bool act = k < cnt;
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            float v[16];
            tc_ld16(TD + 64u * d + lane_off + 16 * hh, v);
            if (hh == 1) {  // both loads complete (warp-collective waits): one arrival for the warp
              tc_fence_before();
              if (lane == 0) ms_arrive(B(WB_DFREE + d));
            }
            if (act) {
#pragma unroll
              for (int p = 0; p < 8; ++p) {
                const __nv_bfloat162 u =
                    __hadd2(__floats2bfloat162_rn(v[2 * p], v[2 * p + 1]), u32_bf2(pr[8 * hh + p]));
                uint32_t th;
                asm("tanh.approx.bf16x2 %0, %1;" : "=r"(th) : "r"(bf2_u32(u)));
                add_bf16x2_f32(acc[16 * hh + 2 * p], acc[16 * hh + 2 * p + 1], bf2_u32(__hfma2(u, u32_bf2(th), u)));
              }
            }
          }
        }
        if (!ok) break;
        // the sums as BF16 high and low parts, the operands of their W2 product
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t oh[8], ol[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const float s0 = acc[16 * hh + 2 * p], s1 = acc[16 * hh + 2 * p + 1];
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(s0, s1);
            const float2 hf = __bfloat1622float2(h2);
            oh[p] = bf2_u32(h2);
            ol[p] = bf2_u32(__floats2bfloat162_rn(s0 - hf.x, s1 - hf.y));
          }
          *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh)) = make_uint4(oh[0], oh[1], oh[2], oh[3]);
          *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh + 1)) = make_uint4(oh[4], oh[5], oh[6], oh[7]);
          *reinterpret_cast<uint4*>(TL + sw128(r, ch * 4 + 2 * hh)) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
          *reinterpret_cast<uint4*>(TL + sw128(r, ch * 4 + 2 * hh + 1)) = make_uint4(ol[4], ol[5], ol[6], ol[7]);
        }
        fence_async_smem();
        tc_fence_before();
        ms_arrive(B(WB_HL));
        // m_i = (sum_j silu(z_ij)) W2 + n_i b2
        if (!(ok = ms_wait_warp(B(WB_DM), nmsg & 1, abort_flag))) break;
        tc_fence_after();
        ++nmsg;
        const float fc = (float)cnt;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16];
          tc_ld16(TDM + lane_off + 16 * hh, v);
          uint32_t o[8];
#pragma unroll
          for (int p = 0; p < 8; ++p) {
            const int col = 32 * ch + 16 * hh + 2 * p;
            o[p] = bf2_u32(
                __floats2bfloat162_rn(fmaf(fc, b2e[col], v[2 * p]), fmaf(fc, b2e[col + 1], v[2 * p + 1])));
          }
          const uint4 o0 = make_uint4(o[0], o[1], o[2], o[3]), o1 = make_uint4(o[4], o[5], o[6], o[7]);
          *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh)) = o0;
          *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh + 1)) = o1;
          if (a.m_out && valid) {
            uint4* mo = reinterpret_cast<uint4*>(a.m_out + (int64_t)node * HID + 32 * ch + 16 * hh);
            mo[0] = o0;
            mo[1] = o1;
          }
        }
      } else {  // no messages: m_i = 0
#pragma unroll
        for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + c)) = make_uint4(0u, 0u, 0u, 0u);
      }
      fence_async_smem();
      tc_fence_before();
      ms_arrive(B(WB_M));
      // node MLP: z = [h_i, m_i] W1 + b1, hidden layer silu(z) into TM
      if (!(ok = ms_wait_warp(B(WB_Z), it & 1, abort_flag))) break;
      tc_fence_after();
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float v[16];
        tc_ld16(TZ + lane_off + 16 * hh, v);
        uint32_t o[8];
#pragma unroll
        for (int p = 0; p < 8; ++p) {
          const int col = 32 * ch + 16 * hh + 2 * p;
          o[p] = bf2_u32(__floats2bfloat162_rn(silu(v[2 * p] + b1n[col]), silu(v[2 * p + 1] + b1n[col + 1])));
        }
        *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh)) = make_uint4(o[0], o[1], o[2], o[3]);
        *reinterpret_cast<uint4*>(TM + sw128(r, ch * 4 + 2 * hh + 1)) = make_uint4(o[4], o[5], o[6], o[7]);
      }
      fence_async_smem();
      tc_fence_before();
      ms_arrive(B(WB_ZT));
      // h'_i = h_i + silu(z) W2 + b2
      if (!(ok = ms_wait_warp(B(WB_O), it & 1, abort_flag))) break;
      tc_fence_after();
      const unsigned char* HI = THI + tb * TC_TILE_BYTES;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float v[16];
        tc_ld16(TO + lane_off + 16 * hh, v);
        uint32_t o[8];
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const uint4 hv = *reinterpret_cast<const uint4*>(HI + sw128(r, ch * 4 + 2 * hh + cc));
          const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int pp = 4 * cc + p, col = 32 * ch + 16 * hh + 2 * pp;
            const float2 hf = __bfloat1622float2(u32_bf2(hw[p]));
            o[pp] = bf2_u32(
                __floats2bfloat162_rn(hf.x + v[2 * pp] + b2n[col], hf.y + v[2 * pp + 1] + b2n[col + 1]));
          }
        }
        if (valid) {
          uint4* ho = reinterpret_cast<uint4*>(a.h_out + (int64_t)node * HID + 32 * ch + 16 * hh);
          ho[0] = make_uint4(o[0], o[1], o[2], o[3]);
          ho[1] = make_uint4(o[4], o[5], o[6], o[7]);
        }
      }
      tc_fence_before();
      ms_arrive(B(WB_HFREE + tb));
      ms_arrive(B(WB_IFREE + tb));
    }
  } else if (lane == 0) {
    // ---- the MMA thread ----
    const uint64_t dW[MS_NW] = {tc_desc(smem_u32(W)), tc_desc(smem_u32(W + MS_W_BYTES)),
                                tc_desc(smem_u32(W + 2 * MS_W_BYTES)), tc_desc(smem_u32(W + 3 * MS_W_BYTES)),
                                tc_desc(smem_u32(W + 4 * MS_W_BYTES)), tc_desc(smem_u32(W + 5 * MS_W_BYTES)),
                                tc_desc(smem_u32(W + 6 * MS_W_BYTES))};
    auto mma_k64 = [&](uint32_t d, uint64_t dA, int w, bool accumulate) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) tc_mma(d, dA + 2 * kk, dW[w] + 2 * kk, (accumulate || kk > 0) ? 1u : 0u);
    };
    const uint64_t dTG = tc_desc(smem_u32(TG)), dTH = tc_desc(smem_u32(TH));
    const uint64_t dTHI = tc_desc(smem_u32(THI)), dTM = tc_desc(smem_u32(TM));
    constexpr uint64_t tile16 = TC_TILE_BYTES >> 4;  // descriptor address step of one tile
    const uint64_t dTL = tc_desc(smem_u32(TL));
    uint32_t gs = 0;
    int it = 0, nmsg = 0;
    bool ok = true;
    for (;; ++it) {
      const int tb = it & 1;
      if (!(ok = ms_wait(B(WB_IFULL + tb), (it >> 1) & 1, abort_flag))) break;
      if (info[tb * MS_INFO + 257] >= ntiles) break;
      const int kmax = info[tb * MS_INFO + 256];
      if (!(ok = ms_wait(B(WB_HFULL + tb), (it >> 1) & 1, abort_flag))) break;
      tc_fence_after();
      const uint64_t dHI = dTHI + tb * tile16;
      if (kmax > 0) {
        mma_k64(TPR, dHI, WR, false);  // P_r / 2 = h_i W_r / 2
        tc_commit(B(WB_PR));
        for (int k = 0; k < kmax; ++k, ++gs) {
          const int s = (int)(gs % MS_NS), d = (int)(gs % MS_ND);
          if (!(ok = ms_wait(B(WB_SFULL + s), (uint32_t)((gs / MS_NS) & 1), abort_flag))) break;
          if (!(ok = ms_wait(B(WB_DFREE + d), (uint32_t)((gs / MS_ND) & 1) ^ 1u, abort_flag))) break;
          tc_fence_after();
          const uint32_t dd = TD + 64u * d;
          tc_mma(dd, dTG + (s >> 2) * tile16 + 2 * (s & 3), dW[WG], 0u);
          const uint64_t dA = dTH + (s >> 1) * tile16 + 4 * (s & 1);
#pragma unroll
          for (int kk = 0; kk < SEND / 16; ++kk) tc_mma(dd, dA + 2 * kk, dW[WS] + 2 * kk, 1u);
          tc_commit(B(WB_DFULL + d));
          tc_commit(B(WB_SFREE + s));
        }
        if (!ok) break;
        // (sum_j silu) W2 from the high and low parts
        if (!(ok = ms_wait(B(WB_HL), nmsg & 1, abort_flag))) break;
        ++nmsg;
        tc_fence_after();
        mma_k64(TDM, dTM, WE2, false);
        mma_k64(TDM, dTL, WE2, true);
        tc_commit(B(WB_DM));
      }
      // node MLP: z = [h_i, m_i] W1 + b1, then the output layer
      if (!(ok = ms_wait(B(WB_M), it & 1, abort_flag))) break;
      tc_fence_after();
      mma_k64(TZ, dHI, WH, false);
      mma_k64(TZ, dTM, WM, true);
      tc_commit(B(WB_Z));
      if (!(ok = ms_wait(B(WB_ZT), it & 1, abort_flag))) break;
      tc_fence_after();
      mma_k64(TO, dTM, WN2, false);
      tc_commit(B(WB_O));
    }
    // every MMA issued has completed before TMEM is released
    tc_commit(B(WB_FIN));
    mbar_wait(B(WB_FIN), 0u);
  }
  tc_fence_before();
  __syncthreads();
  if (t == 0 && *abort_flag) atomicOr(a.status, (unsigned)kStatTimeout);
  if (warp == 16) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(512) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Backward of one fused MLP over its rows: recompute z1 = X W1 + b1 and
// a1 = silu(z1); dA1 = dOut W2^T; dZ = dA1 * silu'(z1); dX = dZ W1^T,
// scattered to the gather sources; dW1 += X^T dZ, dW2 += a1^T dOut,
// db1 += sum dZ, db2 += sum dOut. Each warp owns a fixed set of the weight-
// gradient tiles and accumulates them in shared memory across the CTA's row
// tiles; one atomic add per element and CTA at the end.
// ---------------------------------------------------------------------------
template <int KP, int NP>
struct BwdSmem {
  static constexpr int LDX = KP + 8, LDH = HID + 8, LDO = NP + 8, LDW1 = HID + 8;
  // W1t [64][LDX], W1r [KP][LDW1], W2r [64][LDO], W2t (not needed), X [64][LDX],
  // A1 [64][LDH], DZ [64][LDH], DO [64][LDO]; FP32: gW1 [KP][64], gW2 [64][NP], gb1 [64], gb2 [NP], B1 [64]
  static constexpr size_t bf_elems = (size_t)HID * LDX + (size_t)KP * LDW1 + (size_t)HID * LDO +
                                     (size_t)TILE * LDX + 2 * (size_t)TILE * LDH + (size_t)TILE * LDO;
  static constexpr size_t f_elems = (size_t)KP * HID + (size_t)HID * NP + HID + NP + HID;
  static constexpr size_t bytes = bf_elems * 2 + f_elems * 4;
};

template <int MODE, int KP, int NP>
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_bwd(MlpArgs a) {
  using S = BwdSmem<KP, NP>;
  extern __shared__ __align__(16) unsigned char smem[];
  bf16* W1t = reinterpret_cast<bf16*>(smem);   // [64][LDX]   W1t[c][k] = W1[k][c]
  bf16* W1r = W1t + HID * S::LDX;               // [KP][LDW1]  W1r[k][c] = W1[k][c]
  bf16* W2r = W1r + KP * S::LDW1;               // [64][LDO]   W2r[c][o] = W2[c][o]
  bf16* X = W2r + HID * S::LDO;                 // [64][LDX]
  bf16* A1 = X + TILE * S::LDX;                 // [64][LDH]
  bf16* DZ = A1 + TILE * S::LDH;                // [64][LDH]
  bf16* DO = DZ + TILE * S::LDH;                // [64][LDO]
  float* gW1 = reinterpret_cast<float*>(DO + TILE * S::LDO);  // [KP][64]
  float* gW2 = gW1 + KP * HID;                  // [64][NP]
  float* gB1 = gW2 + HID * NP;
  float* gB2 = gB1 + HID;
  float* B1 = gB2 + NP;
  const bf16 zero = __float2bfloat16(0.f);
  for (int idx = threadIdx.x; idx < HID * KP; idx += MLP_THREADS) {
    int c = idx / KP, k = idx % KP;
    const int pr = param_row<MODE>(a, k);
    bf16 v = pr >= 0 ? a.w1[pr * HID + c] : zero;
    W1t[c * S::LDX + k] = v;
    W1r[k * S::LDW1 + c] = v;
  }
  for (int idx = threadIdx.x; idx < HID * NP; idx += MLP_THREADS) {
    int c = idx / NP, o = idx % NP;
    W2r[c * S::LDO + o] = o < a.nout ? a.w2[c * a.nout + o] : zero;
  }
  for (int idx = threadIdx.x; idx < KP * HID + HID * NP + HID + NP; idx += MLP_THREADS) gW1[idx] = 0.f;
  for (int idx = threadIdx.x; idx < HID; idx += MLP_THREADS) B1[idx] = a.b1[idx];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int m0 = warp * 16;
  const int64_t rows = arg_rows(a);
  const int dstride = (MODE == MODE_LIST) ? a.nout : HID;  // incoming gradient row width
  for (int64_t tile = blockIdx.x; tile * TILE < rows; tile += gridDim.x) {
    const int64_t row0 = tile * TILE;
    load_tile<MODE, KP>(a, row0, rows, X, S::LDX);
    for (int idx = threadIdx.x; idx < TILE * NP; idx += MLP_THREADS) {
      int r = idx / NP, o = idx % NP;
      int64_t row = row0 + r;
      float v = (row < rows && o < a.nout) ? a.dout[row * dstride + o] : 0.f;
      DO[r * S::LDO + o] = __float2bfloat16(v);
    }
    __syncthreads();
    // bias gradient of the second layer from the FP32 incoming gradient
    for (int o = threadIdx.x; o < a.nout; o += MLP_THREADS) {
      float sacc = 0.f;
      for (int r = 0; r < TILE && row0 + r < rows; ++r) sacc += a.dout[(row0 + r) * dstride + o];
      gB2[o] += sacc;
    }
    // recompute z1 (warp's 16 rows x 64)
    float z[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KP / 16; ++kt) {
      uint32_t af[4];
      frag_a_rm(af, X, S::LDX, m0, kt * 16);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t bfr[2];
        frag_b_nk(bfr, W1t, S::LDX, kt * 16, nt * 8);
        mma16816(z[nt], af, bfr);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int r = m0 + g + (q >> 1) * 8, c = nt * 8 + 2 * t + (q & 1);
        z[nt][q] += B1[c];
        A1[r * S::LDH + c] = __float2bfloat16(silu(z[nt][q]));
      }
    }
    // dA1 = dOut W2^T  (B[k=o][n=c] = W2[c][o] = W2r[c][o] -> stored [n][k])
    float da[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) da[nt][0] = da[nt][1] = da[nt][2] = da[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < NP / 16; ++kt) {
      uint32_t af[4];
      frag_a_rm(af, DO, S::LDO, m0, kt * 16);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        uint32_t bfr[2];
        frag_b_nk(bfr, W2r, S::LDO, kt * 16, nt * 8);
        mma16816(da[nt], af, bfr);
      }
    }
    // dZ = dA1 * silu'(z1); bias gradient of the first layer
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float cs0 = 0.f, cs1 = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int r = m0 + g + (q >> 1) * 8, c = nt * 8 + 2 * t + (q & 1);
        bool valid = row0 + r < rows;
        float dz = valid ? da[nt][q] * silu_grad(z[nt][q]) : 0.f;
        DZ[r * S::LDH + c] = __float2bfloat16(dz);
        if (q & 1) cs1 += dz; else cs0 += dz;
      }
      for (int off = 4; off < 32; off <<= 1) {
        cs0 += __shfl_xor_sync(0xffffffffu, cs0, off);
        cs1 += __shfl_xor_sync(0xffffffffu, cs1, off);
      }
      if (g == 0) {
        atomicAdd(&gB1[nt * 8 + 2 * t], cs0);
        atomicAdd(&gB1[nt * 8 + 2 * t + 1], cs1);
      }
    }
    __syncthreads();
    // dX = dZ W1^T (B[k=c][n=k_in] = W1[k_in][c] = W1r[k_in][c] -> stored [n][k]); scatter
    if (MODE != MODE_DIRECT) {
#pragma unroll 1
      for (int nt = 0; nt < KP / 8; ++nt) {
        float dx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < HID / 16; ++kt) {
          uint32_t af[4], bfr[2];
          frag_a_rm(af, DZ, S::LDH, m0, kt * 16);
          frag_b_nk(bfr, W1r, S::LDW1, kt * 16, nt * 8);
          mma16816(dx, af, bfr);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int r = m0 + g + (q >> 1) * 8, k = nt * 8 + 2 * t + (q & 1);
          int64_t row = row0 + r;
          if (row >= rows || param_row<MODE>(a, k) < 0) continue;
          float v = dx[q];
          if (MODE == MODE_LIST) {
            a.dh[(int64_t)a.list[row] * HID + k] = v;
          } else if (MODE == MODE_EDGE) {  // edge inputs take no gradient; h_i, h_j scatter
            if (k < 16) continue;
            if (k < 16 + HID) atomicAdd(&a.dh[(int64_t)a.recv[row] * HID + k - 16], v);
            else atomicAdd(&a.dh[(int64_t)a.send[row] * HID + k - 16 - HID], v);
          } else {  // MODE_NODE
            if (k < HID) a.din_row[row * HID + k] = a.dout[row * HID + k] + v;
            else a.dagg[row * HID + k - HID] = v;
          }
        }
      }
    }
    // weight gradients: tiles (mt, nt) of dW1 [KP x 64] and dW2 [64 x NP], round-robin over warps
    {
      constexpr int T1 = (KP / 16) * 8;
      for (int tt = warp; tt < T1; tt += 4) {
        int mt = tt / 8, nt = tt % 8;
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < TILE / 16; ++kt) {
          uint32_t af[4], bfr[2];
          frag_a_t(af, X, S::LDX, mt * 16, kt * 16);     // A[m=k_in][k=row] = X[row][k_in]
          frag_b_kn(bfr, DZ, S::LDH, kt * 16, nt * 8);   // B[k=row][n=c] = DZ[row][c]
          mma16816(c, af, bfr);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int m = mt * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          gW1[m * HID + n] += c[q];
        }
      }
      constexpr int T2 = (HID / 16) * (NP / 8);
      for (int tt = warp; tt < T2; tt += 4) {
        int mt = tt / (NP / 8), nt = tt % (NP / 8);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < TILE / 16; ++kt) {
          uint32_t af[4], bfr[2];
          frag_a_t(af, A1, S::LDH, mt * 16, kt * 16);    // A[m=c][k=row] = A1[row][c]
          frag_b_kn(bfr, DO, S::LDO, kt * 16, nt * 8);   // B[k=row][n=o] = DO[row][o]
          mma16816(c, af, bfr);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int m = mt * 16 + g + (q >> 1) * 8, n = nt * 8 + 2 * t + (q & 1);
          gW2[m * NP + n] += c[q];
        }
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < KP * HID; idx += MLP_THREADS) {
    const int pr = param_row<MODE>(a, idx / HID);
    if (pr >= 0) atomicAdd(&a.gw1[pr * HID + idx % HID], gW1[idx]);
  }
  for (int idx = threadIdx.x; idx < HID * a.nout; idx += MLP_THREADS) {
    int c = idx / a.nout, o = idx % a.nout;
    atomicAdd(&a.gw2[idx], gW2[c * NP + o]);
  }
  for (int idx = threadIdx.x; idx < HID; idx += MLP_THREADS) atomicAdd(&a.gb1[idx], gB1[idx]);
  for (int idx = threadIdx.x; idx < a.nout; idx += MLP_THREADS) atomicAdd(&a.gb2[idx], gB2[idx]);
}

// ---------------------------------------------------------------------------
// Graph, features, loss, optimiser
// ---------------------------------------------------------------------------
// Node inputs and packs. Node input (BF16, 8 wide): (U, rho/rho0 - 1, phi')
// minus the mean over the std, then the dummy flag, with the hydrostatic
// split phi' = phi - phi_hs(x), phi_hs = G.x + |G| H (FP64, like the mixed
// path). Pack (FP32, 32 B per node) for the edge inputs: (x, y, z, phi') and (U, 0).
__global__ void k_sg_nodes(Params p, State s, int64_t n, const float* mean, const float* stdv, bf16* nf_out,
                           float4* pack) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double phs = p.phs0, xs[3] = {0.0, 0.0, 0.0}, us[3] = {0.0, 0.0, 0.0};
  for (int d = 0; d < p.dim; ++d) {
    xs[d] = s.x[d * n + i];
    us[d] = s.u[d * n + i];
    phs = fma(p.g[d], xs[d], phs);
  }
  const double phip = s.phi[i] - phs;
  float v[FEAT] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = 0; d < p.dim; ++d) v[d] = (float)us[d];
  // rho/rho0 - 1 in FP32 (the input is rounded to BF16): expm1 of phi/C0^2
  // (linear EOS) or the Tait power minus one
  const float phf = (float)s.phi[i];
  if (p.eos == 0) {
    v[p.dim] = expm1f(phf * p.inv_c0sq_f);
  } else {
    const float gm1 = (float)(p.gamma - 1.0);
    v[p.dim] = powf(fmaf(gm1 * phf, p.inv_c0sq_f, 1.f), 1.f / gm1) - 1.f;
  }
  v[p.dim + 1] = (float)phip;
  for (int k = 0; k < p.dim + 2; ++k) v[k] = (v[k] - mean[k]) / stdv[k];
  v[p.dim + 2] = s.type[i] == kFluid ? 0.f : 1.f;
  uint4 o;
  o.x = pack2(__float2bfloat16(v[0]), __float2bfloat16(v[1]));
  o.y = pack2(__float2bfloat16(v[2]), __float2bfloat16(v[3]));
  o.z = pack2(__float2bfloat16(v[4]), __float2bfloat16(v[5]));
  o.w = pack2(__float2bfloat16(v[6]), __float2bfloat16(v[7]));
  *reinterpret_cast<uint4*>(nf_out + i * FEAT) = o;
  pack[2 * i] = make_float4((float)xs[0], (float)xs[1], (float)xs[2], (float)phip);
  pack[2 * i + 1] = make_float4((float)us[0], (float)us[1], (float)us[2], 0.f);
}

// Training graph: edges (receiver, sender) in CSR order by receiver and
// their inputs (edge_features, the same function the fused layer uses), for
// the backward pass. A warp covers the receivers g0 .. g0 + 31 and the
// contiguous range of their edges; lane l takes edges l, l + 32, ... of that
// range and finds its receiver by a binary search over the lanes' row
// starts, so every store of recv, send and the 16-byte input rows coalesces.
__global__ void k_sg_fill(int dim, Work w, int64_t nf, const uint32_t* row_ptr, const float4* pack,
                          float inv_h, float inv_su, float inv_sphi, uint32_t* recv,
                          uint32_t* send, bf16* efeat) {
  const int lane = threadIdx.x & 31;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane;
  if (g0 >= nf) return;  // whole warps leave together
  const int64_t gl = g0 + lane;
  const uint32_t start = row_ptr[gl < nf ? gl : nf];  // row_ptr holds nf + 1 entries
  const uint32_t e_end = __shfl_sync(0xffffffffu, start, 31) + (g0 + 31 < nf ? w.nbr_cnt[g0 + 31] : 0u);
  const uint32_t e_beg = __shfl_sync(0xffffffffu, start, 0);
  for (uint32_t e0 = e_beg; e0 < e_end; e0 += 32) {
    const uint32_t e = e0 + (uint32_t)lane;
    int r = 0;  // receiver lane: the last lane whose row starts at or before e
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const uint32_t st_c = __shfl_sync(0xffffffffu, start, r + step);
      if (r + step < 32 && g0 + r + step < nf && st_c <= e) r += step;
    }
    const uint32_t st_r = __shfl_sync(0xffffffffu, start, r);
    if (e >= e_end) continue;
    const uint32_t i = w.fluid_list[g0 + r];
    const uint32_t j = w.nbr[(int64_t)(e - st_r) * nf + g0 + r];  // every list entry is an exact neighbour
    recv[e] = i;
    send[e] = j;
    *reinterpret_cast<uint4*>(efeat + (int64_t)e * FEAT) =
        edge_features(dim, __ldg(pack + 2 * i), __ldg(pack + 2 * i + 1), __ldg(pack + 2 * j), __ldg(pack + 2 * j + 1),
                      inv_h, inv_su, inv_sphi);
  }
}

// de_e = dm_recv(e): the gradient of a receiver's message sum reaches each of its edges
__global__ void k_sg_aggregate_bwd(const uint32_t* fluid_list, int64_t nf, const uint32_t* row_ptr,
                                   const float* dagg_rows, float* de) {
  int64_t gi = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (gi >= nf) return;
  uint32_t i = fluid_list[gi];
  float2 g = reinterpret_cast<const float2*>(dagg_rows + (int64_t)i * HID)[lane];
  for (uint32_t k = row_ptr[gi]; k < row_ptr[gi + 1]; ++k) reinterpret_cast<float2*>(de + (int64_t)k * HID)[lane] = g;
}

// normalised targets from the plain rates; loss and its gradient (fluid rows)
__global__ void k_sg_loss(int dim, Work w, int64_t n, int64_t nf, const float* out, const float* tmean,
                          const float* tstd, float* dout, double* loss) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double l = 0.0;
  int no = dim + 1;
  if (gi < nf) {
    uint32_t i = w.fluid_list[gi];
    for (int o = 0; o < no; ++o) {
      double y = o < dim ? w.dudt[o * n + i] : w.dphidt[i];
      float tn = (float)((y - tmean[o]) / tstd[o]);
      float d = out[gi * no + o] - tn;
      l += (double)d * d;
      dout[gi * no + o] = 2.f * d / (float)(nf * no);
    }
  }
  for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l / (double)(nf * no));
}

// Control of the gain test: the rates of the last plain stage of a rollout,
// kept per particle (by original id) and replayed in later stages.
__global__ void k_frozen_store(int dim, Work w, const uint32_t* oid, int64_t n, int64_t nf, double* frozen,
                               int64_t cap) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= nf) return;
  const uint32_t i = w.fluid_list[gi], o = oid[i];
  for (int d = 0; d < dim; ++d) frozen[d * cap + o] = w.dudt[d * n + i];
  frozen[dim * cap + o] = w.dphidt[i];
}
__global__ void k_frozen_rates(int dim, Work w, const uint32_t* oid, int64_t n, int64_t nf, const double* frozen,
                               int64_t cap) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= nf) return;
  const uint32_t i = w.fluid_list[gi], o = oid[i];
  for (int d = 0; d < dim; ++d) {
    w.dudt[d * n + i] = frozen[d * cap + o];
    w.dushift[d * n + i] = 0.0;
  }
  w.dphidt[i] = frozen[dim * cap + o];
}

__global__ void k_adam(int64_t np, float* p, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2, bf16* pb) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= np) return;
  float gk = g[k];
  float mk = b1 * m[k] + (1.f - b1) * gk;
  float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  p[k] = pk;
  pb[k] = __float2bfloat16(pk);
}

__global__ void k_to_bf16(int64_t np, const float* p, bf16* pb) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < np) pb[k] = __float2bfloat16(p[k]);
}

struct Block {
  int kin, nout;
  int64_t w1, b1, w2, b2;  // offsets into the flat parameter vector
};

}  // namespace

// ---------------------------------------------------------------------------
// Surrogate object
// ---------------------------------------------------------------------------
struct wbsph_surrogate_s {
  wbsph_surrogate_config cfg;
  int dim = 2, layers = 3, mode = WBSPH_SURROGATE_NETWORK;
  std::vector<Block> blocks;
  int64_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16* pb = nullptr;
  float* norm = nullptr;  // node mean[8], node std[8], target mean[4], target std[4], edge std[2]
  float edge_std[2] = {1.f, 1.f};
  int64_t adam_t = 0;
  // node buffers (inference and training), sized on demand
  int64_t cap_n = 0, cap_nf = 0;
  bf16* nfeat = nullptr;
  float4* pack = nullptr;  // per node: (x, y, z, phi'), (U, 0)
  std::vector<bf16*> hs;
  float* out = nullptr;
  // training: the graph, message sums and gradients
  int64_t cap_tn = 0, cap_e = 0;
  uint32_t *row_ptr = nullptr, *recv = nullptr, *send = nullptr, *scan_tmp = nullptr;
  bf16* efeat = nullptr;
  std::vector<bf16*> ms;
  float *dout = nullptr, *dh = nullptr, *de = nullptr, *dagg = nullptr;
  double* loss = nullptr;
  int64_t E = 0;
  // frozen-rates control: rates by original id
  double* frozen = nullptr;
  int64_t cap_frozen = 0;
  int* tile_ctr = nullptr;  // dynamic tile counter of the fused layer
  std::string err;
};

namespace {

int sfail(wbsph_surrogate s, int code, const char* msg) {
  if (s) s->err = msg;
  return code;
}

// flat layout: node encoder, (edge MLP, node MLP) per layer, decoder
void build_blocks(wbsph_surrogate s) {
  int d = s->dim;
  int64_t off = 0;
  auto add = [&](int kin, int nout) {
    Block b;
    b.kin = kin; b.nout = nout;
    b.w1 = off; off += (int64_t)kin * HID;
    b.b1 = off; off += HID;
    b.w2 = off; off += (int64_t)HID * nout;
    b.b2 = off; off += nout;
    s->blocks.push_back(b);
  };
  add(d + 3, HID);
  for (int l = 0; l < s->layers; ++l) {
    add(2 * d + 2 + HID + EDGE_SEND, HID);
    add(2 * HID, HID);
  }
  add(HID, d + 1);
  s->np = off;
}

template <class T>
bool dalloc(T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *p = (T*)q;
  return true;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_train(wbsph_surrogate s) {
  dfree(s->row_ptr); dfree(s->recv); dfree(s->send); dfree(s->efeat); dfree(s->scan_tmp);
  for (auto* q : s->ms) dfree(q);
  s->ms.clear();
  dfree(s->dout); dfree(s->dh); dfree(s->de); dfree(s->dagg);
  s->row_ptr = s->recv = s->send = s->scan_tmp = nullptr;
  s->efeat = nullptr;
  s->dout = s->dh = s->de = s->dagg = nullptr;
  s->cap_tn = s->cap_e = 0;
}

void free_graph(wbsph_surrogate s) {
  free_train(s);
  dfree(s->nfeat); dfree(s->pack); dfree(s->out);
  for (auto* q : s->hs) dfree(q);
  s->hs.clear();
  s->nfeat = nullptr;
  s->pack = nullptr;
  s->out = nullptr;
  s->cap_n = s->cap_nf = 0;
}

int ensure_nodes(wbsph_surrogate s, int64_t n, int64_t nf) {
  if (n <= s->cap_n && nf <= s->cap_nf) return WBSPH_OK;
  free_graph(s);
  s->cap_n = n; s->cap_nf = nf;
  bool ok = dalloc(&s->nfeat, n * FEAT) && dalloc(&s->pack, 2 * n) && dalloc(&s->out, nf * 4);
  for (int l = 0; ok && l <= s->layers; ++l) {
    bf16* q = nullptr;
    ok = dalloc(&q, n * HID);
    s->hs.push_back(q);
  }
  return ok ? WBSPH_OK : sfail(s, WBSPH_E_NOMEM, "surrogate node buffers");
}

int ensure_train_nodes(wbsph_surrogate s, int64_t n, int64_t nf) {
  if (n <= s->cap_tn && nf <= s->cap_nf && s->row_ptr) return WBSPH_OK;
  free_train(s);
  s->cap_tn = n;
  bool ok = dalloc(&s->row_ptr, s->cap_nf + 1) && dalloc(&s->dout, s->cap_nf * 4) && dalloc(&s->dh, n * HID) &&
            dalloc(&s->dagg, n * HID) && dalloc(&s->scan_tmp, (size_t)scan_scratch_words(s->cap_nf + 1));
  for (int l = 0; ok && l < s->layers; ++l) {
    bf16* q = nullptr;
    ok = dalloc(&q, n * HID);
    s->ms.push_back(q);
  }
  return ok ? WBSPH_OK : sfail(s, WBSPH_E_NOMEM, "surrogate training buffers");
}

int ensure_edges(wbsph_surrogate s, int64_t E) {
  if (E <= s->cap_e) return WBSPH_OK;
  dfree(s->recv); dfree(s->send); dfree(s->efeat); dfree(s->de);
  int64_t cap = E + E / 4 + 1024;
  bool ok = dalloc(&s->recv, cap) && dalloc(&s->send, cap) && dalloc(&s->efeat, cap * FEAT) &&
            dalloc(&s->de, cap * HID);
  s->cap_e = ok ? cap : 0;
  return ok ? WBSPH_OK : sfail(s, WBSPH_E_NOMEM, "surrogate edge buffers");
}

// Persistent grid of every block that fits at once (the tile loop strides by
// the grid, so blocks beyond the resident ones would start late).
// returns the launch's error, which a later runtime call could otherwise consume
template <int MODE, int KP, int NP>
cudaError_t launch_fwd(const MlpArgs& a, int64_t max_rows, cudaStream_t st) {
  size_t sm = FwdSmem<MODE, KP, NP>::bytes;
  static int resident = 0;
  if (!resident) {
    cudaFuncSetAttribute(k_mlp_fwd<MODE, KP, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_fwd<MODE, KP, NP>, MLP_THREADS, sm);
    resident = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 4);
  }
  int64_t tiles = div_up(max_rows > 0 ? max_rows : 1, TILE);
  int grid = (int)(tiles < resident ? tiles : resident);
  k_mlp_fwd<MODE, KP, NP><<<grid, MLP_THREADS, sm, st>>>(a);
  return cudaGetLastError();
}

template <int MODE, int KP, int NP>
void launch_bwd(const MlpArgs& a, int64_t max_rows, cudaStream_t st) {
  size_t sm = BwdSmem<KP, NP>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_bwd<MODE, KP, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  int64_t tiles = div_up(max_rows > 0 ? max_rows : 1, TILE);
  int grid = (int)(tiles < 152 ? tiles : 152);
  k_mlp_bwd<MODE, KP, NP><<<grid, MLP_THREADS, sm, st>>>(a);
}

MlpArgs block_args(wbsph_surrogate s, int bi) {
  const Block& b = s->blocks[bi];
  MlpArgs a;
  memset(&a, 0, sizeof a);
  a.kin = b.kin;
  a.nout = b.nout;
  a.w1 = s->pb + b.w1; a.b1 = s->p + b.b1; a.w2 = s->pb + b.w2; a.b2 = s->p + b.b2;
  a.gw1 = s->g + b.w1; a.gb1 = s->g + b.b1; a.gw2 = s->g + b.w2; a.gb2 = s->g + b.b2;
  return a;
}

// One fused message-passing layer (k_message_tc): persistent CTAs, one per
// SM (221 KB of shared memory and 512 TMEM columns each); returns the
// launch's error.
cudaError_t launch_message(wbsph_surrogate s, const Params& p, const Work& w, int64_t nf, int64_t nd, int l,
                           const bf16* h_in, bf16* h_out, bf16* m_out, cudaStream_t st) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    cudaFuncSetAttribute(k_message_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MS_SMEM_BYTES);
  }
  const Block& be = s->blocks[1 + 2 * l];
  const Block& bn = s->blocks[2 + 2 * l];
  MsgArgs a;
  memset(&a, 0, sizeof a);
  a.nf = nf; a.nd = nd;
  a.fluid_list = w.fluid_list; a.dummy_list = w.dummy_list; a.nbr = w.nbr; a.nbr_cnt = w.nbr_cnt;
  a.pack = s->pack;
  a.h_in = h_in; a.h_out = h_out; a.m_out = m_out;
  a.we_w1 = s->pb + be.w1; a.we_b1 = s->p + be.b1; a.we_w2 = s->pb + be.w2; a.we_b2 = s->p + be.b2;
  a.wn_w1 = s->pb + bn.w1; a.wn_b1 = s->p + bn.b1; a.wn_w2 = s->pb + bn.w2; a.wn_b2 = s->p + bn.b2;
  a.dim = p.dim; a.kg = 2 * p.dim + 2;
  a.inv_h = (float)(1.0 / p.h);
  a.inv_su = 1.f / s->edge_std[0];
  a.inv_sphi = 1.f / s->edge_std[1];
  a.status = w.status;
  a.tile_ctr = s->tile_ctr;
  const int64_t tiles = div_up(nf, 128) + div_up(nd, 128);
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)(tiles < sms ? tiles : sms);
  cudaMemsetAsync(s->tile_ctr, 0, sizeof(int), st);
  k_message_tc<<<grid, MS_THREADS, MS_SMEM_BYTES, st>>>(a);
  return cudaGetLastError();
}

// node inputs and packs of the sim's current state (wall particles updated)
void node_inputs(wbsph_surrogate s, const Params& p, const State& st, int64_t n, cudaStream_t cs) {
  if (n > 0)
    k_sg_nodes<<<(unsigned)div_up(n, 256), 256, 0, cs>>>(p, st, n, s->norm, s->norm + 8, s->nfeat, s->pack);
}

// Training graph of the sim's current state (neighbour lists built).
int build_graph(wbsph_surrogate s, const Params& p, const Work& w, int64_t n, int64_t nf, cudaStream_t cs) {
  int rc = ensure_train_nodes(s, n, nf);
  if (rc) return rc;
  // edges of receiver gi = its neighbour list (exact neighbours, built by k_nbr_list)
  if (nf > 0) cudaMemcpyAsync(s->row_ptr, w.nbr_cnt, nf * 4, cudaMemcpyDeviceToDevice, cs);
  cudaMemsetAsync(s->row_ptr + nf, 0, 4, cs);
  launch_scan_exclusive_chunked(s->row_ptr, nf + 1, s->scan_tmp, cs);
  uint32_t E = 0;
  cudaMemcpyAsync(&E, s->row_ptr + nf, 4, cudaMemcpyDeviceToHost, cs);
  if (cudaStreamSynchronize(cs) != cudaSuccess) return sfail(s, WBSPH_E_CUDA, "graph build");
  s->E = E;
  rc = ensure_edges(s, E);
  if (rc) return rc;
  if (nf > 0)
    k_sg_fill<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, nf, s->row_ptr, s->pack,
                                                         (float)(1.0 / p.h), 1.f / s->edge_std[0],
                                                         1.f / s->edge_std[1], s->recv, s->send, s->efeat);
  return WBSPH_OK;
}

// encoder, layers, decoder; with `train` the message sums of every layer are kept
// to_rates: the decoder writes the stage rates (DU/Dt, Dphi/Dt, zero
// shifting) into the work arrays instead of the normalised outputs
int forward(wbsph_surrogate s, const Params& p, const Work& w, int64_t n, int64_t nf, bool train, cudaStream_t cs,
            bool to_rates = false) {
  const int L = s->layers;
  {  // node encoder (rows of 8 inputs)
    MlpArgs a = block_args(s, 0);
    a.rows = n; a.in = s->nfeat; a.out_bf = s->hs[0];
    const cudaError_t e = launch_fwd<MODE_DIRECT, 16, 64>(a, n, cs);
    if (e != cudaSuccess) return sfail(s, WBSPH_E_CUDA, cudaGetErrorString(e));
  }
  for (int l = 0; l < L; ++l) {
    bf16* m_out = train ? s->ms[l] : nullptr;
    if (m_out) cudaMemsetAsync(m_out, 0, (size_t)n * HID * 2, cs);  // rows of wall particles stay zero
    const cudaError_t e = launch_message(s, p, w, nf, n - nf, l, s->hs[l], s->hs[l + 1], m_out, cs);
    if (e != cudaSuccess) return sfail(s, WBSPH_E_CUDA, cudaGetErrorString(e));
  }
  {  // decoder over fluid rows
    MlpArgs a = block_args(s, 1 + 2 * L);
    a.rows = nf; a.in = s->hs[L]; a.list = w.fluid_list; a.out_f = s->out;
    if (to_rates) {
      a.r_dudt = w.dudt; a.r_dphidt = w.dphidt; a.r_shift = w.dushift;
      a.r_mean = s->norm + 16; a.r_std = s->norm + 20; a.r_n = n;
    }
    const cudaError_t e = launch_fwd<MODE_LIST, 64, 16>(a, nf, cs);
    if (e != cudaSuccess) return sfail(s, WBSPH_E_CUDA, cudaGetErrorString(e));
  }
  return WBSPH_OK;
}

void backward(wbsph_surrogate s, const Params& p, const Work& w, int64_t n, int64_t nf, cudaStream_t cs) {
  const int64_t E = s->E;
  const int L = s->layers;
  cudaMemsetAsync(s->g, 0, (size_t)s->np * 4, cs);
  cudaMemsetAsync(s->dh, 0, (size_t)n * HID * 4, cs);
  {  // decoder: dh_L[fluid] = dX
    MlpArgs a = block_args(s, 1 + 2 * L);
    a.rows = nf; a.in = s->hs[L]; a.list = w.fluid_list; a.dout = s->dout; a.dh = s->dh;
    launch_bwd<MODE_LIST, 64, 16>(a, nf, cs);
  }
  for (int l = L - 1; l >= 0; --l) {
    MlpArgs b = block_args(s, 2 + 2 * l);  // node MLP: dh_l = dh_{l+1} + dX[:64], dm = dX[64:]
    b.rows = n; b.h = s->hs[l]; b.agg = s->ms[l]; b.dout = s->dh; b.din_row = s->dh; b.dagg = s->dagg;
    launch_bwd<MODE_NODE, 128, 64>(b, n, cs);
    if (nf > 0)
      k_sg_aggregate_bwd<<<(unsigned)div_up(nf, 4), 128, 0, cs>>>(w.fluid_list, nf, s->row_ptr, s->dagg, s->de);
    MlpArgs a = block_args(s, 1 + 2 * l);  // edge MLP on [g, h_i, h_j[:32]]: dh += scatter of dX[16:]
    a.rows = E; a.e = s->efeat; a.h = s->hs[l]; a.recv = s->recv; a.send = s->send; a.kg = 2 * p.dim + 2;
    a.dout = s->de; a.dh = s->dh;
    launch_bwd<MODE_EDGE, EDGE_KP, 64>(a, E, cs);
  }
  {  // node encoder: weight gradients only
    MlpArgs b = block_args(s, 0);
    b.rows = n; b.in = s->nfeat; b.dout = s->dh;
    launch_bwd<MODE_DIRECT, 16, 64>(b, n, cs);
  }
}

}  // namespace

// Called by the engine for a surrogate stage: node inputs, forward pass,
// de-normalised rates into the stage rate arrays (or, in the frozen-rates
// control mode, the rates kept from the last plain stage).
namespace wbsph {
int surrogate_stage_rates(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n,
                          int64_t nf, cudaStream_t cs) {
  if (s->mode == WBSPH_SURROGATE_FROZEN) {
    if (!s->frozen) return sfail(s, WBSPH_E_STATE, "frozen-rates mode has no stored rates");
    if (nf > 0)
      k_frozen_rates<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, st.oid, n, nf, s->frozen, s->cap_frozen);
    return WBSPH_OK;
  }
  launch_nbr_list(p, st, w, n, nf, cs, true);
  int rc = ensure_nodes(s, n, nf);
  if (rc) return rc;
  node_inputs(s, p, st, n, cs);
  return forward(s, p, w, n, nf, false, cs, true);
}

int surrogate_mode(wbsph_surrogate s) { return s->mode; }

// Kernel launches of one surrogate stage (surrogate_stage_rates).
int surrogate_stage_launches(wbsph_surrogate s, int64_t nf) {
  if (nf == 0) return 0;
  if (s->mode == WBSPH_SURROGATE_FROZEN) return 1;
  return 1 + 1 + 1 + s->layers + 1;  // lists, node inputs, encoder, layers, decoder (writes the rates)
}

// The rates of a plain stage of a rollout (fluid particles): kept by the
// frozen-rates control; nothing in network mode.
int surrogate_plain_rates(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n, int64_t nf,
                          int64_t n_ids, cudaStream_t cs) {
  if (s->mode != WBSPH_SURROGATE_FROZEN || nf == 0) return WBSPH_OK;
  if (n_ids > s->cap_frozen) {
    dfree(s->frozen);
    s->frozen = nullptr;
    s->cap_frozen = 0;
    if (!dalloc(&s->frozen, (size_t)(p.dim + 1) * n_ids)) return sfail(s, WBSPH_E_NOMEM, "frozen rates");
    s->cap_frozen = n_ids;
  }
  k_frozen_store<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, st.oid, n, nf, s->frozen, s->cap_frozen);
  return WBSPH_OK;
}

// Loss of the surrogate against the rates currently in the work arrays
// (the plain pass of the same state); with `train`, backward and Adam.
int surrogate_loss(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n, int64_t nf,
                   cudaStream_t cs, int train, float lr, double* loss_out, const float* dout_override,
                   float* grad_out) {
  if (s->mode != WBSPH_SURROGATE_NETWORK) return sfail(s, WBSPH_E_STATE, "loss needs the network mode");
  launch_nbr_list(p, st, w, n, nf, cs, true);
  int rc = ensure_nodes(s, n, nf);
  if (rc) return rc;
  node_inputs(s, p, st, n, cs);
  if ((rc = build_graph(s, p, w, n, nf, cs))) return rc;
  if ((rc = forward(s, p, w, n, nf, true, cs))) return rc;
  cudaMemsetAsync(s->loss, 0, 8, cs);
  if (nf > 0)
    k_sg_loss<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, n, nf, s->out, s->norm + 16, s->norm + 20,
                                                          s->dout, s->loss);
  if (dout_override)
    cudaMemcpyAsync(s->dout, dout_override, (size_t)nf * (p.dim + 1) * 4, cudaMemcpyHostToDevice, cs);
  if (train || grad_out) backward(s, p, w, n, nf, cs);
  if (grad_out) cudaMemcpyAsync(grad_out, s->g, (size_t)s->np * 4, cudaMemcpyDeviceToHost, cs);
  if (train) {
    s->adam_t += 1;
    const wbsph_surrogate_config& c = s->cfg;
    float c1 = 1.f - powf(c.beta1, (float)s->adam_t), c2 = 1.f - powf(c.beta2, (float)s->adam_t);
    k_adam<<<(unsigned)div_up(s->np, 256), 256, 0, cs>>>(s->np, s->p, s->g, s->m, s->v, lr, c.beta1, c.beta2,
                                                         c.eps, c1, c2, s->pb);
  }
  double l = 0.0;
  cudaMemcpyAsync(&l, s->loss, 8, cudaMemcpyDeviceToHost, cs);
  cudaError_t e = cudaStreamSynchronize(cs);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return sfail(s, WBSPH_E_CUDA, cudaGetErrorString(e));
  if (loss_out) *loss_out = l;
  return WBSPH_OK;
}

int64_t surrogate_edges(wbsph_surrogate s) { return s->E; }

void launch_wait_probe(unsigned* status, uint32_t limit, cudaStream_t st) {
  k_wait_probe<<<1, 64, 0, st>>>(status, limit);
}
const float* surrogate_out(wbsph_surrogate s) { return s->out; }
const uint32_t* surrogate_recv(wbsph_surrogate s) { return s->recv; }
const uint32_t* surrogate_send(wbsph_surrogate s) { return s->send; }
const bf16* surrogate_efeat(wbsph_surrogate s) { return s->efeat; }
const bf16* surrogate_nfeat(wbsph_surrogate s) { return s->nfeat; }
}  // namespace wbsph

// ---------------------------------------------------------------------------
// C-ABI: create / parameters / normalisation / destroy
// ---------------------------------------------------------------------------
extern "C" int wbsph_surrogate_config_default(wbsph_surrogate_config* c, int dim) {
  if (!c || (dim != 2 && dim != 3)) return WBSPH_E_INVAL;
  memset(c, 0, sizeof *c);
  c->dim = dim;
  c->hidden = HID;
  c->layers = 3;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
  c->device = 0;
  return WBSPH_OK;
}

extern "C" int wbsph_surrogate_create(const wbsph_surrogate_config* c, wbsph_surrogate* out) {
  if (!c || !out) return WBSPH_E_INVAL;
  *out = nullptr;
  if (c->dim != 2 && c->dim != 3) return WBSPH_E_INVAL;
  if (c->hidden != HID || c->layers < 1 || c->layers > 8) return WBSPH_E_INVAL;
  if (cudaSetDevice(c->device) != cudaSuccess) { cudaGetLastError(); return WBSPH_E_CUDA; }
  wbsph_surrogate s = new wbsph_surrogate_s();
  s->cfg = *c;
  s->dim = c->dim;
  s->layers = c->layers;
  build_blocks(s);
  bool ok = dalloc(&s->p, s->np) && dalloc(&s->g, s->np) && dalloc(&s->m, s->np) && dalloc(&s->v, s->np) &&
            dalloc(&s->pb, s->np) && dalloc(&s->norm, 32) && dalloc(&s->loss, 1) && dalloc(&s->tile_ctr, 1);
  if (!ok) {
    wbsph_surrogate_destroy(s);
    return WBSPH_E_NOMEM;
  }
  cudaMemset(s->p, 0, s->np * 4);
  cudaMemset(s->m, 0, s->np * 4);
  cudaMemset(s->v, 0, s->np * 4);
  cudaMemset(s->pb, 0, s->np * 2);
  std::vector<float> nrm(32, 0.f);
  for (int k = 8; k < 16; ++k) nrm[k] = 1.f;
  for (int k = 20; k < 24; ++k) nrm[k] = 1.f;
  cudaMemcpy(s->norm, nrm.data(), 32 * 4, cudaMemcpyHostToDevice);
  *out = s;
  return WBSPH_OK;
}

extern "C" void wbsph_surrogate_destroy(wbsph_surrogate s) {
  if (!s) return;
  cudaSetDevice(s->cfg.device);
  cudaDeviceSynchronize();
  free_graph(s);
  dfree(s->p); dfree(s->g); dfree(s->m); dfree(s->v); dfree(s->pb); dfree(s->norm); dfree(s->loss);
  dfree(s->frozen);
  dfree(s->tile_ctr);
  delete s;
}

extern "C" int64_t wbsph_surrogate_num_params(wbsph_surrogate s) { return s ? s->np : WBSPH_E_INVAL; }

extern "C" int wbsph_surrogate_set_params(wbsph_surrogate s, const float* params) {
  if (!s || !params) return WBSPH_E_INVAL;
  cudaSetDevice(s->cfg.device);
  if (cudaMemcpy(s->p, params, s->np * 4, cudaMemcpyHostToDevice) != cudaSuccess) return WBSPH_E_CUDA;
  cudaMemset(s->m, 0, s->np * 4);
  cudaMemset(s->v, 0, s->np * 4);
  s->adam_t = 0;
  k_to_bf16<<<(unsigned)div_up(s->np, 256), 256>>>(s->np, s->p, s->pb);
  return cudaDeviceSynchronize() == cudaSuccess ? WBSPH_OK : WBSPH_E_CUDA;
}

extern "C" int wbsph_surrogate_get_params(wbsph_surrogate s, float* params) {
  if (!s || !params) return WBSPH_E_INVAL;
  cudaSetDevice(s->cfg.device);
  cudaDeviceSynchronize();
  return cudaMemcpy(params, s->p, s->np * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? WBSPH_OK : WBSPH_E_CUDA;
}

extern "C" int wbsph_surrogate_set_normalization(wbsph_surrogate s, const float* node_mean,
                                                 const float* node_std, const float* edge_std,
                                                 const float* out_mean, const float* out_std) {
  if (!s || !node_mean || !node_std || !edge_std || !out_mean || !out_std) return WBSPH_E_INVAL;
  std::vector<float> nrm(32, 0.f);
  int fn = s->dim + 2, fo = s->dim + 1;
  for (int k = 0; k < 8; ++k) nrm[8 + k] = 1.f;
  for (int k = 0; k < fn; ++k) {
    if (!(node_std[k] > 0)) return sfail(s, WBSPH_E_INVAL, "node std must be positive");
    nrm[k] = node_mean[k];
    nrm[8 + k] = node_std[k];
  }
  for (int k = 0; k < 4; ++k) nrm[20 + k] = 1.f;
  for (int k = 0; k < fo; ++k) {
    if (!(out_std[k] > 0)) return sfail(s, WBSPH_E_INVAL, "output std must be positive");
    nrm[16 + k] = out_mean[k];
    nrm[20 + k] = out_std[k];
  }
  for (int k = 0; k < 2; ++k) {
    if (!(edge_std[k] > 0)) return sfail(s, WBSPH_E_INVAL, "edge scales must be positive");
    nrm[24 + k] = edge_std[k];
    s->edge_std[k] = edge_std[k];
  }
  cudaSetDevice(s->cfg.device);
  return cudaMemcpy(s->norm, nrm.data(), 32 * 4, cudaMemcpyHostToDevice) == cudaSuccess ? WBSPH_OK : WBSPH_E_CUDA;
}

extern "C" int wbsph_surrogate_set_mode(wbsph_surrogate s, int mode) {
  if (!s) return WBSPH_E_INVAL;
  if (mode != WBSPH_SURROGATE_NETWORK && mode != WBSPH_SURROGATE_FROZEN)
    return sfail(s, WBSPH_E_INVAL, "unknown surrogate mode");
  s->mode = mode;
  return WBSPH_OK;
}

extern "C" const char* wbsph_surrogate_last_error(wbsph_surrogate s) { return s ? s->err.c_str() : "null"; }

// relative L2 error of DU/Dt: sums[0] += |a - a_ref|^2, sums[1] += |a|^2 over fluid
namespace {
__global__ void k_rel_err(int dim, Work w, int64_t n, int64_t nf, const double* a_ref, double* sums) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e2 = 0.0, r2 = 0.0;
  if (gi < nf) {
    uint32_t i = w.fluid_list[gi];
    for (int d = 0; d < dim; ++d) {
      double a = w.dudt[d * n + i], b = a_ref[d * n + i];
      e2 += (b - a) * (b - a);
      r2 += a * a;
    }
  }
  for (int off = 16; off; off >>= 1) {
    e2 += __shfl_xor_sync(0xffffffffu, e2, off);
    r2 += __shfl_xor_sync(0xffffffffu, r2, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], e2);
    atomicAdd(&sums[1], r2);
  }
}
}  // namespace

namespace wbsph {
void launch_rel_err(const Params& p, const Work& w, int64_t n, int64_t nf, const double* a_ref_copy,
                    double* sums, cudaStream_t st) {
  cudaMemsetAsync(sums, 0, 16, st);
  if (nf > 0) k_rel_err<<<(unsigned)div_up(nf, 128), 128, 0, st>>>(p.dim, w, n, nf, a_ref_copy, sums);
}
}  // namespace wbsph
