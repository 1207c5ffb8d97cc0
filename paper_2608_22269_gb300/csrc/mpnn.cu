// mpnn.cu -- BF16 message-passing surrogate of the pair pass: graph over the
// same neighbour lists, fused two-layer MLP kernels on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation) for inference and
// training, segment sums, loss, Adam, and the surrogate stage rates.
//
// Network (the paper has no learned part): node input f_i = normalised
// (U_i, rho_i/rho0 - 1, phi_i) plus a dummy flag; edge input
// ((x_j - x_i)/h, |x_j - x_i|/h, (U_j - U_i)/s_U, (phi_j - phi_i)/s_phi) for
// every fluid receiver i and every particle j within 2h (s = node scales); MLP(x) = W2 silu(W1 x + b1) + b2; node and edge encoders,
// three layers of e <- e + MLP_e([e, h_i, h_j]), a_i = sum_j e_ij,
// h <- h + MLP_n([h, a]), and a decoder to normalised (DU/Dt, Dphi/Dt).
// Flat parameter layout: blocks node encoder, edge encoder, (edge MLP,
// node MLP) per layer, decoder; each block W1 [in][64], b1, W2 [64][out], b2.
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

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
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
  const bf16* e;             // EDGE: [E][64]
  const bf16* h;             // EDGE, NODE: [n][64]
  const uint32_t* recv;      // EDGE
  const uint32_t* send;      // EDGE
  const bf16* agg;           // NODE: [n][64]
  int kin, nout;             // true widths
  const bf16* w1; const float* b1; const bf16* w2; const float* b2;  // block parameters
  // forward outputs
  bf16* out_bf;              // [rows][64] (+ residual for EDGE/NODE)
  float* out_f;              // [rows][nout] (decoder)
  // backward
  const float* dout;         // [rows][nout] incoming gradient (EDGE/NODE/DIRECT: [rows][64])
  float* din_row;            // EDGE: de_in, NODE: dh_in ([rows][64], = dout + dX[0:64])
  float* dh;                 // EDGE: atomics into [n][64]; LIST: writes dh[list[row]]
  float* dagg;               // NODE: [rows][64]
  float* gw1; float* gb1; float* gw2; float* gb2;  // FP32 parameter gradients
};

__device__ __forceinline__ int64_t arg_rows(const MlpArgs& a) {
  return a.rows_dev ? (int64_t)*a.rows_dev : a.rows;
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
    if (k < HID) return *reinterpret_cast<const uint32_t*>(a.e + row * HID + k);
    if (k < 2 * HID) return *reinterpret_cast<const uint32_t*>(a.h + (int64_t)a.recv[row] * HID + k - HID);
    return *reinterpret_cast<const uint32_t*>(a.h + (int64_t)a.send[row] * HID + k - 2 * HID);
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
  if (MODE == MODE_EDGE) {
    if (c8 < 8) return a.e + row * HID + c8 * 8;
    if (c8 < 16) return a.h + (int64_t)I[r] * HID + (c8 - 8) * 8;
    return a.h + (int64_t)I[TILE + r] * HID + (c8 - 16) * 8;
  }
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
    if (a.out_f) {  // decoder: FP32 outputs, few columns
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
          if (MODE == MODE_EDGE || MODE == MODE_NODE) {
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
// Node projections for the split edge MLP. The first layer of the edge MLP
// acts on [e_ij, h_i, h_j], so z1 = e_ij W1e + h_i W1r + h_j W1s + b1 with
// W1 = [W1e; W1r; W1s] (64 rows each): the two node terms are computed once
// per node here, P_i = [h_i W1r + b1 | h_i W1s] (BF16, FP32 accumulation), and
// the edge kernel gathers them instead of h, leaving a 64-wide GEMM per edge.
// ---------------------------------------------------------------------------
constexpr int PJ_LD = HID + 8, PJ_LDO = 2 * HID + 8;

__global__ void __launch_bounds__(MLP_THREADS) k_node_proj(const bf16* __restrict__ h, int64_t n,
                                                           const bf16* __restrict__ w1, const float* __restrict__ b1,
                                                           bf16* __restrict__ P) {
  __shared__ __align__(16) bf16 Bt[2 * HID * PJ_LD];  // Bt[o][k] = W1[64 + k][o] | W1[128 + k][o - 64]
  __shared__ __align__(16) bf16 At[TILE * PJ_LD];
  __shared__ __align__(16) bf16 Ot[TILE * PJ_LDO];
  for (int idx = threadIdx.x; idx < 2 * HID * HID; idx += MLP_THREADS) {
    int o = idx / HID, k = idx % HID;
    Bt[o * PJ_LD + k] = w1[(int64_t)(HID + (o >= HID ? HID : 0) + k) * HID + (o % HID)];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int m0 = warp * 16;
  for (int64_t tile = blockIdx.x; tile * TILE < n; tile += gridDim.x) {
    const int64_t row0 = tile * TILE;
    __syncthreads();  // Bt staged / At and Ot free
    for (int idx = threadIdx.x; idx < TILE * (HID / 8); idx += MLP_THREADS) {
      int r = idx / (HID / 8), c8 = idx % (HID / 8);
      int64_t row = row0 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < n) v = *reinterpret_cast<const uint4*>(h + row * HID + c8 * 8);
      *reinterpret_cast<uint4*>(At + r * PJ_LD + c8 * 8) = v;
    }
    __syncthreads();
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < HID / 16; ++kt) {
      uint32_t af[4];
      ldsm_a(af, At, PJ_LD, m0, kt * 16);
#pragma unroll
      for (int nt = 0; nt < 16; nt += 2) {
        uint32_t bq[4];
        ldsm_b2(bq, Bt, PJ_LD, kt * 16, nt * 8);
        mma16816(acc[nt], af, bq);
        mma16816(acc[nt + 1], af, bq + 2);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      int c = nt * 8 + 2 * t;
      // the first-layer bias rides on the receiver half
      const float c0 = nt < 8 ? __ldg(b1 + c) : 0.f, c1 = nt < 8 ? __ldg(b1 + c + 1) : 0.f;
      *reinterpret_cast<__nv_bfloat162*>(Ot + (m0 + g) * PJ_LDO + c) =
          __floats2bfloat162_rn(acc[nt][0] + c0, acc[nt][1] + c1);
      *reinterpret_cast<__nv_bfloat162*>(Ot + (m0 + g + 8) * PJ_LDO + c) =
          __floats2bfloat162_rn(acc[nt][2] + c0, acc[nt][3] + c1);
    }
    __syncwarp();
    // the warp's 16 rows of 256 bytes, 16-byte chunks
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      int idx = q * 32 + lane, r = m0 + (idx >> 4), c16 = idx & 15;
      int64_t row = row0 + r;
      if (row < n)
        *reinterpret_cast<uint4*>(P + row * 2 * HID + c16 * 8) = *reinterpret_cast<const uint4*>(Ot + r * PJ_LDO + c16 * 8);
    }
  }
}

// ---------------------------------------------------------------------------
// Edge MLP of a message-passing layer on the 5th-generation tensor cores
// (tcgen05). Per tile of 128 edges:
//   z1 = e W1e + P_recv + P_send + b1    (64 x 64 GEMM, node terms from k_node_proj)
//   e' = e + silu(z1) W2 + b2            (64 x 64 GEMM)
// Operands sit in shared memory in the K-major 128-byte-swizzled layout the
// tensor core reads through matrix descriptors (row r of 64 BF16 = 128 B at
// r * 128, 16-byte chunk c stored at chunk c ^ (r % 8); 8-row groups 1024 B
// apart); the FP32 accumulators live in tensor memory (TMEM, 64 columns per
// tile in flight, lane = tile row) and are read back by the warp that owns
// those 32 lanes. One thread issues the MMAs and their commit to an
// mbarrier; every wait on an mbarrier is bounded and a timeout is reported
// through the error word.
// ---------------------------------------------------------------------------
constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_TILE_BYTES = TC_ROWS * 128;        // 128 rows x 64 BF16
#ifndef WBSPH_TC_SLOTS
#define WBSPH_TC_SLOTS 2
#endif
// tiles in flight per CTA (operand slots of 2 x 16 KB each)
constexpr int TC_SLOTS = WBSPH_TC_SLOTS;
static_assert(TC_SLOTS >= 2 && TC_SLOTS <= 8, "slot count");
constexpr size_t TC_SMEM_BYTES =
    1024 + 2 * TC_SLOTS * TC_TILE_BYTES + 3 * 8192 + 2 * 64 * 4 + 128;  // slots, W, biases, barriers
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

// all 64 FP32 columns of this thread's TMEM lane in one load and one wait
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float v[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

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

// TMA: 2D tile load into shared memory, completing on an mbarrier with a
// byte count; 2D tile store from shared memory in a bulk group.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void tma_store_read_wait() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Check of the bounded wait itself: one thread waits on an mbarrier that
// nothing arrives on; when the limit runs out it reports a timeout through the
// status word, as the MLP kernels do, and the kernel ends normally.
__global__ void k_wait_probe(unsigned* status, uint32_t limit) {
  __shared__ uint64_t bar;
  const uint32_t mb = smem_u32(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
  if (!mbar_wait(mb, 0u, limit)) atomicOr(status, (unsigned)kStatTimeout);
}

// silu(z) = z sigmoid(z) = z (1 + tanh(z / 2)) / 2 with the hardware tanh
// approximation (one special-function op instead of an exponential and a
// reciprocal; absolute error ~1e-3 |z|, below the BF16 rounding of the result)
__device__ __forceinline__ float silu_tanh(float z) {
  float h = 0.5f * z, th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(h));
  return fmaf(h, th, h);
}

// Modes. TC_EDGE: the edge MLP above. TC_ENC: an encoder MLP on rows of 8
// BF16 input features (K = 16, zero padded): z1 = f W1 + b1,
// out = silu(z1) W2 + b2, no projections, no residual. TC_NODE: the node MLP
// of a layer, h' = h + silu([h, a] W1 + b1) W2 + b2 (K = 128: the h tile and
// the aggregate tile are the two 64-wide K blocks of the first GEMM).
//
// Pipeline over the CTA's tiles: TC_SLOTS operand slots (tile i in slot
// i % TC_SLOTS), each with its own e tile, sender-projection tile (which
// then holds silu(z1)) and TMA mbarrier, and two TMEM accumulators of 64
// columns with their MMA mbarriers (tile i in accumulator i % 2). Iteration
// i runs: epilogue 1 of tile i, MMA2 of tile i issued, MMA1 of tile i+1
// issued (its loads were issued TC_SLOTS - 1 iterations earlier), epilogue
// 2 and store of tile i, loads of tile i + TC_SLOTS into tile i's slot. So
// each tile's GEMMs run while the other tile's epilogues do, and the loads
// of TC_SLOTS - 1 tiles are in flight.
// (The explicit minimum of one block lets the compiler keep the edge mode's
// receiver projections and accumulator values in registers without spills.)
enum { TC_EDGE = 0, TC_ENC = 1, TC_NODE = 2 };

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1) k_edge_mlp_tc(const bf16* __restrict__ e_in, bf16* __restrict__ e_out,
                                                           int64_t E, const uint32_t* __restrict__ recv,
                                                           const uint32_t* __restrict__ send,
                                                           const bf16* __restrict__ P, const bf16* __restrict__ w1,
                                                           int kin, const float* __restrict__ b1g,
                                                           const bf16* __restrict__ w2,
                                                           const float* __restrict__ b2g, unsigned* err,
                                                           const __grid_constant__ CUtensorMap tm_a,
                                                           const __grid_constant__ CUtensorMap tm_b,
                                                           const __grid_constant__ CUtensorMap tm_out) {
  // tm_a: rows of e_in (edge, node: h) and tm_b: rows of the aggregates (node),
  // tm_out: rows of e_out; [rows][64] BF16, 128-row boxes, 128-byte swizzle.
  // The encoder mode (8-feature rows) gathers and stores with plain loads.
  constexpr bool ENC = MODE == TC_ENC, NODE = MODE == TC_NODE, EDGE = MODE == TC_EDGE;
  extern __shared__ unsigned char tc_raw[];
  unsigned char* base = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);  // 1024-byte aligned
  // slot s: e (or h) tile at s * 32 KB; sender projections (or aggregates),
  // then silu(z1), at s * 32 KB + 16 KB
  unsigned char* B1 = base + 2 * TC_SLOTS * TC_TILE_BYTES;  // W1[0:64]^T [n][k]
  unsigned char* B2 = B1 + 8192;                 // W2^T [n][k]
  unsigned char* B1b = B2 + 8192;                // W1[64:128]^T [n][k] (node MLP)
  float* b2 = reinterpret_cast<float*>(B1b + 8192);
  float* b1 = b2 + 64;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b1 + 64);  // MMA completion, one per accumulator
  uint64_t* lbar = mbar + 2;                               // TMA tile arrival, one per slot
  uint32_t* tslot = reinterpret_cast<uint32_t*>(lbar + TC_SLOTS);
  auto Et = [&](int sl) { return base + sl * 2 * TC_TILE_BYTES; };
  auto Pt = [&](int sl) { return base + sl * 2 * TC_TILE_BYTES + TC_TILE_BYTES; };
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

  // weights (K-major swizzled), biases, barriers, tensor memory
  for (int idx = t; idx < 64 * 64; idx += TC_THREADS) {
    int n = idx >> 6, k = idx & 63;
    uint32_t off = sw128(n, k >> 3) + (k & 7) * 2;
    *reinterpret_cast<bf16*>(B1 + off) = k < kin ? w1[k * HID + n] : __float2bfloat16(0.f);
    *reinterpret_cast<bf16*>(B2 + off) = w2[k * HID + n];
    if (NODE) *reinterpret_cast<bf16*>(B1b + off) = w1[(HID + k) * HID + n];
  }
  if (t < 64) {
    b2[t] = b2g[t];
    b1[t] = EDGE ? 0.f : b1g[t];  // the edge MLP's b1 rides on the receiver projections
  }
  if (t == 0) {
    for (int k = 0; k < 2 + TC_SLOTS; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar + k)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;\n" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;  // slot s accumulator: columns 64 s .. 64 s + 63
  const uint32_t t_lane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint64_t dB1 = tc_desc(smem_u32(B1)), dB2 = tc_desc(smem_u32(B2)), dB1b = tc_desc(smem_u32(B1b));
  const int64_t ntiles = div_up(E, TC_ROWS);
  const int64_t stride = gridDim.x;

  // gathers of tile `tile` into slot `sl`: e rows (or features) and sender
  // projections of the warp's 32 rows. Edge rows: lane l moves 16-byte chunk
  // l % 8 of row 4 k + l / 8, so each instruction covers 4 whole rows
  // (512 contiguous bytes of e); `sd` is the sender of this thread's row.
  auto issue = [&](int64_t tile, int sl, uint32_t sd) {
    unsigned char* Ae = Et(sl);
    if (ENC) {  // row t: 8 features, then zeros up to K = 16
      const int64_t row = tile * TC_ROWS + t;
      const bool valid = tile < ntiles && row < E;
      cp_async16(Ae + sw128(t, 0), e_in + (valid ? row : 0) * FEAT, valid);
      cp_async16(Ae + sw128(t, 1), e_in, false);
    } else {
      // e (or h) tile, and the aggregate tile of a node MLP, by TMA (rows past
      // the end read as zeros); the store of the tile held here before must
      // have finished reading it
      if (t == 0 && tile < ntiles) {
        tma_store_read_wait();
        mbar_expect_tx(smem_u32(lbar + sl), NODE ? 2 * TC_TILE_BYTES : TC_TILE_BYTES);
        tma_load_2d(smem_u32(Ae), &tm_a, 0, (int)(tile * TC_ROWS), smem_u32(lbar + sl));
        if (NODE) tma_load_2d(smem_u32(Pt(sl)), &tm_b, 0, (int)(tile * TC_ROWS), smem_u32(lbar + sl));
      }
      if (EDGE) {  // sender projections: lane l moves chunk l % 8 of row 4 k + l / 8
        const int c = lane & 7;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int rl = k * 4 + (lane >> 3), r = warp * 32 + rl;
          const uint32_t sdr = __shfl_sync(0xffffffffu, sd, rl);
          const int64_t row = tile * TC_ROWS + r;
          const bool valid = tile < ntiles && row < E;
          cp_async16(Pt(sl) + sw128(r, c), P + (int64_t)(valid ? sdr : 0u) * 2 * HID + HID + c * 8, valid);
        }
      }
    }
    cp_async_commit();
  };
  auto index_of = [&](const uint32_t* a, int64_t tile) -> uint32_t {
    const int64_t row = tile * TC_ROWS + t;
    return (EDGE && tile < ntiles && row < E) ? __ldg(a + row) : 0u;
  };
  // receiver projections (+ b1) of this thread's row, in registers, one tile ahead
  uint4 pr[8];
  auto load_pr = [&](uint32_t rv) {
    if (EDGE) {
      const uint4* prg = reinterpret_cast<const uint4*>(P + (int64_t)rv * 2 * HID);
#pragma unroll
      for (int c = 0; c < 8; ++c) pr[c] = __ldg(prg + c);
    }
  };
  // accumulator ac (TMEM columns 64 ac .. 64 ac + 63) of the tile in slot sl
  auto mma1 = [&](int sl, int ac) {  // z1 = e W1e (or f W1, or [h, a] W1)
    tc_fence_after();
    const uint64_t dA = tc_desc(smem_u32(Et(sl)));
#pragma unroll
    for (int k = 0; k < (ENC ? 1 : 4); ++k) tc_mma(tmem + 64 * ac, dA + 2 * k, dB1 + 2 * k, k > 0);
    if (NODE) {  // second K block: the aggregates
      const uint64_t dA2 = tc_desc(smem_u32(Pt(sl)));
#pragma unroll
      for (int k = 0; k < 4; ++k) tc_mma(tmem + 64 * ac, dA2 + 2 * k, dB1b + 2 * k, 1u);
    }
    tc_commit(smem_u32(mbar + ac));
  };
  auto mma2 = [&](int sl, int ac) {  // z2 = silu(z1) W2, same columns
    tc_fence_after();
    const uint64_t dA = tc_desc(smem_u32(Pt(sl)));
#pragma unroll
    for (int k = 0; k < 4; ++k) tc_mma(tmem + 64 * ac, dA + 2 * k, dB2 + 2 * k, k > 0);
    tc_commit(smem_u32(mbar + ac));
  };
  // bit b: parity of mbarrier b's next phase (0, 1: MMA per accumulator;
  // 2 + s: TMA arrival of slot s)
  uint32_t phases = 0u;
  auto wait_slot = [&](int ac) -> bool {  // bounded; every thread gets the CTA's decision
    bool w_ok = mbar_wait(smem_u32(mbar + ac), (phases >> ac) & 1u);
    phases ^= 1u << ac;
    return __syncthreads_and(w_ok) != 0;
  };
  // this thread's gathers of slot sl are complete and the slot's TMA tiles
  // have arrived (bounded wait); followed by a CTA barrier. In the prologue
  // all TC_SLOTS slots are in flight, later TC_SLOTS - 1 of them.
  auto wait_loads = [&](int sl, bool prologue) -> bool {
    if (prologue) cp_async_wait<TC_SLOTS - 1>(); else cp_async_wait<TC_SLOTS - 2>();
    bool w_ok = true;
    if (!ENC) {
      w_ok = mbar_wait(smem_u32(lbar + sl), (phases >> (2 + sl)) & 1u);
      phases ^= 1u << (2 + sl);
    }
    fence_async_smem();  // gathered tiles are read by the tensor core
    tc_fence_before();
    return __syncthreads_and(w_ok) != 0;
  };

  int64_t tile = blockIdx.x;
  // prologue: gathers of the first TC_SLOTS tiles, MMA1 of the first
#pragma unroll
  for (int q = 0; q < TC_SLOTS; ++q) issue(tile + q * stride, q, index_of(send, tile + q * stride));
  load_pr(index_of(recv, tile));
  uint32_t rv_n1 = index_of(recv, tile + stride);                // receiver indices of the next tile
  uint32_t sd_nx = index_of(send, tile + TC_SLOTS * stride);     // senders of the next tile to gather
  bool ok = true;
  if (tile < ntiles) {
    ok = wait_loads(0, true);
    if (ok && t == 0) mma1(0, 0);
  }

  for (int it = 0; tile < ntiles; ++it, tile += stride) {
    const int ac = it & 1;              // accumulator of this tile
    const int sl = it % TC_SLOTS;       // operand slot of this tile
    const int sn = (it + 1) % TC_SLOTS; // and of the next one
    const int64_t row0 = tile * TC_ROWS;
    unsigned char* A = Et(sl);
    unsigned char* PS = Pt(sl);
    if (!wait_slot(ac)) { ok = false; break; }  // MMA1 of this tile
    tc_fence_after();
    // ---- silu(z1 + P_recv + P_send) (or + b1) -> PS, in place, BF16 swizzled ----
    {
      float va[64];
      tc_ld64(t_lane + 64 * ac, va);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float* v = va + 8 * c;
        uint4 o;
        uint32_t* o32 = reinterpret_cast<uint32_t*>(&o);
        if (!EDGE) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int col = c * 8 + 2 * j;
            __nv_bfloat162 a2 = __floats2bfloat162_rn(silu_tanh(v[2 * j] + b1[col]),
                                                      silu_tanh(v[2 * j + 1] + b1[col + 1]));
            o32[j] = *reinterpret_cast<uint32_t*>(&a2);
          }
        } else {
          uint4 ps = *reinterpret_cast<const uint4*>(PS + sw128(t, c));
          const __nv_bfloat162* r2 = reinterpret_cast<const __nv_bfloat162*>(&pr[c]);
          const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(&ps);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float2 fr = __bfloat1622float2(r2[j]), fs = __bfloat1622float2(s2[j]);
            __nv_bfloat162 a2 = __floats2bfloat162_rn(silu_tanh(v[2 * j] + fr.x + fs.x),
                                                      silu_tanh(v[2 * j + 1] + fr.y + fs.y));
            o32[j] = *reinterpret_cast<uint32_t*>(&a2);
          }
        }
        *reinterpret_cast<uint4*>(PS + sw128(t, c)) = o;
      }
    }
    fence_async_smem();  // silu(z1) is read by the tensor core
    tc_fence_before();
    __syncthreads();
    if (t == 0) mma2(sl, ac);
    load_pr(rv_n1);  // next tile's receiver projections
    rv_n1 = index_of(recv, tile + 2 * stride);
    // ---- MMA1 of the next tile (its gathers were issued TC_SLOTS - 1 iterations ago) ----
    if (tile + stride < ntiles) {
      if (!wait_loads(sn, false)) { ok = false; break; }
      if (t == 0) mma1(sn, ac ^ 1);
    }
    if (!wait_slot(ac)) { ok = false; break; }  // MMA2 of this tile
    tc_fence_after();
    // ---- e' = e + z2 + b2, in place into the e tile ----
    {
      float va[64];
      tc_ld64(t_lane + 64 * ac, va);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float* v = va + 8 * c;
        uint4 ev = make_uint4(0u, 0u, 0u, 0u);  // residual (none for an encoder)
        if (!ENC) ev = *reinterpret_cast<const uint4*>(A + sw128(t, c));
        const __nv_bfloat162* e2 = reinterpret_cast<const __nv_bfloat162*>(&ev);
        uint4 o;
        uint32_t* o32 = reinterpret_cast<uint32_t*>(&o);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = c * 8 + 2 * j;
          float2 fe = __bfloat1622float2(e2[j]);
          __nv_bfloat162 a2 = __floats2bfloat162_rn(v[2 * j] + b2[col] + fe.x,
                                                    v[2 * j + 1] + b2[col + 1] + fe.y);
          o32[j] = *reinterpret_cast<uint32_t*>(&a2);
        }
        *reinterpret_cast<uint4*>(A + sw128(t, c)) = o;
      }
    }
    if (ENC) {
      __syncwarp();
      // the warp's 32 output rows, 4 whole rows (512 B) per store instruction
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = warp * 32 + k * 4 + (lane >> 3), c = lane & 7;
        const int64_t row = row0 + r;
        if (row < E)
          *reinterpret_cast<uint4*>(e_out + row * HID + c * 8) = *reinterpret_cast<const uint4*>(A + sw128(r, c));
      }
      __syncwarp();
    } else {  // the whole tile by one TMA store (rows past the end are not written)
      fence_async_smem();
      __syncthreads();
      if (t == 0) tma_store_2d(&tm_out, 0, (int)row0, smem_u32(A));
    }
    // ---- gathers of the tile TC_SLOTS ahead into this slot (its e and silu(z1) tiles are free) ----
    issue(tile + TC_SLOTS * stride, sl, sd_nx);
    sd_nx = index_of(send, tile + (TC_SLOTS + 1) * stride);
  }
  cp_async_wait<0>();  // gathers issued for tiles past the end
  if (t == 0) tma_store_wait();
  if (!ok && t == 0) atomicOr(err, (unsigned)kStatTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;\n" ::"r"(tmem) : "memory");
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
    bf16 v = k < a.kin ? a.w1[k * HID + c] : zero;
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
          if (row >= rows || k >= a.kin) continue;
          float v = dx[q];
          if (MODE == MODE_LIST) {
            a.dh[(int64_t)a.list[row] * HID + k] = v;
          } else if (MODE == MODE_EDGE) {
            if (k < HID) a.din_row[row * HID + k] = a.dout[row * HID + k] + v;
            else if (k < 2 * HID) atomicAdd(&a.dh[(int64_t)a.recv[row] * HID + k - HID], v);
            else atomicAdd(&a.dh[(int64_t)a.send[row] * HID + k - 2 * HID], v);
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
  for (int idx = threadIdx.x; idx < a.kin * HID; idx += MLP_THREADS) atomicAdd(&a.gw1[idx], gW1[idx]);
  for (int idx = threadIdx.x; idx < HID * a.nout; idx += MLP_THREADS) {
    int c = idx / a.nout, o = idx % a.nout;
    atomicAdd(&a.gw2[idx], gW2[c * NP + o]);
  }
  for (int idx = threadIdx.x; idx < HID; idx += MLP_THREADS) atomicAdd(&a.gb1[idx], gB1[idx]);
  for (int idx = threadIdx.x; idx < a.nout; idx += MLP_THREADS) atomicAdd(&a.gb2[idx], gB2[idx]);
}

// ---------------------------------------------------------------------------
// Graph, features, aggregation, loss, optimiser
// ---------------------------------------------------------------------------
// FP32 value of a double by truncating its IEEE fields with integer
// instructions (magnitudes below 2^-126 give zero; no infinities arise
// here). Feature inputs are rounded to BF16 afterwards, so truncation is
// immaterial, and the FP64 pipe stays free.
__device__ __forceinline__ float d2f_fields(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7FFu;
  if (e <= 1023u - 127u) return 0.f;
  return __uint_as_float((hi & 0x80000000u) | ((e - (1023u - 127u)) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// Edges and edge features. A warp covers the receivers g0 .. g0 + 31 and
// the contiguous range of their edges; lane l takes edges l, l + 32, ... of
// that range, finds its receiver by a binary search over the lanes' row
// starts, and receives the receiver's data by shuffle: every store of
// recv, send and the 16-byte feature rows is coalesced.
__global__ void k_sg_fill(Params p, State s, Work w, int64_t n, int64_t nf, const uint32_t* row_ptr,
                          uint32_t* recv, uint32_t* send, bf16* efeat, const float* node_std) {
  const int lane = threadIdx.x & 31;
  const int64_t g0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x - lane;
  if (g0 >= nf) return;  // whole warps leave together
  const int64_t gl = g0 + lane;
  const uint32_t start = row_ptr[gl < nf ? gl : nf];  // row_ptr holds nf + 1 entries
  const uint32_t e_end = __shfl_sync(0xffffffffu, start, 31) +
                         (g0 + 31 < nf ? w.nbr_cnt[g0 + 31] : 0u);  // end of the last receiver's row
  const uint32_t e_beg = __shfl_sync(0xffffffffu, start, 0);
  const float inv_h = (float)(1.0 / p.h);
  float inv_su[3] = {0.f, 0.f, 0.f};
  for (int d = 0; d < p.dim; ++d) inv_su[d] = 1.f / node_std[d];
  const float inv_sphi = 1.f / node_std[p.dim + 1];
  // this lane's receiver: FP32 position, velocity and potential narrowed on
  // the IEEE fields (BF16 features need no FP64 arithmetic)
  uint32_t i_l = 0u;
  float4 x_l = make_float4(0.f, 0.f, 0.f, 0.f);
  float u_l[3] = {0.f, 0.f, 0.f}, phi_l = 0.f;
  if (gl < nf) {
    i_l = w.fluid_list[gl];
    x_l = w.xf[i_l];
    for (int d = 0; d < p.dim; ++d) u_l[d] = d2f_fields(s.u[d * n + i_l]);
    phi_l = d2f_fields(s.phi[i_l]);
  }
  for (uint32_t e0 = e_beg; e0 < e_end; e0 += 32) {
    const uint32_t e = e0 + (uint32_t)lane;
    // receiver lane r: the last lane whose row starts at or before e
    int r = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {
      const uint32_t st_c = __shfl_sync(0xffffffffu, start, r + step);
      if (r + step < 32 && g0 + r + step < nf && st_c <= e) r += step;
    }
    const uint32_t i = __shfl_sync(0xffffffffu, i_l, r);
    const float xi = __shfl_sync(0xffffffffu, x_l.x, r), yi = __shfl_sync(0xffffffffu, x_l.y, r),
                zi = __shfl_sync(0xffffffffu, x_l.z, r);
    float ui[3];
    for (int d = 0; d < 3; ++d) ui[d] = __shfl_sync(0xffffffffu, u_l[d], r);
    const float phii = __shfl_sync(0xffffffffu, phi_l, r);
    const uint32_t st_r = __shfl_sync(0xffffffffu, start, r);
    if (e >= e_end) continue;
    const uint32_t k = e - st_r;
    const uint32_t j = w.nbr[(int64_t)k * nf + g0 + r];  // every list entry is an exact neighbour
    const float4 xj = __ldg(&w.xf[j]);
    const float rv[3] = {xj.x - xi, xj.y - yi, xj.z - zi};
    recv[e] = i;
    send[e] = j;
    // features (r/h, |r|/h, dU/s_U, dphi/s_phi), zero padded to 8, one 16-byte store
    float f[FEAT] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float r2 = 0.f;
    for (int d = 0; d < p.dim; ++d) {
      f[d] = rv[d] * inv_h;
      r2 = fmaf(rv[d], rv[d], r2);
      f[p.dim + 1 + d] = (d2f_fields(s.u[d * n + j]) - ui[d]) * inv_su[d];
    }
    f[p.dim] = sqrtf(r2) * inv_h;
    f[2 * p.dim + 1] = (d2f_fields(s.phi[j]) - phii) * inv_sphi;
    uint4 v;
    v.x = pack2(__float2bfloat16(f[0]), __float2bfloat16(f[1]));
    v.y = pack2(__float2bfloat16(f[2]), __float2bfloat16(f[3]));
    v.z = pack2(__float2bfloat16(f[4]), __float2bfloat16(f[5]));
    v.w = pack2(__float2bfloat16(f[6]), __float2bfloat16(f[7]));
    *reinterpret_cast<uint4*>(efeat + (int64_t)e * FEAT) = v;
  }
}

// node features: (U, rho/rho0 - 1, phi) normalised by (mean, std), dummy flag
__global__ void k_sg_nodes(Params p, State s, int64_t n, const float* mean, const float* stdv, bf16* nf_out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v[FEAT] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = 0; d < p.dim; ++d) v[d] = (float)s.u[d * n + i];
  double rho = eos_density(p, s.phi[i]);
  v[p.dim] = (float)(rho / p.rho0 - 1.0);
  v[p.dim + 1] = (float)s.phi[i];
  for (int k = 0; k < p.dim + 2; ++k) v[k] = (v[k] - mean[k]) / stdv[k];
  v[p.dim + 2] = s.type[i] == kFluid ? 0.f : 1.f;
  for (int k = 0; k < FEAT; ++k) nf_out[i * FEAT + k] = __float2bfloat16(v[k]);
}

// a_i = sum of the receiver's edge states (fluid rows; other nodes keep zero)
__global__ void k_sg_aggregate(const uint32_t* fluid_list, int64_t nf, const uint32_t* row_ptr,
                               const bf16* e, bf16* agg) {
  int64_t gi = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (gi >= nf) return;
  uint32_t i = fluid_list[gi];
  float s0 = 0.f, s1 = 0.f;
  for (uint32_t k = row_ptr[gi]; k < row_ptr[gi + 1]; ++k) {
    __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162*>(e + (int64_t)k * HID)[lane];
    s0 += __bfloat162float(v.x);
    s1 += __bfloat162float(v.y);
  }
  reinterpret_cast<__nv_bfloat162*>(agg + (int64_t)i * HID)[lane] = __floats2bfloat162_rn(s0, s1);
}

// de_e += dagg_recv(e)
__global__ void k_sg_aggregate_bwd(const uint32_t* fluid_list, int64_t nf, const uint32_t* row_ptr,
                                   const float* dagg_rows, float* de) {
  int64_t gi = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (gi >= nf) return;
  uint32_t i = fluid_list[gi];
  float2 g = reinterpret_cast<const float2*>(dagg_rows + (int64_t)i * HID)[lane];
  for (uint32_t k = row_ptr[gi]; k < row_ptr[gi + 1]; ++k) {
    float2* p2 = reinterpret_cast<float2*>(de + (int64_t)k * HID) + lane;
    float2 v = *p2;
    v.x += g.x;
    v.y += g.y;
    *p2 = v;
  }
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

// de-normalised outputs -> stage rates (shifting velocity zero)
__global__ void k_sg_rates(int dim, Work w, int64_t n, int64_t nf, const float* out, const float* tmean,
                           const float* tstd) {
  int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gi >= nf) return;
  uint32_t i = w.fluid_list[gi];
  int no = dim + 1;
  for (int o = 0; o < dim; ++o) {
    w.dudt[o * n + i] = (double)out[gi * no + o] * tstd[o] + tmean[o];
    w.dushift[o * n + i] = 0.0;
  }
  w.dphidt[i] = (double)out[gi * no + dim] * tstd[dim] + tmean[dim];
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
  int dim = 2, layers = 3;
  std::vector<Block> blocks;
  int64_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16* pb = nullptr;
  float* norm = nullptr;  // node mean[8], node std[8], target mean[4], target std[4]
  int64_t adam_t = 0;
  // graph and activations, sized on demand
  int64_t cap_n = 0, cap_nf = 0, cap_e = 0;
  uint32_t *row_ptr = nullptr, *recv = nullptr, *send = nullptr, *scan_tmp = nullptr;
  bf16 *efeat = nullptr, *nfeat = nullptr, *proj = nullptr;
  std::vector<bf16*> hs, es, aggs;
  float *out = nullptr, *dout = nullptr, *dh = nullptr, *de = nullptr, *dagg = nullptr;
  double* loss = nullptr;
  int64_t E = 0;
  std::string err;
};

namespace {

int sfail(wbsph_surrogate s, int code, const char* msg) {
  if (s) s->err = msg;
  return code;
}

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
  add(2 * d + 2, HID);
  for (int l = 0; l < s->layers; ++l) {
    add(3 * HID, HID);
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

void free_graph(wbsph_surrogate s) {
  dfree(s->row_ptr); dfree(s->recv); dfree(s->send); dfree(s->efeat); dfree(s->nfeat);
  dfree(s->proj); dfree(s->scan_tmp);
  s->proj = nullptr;
  s->scan_tmp = nullptr;
  for (auto* q : s->hs) dfree(q);
  for (auto* q : s->es) dfree(q);
  for (auto* q : s->aggs) dfree(q);
  s->hs.clear(); s->es.clear(); s->aggs.clear();
  dfree(s->out); dfree(s->dout); dfree(s->dh); dfree(s->de); dfree(s->dagg);
  s->row_ptr = s->recv = s->send = nullptr;
  s->efeat = s->nfeat = nullptr;
  s->out = s->dout = s->dh = s->de = s->dagg = nullptr;
  s->cap_n = s->cap_nf = s->cap_e = 0;
}

int ensure_nodes(wbsph_surrogate s, int64_t n, int64_t nf) {
  if (n <= s->cap_n && nf <= s->cap_nf) return WBSPH_OK;
  free_graph(s);
  s->cap_n = n; s->cap_nf = nf;
  bool ok = dalloc(&s->row_ptr, nf + 1) && dalloc(&s->nfeat, n * FEAT) &&
            dalloc(&s->out, nf * 4) && dalloc(&s->dout, nf * 4) && dalloc(&s->dh, n * HID) &&
            dalloc(&s->dagg, n * HID) && dalloc(&s->proj, n * 2 * HID) &&
            dalloc(&s->scan_tmp, (size_t)scan_scratch_words(nf + 1));
  for (int l = 0; ok && l <= s->layers; ++l) {
    bf16* q = nullptr;
    ok = dalloc(&q, n * HID);
    s->hs.push_back(q);
    if (ok && l < s->layers) {
      ok = dalloc(&q, n * HID);
      s->aggs.push_back(q);
    }
  }
  return ok ? WBSPH_OK : sfail(s, WBSPH_E_NOMEM, "surrogate node buffers");
}

int ensure_edges(wbsph_surrogate s, int64_t E) {
  if (E <= s->cap_e) return WBSPH_OK;
  dfree(s->recv); dfree(s->send); dfree(s->efeat); dfree(s->de);
  for (auto* q : s->es) dfree(q);
  s->es.clear();
  int64_t cap = E + E / 4 + 1024;
  bool ok = dalloc(&s->recv, cap) && dalloc(&s->send, cap) && dalloc(&s->efeat, cap * FEAT) &&
            dalloc(&s->de, cap * HID);
  for (int l = 0; ok && l <= s->layers; ++l) {
    bf16* q = nullptr;
    ok = dalloc(&q, cap * HID);
    s->es.push_back(q);
  }
  s->cap_e = ok ? cap : 0;
  return ok ? WBSPH_OK : sfail(s, WBSPH_E_NOMEM, "surrogate edge buffers");
}

template <int MODE, int KP, int NP>
void launch_fwd(const MlpArgs& a, int64_t max_rows, cudaStream_t st) {
  size_t sm = FwdSmem<MODE, KP, NP>::bytes;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_fwd<MODE, KP, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  int64_t tiles = div_up(max_rows > 0 ? max_rows : 1, TILE);
  int grid = (int)(tiles < 152 * 4 ? tiles : 152 * 4);
  k_mlp_fwd<MODE, KP, NP><<<grid, MLP_THREADS, sm, st>>>(a);
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

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point
// query (no link-time dependency on libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

// TMA map of a [rows][64] BF16 row-major array: 128-row boxes, 128-byte swizzle
// (the tensor core's K-major operand layout), zero fill past the last row.
static bool rows_map(CUtensorMap* m, const bf16* base, int64_t rows) {
  auto fn = tensor_map_encoder();
  if (!fn || rows <= 0 || rows > 0x7FFFFFFF) return false;
  cuuint64_t dims[2] = {(cuuint64_t)HID, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)HID * sizeof(bf16)};
  cuuint32_t box[2] = {(cuuint32_t)HID, (cuuint32_t)TC_ROWS};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// in: rows of e (edge), 8-feature rows (encoder) or h (node); P: projections
// (edge) or aggregates (node); out: [rows][64]. Returns false when a TMA map
// cannot be built (the caller reports it).
template <int MODE>
bool launch_tc(const bf16* in, bf16* out, int64_t rows, const uint32_t* recv, const uint32_t* send,
               const bf16* P, const MlpArgs& blk, unsigned* status, cudaStream_t st) {
  if (rows <= 0) return true;
  static int sms = 0, per_sm = 1;
  if (!sms) {
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncSetAttribute(k_edge_mlp_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM_BYTES);
    // all of the unified L1/shared storage as shared memory; the persistent
    // grid holds as many CTAs per SM as their shared memory allows (two with
    // two slots), at most four (their TMEM columns then fill the 512)
    cudaFuncSetAttribute(k_edge_mlp_tc<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    per_sm = smem_sm > 0 ? smem_sm / (int)(TC_SMEM_BYTES + (size_t)reserved) : 1;
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    if (sms <= 0) sms = 152;
  }
  CUtensorMap ma, mb, mo;
  memset(&ma, 0, sizeof ma);
  memset(&mb, 0, sizeof mb);
  memset(&mo, 0, sizeof mo);
  if (MODE != TC_ENC) {
    if (!rows_map(&ma, in, rows) || !rows_map(&mo, out, rows)) return false;
    if (MODE == TC_NODE && !rows_map(&mb, P, rows)) return false;
  }
  int64_t tiles = div_up(rows, TC_ROWS);
  int grid = (int)(tiles < (int64_t)per_sm * sms ? tiles : (int64_t)per_sm * sms);
  k_edge_mlp_tc<MODE><<<grid, TC_THREADS, TC_SMEM_BYTES, st>>>(in, out, rows, recv, send, P, blk.w1, blk.kin,
                                                               blk.b1, blk.w2, blk.b2, status, ma, mb, mo);
  return true;
}

// Edge MLP of one layer on tcgen05: persistent CTAs, 2 per SM (83 KB of
// shared memory and 128 TMEM columns each).
bool launch_edge_tc(const bf16* e_in, bf16* e_out, int64_t E, const uint32_t* recv, const uint32_t* send,
                    const bf16* P, const MlpArgs& blk, unsigned* status, cudaStream_t st) {
  return launch_tc<TC_EDGE>(e_in, e_out, E, recv, send, P, blk, status, st);
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

// Graph of the sim's current state (candidate lists must be built).
int build_graph(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n,
                int64_t nf, cudaStream_t cs) {
  int rc = ensure_nodes(s, n, nf);
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
    k_sg_fill<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p, st, w, n, nf, s->row_ptr, s->recv, s->send, s->efeat,
                                                         s->norm + 8);
  k_sg_nodes<<<(unsigned)div_up(n > 0 ? n : 1, 256), 256, 0, cs>>>(p, st, n, s->norm, s->norm + 8, s->nfeat);
  return WBSPH_OK;
}

int forward(wbsph_surrogate s, const Work& w, int64_t n, int64_t nf, cudaStream_t cs) {
  const int64_t E = s->E;
  int L = s->layers;
  // node and edge encoders (tcgen05, K = 16)
  const char* tma_err = "TMA tensor map of the surrogate activations could not be built";
  launch_tc<TC_ENC>(s->nfeat, s->hs[0], n, nullptr, nullptr, nullptr, block_args(s, 0), w.status, cs);
  launch_tc<TC_ENC>(s->efeat, s->es[0], E, nullptr, nullptr, nullptr, block_args(s, 1), w.status, cs);
  const int pgrid = (int)(div_up(n > 0 ? n : 1, TILE) < 152 * 4 ? div_up(n > 0 ? n : 1, TILE) : 152 * 4);
  for (int l = 0; l < L; ++l) {
    MlpArgs a = block_args(s, 2 + 2 * l);
    k_node_proj<<<pgrid, MLP_THREADS, 0, cs>>>(s->hs[l], n, a.w1, a.b1, s->proj);
    if (!launch_edge_tc(s->es[l], s->es[l + 1], E, s->recv, s->send, s->proj, a, w.status, cs))
      return sfail(s, WBSPH_E_CUDA, tma_err);
    cudaMemsetAsync(s->aggs[l], 0, (size_t)n * HID * 2, cs);
    if (nf > 0)
      k_sg_aggregate<<<(unsigned)div_up(nf, 4), 128, 0, cs>>>(w.fluid_list, nf, s->row_ptr, s->es[l + 1], s->aggs[l]);
    // node MLP (tcgen05): h_{l+1} = h_l + MLP_n([h_l, a_l])
    if (!launch_tc<TC_NODE>(s->hs[l], s->hs[l + 1], n, nullptr, nullptr, s->aggs[l], block_args(s, 3 + 2 * l),
                       w.status, cs))
      return sfail(s, WBSPH_E_CUDA, tma_err);
  }
  {  // decoder over fluid rows
    MlpArgs a = block_args(s, 2 + 2 * L);
    a.rows = nf; a.in = s->hs[L]; a.list = w.fluid_list; a.out_f = s->out;
    launch_fwd<MODE_LIST, 64, 16>(a, nf, cs);
  }
  return WBSPH_OK;
}

void backward(wbsph_surrogate s, const Work& w, int64_t n, int64_t nf, cudaStream_t cs) {
  const int64_t E = s->E;
  int L = s->layers;
  cudaMemsetAsync(s->g, 0, (size_t)s->np * 4, cs);
  cudaMemsetAsync(s->dh, 0, (size_t)n * HID * 4, cs);
  cudaMemsetAsync(s->de, 0, (size_t)E * HID * 4 + 4, cs);
  {  // decoder: dh_L[fluid] = dX
    MlpArgs a = block_args(s, 2 + 2 * L);
    a.rows = nf; a.in = s->hs[L]; a.list = w.fluid_list; a.dout = s->dout; a.dh = s->dh;
    launch_bwd<MODE_LIST, 64, 16>(a, nf, cs);
  }
  for (int l = L - 1; l >= 0; --l) {
    MlpArgs b = block_args(s, 3 + 2 * l);  // node MLP: dh_l = dh_{l+1} + dX[:64], dagg = dX[64:]
    b.rows = n; b.h = s->hs[l]; b.agg = s->aggs[l]; b.dout = s->dh; b.din_row = s->dh; b.dagg = s->dagg;
    launch_bwd<MODE_NODE, 128, 64>(b, n, cs);
    if (nf > 0)
      k_sg_aggregate_bwd<<<(unsigned)div_up(nf, 4), 128, 0, cs>>>(w.fluid_list, nf, s->row_ptr, s->dagg, s->de);
    MlpArgs a = block_args(s, 2 + 2 * l);  // edge MLP: de_l = de_{l+1} + dX[:64], dh += scatter
    a.rows = E; a.e = s->es[l]; a.h = s->hs[l]; a.recv = s->recv; a.send = s->send;
    a.dout = s->de; a.din_row = s->de; a.dh = s->dh;
    launch_bwd<MODE_EDGE, 192, 64>(a, E, cs);
  }
  {  // encoders: weight gradients only
    MlpArgs a = block_args(s, 1);
    a.rows = E; a.in = s->efeat; a.dout = s->de;
    launch_bwd<MODE_DIRECT, 16, 64>(a, E, cs);
    MlpArgs b = block_args(s, 0);
    b.rows = n; b.in = s->nfeat; b.dout = s->dh;
    launch_bwd<MODE_DIRECT, 16, 64>(b, n, cs);
  }
}

}  // namespace

// Called by the engine for a surrogate stage: graph over the candidate lists,
// forward pass, de-normalised rates into the stage rate arrays.
namespace wbsph {
int surrogate_stage_rates(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n,
                          int64_t nf, cudaStream_t cs) {
  launch_nbr_list(p, st, w, n, nf, cs, true);
  int rc = build_graph(s, p, st, w, n, nf, cs);
  if (rc) return rc;
  if ((rc = forward(s, w, n, nf, cs))) return rc;
  if (nf > 0)
    k_sg_rates<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, n, nf, s->out, s->norm + 16, s->norm + 20);
  return WBSPH_OK;
}

// Loss of the surrogate against the rates currently in the work arrays
// (the plain pass of the same state); with `train`, backward and Adam.
int surrogate_loss(wbsph_surrogate s, const Params& p, const State& st, const Work& w, int64_t n, int64_t nf,
                   cudaStream_t cs, int train, float lr, double* loss_out, const float* dout_override,
                   float* grad_out) {
  launch_nbr_list(p, st, w, n, nf, cs, true);
  int rc = build_graph(s, p, st, w, n, nf, cs);
  if (rc) return rc;
  if ((rc = forward(s, w, n, nf, cs))) return rc;
  cudaMemsetAsync(s->loss, 0, 8, cs);
  if (nf > 0)
    k_sg_loss<<<(unsigned)div_up(nf, 128), 128, 0, cs>>>(p.dim, w, n, nf, s->out, s->norm + 16, s->norm + 20,
                                                          s->dout, s->loss);
  if (dout_override)
    cudaMemcpyAsync(s->dout, dout_override, (size_t)nf * (p.dim + 1) * 4, cudaMemcpyHostToDevice, cs);
  if (train || grad_out) backward(s, w, n, nf, cs);
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
  k_wait_probe<<<1, 1, 0, st>>>(status, limit);
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
            dalloc(&s->pb, s->np) && dalloc(&s->norm, 32) && dalloc(&s->loss, 1);
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
                                                 const float* node_std, const float* out_mean,
                                                 const float* out_std) {
  if (!s || !node_mean || !node_std || !out_mean || !out_std) return WBSPH_E_INVAL;
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
  cudaSetDevice(s->cfg.device);
  return cudaMemcpy(s->norm, nrm.data(), 32 * 4, cudaMemcpyHostToDevice) == cudaSuccess ? WBSPH_OK : WBSPH_E_CUDA;
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
