// noalloc.cu -- wbsph_sort_cells_noalloc: cell keys and the stable radix sort
// of the neighbour build without any device allocation.
//
// Some callers cannot let a library allocate device memory: applications
// whose framework owns the whole device memory pool and forbids allocations
// behind its back, and latency-critical loops in which the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable. For them this
// entry point keeps its scratch (radix histograms, the ping-pong key/index
// buffers and a status word) in one file-scope device array instead of
// allocating it. The array exists once per GPU that loads the library and
// stays allocated until the process exits.
#include <mutex>

#include "../../include/wbsph.h"
#include "common.cuh"

namespace wbsph {
const Params* handle_params(wbsph_handle h);
cudaStream_t handle_stream(wbsph_handle h);
int handle_device(wbsph_handle h);
int handle_fail(wbsph_handle h, int code, const char* msg);
}  // namespace wbsph

using namespace wbsph;

namespace {

constexpr int64_t kMaxN = WBSPH_NOALLOC_MAX_N;
constexpr int64_t kTile = 4096;  // keys per radix tile (256 threads x 16)
constexpr int64_t kHistWords = 256 * ((kMaxN + kTile - 1) / kTile) + 256;  // table + row totals
// layout (32-bit words): [keys kMaxN][ids kMaxN][histograms kHistWords][status 64]
constexpr int64_t kScratchWords = 2 * kMaxN + kHistWords + 64;

static __device__ __align__(256) uint32_t g_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_dev_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch for device `dev` (current). The host-side name
// g_scratch is only a stand-in for the symbol, never a device address.
int scratch_address(int dev, uint32_t** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return WBSPH_E_CUDA;
    }
    g_dev_ptr[dev] = (uint32_t*)p;
  }
  *out = g_dev_ptr[dev];
  return WBSPH_OK;
}

int sort_on_device(wbsph_handle h, int dev, const double* x, int64_t n, uint32_t* keys_sorted,
                   uint32_t* ids_sorted);

}  // namespace

extern "C" int wbsph_sort_cells_noalloc(wbsph_handle h, const double* x, int64_t n,
                                        uint32_t* keys_sorted, uint32_t* ids_sorted) {
  if (!h) return WBSPH_E_INVAL;
  if (n < 0) return handle_fail(h, WBSPH_E_INVAL, "n < 0");
  if (n > kMaxN)
    return handle_fail(h, WBSPH_E_CAPACITY,
                       "n exceeds the no-allocation limit WBSPH_NOALLOC_MAX_N (524288 particles)");
  if (n == 0) return WBSPH_OK;
  if (!x || !keys_sorted || !ids_sorted) return handle_fail(h, WBSPH_E_INVAL, "null pointer");
  int dev = handle_device(h);
  if (dev < 0 || dev >= kMaxDevices) return handle_fail(h, WBSPH_E_INVAL, "device ordinal out of range");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return handle_fail(h, WBSPH_E_CUDA, "cudaGetDevice failed");
  }
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return handle_fail(h, WBSPH_E_CUDA, "cudaSetDevice failed");
  }
  int rc = sort_on_device(h, dev, x, n, keys_sorted, ids_sorted);
  if (prev != dev) cudaSetDevice(prev);  // the caller's current device, as it was
  return rc;
}

namespace {

int sort_on_device(wbsph_handle h, int dev, const double* x, int64_t n, uint32_t* keys_sorted,
                   uint32_t* ids_sorted) {
  uint32_t* base = nullptr;
  if (scratch_address(dev, &base) != WBSPH_OK)
    return handle_fail(h, WBSPH_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
  cudaStream_t st = handle_stream(h);
  const Params& p = *handle_params(h);

  State s{};
  s.x = const_cast<double*>(x);
  Work w{};
  w.key = keys_sorted;
  w.perm = ids_sorted;
  w.key_alt = base;
  w.perm_alt = base + kMaxN;
  w.hist = base + 2 * kMaxN;
  w.status = base + 2 * kMaxN + kHistWords;
  // the status word must start at zero; histograms are fully rewritten per pass
  if (cudaMemsetAsync(w.status, 0, sizeof(unsigned), st) != cudaSuccess) {
    cudaGetLastError();
    return handle_fail(h, WBSPH_E_CUDA, "clearing the status word failed");
  }
  launch_cell_keys(p, s, w, n, st);
  int launches = 0;
  Work r = w;
  launch_radix_sort(p, r, n, st, &launches);  // r.key / r.perm: buffers holding the result
  if (r.key != keys_sorted)
    cudaMemcpyAsync(keys_sorted, r.key, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  if (r.perm != ids_sorted)
    cudaMemcpyAsync(ids_sorted, r.perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
  unsigned status = 0;
  cudaMemcpyAsync(&status, w.status, sizeof status, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return handle_fail(h, WBSPH_E_CUDA, cudaGetErrorString(e));
  if (status & kStatDomain) return handle_fail(h, WBSPH_E_DOMAIN, "a particle is outside the domain");
  return WBSPH_OK;
}

}  // namespace
