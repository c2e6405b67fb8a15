// Morton keys + stable sort of the particles with no device allocation.
//
// Some callers cannot allocate device memory while they run: a host code that
// reserves all of its device memory up front and forbids further allocation
// inside its time-step loop, or a plug-in that only receives buffers from the
// application that owns the GPU. For them this file provides one entry point
// that keeps all of its scratch memory in a fixed, file-scope device array,
// so the call itself never allocates or frees anything.
//
// The array is sized for at most TREVR_NOALLOC_MAX_N particles. Every GPU that
// loads this library holds it (about 12.3 MiB) until the process exits. All
// calls share it, and each call overwrites it: two calls whose work overlaps on
// the GPU (other streams, other host threads) race on the same scratch.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "morton.cuh"
#include "primitives.cuh"
#include "trevr.h"
#include "trevr_internal.cuh"

namespace trevr {
namespace {

constexpr int kMaxN = TREVR_NOALLOC_MAX_N;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// layout of the scratch array
constexpr size_t kOffK2 = 0;
constexpr size_t kOffV2 = kOffK2 + align256((size_t)kMaxN * sizeof(unsigned long long));
constexpr size_t kOffCounts = kOffV2 + align256((size_t)kMaxN * sizeof(unsigned));
constexpr size_t kCountWords = (size_t)256 * ((kMaxN + kSortTile - 1) / kSortTile);
constexpr size_t kOffScan = kOffCounts + align256(kCountWords * sizeof(unsigned));
constexpr size_t kScanWords = 4096;  // >= scan_scratch_words(kCountWords), checked at set-up
constexpr size_t kOffStatus = kOffScan + align256(kScanWords * sizeof(unsigned));
constexpr size_t kScratchBytes = kOffStatus + 256;

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once per
// device (the host-side name of a __device__ array is not a device address).
// The cached address belongs to the device's current context: after
// cudaDeviceReset the module is loaded again and the array may move, so a
// process that resets a device must not call this entry point on it again.
cudaError_t scratch_on_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void noalloc_keys_kernel(const float* __restrict__ xyz, int n, Domain32 D,
                                    unsigned long long* __restrict__ keys,
                                    unsigned* __restrict__ vals, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x = xyz[i], y = xyz[(size_t)n + i], z = xyz[2 * (size_t)n + i];
  unsigned long long k = 0;
  if (in_dom(x, D.lo[0], D.hi[0]) && in_dom(y, D.lo[1], D.hi[1]) && in_dom(z, D.lo[2], D.hi[2])) {
    k = (expand3(quantize(x, D.lo[0], D.scale)) << 2) |
        (expand3(quantize(y, D.lo[1], D.scale)) << 1) | expand3(quantize(z, D.lo[2], D.scale));
  } else {
    atomicOr(status, kStatusOutOfDomain);
  }
  keys[i] = k;
  vals[i] = (unsigned)i;
}

}  // namespace
}  // namespace trevr

using namespace trevr;

extern "C" int trevr_morton_sort_noalloc(const float* gas_xyz, long long n_gas,
                                         const trevr_domain* dom, unsigned long long* keys_out,
                                         int* perm_out, void* stream) {
  if (!gas_xyz || !dom || !keys_out || !perm_out) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_gas < 1 || n_gas > kMaxN) return TREVR_ERR_INVALID_ARGUMENT;
  if (!(dom->side > 0.0f) || !std::isfinite(dom->side)) return TREVR_ERR_INVALID_ARGUMENT;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(dom->lo[d]) || !std::isfinite(dom->lo[d] + dom->side))
      return TREVR_ERR_INVALID_ARGUMENT;
  if (scan_scratch_words((int)sort_count_words((int)n_gas)) > kScanWords)
    return TREVR_ERR_INVALID_ARGUMENT;
  unsigned char* base = nullptr;
  cudaError_t err = scratch_on_current_device(&base);
  if (err != cudaSuccess) return cuda_to_error(err);
  cudaStream_t s = (cudaStream_t)stream;
  const int n = (int)n_gas;
  SortScratch S;
  S.k2 = reinterpret_cast<unsigned long long*>(base + kOffK2);
  S.v2 = reinterpret_cast<unsigned*>(base + kOffV2);
  S.counts = reinterpret_cast<unsigned*>(base + kOffCounts);
  S.scan_scratch = reinterpret_cast<unsigned*>(base + kOffScan);
  int* status = reinterpret_cast<int*>(base + kOffStatus);
  // the status word must start at zero; the rest of the scratch is fully
  // overwritten before it is read
  err = cudaMemsetAsync(status, 0, sizeof(int), s);
  if (err != cudaSuccess) return cuda_to_error(err);
  Domain32 D;
  for (int d = 0; d < 3; ++d) {
    volatile float lo = dom->lo[d], side = dom->side;
    D.lo[d] = lo;
    D.hi[d] = lo + side;
  }
  {
    volatile float side = dom->side;
    D.scale = 2097152.0f / side;
    D.h = side * (1.0f / 2097152.0f);
  }
  noalloc_keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(gas_xyz, n, D, keys_out,
                                                       reinterpret_cast<unsigned*>(perm_out),
                                                       status);
  note_launch();
  radix_sort(keys_out, reinterpret_cast<unsigned*>(perm_out), n, 63, S, s);
  int h_status = 0;
  err = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_to_error(err);
  return status_to_error(h_status);
}
