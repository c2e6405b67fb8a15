// Block-level primitives and the device-wide scan / radix sort used by the tree build.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace trevr {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Exclusive scan of one unsigned value per thread over the block (blockDim.x <= 1024,
// multiple of 32). `smem` needs 32 entries. Returns the exclusive prefix; *total gets
// the block sum. Contains __syncthreads: every thread of the block must call it.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* smem,
                                                         unsigned* total) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned s = lane < nwarps ? smem[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= (unsigned)o) s += y;
    }
    smem[lane] = s;  // inclusive prefix of warp sums
  }
  __syncthreads();
  unsigned warp_off = warp ? smem[warp - 1] : 0u;
  *total = smem[nwarps - 1];
  __syncthreads();
  return warp_off + x - v;
}

__device__ __forceinline__ unsigned long long block_reduce_add(unsigned long long v,
                                                               unsigned long long* smem) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  unsigned long long s = 0;
  if (threadIdx.x == 0)
    for (unsigned w = 0; w < nwarps; ++w) s += smem[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// ---- device-wide exclusive scan of unsigned (in place), host driver in build.cu
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// ---- LSD radix sort of (uint64 key, uint32 value), stable, 8-bit digits
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;

}  // namespace trevr
