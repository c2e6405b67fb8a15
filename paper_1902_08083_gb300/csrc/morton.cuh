// Morton-key helpers shared by the tree build and the fixed-scratch sort entry point.
#pragma once

#include <cuda_runtime.h>

#include "trevr_internal.cuh"

namespace trevr {

__device__ __forceinline__ unsigned long long expand3(unsigned v) {
  unsigned long long x = v & 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ unsigned compact3(unsigned long long x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (unsigned)x;
}

// grid coordinate of key along axis a (0 = x, the most significant)
__device__ __forceinline__ unsigned key_coord(unsigned long long key, int a) {
  return compact3(key >> (2 - a));
}

struct Domain32 {
  float lo[3], hi[3], scale, h;
};

// q = floor((x - lo) * scale) in fp32 (one rounded subtraction, one rounded
// multiplication), clamped to 2^21 - 1. Caller has checked lo <= x < hi.
__device__ __forceinline__ unsigned quantize(float x, float lo, float scale) {
  float t = __fmul_rn(__fsub_rn(x, lo), scale);
  unsigned q = __float2uint_rz(t);
  return q > (unsigned)(kGridMax - 1) ? (unsigned)(kGridMax - 1) : q;
}

__device__ __forceinline__ bool in_dom(float x, float lo, float hi) { return x >= lo && x < hi; }

}  // namespace trevr
