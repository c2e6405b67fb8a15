// Internal declarations shared by the CUDA translation units of libtrevr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "trevr.h"

namespace trevr {
struct TreeView;
}

namespace trevr {

constexpr int kGridBits = 21;
constexpr int kGridMax = 1 << kGridBits;  // cells per axis of the integer grid
constexpr int kRoot = 1;                  // breadth-first numbering, root at 1
constexpr int kMaxLevels = 66;            // depth <= 63 (one key bit per cut), plus slack
constexpr int kDefaultStack = 64;         // >= max depth + 1: a walk can never overflow it
constexpr int kMaxStack = 128;
constexpr int kDefaultChunk = 32;         // sinks per warp of the walk (one per lane)
constexpr int kDefaultVariant = 3;        // walk variant used when the caller passes 0
// kernel-integral table of the sub-bucket trace: Phi(x, sigma) on a uniform grid of
// x = b^2/h^2 in [0, 4] (kKintNX intervals) by sigma = s/h in [0, 2] (kKintNS intervals)
constexpr int kKintNX = 1024;
constexpr int kKintNS = 1024;

// device status bits (OR-ed by kernels, mapped to TREVR_ERR_* on the host)
constexpr int kStatusOutOfDomain = 1;
constexpr int kStatusInvalid = 2;
constexpr int kStatusStackOverflow = 4;
constexpr int kStatusIterationLimit = 8;

// Device-side view of a built tree (all pointers are device memory).
struct TreeView {
  int n_gas, n_src, n_nodes_cap;
  int bucket;
  float lo[3], side, h;
  // particles, Morton order
  const unsigned long long* key;
  const int* perm;     // sorted -> caller
  const int* rank;     // caller -> sorted
  const int* leaf_of;  // sorted -> leaf cell
  const float4* pos;   // (x, y, z, alpha), sorted
  const float* w;      // sorted weights
  // cells, breadth-first numbering (root = 1, children 2k, 2k+1)
  const float4* nA;  // (lo.x, lo.y, lo.z, abar)
  const float4* nB;  // (hi.x, hi.y, hi.z, alpha_max - alpha_min)
  const float4* nS;  // (cen.x, cen.y, cen.z, L)
  const int4* nT;    // (child or -1, parent, src_first, src_count)
  const float* nl2;  // l^2 (furthest vertex from the centre of luminosity)
  const float2* nSP; // (split plane relative to lo, split axis as int bits), internal cells
  const int* ndepth;
  const int4* nglo;  // integer box lower corner, w = split axis (-1 for a leaf)
  const int* nfirst;
  const int* ncount;
  // sources sorted by the first particle of their leaf
  const float4* src;  // (y.x, y.y, y.z, L)
  const int* src_order;
  const int* n_nodes;  // device scalar
  // several bands (trevr_build_tree_bands): up to 4 per record, unused slots 0
  int n_bands;         // 0 for a single-band tree
  const float4* bA;    // per cell: mean absorption of each band
  const float4* bLc;   // per cell: luminosity of each band
  const float4* bLs;   // per sorted source: luminosity of each band
  // sub-bucket particle trace (null unless smoothing lengths are set)
  const float4* sp;    // per sorted particle (x, y, z, h)
  const float* aw;     // per sorted particle alpha * w
  const float* dbk;    // per cell: alpha spread of a leaf's particles
  const unsigned* nbr_first;
  const int2* nbr_ja;    // per list entry: the neighbour's sorted index and alpha * w (bits)
  const float4* nbr_sp;  // per list entry: the neighbour's (x, y, z, 1/h), contiguous per leaf
  // kernel-integral table: per cell (i, j) of the kKintNX x kKintNS grid, sigma fastest,
  // the values at its corners (i, j), (i, j + 1), (i + 1, j), (i + 1, j + 1)
  const float4* kint4;
};

}  // namespace trevr

// Batch of independent trees for the persistent launch (host object behind the C handle).
struct trevr_batch {
  int device, n_trees, n_sm;
  int item;           // sinks per work item (current)
  int n_items;
  long long n_sinks;  // all gas particles of all trees
  trevr::TreeView* views;  // device, n_trees
  int2* items;             // device, work items (tree, first sorted sink)
  unsigned* counter;       // device work counter
  int* status;             // device status word
  unsigned long long* d_stats;
  long long* h_sizes;      // host, particles per tree
};

// Host-side tree object behind the opaque C handle.
struct trevr_tree {
  int device;
  long long n_gas, n_src, n_nodes;
  int max_depth;
  int bucket;
  float lo[3], side, h;
  size_t cap_nodes;
  // particles
  unsigned long long* key;
  int* perm;
  int* rank;
  int* leaf_of;
  float4* pos;
  float* w;
  // cells
  float4* nA;
  float4* nB;
  float4* nS;
  int4* nT;
  float* nl2;
  float2* nSP;
  int* ndepth;
  int* nfirst;
  int* ncount;
  int4* nglo;  // (x, y, z, split axis or -1)
  int4* nghi;
  // sources
  float4* src;
  int* src_order;
  int* src_leaf;  // leaf cell of each sorted source
  double* nW;     // sum of the volume weights of each cell (for the adjoint)
  int n_bands;    // several bands (trevr_build_tree_bands), else 0
  float4* bA;     // per cell, band means of the absorption
  float4* bLc;    // per cell, band luminosities
  float4* bLs;    // per sorted source, band luminosities
  // sub-bucket particle trace (trevr_tree_set_smoothing), else null
  float4* sp;        // per sorted particle (x, y, z, h)
  float* aw;         // per sorted particle alpha * w (absorbing mass kappa m)
  float* dbk;        // per cell: max - min of alpha over a leaf's particles (0 inside)
  unsigned* nbr_first;  // per cell + 1: start of the leaf's neighbour list
  int2* nbr_ja;      // the particles whose kernel support meets the leaf: sorted index and
                     // alpha * w (float bits)
  float4* nbr_sp;    // the same entries' (x, y, z, 1/h), so a leaf's list is read coalesced
  long long n_nbr;
  float4* kint4;     // kernel-integral table of the sub-bucket trace (see TreeView)
  int h_levels[2 * trevr::kMaxLevels];  // host copy of the level ranges
  // bookkeeping
  int* levels;    // kMaxLevels x 2 (begin, end)
  int* d_n_nodes;
  int* status;    // device status word
  unsigned long long* d_stats;  // 4 counters
  trevr::TreeView view() const;
};

namespace trevr {

// ---- build.cu
int build_tree_impl(const float* gas_xyz, const float* alpha, const float* weight, long long n_gas,
                    const float* src_xyz, const float* src_lum, long long n_src,
                    const trevr_domain* dom, int bucket, cudaStream_t s, trevr_tree** out,
                    float* build_ms);
// ---- bands.cu
int build_tree_bands_impl(const float* gas_xyz, const float* alpha_bands, const float* weight,
                          long long n_gas, const float* src_xyz, const float* lum_bands,
                          long long n_src, int n_bands, const trevr_domain* dom, int bucket,
                          cudaStream_t s, trevr_tree** out, float* build_ms);

// ---- build.cu: stable LSD radix sort of (uint64 key, uint32 value) pairs
struct SortScratch {
  unsigned long long* k2;  // n keys
  unsigned* v2;            // n values
  unsigned* counts;        // sort_count_words(n)
  unsigned* scan_scratch;  // scan_scratch_words(sort_count_words(n))
};
size_t sort_count_words(int n);
size_t scan_scratch_words(int n);
int scan_tiles(int n);
// sorts (k, v) in place by bits [0, bits) of k
void radix_sort(unsigned long long* k, unsigned* v, int n, int bits, const SortScratch& S,
                cudaStream_t s);
// exclusive prefix sum of n words in place; scratch holds scan_scratch_words(n) words
void exclusive_scan_u32(unsigned* data, int n, unsigned* scratch, cudaStream_t s);
// ---- subbucket.cu
int set_smoothing_impl(trevr_tree* t, const float* h, cudaStream_t s);

// ---- walk.cu
struct WalkParams {
  float theta2;  // theta_open^2 (fp32)
  float tau_ref;
  float smin2;   // (1e-12 side)^2 (fp32): coincident-source cut
  int stack_depth;
  int sinks_per_warp;  // sinks in each warp's chunk (0 = default)
  int variant;         // 1 = per-lane walk, 2 = warp-shared walk
  float bg_radius;     // > 0: sources are background sources on this sphere (Sec. 2.2.4)
  float tau_stop;      // early ray termination threshold (+inf = off)
  int sub_bucket;      // sub-bucket particle trace (the tree has smoothing lengths)
  int topdown;         // 1: top-down ray walk (a ray starts as its common ancestor cell)
};
// accumulators of the adjoint (FP64, zeroed by the caller)
struct AdjointArgs {
  const float* grad_flux;  // dLoss/dF per sink, caller order of the sinks
  double* G;               // per cell: sum of -g f l over segments using the cell
  double* a;               // per cell: sum of g f / L_C over merged interactions
  double* b;               // per cell, 3: sum of g grad_q f / L_C
  double* e;               // per sorted source: sum of g f / L_j over single-source rays
};
cudaError_t launch_walk_adjoint(const TreeView& T, const long long* sink_idx, int n_sink,
                                const WalkParams& wp, const AdjointArgs& J, int* status,
                                cudaStream_t s);
cudaError_t launch_walk_batched(const TreeView* views, float* const* flux_out, const int2* items,
                                int n_items, int item, unsigned* counter, const WalkParams& wp,
                                unsigned long long* stats, int* status, int block_size,
                                int n_sm, cudaStream_t s);
cudaError_t launch_walk_moments(const TreeView& T, const long long* sink_idx, int n_sink,
                                const WalkParams& wp, float* flux_out, float* fvec, float* press,
                                int* status, cudaStream_t s);
cudaError_t launch_walk(const TreeView& T, const long long* sink_idx, int n_sink,
                        const WalkParams& wp, float* flux_out, int* counters,
                        unsigned long long* stats, int* status, int block_size,
                        cudaStream_t s);
cudaError_t launch_walk_bands(const TreeView& T, const long long* sink_idx, int n_sink,
                              const WalkParams& wp, float* flux_out, int* counters,
                              unsigned long long* stats, int* status, cudaStream_t s);

// ---- adjoint.cu: from the cell accumulators to the caller's gradients
cudaError_t adjoint_finalize(const trevr_tree* t, const AdjointArgs& J, float* grad_lum,
                             float* grad_alpha, double* H, cudaStream_t s);

// ---- api.cu helpers
// Stream-ordered allocation from the library's own memory pool on the current device.
// The pool keeps freed memory for reuse (the process's default pool would return it to
// the driver at every synchronisation, and every tree build would map its buffers
// again). Free with cudaFreeAsync, or cudaFree.
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s);
int status_to_error(int status_bits);
void note_launch(int n = 1);  // count kernels launched by the library
int cuda_to_error(cudaError_t e);

}  // namespace trevr
