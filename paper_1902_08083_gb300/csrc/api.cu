// C ABI of libtrevr: argument checks, status mapping, dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "trevr.h"
#include "trevr_internal.cuh"

namespace trevr {

int status_to_error(int bits) {
  if (bits & kStatusInvalid) return TREVR_ERR_INVALID_ARGUMENT;
  if (bits & kStatusOutOfDomain) return TREVR_ERR_OUT_OF_DOMAIN;
  if (bits & kStatusStackOverflow) return TREVR_ERR_STACK_OVERFLOW;
  if (bits & kStatusIterationLimit) return TREVR_ERR_ITERATION_LIMIT;
  return TREVR_OK;
}

static std::atomic<unsigned long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

constexpr int kMaxPoolDevices = 64;
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaMallocAsync(p, bytes, s);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np = nullptr;
      e = cudaMemPoolCreate(&np, &props);
      if (e != cudaSuccess) return e;
      unsigned long long keep = ~0ull;  // never trim: freed memory stays for reuse
      e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      g_pools[dev] = np;
    }
    pool = g_pools[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int cuda_to_error(cudaError_t e) {
  if (e == cudaSuccess) return TREVR_OK;
  if (e == cudaErrorMemoryAllocation) return TREVR_ERR_OUT_OF_MEMORY;
  return TREVR_ERR_CUDA;
}

static WalkParams walk_params(const trevr_tree* t, const trevr_params* prm) {
  WalkParams wp;
  volatile float th = prm->theta_open;
  wp.theta2 = th * th;
  wp.tau_ref = prm->tau_ref;
  volatile float smin = 1e-12f * t->side;
  wp.smin2 = smin * smin;
  wp.stack_depth = prm->stack_depth > 0 ? prm->stack_depth : kDefaultStack;
  wp.sinks_per_warp = prm->sinks_per_warp;
  wp.variant = prm->walk_variant > 0 ? prm->walk_variant : kDefaultVariant;
  wp.bg_radius = prm->bg_radius;
  wp.tau_stop = prm->tau_stop > 0.0f ? prm->tau_stop : INFINITY;
  wp.sub_bucket = prm->sub_bucket;
  wp.topdown = prm->ray_walk;
  // background sources, early termination, the sub-bucket trace and the top-down ray
  // walk are built into the merged-ray walk only
  if (wp.bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket || prm->ray_walk)
    wp.variant = 3;
  return wp;
}

static bool params_ok(const trevr_params* prm) {
  if (!prm) return false;
  if (!(prm->theta_open >= 0.0f) || !std::isfinite(prm->theta_open)) return false;
  if (std::isnan(prm->tau_ref)) return false;
  if (prm->stack_depth < 0 || prm->stack_depth > kMaxStack) return false;
  if (prm->block_size < 0 || prm->block_size > 1024 || (prm->block_size % 32) != 0) return false;
  if (prm->sinks_per_warp < 0) return false;
  if (prm->walk_variant < 0 || prm->walk_variant > 3) return false;
  if (!(prm->bg_radius >= 0.0f) || !std::isfinite(prm->bg_radius)) return false;
  if (!(prm->tau_stop >= 0.0f)) return false;
  if (prm->sub_bucket != 0 && prm->sub_bucket != 1) return false;
  if (prm->ray_walk != 0 && prm->ray_walk != 1) return false;
  return true;
}

}  // namespace trevr

using namespace trevr;

TreeView trevr_tree::view() const {
  TreeView v;
  v.n_gas = (int)n_gas;
  v.n_src = (int)n_src;
  v.n_nodes_cap = (int)(n_nodes + 1);
  v.bucket = bucket;
  for (int d = 0; d < 3; ++d) v.lo[d] = lo[d];
  v.side = side;
  v.h = h;
  v.key = key;
  v.perm = perm;
  v.rank = rank;
  v.leaf_of = leaf_of;
  v.pos = pos;
  v.w = w;
  v.nA = nA;
  v.nB = nB;
  v.nS = nS;
  v.nT = nT;
  v.nl2 = nl2;
  v.nSP = nSP;
  v.ndepth = ndepth;
  v.nglo = nglo;
  v.nfirst = nfirst;
  v.ncount = ncount;
  v.src = src;
  v.src_order = src_order;
  v.n_nodes = d_n_nodes;
  v.n_bands = n_bands;
  v.bA = bA;
  v.bLc = bLc;
  v.bLs = bLs;
  v.sp = sp;
  v.aw = aw;
  v.dbk = dbk;
  v.nbr_first = nbr_first;
  v.nbr_ja = nbr_ja;
  v.nbr_sp = nbr_sp;
  v.kint4 = kint4;
  return v;
}

extern "C" {

int trevr_build_tree(const float* gas_xyz, const float* alpha, const float* weight,
                     long long n_gas, const float* src_xyz, const float* src_lum, long long n_src,
                     const trevr_domain* dom, const trevr_params* prm, void* stream,
                     trevr_tree** out) {
  if (!out) return TREVR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!gas_xyz || !alpha || !dom || !prm) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_gas < 1 || n_gas > (1ll << 30) || n_src < 0 || n_src > (1ll << 30))
    return TREVR_ERR_INVALID_ARGUMENT;
  if (n_src > 0 && (!src_xyz || !src_lum)) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bucket < 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (!(dom->side > 0.0f) || !std::isfinite(dom->side)) return TREVR_ERR_INVALID_ARGUMENT;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(dom->lo[d]) || !std::isfinite(dom->lo[d] + dom->side))
      return TREVR_ERR_INVALID_ARGUMENT;
  float ms = 0.0f;
  return build_tree_impl(gas_xyz, alpha, weight, n_gas, src_xyz, src_lum, n_src, dom,
                         prm->bucket, (cudaStream_t)stream, out, &ms);
}

int trevr_build_tree_bands(const float* gas_xyz, const float* alpha_bands, const float* weight,
                           long long n_gas, const float* src_xyz, const float* lum_bands,
                           long long n_src, int n_bands, const trevr_domain* dom,
                           const trevr_params* prm, void* stream, trevr_tree** out) {
  if (!out) return TREVR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (n_bands < 1 || n_bands > TREVR_MAX_BANDS) return TREVR_ERR_INVALID_ARGUMENT;
  if (!gas_xyz || !alpha_bands || !dom || !prm) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_gas < 1 || n_gas > (1ll << 30) || n_src < 0 || n_src > (1ll << 30))
    return TREVR_ERR_INVALID_ARGUMENT;
  if ((long long)n_bands * n_gas > (1ll << 31) - 1 || (long long)n_bands * n_src > (1ll << 31) - 1)
    return TREVR_ERR_INVALID_ARGUMENT;
  if (n_src > 0 && (!src_xyz || !lum_bands)) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bucket < 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (!(dom->side > 0.0f) || !std::isfinite(dom->side)) return TREVR_ERR_INVALID_ARGUMENT;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(dom->lo[d]) || !std::isfinite(dom->lo[d] + dom->side))
      return TREVR_ERR_INVALID_ARGUMENT;
  float ms = 0.0f;
  return build_tree_bands_impl(gas_xyz, alpha_bands, weight, n_gas, src_xyz, lum_bands, n_src,
                               n_bands, dom, prm->bucket, (cudaStream_t)stream, out, &ms);
}

int trevr_tree_set_smoothing(trevr_tree* t, const float* hsml, void* stream) {
  if (!t || !hsml || t->n_bands > 1) return TREVR_ERR_INVALID_ARGUMENT;
  return set_smoothing_impl(t, hsml, (cudaStream_t)stream);
}

int trevr_compute_flux_bands(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                             const trevr_params* prm, float* flux_out, int* sink_counters,
                             trevr_stats* stats, void* stream) {
  if (!t || !params_ok(prm) || t->n_bands < 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket || prm->ray_walk)
    return TREVR_ERR_INVALID_ARGUMENT;
  if (t->n_bands == 1)  // one band is the plain method on the same records
    return trevr_compute_flux(t, sink_idx, n_sink, prm, flux_out, sink_counters, stats, stream);
  if (n_sink < 0 || n_sink > (1ll << 30) || (long long)t->n_bands * n_sink > (1ll << 31) - 1)
    return TREVR_ERR_INVALID_ARGUMENT;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_sink == 0) return TREVR_OK;
  if (!flux_out) return TREVR_ERR_INVALID_ARGUMENT;
  if (!sink_idx && n_sink != t->n_gas) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  WalkParams wp = walk_params(t, prm);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (stats) {
    cudaMemsetAsync(t->d_stats, 0, 7 * sizeof(unsigned long long), s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  cudaError_t err = launch_walk_bands(t->view(), sink_idx, (int)n_sink, wp, flux_out,
                                      sink_counters, stats ? t->d_stats : nullptr, t->status, s);
  if (err != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return cuda_to_error(err);
  }
  unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
  if (stats) {
    cudaEventRecord(e1, s);
    cudaMemcpyAsync(h, t->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s);
  }
  int status = 0;
  cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  err = cudaStreamSynchronize(s);
  float ms = 0.0f;
  if (stats && err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_to_error(err);
  if (stats) {
    stats->interactions = (long long)h[0];
    stats->segments = (long long)h[1];
    stats->src_nodes_visited = (long long)h[2];
    stats->refine_expansions = (long long)h[3];
    stats->cells_clipped = (long long)h[4];
    stats->walk_ms = ms;
  }
  if (status) {
    cudaMemsetAsync(t->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return status_to_error(status);
  }
  return TREVR_OK;
}

int trevr_compute_flux(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                       const trevr_params* prm, float* flux_out, int* sink_counters,
                       trevr_stats* stats, void* stream) {
  if (!t || !params_ok(prm) || t->n_bands > 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink < 0 || n_sink > (1ll << 30)) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->sub_bucket && (!t->nbr_first || prm->bg_radius > 0.0f || prm->tau_stop > 0.0f))
    return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->ray_walk && (prm->bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket))
    return TREVR_ERR_INVALID_ARGUMENT;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_sink == 0) return TREVR_OK;
  if (!flux_out) return TREVR_ERR_INVALID_ARGUMENT;
  if (!sink_idx && n_sink != t->n_gas) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  WalkParams wp = walk_params(t, prm);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (stats) {
    cudaMemsetAsync(t->d_stats, 0, 7 * sizeof(unsigned long long), s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  cudaError_t err = launch_walk(t->view(), sink_idx, (int)n_sink, wp, flux_out, sink_counters,
                                stats ? t->d_stats : nullptr, t->status, prm->block_size, s);
  if (err != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return cuda_to_error(err);
  }
  if (!stats) return TREVR_OK;
  cudaEventRecord(e1, s);
  unsigned long long h[7];
  int status = 0;
  cudaMemcpyAsync(h, t->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  err = cudaStreamSynchronize(s);
  float ms = 0.0f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_to_error(err);
  stats->interactions = (long long)h[0];
  stats->segments = (long long)h[1];
  stats->src_nodes_visited = (long long)h[2];
  stats->refine_expansions = (long long)h[3];
  stats->cells_clipped = (long long)h[4];
  stats->rays_terminated = (long long)h[5];
  stats->sub_bucket_segments = (long long)h[6];
  stats->walk_ms = ms;
  if (status) {
    cudaMemsetAsync(t->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return status_to_error(status);
  }
  return TREVR_OK;
}

int trevr_compute_flux_moments(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                               const trevr_params* prm, float* flux_out, float* fvec_out,
                               float* press_out, void* stream) {
  if (!t || !params_ok(prm) || t->n_bands > 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink < 0 || n_sink > (1ll << 30)) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket || prm->ray_walk)
    return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink == 0) return TREVR_OK;
  if (!flux_out || !fvec_out) return TREVR_ERR_INVALID_ARGUMENT;
  if (!sink_idx && n_sink != t->n_gas) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  WalkParams wp = walk_params(t, prm);
  cudaError_t err = launch_walk_moments(t->view(), sink_idx, (int)n_sink, wp, flux_out, fvec_out,
                                        press_out, t->status, s);
  if (err != cudaSuccess) return cuda_to_error(err);
  int status = 0;
  cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_to_error(err);
  if (status) {
    cudaMemsetAsync(t->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return status_to_error(status);
  }
  return TREVR_OK;
}

int trevr_compute_flux_backward(const trevr_tree* t, const long long* sink_idx, long long n_sink,
                                const trevr_params* prm, const float* grad_flux, float* grad_lum,
                                float* grad_alpha, void* stream) {
  if (!t || !params_ok(prm) || t->n_bands > 1) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink < 0 || n_sink > (1ll << 30)) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink > 0 && !grad_flux) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket || prm->ray_walk)
    return TREVR_ERR_INVALID_ARGUMENT;
  if (n_sink > 0 && !sink_idx && n_sink != t->n_gas) return TREVR_ERR_INVALID_ARGUMENT;
  if ((t->n_src > 0 && !grad_lum) || !grad_alpha) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nc = (size_t)t->n_nodes + 1, ns = (size_t)(t->n_src > 0 ? t->n_src : 1);
  // accumulators: G, a, b (3 per cell), e (per source), H (per cell prefix)
  const size_t words = 5 * nc + ns + nc;
  double* buf = nullptr;
  cudaError_t err = pool_malloc_async((void**)&buf, words * sizeof(double), s);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return TREVR_ERR_OUT_OF_MEMORY;
  }
  cudaMemsetAsync(buf, 0, words * sizeof(double), s);
  AdjointArgs J;
  J.grad_flux = grad_flux;
  J.G = buf;
  J.a = buf + nc;
  J.b = buf + 2 * nc;
  J.e = buf + 5 * nc;
  double* H = buf + 5 * nc + ns;
  WalkParams wp = walk_params(t, prm);
  err = launch_walk_adjoint(t->view(), sink_idx, (int)n_sink, wp, J, t->status, s);
  if (err == cudaSuccess) err = adjoint_finalize(t, J, grad_lum, grad_alpha, H, s);
  cudaFreeAsync(buf, s);
  if (err != cudaSuccess) return cuda_to_error(err);
  int status = 0;
  cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_to_error(err);
  if (status) {
    cudaMemsetAsync(t->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return status_to_error(status);
  }
  return TREVR_OK;
}

int trevr_batch_create(trevr_tree* const* trees, int n_trees, trevr_batch** out) {
  if (!out) return TREVR_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!trees || n_trees < 1) return TREVR_ERR_INVALID_ARGUMENT;
  for (int b = 0; b < n_trees; ++b)
    if (!trees[b] || trees[b]->n_bands > 1) return TREVR_ERR_INVALID_ARGUMENT;
  trevr_batch* B = new trevr_batch();
  std::memset(B, 0, sizeof(*B));
  cudaGetDevice(&B->device);
  cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, B->device);
  B->n_trees = n_trees;
  B->h_sizes = new long long[n_trees];
  std::vector<TreeView> views(n_trees);
  for (int b = 0; b < n_trees; ++b) {
    views[b] = trees[b]->view();
    B->h_sizes[b] = trees[b]->n_gas;
    B->n_sinks += trees[b]->n_gas;
  }
  cudaError_t e = cudaMalloc(&B->views, sizeof(TreeView) * n_trees);
  if (e == cudaSuccess) e = cudaMalloc(&B->counter, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&B->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&B->d_stats, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMemcpy(B->views, views.data(), sizeof(TreeView) * n_trees, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(B->status, 0, sizeof(int));
  if (e != cudaSuccess) {
    trevr_batch_free(B);
    cudaGetLastError();
    return cuda_to_error(e);
  }
  *out = B;
  return TREVR_OK;
}

// (Re)build the work items for `item` sinks per item: trees in decreasing size, so
// the largest boxes start first and the small ones fill the tail.
static int batch_items(trevr_batch* B, int item) {
  if (B->items && B->item == item) return TREVR_OK;
  std::vector<int> order(B->n_trees);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return B->h_sizes[a] > B->h_sizes[b]; });
  std::vector<int2> items;
  for (int b : order)
    for (long long f = 0; f < B->h_sizes[b]; f += item) items.push_back(make_int2(b, (int)f));
  if (B->items) cudaFree(B->items);
  B->items = nullptr;
  cudaError_t e = cudaMalloc(&B->items, sizeof(int2) * (items.empty() ? 1 : items.size()));
  if (e == cudaSuccess)
    e = cudaMemcpy(B->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_to_error(e);
  B->item = item;
  B->n_items = (int)items.size();
  return TREVR_OK;
}

int trevr_compute_flux_batched(trevr_batch* B, const trevr_params* prm, float* const* flux_out,
                               trevr_stats* stats, void* stream) {
  if (!B || !flux_out || !params_ok(prm)) return TREVR_ERR_INVALID_ARGUMENT;
  if (prm->bg_radius > 0.0f || prm->tau_stop > 0.0f || prm->sub_bucket || prm->ray_walk)
    return TREVR_ERR_INVALID_ARGUMENT;
  const int item = prm->sinks_per_warp > 0 ? prm->sinks_per_warp : 64;
  if (item % 32 != 0 || item > (1 << 20)) return TREVR_ERR_INVALID_ARGUMENT;
  int rc = batch_items(B, item);
  if (rc != TREVR_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  WalkParams wp;
  {
    volatile float th = prm->theta_open;
    wp.theta2 = th * th;
  }
  wp.tau_ref = prm->tau_ref;
  wp.stack_depth = prm->stack_depth > 0 ? prm->stack_depth : kDefaultStack;
  wp.smin2 = 0.0f;  // set per tree by the kernel from the tree's side
  wp.sinks_per_warp = item;
  wp.variant = prm->walk_variant > 0 ? prm->walk_variant : kDefaultVariant;
  wp.bg_radius = 0.0f;
  wp.tau_stop = INFINITY;
  wp.sub_bucket = 0;
  wp.topdown = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    cudaMemsetAsync(B->d_stats, 0, 5 * sizeof(unsigned long long), s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
  }
  const int bs = prm->block_size > 0 ? prm->block_size : 128;
  cudaError_t err = launch_walk_batched(B->views, flux_out, B->items, B->n_items, item, B->counter,
                                        wp, stats ? B->d_stats : nullptr, B->status, bs, B->n_sm,
                                        s);
  if (err != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return cuda_to_error(err);
  }
  if (!stats) return TREVR_OK;
  cudaEventRecord(e1, s);
  unsigned long long h[5];
  int status = 0;
  cudaMemcpyAsync(h, B->d_stats, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&status, B->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  err = cudaStreamSynchronize(s);
  float ms = 0.0f;
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return cuda_to_error(err);
  stats->interactions = (long long)h[0];
  stats->segments = (long long)h[1];
  stats->src_nodes_visited = (long long)h[2];
  stats->refine_expansions = (long long)h[3];
  stats->cells_clipped = (long long)h[4];
  stats->walk_ms = ms;
  if (status) {
    cudaMemsetAsync(B->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return status_to_error(status);
  }
  return TREVR_OK;
}

int trevr_batch_check(const trevr_batch* B, void* stream) {
  if (!B) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  int status = 0;
  cudaMemcpyAsync(&status, B->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_to_error(err);
  if (status) {
    cudaMemsetAsync(B->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
  }
  return status_to_error(status);
}

void trevr_batch_free(trevr_batch* B) {
  if (!B) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(B->device);
  cudaDeviceSynchronize();
  if (B->views) cudaFree(B->views);
  if (B->items) cudaFree(B->items);
  if (B->counter) cudaFree(B->counter);
  if (B->status) cudaFree(B->status);
  if (B->d_stats) cudaFree(B->d_stats);
  delete[] B->h_sizes;
  cudaSetDevice(cur);
  delete B;
}

int trevr_check(const trevr_tree* t, void* stream) {
  if (!t) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  int status = 0;
  cudaMemcpyAsync(&status, t->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return cuda_to_error(err);
  if (status) {
    cudaMemsetAsync(t->status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
  }
  return status_to_error(status);
}

int trevr_tree_info(const trevr_tree* t, long long* n_nodes, int* max_depth, long long* n_gas,
                    long long* n_src) {
  if (!t) return TREVR_ERR_INVALID_ARGUMENT;
  if (n_nodes) *n_nodes = t->n_nodes;
  if (max_depth) *max_depth = t->max_depth;
  if (n_gas) *n_gas = t->n_gas;
  if (n_src) *n_src = t->n_src;
  return TREVR_OK;
}

namespace {
__global__ void export_kernel(int ncell, const int4* nglo, const int4* nghi, const int4* nT,
                              const float4* nA, const float4* nB, const float4* nS, int* child,
                              int* parent, int* glo, int* ghi, float* abar, float* dalpha,
                              float* lum, float* cen, int* src_first, int* src_count) {
  int X = blockIdx.x * blockDim.x + threadIdx.x;
  if (X >= ncell) return;
  int4 t = nT[X];
  if (child) child[X] = t.x;
  if (parent) parent[X] = t.y;
  if (src_first) src_first[X] = t.z;
  if (src_count) src_count[X] = t.w;
  int4 a = nglo[X], b = nghi[X];
  if (glo) {
    glo[3 * X] = a.x;
    glo[3 * X + 1] = a.y;
    glo[3 * X + 2] = a.z;
  }
  if (ghi) {
    ghi[3 * X] = b.x;
    ghi[3 * X + 1] = b.y;
    ghi[3 * X + 2] = b.z;
  }
  float4 A = nA[X], B = nB[X], S = nS[X];
  if (abar) abar[X] = A.w;
  if (dalpha) dalpha[X] = B.w;
  if (lum) lum[X] = S.w;
  if (cen) {
    cen[3 * X] = S.x;
    cen[3 * X + 1] = S.y;
    cen[3 * X + 2] = S.z;
  }
}
}  // namespace

int trevr_tree_export(const trevr_tree* t, unsigned long long* key, int* perm, int* leaf_of,
                      int* first, int* count, int* child, int* parent, int* depth, int* glo,
                      int* ghi, float* abar, float* dalpha, float* lum, float* cen, float* l2,
                      int* src_first, int* src_count, int* src_order, void* stream) {
  if (!t) return TREVR_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)t->n_gas, nc = (size_t)t->n_nodes + 1;
  if (key) cudaMemcpyAsync(key, t->key, n * sizeof(*key), cudaMemcpyDeviceToDevice, s);
  if (perm) cudaMemcpyAsync(perm, t->perm, n * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (leaf_of) cudaMemcpyAsync(leaf_of, t->leaf_of, n * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (first) cudaMemcpyAsync(first, t->nfirst, nc * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (count) cudaMemcpyAsync(count, t->ncount, nc * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (depth) cudaMemcpyAsync(depth, t->ndepth, nc * sizeof(int), cudaMemcpyDeviceToDevice, s);
  if (l2) cudaMemcpyAsync(l2, t->nl2, nc * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (src_order && t->n_src > 0)
    cudaMemcpyAsync(src_order, t->src_order, (size_t)t->n_src * sizeof(int),
                    cudaMemcpyDeviceToDevice, s);
  export_kernel<<<(int)((nc + 255) / 256), 256, 0, s>>>(
      (int)nc, t->nglo, t->nghi, t->nT, t->nA, t->nB, t->nS, child, parent, glo, ghi, abar, dalpha,
      lum, cen, src_first, src_count);
  note_launch();
  cudaError_t err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = cudaGetLastError();
  return cuda_to_error(err);
}

void trevr_tree_free(trevr_tree* t) {
  if (!t) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  void* ptrs[] = {t->nSP, t->key, t->perm,   t->rank,   t->leaf_of, t->pos,    t->w,      t->nA,
                  t->nB,  t->nS,     t->nT,     t->nl2,     t->ndepth, t->nfirst, t->ncount,
                  t->nglo, t->nghi,  t->src,    t->src_order, t->levels, t->d_n_nodes,
                  t->status, t->d_stats, t->src_leaf, t->nW, t->bA, t->bLc, t->bLs, t->sp, t->aw,
                  t->dbk, t->nbr_first, t->nbr_ja, t->nbr_sp, t->kint4};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  cudaSetDevice(cur);
  delete t;
}

unsigned long long trevr_kernel_launches(void) {
  return g_launches.load(std::memory_order_relaxed);
}

const char* trevr_status_string(int code) {
  switch (code) {
    case TREVR_OK: return "ok";
    case TREVR_ERR_INVALID_ARGUMENT: return "invalid argument";
    case TREVR_ERR_OUT_OF_DOMAIN: return "point outside the domain";
    case TREVR_ERR_STACK_OVERFLOW: return "traversal stack overflow";
    case TREVR_ERR_ITERATION_LIMIT: return "walk iteration limit reached";
    case TREVR_ERR_CUDA: return "CUDA error";
    case TREVR_ERR_OUT_OF_MEMORY: return "out of device memory";
    default: return "unknown status";
  }
}

}  // extern "C"
