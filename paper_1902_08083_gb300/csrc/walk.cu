// Sink walk, reverse ray and flux sum (Grond et al. 2019, Sec. 2.2.1-2.2.3).
//
// One lane per sink; sinks in Morton order, so the 32 sinks of a warp are
// neighbours in space and walk almost the same cells. Per sink:
//   * source walk: a cell with L > 0 is merged into one pseudo-source at its
//     centre of luminosity when theta_open > l/r (Eq. openangle), tested as
//     l^2 < theta^2 r^2 in fp32; otherwise it is opened, and an opened leaf
//     gives its sources one by one;
//   * reverse ray to each pseudo-source: the segments are the sink's leaf S,
//     the pseudo-source's cell C and the siblings of the cells on the two
//     paths up to the children of their lowest common ancestor A; each segment
//     uses the cell's mean absorption unless (alpha_max - alpha_min) * l >
//     tau_ref (Eq. refcrit), in which case its children are used instead;
//   * flux: sum of L exp(-tau) / (4 pi s^2) (Eq. simpint).
// The decisions (opening angle, refinement, "does the ray touch the cell")
// are evaluated with explicitly rounded fp32 operations in a fixed order.
//
// GPU form. Every lane runs one flat loop whose iterations are either one
// walk step or one cell clip, so the lanes of a warp stay converged on the
// clip work, which dominates (tens of clips per ray). The ancestors of the
// sink's leaf are listed once per sink, and the walk keeps its depth-first
// path, so the segment list of a ray is known without chasing parent links:
// the sibling of a cell is its index XOR 1 (children are allocated in pairs),
// and the common ancestor's depth is the length of the common prefix of the
// two ancestor lists, kept as a bit mask during the walk.
#include <cuda_runtime.h>
#include <stdint.h>

#include "trevr_internal.cuh"

namespace trevr {

namespace {

constexpr int kDepth = 64;  // > max cell depth (63): stacks and ancestor lists never overflow

struct Ray {
  float px, py, pz;
  float dx, dy, dz;
  float ix, iy, iz;
  float len;
};

// Length of the ray inside the box [a.xyz, b.xyz] (slab method, fp32); 0 if it misses.
__device__ __forceinline__ float clip_len(const Ray& R, const float4& a, const float4& b) {
  float t0 = 0.0f, t1 = 1.0f;
  if (R.dx != 0.0f) {
    float ta = __fmul_rn(__fsub_rn(a.x, R.px), R.ix);
    float tb = __fmul_rn(__fsub_rn(b.x, R.px), R.ix);
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  } else if (R.px < a.x || R.px > b.x) {
    return 0.0f;
  }
  if (R.dy != 0.0f) {
    float ta = __fmul_rn(__fsub_rn(a.y, R.py), R.iy);
    float tb = __fmul_rn(__fsub_rn(b.y, R.py), R.iy);
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  } else if (R.py < a.y || R.py > b.y) {
    return 0.0f;
  }
  if (R.dz != 0.0f) {
    float ta = __fmul_rn(__fsub_rn(a.z, R.pz), R.iz);
    float tb = __fmul_rn(__fsub_rn(b.z, R.pz), R.iz);
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  } else if (R.pz < a.z || R.pz > b.z) {
    return 0.0f;
  }
  return t1 > t0 ? __fmul_rn(__fsub_rn(t1, t0), R.len) : 0.0f;
}

// The same clip (identical length, so identical decisions) plus the gradient of the
// length with respect to the ray's end point q. A slab parameter t = (b - p_k)/d_k
// moves as dt/dq_k = -t/d_k; a parameter clamped to 0 or 1 does not move.
__device__ __forceinline__ float clip_len_grad(const Ray& R, const float4& a, const float4& b,
                                               float g[3]) {
  float t0 = 0.0f, t1 = 1.0f;
  int k0 = -1, k1 = -1;
  const float pp[3] = {R.px, R.py, R.pz}, dd[3] = {R.dx, R.dy, R.dz}, ii[3] = {R.ix, R.iy, R.iz};
  const float lo[3] = {a.x, a.y, a.z}, hi[3] = {b.x, b.y, b.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (dd[k] != 0.0f) {
      float ta = __fmul_rn(__fsub_rn(lo[k], pp[k]), ii[k]);
      float tb = __fmul_rn(__fsub_rn(hi[k], pp[k]), ii[k]);
      float tn = fminf(ta, tb), tx = fmaxf(ta, tb);
      if (tn > t0) { t0 = tn; k0 = k; }
      if (tx < t1) { t1 = tx; k1 = k; }
    } else if (pp[k] < lo[k] || pp[k] > hi[k]) {
      g[0] = g[1] = g[2] = 0.0f;
      return 0.0f;
    }
  }
  if (!(t1 > t0)) {
    g[0] = g[1] = g[2] = 0.0f;
    return 0.0f;
  }
  const float l = __fmul_rn(__fsub_rn(t1, t0), R.len);
  const float w = (t1 - t0) / R.len;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float dt = 0.0f;
    if (k1 == k) dt -= t1 * ii[k];
    if (k0 == k) dt += t0 * ii[k];
    g[k] = dt * R.len + w * dd[k];
  }
  return l;
}

// Neumaier-compensated fp32 sum.
struct CSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float t = __fadd_rn(s, x);
    if (fabsf(s) >= fabsf(x)) c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), x));
    else c = __fadd_rn(c, __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  __device__ __forceinline__ float get() const { return __fadd_rn(s, c); }
};

}  // namespace

struct SinkCounters {
  int rays = 0, segs = 0, visit = 0, ref = 0, clip = 0;
};

// warp-reduce the counters and add them to the device totals (all lanes call it)
__device__ __forceinline__ void add_stats(const SinkCounters& c, unsigned long long* stats) {
  unsigned long long v[5] = {(unsigned long long)c.rays, (unsigned long long)c.segs,
                             (unsigned long long)c.visit, (unsigned long long)c.ref,
                             (unsigned long long)c.clip};
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[q], x);
  }
}

// The whole hot path for one sink (sorted position i): the source walk, the
// reverse rays with refinement and the flux sum; returns the flux (forward) or
// scatters the adjoint contributions for dLoss/dF = gk (ADJ).
template <bool ADJ>
__device__ __forceinline__ float walk_sink(const TreeView& T, const int i, const float gk,
                                           const WalkParams& P, int* status,
                                           const AdjointArgs& J, SinkCounters& cnt) {
  const float4 p = T.pos[i];
  const int S = T.leaf_of[i];
  const int dS = __ldg(&T.ndepth[S]);
  const int stack_limit = P.stack_depth < kDepth ? P.stack_depth : kDepth;

  int anc[kDepth];     // ancestors of S by depth (anc[dS] = S)
  int path[kDepth];    // current depth-first path of the walk
  int wstack[kDepth];  // walk stack: cell index
  int wdepth[kDepth];  //             and its depth
  int rstack[kDepth];  // cells waiting to be clipped (refinement)
  {
    int u = S;
    for (int d = dS; d >= 0; --d) {
      anc[d] = u;
      u = __ldg(&T.nT[u].y);
    }
  }
  unsigned long long on_path = 0;  // bit d: path[d] is an ancestor of S (or S)
  wstack[0] = kRoot;
  wdepth[0] = 0;
  int sp = 1;

  CSum F;
  // ray state
  bool in_ray = false;
  Ray R;
  R.px = p.x;
  R.py = p.y;
  R.pz = p.z;
  CSum tau;
  float rayL = 0.0f, s2 = 0.0f;
  int C = 0, dC = 0, dstar = 0, nb = 0, b = 0, rsp = 0;
  // single sources of an opened leaf
  int j = 0, j_end = 0, leafC = 0, dleaf = 0;
  const int box_limit = 2 * T.n_nodes_cap + 4;
  int boxes = 0;
  // adjoint state
  int pass = 1, src_j = -1;
  float gq0 = 0.0f, gq1 = 0.0f, gq2 = 0.0f, fcur = 0.0f;

  while (true) {
    if (in_ray) {
      int box;
      if (rsp > 0) {
        box = rstack[--rsp];
      } else if (b < nb) {
        const int nS_side = dS - dstar - 1;  // siblings on the sink side
        if (b == 0) box = S;
        else if (b <= nS_side) box = anc[dS - b + 1] ^ 1;
        else if (b == nS_side + 1) box = C;
        else box = path[dC - (b - nS_side - 2)] ^ 1;
        ++b;
      } else {
        const float t = tau.get();
        const float f = rayL * expf(-t) / (12.566370614359172f * s2);
        if (!ADJ) {
          F.add(f);
          ++cnt.rays;
          in_ray = false;
        } else if (pass == 1) {
          // second pass over the same cells, now that f is known
          fcur = f;
          pass = 2;
          b = 0;
          rsp = 0;
          boxes = 0;
        } else {
          const float gf = gk * fcur;
          if (src_j >= 0) {
            atomicAdd(&J.e[src_j], (double)(gf / rayL));
          } else {
            const float c = gf / rayL, inv_s2 = 2.0f / s2;
            atomicAdd(&J.a[C], (double)c);
            atomicAdd(&J.b[3 * C + 0], (double)(c * (-R.dx * inv_s2 - gq0)));
            atomicAdd(&J.b[3 * C + 1], (double)(c * (-R.dy * inv_s2 - gq1)));
            atomicAdd(&J.b[3 * C + 2], (double)(c * (-R.dz * inv_s2 - gq2)));
          }
          ++cnt.rays;
          in_ray = false;
        }
        continue;
      }
      if (++boxes > box_limit) {
        atomicOr(status, kStatusIterationLimit);
        break;
      }
      const float4 a = __ldg(&T.nA[box]);
      const float4 bb = __ldg(&T.nB[box]);
      float gl[3];
      const bool want_grad = ADJ && pass == 1 && src_j < 0;
      const float l = want_grad ? clip_len_grad(R, a, bb, gl) : clip_len(R, a, bb);
      ++cnt.clip;
      if (!(l > 0.0f)) continue;
      if (P.tau_ref <= 0.0f || __fmul_rn(bb.w, l) > P.tau_ref) {
        const int child = __ldg(&T.nT[box].x);
        if (child >= 0) {
          if (rsp + 2 > stack_limit) {
            atomicOr(status, kStatusStackOverflow);
            break;
          }
          ++cnt.ref;
          rstack[rsp++] = child + 1;
          rstack[rsp++] = child;
          continue;
        }
      }
      if (ADJ && pass == 2) {
        atomicAdd(&J.G[box], (double)(-gk * fcur * l));
        continue;
      }
      tau.add(a.w * l);
      if (want_grad) {
        gq0 = fmaf(a.w, gl[0], gq0);
        gq1 = fmaf(a.w, gl[1], gq1);
        gq2 = fmaf(a.w, gl[2], gq2);
      }
      ++cnt.segs;
      continue;
    }

    // ---- walk step: next pseudo-source
    float qx, qy, qz, L;
    if (j < j_end) {
      const float4 y = __ldg(&T.src[j]);
      ++j;
      if (!(y.w > 0.0f)) continue;
      C = leafC;
      dC = dleaf;
      src_j = j - 1;
      qx = y.x;
      qy = y.y;
      qz = y.z;
      L = y.w;
    } else {
      if (sp == 0) break;
      --sp;
      const int X = wstack[sp];
      const int dX = wdepth[sp];
      path[dX] = X;
      const unsigned long long bit = 1ull << dX;
      on_path = (dX <= dS && anc[dX] == X) ? (on_path | bit) : (on_path & ~bit);
      const float4 s = __ldg(&T.nS[X]);
      if (!(s.w > 0.0f)) continue;
      ++cnt.visit;
      const float4 a = __ldg(&T.nA[X]);
      const float4 bb = __ldg(&T.nB[X]);
      const float ex = fmaxf(fmaxf(__fsub_rn(a.x, p.x), __fsub_rn(p.x, bb.x)), 0.0f);
      const float ey = fmaxf(fmaxf(__fsub_rn(a.y, p.y), __fsub_rn(p.y, bb.y)), 0.0f);
      const float ez = fmaxf(fmaxf(__fsub_rn(a.z, p.z), __fsub_rn(p.z, bb.z)), 0.0f);
      const float r2 =
          __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
      if (!(__ldg(&T.nl2[X]) < __fmul_rn(P.theta2, r2))) {
        const int4 t = __ldg(&T.nT[X]);
        if (t.x < 0) {
          j = t.z;
          j_end = t.z + t.w;
          leafC = X;
          dleaf = dX;
        } else {
          if (sp + 2 > stack_limit) {
            atomicOr(status, kStatusStackOverflow);
            break;
          }
          wstack[sp] = t.x + 1;
          wdepth[sp] = dX + 1;
          wstack[sp + 1] = t.x;
          wdepth[sp + 1] = dX + 1;
          sp += 2;
        }
        continue;
      }
      C = X;
      dC = dX;
      src_j = -1;
      qx = s.x;
      qy = s.y;
      qz = s.z;
      L = s.w;
    }
    // ---- start the reverse ray from the sink to (q, L) in cell C
    R.dx = __fsub_rn(qx, p.x);
    R.dy = __fsub_rn(qy, p.y);
    R.dz = __fsub_rn(qz, p.z);
    s2 = __fadd_rn(__fadd_rn(__fmul_rn(R.dx, R.dx), __fmul_rn(R.dy, R.dy)),
                   __fmul_rn(R.dz, R.dz));
    if (s2 < P.smin2) continue;  // a source on top of the sink adds nothing
    R.len = __fsqrt_rn(s2);
    R.ix = R.dx != 0.0f ? __frcp_rn(R.dx) : 0.0f;
    R.iy = R.dy != 0.0f ? __frcp_rn(R.dy) : 0.0f;
    R.iz = R.dz != 0.0f ? __frcp_rn(R.dz) : 0.0f;
    rayL = L;
    tau = CSum();
    pass = 1;
    gq0 = gq1 = gq2 = 0.0f;
    b = 0;
    rsp = 0;
    boxes = 0;
    if (C == S) {
      nb = 1;
    } else {
      // depth of the lowest common ancestor: the common prefix of path and anc
      const int mn = dC < dS ? dC : dS;
      const unsigned long long m = on_path & ((2ull << mn) - 1ull);  // mn <= 62
      dstar = __ffsll((long long)~m) - 2;
      nb = dS + dC - 2 * dstar;
    }
    in_ray = true;
  }
  return F.get();
}

// ADJ = false: forward flux. ADJ = true: the adjoint with the same decisions; every
// ray is traced twice, first for tau and d(tau)/dq, then, with the contribution f
// known, to scatter -g f l_X into each segment cell (FP64 atomics).
template <bool ADJ>
__global__ void __launch_bounds__(128) walk_flat_kernel(TreeView T, const long long* sink_idx,
                                                        int n_sink, WalkParams P, float* flux_out,
                                                        int* counters,
                                                        unsigned long long* stats, int* status,
                                                        AdjointArgs J) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  SinkCounters cnt;
  bool valid = k < n_sink;
  if (valid && sink_idx) {
    const long long si = sink_idx[k];
    if (si < 0 || si >= T.n_gas) {
      atomicOr(status, kStatusInvalid);
      if (!ADJ) flux_out[k] = 0.0f;
      if (counters) reinterpret_cast<int4*>(counters)[k] = make_int4(0, 0, 0, 0);
      valid = false;
    }
  }
  if (ADJ && valid) {
    // the adjoint skips sinks whose dLoss/dF (caller order, like the fluxes) is zero
    const int i0 = sink_idx ? T.rank[sink_idx[k]] : k;
    if (J.grad_flux[sink_idx ? k : T.perm[i0]] == 0.0f) valid = false;
  }
  if (valid) {
    const int i = sink_idx ? T.rank[sink_idx[k]] : k;
    const float gk = ADJ ? J.grad_flux[sink_idx ? k : T.perm[i]] : 0.0f;
    const float Fv = walk_sink<ADJ>(T, i, gk, P, status, J, cnt);
    if (!ADJ) {
      const int out = sink_idx ? k : T.perm[i];
      flux_out[out] = Fv;
      if (counters)
        reinterpret_cast<int4*>(counters)[out] = make_int4(cnt.rays, cnt.segs, cnt.visit, cnt.ref);
    }
  }
  if (stats) add_stats(cnt, stats);
}

// Many independent trees in one persistent launch. Work items are runs of
// `item` consecutive sinks (Morton order) of one tree; each warp takes the next
// item from a device counter, so warps that finish early keep pulling work from
// the boxes that are left. Per-sink arithmetic is the same as walk_flat_kernel.
template <int BS>
__global__ void __launch_bounds__(BS) walk_batched_kernel(const TreeView* __restrict__ views,
                                                         float* const* __restrict__ flux_out,
                                                         const int2* __restrict__ items,
                                                         int n_items, int item,
                                                         unsigned* counter, WalkParams P,
                                                         unsigned long long* stats, int* status) {
  const unsigned lane = threadIdx.x & 31u;
  SinkCounters cnt;
  while (true) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)n_items) break;
    const int2 w = items[it];
    const TreeView T = views[w.x];
    float* out = flux_out[w.x];
    WalkParams Pt = P;  // the coincident-source cut (1e-12 side)^2 of this tree, in fp32
    const float smin = __fmul_rn(1e-12f, T.side);
    Pt.smin2 = __fmul_rn(smin, smin);
    const int end = min(w.y + item, T.n_gas);
    for (int i = w.y + (int)lane; i < end; i += 32) {
      const float f = walk_sink<false>(T, i, 0.0f, Pt, status, AdjointArgs{}, cnt);
      out[T.perm[i]] = f;
    }
  }
  if (stats) add_stats(cnt, stats);
}

cudaError_t launch_walk_batched(const TreeView* views, float* const* flux_out, const int2* items,
                                int n_items, int item, unsigned* counter, const WalkParams& wp,
                                unsigned long long* stats, int* status, int block_size,
                                int n_sm, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (block_size <= 64) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_batched_kernel<64>, 64, 0);
    walk_batched_kernel<64><<<n_sm * per_sm, 64, 0, s>>>(views, flux_out, items, n_items, item,
                                                         counter, wp, stats, status);
  } else if (block_size <= 128) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_batched_kernel<128>, 128, 0);
    walk_batched_kernel<128><<<n_sm * per_sm, 128, 0, s>>>(views, flux_out, items, n_items, item,
                                                           counter, wp, stats, status);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_batched_kernel<256>, 256, 0);
    walk_batched_kernel<256><<<n_sm * per_sm, 256, 0, s>>>(views, flux_out, items, n_items, item,
                                                           counter, wp, stats, status);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_walk(const TreeView& T, const long long* sink_idx, int n_sink,
                        const WalkParams& wp, float* flux_out, int* counters,
                        unsigned long long* stats, int* status, int block_size,
                        cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  const int threads = 128;
  (void)block_size;
  const int blocks = (n_sink + threads - 1) / threads;
  walk_flat_kernel<false><<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, flux_out, counters,
                                                     stats, status, AdjointArgs{});
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_walk_adjoint(const TreeView& T, const long long* sink_idx, int n_sink,
                                const WalkParams& wp, const AdjointArgs& J, int* status,
                                cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (n_sink + threads - 1) / threads;
  walk_flat_kernel<true><<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, nullptr, nullptr,
                                                    nullptr, status, J);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trevr
