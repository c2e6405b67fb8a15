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

__global__ void __launch_bounds__(128) walk_flat_kernel(TreeView T, const long long* sink_idx,
                                                        int n_sink, WalkParams P, float* flux_out,
                                                        int* counters,
                                                        unsigned long long* stats, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int c_rays = 0, c_segs = 0, c_visit = 0, c_ref = 0, c_clip = 0;
  bool valid = k < n_sink;
  if (valid && sink_idx) {
    const long long si = sink_idx[k];
    if (si < 0 || si >= T.n_gas) {
      atomicOr(status, kStatusInvalid);
      flux_out[k] = 0.0f;
      if (counters) reinterpret_cast<int4*>(counters)[k] = make_int4(0, 0, 0, 0);
      valid = false;
    }
  }
  if (valid) {
    const int i = sink_idx ? T.rank[sink_idx[k]] : k;
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
          F.add(rayL * expf(-t) / (12.566370614359172f * s2));
          ++c_rays;
          in_ray = false;
          continue;
        }
        if (++boxes > box_limit) {
          atomicOr(status, kStatusIterationLimit);
          break;
        }
        const float4 a = __ldg(&T.nA[box]);
        const float4 bb = __ldg(&T.nB[box]);
        const float l = clip_len(R, a, bb);
        ++c_clip;
        if (!(l > 0.0f)) continue;
        if (P.tau_ref <= 0.0f || __fmul_rn(bb.w, l) > P.tau_ref) {
          const int child = __ldg(&T.nT[box].x);
          if (child >= 0) {
            if (rsp + 2 > stack_limit) {
              atomicOr(status, kStatusStackOverflow);
              break;
            }
            ++c_ref;
            rstack[rsp++] = child + 1;
            rstack[rsp++] = child;
            continue;
          }
        }
        tau.add(a.w * l);
        ++c_segs;
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
        ++c_visit;
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
    const int out = sink_idx ? k : T.perm[i];
    flux_out[out] = F.get();
    if (counters)
      reinterpret_cast<int4*>(counters)[out] = make_int4(c_rays, c_segs, c_visit, c_ref);
  }
  if (stats) {
    unsigned long long v[5] = {(unsigned long long)c_rays, (unsigned long long)c_segs,
                               (unsigned long long)c_visit, (unsigned long long)c_ref,
                               (unsigned long long)c_clip};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      unsigned long long x = v[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[q], x);
    }
  }
}

cudaError_t launch_walk(const TreeView& T, const long long* sink_idx, int n_sink,
                        const WalkParams& wp, float* flux_out, int* counters,
                        unsigned long long* stats, int* status, int block_size,
                        cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  const int threads = 128;
  (void)block_size;
  const int blocks = (n_sink + threads - 1) / threads;
  walk_flat_kernel<<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, flux_out, counters, stats,
                                              status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trevr
