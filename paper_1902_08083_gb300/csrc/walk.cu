// Sink walk, reverse ray and flux sum (Grond et al. 2019, Sec. 2.2.1-2.2.3).
//
// One thread per sink; sinks in Morton order, so the 32 sinks of a warp are
// neighbours in space and walk almost the same cells. Per sink:
//   * source walk: a cell with L > 0 is merged into one pseudo-source at its
//     centre of luminosity when theta_open > l/r (Eq. openangle), tested as
//     l^2 < theta^2 r^2 in fp32; otherwise it is opened, and an opened leaf
//     gives its sources one by one;
//   * reverse ray to each pseudo-source: the segments are the sink's leaf S,
//     the pseudo-source's cell C and the siblings of the cells on the two
//     paths up to the children of their lowest common ancestor; each segment
//     uses the cell's mean absorption unless (alpha_max - alpha_min) * l >
//     tau_ref (Eq. refcrit), in which case its children are used instead;
//   * flux: sum of L exp(-tau) / (4 pi s^2) (Eq. simpint).
// The decisions (opening angle, refinement, "does the ray touch the cell")
// are evaluated with explicitly rounded fp32 operations in a fixed order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "trevr_internal.cuh"

namespace trevr {

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

struct Counters {
  int rays = 0, segs = 0, visited = 0, refines = 0, clips = 0;
};

template <int STACK>
struct RayTracer {
  const TreeView& T;
  const WalkParams& P;
  Ray R;
  CSum tau;
  Counters& cnt;
  int* status;

  __device__ RayTracer(const TreeView& t, const WalkParams& p, Counters& c, int* st)
      : T(t), P(p), cnt(c), status(st) {}

  // optical depth through cell X, refined where Eq. refcrit asks
  __device__ __forceinline__ void seg(int X) {
    int stack[STACK];
    int sp = 0;
    stack[sp++] = X;
    while (sp > 0) {
      const int Y = stack[--sp];
      const float4 a = __ldg(&T.nA[Y]);
      const float4 b = __ldg(&T.nB[Y]);
      const float l = clip_len(R, a, b);
      ++cnt.clips;
      if (!(l > 0.0f)) continue;
      const int child = __ldg(&T.nT[Y].x);
      if (child >= 0 && (P.tau_ref <= 0.0f || __fmul_rn(b.w, l) > P.tau_ref)) {
        if (sp + 2 > STACK) {
          atomicOr(status, kStatusStackOverflow);
          return;
        }
        ++cnt.refines;
        stack[sp++] = child + 1;
        stack[sp++] = child;
        continue;
      }
      tau.add(a.w * l);
      ++cnt.segs;
    }
  }

  // flux of luminosity L at q (inside cell C) seen from the sink at p in leaf S
  __device__ float contribute(float px, float py, float pz, int S, int C, float qx, float qy,
                              float qz, float L) {
    R.px = px;
    R.py = py;
    R.pz = pz;
    R.dx = __fsub_rn(qx, px);
    R.dy = __fsub_rn(qy, py);
    R.dz = __fsub_rn(qz, pz);
    const float s2 =
        __fadd_rn(__fadd_rn(__fmul_rn(R.dx, R.dx), __fmul_rn(R.dy, R.dy)), __fmul_rn(R.dz, R.dz));
    if (s2 < P.smin2) return 0.0f;  // a source on top of the sink adds nothing
    R.len = __fsqrt_rn(s2);
    R.ix = R.dx != 0.0f ? __frcp_rn(R.dx) : 0.0f;
    R.iy = R.dy != 0.0f ? __frcp_rn(R.dy) : 0.0f;
    R.iz = R.dz != 0.0f ? __frcp_rn(R.dz) : 0.0f;
    tau = CSum();
    seg(S);
    if (S != C) {
      seg(C);
      int u = S, v = C;
      int du = __ldg(&T.ndepth[u]), dv = __ldg(&T.ndepth[v]);
      while (du > dv) {
        seg(u ^ 1);
        u = __ldg(&T.nT[u].y);
        --du;
      }
      while (dv > du) {
        seg(v ^ 1);
        v = __ldg(&T.nT[v].y);
        --dv;
      }
      while (true) {
        const int pu = __ldg(&T.nT[u].y), pv = __ldg(&T.nT[v].y);
        if (pu == pv) break;
        seg(u ^ 1);
        seg(v ^ 1);
        u = pu;
        v = pv;
      }
    }
    ++cnt.rays;
    const float t = tau.get();
    return L * expf(-t) / (12.566370614359172f * s2);
  }
};

template <int STACK>
__global__ void __launch_bounds__(128) walk_plain_kernel(TreeView T, const long long* sink_idx,
                                                         int n_sink, WalkParams P, float* flux_out,
                                                         int* counters,
                                                         unsigned long long* stats, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  Counters cnt;
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
    int i = sink_idx ? T.rank[sink_idx[k]] : k;
    const float4 p = T.pos[i];
    const int S = T.leaf_of[i];
    RayTracer<STACK> rt(T, P, cnt, status);
    CSum F;
    int stack[STACK];
    int sp = 0;
    stack[sp++] = kRoot;
    const int limit = 2 * T.n_nodes_cap + 2;
    int iters = 0;
    while (sp > 0) {
      const int X = stack[--sp];
      if (++iters > limit) {
        atomicOr(status, kStatusIterationLimit);
        break;
      }
      const float4 s = __ldg(&T.nS[X]);
      if (!(s.w > 0.0f)) continue;
      ++cnt.visited;
      const float4 a = __ldg(&T.nA[X]);
      const float4 b = __ldg(&T.nB[X]);
      const float ex = fmaxf(fmaxf(__fsub_rn(a.x, p.x), __fsub_rn(p.x, b.x)), 0.0f);
      const float ey = fmaxf(fmaxf(__fsub_rn(a.y, p.y), __fsub_rn(p.y, b.y)), 0.0f);
      const float ez = fmaxf(fmaxf(__fsub_rn(a.z, p.z), __fsub_rn(p.z, b.z)), 0.0f);
      const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
      if (__ldg(&T.nl2[X]) < __fmul_rn(P.theta2, r2)) {
        F.add(rt.contribute(p.x, p.y, p.z, S, X, s.x, s.y, s.z, s.w));
        continue;
      }
      const int4 t = __ldg(&T.nT[X]);
      if (t.x < 0) {
        for (int j = t.z; j < t.z + t.w; ++j) {
          const float4 y = __ldg(&T.src[j]);
          if (!(y.w > 0.0f)) continue;
          F.add(rt.contribute(p.x, p.y, p.z, S, X, y.x, y.y, y.z, y.w));
        }
      } else {
        if (sp + 2 > STACK) {
          atomicOr(status, kStatusStackOverflow);
          break;
        }
        stack[sp++] = t.x + 1;
        stack[sp++] = t.x;
      }
    }
    const int out = sink_idx ? k : T.perm[i];
    flux_out[out] = F.get();
    if (counters) {
      int4 c = make_int4(cnt.rays, cnt.segs, cnt.visited, cnt.refines);
      reinterpret_cast<int4*>(counters)[out] = c;
    }
  }
  if (stats) {
    unsigned long long v[5] = {(unsigned long long)cnt.rays, (unsigned long long)cnt.segs,
                               (unsigned long long)cnt.visited, (unsigned long long)cnt.refines,
                               (unsigned long long)cnt.clips};
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      unsigned long long x = v[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[j], x);
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
  if (wp.stack_depth <= 4)  // only useful to exercise the overflow check
    walk_plain_kernel<4><<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, flux_out, counters,
                                                    stats, status);
  else if (wp.stack_depth <= 32)
    walk_plain_kernel<32><<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, flux_out, counters,
                                                     stats, status);
  else
    walk_plain_kernel<64><<<blocks, threads, 0, s>>>(T, sink_idx, n_sink, wp, flux_out, counters,
                                                     stats, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trevr
