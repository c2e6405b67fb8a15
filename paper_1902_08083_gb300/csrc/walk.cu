// Sink walk, reverse ray and flux sum (Grond et al. 2019, Sec. 2.2.1-2.2.3).
//
// Per sink (a gas particle at p in leaf S):
//   * source walk: a cell with L > 0 is merged into one pseudo-source at its
//     centre of luminosity when theta_open > l/r (Eq. openangle), tested as
//     l^2 < theta^2 r^2 in fp32; otherwise it is opened, and an opened leaf
//     gives its sources one by one;
//   * reverse ray to each pseudo-source: the segments are S, the pseudo-source's
//     cell C and the siblings of the cells on the two paths up to the children
//     of their lowest common ancestor A; each segment uses the cell's mean
//     absorption unless (alpha_max - alpha_min) * l > tau_ref (Eq. refcrit), in
//     which case its children are used instead;
//   * flux: sum of L exp(-tau) / (4 pi s^2) (Eq. simpint).
// The decisions (opening angle, refinement, "does the ray touch the cell") are
// evaluated with explicitly rounded fp32 operations in a fixed order. Positions,
// centres of luminosity and cell planes are stored relative to the domain's lower
// corner (planes g * h), so their fp32 rounding depends on the domain's size and not
// on its offset from the origin.
//
// GPU form (sinks in Morton order, so the lanes of a warp are neighbours in space).
//   * Variant 1 (walk_kernel): one lane per sink, a flat loop in which one
//     iteration is a walk step or a cell clip, cells picked with selects from one
//     per-lane list; a lane that finishes takes the next sink of its warp's chunk.
//   * Variant 2 (walk_warp_kernel, MERGE = false): the 32 lanes walk one shared
//     stack in shared memory with a mask of the lanes that still need each cell,
//     and trace together the rays to a cell they accept together.
//   * Variant 3 (MERGE = true, the default): as 2, but a lane keeps its next ray
//     pending, and the pending rays of all lanes (to different cells) are traced
//     together, so more lanes share each traced step.
//   * The segment cells of a ray are known without following parent links: the
//     sibling of a cell is its index XOR 1 (children are allocated in pairs) and
//     the common ancestor's depth is the length of the common prefix of the
//     sink's ancestor list and the walk path, kept as a 64-bit mask. Refined
//     children are clipped after the ray's base segments.
// Template options of the warp walk: ADJ (adjoint accumulation, Sec. 2.2 with the
// decisions frozen), MOM (flux vector and pressure moments), BG (background
// sources moved onto a sphere), STOP (early ray termination), NB (several bands)
// and SUB (sub-bucket particle trace).
#include <cuda_runtime.h>
#include <stdint.h>

#include "trevr_internal.cuh"

namespace trevr {

namespace {

constexpr int kDepth = 64;  // > max cell depth (63): lists and stacks never overflow
constexpr int kAnc = 0;     // offsets of the three parts of the per-lane list
constexpr int kPath = kDepth;
constexpr int kRef = 2 * kDepth;
constexpr float kFourPi = 12.566370614359172f;
// refinement stack of the warp walk: refined base segments (at most 2 x 63 + 1) are
// queued first, then each popped pair adds at most one entry per level below
constexpr int kRayStack = 4 * kDepth;
constexpr int kSegBuf = 64;  // segments of one ray kept for the adjoint's second pass

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

// Kahan-compensated fp32 running sum (branch-free), for the optical depth of one
// ray in the warp walks: c carries the low-order part that each addition loses,
// so the error of the sum stays within about 2 ulp of the total however many
// terms a refined ray has.
struct KSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ float get() const { return s; }
};

// one slab of the clip: (lo - p) * (1/d), (hi - p) * (1/d), rounded after each step;
// along an axis the ray does not move on, the box is half-open [lo, hi), so a ray
// lying in the face between two cells belongs to the upper one only
__device__ __forceinline__ void slab(float lo, float hi, float p, float d, float inv, float& t0,
                                     float& t1, bool& miss) {
  if (d != 0.0f) {
    const float ta = __fmul_rn(__fsub_rn(lo, p), inv);
    const float tb = __fmul_rn(__fsub_rn(hi, p), inv);
    t0 = fmaxf(t0, fminf(ta, tb));
    t1 = fminf(t1, fmaxf(ta, tb));
  } else {
    miss = miss || p < lo || p >= hi;
  }
}

// the slab of an axis the ray moves along (d != 0): the same steps as slab()
__device__ __forceinline__ void slab_nz(float lo, float hi, float p, float inv, float& t0,
                                        float& t1) {
  const float ta = __fmul_rn(__fsub_rn(lo, p), inv);
  const float tb = __fmul_rn(__fsub_rn(hi, p), inv);
  t0 = fmaxf(t0, fminf(ta, tb));
  t1 = fminf(t1, fmaxf(ta, tb));
}

__device__ __forceinline__ void slab_g_nz(int k, float lo, float hi, float p, float inv,
                                          float& t0, float& t1, int& k0, int& k1) {
  const float ta = __fmul_rn(__fsub_rn(lo, p), inv);
  const float tb = __fmul_rn(__fsub_rn(hi, p), inv);
  const float tn = fminf(ta, tb), tx = fmaxf(ta, tb);
  if (tn > t0) { t0 = tn; k0 = k; }
  if (tx < t1) { t1 = tx; k1 = k; }
}

// gradient-carrying slab: remembers which axis sets t0 / t1
__device__ __forceinline__ void slab_g(int k, float lo, float hi, float p, float d, float inv,
                                       float& t0, float& t1, int& k0, int& k1, bool& miss) {
  if (d != 0.0f) {
    const float ta = __fmul_rn(__fsub_rn(lo, p), inv);
    const float tb = __fmul_rn(__fsub_rn(hi, p), inv);
    const float tn = fminf(ta, tb), tx = fmaxf(ta, tb);
    if (tn > t0) {
      t0 = tn;
      k0 = k;
    }
    if (tx < t1) {
      t1 = tx;
      k1 = k;
    }
  } else {
    miss = miss || p < lo || p >= hi;
  }
}

}  // namespace

struct SinkCounters {
  int rays = 0, segs = 0, visit = 0, ref = 0, clip = 0, cut = 0, sub = 0;
};

// warp-reduce the counters and add them to the device totals (all lanes call it)
__device__ __forceinline__ void add_stats(const SinkCounters& c, unsigned long long* stats) {
  unsigned long long v[7] = {(unsigned long long)c.rays, (unsigned long long)c.segs,
                             (unsigned long long)c.visit, (unsigned long long)c.ref,
                             (unsigned long long)c.clip, (unsigned long long)c.cut,
                             (unsigned long long)c.sub};
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    unsigned long long x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&stats[q], x);
  }
}

// Per-lane lists, kept apart from the scalar state so that the state stays in
// registers: the ancestors of S | the depth-first path | cells to clip, and the
// walk stack (cell, depth).
struct Lists {
  int lst[3 * kDepth];
  int wstack[kDepth];
  int wdepth[kDepth];
};

// State of one lane: the sink it works on, its walk and its current ray.
// ADJ = false computes the flux. ADJ = true is the adjoint with the same
// decisions: every ray is traced twice, first for tau and d(tau)/dq, then, with
// the contribution f known, to scatter -g f l_X into each segment cell.
template <bool ADJ>
struct Lane {
  // sink
  int i;     // sorted position
  float gk;  // dLoss/dF of this sink (adjoint)
  float px, py, pz;
  int S, dS;
  unsigned long long on_path;  // bit d: path[d] is an ancestor of S
  int sp;                      // walk stack size
  CSum F;
  SinkCounters cnt;  // this sink's counters
  // ray
  bool in_ray;
  float dx, dy, dz, ix, iy, iz, len, s2, rayL;
  CSum tau;
  int C, dC, nSs, nb, b, rsp, boxes;
  // single sources of an opened leaf
  int j, j_end, leafC, dleaf;
  // adjoint
  int pass, src_j;
  float gq0, gq1, gq2, fcur;
  __device__ __forceinline__ void begin(const TreeView& T, int i_, float g, Lists& L_) {
    int* lst = L_.lst;
    int* wstack = L_.wstack;
    int* wdepth = L_.wdepth;
    i = i_;
    gk = g;
    const float4 p = T.pos[i];
    px = p.x;
    py = p.y;
    pz = p.z;
    S = T.leaf_of[i];
    dS = __ldg(&T.ndepth[S]);
    int u = S;
    for (int d = dS; d >= 0; --d) {
      lst[kAnc + d] = u;
      u = __ldg(&T.nT[u].y);
    }
    on_path = 0;
    wstack[0] = kRoot;
    wdepth[0] = 0;
    sp = 1;
    F = CSum();
    cnt = SinkCounters();
    in_ray = false;
    j = j_end = 0;
  }

  // One iteration. Returns false when the sink is finished.
  __device__ __forceinline__ bool step(const TreeView& T, const WalkParams& P, int stack_limit,
                                       int box_limit, int* status, const AdjointArgs& J,
                                       Lists& L_) {
    int* lst = L_.lst;
    int* wstack = L_.wstack;
    int* wdepth = L_.wdepth;
    if (in_ray) {
      const bool from_stack = rsp > 0;
      if (!from_stack && b >= nb) {
        finish_ray(J);
        return true;
      }
      // the next cell, by selects: refinement stack, else S, sink-side siblings,
      // C, pseudo-source-side siblings
      int off = kRef + rsp - 1;
      if (!from_stack) off = (b <= nSs) ? (kAnc + dS - b + 1) : (kPath + dC - (b - nSs - 2));
      const int v = lst[off];
      const int box = from_stack ? v : ((b == 0) ? S : ((b == nSs + 1) ? C : (v ^ 1)));
      rsp -= from_stack ? 1 : 0;
      b += from_stack ? 0 : 1;
      if (++boxes > box_limit) {
        atomicOr(status, kStatusIterationLimit);
        return false;
      }
      const float4 a = __ldg(&T.nA[box]);
      const float4 bb = __ldg(&T.nB[box]);
      const bool want_grad = ADJ && pass == 1 && src_j < 0;
      float t0 = 0.0f, t1 = 1.0f;
      bool miss = false;
      int k0 = -1, k1 = -1;
      if (want_grad) {
        slab_g(0, a.x, bb.x, px, dx, ix, t0, t1, k0, k1, miss);
        slab_g(1, a.y, bb.y, py, dy, iy, t0, t1, k0, k1, miss);
        slab_g(2, a.z, bb.z, pz, dz, iz, t0, t1, k0, k1, miss);
      } else {
        slab(a.x, bb.x, px, dx, ix, t0, t1, miss);
        slab(a.y, bb.y, py, dy, iy, t0, t1, miss);
        slab(a.z, bb.z, pz, dz, iz, t0, t1, miss);
      }
      const float l = (!miss && t1 > t0) ? __fmul_rn(__fsub_rn(t1, t0), len) : 0.0f;
      ++cnt.clip;
      if (!(l > 0.0f)) return true;
      if (P.tau_ref <= 0.0f || __fmul_rn(bb.w, l) > P.tau_ref) {
        const int child = __ldg(&T.nT[box].x);
        if (child >= 0) {
          if (rsp + 2 > stack_limit) {
            atomicOr(status, kStatusStackOverflow);
            return false;
          }
          ++cnt.ref;
          lst[kRef + rsp] = child + 1;
          lst[kRef + rsp + 1] = child;
          rsp += 2;
          return true;
        }
      }
      if (ADJ && pass == 2) {
        atomicAdd(&J.G[box], (double)(-gk * fcur * l));
        return true;
      }
      tau.add(a.w * l);
      if (want_grad) {
        // d l / d q: a slab parameter t = (b - p_k)/d_k moves as -t/d_k along q_k;
        // one clamped to 0 or 1 does not move
        const float w = (t1 - t0) / len;
        const float g0 = (k1 == 0 ? -t1 * ix : 0.0f) + (k0 == 0 ? t0 * ix : 0.0f);
        const float g1 = (k1 == 1 ? -t1 * iy : 0.0f) + (k0 == 1 ? t0 * iy : 0.0f);
        const float g2 = (k1 == 2 ? -t1 * iz : 0.0f) + (k0 == 2 ? t0 * iz : 0.0f);
        gq0 = fmaf(a.w, g0 * len + w * dx, gq0);
        gq1 = fmaf(a.w, g1 * len + w * dy, gq1);
        gq2 = fmaf(a.w, g2 * len + w * dz, gq2);
      }
      ++cnt.segs;
      return true;
    }

    // ---- walk step: find the next pseudo-source
    float qx, qy, qz, L;
    if (j < j_end) {
      const float4 y = __ldg(&T.src[j]);
      ++j;
      if (!(y.w > 0.0f)) return true;
      C = leafC;
      dC = dleaf;
      src_j = j - 1;
      qx = y.x;
      qy = y.y;
      qz = y.z;
      L = y.w;
    } else {
      if (sp == 0) return false;  // the sink is done
      --sp;
      const int X = wstack[sp];
      const int dX = wdepth[sp];
      lst[kPath + dX] = X;
      const unsigned long long bit = 1ull << dX;
      on_path = (dX <= dS && lst[kAnc + dX] == X) ? (on_path | bit) : (on_path & ~bit);
      const float4 s = __ldg(&T.nS[X]);
      if (!(s.w > 0.0f)) return true;
      ++cnt.visit;
      const float4 a = __ldg(&T.nA[X]);
      const float4 bb = __ldg(&T.nB[X]);
      const float ex = fmaxf(fmaxf(__fsub_rn(a.x, px), __fsub_rn(px, bb.x)), 0.0f);
      const float ey = fmaxf(fmaxf(__fsub_rn(a.y, py), __fsub_rn(py, bb.y)), 0.0f);
      const float ez = fmaxf(fmaxf(__fsub_rn(a.z, pz), __fsub_rn(pz, bb.z)), 0.0f);
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
            return false;
          }
          wstack[sp] = t.x + 1;
          wdepth[sp] = dX + 1;
          wstack[sp + 1] = t.x;
          wdepth[sp + 1] = dX + 1;
          sp += 2;
        }
        return true;
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
    dx = __fsub_rn(qx, px);
    dy = __fsub_rn(qy, py);
    dz = __fsub_rn(qz, pz);
    s2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (s2 < P.smin2) return true;  // a source on top of the sink adds nothing
    len = __fsqrt_rn(s2);
    ix = dx != 0.0f ? __frcp_rn(dx) : 0.0f;
    iy = dy != 0.0f ? __frcp_rn(dy) : 0.0f;
    iz = dz != 0.0f ? __frcp_rn(dz) : 0.0f;
    rayL = L;
    tau = CSum();
    pass = 1;
    gq0 = gq1 = gq2 = 0.0f;
    b = 0;
    rsp = 0;
    boxes = 0;
    if (C == S) {
      nSs = 0;
      nb = 1;
    } else {
      // depth of the lowest common ancestor: the common prefix of path and anc
      const int mn = dC < dS ? dC : dS;
      const unsigned long long m = on_path & ((2ull << mn) - 1ull);  // mn <= 62
      const int dstar = __ffsll((long long)~m) - 2;
      nSs = dS - dstar - 1;  // siblings on the sink side
      nb = dS + dC - 2 * dstar;
    }
    in_ray = true;
    return true;
  }

  __device__ __forceinline__ void finish_ray(const AdjointArgs& J) {
    const float t = tau.get();
    const float f = rayL * expf(-t) / (kFourPi * s2);
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
        atomicAdd(&J.b[3 * C + 0], (double)(c * (-dx * inv_s2 - gq0)));
        atomicAdd(&J.b[3 * C + 1], (double)(c * (-dy * inv_s2 - gq1)));
        atomicAdd(&J.b[3 * C + 2], (double)(c * (-dz * inv_s2 - gq2)));
      }
      ++cnt.rays;
      in_ray = false;
    }
  }
};

// Where a finished sink's results go.
struct SinkOut {
  float* flux;    // flux per sink (caller order), or nullptr
  int* counters;  // 4 int per sink, or nullptr
  float* fvec;    // flux vector, 3 x n_sink (SoA), or nullptr
  float* press;   // second moment, 6 x n_sink (SoA: xx yy zz xy xz yz), or nullptr
  int n_out;      // n_sink (stride of the SoA blocks)
};

// Direction moments of the intensity at one sink: sum f n and sum f n n^T, n the
// unit vector from the pseudo-source to the sink (Eq. simpflux; Sec. 2.1).
struct Moments {
  CSum v[9];  // x y z | xx yy zz xy xz yz
};

// Runs the sinks [first, end) of a chunk with one warp: the lanes start on the
// first 32 and take the next unclaimed sink of the chunk when theirs is done.
// `map` turns a chunk position into (sorted position, output slot, dLoss/dF);
// positions it rejects are skipped. Every lane of the warp must call it.
template <bool ADJ, class Map>
__device__ __forceinline__ void run_chunk(const TreeView& T, const WalkParams& P, int first,
                                          int end, const Map& map, const SinkOut& out,
                                          int* status, const AdjointArgs& J, SinkCounters& tot) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  const int stack_limit = P.stack_depth < kDepth ? P.stack_depth : kDepth;
  const int box_limit = 2 * T.n_nodes_cap + 4;
  Lane<ADJ> st;
  Lists lists;
  int next = first;     // next unclaimed chunk position (same value in every lane)
  bool active = false;  // this lane holds a sink
  int slot = -1;        // output slot of the lane's sink
  while (true) {
    // idle lanes claim the next positions of the chunk, in lane order
    const unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (idle) {
      if (next >= end) {
        if (idle == 0xffffffffu) break;
      } else {
        const int pos = next + (int)__popc(idle & lt);
        if (!active && pos < end) {
          int i;
          float g;
          if (map(pos, i, slot, g)) {
            st.begin(T, i, g, lists);
            active = true;
          }
        }
        next += (int)__popc(idle);
        continue;  // a lane whose position was rejected claims again next round
      }
    }
    if (active && !st.step(T, P, stack_limit, box_limit, status, J, lists)) {
      active = false;
      if (!ADJ) {
        if (out.flux) out.flux[slot] = st.F.get();
        if (out.counters)
          reinterpret_cast<int4*>(out.counters)[slot] =
              make_int4(st.cnt.rays, st.cnt.segs, st.cnt.visit, st.cnt.ref);
      }
      tot.rays += st.cnt.rays;
      tot.segs += st.cnt.segs;
      tot.visit += st.cnt.visit;
      tot.ref += st.cnt.ref;
      tot.clip += st.cnt.clip;
    }
  }
}

// Sinks of a plain call: chunk position k is the k-th requested sink.
template <bool ADJ>
struct PlainMap {
  const TreeView* T;
  const long long* sink_idx;
  const float* grad_flux;
  int* status;
  __device__ __forceinline__ bool operator()(int k, int& i, int& slot, float& g) const {
    if (sink_idx) {
      const long long si = sink_idx[k];
      if (si < 0 || si >= T->n_gas) {
        atomicOr(status, kStatusInvalid);
        return false;
      }
      i = T->rank[si];
      slot = k;
    } else {
      i = k;
      slot = T->perm[k];
    }
    g = ADJ ? grad_flux[slot] : 0.0f;
    return !ADJ || g != 0.0f;  // the adjoint skips sinks with dLoss/dF = 0
  }
};

template <bool ADJ>
__global__ void __launch_bounds__(128) walk_kernel(TreeView T, const long long* sink_idx,
                                                   int n_sink, int chunk, WalkParams P,
                                                   SinkOut out, unsigned long long* stats,
                                                   int* status, AdjointArgs J) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long first = warp * chunk;
  SinkCounters tot;
  if (first < n_sink) {
    const int end = (int)min((long long)n_sink, first + chunk);
    if (!ADJ && sink_idx) {  // sinks with an index out of range get zeros
      for (int k = (int)first + (int)(threadIdx.x & 31); k < end; k += 32) {
        const long long si = sink_idx[k];
        if (si < 0 || si >= T.n_gas) {
          if (out.flux) out.flux[k] = 0.0f;
          if (out.counters) reinterpret_cast<int4*>(out.counters)[k] = make_int4(0, 0, 0, 0);
        }
      }
    }
    PlainMap<ADJ> map{&T, sink_idx, J.grad_flux, status};
    run_chunk<ADJ>(T, P, (int)first, end, map, out, status, J, tot);
  }
  if (stats) add_stats(tot, stats);
}

// Batched form: sorted positions of one tree, output in that tree's caller order.
struct TreeMap {
  const TreeView* T;
  __device__ __forceinline__ bool operator()(int k, int& i, int& slot, float& g) const {
    i = k;
    slot = T->perm[k];
    g = 0.0f;
    return true;
  }
};

// Many independent trees in one persistent launch. Work items are runs of
// `item` consecutive sinks (Morton order) of one tree; each warp takes the next
// item from a device counter, so warps that finish early keep pulling work from
// the boxes that are left. Per-sink arithmetic is the same as walk_kernel.
template <int BS>
__global__ void __launch_bounds__(BS) walk_batched_kernel(const TreeView* __restrict__ views,
                                                         float* const* __restrict__ flux_out,
                                                         const int2* __restrict__ items,
                                                         int n_items, int item,
                                                         unsigned* counter, WalkParams P,
                                                         unsigned long long* stats, int* status) {
  const unsigned lane = threadIdx.x & 31u;
  SinkCounters tot;
  while (true) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)n_items) break;
    const int2 w = items[it];
    const TreeView T = views[w.x];
    WalkParams Pt = P;  // the coincident-source cut (1e-12 side)^2 of this tree, in fp32
    const float smin = __fmul_rn(1e-12f, T.side);
    Pt.smin2 = __fmul_rn(smin, smin);
    SinkOut out{flux_out[w.x], nullptr, nullptr, nullptr, 0};
    TreeMap map{&T};
    run_chunk<false>(T, Pt, w.y, min(w.y + item, T.n_gas), map, out, status, AdjointArgs{}, tot);
  }
  if (stats) add_stats(tot, stats);
}

// ---------------------------------------------------------------------------
// Warp-shared walk (variant 2). The 32 lanes of a warp (32 consecutive sinks in
// Morton order) walk ONE depth-first stack held in shared memory; each entry
// carries the mask of lanes that still need the cell. A cell that several
// lanes accept is traced by all of them at once, to the same pseudo-source, so
// the cells on the pseudo-source's side and the shared part of the sinks' side
// are the same addresses in every lane (one broadcast load). The segment order
// is chosen for that: C, then C's side from deep to shallow, then the sink's
// side from shallow to deep, then S.
// ---------------------------------------------------------------------------
struct WarpStack {
  int node[kDepth + 2];
  int depth[kDepth + 2];
  unsigned mask[kDepth + 2];
  int path[kDepth];  // the walk's depth-first path
};

// Sum of v over the lanes that asked (key >= 0) when they all name the same cell,
// else one atomic per lane. Every lane of the warp must call it.
__device__ __forceinline__ void warp_atomic_add(double* base, int key, float v) {
  const unsigned FULL = 0xffffffffu;
  const unsigned want = __ballot_sync(FULL, key >= 0);
  if (!want) return;
  const int k0 = __shfl_sync(FULL, key, __ffs(want) - 1);
  if (__all_sync(FULL, key < 0 || key == k0)) {
    float x = key >= 0 ? v : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&base[k0], (double)x);
  } else if (key >= 0) {
    atomicAdd(&base[key], (double)v);
  }
}

// ---------------------------------------------------------------------------
// Sub-bucket particle trace (Sec. 2.2.3, 3.1.3). The absorption below the bucket
// scale is the SPH field sum_j alpha_j w_j W(|x - x_j|, h_j), W(r, h) = w(r/h)/(pi h^3)
// the cubic spline of support 2h. Along a ray at impact parameter b from x_j, with s
// measured from the closest approach, the column over [s0, s1] is
// (Phi(x, s1/h) - Phi(x, s0/h)) / (pi h^2), x = b^2/h^2, where Phi(x, sigma) is the
// integral of w(sqrt(x + t^2)) over t in [0, sigma]: odd in sigma and constant beyond
// the support. Phi comes from the tree's pre-computed table (the paper's pre-computed
// kernel integral), bilinear in (x, sigma).
__device__ __forceinline__ float kint_phi(const float4* __restrict__ tab, float x, float sigma) {
  const float a = fminf(fabsf(sigma), 2.0f);
  const float fx = x * (0.25f * (float)kKintNX), fs = a * (0.5f * (float)kKintNS);
  const int i = min((int)fx, kKintNX - 1), j = min((int)fs, kKintNS - 1);
  const float u = fx - (float)i, v = fs - (float)j;
  const float4 c = __ldg(tab + (size_t)i * kKintNS + j);  // the cell's four corners
  const float p0 = fmaf(v, c.y - c.x, c.x);
  const float p1 = fmaf(v, c.w - c.z, c.z);
  const float p = fmaf(u, p1 - p0, p0);
  return sigma < 0.0f ? -p : p;
}

// Per-warp queue of the neighbours whose support meets the chord, so that the
// quadrature runs on full warps: (x, sigma_0, sigma_1, alpha w / (pi h^2)).
struct SubQueue {
  float4 g[64];
};

// Optical depth of lane src's chord p + t d, t in [t0, t1], through the particles
// listed for its leaf, the receiving particle (sorted index si) left out. The 32
// lanes of the warp test one neighbour each per round, with the next round's
// entries already loading; the neighbours that reach the chord are queued in shared
// memory and integrated 32 at a time: (Phi(x, sigma_1) - Phi(x, sigma_0)) times
// alpha w / (pi h^2), with x = b^2 / h^2 and sigma = s / h. Every lane must call it;
// all lanes return the sum.
__device__ __forceinline__ float sub_bucket_tau_warp(const TreeView& T, int src, int box, int si,
                                                     float px, float py, float pz, float dx,
                                                     float dy, float dz, float s2, float len,
                                                     float t0, float t1) {
  const unsigned FULL = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  __shared__ SubQueue queues[4];  // one per warp of a 128-thread block
  SubQueue& Q = queues[threadIdx.x >> 5];
  box = __shfl_sync(FULL, box, src);
  si = __shfl_sync(FULL, si, src);
  px = __shfl_sync(FULL, px, src);
  py = __shfl_sync(FULL, py, src);
  pz = __shfl_sync(FULL, pz, src);
  dx = __shfl_sync(FULL, dx, src);
  dy = __shfl_sync(FULL, dy, src);
  dz = __shfl_sync(FULL, dz, src);
  s2 = __shfl_sync(FULL, s2, src);
  len = __shfl_sync(FULL, len, src);
  t0 = __shfl_sync(FULL, t0, src);
  t1 = __shfl_sync(FULL, t1, src);
  const float inv_s2 = 1.0f / s2;
  float part = 0.0f;
  int qn = 0;  // queued entries (warp-uniform)
  const unsigned k0 = __ldg(&T.nbr_first[box]), k1 = __ldg(&T.nbr_first[box + 1]);
  int2 nja = make_int2(-1, 0);  // the next round's entries
  float4 nq = make_float4(0.0f, 0.0f, 0.0f, 1.0f);
  if (k0 + lane < k1) {
    nja = __ldg(&T.nbr_ja[k0 + lane]);
    nq = __ldg(&T.nbr_sp[k0 + lane]);
  }
  for (unsigned base = k0; base < k1; base += 32u) {
    const unsigned k = base + lane;
    const int2 ja = nja;
    const float4 q = nq;
    if (k + 32u < k1) {
      nja = __ldg(&T.nbr_ja[k + 32u]);
      nq = __ldg(&T.nbr_sp[k + 32u]);
    }
    const float a = __int_as_float(ja.y);
    bool pass = false;
    float x = 0.0f, sa = 0.0f, sb = 0.0f;
    if (k < k1 && ja.x != si && a > 0.0f) {
      const float ux = q.x - px, uy = q.y - py, uz = q.z - pz;
      const float tc = (ux * dx + uy * dy + uz * dz) * inv_s2;
      const float ex = ux - tc * dx, ey = uy - tc * dy, ez = uz - tc * dz;
      const float b2 = ex * ex + ey * ey + ez * ez;
      const float ih = q.w;
      x = b2 * ih * ih;
      sa = ((t0 - tc) * len) * ih;
      sb = ((t1 - tc) * len) * ih;
      if (x < 4.0f) {  // the chord [sa, sb] must meet the support |sigma| < sqrt(4 - x)
        const float u22 = 4.0f - x;
        pass = (sb > 0.0f || sb * sb < u22) && (sa < 0.0f || sa * sa < u22);
      }
    }
    const unsigned m = __ballot_sync(FULL, pass);
    if (pass) {
      const float ih = q.w;
      Q.g[qn + __popc(m & ((1u << lane) - 1u))] =
          make_float4(x, sa, sb, a * (ih * ih * 0.318309886f));
    }
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {
      const float4 g = Q.g[qn - 32 + (int)lane];
      part += g.w * (kint_phi(T.kint4, g.x, g.z) - kint_phi(T.kint4, g.x, g.y));
      qn -= 32;
      __syncwarp();
    }
  }
  if ((int)lane < qn) {
    const float4 g = Q.g[lane];
    part += g.w * (kint_phi(T.kint4, g.x, g.z) - kint_phi(T.kint4, g.x, g.y));
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(FULL, part, o);
  return part;
}

// Rays from the sinks of the lanes in `on` to (q, L) inside cell C; every lane
// of the warp must call it (the loop runs while any lane has cells left).
// STOP: early ray termination (Sec. 4): a lane whose running optical depth passes
// P.tau_stop drops the rest of its ray, and the ray adds nothing.
// NB > 1: several bands (2 or 4 slots of the band records): every band sums its own
// optical depth over the shared segments, and F[b] gets band b's flux.
// SUB: the sub-bucket particle trace for leaves whose own particles ask for
// refinement (the sink's sorted index si is left out of the sum).
// TD: the top-down ray walk (Sec. 3.1.3, Sec. 4): the ray's only base segment is the
// common ancestor A = path[d*], and Eq. refcrit alone splits it through the same
// refinement stack; without TD the base segments are C, the siblings up both paths
// and S, as in the paper's walk.
template <bool ADJ, bool MOM, bool STOP = false, int NB = 1, bool SUB = false, bool CNT = true,
          bool TD = false>
__device__ __forceinline__ void warp_ray(const TreeView& T, const WalkParams& P, const bool on,
                                         const float px, const float py, const float pz,
                                         const int S, const int dS, const int* anc, int* rst,
                                         const unsigned long long on_path, const int* path,
                                         const int C, const int dC, const float qx,
                                         const float qy, const float qz, const float L,
                                         const int src_j, const float gk, const int stack_limit,
                                         const int box_limit, int* status, const AdjointArgs& J,
                                         SinkCounters& cnt, CSum* F, Moments* mom,
                                         const int si = -1) {
  static_assert(NB == 1 || NB == 2 || NB == 4, "band slots: 1, 2 or 4");
  static_assert(!SUB || (!ADJ && !MOM && !STOP && NB == 1), "sub-bucket trace: plain flux only");
  static_assert(NB == 1 || !(ADJ || MOM || STOP), "bands: plain flux only");
  const unsigned FULL = 0xffffffffu;
  float dx = 0.0f, dy = 0.0f, dz = 0.0f, s2 = 1.0f, len = 1.0f, ix = 0.0f, iy = 0.0f, iz = 0.0f;
  int nCs = 0, nSs = 0, nb = 0, dstar = 0;
  int base1 = S;  // the base segment of a one-segment ray: S, or A for the top-down walk
  bool active = false;
  if (on) {
    dx = __fsub_rn(qx, px);
    dy = __fsub_rn(qy, py);
    dz = __fsub_rn(qz, pz);
    s2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    if (!(s2 < P.smin2)) {  // a source on top of the sink adds nothing
      active = true;
      len = __fsqrt_rn(s2);
      ix = dx != 0.0f ? __frcp_rn(dx) : 0.0f;
      iy = dy != 0.0f ? __frcp_rn(dy) : 0.0f;
      iz = dz != 0.0f ? __frcp_rn(dz) : 0.0f;
      if (C == S) {
        nb = 1;
      } else {
        const int mn = dC < dS ? dC : dS;
        const unsigned long long m = on_path & ((2ull << mn) - 1ull);  // mn <= 62
        dstar = __ffsll((long long)~m) - 2;
        if (TD) {
          nb = 1;
          base1 = path[dstar];
        } else {
          nCs = dC - dstar - 1;
          nSs = dS - dstar - 1;
          nb = nCs + nSs + 2;
        }
      }
    }
  }
  const bool traced = active;
  const bool nz = dx != 0.0f && dy != 0.0f && dz != 0.0f;  // the ray moves along every axis
  KSum tau;
  KSum taub[NB];  // (NB > 1) optical depth of each band
  bool cut = false;
  int b = 0, rsp = 0, boxes = 0, pass = 1;
  int slot = -1;  // the upper child of the pair popped last: clipped next
  // adjoint: the first pass records its segment cells and lengths (up to kSegBuf),
  // so the second pass replays them instead of tracing the ray again
  int segb[ADJ ? kSegBuf : 1];
  float segl[ADJ ? kSegBuf : 1];
  int nseg = 0, kk = 0;
  bool seg_over = false;
  float gq0 = 0.0f, gq1 = 0.0f, gq2 = 0.0f, fcur = 0.0f;
  bool need_sub = false;  // (SUB) this step's leaf is traced through its particles
  int sub_box = 0;
  float sub_t0 = 0.0f, sub_t1 = 0.0f;
  while (__any_sync(FULL, active)) {
    int akey = -1;
    float aval = 0.0f;
    if (ADJ && active && pass == 3) {
      if (kk < nseg) {
        // four recorded segments per iteration: 2.2 % faster backward than one
        // (145.5 against 148.8 ms at 2^21), eight were slower (154 ms)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (kk + u < nseg) atomicAdd(&J.G[segb[kk + u]], (double)(-gk * fcur * segl[kk + u]));
        kk += 4;
      } else {
        if (CNT) ++cnt.rays;
        active = false;
      }
    } else if (active) {
      const bool from_stack = b >= nb && (rsp > 0 || slot >= 0);  // base segments first
      if (!from_stack && b >= nb) {
        const float f = L * expf(-tau.get()) / (kFourPi * s2);
        if (!ADJ && STOP && cut) {
          if (CNT) ++cnt.cut;
          if (CNT) ++cnt.rays;
          active = false;
        } else if (!ADJ) {
          if (NB > 1) {
            // the band luminosities of the source, or of the merged cell C
            const float4 Lb = src_j >= 0 ? __ldg(&T.bLs[src_j]) : __ldg(&T.bLc[C]);
            F[0].add(Lb.x * expf(-taub[0].get()) / (kFourPi * s2));
            F[1].add(Lb.y * expf(-taub[1].get()) / (kFourPi * s2));
            if (NB > 2) {
              F[NB > 2 ? 2 : 0].add(Lb.z * expf(-taub[NB > 2 ? 2 : 0].get()) / (kFourPi * s2));
              F[NB > 2 ? 3 : 0].add(Lb.w * expf(-taub[NB > 2 ? 3 : 0].get()) / (kFourPi * s2));
            }
          } else {
            F[0].add(f);
          }
          if (MOM) {
            const float il = 1.0f / len;
            const float n0 = -dx * il, n1 = -dy * il, n2 = -dz * il;
            mom->v[0].add(f * n0);
            mom->v[1].add(f * n1);
            mom->v[2].add(f * n2);
            mom->v[3].add(f * n0 * n0);
            mom->v[4].add(f * n1 * n1);
            mom->v[5].add(f * n2 * n2);
            mom->v[6].add(f * n0 * n1);
            mom->v[7].add(f * n0 * n2);
            mom->v[8].add(f * n1 * n2);
          }
          if (CNT) ++cnt.rays;
          active = false;
        } else if (pass == 1) {
          fcur = f;  // second pass over the same cells, now that f is known
          if (!seg_over) {
            pass = 3;  // replay the recorded segments
            kk = 0;
          } else {
            pass = 2;  // too many segments to record: trace the ray again
            b = 0;
            rsp = 0;
            slot = -1;
            boxes = 0;
          }
        } else {
          if (CNT) ++cnt.rays;
          active = false;
        }
      } else {
        int box;
        if (from_stack) {
          if (slot >= 0) {
            box = slot;
            slot = -1;
          } else {
            // a refined cell's pair of children (clip the lower, keep the upper), or
            // the one child the ray crosses
            const int e = rst[--rsp];
            if (e < 0) {
              box = ~e;
              slot = box + 1;
            } else {
              box = e;
            }
          }
        } else {
          if (nb == 1) {
            box = base1;
          } else if (b <= nCs) {  // C = path[dC], then the siblings up C's path
            box = path[dC - max(b - 1, 0)] ^ (b > 0 ? 1 : 0);
          } else {  // the siblings down S's path, then S = anc[dS]
            const int j = b - nCs;
            box = anc[dstar + 1 + min(j, nSs)] ^ (j <= nSs ? 1 : 0);
          }
          ++b;
        }
        // Each iteration clips one base segment or one child of a pushed pair, and the
        // pushes are capped by box_limit below, so a ray ends after at most
        // nb + 2 box_limit iterations (the walk's hang guard).
        {
          const float4 a = __ldg(&T.nA[box]);
          const float4 bb = __ldg(&T.nB[box]);
          const bool want_grad = ADJ && pass == 1 && src_j < 0;
          float t0 = 0.0f, t1 = 1.0f;
          bool miss = false;
          int k0 = -1, k1 = -1;
          if (want_grad && nz) {
            slab_g_nz(0, a.x, bb.x, px, ix, t0, t1, k0, k1);
            slab_g_nz(1, a.y, bb.y, py, iy, t0, t1, k0, k1);
            slab_g_nz(2, a.z, bb.z, pz, iz, t0, t1, k0, k1);
          } else if (want_grad) {
            slab_g(0, a.x, bb.x, px, dx, ix, t0, t1, k0, k1, miss);
            slab_g(1, a.y, bb.y, py, dy, iy, t0, t1, k0, k1, miss);
            slab_g(2, a.z, bb.z, pz, dz, iz, t0, t1, k0, k1, miss);
          } else if (nz) {  // no axis along which the ray stays still: no face tests
            slab_nz(a.x, bb.x, px, ix, t0, t1);
            slab_nz(a.y, bb.y, py, iy, t0, t1);
            slab_nz(a.z, bb.z, pz, iz, t0, t1);
          } else {
            slab(a.x, bb.x, px, dx, ix, t0, t1, miss);
            slab(a.y, bb.y, py, dy, iy, t0, t1, miss);
            slab(a.z, bb.z, pz, dz, iz, t0, t1, miss);
          }
          const float l = (!miss && t1 > t0) ? __fmul_rn(__fsub_rn(t1, t0), len) : 0.0f;
          if (CNT) ++cnt.clip;
          if (l > 0.0f) {
            bool pushed = false;
            if (P.tau_ref <= 0.0f || __fmul_rn(bb.w, l) > P.tau_ref) {
              const int child = __ldg(&T.nT[box].x);
              if (child >= 0) {
                if (rsp + 1 > kRayStack) {
                  atomicOr(status, kStatusStackOverflow);
                  active = false;
                } else if (++boxes > box_limit) {
                  atomicOr(status, kStatusIterationLimit);
                  active = false;
                } else {
                  if (CNT) ++cnt.ref;
                  // The children's intervals are this cell's cut at the split plane,
                  // whose t is the one their clips would compute ((P - p) * (1/d),
                  // with min / max exact), so a child the ray misses is not queued
                  // (22 % fewer clips on the clumpy workload, bit-identical fluxes).
                  bool lo_t = true, hi_t = true;
                  {
                    const float2 sp = __ldg(&T.nSP[box]);
                    const int ax = __float_as_int(sp.y);
                    const float Pl = sp.x;
                    const float pa = ax == 0 ? px : (ax == 1 ? py : pz);
                    const float ia = ax == 0 ? ix : (ax == 1 ? iy : iz);
                    if (ia != 0.0f) {
                      const float tP = __fmul_rn(__fsub_rn(Pl, pa), ia);
                      const bool fwd = ia > 0.0f;
                      lo_t = fwd ? tP > t0 : tP < t1;
                      hi_t = fwd ? tP < t1 : tP > t0;
                    } else {  // the ray lies in a plane of this axis: half-open children
                      lo_t = pa < Pl;
                      hi_t = !lo_t;
                    }
                  }
                  // both children, clipped after the base segments, or the crossed one
                  rst[rsp++] = lo_t && hi_t ? ~child : (lo_t ? child : child + 1);
                }
                pushed = true;
              }
            }
            if (!pushed) {
              if (ADJ && pass == 2) {
                akey = box;
                aval = -gk * fcur * l;
              } else {
                if (NB > 1) {
                  const float4 ab = __ldg(&T.bA[box]);
                  taub[0].add(__fmul_rn(ab.x, l));
                  taub[1].add(__fmul_rn(ab.y, l));
                  if (NB > 2) {
                    taub[NB > 2 ? 2 : 0].add(__fmul_rn(ab.z, l));
                    taub[NB > 2 ? 3 : 0].add(__fmul_rn(ab.w, l));
                  }
                } else if (SUB && (P.tau_ref <= 0.0f ||
                                   __fmul_rn(__ldg(&T.dbk[box]), l) > P.tau_ref)) {
                  // a bucket that still asks for refinement: its particles are traced
                  // by the whole warp at the end of this step
                  need_sub = true;
                  sub_box = box;
                  sub_t0 = t0;
                  sub_t1 = t1;
                  if (CNT) ++cnt.sub;
                } else {
                  tau.add(__fmul_rn(a.w, l));
                }
                if (!ADJ && STOP && tau.get() > P.tau_stop) {
                  cut = true;  // the rest of the ray is not traced
                  b = nb;
                  rsp = 0;
                  slot = -1;
                }
                if (ADJ) {
                  if (nseg < kSegBuf) {
                    segb[nseg] = box;
                    segl[nseg] = l;
                    ++nseg;
                  } else {
                    seg_over = true;
                  }
                }
                if (want_grad) {
                  const float w = (t1 - t0) / len;
                  const float g0 = (k1 == 0 ? -t1 * ix : 0.0f) + (k0 == 0 ? t0 * ix : 0.0f);
                  const float g1 = (k1 == 1 ? -t1 * iy : 0.0f) + (k0 == 1 ? t0 * iy : 0.0f);
                  const float g2 = (k1 == 2 ? -t1 * iz : 0.0f) + (k0 == 2 ? t0 * iz : 0.0f);
                  gq0 = fmaf(a.w, g0 * len + w * dx, gq0);
                  gq1 = fmaf(a.w, g1 * len + w * dy, gq1);
                  gq2 = fmaf(a.w, g2 * len + w * dz, gq2);
                }
                if (CNT) ++cnt.segs;
              }
            }
          }
        }
      }
    }
    if (SUB) {
      // the leaves of this step that need the particle trace, one after another
      unsigned m = __ballot_sync(FULL, need_sub);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1u;
        const float t = sub_bucket_tau_warp(T, src, sub_box, si, px, py, pz, dx, dy, dz, s2, len,
                                            sub_t0, sub_t1);
        if ((int)(threadIdx.x & 31u) == src) tau.add(t);
      }
      need_sub = false;
    }
    // a retraced segment's gradient (a ray with more segments than were recorded): the
    // lanes trace different rays, so the cells differ and each lane adds its own, as the
    // replay does (1.4 % faster than trying a warp-wide sum first)
    if (ADJ && akey >= 0) atomicAdd(&J.G[akey], (double)aval);
  }
  if (ADJ) {
    // the pseudo-source's terms. The lanes of one call may mix single sources and
    // merged cells (merged pending rays), so every lane takes part in every
    // warp-wide sum, naming no key (-1) for a term that is not its own.
    const bool single = traced && src_j >= 0, merged = traced && src_j < 0;
    const float gf = traced ? gk * fcur : 0.0f;
    const float c = traced ? gf / L : 0.0f, inv_s2 = 2.0f / s2;
    warp_atomic_add(J.e, single ? src_j : -1, c);
    warp_atomic_add(J.a, merged ? C : -1, c);
    warp_atomic_add(J.b + 0, merged ? 3 * C : -1, c * (-dx * inv_s2 - gq0));
    warp_atomic_add(J.b + 1, merged ? 3 * C : -1, c * (-dy * inv_s2 - gq1));
    warp_atomic_add(J.b + 2, merged ? 3 * C : -1, c * (-dz * inv_s2 - gq2));
  }
}

// Background sources (Sec. 2.2.4): the centre of luminosity c (s.xyz) of an accepted
// cell moved radially onto the sphere of radius P.bg_radius around the domain centre
// o (side / 2 in coordinates relative to the lower corner), in fp32 as d = c - o,
// s = sqrt((dx^2 + dy^2) + dz^2), q = o + d * (R / s); and the leaf Y holding q (grid
// coordinates clamped to the grid), found by descending the cut planes from the root,
// with its ancestors cpath[0 .. dY].
__device__ __forceinline__ void bg_move(const TreeView& T, const WalkParams& P, const float4 s,
                                        float& qx, float& qy, float& qz, int& Y, int& dY,
                                        int* cpath) {
  const float ox = __fmul_rn(T.side, 0.5f), oy = ox, oz = ox;
  const float ddx = __fsub_rn(s.x, ox), ddy = __fsub_rn(s.y, oy), ddz = __fsub_rn(s.z, oz);
  const float sn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy)),
                                        __fmul_rn(ddz, ddz)));
  if (sn > 0.0f) {
    const float kk = __fdiv_rn(P.bg_radius, sn);
    qx = __fadd_rn(ox, __fmul_rn(ddx, kk));
    qy = __fadd_rn(oy, __fmul_rn(ddy, kk));
    qz = __fadd_rn(oz, __fmul_rn(ddz, kk));
  }
  const float scale = __fdiv_rn(2097152.0f, T.side);
  const float q[3] = {qx, qy, qz};
  int g[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float t = __fmul_rn(q[d], scale);
    if (!(t >= 0.0f)) t = 0.0f;
    const unsigned v = __float2uint_rz(t);
    g[d] = (int)(v > (unsigned)(kGridMax - 1) ? (unsigned)(kGridMax - 1) : v);
  }
  Y = kRoot;
  dY = 0;
  cpath[0] = kRoot;
  for (int it = 0; it < kDepth - 1; ++it) {
    const int ch = __ldg(&T.nT[Y].x);
    if (ch < 0) break;
    const int ax = __ldg(&T.nglo[Y].w);
    const int4 up = __ldg(&T.nglo[ch + 1]);
    const int plane = ax == 0 ? up.x : (ax == 1 ? up.y : up.z);
    Y = g[ax] >= plane ? ch + 1 : ch;
    cpath[++dY] = Y;
  }
}

// The hot path for the 32 sinks of one warp (lane holds sorted position i if
// `has`); every lane of the warp must call it. Accumulates the lane's flux in F.
// MERGE = true: a lane that accepts a cell (or reaches a single source) does not
// trace the ray at once; it keeps it pending, and the pending rays of all lanes are
// traced together (each lane to its own cell) when a lane needs its slot again or
// when the walk is about to overwrite the part of the path a pending ray uses. More
// lanes then share each traced batch; every lane still gets the same rays.
// BG = true (with MERGE): background sources (Sec. 2.2.4). A merged cell's centre of
// luminosity c is moved radially onto the sphere of radius R around the domain centre
// o before its ray is traced, in fp32 as d = c - o, s = sqrt((dx^2 + dy^2) + dz^2),
// q = o + d * (R / s); the ray then ends in the leaf that holds q, whose ancestors the
// lane finds by descending the cut planes from the root and keeps for that ray.
template <bool ADJ, bool MERGE, bool MOM = false, bool BG = false, bool STOP = false, int NB = 1,
          bool SUB = false, bool CNT = true, bool TD = false>
__device__ __forceinline__ void warp_walk(const TreeView& T, const WalkParams& P, const bool has,
                                          const int i, const float gk, WarpStack& ws,
                                          int* status, const AdjointArgs& J,
                                          SinkCounters& cnt, CSum* F, Moments* mom = nullptr) {
  const unsigned FULL = 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  const int stack_limit = P.stack_depth < kDepth ? P.stack_depth : kDepth;
  const int box_limit = 2 * T.n_nodes_cap + 4;
  int anc[kDepth];     // ancestors of S by depth
  int rst[kRayStack];  // this lane's cells waiting to be clipped (refinement)
  float px = 0.0f, py = 0.0f, pz = 0.0f;
  int S = 0, dS = 0;
  if (has) {
    const float4 p = T.pos[i];
    px = p.x;
    py = p.y;
    pz = p.z;
    S = T.leaf_of[i];
    dS = __ldg(&T.ndepth[S]);
    int u = S;
    for (int d = dS; d >= 0; --d) {
      anc[d] = u;
      u = __ldg(&T.nT[u].y);
    }
  }
  unsigned long long on_path = 0;
  const unsigned live = __ballot_sync(FULL, has);
  if (lane == 0) {
    ws.node[0] = kRoot;
    ws.depth[0] = 0;
    ws.mask[0] = live;
  }
  int sp = live ? 1 : 0;
  // this lane's pending ray (MERGE)
  bool pnd = false;
  bool pbg = false;          // (BG) the pending ray ends at a moved source: path in cpath
  int cpath[BG ? kDepth : 1] = {};  // (BG) ancestors of the leaf holding the moved source
  int pC = 0, pdC = 0, psrc = -1;
  float pqx = 0.0f, pqy = 0.0f, pqz = 0.0f, pL = 0.0f;
  auto flush = [&]() {
    if (BG) {
      // a ray to a moved source uses its own path: the common-prefix mask of that
      // path and the sink's ancestors
      unsigned long long onp = on_path;
      const int* pp = ws.path;
      if (pnd && pbg) {
        onp = 0;
        const int mn = pdC < dS ? pdC : dS;
        for (int d = 0; d <= mn && cpath[d] == anc[d]; ++d) onp |= 1ull << d;
        pp = cpath;
      }
      warp_ray<ADJ, MOM, STOP, NB, SUB, CNT, TD>(T, P, pnd, px, py, pz, S, dS, anc, rst, onp, pp, pC, pdC, pqx, pqy,
                         pqz, pL, psrc, gk, stack_limit, box_limit, status, J, cnt, F, mom,
                         i);
    } else {
      warp_ray<ADJ, MOM, STOP, NB, SUB, CNT, TD>(T, P, pnd, px, py, pz, S, dS, anc, rst, on_path, ws.path, pC, pdC,
                         pqx, pqy, pqz, pL, psrc, gk, stack_limit, box_limit, status, J, cnt, F,
                         mom, i);
    }
    pnd = false;
    pbg = false;
  };
  __syncwarp();
  while (sp > 0) {
    --sp;
    const int X = ws.node[sp], dX = ws.depth[sp];
    const unsigned M = ws.mask[sp];
    __syncwarp();
    // a pending ray reads the path up to its cell's depth: trace it before that changes
    if (MERGE && __any_sync(FULL, pnd && !pbg && pdC >= dX)) flush();
    if (lane == 0) ws.path[dX] = X;
    const unsigned long long bit = 1ull << dX;
    if (has) on_path = (dX <= dS && anc[dX] == X) ? (on_path | bit) : (on_path & ~bit);
    __syncwarp();
    const float4 s = __ldg(&T.nS[X]);
    if (!(s.w > 0.0f)) continue;
    bool acc = false, opn = false;
    if ((M >> lane) & 1u) {
      if (CNT) ++cnt.visit;
      const float4 a = __ldg(&T.nA[X]);
      const float4 bb = __ldg(&T.nB[X]);
      const float ex = fmaxf(fmaxf(__fsub_rn(a.x, px), __fsub_rn(px, bb.x)), 0.0f);
      const float ey = fmaxf(fmaxf(__fsub_rn(a.y, py), __fsub_rn(py, bb.y)), 0.0f);
      const float ez = fmaxf(fmaxf(__fsub_rn(a.z, pz), __fsub_rn(pz, bb.z)), 0.0f);
      const float r2 =
          __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
      acc = __ldg(&T.nl2[X]) < __fmul_rn(P.theta2, r2);
      opn = !acc;
    }
    const unsigned accM = __ballot_sync(FULL, acc);
    const unsigned opnM = __ballot_sync(FULL, opn);
    if (MERGE) {
      if (__any_sync(FULL, acc && pnd)) flush();
      if (acc) {
        pnd = true;
        pC = X;
        pdC = dX;
        pqx = s.x;
        pqy = s.y;
        pqz = s.z;
        pL = s.w;
        psrc = -1;
        if (BG) {
          bg_move(T, P, s, pqx, pqy, pqz, pC, pdC, cpath);
          pbg = true;
        }
      }
    } else if (accM) {
      warp_ray<ADJ, MOM, STOP, NB, SUB, CNT, TD>(T, P, acc, px, py, pz, S, dS, anc, rst, on_path, ws.path, X, dX, s.x,
                         s.y, s.z, s.w, -1, gk, stack_limit, box_limit, status, J, cnt, F, mom,
                         i);
    }
    if (opnM) {
      const int4 t = __ldg(&T.nT[X]);
      if (t.x < 0) {
        for (int jj = t.z; jj < t.z + t.w; ++jj) {
          const float4 y = __ldg(&T.src[jj]);
          if (!(y.w > 0.0f)) continue;
          if (MERGE) {
            if (__any_sync(FULL, opn && pnd)) flush();
            if (opn) {
              pnd = true;
              pC = X;
              pdC = dX;
              pqx = y.x;
              pqy = y.y;
              pqz = y.z;
              pL = y.w;
              psrc = jj;
            }
          } else {
            warp_ray<ADJ, MOM, STOP, NB, SUB, CNT, TD>(T, P, opn, px, py, pz, S, dS, anc, rst, on_path, ws.path, X, dX,
                               y.x, y.y, y.z, y.w, jj, gk, stack_limit, box_limit, status, J, cnt,
                               F, mom, i);
          }
        }
      } else {
        if (sp + 2 > stack_limit) {
          if (lane == 0) atomicOr(status, kStatusStackOverflow);
          break;
        }
        if (lane == 0) {
          ws.node[sp] = t.x + 1;
          ws.depth[sp] = dX + 1;
          ws.mask[sp] = opnM;
          ws.node[sp + 1] = t.x;
          ws.depth[sp + 1] = dX + 1;
          ws.mask[sp + 1] = opnM;
        }
        sp += 2;
        __syncwarp();
      }
    }
  }
  if (MERGE && __any_sync(FULL, pnd)) flush();
}

// 8 blocks of 128 per SM (at most 64 registers): measured 4% faster forward and 8%
// faster adjoint than the compiler's own 70 registers at 7 blocks. The adjoint keeps
// no counters (the backward call reports none) and stays at 8 blocks: 3% faster
// than with counters; 10 and 12 blocks spilled and were 6% and 13% slower. Without
// counters (CNT = false, the plain flux when the caller asks for no counters or
// stats) the walk runs 12 blocks (40 registers, spilling to L1): 2.7% faster than
// 9 blocks (56 registers) on the clumpy workload, 119.8 against 123.2 ms; 10
// blocks were slower (141 ms).
// CNT = false keeps no per-sink counters; the fluxes are bit-identical. The band
// walks without counters fit 6 blocks (74 registers, no spills) instead of 4:
// 245 ms against 262 ms for four bands on the clumpy workload. The sub-bucket walk
// runs 8 blocks (64 registers, spilling): 325.6 ms against 343.0 ms at 4 blocks
// (114 registers) on 2^18 particles, without counters.
template <bool ADJ, bool MERGE, bool MOM = false, bool BG = false, bool STOP = false, int NB = 1,
          bool SUB = false, bool CNT = true, bool TD = false>
__global__ void __launch_bounds__(128, SUB ? 8 : ADJ ? 8 : (NB > 1 ? (CNT ? 4 : 6) : (CNT ? 8 : 12))) walk_warp_kernel(TreeView T, const long long* sink_idx,
                                                        int n_sink, WalkParams P, SinkOut out,
                                                        unsigned long long* stats, int* status,
                                                        AdjointArgs J) {
  __shared__ WarpStack stacks[4];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  WarpStack& ws = stacks[threadIdx.x >> 5];
  SinkCounters cnt;
  int i = 0, slot = 0;
  float g = 0.0f;
  bool has = false;
  if (k < n_sink) {
    PlainMap<ADJ> map{&T, sink_idx, J.grad_flux, status};
    has = map(k, i, slot, g);
    if (!has && !ADJ && sink_idx) {
      if (out.flux)
        for (int b = 0; b < (NB > 1 ? T.n_bands : 1); ++b) out.flux[(size_t)b * out.n_out + k] = 0.0f;
      if (out.counters) reinterpret_cast<int4*>(out.counters)[k] = make_int4(0, 0, 0, 0);
    }
  }
  CSum F[NB];
  Moments mom;
  if (__any_sync(0xffffffffu, has))
    warp_walk<ADJ, MERGE, MOM, BG, STOP, NB, SUB, CNT, TD>(T, P, has, i, g, ws, status, J, cnt, F,
                                                  MOM ? &mom : nullptr);
  if (MOM && has) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (out.fvec) out.fvec[(size_t)q * out.n_out + slot] = mom.v[q].get();
#pragma unroll
    for (int q = 0; q < 6; ++q)
      if (out.press) out.press[(size_t)q * out.n_out + slot] = mom.v[3 + q].get();
  }
  if (!ADJ && has) {
    if (NB > 1) {
      // band-major output: band b of sink slot at b * n_out + slot
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (out.flux && b < T.n_bands) out.flux[(size_t)b * out.n_out + slot] = F[b].get();
    } else if (out.flux) {
      out.flux[slot] = F[0].get();
    }
    if (out.counters)
      reinterpret_cast<int4*>(out.counters)[slot] = make_int4(cnt.rays, cnt.segs, cnt.visit, cnt.ref);
  }
  if (stats) add_stats(cnt, stats);
}

// Batched form of the warp-shared walk: each work item is cut into groups of 32
// consecutive sinks, one warp walk per group.
// CNT = false (no stats asked for): no counters, and 12 blocks-of-128 worth of
// threads per SM instead of 8, as for the single-tree walk (2.8% faster than 9 on
// the 64 boxes).
template <int BS, bool MERGE, bool CNT = true>
__global__ void __launch_bounds__(BS, CNT ? 1024 / BS : 1536 / BS) walk_warp_batched_kernel(
    const TreeView* __restrict__ views, float* const* __restrict__ flux_out,
    const int2* __restrict__ items, int n_items, int item, unsigned* counter, WalkParams P,
    unsigned long long* stats, int* status) {
  __shared__ WarpStack stacks[BS / 32];
  WarpStack& ws = stacks[threadIdx.x >> 5];
  const unsigned lane = threadIdx.x & 31u;
  SinkCounters tot;
  while (true) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)n_items) break;
    const int2 w = items[it];
    const TreeView T = views[w.x];
    WalkParams Pt = P;  // the coincident-source cut (1e-12 side)^2 of this tree, in fp32
    const float smin = __fmul_rn(1e-12f, T.side);
    Pt.smin2 = __fmul_rn(smin, smin);
    const int end = min(w.y + item, T.n_gas);
    for (int g0 = w.y; g0 < end; g0 += 32) {
      const int i = g0 + (int)lane;
      const bool has = i < end;
      SinkCounters cnt;
      CSum F;
      warp_walk<false, MERGE, false, false, false, 1, false, CNT>(T, Pt, has, i, 0.0f, ws, status,
                                                                 AdjointArgs{}, cnt, &F);
      if (has) flux_out[w.x][T.perm[i]] = F.get();
      if (CNT) {
        tot.rays += cnt.rays;
        tot.segs += cnt.segs;
        tot.visit += cnt.visit;
        tot.ref += cnt.ref;
        tot.clip += cnt.clip;
      }
    }
  }
  if (CNT && stats) add_stats(tot, stats);
}

cudaError_t launch_walk_batched(const TreeView* views, float* const* flux_out, const int2* items,
                                int n_items, int item, unsigned* counter, const WalkParams& wp,
                                unsigned long long* stats, int* status, int block_size,
                                int n_sm, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (wp.variant >= 2) {
    const int bs = block_size <= 64 ? 64 : (block_size <= 128 ? 128 : 256);
    const bool merge = wp.variant == 3;
#define TREVR_WB(BSV, MV)                                                                     \
  do {                                                                                         \
    if (stats) {                                                                               \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk_warp_batched_kernel<BSV, MV>, \
                                                    BSV, 0);                                   \
      walk_warp_batched_kernel<BSV, MV><<<n_sm * per_sm, BSV, 0, s>>>(                        \
          views, flux_out, items, n_items, item, counter, wp, stats, status);                  \
    } else {                                                                                   \
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(                                           \
          &per_sm, walk_warp_batched_kernel<BSV, MV, false>, BSV, 0);                          \
      walk_warp_batched_kernel<BSV, MV, false><<<n_sm * per_sm, BSV, 0, s>>>(                 \
          views, flux_out, items, n_items, item, counter, wp, nullptr, status);                \
    }                                                                                          \
  } while (0)
    if (bs == 64) {
      if (merge) TREVR_WB(64, true);
      else TREVR_WB(64, false);
    } else if (bs == 128) {
      if (merge) TREVR_WB(128, true);
      else TREVR_WB(128, false);
    } else {
      if (merge) TREVR_WB(256, true);
      else TREVR_WB(256, false);
    }
#undef TREVR_WB
  } else if (block_size <= 64) {
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

cudaError_t launch_walk_moments(const TreeView& T, const long long* sink_idx, int n_sink,
                                const WalkParams& wp, float* flux_out, float* fvec, float* press,
                                int* status, cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  walk_warp_kernel<false, true, true><<<(n_sink + 127) / 128, 128, 0, s>>>(
      T, sink_idx, n_sink, wp, SinkOut{flux_out, nullptr, fvec, press, n_sink}, nullptr, status,
      AdjointArgs{});
  note_launch();
  return cudaGetLastError();
}

// Several bands: 2 band slots for 2 bands, 4 slots for 3 or 4 (an unused slot holds
// zeros and is not written). One band is the plain walk.
cudaError_t launch_walk_bands(const TreeView& T, const long long* sink_idx, int n_sink,
                              const WalkParams& wp, float* flux_out, int* counters,
                              unsigned long long* stats, int* status, cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  const dim3 grid((n_sink + 127) / 128);
  const SinkOut o{flux_out, counters, nullptr, nullptr, n_sink};
  const bool cnt = counters || stats;
  if (T.n_bands <= 2 && cnt)
    walk_warp_kernel<false, true, false, false, false, 2><<<grid, 128, 0, s>>>(
        T, sink_idx, n_sink, wp, o, stats, status, AdjointArgs{});
  else if (T.n_bands <= 2)
    walk_warp_kernel<false, true, false, false, false, 2, false, false><<<grid, 128, 0, s>>>(
        T, sink_idx, n_sink, wp, o, nullptr, status, AdjointArgs{});
  else if (cnt)
    walk_warp_kernel<false, true, false, false, false, 4><<<grid, 128, 0, s>>>(
        T, sink_idx, n_sink, wp, o, stats, status, AdjointArgs{});
  else
    walk_warp_kernel<false, true, false, false, false, 4, false, false><<<grid, 128, 0, s>>>(
        T, sink_idx, n_sink, wp, o, nullptr, status, AdjointArgs{});
  note_launch();
  return cudaGetLastError();
}

static int chunk_of(const WalkParams& wp) {
  return wp.sinks_per_warp > 0 ? wp.sinks_per_warp : kDefaultChunk;
}

cudaError_t launch_walk(const TreeView& T, const long long* sink_idx, int n_sink,
                        const WalkParams& wp, float* flux_out, int* counters,
                        unsigned long long* stats, int* status, int block_size,
                        cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  (void)block_size;
  if (wp.sub_bucket) {
    if (counters || stats)
      walk_warp_kernel<false, true, false, false, false, 1, true><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{flux_out, counters, nullptr, nullptr, n_sink}, stats,
          status, AdjointArgs{});
    else
      walk_warp_kernel<false, true, false, false, false, 1, true, false><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{flux_out, nullptr, nullptr, nullptr, n_sink}, nullptr,
          status, AdjointArgs{});
    note_launch();
    return cudaGetLastError();
  }
  if (wp.bg_radius > 0.0f || wp.tau_stop < INFINITY) {
    const dim3 grid((n_sink + 127) / 128);
    const SinkOut o{flux_out, counters, nullptr, nullptr, n_sink};
    const bool bg = wp.bg_radius > 0.0f, stop = wp.tau_stop < INFINITY;
    if (counters || stats) {
      if (bg && stop)
        walk_warp_kernel<false, true, false, true, true><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, stats, status, AdjointArgs{});
      else if (bg)
        walk_warp_kernel<false, true, false, true><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, stats, status, AdjointArgs{});
      else
        walk_warp_kernel<false, true, false, false, true><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, stats, status, AdjointArgs{});
    } else {  // no counters asked for: the walk keeps none
      if (bg && stop)
        walk_warp_kernel<false, true, false, true, true, 1, false, false><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, nullptr, status, AdjointArgs{});
      else if (bg)
        walk_warp_kernel<false, true, false, true, false, 1, false, false><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, nullptr, status, AdjointArgs{});
      else
        walk_warp_kernel<false, true, false, false, true, 1, false, false><<<grid, 128, 0, s>>>(
            T, sink_idx, n_sink, wp, o, nullptr, status, AdjointArgs{});
    }
    note_launch();
    return cudaGetLastError();
  }
  if (wp.topdown) {  // the top-down ray walk (merged-ray walk only)
    const SinkOut o{flux_out, counters, nullptr, nullptr, n_sink};
    if (counters || stats)
      walk_warp_kernel<false, true, false, false, false, 1, false, true, true>
          <<<(n_sink + 127) / 128, 128, 0, s>>>(T, sink_idx, n_sink, wp, o, stats, status,
                                                AdjointArgs{});
    else
      walk_warp_kernel<false, true, false, false, false, 1, false, false, true>
          <<<(n_sink + 127) / 128, 128, 0, s>>>(T, sink_idx, n_sink, wp, o, nullptr, status,
                                                AdjointArgs{});
    note_launch();
    return cudaGetLastError();
  }
  if (wp.variant >= 2) {
    if (wp.variant == 3 && (counters || stats))
      walk_warp_kernel<false, true><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{flux_out, counters, nullptr, nullptr, n_sink}, stats, status, AdjointArgs{});
    else if (wp.variant == 3)  // no counters asked for: the walk keeps none
      walk_warp_kernel<false, true, false, false, false, 1, false, false><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{flux_out, nullptr, nullptr, nullptr, n_sink}, nullptr, status, AdjointArgs{});
    else
      walk_warp_kernel<false, false><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{flux_out, counters, nullptr, nullptr, n_sink}, stats, status, AdjointArgs{});
    note_launch();
    return cudaGetLastError();
  }
  const int chunk = chunk_of(wp);
  const long long warps = ((long long)n_sink + chunk - 1) / chunk;
  const int blocks = (int)((warps * 32 + 127) / 128);
  walk_kernel<false><<<blocks, 128, 0, s>>>(T, sink_idx, n_sink, chunk, wp,
                                            SinkOut{flux_out, counters, nullptr, nullptr, n_sink}, stats, status,
                                            AdjointArgs{});
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_walk_adjoint(const TreeView& T, const long long* sink_idx, int n_sink,
                                const WalkParams& wp, const AdjointArgs& J, int* status,
                                cudaStream_t s) {
  if (n_sink <= 0) return cudaSuccess;
  if (wp.variant >= 2) {
    if (wp.variant == 3)
      walk_warp_kernel<true, true, false, false, false, 1, false, false><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{nullptr, nullptr, nullptr, nullptr, n_sink}, nullptr, status, J);
    else
      walk_warp_kernel<true, false><<<(n_sink + 127) / 128, 128, 0, s>>>(
          T, sink_idx, n_sink, wp, SinkOut{nullptr, nullptr, nullptr, nullptr, n_sink}, nullptr, status, J);
    note_launch();
    return cudaGetLastError();
  }
  const int chunk = chunk_of(wp);
  const long long warps = ((long long)n_sink + chunk - 1) / chunk;
  const int blocks = (int)((warps * 32 + 127) / 128);
  walk_kernel<true><<<blocks, 128, 0, s>>>(T, sink_idx, n_sink, chunk, wp,
                                           SinkOut{nullptr, nullptr, nullptr, nullptr, n_sink}, nullptr, status, J);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trevr
