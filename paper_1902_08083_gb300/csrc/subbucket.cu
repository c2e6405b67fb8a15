// Smoothing lengths and neighbour lists for the sub-bucket particle trace
// (Sec. 2.2.3, 3.1.3).
//
// Below the bucket scale, the absorption is the SPH field
// alpha(x) = sum_j alpha_j w_j W(|x - x_j|, h_j), with W the cubic spline of support
// 2h. A bucket whose own particles still ask for refinement gets this field
// integrated along the ray's chord inside it. The particles that can add to the
// field inside a leaf are those whose support sphere (radius 2 h_j) meets the leaf's
// box. This file lists them once per tree, for every leaf, by a tree search that
// prunes cells with the largest smoothing length below them. It also stores each
// leaf's spread max - min of its particles' alpha, which the sub-bucket refinement
// test uses, and the kernel-integral table the trace interpolates (the pre-computed
// kernel integral of an SPHRay-like trace, Sec. 2.2.3).
#include <cstring>

#include "trevr_internal.cuh"

namespace trevr {
namespace {

constexpr int kNbrStack = 2 * kMaxLevels + 4;

__global__ void smoothing_kernel(const float* __restrict__ h, const int* __restrict__ perm,
                                 const float4* __restrict__ pos, const float* __restrict__ w,
                                 int n, float4* __restrict__ sp, float* __restrict__ aw,
                                 int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float H = h[perm[i]];
    if (!(H > 0.0f) || !isfinite(H)) atomicOr(status, kStatusInvalid);
    const float4 p = pos[i];
    sp[i] = make_float4(p.x, p.y, p.z, H);
    aw[i] = __fmul_rn(p.w, w[i]);
  }
}

// bottom-up, one level: the largest h below each cell, and each leaf's alpha spread
__global__ void hmax_level_kernel(const int4* __restrict__ nT, const int* __restrict__ nfirst,
                                  const int* __restrict__ ncount, const float4* __restrict__ sp,
                                  const float4* __restrict__ pos, const int* __restrict__ levels,
                                  int Lv, float* __restrict__ hmax, float* __restrict__ dbk) {
  const int begin = levels[2 * Lv], end = levels[2 * Lv + 1];
  for (int X = begin + blockIdx.x * blockDim.x + threadIdx.x; X < end;
       X += gridDim.x * blockDim.x) {
    const int c = nT[X].x;
    if (c < 0) {
      float hm = 0.0f, amin = INFINITY, amax = -INFINITY;
      for (int i = nfirst[X]; i < nfirst[X] + ncount[X]; ++i) {
        hm = fmaxf(hm, sp[i].w);
        amin = fminf(amin, pos[i].w);
        amax = fmaxf(amax, pos[i].w);
      }
      hmax[X] = hm;
      dbk[X] = __fsub_rn(amax, amin);
    } else {
      hmax[X] = fmaxf(hmax[c], hmax[c + 1]);
      dbk[X] = 0.0f;
    }
  }
}

struct NbrArgs {
  const int4* nT;
  const float4* nA;  // lower corner (xyz)
  const float4* nB;  // upper corner (xyz)
  const int* nfirst;
  const int* ncount;
  const float4* sp;
  const float* hmax;
  int n_end;         // cells are kRoot .. n_end - 1
  float pad;         // absolute slack added to every support radius
  unsigned* count;   // count pass: per cell
  const unsigned* first;  // fill pass: per cell start
  const float* aw;        // per sorted particle alpha * w
  int2* nbr_ja;           // fill pass: output, the entry's sorted index and alpha * w (bits)
  float4* nbr_sp;         // fill pass: output, the entry's (x, y, z, 1/h)
  int* status;
};

__device__ __forceinline__ float box_gap2(float4 alo, float4 ahi, float4 blo, float4 bhi) {
  const float gx = fmaxf(fmaxf(__fsub_rn(blo.x, ahi.x), __fsub_rn(alo.x, bhi.x)), 0.0f);
  const float gy = fmaxf(fmaxf(__fsub_rn(blo.y, ahi.y), __fsub_rn(alo.y, bhi.y)), 0.0f);
  const float gz = fmaxf(fmaxf(__fsub_rn(blo.z, ahi.z), __fsub_rn(alo.z, bhi.z)), 0.0f);
  return gx * gx + gy * gy + gz * gz;
}

// one thread per leaf: every particle whose support sphere meets the leaf's box
// (radius 2h (1 + 1e-5) + pad, so that rounding can only add a harmless neighbour)
template <bool FILL>
__global__ void nbr_kernel(NbrArgs A) {
  for (int X = kRoot + blockIdx.x * blockDim.x + threadIdx.x; X < A.n_end;
       X += gridDim.x * blockDim.x) {
    if (A.nT[X].x >= 0) continue;
    const float4 lo = A.nA[X], hi = A.nB[X];
    int stack[kNbrStack];
    int sp = 0;
    stack[sp++] = kRoot;
    unsigned c = 0;
    unsigned out = FILL ? A.first[X] : 0u;
    const unsigned out_end = FILL ? A.first[X + 1] : 0u;  // the count pass's total
    while (sp > 0) {
      const int Y = stack[--sp];
      const float R = fmaf(2.0f * A.hmax[Y], 1.00001f, A.pad);
      if (box_gap2(lo, hi, A.nA[Y], A.nB[Y]) >= R * R) continue;
      const int ch = A.nT[Y].x;
      if (ch >= 0) {
        if (sp + 2 > kNbrStack) {
          atomicOr(A.status, kStatusStackOverflow);
          break;
        }
        stack[sp++] = ch + 1;
        stack[sp++] = ch;
        continue;
      }
      for (int i = A.nfirst[Y]; i < A.nfirst[Y] + A.ncount[Y]; ++i) {
        const float4 q = A.sp[i];
        const float ex = fmaxf(fmaxf(__fsub_rn(lo.x, q.x), __fsub_rn(q.x, hi.x)), 0.0f);
        const float ey = fmaxf(fmaxf(__fsub_rn(lo.y, q.y), __fsub_rn(q.y, hi.y)), 0.0f);
        const float ez = fmaxf(fmaxf(__fsub_rn(lo.z, q.z), __fsub_rn(q.z, hi.z)), 0.0f);
        const float r = fmaf(2.0f * q.w, 1.00001f, A.pad);
        if (ex * ex + ey * ey + ez * ez < r * r) {
          if (FILL && out < out_end) {
            A.nbr_ja[out] = make_int2(i, __float_as_int(A.aw[i]));
            A.nbr_sp[out] = make_float4(q.x, q.y, q.z, __frcp_rn(q.w));
            ++out;
          }
          ++c;
        }
      }
    }
    if (!FILL) A.count[X] = c;
  }
}

// The dimensionless cubic spline w(q): W(r, h) = w(r/h) / (pi h^3), support 2h.
__device__ __forceinline__ float spline_q(float q) {
  if (q < 1.0f) return 1.0f - 1.5f * q * q + 0.75f * q * q * q;
  if (q < 2.0f) {
    const float t = 2.0f - q;
    return 0.25f * t * t * t;
  }
  return 0.0f;
}

// integral of w(sqrt(x + t^2)) dt over [a, c], Gauss-Legendre with 6 points on each half
// (nodes and weights of Abramowitz & Stegun, Table 25.4)
__device__ float gl6_halves(float x, float a, float c) {
  if (!(c > a)) return 0.0f;
  const float g[3] = {0.2386191860831969f, 0.6612093864662645f, 0.9324695142031521f};
  const float wt[3] = {0.4679139345726910f, 0.3607615730481386f, 0.1713244923791704f};
  float acc = 0.0f;
  for (int half = 0; half < 2; ++half) {
    const float lo = half ? 0.5f * (a + c) : a, hi = half ? c : 0.5f * (a + c);
    const float m = 0.5f * (lo + hi), hw = 0.5f * (hi - lo);
    float part = 0.0f;
    for (int k = 0; k < 3; ++k) {
      const float u = hw * g[k];
      part += wt[k] * (spline_q(sqrtf(x + (m - u) * (m - u))) +
                       spline_q(sqrtf(x + (m + u) * (m + u))));
    }
    acc += part * hw;
  }
  return acc;
}

// Phi(x, sigma) = integral over t in [0, sigma] of w(sqrt(x + t^2)): the column of the
// kernel through a chord at impact parameter b = h sqrt(x), from the closest approach
// to s = h sigma, in units of 1 / (pi h^2). The integrand's break points t = sqrt(1 - x)
// (q = 1) and t = sqrt(4 - x) (q = 2) separate the smooth pieces.
__global__ void kint_table_kernel(float* __restrict__ tab) {
  const int n = (kKintNX + 1) * (kKintNS + 1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int i = e / (kKintNS + 1), j = e - i * (kKintNS + 1);
    const float x = 4.0f * (float)i / (float)kKintNX;
    const float sigma = 2.0f * (float)j / (float)kKintNS;
    const float t1 = x < 1.0f ? sqrtf(1.0f - x) : 0.0f;
    const float t2 = x < 4.0f ? sqrtf(4.0f - x) : 0.0f;
    const float c1 = fminf(sigma, t1), c2 = fminf(sigma, t2);
    tab[e] = gl6_halves(x, 0.0f, c1) + gl6_halves(x, c1, c2);
  }
}

// the table by cells: the four corner values of each cell of the grid in one record,
// so that a bilinear lookup reads 16 bytes once
__global__ void kint_cells_kernel(const float* __restrict__ tab, float4* __restrict__ cells) {
  const int n = kKintNX * kKintNS;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int i = e / kKintNS, j = e - i * kKintNS;
    const float* r0 = tab + (size_t)i * (kKintNS + 1) + j;
    const float* r1 = r0 + (kKintNS + 1);
    cells[e] = make_float4(r0[0], r0[1], r1[0], r1[1]);
  }
}

inline int grid_of(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

template <class T>
void free_dev(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

}  // namespace

int set_smoothing_impl(trevr_tree* t, const float* h, cudaStream_t s) {
  const int n = (int)t->n_gas;
  const size_t ncell = (size_t)t->n_nodes + kRoot;
  cudaStreamSynchronize(s);
  free_dev(t->sp);
  free_dev(t->aw);
  free_dev(t->dbk);
  free_dev(t->nbr_first);
  free_dev(t->nbr_ja);
  free_dev(t->nbr_sp);
  free_dev(t->kint4);
  t->n_nbr = 0;
  float* hmax = nullptr;
  float* tab = nullptr;  // the kernel-integral table on the grid's nodes, before packing
  unsigned* scratch = nullptr;
  int* st = nullptr;
  cudaError_t e = cudaMalloc(&t->sp, sizeof(float4) * n);
  if (e == cudaSuccess) e = cudaMalloc(&t->aw, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc(&t->dbk, sizeof(float) * ncell);
  if (e == cudaSuccess) e = cudaMalloc(&t->nbr_first, sizeof(unsigned) * (ncell + 1));
  if (e == cudaSuccess) e = cudaMalloc(&hmax, sizeof(float) * ncell);
  if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(unsigned) * scan_scratch_words((int)ncell + 1));
  if (e == cudaSuccess) e = cudaMalloc(&st, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&tab, sizeof(float) * (size_t)(kKintNX + 1) * (kKintNS + 1));
  if (e == cudaSuccess) e = cudaMalloc(&t->kint4, sizeof(float4) * (size_t)kKintNX * kKintNS);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->nbr_first, 0, sizeof(unsigned) * (ncell + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hmax, 0, sizeof(float) * ncell, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->dbk, 0, sizeof(float) * ncell, s);
  NbrArgs A;
  std::memset(&A, 0, sizeof(A));
  unsigned total = 0;
  int bad = 0;
  if (e == cudaSuccess) {
    smoothing_kernel<<<grid_of(n, 256), 256, 0, s>>>(h, t->perm, t->pos, t->w, n, t->sp, t->aw, st);
    note_launch();
    kint_table_kernel<<<grid_of((long long)(kKintNX + 1) * (kKintNS + 1), 256), 256, 0, s>>>(
        tab);
    note_launch();
    kint_cells_kernel<<<grid_of((long long)kKintNX * kKintNS, 256), 256, 0, s>>>(tab, t->kint4);
    note_launch();
    for (int L = t->max_depth; L >= 0; --L) {
      const int m = t->h_levels[2 * L + 1] - t->h_levels[2 * L];
      hmax_level_kernel<<<grid_of(m, 128), 128, 0, s>>>(t->nT, t->nfirst, t->ncount, t->sp,
                                                         t->pos, t->levels, L, hmax, t->dbk);
      note_launch();
    }
    A.nT = t->nT;
    A.nA = t->nA;
    A.nB = t->nB;
    A.nfirst = t->nfirst;
    A.ncount = t->ncount;
    A.sp = t->sp;
    A.hmax = hmax;
    A.n_end = (int)ncell;
    A.pad = 1e-6f * t->side;
    A.count = t->nbr_first;
    A.status = st;
    nbr_kernel<false><<<grid_of((long long)ncell, 128), 128, 0, s>>>(A);
    note_launch();
    exclusive_scan_u32(t->nbr_first, (int)ncell + 1, scratch, s);
    cudaMemcpyAsync(&total, t->nbr_first + ncell, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&bad, st, sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess && !bad) {
    if (total > 0x7fffffffu) {
      e = cudaErrorMemoryAllocation;
    } else {
      const size_t m = total > 0 ? total : 1;
      e = cudaMalloc(&t->nbr_ja, sizeof(int2) * m);
      if (e == cudaSuccess) e = cudaMalloc(&t->nbr_sp, sizeof(float4) * m);
      if (e == cudaSuccess) {
        A.first = t->nbr_first;
        A.aw = t->aw;
        A.nbr_ja = t->nbr_ja;
        A.nbr_sp = t->nbr_sp;
        nbr_kernel<true><<<grid_of((long long)ncell, 128), 128, 0, s>>>(A);
        note_launch();
        cudaMemcpyAsync(&bad, st, sizeof(int), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        t->n_nbr = total;
      }
    }
  }
  if (hmax) cudaFree(hmax);
  if (tab) cudaFree(tab);
  if (scratch) cudaFree(scratch);
  if (st) cudaFree(st);
  if (e != cudaSuccess || bad) {
    free_dev(t->sp);
    free_dev(t->aw);
    free_dev(t->dbk);
    free_dev(t->nbr_first);
    free_dev(t->nbr_ja);
    free_dev(t->nbr_sp);
    free_dev(t->kint4);
    t->n_nbr = 0;
    if (e == cudaErrorMemoryAllocation) return TREVR_ERR_OUT_OF_MEMORY;
    return e != cudaSuccess ? cuda_to_error(e) : status_to_error(bad);
  }
  return TREVR_OK;
}

}  // namespace trevr
