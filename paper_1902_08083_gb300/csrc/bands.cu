// Trees with several bands (Sec. 4: many bands for a constant factor in cost).
//
// Band b has its own absorption alpha_b per particle and luminosity L_b per source.
// The bands share the walk and the rays. The tree is built as a single-band tree
// whose absorption is band 0's and whose source luminosity is the band sum
// L = sum_b L_b (FP64 in band order, rounded to fp32 per source). The centres of
// luminosity and the opening-angle test therefore see the summed light. A second
// bottom-up pass per band then fills the band records of every cell:
//   bA[X].b  = fp32(sum_i w_i alpha_b,i / sum_i w_i)          (Sec. 2.2.3, 2.3)
//   bLc[X].b = fp32(sum_j L_b,j)
//   nB[X].w  = max over the bands of fp32(alpha_max,b - alpha_min,b)
// The last line makes a cell refine (Eq. refcrit) when any band asks for it. The
// directional alpha_min / alpha_max recursion and the FP64 operation order are those
// of the single-band moments.
#include <cstring>

#include "trevr_internal.cuh"

namespace trevr {
namespace {

struct BandMom {
  double WA, L, amin[3], amax[3];
};

struct BandArgs {
  const int4* nT;
  const int4* nglo;
  const int4* nghi;
  const int* nfirst;
  const int* ncount;
  const float* w;       // sorted volume weights
  const float* as;      // band b's absorption, sorted
  const float* bLs;     // per sorted source, 4 band luminosities
  const double* nW;     // per cell, sum of the volume weights
  const int* levels;
  BandMom* mom;
  float* bA;            // per cell, 4 slots
  float* bLc;           // per cell, 4 slots
  float4* nB;
  int b;
};

// L_j = fp32(sum_b L_b,j) in band order; a negative or non-finite band luminosity is
// an invalid argument
__global__ void band_lsum_kernel(const float* __restrict__ lum_bands, int ns, int nb,
                                 float* __restrict__ lsum, int* status) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) {
      const float L = lum_bands[(size_t)b * ns + j];
      if (!(L >= 0.0f) || !isfinite(L)) atomicOr(status, kStatusInvalid);
      t = __dadd_rn(t, (double)L);
    }
    lsum[j] = __double2float_rn(t);
  }
}

__global__ void band_src_kernel(const float* __restrict__ lum_bands, int ns, int nb,
                                const int* __restrict__ src_order, float* __restrict__ bLs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
    const int o = src_order[j];
    for (int b = 0; b < nb; ++b) bLs[4 * (size_t)j + b] = lum_bands[(size_t)b * ns + o];
  }
}

__global__ void band_alpha_kernel(const float* __restrict__ alpha_b, const int* __restrict__ perm,
                                  int n, float* __restrict__ as, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float a = alpha_b[perm[i]];
    if (!(a >= 0.0f) || !isfinite(a)) atomicOr(status, kStatusInvalid);
    as[i] = a;
  }
}

__global__ void band_moments_level_kernel(BandArgs A, int Lv) {
  const int begin = A.levels[2 * Lv], end = A.levels[2 * Lv + 1];
  for (int X = begin + blockIdx.x * blockDim.x + threadIdx.x; X < end;
       X += gridDim.x * blockDim.x) {
    const int4 t = A.nT[X];
    BandMom m;
    if (t.x < 0) {
      double swa = 0.0;
      const int f = A.nfirst[X], c = A.ncount[X];
      for (int i = f; i < f + c; ++i)
        swa = __dadd_rn(swa, __dmul_rn((double)A.w[i], (double)A.as[i]));
      double sl = 0.0;
      for (int s = t.z; s < t.z + t.w; ++s) sl = __dadd_rn(sl, (double)A.bLs[4 * (size_t)s + A.b]);
      m.WA = swa;
      m.L = sl;
      const double ab = __ddiv_rn(swa, A.nW[X]);
      for (int d = 0; d < 3; ++d) m.amin[d] = m.amax[d] = ab;
    } else {
      const BandMom& m1 = A.mom[t.x];
      const BandMom& m2 = A.mom[t.x + 1];
      m.WA = __dadd_rn(m1.WA, m2.WA);
      m.L = __dadd_rn(m1.L, m2.L);
      const int a = A.nglo[X].w;
      const int4 l1 = A.nglo[t.x], h1 = A.nghi[t.x], l2 = A.nglo[t.x + 1], h2 = A.nghi[t.x + 1];
      const int4 lX = A.nglo[X], hX = A.nghi[X];
      const int lo1[3] = {l1.x, l1.y, l1.z}, hi1[3] = {h1.x, h1.y, h1.z};
      const int lo2[3] = {l2.x, l2.y, l2.z}, hi2[3] = {h2.x, h2.y, h2.z};
      const int loX[3] = {lX.x, lX.y, lX.z}, hiX[3] = {hX.x, hX.y, hX.z};
      for (int d = 0; d < 3; ++d) {
        if (d == a) {
          const double w1 = (double)(hi1[d] - lo1[d]);
          const double w2 = (double)(hi2[d] - lo2[d]);
          const double Wd = (double)(hiX[d] - loX[d]);
          m.amin[d] =
              __ddiv_rn(__dadd_rn(__dmul_rn(m1.amin[d], w1), __dmul_rn(m2.amin[d], w2)), Wd);
          m.amax[d] =
              __ddiv_rn(__dadd_rn(__dmul_rn(m1.amax[d], w1), __dmul_rn(m2.amax[d], w2)), Wd);
        } else {
          m.amin[d] = fmin(m1.amin[d], m2.amin[d]);
          m.amax[d] = fmax(m1.amax[d], m2.amax[d]);
        }
      }
    }
    A.mom[X] = m;
    const double amin = fmin(fmin(m.amin[0], m.amin[1]), m.amin[2]);
    const double amax = fmax(fmax(m.amax[0], m.amax[1]), m.amax[2]);
    A.bA[4 * (size_t)X + A.b] = __double2float_rn(__ddiv_rn(m.WA, A.nW[X]));
    A.bLc[4 * (size_t)X + A.b] = __double2float_rn(m.L);
    const float dal = __double2float_rn(__dsub_rn(amax, amin));
    if (dal > A.nB[X].w) A.nB[X].w = dal;
  }
}

inline int grid_of(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int build_tree_bands_impl(const float* gas_xyz, const float* alpha_bands, const float* weight,
                          long long n_gas, const float* src_xyz, const float* lum_bands,
                          long long n_src, int n_bands, const trevr_domain* dom, int bucket,
                          cudaStream_t s, trevr_tree** out, float* build_ms) {
  const int n = (int)n_gas, ns = (int)n_src, nb = n_bands;
  float* lsum = nullptr;
  int* st = nullptr;
  cudaError_t e = pool_malloc_async((void**)&lsum, sizeof(float) * (ns > 0 ? ns : 1), s);
  if (e == cudaSuccess) e = pool_malloc_async((void**)&st, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    if (lsum) cudaFreeAsync(lsum, s);
    if (st) cudaFreeAsync(st, s);
    return cuda_to_error(e);
  }
  if (ns > 0) {
    band_lsum_kernel<<<grid_of(ns, 256), 256, 0, s>>>(lum_bands, ns, nb, lsum, st);
    note_launch();
  }
  int bad = 0;
  cudaMemcpyAsync(&bad, st, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || bad) {
    cudaFreeAsync(lsum, s);
    cudaFreeAsync(st, s);
    return e != cudaSuccess ? cuda_to_error(e) : status_to_error(bad);
  }
  trevr_tree* t = nullptr;
  float ms = 0.0f;
  int rc = build_tree_impl(gas_xyz, alpha_bands, weight, n_gas, src_xyz, lsum, n_src, dom, bucket,
                           s, &t, &ms);
  cudaFreeAsync(lsum, s);
  if (rc != TREVR_OK) {
    cudaFreeAsync(st, s);
    return rc;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const size_t ncell = (size_t)t->n_nodes + kRoot;
  float* as = nullptr;
  BandMom* mom = nullptr;
  e = cudaMalloc(&t->bA, sizeof(float4) * ncell);
  if (e == cudaSuccess) e = cudaMalloc(&t->bLc, sizeof(float4) * ncell);
  if (e == cudaSuccess) e = cudaMalloc(&t->bLs, sizeof(float4) * (ns > 0 ? ns : 1));
  if (e == cudaSuccess) e = pool_malloc_async((void**)&as, sizeof(float) * n, s);
  if (e == cudaSuccess) e = pool_malloc_async((void**)&mom, sizeof(BandMom) * ncell, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->bA, 0, sizeof(float4) * ncell, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->bLc, 0, sizeof(float4) * ncell, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(t->bLs, 0, sizeof(float4) * (ns > 0 ? ns : 1), s);
  if (e == cudaSuccess) {
    t->n_bands = nb;
    if (ns > 0) {
      band_src_kernel<<<grid_of(ns, 256), 256, 0, s>>>(lum_bands, ns, nb, t->src_order,
                                                        reinterpret_cast<float*>(t->bLs));
      note_launch();
    }
    BandArgs A;
    A.nT = t->nT;
    A.nglo = t->nglo;
    A.nghi = t->nghi;
    A.nfirst = t->nfirst;
    A.ncount = t->ncount;
    A.w = t->w;
    A.as = as;
    A.bLs = reinterpret_cast<const float*>(t->bLs);
    A.nW = t->nW;
    A.levels = t->levels;
    A.mom = mom;
    A.bA = reinterpret_cast<float*>(t->bA);
    A.bLc = reinterpret_cast<float*>(t->bLc);
    A.nB = t->nB;
    for (int b = 0; b < nb; ++b) {
      band_alpha_kernel<<<grid_of(n, 256), 256, 0, s>>>(alpha_bands + (size_t)b * n, t->perm, n,
                                                         as, st);
      note_launch();
      A.b = b;
      for (int L = t->max_depth; L >= 0; --L) {
        const int m = t->h_levels[2 * L + 1] - t->h_levels[2 * L];
        band_moments_level_kernel<<<grid_of(m, 128), 128, 0, s>>>(A, L);
        note_launch();
      }
    }
    e = cudaGetLastError();
  }
  if (as) cudaFreeAsync(as, s);
  if (mom) cudaFreeAsync(mom, s);
  cudaEventRecord(e1, s);
  bad = 0;
  cudaMemcpyAsync(&bad, st, sizeof(int), cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  float ms2 = 0.0f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms2, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(st);
  if (e != cudaSuccess || bad) {
    trevr_tree_free(t);
    return e != cudaSuccess ? cuda_to_error(e) : status_to_error(bad);
  }
  if (build_ms) *build_ms = ms + ms2;
  *out = t;
  return TREVR_OK;
}

}  // namespace trevr
