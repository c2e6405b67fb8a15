// Adjoint of the flux (differentiation with the decisions of the forward pass
// frozen): from the per-cell accumulators of the adjoint walk to the gradients
// with respect to the source luminosities and the particle absorption
// coefficients, in the caller's order.
//
//   dLoss/dL_j   = e_j + sum over the cells C holding source j (its leaf and
//                  every ancestor) of a_C + b_C . (y_j - c_C)
//                  (a merged source sits at the centre of luminosity c_C, which
//                  moves as dc_C/dL_j = (y_j - c_C) / L_C)
//   dLoss/dalpha_i = w_i * sum over the cells X holding particle i of G_X / W_X
//                  (the mean absorption of X is sum(w alpha) / W_X)
#include <cuda_runtime.h>

#include "trevr_internal.cuh"

namespace trevr {
namespace {

__global__ void lum_grad_kernel(int n_src, const float4* __restrict__ src,
                                const int* __restrict__ src_order, const int* __restrict__ src_leaf,
                                const int4* __restrict__ nT, const float4* __restrict__ nS,
                                const double* __restrict__ a, const double* __restrict__ b,
                                const double* __restrict__ e, float* grad_lum) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_src) return;
  const float4 y = src[k];
  double g = e[k];
  int C = src_leaf[k];
  for (int it = 0; it < kMaxLevels && C > 0; ++it) {
    const float4 c = nS[C];
    g += a[C] + b[3 * C] * (double)(y.x - c.x) + b[3 * C + 1] * (double)(y.y - c.y) +
         b[3 * C + 2] * (double)(y.z - c.z);
    C = nT[C].y;
  }
  grad_lum[src_order[k]] = (float)g;
}

// H_X = H_parent + G_X / W_X for the cells of one level (top-down).
__global__ void alpha_prefix_kernel(const int* __restrict__ levels, int L,
                                    const int4* __restrict__ nT, const double* __restrict__ G,
                                    const double* __restrict__ W, double* H) {
  const int begin = levels[2 * L], end = levels[2 * L + 1];
  for (int X = begin + blockIdx.x * blockDim.x + threadIdx.x; X < end;
       X += gridDim.x * blockDim.x) {
    const int par = nT[X].y;
    H[X] = (par > 0 ? H[par] : 0.0) + G[X] / W[X];
  }
}

__global__ void alpha_grad_kernel(int n, const int* __restrict__ leaf_of,
                                  const int* __restrict__ perm, const float* __restrict__ w,
                                  const double* __restrict__ H, float* grad_alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  grad_alpha[perm[i]] = (float)((double)w[i] * H[leaf_of[i]]);
}

}  // namespace

cudaError_t adjoint_finalize(const trevr_tree* t, const AdjointArgs& J, float* grad_lum,
                             float* grad_alpha, double* H, cudaStream_t s) {
  const int ns = (int)t->n_src, n = (int)t->n_gas;
  if (ns > 0) {
    lum_grad_kernel<<<(ns + 127) / 128, 128, 0, s>>>(ns, t->src, t->src_order, t->src_leaf, t->nT,
                                                     t->nS, J.a, J.b, J.e, grad_lum);
    note_launch();
  }
  for (int L = 0; L <= t->max_depth; ++L) {
    const int m = t->h_levels[2 * L + 1] - t->h_levels[2 * L];
    int blocks = (m + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    alpha_prefix_kernel<<<blocks, 256, 0, s>>>(t->levels, L, t->nT, J.G, t->nW, H);
    note_launch();
  }
  alpha_grad_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, t->leaf_of, t->perm, t->w, H, grad_alpha);
  note_launch();
  return cudaGetLastError();
}

}  // namespace trevr
