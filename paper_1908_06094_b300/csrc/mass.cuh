// mass.cuh -- deterministic FP64 mass sum_interior psi*G (either dtype).
//
// Two levels with a fixed shape: MASS_BLOCKS blocks each own the interior
// rows (j,k) r = b, b + MASS_BLOCKS, ...; a thread owns the points
// i = t, t + 256, ... of each of its block's rows, accumulating in FP64 in
// that fixed order; the block folds its 256 partials in a fixed tree.  One
// more block folds the MASS_BLOCKS partials the same way.  The result does
// not depend on timing, so repeated calls return identical bits.
#pragma once
#include "grid.cuh"

namespace mpd {

constexpr int MASS_BLOCKS = 1184;  // 8 per SM on 148 SMs
constexpr int MASS_THREADS = 256;

__device__ __forceinline__ double block_fold(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] = sh[t] + sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

template <class T>
__global__ void __launch_bounds__(MASS_THREADS)
mass_partial_kernel(Geo g, const T* __restrict__ psi, const T* __restrict__ G,
                    double* __restrict__ part) {
  __shared__ double sh[MASS_THREADS];
  const int rows = g.ny * g.nz;
  double s = 0.0;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int j = r % g.ny, k = r / g.ny;
    const int64_t base = at(g, 0, j, k);
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x)
      s += (double)psi[base + i] * (double)G[base + i];
  }
  double b = block_fold(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

static __global__ void __launch_bounds__(1024)
mass_final_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) s += part[q];
  double b = block_fold(s, sh);
  if (threadIdx.x == 0) *out = b;
}

}  // namespace mpd
