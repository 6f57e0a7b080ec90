// mass.cuh -- deterministic FP64 mass sum_interior psi*G (either dtype).
//
// Two levels with a fixed shape: MASS_BLOCKS blocks each own the interior
// rows (j,k) r = b, b + MASS_BLOCKS, ...; a thread owns the points
// i = t, t + 256, ... of each of its block's rows, accumulating them in that
// fixed order (see MassAcc); the block folds its 256 partials in a fixed
// tree.  One
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

// Per-thread accumulation of psi*G into an FP64 sum.  FP64: one fused
// multiply-add per point.  FP32: the FP64 pipe of the B300 issues 2 lanes
// per SM per clock, so the products are formed exactly as float pairs
// (hi = a*b, lo = fma(a, b, -hi)) and summed in a float-float accumulator
// (Knuth's two-sum on the high parts) over runs of at most 16 points, whose
// total goes into the FP64 sum: the run's error is below 16 * 2^-48 of the
// run's magnitude, far under the FP64 rounding of the final sum.
struct MassAcc64 {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void flush() {}
};
struct MassAcc32 {
  double s = 0.0;
  float hi = 0.f, lo = 0.f;
  int n = 0;
  // every operation explicitly rounded: a contraction of hi + a*b into one
  // fma would break the exactness the two-sum relies on
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b), e = __fmaf_rn(a, b, -p);  // p + e == a*b exactly
    const float t = __fadd_rn(hi, p);                          // two-sum of hi and p
    const float bv = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
    if (++n == 16) flush();
  }
  __device__ __forceinline__ void flush() {
    s += (double)hi + (double)lo;
    hi = lo = 0.f;
    n = 0;
  }
};
template <class T> struct MassAcc;
template <> struct MassAcc<double> { using type = MassAcc64; };
template <> struct MassAcc<float> { using type = MassAcc32; };

template <class T>
__global__ void __launch_bounds__(MASS_THREADS)
mass_partial_kernel(Geo g, const T* __restrict__ psi, const T* __restrict__ G,
                    double* __restrict__ part) {
  __shared__ double sh[MASS_THREADS];
  const int rows = g.ny * g.nz;
  typename MassAcc<T>::type acc;
  // R rows at a time: all their loads are issued before the (fixed-order)
  // accumulation, so each thread keeps 2R loads in flight
  constexpr int R = 4;
  for (int r0 = blockIdx.x; r0 < rows; r0 += R * gridDim.x) {
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      T a[R], b[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = r0 + q * gridDim.x;
        a[q] = b[q] = T(0);
        if (r < rows) {
          const int64_t base = at(g, 0, r % g.ny, r / g.ny);
          a[q] = psi[base + i];
          b[q] = G[base + i];
        }
      }
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (r0 + q * gridDim.x < rows) acc.add(a[q], b[q]);
    }
  }
  acc.flush();
  double b = block_fold(acc.s, sh);
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
