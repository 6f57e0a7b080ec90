// mass.cuh -- deterministic FP64 mass sum_interior psi*G (either dtype).
//
// Two levels with a fixed shape: MASS_BLOCKS blocks each own the interior
// rows (j,k) r = b, b + MASS_BLOCKS, ...; a thread owns the points
// i = t, t + 256, ... of each of its block's rows, accumulating them in a
// fixed order (see MassAcc); the block folds its 256 partials in a fixed
// tree.  One
// more block folds the MASS_BLOCKS partials the same way.  The result does
// not depend on timing, so repeated calls return identical bits.
#pragma once
#include "grid.cuh"

namespace mpd {

constexpr int MASS_BLOCKS = 1184;  // 8 per SM on 148 SMs
constexpr int MASS_THREADS = 256;

// The block's sum in a fixed order, valid in thread 0: lane l of the first
// warp adds the values of threads l, l + 32, l + 64, ... in turn, then the
// 32 lane sums fold pairwise by shuffles.  Only the first warp adds: a tree
// over shared memory had its per-level adds if-converted into every thread,
// log2(n) FP64 adds a thread on the slow FP64 pipe.  blockDim.x is a
// multiple of 32.
__device__ __forceinline__ double block_fold(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  double s = 0.0;
  if (t < 32) {
    s = sh[t];
    for (int q = t + 32; q < (int)blockDim.x; q += 32) s += sh[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// Per-thread accumulation of psi*G into an FP64 sum.  FP64: one fused
// multiply-add per point.  FP32: the FP64 pipe of the B300 issues 2 lanes
// per SM per clock, so the products are formed exactly as float pairs
// (hi = a*b, lo = fma(a, b, -hi)) and summed in a float-float accumulator
// (Knuth's two-sum on the high parts) over one group of at most
// MassAcc<float>::R points, whose total then goes into the FP64 sum: the
// group's error is below R * 2^-48 of its magnitude, far under the FP64
// rounding of the final sum.  The flush is unconditional code after each
// group, so the FP64 work is two conversions and two adds per R points.
struct MassAcc64 {
  static constexpr int R = 4;
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ void flush() {}
};
struct MassAcc32 {
  static constexpr int R = 16;
  double s = 0.0;
  float hi = 0.f, lo = 0.f;
  // every operation explicitly rounded: a contraction of hi + a*b into one
  // fma would break the exactness the two-sum relies on.  A padded point
  // (a = b = 0) leaves hi and lo unchanged.
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b), e = __fmaf_rn(a, b, -p);  // p + e == a*b exactly
    const float t = __fadd_rn(hi, p);                          // two-sum of hi and p
    const float bv = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ void flush() {
    s += (double)hi + (double)lo;
    hi = lo = 0.f;
  }
};
template <class T> struct MassAcc;
template <> struct MassAcc<double> { using type = MassAcc64; };
template <> struct MassAcc<float> { using type = MassAcc32; };

// A block takes the interior rows r0 + q*gridDim.x (q < R) of each group in
// turn; the row bases are computed once per group and all 2R loads of a
// point column are issued before its (fixed-order) accumulation.  Rows past
// the end are skipped (a block-uniform test).
// V2: a thread takes two adjacent points of a row with one 2-element load
// of each field (rows start on an even element: nx and h even), adding the
// second point only inside the interior (the load past the last interior
// point reads the first halo element, which is not added).
template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <class T, bool V2 = false>
__global__ void __launch_bounds__(MASS_THREADS)
mass_partial_kernel(Geo g, const T* __restrict__ psi, const T* __restrict__ G,
                    double* __restrict__ part) {
  pdl_enter();
  __shared__ double sh[MASS_THREADS];
  using Acc = typename MassAcc<T>::type;
  // (V2: half the rows a group, so a group still adds at most Acc::R points)
  constexpr int R = V2 ? (Acc::R / 2 > 0 ? Acc::R / 2 : 1) : Acc::R;
  const int rows = g.ny * g.nz;
  // row r is (j, k) = (r % ny, r / ny); a step of gridDim.x rows moves (j, k)
  // by (dj, dk) with one carry, so only the first row takes a division
  const int dj = (int)(gridDim.x % g.ny), dk = (int)(gridDim.x / g.ny);
  int j = (int)(blockIdx.x % g.ny), k = (int)(blockIdx.x / g.ny);
  Acc acc;
  for (int r0 = blockIdx.x; r0 < rows; r0 += R * gridDim.x) {
    int64_t base[R];
    bool ok[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      ok[q] = r0 + q * (int)gridDim.x < rows;
      base[q] = ok[q] ? at(g, 0, j, k) : 0;
      j += dj;
      k += dk;
      if (j >= g.ny) {
        j -= g.ny;
        ++k;
      }
    }
    if constexpr (V2) {
      using V = typename Vec2<T>::type;
      for (int i = 2 * threadIdx.x; i < g.nx; i += 2 * blockDim.x) {
        const bool two = i + 1 < g.nx;
        V a[R], b[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          a[q] = ok[q] ? *reinterpret_cast<const V*>(psi + base[q] + i) : V{T(0), T(0)};
          b[q] = ok[q] ? *reinterpret_cast<const V*>(G + base[q] + i) : V{T(0), T(0)};
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
          if (ok[q]) {  // rows past the end add nothing
            acc.add(a[q].x, b[q].x);
            if (two) acc.add(a[q].y, b[q].y);
          }
        }
        acc.flush();
      }
    } else {
      for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
        T a[R], b[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
          a[q] = ok[q] ? psi[base[q] + i] : T(0);
          b[q] = ok[q] ? G[base[q] + i] : T(0);
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
          if (ok[q]) acc.add(a[q], b[q]);  // rows past the end add nothing
        acc.flush();
      }
    }
  }
  double b = block_fold(acc.s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

static __global__ void __launch_bounds__(1024)
mass_final_kernel(const double* __restrict__ part, int np, double* __restrict__ out) {
  pdl_enter();
  __shared__ double sh[1024];
  double s = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) s += part[q];
  double b = block_fold(s, sh);
  if (threadIdx.x == 0) *out = b;
}

// The first level of the reduction: the two-point form where every row
// starts on an even element (nx and h even; the fields are 16-byte aligned).
template <class T>
inline void mass_partial_launch(const Geo& g, const T* psi, const T* G, double* part,
                                cudaStream_t s, bool pdl = false) {
  auto k = (g.nx % 2 == 0 && g.h % 2 == 0) ? mass_partial_kernel<T, true>
                                           : mass_partial_kernel<T, false>;
  if (pdl) launch_pdl(k, MASS_BLOCKS, MASS_THREADS, 0, s, g, psi, G, part);
  else k<<<MASS_BLOCKS, MASS_THREADS, 0, s>>>(g, psi, G, part);
}

}  // namespace mpd
