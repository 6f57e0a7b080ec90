// probe.cu -- a measurement helper, not part of the method: the FP64 FMA
// rate of the device, which bounds every FP64 kernel of the step on the
// B300 (its FP64 pipe issues 2 lanes per SM per clock).  The benchmark
// divides its FP64 kernels' algorithmic FLOP rates by the rate this kernel
// reaches on the same device, in the same run.
#include <cuda_runtime.h>

#include "../../include/mpdata.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent FMA chains per thread (hides the latency)

// Each thread runs kProbeChains independent chains a <- a*x + y for iters
// rounds: 2 flops per FMA.  x just below 1 and a small y keep every value
// finite and normal.  The only store happens if a chain hits a value it
// never reaches, so the compiler keeps the work and nothing is written.
__global__ void __launch_bounds__(kProbeThreads)
fp64_fma_probe_kernel(double* __restrict__ out, int iters, double x, double y) {
  double a[kProbeChains];
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) a[q] = 1.0 + 1e-3 * (threadIdx.x + q);
  for (int r = 0; r < iters; ++r) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) a[q] = __fma_rn(a[q], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += a[q];
  if (s == -1.0) out[0] = s;  // never true: the chains stay positive
}

}  // namespace

extern "C" int mpdata_probe_fp64_fma(double* out_dev, int blocks, int iters, void* cuda_stream,
                                     double* flops) {
  if (!out_dev || blocks < 1 || iters < 1 || !flops) return MPDATA_EINVAL;
  fp64_fma_probe_kernel<<<blocks, kProbeThreads, 0, (cudaStream_t)cuda_stream>>>(
      out_dev, iters, 0.9999999, 1e-7);
  if (cudaGetLastError() != cudaSuccess) return MPDATA_ECUDA;
  *flops = 2.0 * kProbeChains * (double)iters * kProbeThreads * (double)blocks;
  return MPDATA_OK;
}
