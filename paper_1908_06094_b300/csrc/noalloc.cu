// noalloc.cu -- mpdata_mass_noalloc: the mass reduction for callers that
// cannot allocate device memory.
//
// mpdata_mass needs a context, and creating a context calls cudaMalloc for
// the step's scratch.  Some callers cannot do that: applications whose
// device memory is entirely handed out by their own pool or arena, and
// hosts that forbid allocation after start-up (real-time or certified
// codes).  This entry point needs no context: its only scratch,
// the per-block partial sums of the two-level reduction, lives in the
// file-scope array below, which every GPU that loads the library keeps
// until the process exits.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>

#include "../../include/mpdata.h"
#include "grid.cuh"
#include "mass.cuh"

namespace {

// The reduction's scratch: one FP64 partial per block of the first level
// (MPDATA_MASS_NOALLOC_PARTIALS entries, 9472 bytes).  Every call writes
// all of it before reading it, so nothing needs clearing between calls.
static_assert(mpd::MASS_BLOCKS == MPDATA_MASS_NOALLOC_PARTIALS,
              "the header states the scratch size");
static __device__ __align__(256) double g_mass_partials[mpd::MASS_BLOCKS];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
double* g_partials_addr[kMaxDevices] = {};

// Device address of g_mass_partials on the current device, looked up once
// per device (in host code the array's name is only a stand-in) and kept for
// the life of the process: a cudaDeviceReset of that device makes the kept
// address stale, which the header states.
int partials_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MPDATA_EDEVICE;
  }
  if (dev < 0 || dev >= kMaxDevices) return MPDATA_EDEVICE;
  std::lock_guard<std::mutex> lock(g_setup_lock);
  if (!g_partials_addr[dev]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_mass_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return MPDATA_ECUDA;
    }
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return MPDATA_OK;
}

template <class T>
int launch(const mpd::Geo& g, const T* psi, const T* G, double* part, double* out,
           cudaStream_t s) {
  mpd::mass_partial_launch<T>(g, psi, G, part, s);
  mpd::mass_final_kernel<<<1, 1024, 0, s>>>(part, mpd::MASS_BLOCKS, out);
  if (cudaGetLastError() != cudaSuccess) return MPDATA_ECUDA;
  return MPDATA_OK;
}

}  // namespace

extern "C" int mpdata_mass_noalloc(const void* psi, const void* g, int nx, int ny, int nz,
                                   int halo, int dtype, double* out_dev, void* cuda_stream) {
  if (!psi || !g || !out_dev) return MPDATA_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1 || halo < 0) return MPDATA_EINVAL;
  if (dtype != MPDATA_F64 && dtype != MPDATA_F32) return MPDATA_EINVAL;
  if ((reinterpret_cast<uintptr_t>(psi) & 15u) || (reinterpret_cast<uintptr_t>(g) & 15u) ||
      (reinterpret_cast<uintptr_t>(out_dev) & 7u))
    return MPDATA_EALIGN;
  // the reduction indexes rows (j,k) and padded planes with 32-bit integers;
  // its row counter runs up to 16 x MASS_BLOCKS rows past the last row
  static_assert(MPDATA_MASS_NOALLOC_MAX_ROWS + 16LL * mpd::MASS_BLOCKS <= (long long)INT_MAX,
                "the row bound leaves the row counter's margin");
  if ((int64_t)ny * nz > MPDATA_MASS_NOALLOC_MAX_ROWS) return MPDATA_ERANGE;
  if ((int64_t)(nx + 2 * (int64_t)halo) * (ny + 2 * (int64_t)halo) > (int64_t)INT_MAX)
    return MPDATA_ERANGE;
  double* part = nullptr;
  int rc = partials_for_current_device(&part);
  if (rc) return rc;
  const mpd::Geo geo = mpd::make_geo(nx, ny, nz, halo);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (dtype == MPDATA_F64)
    return launch<double>(geo, (const double*)psi, (const double*)g, part, out_dev, s);
  return launch<float>(geo, (const float*)psi, (const float*)g, part, out_dev, s);
}
