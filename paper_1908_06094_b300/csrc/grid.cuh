// grid.cuh -- index geometry of the halo-padded fields and the boundary rules.
//
// Every field is [nz+2h][ny+2h][nx+2h], i fastest.  The step kernels never
// read a halo: periodic neighbours in i and j are taken by wrapping the
// interior index, the k neighbours of psi by clamping (edge copy), and the
// vertical faces k = -1/2 and k = nz-1/2 are closed (the boundary factor
// pivbz = 0 of Listing 7), so what the caller leaves in the halos never
// matters.
#pragma once
#include <cstdint>

namespace mpd {

struct Geo {
  int nx, ny, nz, h;
  int64_t px;    // padded row length (elements)
  int64_t pxy;   // padded plane size (elements)
  int64_t off0;  // offset of interior point (0,0,0)
  int64_t total; // padded field size (elements)
};

inline Geo make_geo(int nx, int ny, int nz, int h) {
  Geo g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.h = h;
  g.px = nx + 2 * (int64_t)h;
  g.pxy = g.px * (ny + 2 * (int64_t)h);
  g.off0 = h * g.pxy + h * g.px + h;
  g.total = g.pxy * (nz + 2 * (int64_t)h);
  return g;
}

__host__ __device__ __forceinline__ int64_t at(const Geo& g, int i, int j, int k) {
  return g.off0 + (int64_t)k * g.pxy + (int64_t)j * g.px + i;
}
__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int clampk(int k, int nz) { return k < 0 ? 0 : (k >= nz ? nz - 1 : k); }

// Donor-cell (upwind) flux through a face: left value L, right value R,
// face Courant number C (Listings 4/5).
template <class T>
__device__ __forceinline__ T donor(T L, T R, T C) {
  return fmax(C, T(0)) * L + fmin(C, T(0)) * R;
}

template <class T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 1e-15; };
template <> struct Eps<float> { static constexpr float v = 1e-15f; };

}  // namespace mpd
