// exchange.cuh -- pack and unpack the halo strips of one slab of an i-j
// decomposed domain (the halo exchange that Sec. 3.1.1, item 2, lists as a
// library component; the domain decomposition of Fig. 8).
//
// A slab is a padded grid whose i-j halo belongs to its neighbours.  Its
// step reads that halo instead of wrapping (Geo::openij), so before a step
// the halo of psi must hold the neighbours' edge values, to the depth the
// step reads (3 for the one-kernel step).  Face f of a slab: 0 = -x, 1 = +x,
// 2 = -y, 3 = +y.  pack(f) copies the h-deep interior strip next to face f
// into a contiguous buffer; the neighbour across f receives it and
// unpack(f ^ 1) writes it into its halo strip beyond face f ^ 1.  The x faces
// carry interior rows only (j in [0, ny)); the y faces carry whole padded
// rows (i in [-h, nx + h)), so running the x exchange first and the y one
// second fills the corners of the halo too.  Levels k in [0, nz): the step
// takes its vertical neighbours by clamping or wrapping k, never from the
// k halo.
//
// Buffer layout: [nz][rows][cols] with (rows, cols) = (ny, h) for an x
// face and (h, nx + 2h) for a y face.
#pragma once
#include "grid.cuh"

namespace mpd {
namespace xch {

struct Strip {
  int i0, j0;      // first (i, j) of the strip (interior coordinates)
  int rows, cols;  // extent in j and in i
  int64_t n;       // elements: nz * rows * cols
};

// The strip a slab sends across face f (pack) or receives beyond face f
// (unpack).
__host__ __device__ inline Strip strip(const Geo& g, int face, bool unpack) {
  Strip s;
  const int h = g.h;
  if (face < 2) {  // x faces: interior rows
    s.rows = g.ny;
    s.cols = h;
    s.j0 = 0;
    if (face == 0) s.i0 = unpack ? -h : 0;
    else s.i0 = unpack ? g.nx : g.nx - h;
  } else {  // y faces: whole padded rows, corners included
    s.rows = h;
    s.cols = g.nx + 2 * h;
    s.i0 = -h;
    if (face == 2) s.j0 = unpack ? -h : 0;
    else s.j0 = unpack ? g.ny : g.ny - h;
  }
  s.n = (int64_t)g.nz * s.rows * s.cols;
  return s;
}

// One thread per element (grid-stride); UNPACK: buffer -> field, else
// field -> buffer.  Reads and writes are contiguous along a strip row.
template <class T, bool UNPACK>
__global__ void __launch_bounds__(256)
strip_kernel(Geo g, Strip s, const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t per_level = (int64_t)s.rows * s.cols;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < s.n;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / per_level);
    const int64_t r = q - k * per_level;
    const int j = s.j0 + (int)(r / s.cols);
    const int i = s.i0 + (int)(r % s.cols);
    const int64_t f = at(g, i, j, k);
    if (UNPACK) dst[f] = src[q];
    else dst[q] = src[f];
  }
}

}  // namespace xch
}  // namespace mpd
