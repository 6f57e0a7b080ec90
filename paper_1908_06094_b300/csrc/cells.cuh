// cells.cuh -- the cell-neighbour reduction of Table 1 (the on_cells
// operation of Fig. 5): for every cell s and level k,
//   B[k][s] = fac * (A[k][n0] + A[k][n1] + A[k][n2]),
// n0..n2 the cells across s's three edges, summed in that order.  Fields are
// level-major [nz][ncells] in the numbering's storage order.
//
// Two access methods (Sec. 3.2):
//   direct (DA)   structured numbering (row, colour, column) ->
//                 (2 r + colour) nc + c of a periodic nr x nc patch; the
//                 neighbours are index arithmetic: U(r,c) borders D(r-1,c),
//                 D(r,c+1), D(r,c); D(r,c) borders U(r,c), U(r+1,c), U(r,c-1);
//   indirect (IA) a neighbour table [3][ncells] (int32) in any numbering.
// A thread owns one cell and a chunk of levels: the neighbour indices are
// found (or read) once and every level's three loads are independent.
#pragma once
#include <cstdint>

namespace mpd {
namespace cells {

constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads)
cells_sum_direct_kernel(int nr, int nc, int nz, int kc, const T* __restrict__ A,
                        T* __restrict__ B, T fac) {
  const int64_t ncells = 2LL * nr * nc;
  const int64_t s = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (s >= ncells) return;
  const int c = (int)(s % nc);
  const int rk = (int)(s / nc);
  const int colour = rk & 1, r = rk >> 1;
  const int rm = r == 0 ? nr - 1 : r - 1, rp = r + 1 == nr ? 0 : r + 1;
  const int cm = c == 0 ? nc - 1 : c - 1, cp = c + 1 == nc ? 0 : c + 1;
  auto id = [&](int rr, int k, int cc) { return ((int64_t)(2 * rr + k)) * nc + cc; };
  int64_t n0, n1, n2;
  if (colour == 0) { n0 = id(rm, 1, c); n1 = id(r, 1, cp); n2 = id(r, 1, c); }
  else             { n0 = id(r, 0, c);  n1 = id(rp, 0, c); n2 = id(r, 0, cm); }
  const int k0 = blockIdx.y * kc, k1 = min(nz, k0 + kc);
  for (int k = k0; k < k1; ++k) {
    const T* a = A + k * ncells;
    B[k * ncells + s] = (a[n0] + a[n1] + a[n2]) * fac;
  }
}

template <class T>
__global__ void __launch_bounds__(kThreads)
cells_sum_table_kernel(int64_t ncells, int nz, int kc, const int* __restrict__ t,
                       const T* __restrict__ A, T* __restrict__ B, T fac) {
  const int64_t s = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (s >= ncells) return;
  const int64_t n0 = t[s], n1 = t[ncells + s], n2 = t[2 * ncells + s];
  const int k0 = blockIdx.y * kc, k1 = min(nz, k0 + kc);
  for (int k = k0; k < k1; ++k) {
    const T* a = A + k * ncells;
    B[k * ncells + s] = (a[n0] + a[n1] + a[n2]) * fac;
  }
}

}  // namespace cells
}  // namespace mpd
