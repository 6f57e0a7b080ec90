// edge.cuh -- the edge-based flux stages of the paper's MPDATA dwarf on a
// structured triangular (octahedral-grid) patch: the upwind flux on edges
// (Listings 4/5), the vertical upwind flux (Listings 6/7), the flux
// divergence over each node's dual cell and the advance (Listing 8).
//
// The patch is nr x nc nodes, periodic in both directions.  Structured
// numbering with direct access (Figs. 9 and 11): node (r, c) and its three
// own edges of colours 0: (r,c)->(r,c+1), 1: (r,c)->(r+1,c), 2:
// (r,c)->(r+1,c+1); a node is the second node of its neighbours' edges
// (r,c-1) colour 0, (r-1,c) colour 1 and (r-1,c-1) colour 2.  No table is
// read: the neighbours are index arithmetic.  Level-major fields:
//   pD, rho [nz][nr][nc];  vn [nz][nr][3][nc];  wn [nz+1][nr][nc] (face k
//   between levels k-1 and k; faces 0 and nz are never read);  vol [nr][nc].
//
// Two organisations (Table 2):
//   staged  four kernels as the four subroutine calls of Listing 8, the
//           edge fluxes, vertical fluxes and divergence through memory;
//   fused   one kernel as the composition of Listing 9: every node-level
//           forms its six edge fluxes and two vertical fluxes on chip.
#pragma once
#include "grid.cuh"

namespace mpd {
namespace edge {

struct Patch {
  int nr, nc, nz;
  int64_t plane;   // nr * nc
  int64_t eplane;  // 3 * nr * nc
};

constexpr int BX = 32, BY = 8;  // node tile of a block: columns x rows

__host__ __device__ inline Patch make_patch(int nr, int nc, int nz) {
  Patch p;
  p.nr = nr; p.nc = nc; p.nz = nz;
  p.plane = (int64_t)nr * nc;
  p.eplane = 3 * p.plane;
  return p;
}

struct Node {
  int r, c, k;
  bool ok;
};

__device__ __forceinline__ Node node_of(const Patch& p) {
  Node n;
  n.c = blockIdx.x * BX + threadIdx.x;
  n.r = blockIdx.y * BY + threadIdx.y;
  n.k = blockIdx.z;
  n.ok = n.c < p.nc && n.r < p.nr;
  return n;
}

__device__ __forceinline__ int up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }

// offsets within a level
__device__ __forceinline__ int64_t nidx(const Patch& p, int r, int c) { return (int64_t)r * p.nc + c; }
__device__ __forceinline__ int64_t eidx(const Patch& p, int r, int col, int c) {
  return ((int64_t)r * 3 + col) * p.nc + c;
}

// ---------------------------------------------------------------- staged --

// compute_upwind_flux (Listing 5): the three own edges of every node-level.
template <class T>
__global__ void __launch_bounds__(BX * BY)
edge_flux_kernel(Patch p, const T* __restrict__ pD, const T* __restrict__ vn,
                 T* __restrict__ flux) {
  const Node n = node_of(p);
  if (!n.ok) return;
  const T* P = pD + n.k * p.plane;
  const int rp = up(n.r, p.nr), cp = up(n.c, p.nc);
  const T ps = P[nidx(p, n.r, n.c)];
  const T pn[3] = {P[nidx(p, n.r, cp)], P[nidx(p, rp, n.c)], P[nidx(p, rp, cp)]};
  const int64_t eb = n.k * p.eplane;
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const int64_t e = eb + eidx(p, n.r, col, n.c);
    flux[e] = donor(ps, pn[col], vn[e]);
  }
}

// compute_upwind_fluz (Listing 7): faces 1..nz-1 upwind, the boundary faces
// pivbz times their adjacent interior face's flux.  Launched over nz+1 faces.
template <class T>
__global__ void __launch_bounds__(BX * BY)
edge_fluz_kernel(Patch p, const T* __restrict__ pD, const T* __restrict__ W, T pivbz,
                 T* __restrict__ fluz) {
  const Node n = node_of(p);
  if (!n.ok) return;
  const int64_t q = nidx(p, n.r, n.c);
  const int kf = n.k == 0 ? 1 : (n.k == p.nz ? p.nz - 1 : n.k);  // the face computed
  const T f = donor(pD[(kf - 1) * p.plane + q], pD[kf * p.plane + q], W[kf * p.plane + q]);
  fluz[n.k * p.plane + q] = (kf == n.k) ? f : pivbz * f;
}

// compute_fluxdiv: the signed sum of the six edge fluxes (own edges leave
// the node, the neighbours' enter it) and the vertical flux difference,
// over the dual volume.
template <class T>
__global__ void __launch_bounds__(BX * BY)
edge_fluxdiv_kernel(Patch p, const T* __restrict__ flux, const T* __restrict__ fluz,
                    const T* __restrict__ vol, T* __restrict__ div) {
  const Node n = node_of(p);
  if (!n.ok) return;
  const int rm = dn(n.r, p.nr), cm = dn(n.c, p.nc);
  const T* F = flux + n.k * p.eplane;
  const int64_t q = nidx(p, n.r, n.c);
  T s = F[eidx(p, n.r, 0, n.c)];
  s = s + F[eidx(p, n.r, 1, n.c)];
  s = s + F[eidx(p, n.r, 2, n.c)];
  s = s - F[eidx(p, n.r, 0, cm)];
  s = s - F[eidx(p, rm, 1, n.c)];
  s = s - F[eidx(p, rm, 2, cm)];
  s = s + (fluz[(n.k + 1) * p.plane + q] - fluz[n.k * p.plane + q]);
  div[n.k * p.plane + q] = s * rcp(vol[q]);
}

// advance_solution: pD = pD - divVD / rho (out of place).
template <class T>
__global__ void __launch_bounds__(BX * BY)
edge_advance_kernel(Patch p, const T* __restrict__ pD, const T* __restrict__ div,
                    const T* __restrict__ rho, T* __restrict__ out) {
  const Node n = node_of(p);
  if (!n.ok) return;
  const int64_t q = n.k * p.plane + nidx(p, n.r, n.c);
  out[q] = pD[q] - div[q] * rcp(rho[q]);
}

// ----------------------------------------------------------------- fused --

// The four stages in one pass (the composition of Listing 9), one thread
// per node-level: the six edge fluxes and the two vertical fluxes are
// formed in registers and summed at once, and only the new pD is stored.
// The kernel is bound by memory: a node-level's loads are its own pD, vn
// and rho, the W faces below and above, and pD one level below and above;
// an in-plane neighbour's pD is fetched only in the lanes whose flux takes
// it (a predicated load after the velocity's sign is known), which halves
// that traffic through L1 (measured: 53 us against 63 us with every
// neighbour loaded, FP32, 71424 x 80).  Products are folded into the flux
// sum with FMAs; one reciprocal of vol rho (FP64 is bound by its pipe here).  Boundary faces: face 0 carries pivbz times face 1's flux, face nz
// pivbz times face nz-1's (nz >= 2).
template <class T>
__global__ void __launch_bounds__(BX * BY)
edge_fused_kernel(Patch p, const T* __restrict__ pD, const T* __restrict__ vn,
                  const T* __restrict__ W, const T* __restrict__ rho,
                  const T* __restrict__ vol, T pivbz, T* __restrict__ out) {
  const Node n = node_of(p);
  if (!n.ok) return;
  const int k = n.k, nz = p.nz;
  const int rp = up(n.r, p.nr), cp = up(n.c, p.nc);
  const int rm = dn(n.r, p.nr), cm = dn(n.c, p.nc);
  const int64_t q = nidx(p, n.r, n.c);
  const T* P = pD + k * p.plane;
  const T* V = vn + k * p.eplane;
  const T ps = P[q];
  // own edges: this node is upwind where vn >= 0
  const T v0 = V[eidx(p, n.r, 0, n.c)], v1 = V[eidx(p, n.r, 1, n.c)];
  const T v2 = V[eidx(p, n.r, 2, n.c)];
  const T o0 = nonneg(v0) ? ps : P[nidx(p, n.r, cp)];
  const T o1 = nonneg(v1) ? ps : P[nidx(p, rp, n.c)];
  const T o2 = nonneg(v2) ? ps : P[nidx(p, rp, cp)];
  // the neighbours' edges ending at this node
  const T u0 = V[eidx(p, n.r, 0, cm)], u1 = V[eidx(p, rm, 1, n.c)];
  const T u2 = V[eidx(p, rm, 2, cm)];
  const T i0 = nonneg(u0) ? P[nidx(p, n.r, cm)] : ps;
  const T i1 = nonneg(u1) ? P[nidx(p, rm, n.c)] : ps;
  const T i2 = nonneg(u2) ? P[nidx(p, rm, cm)] : ps;
  T s = v0 * o0;
  s = fma_rn(v1, o1, s);
  s = fma_rn(v2, o2, s);
  s = fma_rn(-u0, i0, s);
  s = fma_rn(-u1, i1, s);
  s = fma_rn(-u2, i2, s);
  // face k below (levels k-1, k) and face k+1 above (levels k, k+1); at
  // k = 0 the face below is pivbz times face 1, at k = nz-1 the face above
  // is pivbz times face nz-1.  The levels above and below are loaded
  // unconditionally, in parallel with W.
  const int kb = k > 0 ? k : 1, ka = k < nz - 1 ? k + 1 : nz - 1;
  const T wb = W[kb * p.plane + q], wa = W[ka * p.plane + q];
  const T pm = pD[(k > 0 ? k - 1 : 1) * p.plane + q];
  const T pu = pD[(k < nz - 1 ? k + 1 : nz - 2) * p.plane + q];
  T fb = (k > 0) ? wb * (nonneg(wb) ? pm : ps) : wb * (nonneg(wb) ? ps : pm);
  T fa = (k < nz - 1) ? wa * (nonneg(wa) ? ps : pu) : wa * (nonneg(wa) ? pu : ps);
  if (k == 0) fb = pivbz * fb;
  if (k == nz - 1) fa = pivbz * fa;
  s = s + (fa - fb);
  const int64_t o = k * p.plane + q;
  out[o] = fma_rn(-s, rcp(vol[q] * rho[o]), ps);
}

// FP32 with nc a multiple of 4: one thread per four consecutive nodes of a
// row (columns c0..c0+3, c0 = 4 x thread column) and one level.  The rows
// it reads are 16-byte vectors (its own four values), and only the columns
// c0-1 and c0+4 of the neighbouring rows are single loads: a fifth of the
// load instructions of the one-node kernel for the same bytes.  The
// arithmetic per node is that kernel's, in the same order.
constexpr int BX4 = 32;  // threads per block row: 128 columns

__device__ __forceinline__ float f4(const float4& v, int j) {
  return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

__global__ void __launch_bounds__(BX4 * BY)
edge_fused4_kernel(Patch p, const float* __restrict__ pD, const float* __restrict__ vn,
                   const float* __restrict__ W, const float* __restrict__ rho,
                   const float* __restrict__ vol, float pivbz, float* __restrict__ out) {
  const int c0 = 4 * (blockIdx.x * BX4 + threadIdx.x);
  const int r = blockIdx.y * BY + threadIdx.y, k = blockIdx.z, nz = p.nz;
  if (c0 >= p.nc || r >= p.nr) return;
  const int rp = up(r, p.nr), rm = dn(r, p.nr);
  const int cl = c0 == 0 ? p.nc - 1 : c0 - 1, cr = c0 + 4 == p.nc ? 0 : c0 + 4;
  const float* P = pD + k * p.plane;
  const float* V = vn + k * p.eplane;
  auto ld4 = [](const float* a, int64_t i) { return *reinterpret_cast<const float4*>(a + i); };
  // pD: own row, the row above (r+1) and below (r-1), and their end columns
  const float4 pr = ld4(P, nidx(p, r, c0)), pu = ld4(P, nidx(p, rp, c0));
  const float4 pdn = ld4(P, nidx(p, rm, c0));
  const float prL = P[nidx(p, r, cl)], prR = P[nidx(p, r, cr)];
  const float puR = P[nidx(p, rp, cr)], pdL = P[nidx(p, rm, cl)];
  // vn: own colours 0..2 (row r), colour 1 and 2 of row r-1, and the end
  // columns of colour 0 (row r) and colour 2 (row r-1)
  const float4 a0 = ld4(V, eidx(p, r, 0, c0)), a1 = ld4(V, eidx(p, r, 1, c0));
  const float4 a2 = ld4(V, eidx(p, r, 2, c0));
  const float4 b1 = ld4(V, eidx(p, rm, 1, c0)), b2 = ld4(V, eidx(p, rm, 2, c0));
  const float a0L = V[eidx(p, r, 0, cl)], b2L = V[eidx(p, rm, 2, cl)];
  // vertical: faces k (below) and k+1 (above) and the levels they join
  const int kb = k > 0 ? k : 1, ka = k < nz - 1 ? k + 1 : nz - 1;
  const float4 wb = ld4(W, kb * p.plane + nidx(p, r, c0));
  const float4 wa = ld4(W, ka * p.plane + nidx(p, r, c0));
  const float4 pbl = ld4(pD, (k > 0 ? k - 1 : 1) * p.plane + nidx(p, r, c0));
  const float4 pal = ld4(pD, (k < nz - 1 ? k + 1 : nz - 2) * p.plane + nidx(p, r, c0));
  const float4 rh = ld4(rho, k * p.plane + nidx(p, r, c0));
  const float4 vo = ld4(vol, nidx(p, r, c0));
  float res[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float ps = f4(pr, j);
    // own edges' second nodes: (r, c+1), (r+1, c), (r+1, c+1)
    const float n0 = j < 3 ? f4(pr, j + 1) : prR;
    const float n1 = f4(pu, j);
    const float n2 = j < 3 ? f4(pu, j + 1) : puR;
    // incoming edges: colour 0 from (r, c-1), 1 from (r-1, c), 2 from (r-1, c-1)
    const float u0 = j > 0 ? f4(a0, j - 1) : a0L;
    const float u1 = f4(b1, j);
    const float u2 = j > 0 ? f4(b2, j - 1) : b2L;
    const float m0 = j > 0 ? f4(pr, j - 1) : prL;
    const float m1 = f4(pdn, j);
    const float m2 = j > 0 ? f4(pdn, j - 1) : pdL;
    const float v0 = f4(a0, j), v1 = f4(a1, j), v2 = f4(a2, j);
    float s = v0 * (nonneg(v0) ? ps : n0);
    s = fma_rn(v1, nonneg(v1) ? ps : n1, s);
    s = fma_rn(v2, nonneg(v2) ? ps : n2, s);
    s = fma_rn(-u0, nonneg(u0) ? m0 : ps, s);
    s = fma_rn(-u1, nonneg(u1) ? m1 : ps, s);
    s = fma_rn(-u2, nonneg(u2) ? m2 : ps, s);
    const float w_b = f4(wb, j), w_a = f4(wa, j);
    float fb, fa;
    if (k > 0) fb = w_b * (nonneg(w_b) ? f4(pbl, j) : ps);
    else fb = w_b * (nonneg(w_b) ? ps : f4(pbl, j));
    if (k < nz - 1) fa = w_a * (nonneg(w_a) ? ps : f4(pal, j));
    else fa = w_a * (nonneg(w_a) ? f4(pal, j) : ps);
    if (k == 0) fb = pivbz * fb;
    if (k == nz - 1) fa = pivbz * fa;
    s = s + (fa - fb);
    res[j] = fma_rn(-s, rcp(f4(vo, j) * f4(rh, j)), ps);
  }
  *reinterpret_cast<float4*>(out + k * p.plane + nidx(p, r, c0)) =
      make_float4(res[0], res[1], res[2], res[3]);
}

}  // namespace edge
}  // namespace mpd
