// fused.cuh -- the whole MPDATA step (iord = 2) in one kernel.
//
// The fused organisation of Listing 9 and Table 2 ("with fusion"): every
// intermediate of the step -- the donor-cell solution psi1, the three
// pseudo-velocity fields, the limiter's beta-up/beta-down and the limited
// face fluxes -- lives in shared memory; device memory sees only the five
// inputs (psi^n, U, V, W, G) and the output psi^(n+1).
//
// Each CTA owns a TX x TY column tile and marches k upward (the "forward"
// vertical sweep of Listing 9).  At iteration t it runs five stages, each on
// the smallest horizontal region the next stage needs (the tile widened by
// the stencil radius still to come):
//   A  psi1 on plane t+2, tile + 2 ring      (donor cell from psi^n, U,V,W,G)
//   B  Ut, Vt on plane t+1 and Wt on face t+3/2, on the faces around tile+1
//   C  bounds and beta on plane t+1, tile + 1
//   D  limited donor fluxes of plane t (x and y faces) and face t+1/2
//   E  psi^(n+1) on plane t = psi1 - (1/G) sum dF, with its halo images.
// psi1 is kept for four planes, the other intermediates for two, in
// shared-memory rings.  Periodic neighbours come from a per-CTA table of
// wrapped column offsets, so the inputs' halos are never read.
//
// A CTA may own only the levels [k0, k1) of its columns (blockIdx.z); it
// then starts five iterations early to rebuild the intermediates its first
// planes need.  Output must not alias psi^n: neighbouring CTAs still read
// psi^n at planes this CTA has already written.
#pragma once
#include "grid.cuh"

namespace mpd {
namespace fused {

template <class T, int TX, int TY>
struct Layout {
  static constexpr int SX = TX + 4, SY = TY + 4, SN = SX * SY;  // radius-2 planes
  static constexpr int CX = TX + 6, CY = TY + 6, CN = CX * CY;  // radius-3 columns
  static constexpr int P1 = 0;            // psi1, 4 planes
  static constexpr int UT = P1 + 4 * SN;  // Ut, 2 planes
  static constexpr int VT = UT + 2 * SN;  // Vt, 2 planes
  static constexpr int WT = VT + 2 * SN;  // Wt, 2 faces
  static constexpr int BU = WT + 2 * SN;  // beta-up, 2 planes
  static constexpr int BD = BU + 2 * SN;  // beta-down, 2 planes
  static constexpr int FX = BD + 2 * SN;  // x-face fluxes of the output plane
  static constexpr int FY = FX + SN;      // y-face fluxes
  static constexpr int FZ = FY + SN;      // z-face fluxes, 2 faces
  static constexpr int NVAL = FZ + 2 * SN;
  static constexpr size_t bytes = NVAL * sizeof(T) + CN * sizeof(int);
};

// One tile of the step: columns [i0, i0+TX) x [j0, j0+TY), levels [k0, k1),
// psi^n P0 -> out.  Called by every thread of the CTA; smem_raw holds
// Layout::bytes.  Starts with a barrier, so consecutive calls from one CTA
// (the persistent batched kernel) may reuse the shared memory.
template <class T, int TX, int TY, int NT, bool LIMIT>
__device__ __forceinline__ void step_tile(const Geo& g, int i0, int j0, int k0, int k1,
                                          const T* __restrict__ P0, const T* __restrict__ U,
                                          const T* __restrict__ V, const T* __restrict__ W,
                                          const T* __restrict__ G, T* __restrict__ out,
                                          unsigned char* smem_raw) {
  using L = Layout<T, TX, TY>;
  T* sm = reinterpret_cast<T*>(smem_raw);
  int* col = reinterpret_cast<int*>(sm + L::NVAL);
  const int tid = threadIdx.x;
  const int nz = g.nz;
  __syncthreads();
  const T eps = Eps<T>::v, zero = T(0);

  // wrapped column offsets (j*px + i) of the tile + 3 ring
  for (int q = tid; q < L::CN; q += NT) {
    int i = i0 + q % L::CX - 3, j = j0 + q / L::CX - 3;
    i = ((i % g.nx) + g.nx) % g.nx;
    j = ((j % g.ny) + g.ny) % g.ny;
    col[q] = j * (int)g.px + i;
  }
  __syncthreads();
  auto C = [&](int x, int y) { return col[(y + 3) * L::CX + (x + 3)]; };
  auto S = [&](int x, int y) { return (y + 2) * L::SX + (x + 2); };
  auto plane = [&](int k) { return g.off0 + (int64_t)k * g.pxy; };
  auto P1 = [&](int k, int x, int y) -> T& { return sm[L::P1 + (k & 3) * L::SN + S(x, y)]; };
  // vertical face value with the closed bottom (k = -1) and top (k = nz-1) faces
  auto Wf = [&](int k, int c) { return (k < 0 || k >= nz - 1) ? zero : W[plane(k) + c]; };

  for (int t = k0 - 5; t < k1; ++t) {
    // ---- A: psi1 on plane a = t+2, tile + 2 ring --------------------------
    const int a = t + 2;
    if (a >= max(0, k0 - 3) && a <= min(nz - 1, k1 + 1)) {
      const int64_t b = plane(a);
      for (int q = tid; q < L::SN; q += NT) {
        const int x = q % L::SX - 2, y = q / L::SX - 2;
        const int c = C(x, y), cxm = C(x - 1, y), cxp = C(x + 1, y);
        const int cym = C(x, y - 1), cyp = C(x, y + 1);
        const T p = P0[b + c];
        const T fxp = donor(p, P0[b + cxp], U[b + c]);
        const T fxm = donor(P0[b + cxm], p, U[b + cxm]);
        const T fyp = donor(p, P0[b + cyp], V[b + c]);
        const T fym = donor(P0[b + cym], p, V[b + cym]);
        const T fzp = a < nz - 1 ? donor(p, P0[b + g.pxy + c], W[b + c]) : zero;
        const T fzm = a > 0 ? donor(P0[b - g.pxy + c], p, W[b - g.pxy + c]) : zero;
        P1(a, x, y) = p - ((fxp - fxm) + (fyp - fym) + (fzp - fzm)) * rcp(G[b + c]);
      }
    }
    __syncthreads();
    // ---- B: pseudo-velocities on plane b = t+1 ----------------------------
    const int bb = t + 1;
    if (bb >= max(0, k0 - 2) && bb <= min(nz - 1, k1)) {
      const int64_t pb = plane(bb);
      const int bp = min(bb + 1, nz - 1), bm = max(bb - 1, 0);
      constexpr int NU = (TX + 3) * (TY + 2);  // x faces of cells [-2,TX] x [-1,TY]
      constexpr int NV = (TX + 2) * (TY + 3);  // y faces of cells [-1,TX] x [-2,TY]
      constexpr int NW = (TX + 2) * (TY + 2);  // z faces of cells [-1,TX] x [-1,TY]
      T* ut = sm + L::UT + (bb & 1) * L::SN;
      T* vt = sm + L::VT + (bb & 1) * L::SN;
      T* wt = sm + L::WT + (bb & 1) * L::SN;
      for (int q = tid; q < NU + NV + NW; q += NT) {
        if (q < NU) {
          const int x = q % (TX + 3) - 2, y = q / (TX + 3) - 1;
          const int c = C(x, y), cr = C(x + 1, y);
          const int cym = C(x, y - 1), crym = C(x + 1, y - 1);
          const T s1p = P1(bb, x + 1, y + 1) + P1(bb, x, y + 1);
          const T s1m = P1(bb, x + 1, y - 1) + P1(bb, x, y - 1);
          const T s2p = P1(bp, x + 1, y) + P1(bp, x, y);
          const T s2m = P1(bm, x + 1, y) + P1(bm, x, y);
          const T vs = V[pb + c] + V[pb + cr] + V[pb + cym] + V[pb + crym];
          const T ws = Wf(bb, c) + Wf(bb, cr) + Wf(bb - 1, c) + Wf(bb - 1, cr);
          ut[S(x, y)] = pseudo_velocity(U[pb + c], G[pb + c] + G[pb + cr], P1(bb, x, y),
                                        P1(bb, x + 1, y), s1p, s1m, s2p, s2m, vs, ws);
        } else if (q < NU + NV) {
          const int r = q - NU;
          const int x = r % (TX + 2) - 1, y = r / (TX + 2) - 2;
          const int c = C(x, y), cu = C(x, y + 1);
          const int cxm = C(x - 1, y), cuxm = C(x - 1, y + 1);
          const T s1p = P1(bb, x + 1, y + 1) + P1(bb, x + 1, y);
          const T s1m = P1(bb, x - 1, y + 1) + P1(bb, x - 1, y);
          const T s2p = P1(bp, x, y + 1) + P1(bp, x, y);
          const T s2m = P1(bm, x, y + 1) + P1(bm, x, y);
          const T us = U[pb + c] + U[pb + cu] + U[pb + cxm] + U[pb + cuxm];
          const T ws = Wf(bb, c) + Wf(bb, cu) + Wf(bb - 1, c) + Wf(bb - 1, cu);
          vt[S(x, y)] = pseudo_velocity(V[pb + c], G[pb + c] + G[pb + cu], P1(bb, x, y),
                                        P1(bb, x, y + 1), s1p, s1m, s2p, s2m, us, ws);
        } else {
          const int r = q - NU - NV;
          const int x = r % (TX + 2) - 1, y = r / (TX + 2) - 1;
          T res = zero;
          if (bb < nz - 1) {  // the top face is closed
            const int c = C(x, y), cxm = C(x - 1, y), cym = C(x, y - 1);
            const int64_t pu = pb + g.pxy;
            const T s1p = P1(bb + 1, x + 1, y) + P1(bb, x + 1, y);
            const T s1m = P1(bb + 1, x - 1, y) + P1(bb, x - 1, y);
            const T s2p = P1(bb + 1, x, y + 1) + P1(bb, x, y + 1);
            const T s2m = P1(bb + 1, x, y - 1) + P1(bb, x, y - 1);
            const T us = U[pb + c] + U[pu + c] + U[pb + cxm] + U[pu + cxm];
            const T vs = V[pb + c] + V[pu + c] + V[pb + cym] + V[pu + cym];
            res = pseudo_velocity(W[pb + c], G[pb + c] + G[pu + c], P1(bb, x, y),
                                  P1(bb + 1, x, y), s1p, s1m, s2p, s2m, us, vs);
          }
          wt[S(x, y)] = res;
        }
      }
    }
    __syncthreads();
    // ---- C: limiter bounds and betas on plane b = t+1, tile + 1 -----------
    if (LIMIT && bb >= max(0, k0 - 1) && bb <= min(nz - 1, k1)) {
      const int64_t pb = plane(bb);
      const int bp = min(bb + 1, nz - 1), bm = max(bb - 1, 0);
      const T* ut = sm + L::UT + (bb & 1) * L::SN;
      const T* vt = sm + L::VT + (bb & 1) * L::SN;
      const T* wt_up = sm + L::WT + (bb & 1) * L::SN;        // face bb+1/2
      const T* wt_dn = sm + L::WT + ((bb - 1) & 1) * L::SN;  // face bb-1/2
      T* bu = sm + L::BU + (bb & 1) * L::SN;
      T* bd = sm + L::BD + (bb & 1) * L::SN;
      constexpr int NB = (TX + 2) * (TY + 2);
      for (int q = tid; q < NB; q += NT) {
        const int x = q % (TX + 2) - 1, y = q / (TX + 2) - 1;
        const int c = C(x, y);
        const T pc = P1(bb, x, y);
        const T pxm = P1(bb, x - 1, y), pxp = P1(bb, x + 1, y);
        const T pym = P1(bb, x, y - 1), pyp = P1(bb, x, y + 1);
        const T pzm = P1(bm, x, y), pzp = P1(bp, x, y);
        const T p0 = P0[pb + c];
        const T n1 = P0[pb + C(x - 1, y)], n2 = P0[pb + C(x + 1, y)];
        const T n3 = P0[pb + C(x, y - 1)], n4 = P0[pb + C(x, y + 1)];
        const T n5 = P0[plane(bm) + c], n6 = P0[plane(bp) + c];
        const T vals[14] = {pc, p0, n1, n2, n3, n4, n5, n6, pxm, pxp, pym, pyp, pzm, pzp};
        T hi, lo;
        bounds(vals, hi, lo);
        const T fxp = donor(pc, pxp, ut[S(x, y)]);
        const T fxm = donor(pxm, pc, ut[S(x - 1, y)]);
        const T fyp = donor(pc, pyp, vt[S(x, y)]);
        const T fym = donor(pym, pc, vt[S(x, y - 1)]);
        const T fzp = bb < nz - 1 ? donor(pc, pzp, wt_up[S(x, y)]) : zero;
        const T fzm = bb > 0 ? donor(pzm, pc, wt_dn[S(x, y)]) : zero;
        const T in = (pos(fxm) - neg(fxp)) + (pos(fym) - neg(fyp)) + (pos(fzm) - neg(fzp));
        const T ou = (pos(fxp) - neg(fxm)) + (pos(fyp) - neg(fym)) + (pos(fzp) - neg(fzm));
        const T gc = G[pb + c];
        bu[S(x, y)] = (hi - pc) * gc * rcp(in + eps);
        bd[S(x, y)] = (pc - lo) * gc * rcp(ou + eps);
      }
    }
    __syncthreads();
    // ---- D: limited donor fluxes of plane t and of face t+1/2 ------------
    if (t >= max(0, k0 - 1) && t <= k1 - 1) {
      const T* ut = sm + L::UT + (t & 1) * L::SN;
      const T* vt = sm + L::VT + (t & 1) * L::SN;
      const T* wt = sm + L::WT + (t & 1) * L::SN;
      const T* bu0 = sm + L::BU + (t & 1) * L::SN;
      const T* bd0 = sm + L::BD + (t & 1) * L::SN;
      const T* bu1 = sm + L::BU + ((t + 1) & 1) * L::SN;
      const T* bd1 = sm + L::BD + ((t + 1) & 1) * L::SN;
      T* fx = sm + L::FX;
      T* fy = sm + L::FY;
      T* fz = sm + L::FZ + (t & 1) * L::SN;
      constexpr int NX = (TX + 1) * TY, NY = TX * (TY + 1), NZ = TX * TY;
      for (int q = tid; q < NX + NY + NZ; q += NT) {
        if (q < NX) {
          const int x = q % (TX + 1) - 1, y = q / (TX + 1);
          T u = ut[S(x, y)];
          if (LIMIT) u = limit_face(u, bu0[S(x, y)], bd0[S(x, y)], bu0[S(x + 1, y)], bd0[S(x + 1, y)]);
          fx[S(x, y)] = donor(P1(t, x, y), P1(t, x + 1, y), u);
        } else if (q < NX + NY) {
          const int r = q - NX;
          const int x = r % TX, y = r / TX - 1;
          T v = vt[S(x, y)];
          if (LIMIT) v = limit_face(v, bu0[S(x, y)], bd0[S(x, y)], bu0[S(x, y + 1)], bd0[S(x, y + 1)]);
          fy[S(x, y)] = donor(P1(t, x, y), P1(t, x, y + 1), v);
        } else {
          const int r = q - NX - NY;
          const int x = r % TX, y = r / TX;
          T f = zero;
          if (t < nz - 1) {
            T w = wt[S(x, y)];
            if (LIMIT) w = limit_face(w, bu0[S(x, y)], bd0[S(x, y)], bu1[S(x, y)], bd1[S(x, y)]);
            f = donor(P1(t, x, y), P1(t + 1, x, y), w);
          }
          fz[S(x, y)] = f;
        }
      }
    }
    __syncthreads();
    // ---- E: advance and write psi^(n+1) on plane t ------------------------
    if (t >= k0) {
      const T* fx = sm + L::FX;
      const T* fy = sm + L::FY;
      const T* fzu = sm + L::FZ + (t & 1) * L::SN;
      const T* fzd = sm + L::FZ + ((t - 1) & 1) * L::SN;
      const int64_t pt = plane(t);
      for (int q = tid; q < TX * TY; q += NT) {
        const int x = q % TX, y = q / TX;
        const int i = i0 + x, j = j0 + y;
        if (i >= g.nx || j >= g.ny) continue;
        const T fzm = t > 0 ? fzd[S(x, y)] : zero;
        const T r = P1(t, x, y) - ((fx[S(x, y)] - fx[S(x - 1, y)]) + (fy[S(x, y)] - fy[S(x, y - 1)]) +
                                   (fzu[S(x, y)] - fzm)) * rcp(G[pt + C(x, y)]);
        // the point and its periodic (i, j) and edge-copied (k) halo images
        const int ni = (i < g.h) ? 1 : ((i >= g.nx - g.h) ? -1 : 0);
        const int nj = (j < g.h) ? 1 : ((j >= g.ny - g.h) ? -1 : 0);
        const int klo = (t == 0) ? -g.h : t, khi = (t == nz - 1) ? nz - 1 + g.h : t;
        for (int kk = klo; kk <= khi; ++kk) {
          if (kk != t && kk >= 0 && kk < nz) continue;
          const int64_t pk = g.off0 + (int64_t)kk * g.pxy;
          for (int a2 = 0; a2 <= (ni != 0); ++a2) {
            const int ii = i + a2 * ni * g.nx;
            for (int b2 = 0; b2 <= (nj != 0); ++b2) {
              const int jj = j + b2 * nj * g.ny;
              out[pk + (int64_t)jj * g.px + ii] = r;
            }
          }
        }
      }
    }
    // no barrier needed here: the next iteration's stage A writes a psi1
    // slot this stage does not read, and every later stage is behind a barrier
  }
}

template <class T, int TX, int TY, int NT, int MINB, bool LIMIT>
__global__ void __launch_bounds__(NT, MINB)
step_kernel(Geo g, int kchunk, const T* __restrict__ P0, const T* __restrict__ U,
            const T* __restrict__ V, const T* __restrict__ W, const T* __restrict__ G,
            T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k0 = blockIdx.z * kchunk;
  step_tile<T, TX, TY, NT, LIMIT>(g, blockIdx.x * TX, blockIdx.y * TY, k0, min(g.nz, k0 + kchunk),
                                  P0, U, V, W, G, out, smem_raw);
}

}  // namespace fused
}  // namespace mpd
