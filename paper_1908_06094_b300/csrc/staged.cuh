// staged.cuh -- the unfused MPDATA step: one simple kernel per stage, one
// thread per interior cell, every intermediate in device memory.
//
// This is the "without fusion" organisation of Table 2 (each stage re-reads
// its inputs from main memory, as the separate Fortran subroutines of
// Listing 8 do).  Each face flux is computed once, by the cell on its left
// (the face's owner), and read by both neighbours, so the flux divergence
// telescopes exactly and mass is conserved to the rounding of psi*G alone.
#pragma once
#include <type_traits>
#include "grid.cuh"

namespace mpd {
namespace staged {

struct Cell {
  int i, j, k;
  bool ok;
};

__device__ __forceinline__ Cell cell_of(const Geo& g) {
  Cell c;
  c.i = blockIdx.x * blockDim.x + threadIdx.x;
  c.j = blockIdx.y * blockDim.y + threadIdx.y;
  c.k = blockIdx.z;
  c.ok = c.i < g.nx && c.j < g.ny;
  return c;
}

// Vertical-face value with the closed bottom and top faces.
template <class T>
__device__ __forceinline__ T wface(const T* w, const Geo& g, int i, int j, int k) {
  return zopen(g, k) ? w[at(g, i, j, kadj(g, k))] : T(0);
}

// Donor-cell fluxes through the three "+" faces of every cell.  RG: also
// store 1/G in rg (the FP64 staged step: this kernel is bound by memory with
// FP64 issue to spare, the advances that read 1/G by the FP64 pipe).
template <class T, bool RG = false>
__global__ void flux_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
                            const T* __restrict__ cv, const T* __restrict__ cw,
                            T* __restrict__ fx, T* __restrict__ fy, T* __restrict__ fz,
                            const T* __restrict__ G = nullptr, T* __restrict__ rg = nullptr) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  int64_t q = at(g, c.i, c.j, c.k);
  if constexpr (RG) rg[q] = rcp(G[q]);
  T p = P[q];
  fx[q] = donor(p, P[at(g, wrap_up(c.i, g.nx), c.j, c.k)], cu[q]);
  fy[q] = donor(p, P[at(g, c.i, wrap_up(c.j, g.ny), c.k)], cv[q]);
  fz[q] = zopen(g, c.k) ? donor(p, P[at(g, c.i, c.j, kadj(g, c.k + 1))], cw[q]) : T(0);
}

// Flux divergence and advance (Listings 8/9): out = P - (1/G) sum dF.
// P and out may be the same buffer (each thread reads and writes only its
// own point), so neither is declared __restrict__.
// RG: 0 forms 1/G here; 1 forms it and also stores it to rg; 2 reads it from
// rg (stored earlier in the same step with the same G: the FP64 advances
// skip the reciprocal's three FMAs for one load).
template <class T, int RG = 0>
__global__ void advance_kernel(Geo g, const T* P, const T* __restrict__ fx,
                               const T* __restrict__ fy, const T* __restrict__ fz,
                               const T* __restrict__ G, T* out, T* rg = nullptr) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  int64_t q = at(g, c.i, c.j, c.k);
  T fxm = fx[at(g, wrap_dn(c.i, g.nx), c.j, c.k)];
  T fym = fy[at(g, c.i, wrap_dn(c.j, g.ny), c.k)];
  T fzm = zopen(g, c.k - 1) ? fz[at(g, c.i, c.j, kadj(g, c.k - 1))] : T(0);
  T r;
  if constexpr (RG == 2) {
    r = rg[q];
  } else {
    r = rcp(G[q]);
    if constexpr (RG == 1) rg[q] = r;
  }
  out[q] = P[q] - ((fx[q] - fxm) + (fy[q] - fym) + (fz[q] - fzm)) * r;
}

// The last corrective pass's limited fluxes and its advance in one kernel
// (the FP64 staged step, whose pseudo-velocity stage formed the donor
// fluxes F of Ut): each cell scales the fluxes of its six faces by their
// limiter factors -- its "-" faces are its neighbours' "+" faces, scaled
// with the same inputs, so both cells see the same bits -- and advances
// with the stored 1/G.  The same bits as limflux_kernel<FIN> followed by
// advance_kernel<RG = 2>, without the limited fluxes' round trip through
// memory (6 products a cell instead of 3: the kernel is bound by neither).
// P and out are distinct.  IMG: each cell also writes its value's images
// in the halo of out (periodic in i and j; in k the edge copies of the
// bottom and top levels, or the periodic images), the separate halo fill's
// work (nx, ny >= 2h: one image a side).
template <class T>
__device__ __forceinline__ void put_images(const Geo& g, int i, int j, int k, T r,
                                           T* __restrict__ out) {
  const int ni = i < g.h ? 1 : (i >= g.nx - g.h ? -1 : 0);
  const int nj = j < g.h ? 1 : (j >= g.ny - g.h ? -1 : 0);
  int klo = (k == 0) ? -g.h : k, khi = (k == g.nz - 1) ? g.nz - 1 + g.h : k;
  if (g.kper) {
    klo = k;
    while (klo - g.nz >= -g.h) klo -= g.nz;
    khi = g.nz - 1 + g.h;
  }
  if (ni == 0 && nj == 0 && klo == k && khi == k) return;
  for (int kk = klo; kk <= khi; kk += g.kper ? g.nz : 1) {
    if (!g.kper && kk != k && kk >= 0 && kk < g.nz) continue;
    for (int a = 0; a <= (ni != 0); ++a)
      for (int b = 0; b <= (nj != 0); ++b)
        if (kk != k || a != 0 || b != 0) out[at(g, i + a * ni * g.nx, j + b * nj * g.ny, kk)] = r;
  }
}
template <class T, bool IMG = false>
__global__ void limadvance_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ ut,
                                  const T* __restrict__ vt, const T* __restrict__ wt,
                                  const T* __restrict__ bu, const T* __restrict__ bd,
                                  const T* __restrict__ fx, const T* __restrict__ fy,
                                  const T* __restrict__ fz, const T* __restrict__ rg,
                                  T* __restrict__ out) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  const int64_t xp = at(g, wrap_up(c.i, g.nx), c.j, c.k), xm = at(g, wrap_dn(c.i, g.nx), c.j, c.k);
  const int64_t yp = at(g, c.i, wrap_up(c.j, g.ny), c.k), ym = at(g, c.i, wrap_dn(c.j, g.ny), c.k);
  const bool zt = zopen(g, c.k), zb = zopen(g, c.k - 1);
  // a closed face takes q as an in-bounds stand-in (its flux is 0)
  const int64_t zp = zt ? at(g, c.i, c.j, kadj(g, c.k + 1)) : q;
  const int64_t zm = zb ? at(g, c.i, c.j, kadj(g, c.k - 1)) : q;
  const T buq = bu[q], bdq = bd[q];
  // the limited flux of the face from L to R
  auto lf = [&](T U, T F, T buL, T bdL, T buR, T bdR) {
    return mul_rn(limit_factor(U, buL, bdL, buR, bdR), F);
  };
  const T fxp = lf(ut[q], fx[q], buq, bdq, bu[xp], bd[xp]);
  const T fxm = lf(ut[xm], fx[xm], bu[xm], bd[xm], buq, bdq);
  const T fyp = lf(vt[q], fy[q], buq, bdq, bu[yp], bd[yp]);
  const T fym = lf(vt[ym], fy[ym], bu[ym], bd[ym], buq, bdq);
  const T fzp = zt ? lf(wt[q], fz[q], buq, bdq, bu[zp], bd[zp]) : T(0);
  const T fzm = zb ? lf(wt[zm], fz[zm], bu[zm], bd[zm], buq, bdq) : T(0);
  const T r = P[q] - ((fxp - fxm) + (fyp - fym) + (fzp - fzm)) * rg[q];
  out[q] = r;
  if constexpr (IMG) put_images(g, c.i, c.j, c.k, r, out);
}

// Antidiffusive pseudo-velocities on the "+" faces of every cell
// (Smolarkiewicz 1984; G-weighted form of Smolarkiewicz & Margolin 1998).
// OPT (kOpt* bits): ABS forms A and B from |psi|; IGA gives the
// infinite-gauge pseudo-fluxes instead; DFL adds the divergent-flow term.
template <class T, int OPT = 0>
__global__ void pseudo_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
                              const T* __restrict__ cv, const T* __restrict__ cw,
                              const T* __restrict__ G, T* __restrict__ ut, T* __restrict__ vt,
                              T* __restrict__ wt) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int i = c.i, j = c.j, k = c.k;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int kp = kadj(g, k + 1), km = kadj(g, k - 1);
  auto p = [&](int a, int b, int d) {
    const T x = P[at(g, a, b, d)];
    return (OPT & kOptABS) ? absv(x) : x;
  };
  auto face = [&](T U, T gsum, T pl, T pr, T s1p, T s1m, T s2p, T s2m, T vsum, T wsum) {
    if constexpr ((OPT & kOptIGA) != 0)
      return pseudo_flux_iga(U, gsum, pl, pr, s1p, s1m, s2p, s2m, vsum, wsum);
    else
      return pseudo_velocity(U, gsum, pl, pr, s1p, s1m, s2p, s2m, vsum, wsum);
  };
  // divergence of the Courant numbers of cell (a, b, d) (closed faces 0)
  auto div = [&](int a, int b, int d) {
    return (cu[at(g, a, b, d)] - cu[at(g, wrap_dn(a, g.nx), b, d)]) +
           (cv[at(g, a, b, d)] - cv[at(g, a, wrap_dn(b, g.ny), d)]) +
           (wface(cw, g, a, b, d) - wface(cw, g, a, b, d - 1));
  };
  const int64_t q = at(g, i, j, k);
  const T pc = p(i, j, k);
  {  // x face between (i) and (ip)
    const T s1p = p(ip, jp, k) + p(i, jp, k), s1m = p(ip, jm, k) + p(i, jm, k);
    const T s2p = p(ip, j, kp) + p(i, j, kp), s2m = p(ip, j, km) + p(i, j, km);
    const T vs = cv[q] + cv[at(g, ip, j, k)] + cv[at(g, i, jm, k)] + cv[at(g, ip, jm, k)];
    const T ws = wface(cw, g, i, j, k) + wface(cw, g, ip, j, k) + wface(cw, g, i, j, k - 1) +
                 wface(cw, g, ip, j, k - 1);
    const T gs = G[q] + G[at(g, ip, j, k)];
    T r = face(cu[q], gs, pc, p(ip, j, k), s1p, s1m, s2p, s2m, vs, ws);
    if constexpr ((OPT & kOptDFL) != 0)
      r = add_rn(r, divergent_flow_term(cu[q], gs, div(i, j, k) + div(ip, j, k)));
    ut[q] = r;
  }
  {  // y face between (j) and (jp)
    const T s1p = p(ip, jp, k) + p(ip, j, k), s1m = p(im, jp, k) + p(im, j, k);
    const T s2p = p(i, jp, kp) + p(i, j, kp), s2m = p(i, jp, km) + p(i, j, km);
    const T us = cu[q] + cu[at(g, i, jp, k)] + cu[at(g, im, j, k)] + cu[at(g, im, jp, k)];
    const T ws = wface(cw, g, i, j, k) + wface(cw, g, i, jp, k) + wface(cw, g, i, j, k - 1) +
                 wface(cw, g, i, jp, k - 1);
    const T gs = G[q] + G[at(g, i, jp, k)];
    T r = face(cv[q], gs, pc, p(i, jp, k), s1p, s1m, s2p, s2m, us, ws);
    if constexpr ((OPT & kOptDFL) != 0)
      r = add_rn(r, divergent_flow_term(cv[q], gs, div(i, j, k) + div(i, jp, k)));
    vt[q] = r;
  }
  if (zopen(g, k)) {  // z face between (k) and (k+1); a zero-flux top face is closed
    const int64_t qp = at(g, i, j, kp);
    const T s1p = p(ip, j, kp) + p(ip, j, k), s1m = p(im, j, kp) + p(im, j, k);
    const T s2p = p(i, jp, kp) + p(i, jp, k), s2m = p(i, jm, kp) + p(i, jm, k);
    const T us = cu[q] + cu[qp] + cu[at(g, im, j, k)] + cu[at(g, im, j, kp)];
    const T vs = cv[q] + cv[qp] + cv[at(g, i, jm, k)] + cv[at(g, i, jm, kp)];
    const T gs = G[q] + G[qp];
    T r = face(cw[q], gs, pc, p(i, j, kp), s1p, s1m, s2p, s2m, us, vs);
    if constexpr ((OPT & kOptDFL) != 0)
      r = add_rn(r, divergent_flow_term(cw[q], gs, div(i, j, k) + div(i, j, kp)));
    wt[q] = r;
  } else {
    wt[q] = T(0);
  }
}

// Non-oscillatory limiter, first half: bounds over the 7-point stencil of
// psi^n (P0) and psi^(m-1) (P), incoming/outgoing antidiffusive fluxes and
// the scale factors beta-up, beta-down (Smolarkiewicz & Grabowski 1990).
// With rin != nullptr the reciprocals 1/(in+eps) and 1/(out+eps) are kept
// too (the adjoint's tape).
// UNIT: the face values ut, vt, wt are the fluxes themselves -- in the
// infinite gauge, and in the FP64 staged step, whose pseudo-velocity stage
// passes the donor fluxes it formed.
template <class T, bool UNIT = false>
__global__ void beta_kernel(Geo g, const T* __restrict__ P0, const T* __restrict__ P,
                            const T* __restrict__ ut, const T* __restrict__ vt,
                            const T* __restrict__ wt, const T* __restrict__ G,
                            T* __restrict__ bu, T* __restrict__ bd, T* __restrict__ rin,
                            T* __restrict__ rout) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const T eps = Eps<T>::v, zero = T(0);
  const int i = c.i, j = c.j, k = c.k;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int kp = kadj(g, k + 1), km = kadj(g, k - 1);
  const int64_t q = at(g, i, j, k);
  const int64_t nb[6] = {at(g, im, j, k), at(g, ip, j, k), at(g, i, jm, k),
                         at(g, i, jp, k), at(g, i, j, km), at(g, i, j, kp)};
  T pc = P[q];
  const T vals[14] = {P0[q], pc, P0[nb[0]], P[nb[0]], P0[nb[1]], P[nb[1]], P0[nb[2]], P[nb[2]],
                      P0[nb[3]], P[nb[3]], P0[nb[4]], P[nb[4]], P0[nb[5]], P[nb[5]]};
  T hi, lo;
  bounds(vals, hi, lo);
  auto fl = [&](T L, T R, T C) { return UNIT ? C : donor(L, R, C); };
  T fxp = fl(pc, P[nb[1]], ut[q]);
  T fxm = fl(P[nb[0]], pc, ut[nb[0]]);
  T fyp = fl(pc, P[nb[3]], vt[q]);
  T fym = fl(P[nb[2]], pc, vt[nb[2]]);
  T fzp = zopen(g, k) ? fl(pc, P[nb[5]], wt[q]) : zero;
  T fzm = zopen(g, k - 1) ? fl(P[nb[4]], pc, wt[nb[4]]) : zero;
  T in = (pos(fxm) - neg(fxp)) + (pos(fym) - neg(fyp)) + (pos(fzm) - neg(fzp));
  T out = (pos(fxp) - neg(fxm)) + (pos(fyp) - neg(fym)) + (pos(fzp) - neg(fzm));
  const T gq = G[q];
  const T nu = (hi - pc) * gq, nd = (pc - lo) * gq;  // >= +0: hi >= pc >= lo, G > 0
  const T di = in + eps, dd = out + eps;              // > 0
  if constexpr (std::is_same<T, double>::value && UNIT) {
    // FP64 staged step: a beta at or above 1 is stored as 1, which the
    // limiter reads only through min(1, beta); beta >= 1 exactly when its
    // numerator reaches its denominator, a test on the bit patterns of two
    // non-negative doubles (integer pipe).  A warp whose betas of one kind
    // are all >= 1 skips that reciprocal (4 FP64 instructions); the adjoint's
    // tape keeps both reciprocals.
    const bool lu = dbits(nu) < dbits(di), ld = dbits(nd) < dbits(dd);
    const unsigned live = __activemask();
    T bu_v = 1.0, bd_v = 1.0;
    if (rin || __any_sync(live, lu)) {
      const T ri = rcp(di);
      if (lu) bu_v = nu * ri;
      if (rin) rin[q] = ri;
    }
    if (rin || __any_sync(live, ld)) {
      const T ro = rcp(dd);
      if (ld) bd_v = nd * ro;
      if (rin) rout[q] = ro;
    }
    bu[q] = bu_v;
    bd[q] = bd_v;
  } else {
    const T ri = rcp(di), ro = rcp(dd);
    bu[q] = nu * ri;
    bd[q] = nd * ro;
    if (rin) {
      rin[q] = ri;
      rout[q] = ro;
    }
  }
}

// Second half: limited velocities on the "+" faces and their donor fluxes.
// With ul != nullptr the limited velocities are kept for a further pass.
// OPT: with ABS a face whose upwind value is negative carries its flux
// against its velocity, so beta-up and beta-down trade places there; with
// IGA the limited values are the fluxes.
// FIN: fx, fy, fz hold on entry the unlimited donor fluxes F(psi_L, psi_R,
// Ut) (stored by the pseudo-velocity stage), and the limited flux is the
// limiter's factor times that flux: one product a face, psi not read (not
// with the signed-field or infinite-gauge options).
template <class T, int OPT = 0, bool FIN = false>
__global__ void limflux_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ ut,
                               const T* __restrict__ vt, const T* __restrict__ wt,
                               const T* __restrict__ bu, const T* __restrict__ bd,
                               T* __restrict__ fx, T* __restrict__ fy, T* __restrict__ fz,
                               T* __restrict__ ul, T* __restrict__ vl, T* __restrict__ wl) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  const int64_t qx = at(g, wrap_up(c.i, g.nx), c.j, c.k);
  const int64_t qy = at(g, c.i, wrap_up(c.j, g.ny), c.k);
  if constexpr (FIN) {
    static_assert((OPT & (kOptABS | kOptIGA)) == 0, "FIN: signed psi only");
    const T buc = bu[q], bdc = bd[q], ux = ut[q], vy = vt[q];
    const bool oz = zopen(g, c.k);
    const int64_t qz = at(g, c.i, c.j, kadj(g, c.k + 1));
    const T wz = oz ? wt[q] : T(0);
    const T cx = limit_factor(ux, buc, bdc, bu[qx], bd[qx]);
    const T cy = limit_factor(vy, buc, bdc, bu[qy], bd[qy]);
    const T cz = oz ? limit_factor(wz, buc, bdc, bu[qz], bd[qz]) : T(0);
    const T Fx = fx[q], Fy = fy[q], Fz = oz ? fz[q] : T(0);
    fx[q] = mul_rn(cx, Fx);
    fy[q] = mul_rn(cy, Fy);
    fz[q] = oz ? mul_rn(cz, Fz) : T(0);
    if (ul) {
      ul[q] = mul_rn(cx, ux);
      vl[q] = mul_rn(cy, vy);
      wl[q] = oz ? mul_rn(cz, wz) : T(0);
    }
    return;
  }
  T pc = P[q], buc = bu[q], bdc = bd[q];
  auto lim = [&](T Ut, int64_t qn) {
    T uL = buc, dL = bdc, uR = bu[qn], dR = bd[qn];
    if constexpr ((OPT & kOptABS) != 0) {
      if (!ge0(ge0(Ut) ? pc : P[qn])) {
        uL = bdc; dL = buc; uR = bd[qn]; dR = bu[qn];
      }
    }
    return limit_face(Ut, uL, dL, uR, dR);
  };
  auto fl = [&](T R, T C) {
    if constexpr ((OPT & kOptIGA) != 0) return C;
    else return donor(pc, R, C);
  };
  T lx = lim(ut[q], qx);
  T ly = lim(vt[q], qy);
  T lz = T(0);
  const bool oz = zopen(g, c.k);
  const int64_t qz = at(g, c.i, c.j, kadj(g, c.k + 1));
  if (oz) lz = lim(wt[q], qz);
  fx[q] = fl(P[qx], lx);
  fy[q] = fl(P[qy], ly);
  fz[q] = oz ? fl(P[qz], lz) : T(0);
  if (ul) { ul[q] = lx; vl[q] = ly; wl[q] = lz; }
}

}  // namespace staged

// Halo kernels.  They visit halo cells only, one thread per cell of a 1D
// enumeration (halo_count cells): first the levels that are all halo -- the
// h levels below and above the interior, and with `top` the interior top
// level too -- px * (ny+2h) cells each, then for every other interior level
// its h-deep bands of rows below and above (2h * px cells) and of columns
// left and right (2h * ny cells).
struct HaloCell {
  int ii, jj, kk;
  bool whole;  // on an all-halo level
};
__device__ __forceinline__ int64_t halo_count(const Geo& g, bool top) {
  const int64_t plane = g.px * (int64_t)(g.ny + 2 * g.h);
  const int64_t band = 2 * (int64_t)g.h * (g.px + g.ny);
  return (2 * g.h + top) * plane + (g.nz - top) * band;
}
__device__ __forceinline__ HaloCell halo_cell(const Geo& g, bool top, int64_t t) {
  const int h = g.h, px = (int)g.px;
  const int64_t plane = g.px * (int64_t)(g.ny + 2 * h);
  const int64_t nwhole = (2 * h + top) * plane;
  HaloCell c;
  if (t < nwhole) {
    const int w = (int)(t / plane), e = (int)(t % plane);
    c.kk = w < h ? w - h : g.nz - top + (w - h);
    c.ii = e % px - h;
    c.jj = e / px - h;
    c.whole = true;
    return c;
  }
  const int64_t band = 2 * (int64_t)h * (g.px + g.ny);
  const int64_t t2 = t - nwhole;
  const int e = (int)(t2 % band);
  c.kk = (int)(t2 / band);
  c.whole = false;
  const int nrow = 2 * h * px;
  if (e < nrow) {
    const int r = e / px;
    c.ii = e % px - h;
    c.jj = r < h ? r - h : g.ny + (r - h);
  } else {
    const int e2 = e - nrow, ci = e2 % (2 * h);
    c.jj = e2 / (2 * h);
    c.ii = ci < h ? ci - h : g.nx + (ci - h);
  }
  return c;
}
__device__ __forceinline__ int64_t padded_at(const Geo& g, const HaloCell& c) {
  return g.off0 + (int64_t)c.kk * g.pxy + (int64_t)c.jj * g.px + c.ii;
}
// the interior value a halo cell copies (periodic in i, j; edge copy in k)
__device__ __forceinline__ int64_t halo_source(const Geo& g, const HaloCell& c) {
  const int is = ((c.ii % g.nx) + g.nx) % g.nx;
  const int js = ((c.jj % g.ny) + g.ny) % g.ny;
  const int ks = g.kper ? ((c.kk % g.nz) + g.nz) % g.nz
                       : (c.kk < 0 ? 0 : (c.kk >= g.nz ? g.nz - 1 : c.kk));
  return at(g, is, js, ks);
}

// Fill: CELL (kind 0) periodic images in i and j, edge copy in k (periodic
// k: the level nz away); WFACE (kind 1) the same, except that with closed
// vertical boundaries the faces k < 0 and k >= nz-1 (the bottom and top
// faces, interior included) are 0.
template <class T>
__global__ void halo_kernel(Geo g, T* __restrict__ f, int kind) {
  pdl_enter();
  const bool top = kind == 1 && !g.kper;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= halo_count(g, top)) return;
  const HaloCell c = halo_cell(g, top, t);
  const bool closed = top && (c.kk < 0 || c.kk >= g.nz - 1);
  f[padded_at(g, c)] = closed ? T(0) : f[halo_source(g, c)];
}

// Reverse of the CELL halo fill for an adjoint field: every halo entry was a
// copy of one interior value, so its adjoint is added to that value (atomic:
// several halo entries copy the same corner values); a second launch
// (halo_zero_kernel) then clears the halo.
template <class T>
__global__ void halo_fold_kernel(Geo g, T* __restrict__ f) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= halo_count(g, false)) return;
  const HaloCell c = halo_cell(g, false, t);
  const T v = f[padded_at(g, c)];
  if (v != T(0)) atomicAdd(&f[halo_source(g, c)], v);
}

// dst[q] = src[q] for the n elements of a padded field (the copy back of a
// one-kernel step run out of place), 16 bytes a thread where both fields
// start on a 16-byte boundary.
template <class T>
__global__ void copy_kernel(const T* __restrict__ src, T* __restrict__ dst, int64_t n,
                            bool vec) {
  pdl_enter();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  constexpr int V = 16 / sizeof(T);
  if (vec) {
    const int64_t nv = n / V;
    for (int64_t q = t; q < nv; q += stride)
      reinterpret_cast<int4*>(dst)[q] = reinterpret_cast<const int4*>(src)[q];
    for (int64_t q = nv * V + t; q < n; q += stride) dst[q] = src[q];
  } else {
    for (int64_t q = t; q < n; q += stride) dst[q] = src[q];
  }
}

template <class T>
__global__ void halo_zero_kernel(Geo g, T* __restrict__ f) {
  pdl_enter();
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= halo_count(g, false)) return;
  f[padded_at(g, halo_cell(g, false, t))] = T(0);
}

}  // namespace mpd
