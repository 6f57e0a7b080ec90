// fusedt.cuh -- the one-kernel FP32 MPDATA step for two tracers of one
// domain at once (the batch's tracer pairs).
//
// The tracers of a batch domain share its Courant fields and metric.  A
// thread owns one column of the tile (the one-column kernel's layout,
// fused2.cuh: the same stages, rings and two barriers a level) and carries
// every tracer-dependent value of its column for two tracers as one float2
// (lane 0 tracer a, lane 1 tracer b), whose sums, differences, products and
// fused multiply-adds are single f32x2 instructions.  What depends on U, V,
// W and G alone is formed once for both lanes: the loads and shared planes
// of U, V, W, G, the face sums of G and of the cross-direction Courant
// numbers, 1/G_f, U/G_f and |U| - U^2/G_f of every face, 1/G of every cell,
// and the upwind sign of every face.  Both tracers' values of a cell sit
// side by side in shared memory, so a neighbour is one 8-byte load.
//
// Every lane performs the one-column kernel's explicitly rounded operations
// in its order (a shared value is the same scalar operation the lane would
// form), so a tracer advanced here has the bits of the single-domain step.
// As in fusedx.cuh, a product that a sum consumes directly is formed per
// lane, since the code generator may fuse a packed product into the packed
// sum that consumes it.
//
// Zero-flux k, periodic i-j domain, no options, no tape (the batch's step).
#pragma once
#include <climits>
#include <type_traits>

#include "fused2.cuh"
#include "fusedx.cuh"
#include "grid.cuh"

namespace mpd {
namespace fusedt {

using fusedx::f2;
using fusedx::mk;
using fusedx::add2;
using fusedx::sub2;
using fusedx::mul2;
using fusedx::fma2;
using fusedx::splat;
using fusedx::rcp2;
using fusedx::pos2;
using fusedx::neg2;
using fusedx::bounds2;

// donor flux of both lanes through a face of Courant number C (shared): one
// sign test, each lane's upwind value, each lane's product (scalar: a sum
// consumes it)
__device__ __forceinline__ f2 donor_s(f2 L, f2 R, float C) {
  const bool up = nonneg(C);
  return mk(mul_rn(C, up ? L.x : R.x), mul_rn(C, up ? L.y : R.y));
}
// the same as one packed product (for fluxes that are stored or bounded)
__device__ __forceinline__ f2 donor_p(f2 L, f2 R, float C) {
  const bool up = nonneg(C);
  return mul2(splat(C), mk(up ? L.x : R.x, up ? L.y : R.y));
}
// donor flux of a face whose Courant number differs per lane (the
// pseudo-velocities and limited velocities are tracer-dependent)
__device__ __forceinline__ f2 donor_l(f2 L, f2 R, f2 C) {
  return mul2(C, mk(nonneg(C.x) ? L.x : R.x, nonneg(C.y) ? L.y : R.y));
}

// The tracer-independent part of a face's pseudo-velocity (the scalar
// pseudo_velocity's operations on U and G_f): q = U/Gf and |U| - U^2/Gf.
struct FaceU {
  float q, diff;
};
__device__ __forceinline__ FaceU face_u(float U, float gsum) {
  const float rG = mul_rn(2.0f, rcp(gsum));
  const float q = mul_rn(U, rG);
  return {q, fma_rn(-U, q, absv(U))};
}
// the tracer-dependent rest, per lane
__device__ __forceinline__ f2 pseudo_t(const FaceU& fu, f2 pl, f2 pr, f2 s1p, f2 s1m, f2 s2p,
                                       f2 s2m, float vsum, float wsum) {
  const f2 eps = splat(Eps<float>::v);
  const f2 A = mul2(sub2(pr, pl), rcp2(add2(add2(pr, pl), eps)));
  const f2 B1 = mul2(sub2(s1p, s1m), rcp2(add2(add2(s1p, s1m), eps)));
  const f2 B2 = mul2(sub2(s2p, s2m), rcp2(add2(add2(s2p, s2m), eps)));
  const f2 cross = mul2(splat(0.125f), fma2(splat(vsum), B1, mul2(splat(wsum), B2)));
  return fma2(splat(fu.diff), A, mul2(splat(-fu.q), cross));
}

// Shared planes (floats): the tracer-dependent ones hold a float2 a cell.
template <int TX, int TY>
struct Layout {
  static constexpr int EX = TX + 4, EY = TY + 4, SN = EX * EY;  // radius-2 planes
  static constexpr int RX = TX + 6, RY = TY + 6, RN = RX * RY;  // radius-3 planes
  static constexpr int NRING = RN - SN;
  static constexpr int P0S = 0;              // psi^n pairs, 4 planes, radius 3
  static constexpr int US = P0S + 8 * RN;    // U, 4 planes, radius 3
  static constexpr int VS = US + 4 * RN;     // V, 4 planes, radius 3
  static constexpr int WS = VS + 4 * RN;     // W, 4 faces
  static constexpr int GS = WS + 4 * SN;     // G, 4 planes
  static constexpr int P1S = GS + 4 * SN;    // psi1 pairs, 4 planes
  static constexpr int UTS = P1S + 8 * SN;   // Ut pairs, 1 plane
  static constexpr int VTS = UTS + 2 * SN;   // Vt pairs, 1 plane
  static constexpr int BUS = VTS + 2 * SN;   // beta-up pairs, 2 planes
  static constexpr int BDS = BUS + 4 * SN;   // beta-down pairs, 2 planes
  static constexpr int FXS = BDS + 4 * SN;   // x-face flux pairs, 2 planes
  static constexpr int FYS = FXS + 4 * SN;   // y-face flux pairs, 2 planes
  static constexpr int NVAL = FYS + 4 * SN;
  static constexpr size_t bytes = (size_t)NVAL * sizeof(float);
  static_assert(RN % 2 == 0 && SN % 2 == 0, "8-byte pairs");
};

// One tile and level chunk of two tracers: Pa, Pb -> Oa, Ob (Pb, Ob carry
// tracer b; with two false the pair holds tracer a alone, lane 1 repeats it
// and writes nothing).  Element offsets are 32-bit (the caller checks that a
// padded field has fewer than 2^31 elements).
template <int TX, int TY, bool LIMIT>
__device__ __forceinline__ void step_tile_t2(const Geo& g, int i0, int j0, int k0, int k1,
                                             const float* __restrict__ Pa,
                                             const float* __restrict__ Pb,
                                             const float* __restrict__ U,
                                             const float* __restrict__ V,
                                             const float* __restrict__ W,
                                             const float* __restrict__ G, float* __restrict__ Oa,
                                             float* __restrict__ Ob, bool two,
                                             unsigned char* smem_raw) {
  using L = Layout<TX, TY>;
  using Map = fused2::TileMap<TX, TY>;
  constexpr int EX = L::EX, RX = L::RX;
  float* sm = reinterpret_cast<float*>(smem_raw);
  f2* p0s = reinterpret_cast<f2*>(sm + L::P0S);
  float* us = sm + L::US;
  float* vs = sm + L::VS;
  float* ws = sm + L::WS;
  float* gs = sm + L::GS;
  f2* p1s = reinterpret_cast<f2*>(sm + L::P1S);
  f2* uts = reinterpret_cast<f2*>(sm + L::UTS);
  f2* vts = reinterpret_cast<f2*>(sm + L::VTS);
  f2* bus = reinterpret_cast<f2*>(sm + L::BUS);
  f2* bds = reinterpret_cast<f2*>(sm + L::BDS);
  f2* fxs = reinterpret_cast<f2*>(sm + L::FXS);
  f2* fys = reinterpret_cast<f2*>(sm + L::FYS);
  const int tid = threadIdx.x;
  const int nz = g.nz;
  const f2 zero2 = splat(0.0f), eps2 = splat(Eps<float>::v);

  // the thread's column and stage regions: the one-column kernel's
  int x, y;
  Map::cell(tid, x, y);
  const int s2 = (y + 2) * EX + (x + 2);
  const int s3 = (y + 3) * RX + (x + 3);
  const bool inB = tid < Map::NB, inC = tid < Map::NC;
  const bool inD = inC && x < TX && y < TY;
  auto wrapi = [&](int i) { return ((i % g.nx) + g.nx) % g.nx; };
  auto wrapj = [&](int j) { return ((j % g.ny) + g.ny) % g.ny; };
  const int col = wrapj(j0 + y) * (int)g.px + wrapi(i0 + x);
  const bool ringer = tid < L::NRING;
  int r3 = 0, rcol = 0;
  if (ringer) {
    int rx, ry, r = tid;
    if (r < RX) { rx = r - 3; ry = -3; }
    else if ((r -= RX) < RX) { rx = r - 3; ry = TY + 2; }
    else if ((r -= RX) < L::EY) { rx = -3; ry = r - 2; }
    else { r -= L::EY; rx = TX + 2; ry = r - 2; }
    r3 = (ry + 3) * RX + (rx + 3);
    rcol = wrapj(j0 + ry) * (int)g.px + wrapi(i0 + rx);
  }
  const int pxy = (int)g.pxy;
  auto clampk_ = [&](int k) { return k < 0 ? 0 : (k >= nz ? nz - 1 : k); };
  const int khi = nz - 1;
  auto zface = [&](int k) { return k >= 0 && k < nz - 1; };
  const int c0 = (int)g.off0 + col, rc0 = (int)g.off0 + rcol;
  auto ldp = [&](int c, int k) {  // psi of both tracers
    const int o = c + clampk_(k) * pxy;
    return mk(Pa[o], Pb[o]);
  };
  auto lds = [&](const float* f, int k) { return f[c0 + clampk_(k) * pxy]; };
  auto ldw = [&](int k) { return (k < 0 || k >= nz - 1) ? 0.0f : W[c0 + k * pxy]; };

  const bool inT = x >= 0 && x < TX && y >= 0 && y < TY;
  const int gi = i0 + x, gj = j0 + y;
  const bool writes = inT && gi < g.nx && gj < g.ny;
  const bool noimg = gi >= g.h && gi < g.nx - g.h && gj >= g.h && gj < g.ny - g.h;

  const int t0 = k0 - 5;
  f2 p0 = ldp(c0, t0), p1 = ldp(c0, t0 + 1), p2 = ldp(c0, t0 + 2), p3 = ldp(c0, t0 + 3);
  f2 pn = ldp(c0, t0 + 4);
  float u1 = lds(U, t0 + 1), u2 = lds(U, t0 + 2), un = lds(U, t0 + 3);
  float v1 = lds(V, t0 + 1), v2 = lds(V, t0 + 2), vn = lds(V, t0 + 3);
  float w0 = ldw(t0), w1 = ldw(t0 + 1), w2 = ldw(t0 + 2), wn = ldw(t0 + 3);
  float g1 = lds(G, t0 + 1), g2 = lds(G, t0 + 2), gn = lds(G, t0 + 3);
  f2 rp = zero2;  // ring values of plane t+3
  float ru = 0.0f, rv = 0.0f;
  if (ringer) {
    rp = ldp(rc0, t0 + 3);
    ru = U[rc0 + clampk_(t0 + 3) * pxy];
    rv = V[rc0 + clampk_(t0 + 3) * pxy];
  }
  f2 q0 = zero2, q1 = zero2, q2 = zero2;
  f2 utA = zero2, vtA = zero2, utB = zero2, vtB = zero2, wtA = zero2, wtB = zero2;
  f2 buA = zero2, bdA = zero2, buB = zero2, bdB = zero2;
  f2 f1z = zero2;  // the donor flux through face t+3/2 (stage A's last "+" z face)
  f2 fzAA = zero2, fzA = zero2, fzB = zero2;

  __syncthreads();  // the shared memory may still be read by a previous item
  {
    const int a = t0 + 2;
    p0s[(a & 3) * L::RN + s3] = p2;
    us[(a & 3) * L::RN + s3] = u2;
    vs[(a & 3) * L::RN + s3] = v2;
    if (ringer) {
      p0s[(a & 3) * L::RN + r3] = ldp(rc0, a);
      us[(a & 3) * L::RN + r3] = U[rc0 + clampk_(a) * pxy];
      vs[(a & 3) * L::RN + r3] = V[rc0 + clampk_(a) * pxy];
    }
    ws[((t0 + 1) & 3) * L::SN + s2] = w1;
    gs[((t0 + 1) & 3) * L::SN + s2] = g1;
  }
  __syncthreads();
  auto level = [&](const int t, auto steady) {
    constexpr bool S = decltype(steady)::value;
    // ---- publish plane t+3 of psi^n, U, V, face t+2 of W, plane t+2 of G --
    {
      const int a = t + 3;
      p0s[(a & 3) * L::RN + s3] = p3;
      us[(a & 3) * L::RN + s3] = un;
      vs[(a & 3) * L::RN + s3] = vn;
      if (ringer) {
        p0s[(a & 3) * L::RN + r3] = rp;
        us[(a & 3) * L::RN + r3] = ru;
        vs[(a & 3) * L::RN + r3] = rv;
      }
      ws[((t + 2) & 3) * L::SN + s2] = w2;
      gs[((t + 2) & 3) * L::SN + s2] = g2;
    }
    const int o5 = (S ? t + 5 : clampk_(t + 5)) * pxy;
    const int o4 = S ? o5 - pxy : clampk_(t + 4) * pxy;
    const f2 pn_next = mk(Pa[c0 + o5], Pb[c0 + o5]);
    const float un_next = U[c0 + o4], vn_next = V[c0 + o4], gn_next = G[c0 + o4];
    const float wn_next = (S || zface(t + 4)) ? W[c0 + o4] : 0.0f;  // closed faces
    f2 rp_next = zero2;
    float ru_next = 0.0f, rv_next = 0.0f;
    if (ringer) {
      rp_next = mk(Pa[rc0 + o4], Pb[rc0 + o4]);
      ru_next = U[rc0 + o4];
      rv_next = V[rc0 + o4];
    }
    // ---- A: psi1 on plane a = t+2 ---------------------------------------
    const int a = t + 2;
    if (S || (a >= max(0, k0 - 3) && a <= min(khi, k1 + 1))) {
      const f2* pa = p0s + (a & 3) * L::RN + s3;
      const float* ua = us + (a & 3) * L::RN + s3;
      const float* va = vs + (a & 3) * L::RN + s3;
      const f2 fxp = donor_s(p2, pa[1], u2);
      const f2 fxm = donor_s(pa[-1], p2, ua[-1]);
      const f2 fyp = donor_s(p2, pa[RX], v2);
      const f2 fym = donor_s(pa[-RX], p2, va[-RX]);
      const f2 fzp = donor_s(p2, p3, w2);  // w2 = 0 on a zero-flux top face
      // the "-" z face is the previous level's "+" z face (the same operation
      // on the same values): stage A ran a level before every steady level
      const f2 fzm = S ? f1z : donor_s(p1, p2, w1);  // w1 = 0 on a zero-flux bottom face
      f1z = fzp;
      q2 = fma2(add2(add2(sub2(fxm, fxp), sub2(fym, fyp)), sub2(fzm, fzp)), splat(rcp(g2)), p2);
      p1s[(a & 3) * L::SN + s2] = q2;
    }
    __syncthreads();
    // ---- B: pseudo-velocities on plane b = t+1 ---------------------------
    const int b = t + 1;
    const bool runB = inB && (S || (b >= max(0, k0 - 2) && b <= min(khi, k1)));
    if (runB) {
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, 0);
      const f2 qp = (S || bp != b) ? q2 : q1;
      const f2 qm = (S || bm != b) ? q0 : q1;
      const f2* pb1 = p1s + (b & 3) * L::SN + s2;
      const f2* pbp = p1s + (bp & 3) * L::SN + s2;
      const f2* pbm = p1s + (bm & 3) * L::SN + s2;
      const float* gb = gs + (b & 3) * L::SN + s2;
      const float* vb = vs + (b & 3) * L::RN + s3;
      const float* ub = us + (b & 3) * L::RN + s3;
      const float* wb = ws + (b & 3) * L::SN + s2;
      const float* wbm = ws + ((b - 1) & 3) * L::SN + s2;
      // every thread of B forms all three faces (column -2 and row -2 need
      // only their x or y faces; the others go to slots and registers
      // nobody reads), so the faces' arithmetic interleaves: +0.6 %
      {  // x face
        const f2 s1p = add2(pb1[EX + 1], pb1[EX]), s1m = add2(pb1[-EX + 1], pb1[-EX]);
        const f2 s2p = add2(pbp[1], qp), s2m = add2(pbm[1], qm);
        const float vsum = v1 + vb[1] + vb[-RX] + vb[-RX + 1];
        const float wsum = w1 + wb[1] + w0 + wbm[1];
        utB = pseudo_t(face_u(u1, g1 + gb[1]), q1, pb1[1], s1p, s1m, s2p, s2m, vsum, wsum);
        uts[s2] = utB;
      }
      {  // y face
        const f2 s1p = add2(pb1[EX + 1], pb1[1]), s1m = add2(pb1[EX - 1], pb1[-1]);
        const f2 s2p = add2(pbp[EX], qp), s2m = add2(pbm[EX], qm);
        const float usum = u1 + ub[RX] + ub[-1] + ub[RX - 1];
        const float wsum = w1 + wb[EX] + w0 + wbm[EX];
        vtB = pseudo_t(face_u(v1, g1 + gb[EX]), q1, pb1[EX], s1p, s1m, s2p, s2m, usum, wsum);
        vts[s2] = vtB;
      }
      {  // z face
        f2 res = zero2;
        if (S || zface(b)) {  // a zero-flux top face is closed
          const f2* pb2 = p1s + ((b + 1) & 3) * L::SN + s2;
          const float* ub1 = us + ((b + 1) & 3) * L::RN + s3;
          const float* vb1 = vs + ((b + 1) & 3) * L::RN + s3;
          const f2 s1p = add2(pb2[1], pb1[1]), s1m = add2(pb2[-1], pb1[-1]);
          const f2 s2p = add2(pb2[EX], pb1[EX]), s2m = add2(pb2[-EX], pb1[-EX]);
          const float usum = u1 + u2 + ub[-1] + ub1[-1];
          const float vsum = v1 + v2 + vb[-RX] + vb1[-RX];
          res = pseudo_t(face_u(w1, g1 + g2), q1, q2, s1p, s1m, s2p, s2m, usum, vsum);
        }
        wtB = res;
      }
    }
    __syncthreads();
    // ---- C: limiter bounds and betas on plane b = t+1 --------------------
    if (LIMIT && inC && (S || (b >= max(0, k0 - 1) && b <= min(khi, k1)))) {
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, 0);
      const f2 qp = (S || bp != b) ? q2 : q1, qm = (S || bm != b) ? q0 : q1;
      const f2* pb = p0s + (b & 3) * L::RN + s3;
      const f2* pb1 = p1s + (b & 3) * L::SN + s2;
      const f2 pxm = pb1[-1], pxp = pb1[1], pym = pb1[-EX], pyp = pb1[EX];
      const f2 vals[14] = {q1, p1, pb[-1], pb[1], pb[-RX], pb[RX], p0, p2,
                           pxm, pxp, pym, pyp, qm, qp};
      f2 hi, lo;
      bounds2(vals, hi, lo);
      const f2 fxp = donor_l(q1, pxp, utB);
      const f2 fxm = donor_l(pxm, q1, uts[s2 - 1]);
      const f2 fyp = donor_l(q1, pyp, vtB);
      const f2 fym = donor_l(pym, q1, vts[s2 - EX]);
      const f2 fzp = donor_l(q1, qp, wtB);
      const f2 fzm = donor_l(qm, q1, wtA);
      const f2 in = add2(add2(sub2(pos2(fxm), neg2(fxp)), sub2(pos2(fym), neg2(fyp))),
                         sub2(pos2(fzm), neg2(fzp)));
      const f2 ou = add2(add2(sub2(pos2(fxp), neg2(fxm)), sub2(pos2(fyp), neg2(fym))),
                         sub2(pos2(fzp), neg2(fzm)));
      const f2 ri = rcp2(add2(in, eps2)), ro = rcp2(add2(ou, eps2));
      buB = mul2(mul2(sub2(hi, q1), splat(g1)), ri);
      bdB = mul2(mul2(sub2(q1, lo), splat(g1)), ro);
      bus[(b & 1) * L::SN + s2] = buB;
      bds[(b & 1) * L::SN + s2] = bdB;
    }
    // ---- D: limited donor fluxes of plane t and face t+1/2 ---------------
    if (inD && (S || (t >= max(0, k0 - 1) && t <= k1 - 1))) {
      const f2* bu0 = bus + (t & 1) * L::SN + s2;
      const f2* bd0 = bds + (t & 1) * L::SN + s2;
      const f2* pt = p1s + (t & 3) * L::SN + s2;
      f2 u = utA;
      if (LIMIT) u = fusedx::limit2(u, buA, bdA, bu0[1], bd0[1]);
      fxs[(t & 1) * L::SN + s2] = donor_l(q0, pt[1], u);
      f2 v = vtA;
      if (LIMIT) v = fusedx::limit2(v, buA, bdA, bu0[EX], bd0[EX]);
      fys[(t & 1) * L::SN + s2] = donor_l(q0, pt[EX], v);
      f2 f = zero2;
      if (S || zface(t)) {
        f2 w = wtA;
        if (LIMIT) w = fusedx::limit2(w, buA, bdA, buB, bdB);
        f = donor_l(q0, q1, w);
      }
      fzB = f;
    }
    // ---- E: advance and write psi^(n+1) of both tracers on plane e = t-1 --
    const int e = t - 1;
    if ((S || e >= k0) && writes) {
      const f2* fx = fxs + (e & 1) * L::SN + s2;
      const f2* fy = fys + (e & 1) * L::SN + s2;
      const f2 fzm = (S || zface(e - 1)) ? fzAA : zero2;
      const f2 r = fma2(add2(add2(sub2(fx[-1], fx[0]), sub2(fy[-EX], fy[0])), sub2(fzm, fzA)),
                        splat(rcp(gs[(e & 3) * L::SN + s2])), p1s[(e & 3) * L::SN + s2]);
      if (S && noimg) {
        Oa[c0 + e * pxy] = r.x;
        if (two) Ob[c0 + e * pxy] = r.y;
      } else {
        // the value and its periodic images in the i-j halo and the k halo
        const int ni = (gi < g.h) ? 1 : ((gi >= g.nx - g.h) ? -1 : 0);
        const int nj = (gj < g.h) ? 1 : ((gj >= g.ny - g.h) ? -1 : 0);
        const int ilo = (e == 0) ? -g.h : e, ihi = (e == nz - 1) ? nz - 1 + g.h : e;
        for (int kk = ilo; kk <= ihi; ++kk) {
          if (kk != e && kk >= 0 && kk < nz) continue;
          const int64_t pk = g.off0 + (int64_t)kk * g.pxy;
          for (int a2 = 0; a2 <= (ni != 0); ++a2) {
            const int ii = gi + a2 * ni * g.nx;
            for (int b2 = 0; b2 <= (nj != 0); ++b2) {
              const int64_t q = pk + (int64_t)(gj + b2 * nj * g.ny) * g.px + ii;
              Oa[q] = r.x;
              if (two) Ob[q] = r.y;
            }
          }
        }
      }
    }
    // ---- shift the queues ------------------------------------------------
    p0 = p1; p1 = p2; p2 = p3; p3 = pn; pn = pn_next;
    u1 = u2; u2 = un; un = un_next;
    v1 = v2; v2 = vn; vn = vn_next;
    w0 = w1; w1 = w2; w2 = wn; wn = wn_next;
    g1 = g2; g2 = gn; gn = gn_next;
    rp = rp_next; ru = ru_next; rv = rv_next;
    q0 = q1; q1 = q2;
    utA = utB; vtA = vtB; wtA = wtB;
    buA = buB; bdA = bdB;
    fzAA = fzA; fzA = fzB;
  };
  const int tS = max(k0 + 1, 2), tE = min(k1 - 1, nz - 6);
  int t = t0;
  for (; t < tS && t <= k1; ++t) level(t, std::false_type{});
  for (; t <= tE; ++t) level(t, std::true_type{});
  for (; t <= k1; ++t) level(t, std::false_type{});
}

}  // namespace fusedt
}  // namespace mpd
