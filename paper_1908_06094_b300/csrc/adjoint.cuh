// adjoint.cuh -- reverse mode of one MPDATA step (iord 1 or 2, with or
// without the limiter) on the GPU.
//
// The forward intermediates of the step (psi1, the pseudo-velocities, the
// betas and the limited velocities) come from a tape recorded by the staged
// forward kernels; the kernels here run the forward stages backwards:
//   * the two advance reverses gather per cell, without atomics, and store
//     their outputs (no zeroing);
//   * the limiter reverse runs inside the second advance reverse, on each
//     limited-velocity adjoint it produces; it and the beta reverse scatter
//     the adjoints of the betas, bounds and fluxes with atomic adds;
//   * the pseudo-velocity reverse, the heaviest, runs on the k-marching
//     tile scaffold of march.cuh: FP64 stores per-face weights and gathers
//     them in a second pass (RevPseudo, rev_pg_kernel), FP32 accumulates
//     them in shared memory in one pass (RevPseudoAcc).
// Periodic and clamped neighbours are addressed by wrapped indices, so the
// reverse of the halo fill is implicit.
//
// Derivatives follow the branch the forward took, with the tie rules
// max(a,b) = a if a >= b, min(a,b) = a if a <= b, d|x| = sign(x) dx with
// sign(0) = 0; the bounds are folded in the order psi^n(c), psi1(c), then
// psi^n and psi1 at the -x, +x, -y, +y, -z, +z neighbours, and the
// derivative of a bound goes to the value that won the fold.
#pragma once
#include "grid.cuh"
#include "staged.cuh"
#include "march.cuh"

namespace mpd {
namespace adj {

using staged::Cell;
using staged::cell_of;

template <class T> __device__ __forceinline__ void aadd(T* p, T v) { atomicAdd(p, v); }

// s = ob/G per interior cell (the FP64 input of the gather form).
template <class T>
__global__ void rev_scale_kernel(Geo g, const T* __restrict__ ob, const T* __restrict__ G,
                                 T* __restrict__ sf) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  sf[q] = ob[q] * rcp(G[q]);
}

// Reverse of the limited velocity of a face (see the tie rules above).
template <class T>
__device__ __forceinline__ void rev_limit_face(T lb, T Ut, T buL, T bdL, T buR, T bdR, T* Utb,
                                               T* buLb, T* bdLb, T* buRb, T* bdRb) {
  const bool p_is_bdL = !leq(T(1), bdL);
  const T m1 = p_is_bdL ? bdL : T(1);
  const bool p_first = leq(m1, buR);
  const T cpos = p_first ? m1 : buR;
  const bool n_is_buL = !leq(T(1), buL);
  const T n1 = n_is_buL ? buL : T(1);
  const bool n_first = leq(n1, bdR);
  const T cneg = n_first ? n1 : bdR;
  const bool ge = ge0(Ut), le = le0(Ut);
  *Utb = lb * ((ge ? cpos : T(0)) + (le ? cneg : T(0)));  // the face's first writer
  // d/d(beta) of c * [Ut]+ (or [Ut]-) is lb * Ut on the branch Ut's sign
  // takes, and exactly zero on the other one or when Ut or lb is zero: only
  // non-zero adjoints are added
  if (ge && le) return;
  const T cb = lb * Ut;
  if (ge0(cb) && le0(cb)) return;
  if (ge) {
    if (!p_first) aadd(buRb, cb);
    else if (p_is_bdL) aadd(bdLb, cb);
  } else {
    if (!n_first) aadd(bdRb, cb);
    else if (n_is_buL) aadd(buLb, cb);
  }
}

// Reverse of the advance out = P - (1/G) sum_d [F(P_c, P_c+d, C_c) -
// F(P_c-d, P_c, C_c-d)] for the adjoint ob of out.
// It runs in gather form, without atomics.  With s = ob/G, the adjoint of
// the flux through face f = (L, R) is Fb = s_R - s_L; cell q takes the
// upwind partial Fb*C of each of its six faces where it is the upwind value
// (C > 0 on its "+" faces, C < 0 on its "-" faces; both partials vanish at
// C = 0), and hands the velocity adjoint Fb*(upwind value) (L + R at
// C = 0) of each of its own three "+" faces to out(fam, q, n, cb, pre) (n
// the face's right cell, pre = out.pre(fam, q, n), the values out reads),
// and its closed top face to out.closed(q).  ADD_P:
// Pb = Pin + the gathered sum and Pin is cleared (its only reader; Pin and
// Pb distinct), else Pb = the sum (the field's first writer).  Pb must not
// alias ob.  S: s comes
// precomputed in sf (FP64, where six neighbour reciprocals would cost 24
// FP64 instructions), else it is formed from ob and G.
// Every load is issued before the first store: the kernel is bound by load
// latency, and with output fields that are not restrict-qualified a load
// placed after a store could not be moved above it.
template <class T, bool ADD_P, bool S, class Out>
__global__ void rev_advance_gather_kernel(Geo g, const T* __restrict__ P,
                                          const T* __restrict__ cu, const T* __restrict__ cv,
                                          const T* __restrict__ cw, const T* __restrict__ G,
                                          const T* __restrict__ ob, const T* __restrict__ sf,
                                          T* Pin, T* Pb, Out out) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  const bool zt = zopen(g, c.k), zb = zopen(g, c.k - 1);
  const int64_t xp = at(g, wrap_up(c.i, g.nx), c.j, c.k), xm = at(g, wrap_dn(c.i, g.nx), c.j, c.k);
  const int64_t yp = at(g, c.i, wrap_up(c.j, g.ny), c.k), ym = at(g, c.i, wrap_dn(c.j, g.ny), c.k);
  // a closed face takes q as an in-bounds stand-in (its values are unused)
  const int64_t zp = zt ? at(g, c.i, c.j, kadj(g, c.k + 1)) : q;
  const int64_t zm = zb ? at(g, c.i, c.j, kadj(g, c.k - 1)) : q;
  auto s_at = [&](int64_t n) { return S ? sf[n] : ob[n] * rcp(G[n]); };
  const T obq = ob[q], pc = P[q];
  const T sq = S ? sf[q] : obq * rcp(G[q]);
  const T sxp = s_at(xp), sxm = s_at(xm), syp = s_at(yp), sym = s_at(ym);
  const T szp = s_at(zp), szm = s_at(zm);
  const T pxp = P[xp], pyp = P[yp], pzp = P[zp];
  const T cx = cu[q], cy = cv[q], cz = cw[q], cxm = cu[xm], cym = cv[ym], czm = cw[zm];
  const T pin = ADD_P ? Pin[q] : T(0);
  const typename Out::Pre ox = out.pre(0, q, xp), oy = out.pre(1, q, yp), oz = out.pre(2, q, zp);
  T acc = obq;
  // "+" face to neighbour n with Courant number C (q is its left value)
  auto plus = [&](T sn, T pn, T C) {
    const T Fb = sn - sq;
    const bool ge = ge0(C), le = le0(C);
    if (ge && le) return Fb * (pc + pn);
    if (ge) acc += Fb * C;
    return Fb * (ge ? pc : pn);
  };
  // "-" face from neighbour n (q is its right value)
  auto minus = [&](T sn, T C) {
    if (!ge0(C)) acc += (sq - sn) * C;
  };
  const T bx = plus(sxp, pxp, cx);
  minus(sxm, cxm);
  const T by = plus(syp, pyp, cy);
  minus(sym, cym);
  T bz = T(0);
  if (zt) bz = plus(szp, pzp, cz);
  if (zb) minus(szm, czm);
  out(0, q, xp, bx, ox);
  out(1, q, yp, by, oy);
  if (zt) out(2, q, zp, bz, oz);
  else out.closed(q);
  if (ADD_P) {
    Pb[q] = pin + acc;
    Pin[q] = T(0);
  } else {
    Pb[q] = acc;
  }
}

// Velocity adjoints of the advance reverse into fields: added (ADD) or
// stored (the fields' first writer; the closed top face gets 0), with the
// carried adjoints au, av, aw of the same velocities added when not null.
template <class T, bool ADD>
struct VelOut {
  T *ub, *vb, *wb;
  const T *au, *av, *aw;
  struct Pre { T a, f; };
  __device__ __forceinline__ Pre pre(int fam, int64_t q, int64_t) const {
    const T* a = fam == 0 ? au : fam == 1 ? av : aw;
    const T* f = fam == 0 ? ub : fam == 1 ? vb : wb;
    return Pre{a ? a[q] : T(0), ADD ? f[q] : T(0)};
  }
  __device__ __forceinline__ void operator()(int fam, int64_t q, int64_t, T cb,
                                             const Pre& p) const {
    T* f = fam == 0 ? ub : fam == 1 ? vb : wb;
    const T* a = fam == 0 ? au : fam == 1 ? av : aw;
    if (a) cb += p.a;
    f[q] = ADD ? p.f + cb : cb;
  }
  __device__ __forceinline__ void closed(int64_t q) const {
    if (!ADD) wb[q] = T(0);
  }
};

// The limiter's reverse applied to each limited-velocity adjoint as the
// advance reverse produces it (the limiter reverse is its only reader):
// stores the unlimited-velocity adjoints and scatters the beta adjoints.
// au, av, aw (when not null): further adjoints of the same limited
// velocities, from the next pass that took them as its input velocities.
template <class T>
struct LimitOut {
  const T *ut, *vt, *wt, *bu, *bd;
  T *utb, *vtb, *wtb, *bub, *bdb;
  const T *au, *av, *aw;
  struct Pre { T a, U, buL, bdL, buR, bdR; };
  __device__ __forceinline__ Pre pre(int fam, int64_t q, int64_t n) const {
    const T* a = fam == 0 ? au : fam == 1 ? av : aw;
    const T* U = fam == 0 ? ut : fam == 1 ? vt : wt;
    return Pre{a ? a[q] : T(0), U[q], bu[q], bd[q], bu[n], bd[n]};
  }
  __device__ __forceinline__ void operator()(int fam, int64_t q, int64_t n, T lb,
                                             const Pre& p) const {
    const T* a = fam == 0 ? au : fam == 1 ? av : aw;
    if (a) lb += p.a;
    T* Ub = fam == 0 ? utb : fam == 1 ? vtb : wtb;
    rev_limit_face(lb, p.U, p.buL, p.bdL, p.buR, p.bdR, &Ub[q], &bub[q], &bdb[q], &bub[n],
                   &bdb[n]);
  }
  __device__ __forceinline__ void closed(int64_t q) const { wtb[q] = T(0); }
};

// Reverse of the beta stage from the tape (beta-up/down, and in FP64 the
// reciprocals ri = 1/(in+eps), ro = 1/(out+eps) of the forward):
//   beta_up = (hi - psi) G ri,  beta_dn = (psi - lo) G ro,
// in = sum of incoming antidiffusive fluxes, out = outgoing.  A cell whose
// two beta adjoints are zero (its betas never won the limiter's min)
// contributes exactly nothing and returns at once.  The adjoint of a face
// flux F from this cell's in/out is outb (F > 0) or -inb (F < 0) on its
// "+" faces, inb or -outb on its "-" faces, and both (outb - inb) when F is
// zero; it then goes to the upwind psi1 value and the face's velocity.
template <class T>
__global__ void rev_beta_kernel(Geo g, const T* __restrict__ P0, const T* __restrict__ P,
                                const T* __restrict__ ut, const T* __restrict__ vt,
                                const T* __restrict__ wt, const T* __restrict__ G,
                                const T* __restrict__ bu, const T* __restrict__ bd,
                                const T* __restrict__ rin, const T* __restrict__ rout,
                                T* __restrict__ bub, T* __restrict__ bdb, T* P0b,
                                T* Pb, T* utb, T* vtb, T* wtb) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int i = c.i, j = c.j, k = c.k;
  const int64_t q = at(g, i, j, k);
  const T ab = bub[q], db = bdb[q];
  if (ge0(ab) && le0(ab) && ge0(db) && le0(db)) return;
  bub[q] = bdb[q] = T(0);  // the only reader: leave them zero for the next step
  const int64_t nb[6] = {at(g, wrap_dn(i, g.nx), j, k), at(g, wrap_up(i, g.nx), j, k),
                         at(g, i, wrap_dn(j, g.ny), k), at(g, i, wrap_up(j, g.ny), k),
                         at(g, i, j, kadj(g, k - 1)), at(g, i, j, kadj(g, k + 1))};
  T hi = P0[q], lo = P0[q];
  T* hip = &P0b[q];
  T* lop = &P0b[q];
  if (!geq(hi, P[q])) { hi = P[q]; hip = &Pb[q]; }
  if (!leq(lo, P[q])) { lo = P[q]; lop = &Pb[q]; }
  for (int s = 0; s < 6; ++s) {
    const int64_t n = nb[s];
    if (!geq(hi, P0[n])) { hi = P0[n]; hip = &P0b[n]; }
    if (!geq(hi, P[n])) { hi = P[n]; hip = &Pb[n]; }
    if (!leq(lo, P0[n])) { lo = P0[n]; lop = &P0b[n]; }
    if (!leq(lo, P[n])) { lo = P[n]; lop = &Pb[n]; }
  }
  const T pc = P[q];
  const T* vel[3] = {ut, vt, wt};
  T* velb[3] = {utb, vtb, wtb};
  // the six face fluxes (0 through the closed bottom and top faces)
  bool hp[3], hm[3];
  T Cp[3], Cm[3], Pr[3], Pl[3], fp[3], fm[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    hp[d] = d != 2 || zopen(g, k);
    hm[d] = d != 2 || zopen(g, k - 1);
    Cp[d] = hp[d] ? vel[d][q] : T(0);
    Pr[d] = P[nb[2 * d + 1]];
    fp[d] = donor(pc, Pr[d], Cp[d]);
    Cm[d] = hm[d] ? vel[d][nb[2 * d]] : T(0);
    Pl[d] = P[nb[2 * d]];
    fm[d] = donor(Pl[d], pc, Cm[d]);
  }
  T ri, ro;
  if constexpr (sizeof(T) == 4) {
    // FP32 re-forms 1/(in+eps), 1/(out+eps) from the fluxes, as the forward
    // did (the same sums in the same order), instead of taping them
    const T in = (pos(fm[0]) - neg(fp[0])) + (pos(fm[1]) - neg(fp[1])) + (pos(fm[2]) - neg(fp[2]));
    const T ou = (pos(fp[0]) - neg(fm[0])) + (pos(fp[1]) - neg(fm[1])) + (pos(fp[2]) - neg(fm[2]));
    ri = rcp(in + Eps<T>::v);
    ro = rcp(ou + Eps<T>::v);
  } else {
    ri = rin[q];
    ro = rout[q];
  }
  const T gc = G[q];
  const T x = ab * gc * ri, y = db * gc * ro;  // d beta_up/d hi, -d beta_dn/d lo
  aadd(hip, x);
  aadd(lop, -y);
  aadd(&Pb[q], y - x);
  const T inb = -ab * bu[q] * ri, outb = -db * bd[q] * ro;
  const T dio = outb - inb;
  // reverse of F = donor(L, R, C) for the adjoint fb: only the upwind value
  // has a non-zero partial (both are 0 * fb when C == 0)
  auto rdonor = [&](T fb, T L, T R, T C, T* Lb, T* Rb, T* Cb) {
    const bool ge = ge0(C), le = le0(C);
    if (ge && le) {
      aadd(Cb, fb * (L + R));
      return;
    }
    aadd(ge ? Lb : Rb, fb * C);
    aadd(Cb, fb * (ge ? L : R));
  };
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (hp[d]) {
      const int64_t r = nb[2 * d + 1];
      const T fpb = ge0(fp[d]) ? (le0(fp[d]) ? dio : outb) : -inb;
      rdonor(fpb, pc, Pr[d], Cp[d], &Pb[q], &Pb[r], &velb[d][q]);
    }
    if (hm[d]) {
      const int64_t l = nb[2 * d];
      const T fmb = ge0(fm[d]) ? (le0(fm[d]) ? -dio : inb) : -outb;
      rdonor(fmb, Pl[d], pc, Cm[d], &Pb[l], &Pb[q], &velb[d][l]);
    }
  }
}

// ---------------------------------------------------------------------------
// Pseudo-velocity reverse in gather form (no atomics).
//
// Pass 1 (face_weights, RevPseudo), per cell and its three "+" faces f, from the
// adjoint ub_f of the pseudo-velocity: adds dJ/dU_f (own face) and stores
// eight weights per face, the adjoint routed to each stencil point:
//   wl, wr    to psi1 at L and R through A,
//   w1p, w1m  to the two psi1 values on each side of the first cross
//             direction (B1), w2p, w2m the same for B2,
//   c1, c2    to each of the four Courant faces of the two cross averages.
// Pass 2 (rev_pg_kernel), per cell q: gathers every weight whose stencil
// point is q (about thirty faces) into dJ/dpsi1_q, and the cross weights
// of the eight faces whose averages contain each of q's three Courant
// faces.  The clamped k neighbours of the boundary levels gather the
// weights of the faces whose clamped index lands on them.
enum { kWL = 0, kWR, kW1P, kW1M, kW2P, kW2M, kC1, kC2, kNW };

// sign(U) with sign(0) = 0
template <class T>
__device__ __forceinline__ T sgn0(T U) {
  return (ge0(U) && le0(U)) ? T(0) : (nonneg(U) ? T(1) : T(-1));
}

// Pass 1 as the face operation of march::march_kernel, which supplies each
// face's ingredients from pair sums shared across the tile.  With
// B1' = N1/D1 = 2 B1, B2' = 2 B2, qh = U/(G_L+G_R) (so U/G_face = 2 qh) and
// X8 = s1 B1' + s2 B2' (8x the cross term Vbar B1 + Wbar B2):
//   dUt/dU = A (sign U - 4 qh) - X8 rG2 / 4 with rG2 = 1/(G_L+G_R);
//   wl, wr = -(ub Dd/DA) (1 + A), (ub Dd/DA) (1 - A), Dd = |U| - U^2/G_face;
//   w1p, w1m = t1 (1 - B1'), -t1 (1 + B1') with t1 = m4 s1 / D1,
//            m4 = -ub qh / 4 (w2p, w2m the same with s2, D2, B2');
//   c1, c2 = m4 B1', m4 B2'.
// The factors 1/4 ride on the reciprocal: rq = 1/(4 (G_L+G_R)) (the 4 an
// exponent step) and qq = -U rq = -qh/4, so that m4 = ub qq, 4 qh = -16 qq,
// 2 U qh = -8 U qq and X8 rG2 / 4 = X8 rq: two FP64 products a face fewer.
// The eight weights and the direct adjoint ub * dUt/dU of one face (see
// above), for the face adjoint ub.
template <class T>
struct FaceW {
  T wl, wr, w1p, w1m, w2p, w2m, c1, c2, du;
};

template <class T>
__device__ __forceinline__ FaceW<T> face_weights(const march::FaceIn<T>& f, T ubv) {
  const T rd = rcp(f.DA), rd1 = rcp(f.D1), rd2 = rcp(f.D2), rq = rcp(march::times4(f.gsum));
  const T A = (f.pr - f.pl) * rd, B1 = f.N1 * rd1, B2 = f.N2 * rd2;
  const T qq = -f.U * rq;
  const T Dd = fma_rn(f.U * T(8), qq, absv(f.U));
  const T X8 = fma_rn(f.s2, B2, f.s1 * B1);
  const T dU = fma_rn(-X8, rq, A * fma_rn(qq, T(16), sgn0(f.U)));
  const T Abr = ubv * Dd * rd;
  const T m4 = ubv * qq;
  const T t1 = m4 * f.s1 * rd1, t2 = m4 * f.s2 * rd2;
  return FaceW<T>{fma_rn(-Abr, A, -Abr), fma_rn(-Abr, A, Abr), fma_rn(-t1, B1, t1),
                  fma_rn(-t1, B1, -t1),  fma_rn(-t2, B2, t2),  fma_rn(-t2, B2, -t2),
                  m4 * B1,               m4 * B2,              ubv * dU};
}

// Pass 1 as the cell operation of march::march_kernel (FP64): stores the
// weights for the gather pass and adds the direct adjoint to ub, vb, wb.
template <class T>
struct RevPseudo {
  using Acc = march::NoAcc;
  static constexpr bool kAccum = false;
  const T *utb, *vtb, *wtb;
  T* wts;
  int64_t F;  // one weight field
  T *ub, *vb, *wb;
  struct Load {
    T x, y, z;  // the face adjoints of the cell's three "+" faces
  };
  __device__ __forceinline__ Load load(int64_t q) const { return {utb[q], vtb[q], wtb[q]}; }
  __device__ __forceinline__ void store(int fam, int64_t q, const FaceW<T>& w) const {
    T* b = wts + (int64_t)fam * kNW * F + q;
    b[kWL * F] = w.wl;
    b[kWR * F] = w.wr;
    b[kW1P * F] = w.w1p;
    b[kW1M * F] = w.w1m;
    b[kW2P * F] = w.w2p;
    b[kW2M * F] = w.w2m;
    b[kC1 * F] = w.c1;
    b[kC2 * F] = w.c2;
  }
  __device__ __forceinline__ void cell(int64_t q, const march::FaceIn<T>& fx,
                                      const march::FaceIn<T>& fy, const march::FaceIn<T>& fz,
                                      bool top, march::CellAt, Load l, Acc&) const {
    // the accumulators' old values are read before the first store (the
    // weight stores could alias them as far as the compiler knows)
    const T u0 = ub[q], v0 = vb[q], w0 = top ? T(0) : wb[q];
    const FaceW<T> x = face_weights(fx, l.x);
    store(0, q, x);
    ub[q] = u0 + x.du;
    const FaceW<T> y = face_weights(fy, l.y);
    store(1, q, y);
    vb[q] = v0 + y.du;
    if (top) {
      store(2, q, FaceW<T>{});
    } else {
      const FaceW<T> z = face_weights(fz, l.z);
      store(2, q, z);
      wb[q] = w0 + z.du;
    }
  }
};

// The pseudo-velocity reverse in one pass (FP32): each cell adds its three
// faces' weights into shared accumulators of psi1-bar, U-, V- and W-bar,
// the contributions of one cell to one point summed first (34 targets per
// cell).  Every warp (one tile row) owns a private strip of each
// accumulator -- the rows above, at and below its own, the tile's columns
// plus the ring -- so for any one target offset its lanes write distinct
// words: plain read-add-write, a __syncwarp between offsets, no atomics.
// Levels: psi1-bar k-1, k, k+1 (a ring of three), U-, V-bar k, k+1 and
// W-bar k-1, k (rings of two).  A level is complete once no later cell of
// the CTA reaches it; its (up to three) strips are then summed in warp
// order and added to the global field with fire-and-forget atomic adds
// (the ring and the chunk's end levels are shared with other CTAs, and a
// reduction never waits for the old value, unlike a plain add).
template <class T>
struct RevPseudoAcc {
  static constexpr int TY = march::TY, C = march::TX + 2, R = TY + 2;
  static constexpr int kStrip = TY * 3 * C;  // words of one accumulator level
  struct Acc {
    T p[3 * kStrip], u[2 * kStrip], v[2 * kStrip], w[2 * kStrip];
  };
  static constexpr bool kAccum = true;
  static constexpr int kWords = 9 * kStrip;
  static constexpr int kPos = (R * C + march::TX * march::TY - 1) / (march::TX * march::TY);
  const T *utb, *vtb, *wtb;
  T *pb, *ub, *vb, *wb;
  struct Load {
    T x, y, z;
  };
  // The flush positions of one thread: shared row r, column c (tile row
  // r-1, column c-1) and the in-plane offset of their (wrapped) global point.
  struct Pos {
    int r, c;
    int64_t off;
  };
  Pos pos[kPos];
  __device__ __forceinline__ Load load(int64_t q) const { return {utb[q], vtb[q], wtb[q]}; }
  __device__ __forceinline__ void zero(Acc& a, int t) {
    T* f = a.p;
    for (int q = t; q < kWords; q += march::TX * march::TY) f[q] = T(0);
  }
  __device__ __forceinline__ void setup(const Geo& g, int i0, int j0, int t) {
#pragma unroll
    for (int m = 0; m < kPos; ++m) {
      const int e = t + m * march::TX * march::TY;
      Pos& P = pos[m];
      P.r = e / C;
      P.c = e % C;
      const int ti = P.c - 1, tj = P.r - 1;
      P.off = e < R * C ? at(g, (i0 + ti + g.nx) % g.nx, (j0 + tj + g.ny) % g.ny, 0) : 0;
    }
  }
  // v into the strip word at row offset sr (0 below, 1 own, 2 above) and
  // column offset dc from the cell, its base b = &strip[ty][0][c]
  template <int SR, int DC>
  __device__ __forceinline__ static void add(T* b, T v) {
    b[SR * C + DC] += v;
    __syncwarp();
  }
  __device__ __forceinline__ void cell(int64_t q, const march::FaceIn<T>& fx,
                                      const march::FaceIn<T>& fy, const march::FaceIn<T>& fz,
                                      bool top, march::CellAt at, Load l, Acc& a) const {
    const T own = at.own ? T(1) : T(0);  // lanes past a ragged edge add zeros
    const FaceW<T> x = face_weights(fx, own * l.x);
    const FaceW<T> y = face_weights(fy, own * l.y);
    const FaceW<T> z = top ? FaceW<T>{} : face_weights(fz, own * l.z);
    const int k = at.k, cb = (at.r - 1) * 3 * C + at.c;
    const int s3 = k % 3, s2 = k & 1;
    T* p0 = a.p + s3 * kStrip + cb;
    T* pq = a.p + (top ? s3 : (s3 == 2 ? 0 : s3 + 1)) * kStrip + cb;  // "+z" level, clamped
    // "-z" level: k-1 (a virtual level -1 under periodic k), clamped to k
    // at a zero-flux bottom
    T* pm = a.p + (k > 0 || at.kper ? (s3 == 0 ? 2 : s3 - 1) : s3) * kStrip + cb;
    // psi1-bar, same level
    add<1, 0>(p0, x.wl + y.wl + z.wl);
    add<1, 1>(p0, x.wr + y.w1p + z.w1p);
    add<2, 0>(p0, x.w1p + y.wr + z.w2p);
    add<2, 1>(p0, x.w1p + y.w1p);
    add<0, 0>(p0, x.w1m + z.w2m);
    add<0, 1>(p0, x.w1m);
    add<2, -1>(p0, y.w1m);
    add<1, -1>(p0, y.w1m + z.w1m);
    // the level above (z faces; the x, y faces' +z points)
    add<1, 0>(pq, x.w2p + y.w2p + z.wr);
    add<1, 1>(pq, x.w2p + z.w1p);
    add<2, 0>(pq, y.w2p + z.w2p);
    if (!top) {
      add<1, -1>(pq, z.w1m);
      add<0, 0>(pq, z.w2m);
    }
    // the level below (the x, y faces' -z points, clamped at the bottom)
    add<1, 0>(pm, x.w2m + y.w2m);
    add<1, 1>(pm, x.w2m);
    add<2, 0>(pm, y.w2m);
    // U-bar and V-bar at k: own face terms and the cross averages
    T* u0 = a.u + s2 * kStrip + cb;
    T* v0 = a.v + s2 * kStrip + cb;
    add<1, 0>(u0, x.du + y.c1 + z.c1);
    add<2, 0>(u0, y.c1);
    add<1, -1>(u0, y.c1 + z.c1);
    add<2, -1>(u0, y.c1);
    add<1, 0>(v0, y.du + x.c1 + z.c2);
    add<1, 1>(v0, x.c1);
    add<0, 0>(v0, x.c1 + z.c2);
    add<0, 1>(v0, x.c1);
    if (!top) {
      T* u1 = a.u + (s2 ^ 1) * kStrip + cb;
      T* v1 = a.v + (s2 ^ 1) * kStrip + cb;
      add<1, 0>(u1, z.c1);
      add<1, -1>(u1, z.c1);
      add<1, 0>(v1, z.c2);
      add<0, 0>(v1, z.c2);
      T* w0 = a.w + s2 * kStrip + cb;  // W-bar at the open face k+1/2
      add<1, 0>(w0, z.du + x.c2 + y.c2);
      add<1, 1>(w0, x.c2);
      add<2, 0>(w0, y.c2);
    }
    if (k > 0 || at.kper) {  // W-bar at the open face k-1/2
      T* wm = a.w + (s2 ^ 1) * kStrip + cb;
      add<1, 0>(wm, x.c2 + y.c2);
      add<1, 1>(wm, x.c2);
      add<2, 0>(wm, y.c2);
    }
  }
  // Sum the strips of one accumulator level (base f) into dst at level kf
  // and clear them.
  __device__ __forceinline__ void flush_one(T* f, T* dst, int kf, const Geo& g) const {
    // virtual levels -1 and nz (periodic k) are the levels nz-1 and 0
    const int kg = kf < 0 ? kf + g.nz : (kf >= g.nz ? kf - g.nz : kf);
    const int64_t ok = (int64_t)kg * g.pxy;
#pragma unroll
    for (int m = 0; m < kPos; ++m) {
      const Pos& P = pos[m];
      if (P.r >= R) continue;
      T v = T(0);
      // warps w = r-2 .. r (within the tile) hold the point in strip row r-w
#pragma unroll
      for (int d = 2; d >= 0; --d) {
        const int w = P.r - d;
        if (w >= 0 && w < TY) {
          T* x = f + (w * 3 + d) * C + P.c;
          v += *x;
          *x = T(0);
        }
      }
      if (ge0(v) && le0(v)) continue;
      atomicAdd(dst + P.off + ok, v);
    }
  }
  // After the cells of level k (and a barrier): psi1-bar and W-bar level k-1
  // and U-, V-bar level k are complete.  After the last level k1-1 (after),
  // psi1-bar k1-1, k1, U-, V-bar k1 and W-bar k1-1 remain.
  __device__ __forceinline__ void flush(Acc& a, int k, bool after, const Geo& g, int i0,
                                       int j0, int k0, int k1, int t) const {
    if (!after) {
      if (k > 0 || g.kper) {
        flush_one(a.p + ((k + 2) % 3) * kStrip, pb, k - 1, g);  // slot of k-1
        flush_one(a.w + ((k - 1) & 1) * kStrip, wb, k - 1, g);
      }
      flush_one(a.u + (k & 1) * kStrip, ub, k, g);
      flush_one(a.v + (k & 1) * kStrip, vb, k, g);
    } else {
      flush_one(a.p + ((k1 - 1) % 3) * kStrip, pb, k1 - 1, g);
      flush_one(a.w + ((k1 - 1) & 1) * kStrip, wb, k1 - 1, g);
      if (k1 < g.nz || g.kper) {
        flush_one(a.p + (k1 % 3) * kStrip, pb, k1, g);
        flush_one(a.u + (k1 & 1) * kStrip, ub, k1, g);
        flush_one(a.v + (k1 & 1) * kStrip, vb, k1, g);
      }
    }
  }
};

template <class T>
__global__ void rev_pg_kernel(Geo g, const T* __restrict__ wts, T* Pb, T* ub, T* vb, T* wb) {
  pdl_enter();
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int i = c.i, j = c.j, k = c.k, nz = g.nz;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int64_t F = g.total;
  const bool kper = g.kper != 0;
  const int kb = kadj(g, k - 1), ka = kadj(g, k + 1);  // the levels below and above
  const bool below = kper || k >= 1;                   // the face k-1/2 is open
  auto W = [&](int fam, int w, int a, int b, int d) -> T {
    return wts[((int64_t)fam * kNW + w) * F + at(g, a, b, d)];
  };
  // the accumulators' old values, read before the first store
  const int64_t q = at(g, i, j, k);
  const T p0 = Pb[q], u0 = ub[q], v0 = vb[q], w0 = zopen(g, k) ? wb[q] : T(0);
  T s = T(0);
  // x faces: A, B1 (y), B2 (z, clamped)
  s += W(0, kWL, i, j, k) + W(0, kWR, im, j, k);
  s += W(0, kW1P, i, jm, k) + W(0, kW1P, im, jm, k) + W(0, kW1M, i, jp, k) + W(0, kW1M, im, jp, k);
  // y faces: A, B1 (x), B2 (z, clamped)
  s += W(1, kWL, i, j, k) + W(1, kWR, i, jm, k);
  s += W(1, kW1P, im, j, k) + W(1, kW1P, im, jm, k) + W(1, kW1M, ip, j, k) + W(1, kW1M, ip, jm, k);
  // z neighbours of the x and y faces: q is the "+z" point of the faces at
  // level kf with kadj(kf+1) == k, the "-z" point where kadj(kf-1) == k
  // (clamped at a zero-flux bottom and top, wrapped under periodic k)
  auto zgather = [&](int kf, int w) {
    s += W(0, w, i, j, kf) + W(0, w, im, j, kf) + W(1, w, i, j, kf) + W(1, w, i, jm, kf);
  };
  if (kper) {
    zgather(kb, kW2P);
    zgather(ka, kW2M);
  } else {
    if (k >= 1) zgather(k - 1, kW2P);
    if (k == nz - 1) zgather(k, kW2P);
    if (k + 1 <= nz - 1) zgather(k + 1, kW2M);
    if (k == 0) zgather(k, kW2M);
  }
  // z faces (a zero-flux top level holds zeros)
  s += W(2, kWL, i, j, k);
  if (below) s += W(2, kWR, i, j, kb);
  s += W(2, kW1P, im, j, k) + W(2, kW1M, ip, j, k) + W(2, kW2P, i, jm, k) + W(2, kW2M, i, jp, k);
  if (below)
    s += W(2, kW1P, im, j, kb) + W(2, kW1M, ip, j, kb) + W(2, kW2P, i, jm, kb) +
         W(2, kW2M, i, jp, kb);
  Pb[q] = p0 + s;
  // cross averages: U (face i+1/2) in y faces and z faces, V in x and z, W in x and y
  T su = W(1, kC1, i, j, k) + W(1, kC1, i, jm, k) + W(1, kC1, ip, j, k) + W(1, kC1, ip, jm, k);
  su += W(2, kC1, i, j, k) + W(2, kC1, ip, j, k);
  if (below) su += W(2, kC1, i, j, kb) + W(2, kC1, ip, j, kb);
  ub[q] = u0 + su;
  T sv = W(0, kC1, i, j, k) + W(0, kC1, im, j, k) + W(0, kC1, i, jp, k) + W(0, kC1, im, jp, k);
  sv += W(2, kC2, i, j, k) + W(2, kC2, i, jp, k);
  if (below) sv += W(2, kC2, i, j, kb) + W(2, kC2, i, jp, kb);
  vb[q] = v0 + sv;
  if (zopen(g, k)) {  // open vertical face
    T sw = W(0, kC2, i, j, k) + W(0, kC2, im, j, k) + W(0, kC2, i, j, ka) + W(0, kC2, im, j, ka);
    sw += W(1, kC2, i, j, k) + W(1, kC2, i, jm, k) + W(1, kC2, i, j, ka) + W(1, kC2, i, jm, ka);
    wb[q] = w0 + sw;
  }
}

}  // namespace adj
}  // namespace mpd
