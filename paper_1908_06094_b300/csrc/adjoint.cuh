// adjoint.cuh -- reverse mode of one MPDATA step (iord 1 or 2, with or
// without the limiter) on the GPU.
//
// The forward intermediates of the step (psi1, the pseudo-velocities, the
// betas and the limited velocities) come from a tape recorded by the staged
// forward kernels; the kernels here run the forward stages backwards, one
// thread per interior cell.  The advance, limiter and beta reverses scatter:
// each thread adds the adjoint of what its cell computed into every value
// that computation read, with atomic adds.  The pseudo-velocity reverse, the
// heaviest, is a gather in two passes without atomics (rev_pw, rev_pg).
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

namespace mpd {
namespace adj {

using staged::Cell;
using staged::cell_of;

template <class T> __device__ __forceinline__ void aadd(T* p, T v) { atomicAdd(p, v); }

// Reverse of F(L,R,C) = max(C,0) L + min(C,0) R for the adjoint fb.
template <class T>
__device__ __forceinline__ void rev_donor(T fb, T L, T R, T C, T* Lb, T* Rb, T* Cb) {
  const bool ge = ge0(C), le = le0(C);
  aadd(Lb, fb * (ge ? C : T(0)));
  aadd(Rb, fb * (le ? C : T(0)));
  aadd(Cb, fb * ((ge ? L : T(0)) + (le ? R : T(0))));
}

// Reverse of out = P - (1/G) sum_d [F(P_c, P_c+d, C_c) - F(P_c-d, P_c, C_c-d)]
// for the adjoint ob of out.
template <class T>
__global__ void rev_advance_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
                                   const T* __restrict__ cv, const T* __restrict__ cw,
                                   const T* __restrict__ G, const T* __restrict__ ob,
                                   T* Pb, T* ub, T* vb, T* wb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  const T a = ob[q];
  const T s = -a * rcp(G[q]);
  const int64_t xp = at(g, wrap_up(c.i, g.nx), c.j, c.k), xm = at(g, wrap_dn(c.i, g.nx), c.j, c.k);
  const int64_t yp = at(g, c.i, wrap_up(c.j, g.ny), c.k), ym = at(g, c.i, wrap_dn(c.j, g.ny), c.k);
  // the own cell's share of all six face terms is added once
  T own = a;
  auto face = [&](T fb, T L, T R, T C, bool own_is_left, int64_t other, T* Cb) {
    const bool ge = ge0(C), le = le0(C);
    const T dl = fb * (ge ? C : T(0)), dr = fb * (le ? C : T(0));
    if (own_is_left) { own += dl; aadd(&Pb[other], dr); }
    else { own += dr; aadd(&Pb[other], dl); }
    aadd(Cb, fb * ((ge ? L : T(0)) + (le ? R : T(0))));
  };
  face(s, P[q], P[xp], cu[q], true, xp, &ub[q]);
  face(-s, P[xm], P[q], cu[xm], false, xm, &ub[xm]);
  face(s, P[q], P[yp], cv[q], true, yp, &vb[q]);
  face(-s, P[ym], P[q], cv[ym], false, ym, &vb[ym]);
  if (c.k < g.nz - 1) face(s, P[q], P[q + g.pxy], cw[q], true, q + g.pxy, &wb[q]);
  if (c.k > 0) face(-s, P[q - g.pxy], P[q], cw[q - g.pxy], false, q - g.pxy, &wb[q - g.pxy]);
  aadd(&Pb[q], own);
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
  aadd(Utb, lb * ((ge ? cpos : T(0)) + (le ? cneg : T(0))));
  const T cpb = lb * (ge ? Ut : T(0)), cnb = lb * (le ? Ut : T(0));
  if (p_first) {
    if (p_is_bdL) aadd(bdLb, cpb);
  } else {
    aadd(buRb, cpb);
  }
  if (n_first) {
    if (n_is_buL) aadd(buLb, cnb);
  } else {
    aadd(bdRb, cnb);
  }
}

template <class T>
__global__ void rev_limit_kernel(Geo g, const T* __restrict__ ut, const T* __restrict__ vt,
                                 const T* __restrict__ wt, const T* __restrict__ bu,
                                 const T* __restrict__ bd, const T* __restrict__ ulb,
                                 const T* __restrict__ vlb, const T* __restrict__ wlb, T* utb,
                                 T* vtb, T* wtb, T* bub, T* bdb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int64_t q = at(g, c.i, c.j, c.k);
  const int64_t xp = at(g, wrap_up(c.i, g.nx), c.j, c.k);
  const int64_t yp = at(g, c.i, wrap_up(c.j, g.ny), c.k);
  rev_limit_face(ulb[q], ut[q], bu[q], bd[q], bu[xp], bd[xp], &utb[q], &bub[q], &bdb[q],
                 &bub[xp], &bdb[xp]);
  rev_limit_face(vlb[q], vt[q], bu[q], bd[q], bu[yp], bd[yp], &vtb[q], &bub[q], &bdb[q],
                 &bub[yp], &bdb[yp]);
  if (c.k < g.nz - 1) {
    const int64_t zp = q + g.pxy;
    rev_limit_face(wlb[q], wt[q], bu[q], bd[q], bu[zp], bd[zp], &wtb[q], &bub[q], &bdb[q],
                   &bub[zp], &bdb[zp]);
  }
}

template <class T>
__global__ void rev_beta_kernel(Geo g, const T* __restrict__ P0, const T* __restrict__ P,
                                const T* __restrict__ ut, const T* __restrict__ vt,
                                const T* __restrict__ wt, const T* __restrict__ G,
                                const T* __restrict__ bub, const T* __restrict__ bdb, T* P0b,
                                T* Pb, T* utb, T* vtb, T* wtb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const T eps = Eps<T>::v;
  const int i = c.i, j = c.j, k = c.k;
  const int64_t q = at(g, i, j, k);
  const int64_t nb[6] = {at(g, wrap_dn(i, g.nx), j, k), at(g, wrap_up(i, g.nx), j, k),
                         at(g, i, wrap_dn(j, g.ny), k), at(g, i, wrap_up(j, g.ny), k),
                         at(g, i, j, clampk(k - 1, g.nz)), at(g, i, j, clampk(k + 1, g.nz))};
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
  const T* vel[3] = {ut, vt, wt};
  T* velb[3] = {utb, vtb, wtb};
  T fp[3], fm[3];
  bool hp[3], hm[3];
  for (int d = 0; d < 3; ++d) {
    hp[d] = !(d == 2 && k == g.nz - 1);
    hm[d] = !(d == 2 && k == 0);
    fp[d] = hp[d] ? donor(P[q], P[nb[2 * d + 1]], vel[d][q]) : T(0);
    fm[d] = hm[d] ? donor(P[nb[2 * d]], P[q], vel[d][nb[2 * d]]) : T(0);
  }
  T in = T(0), out = T(0);
  for (int d = 0; d < 3; ++d) {
    in += (ge0(fm[d]) ? fm[d] : T(0)) - (le0(fp[d]) ? fp[d] : T(0));
    out += (ge0(fp[d]) ? fp[d] : T(0)) - (le0(fm[d]) ? fm[d] : T(0));
  }
  const T gc = G[q];
  const T rin = rcp(in + eps), rout = rcp(out + eps);
  const T bu = (hi - P[q]) * gc * rin, bd = (P[q] - lo) * gc * rout;
  const T ab = bub[q], db = bdb[q];
  aadd(hip, ab * gc * rin);
  aadd(lop, -db * gc * rout);
  aadd(&Pb[q], -ab * gc * rin + db * gc * rout);
  const T inb = -ab * bu * rin, outb = -db * bd * rout;
  for (int d = 0; d < 3; ++d) {
    const T fpb = (le0(fp[d]) ? -inb : T(0)) + (ge0(fp[d]) ? outb : T(0));
    const T fmb = (ge0(fm[d]) ? inb : T(0)) - (le0(fm[d]) ? outb : T(0));
    if (hp[d]) {
      const int64_t r = nb[2 * d + 1];
      rev_donor(fpb, P[q], P[r], vel[d][q], &Pb[q], &Pb[r], &velb[d][q]);
    }
    if (hm[d]) {
      const int64_t l = nb[2 * d];
      rev_donor(fmb, P[l], P[q], vel[d][l], &Pb[l], &Pb[q], &velb[d][l]);
    }
  }
}


// ---------------------------------------------------------------------------
// Pseudo-velocity reverse in gather form (no atomics).
//
// Pass 1 (rev_pw_kernel), per cell and its three "+" faces f, from the
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

template <class T>
__global__ void rev_pw_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
                              const T* __restrict__ cv, const T* __restrict__ cw,
                              const T* __restrict__ G, const T* __restrict__ utb,
                              const T* __restrict__ vtb, const T* __restrict__ wtb,
                              T* __restrict__ wts, T* ub, T* vb, T* wb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const T eps = Eps<T>::v;
  const int i = c.i, j = c.j, k = c.k;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int kp = clampk(k + 1, g.nz), km = clampk(k - 1, g.nz);
  auto A_ = [&](int a, int b, int d) { return at(g, a, b, d); };
  auto wfv = [&](int a, int b, int d) -> T {
    return (d < 0 || d >= g.nz - 1) ? T(0) : cw[at(g, a, b, d)];
  };
  const int64_t q = A_(i, j, k);
  const int64_t F = g.total;  // one weight field
  // fam: 0 x, 1 y, 2 z; fields [fam][kNW]
  auto put = [&](int fam, int w, T v) { wts[((int64_t)fam * kNW + w) * F + q] = v; };
  auto face = [&](int fam, T ubv, T U, T Gf, T pl, T pr, T s1pv, T s1mv, T s2pv, T s2mv,
                  T C1sum, T C2sum, T* Ub) {
    const T rd = rcp(pr + pl + eps);
    const T A = (pr - pl) * rd;
    const T rd1 = rcp(s1pv + s1mv + eps), rd2 = rcp(s2pv + s2mv + eps);
    const T B1 = T(0.5) * (s1pv - s1mv) * rd1, B2 = T(0.5) * (s2pv - s2mv) * rd2;
    const T C1 = T(0.25) * C1sum, C2 = T(0.25) * C2sum;
    const T rG = rcp(Gf);
    const T Dd = absv(U) - U * U * rG;
    const T X = C1 * B1 + C2 * B2;
    const T sg = (ge0(U) && le0(U)) ? T(0) : (nonneg(U) ? T(1) : T(-1));
    *Ub += ubv * (sg * A - T(2) * U * rG * A - X * rG);
    const T Ab = ubv * Dd;
    const T B1b = ubv * (-U * C1 * rG), B2b = ubv * (-U * C2 * rG);
    put(fam, kWL, Ab * (T(-1) - A) * rd);
    put(fam, kWR, Ab * (T(1) - A) * rd);
    put(fam, kW1P, B1b * (T(0.5) - B1) * rd1);
    put(fam, kW1M, B1b * (T(-0.5) - B1) * rd1);
    put(fam, kW2P, B2b * (T(0.5) - B2) * rd2);
    put(fam, kW2M, B2b * (T(-0.5) - B2) * rd2);
    put(fam, kC1, T(0.25) * ubv * (-U * B1 * rG));
    put(fam, kC2, T(0.25) * ubv * (-U * B2 * rG));
  };
  auto p = [&](int a, int b, int d) { return P[A_(a, b, d)]; };
  {  // x face: cross directions y (V) and z (W)
    const int64_t R = A_(ip, j, k);
    face(0, utb[q], cu[q], T(0.5) * (G[q] + G[R]), p(i, j, k), p(ip, j, k),
         p(ip, jp, k) + p(i, jp, k), p(ip, jm, k) + p(i, jm, k),
         p(ip, j, kp) + p(i, j, kp), p(ip, j, km) + p(i, j, km),
         cv[q] + cv[R] + cv[A_(i, jm, k)] + cv[A_(ip, jm, k)],
         wfv(i, j, k) + wfv(ip, j, k) + wfv(i, j, k - 1) + wfv(ip, j, k - 1), &ub[q]);
  }
  {  // y face: cross directions x (U) and z (W)
    const int64_t R = A_(i, jp, k);
    face(1, vtb[q], cv[q], T(0.5) * (G[q] + G[R]), p(i, j, k), p(i, jp, k),
         p(ip, jp, k) + p(ip, j, k), p(im, jp, k) + p(im, j, k),
         p(i, jp, kp) + p(i, j, kp), p(i, jp, km) + p(i, j, km),
         cu[q] + cu[R] + cu[A_(im, j, k)] + cu[A_(im, jp, k)],
         wfv(i, j, k) + wfv(i, jp, k) + wfv(i, j, k - 1) + wfv(i, jp, k - 1), &vb[q]);
  }
  if (k < g.nz - 1) {  // z face: cross directions x (U) and y (V)
    const int64_t R = q + g.pxy;
    face(2, wtb[q], cw[q], T(0.5) * (G[q] + G[R]), p(i, j, k), p(i, j, k + 1),
         p(ip, j, k + 1) + p(ip, j, k), p(im, j, k + 1) + p(im, j, k),
         p(i, jp, k + 1) + p(i, jp, k), p(i, jm, k + 1) + p(i, jm, k),
         cu[q] + cu[R] + cu[A_(im, j, k)] + cu[A_(im, j, k + 1)],
         cv[q] + cv[R] + cv[A_(i, jm, k)] + cv[A_(i, jm, k + 1)], &wb[q]);
  } else {
    for (int w = 0; w < kNW; ++w) put(2, w, T(0));
  }
}

template <class T>
__global__ void rev_pg_kernel(Geo g, const T* __restrict__ wts, T* Pb, T* ub, T* vb, T* wb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int i = c.i, j = c.j, k = c.k, nz = g.nz;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int64_t F = g.total;
  auto W = [&](int fam, int w, int a, int b, int d) -> T {
    return wts[((int64_t)fam * kNW + w) * F + at(g, a, b, d)];
  };
  T s = T(0);
  // x faces: A, B1 (y), B2 (z, clamped)
  s += W(0, kWL, i, j, k) + W(0, kWR, im, j, k);
  s += W(0, kW1P, i, jm, k) + W(0, kW1P, im, jm, k) + W(0, kW1M, i, jp, k) + W(0, kW1M, im, jp, k);
  // y faces: A, B1 (x), B2 (z, clamped)
  s += W(1, kWL, i, j, k) + W(1, kWR, i, jm, k);
  s += W(1, kW1P, im, j, k) + W(1, kW1P, im, jm, k) + W(1, kW1M, ip, j, k) + W(1, kW1M, ip, jm, k);
  // clamped z neighbours of the x and y faces: q is the "+z" point of the
  // faces at level kf with clamp(kf+1) == k, the "-z" point where clamp(kf-1) == k
  auto zgather = [&](int kf, int w) {
    s += W(0, w, i, j, kf) + W(0, w, im, j, kf) + W(1, w, i, j, kf) + W(1, w, i, jm, kf);
  };
  if (k >= 1) zgather(k - 1, kW2P);
  if (k == nz - 1) zgather(k, kW2P);
  if (k + 1 <= nz - 1) zgather(k + 1, kW2M);
  if (k == 0) zgather(k, kW2M);
  // z faces (levels kf in [0, nz-2]; the top level holds zeros)
  s += W(2, kWL, i, j, k);
  if (k >= 1) s += W(2, kWR, i, j, k - 1);
  s += W(2, kW1P, im, j, k) + W(2, kW1M, ip, j, k) + W(2, kW2P, i, jm, k) + W(2, kW2M, i, jp, k);
  if (k >= 1)
    s += W(2, kW1P, im, j, k - 1) + W(2, kW1M, ip, j, k - 1) + W(2, kW2P, i, jm, k - 1) +
         W(2, kW2M, i, jp, k - 1);
  const int64_t q = at(g, i, j, k);
  Pb[q] += s;
  // cross averages: U (face i+1/2) in y faces and z faces, V in x and z, W in x and y
  T su = W(1, kC1, i, j, k) + W(1, kC1, i, jm, k) + W(1, kC1, ip, j, k) + W(1, kC1, ip, jm, k);
  su += W(2, kC1, i, j, k) + W(2, kC1, ip, j, k);
  if (k >= 1) su += W(2, kC1, i, j, k - 1) + W(2, kC1, ip, j, k - 1);
  ub[q] += su;
  T sv = W(0, kC1, i, j, k) + W(0, kC1, im, j, k) + W(0, kC1, i, jp, k) + W(0, kC1, im, jp, k);
  sv += W(2, kC2, i, j, k) + W(2, kC2, i, jp, k);
  if (k >= 1) sv += W(2, kC2, i, j, k - 1) + W(2, kC2, i, jp, k - 1);
  vb[q] += sv;
  if (k <= nz - 2) {  // open vertical face
    T sw = W(0, kC2, i, j, k) + W(0, kC2, im, j, k) + W(0, kC2, i, j, k + 1) + W(0, kC2, im, j, k + 1);
    sw += W(1, kC2, i, j, k) + W(1, kC2, i, jm, k) + W(1, kC2, i, j, k + 1) + W(1, kC2, i, jm, k + 1);
    wb[q] += sw;
  }
}

}  // namespace adj
}  // namespace mpd
