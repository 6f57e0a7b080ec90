// adjoint.cuh -- reverse mode of one MPDATA step (iord 1 or 2, with or
// without the limiter) on the GPU.
//
// The forward intermediates of the step (psi1, the pseudo-velocities, the
// betas and the limited velocities) are recomputed by the staged forward
// kernels from the checkpointed psi^n; the kernels here then run the forward
// stages backwards, one thread per interior cell: each thread takes the
// adjoint of what its cell computed (its update, its "+" face quantities,
// its betas) and adds the contributions to every value that computation
// read, with atomic adds (the neighbours it reads are read by other cells
// too).  Periodic and clamped neighbours are addressed by wrapped indices,
// so the reverse of the halo fill is implicit.
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

// Reverse of one face's pseudo-velocity.  L, R: the two cells; l1p/r1p and
// l1m/r1m: the cells one step up/down the first cross direction (next to L
// and R), the same for the second; k1*: the cross Courant field of the first
// cross direction at the four faces of its average, k2* of the second
// (a negative index marks a closed vertical face, which is constant).
template <class T>
__device__ __forceinline__ void rev_face(T ub, const T* P, int64_t L, int64_t R, int64_t l1p,
                                         int64_t r1p, int64_t l1m, int64_t r1m, int64_t l2p,
                                         int64_t r2p, int64_t l2m, int64_t r2m, T U, T Gf,
                                         const T* c1, const int64_t* k1, const T* c2,
                                         const int64_t* k2, T* Pb, T* Ub, T* c1b, T* c2b) {
  const T eps = Eps<T>::v;
  const T rd = rcp(P[R] + P[L] + eps);
  const T A = (P[R] - P[L]) * rd;
  const T n1 = T(0.5) * (P[r1p] + P[l1p] - P[r1m] - P[l1m]);
  const T rd1 = rcp(P[r1p] + P[l1p] + P[r1m] + P[l1m] + eps);
  const T B1 = n1 * rd1;
  const T n2 = T(0.5) * (P[r2p] + P[l2p] - P[r2m] - P[l2m]);
  const T rd2 = rcp(P[r2p] + P[l2p] + P[r2m] + P[l2m] + eps);
  const T B2 = n2 * rd2;
  T C1 = T(0), C2 = T(0);
  for (int q = 0; q < 4; ++q) {
    if (k1[q] >= 0) C1 += c1[k1[q]];
    if (k2[q] >= 0) C2 += c2[k2[q]];
  }
  C1 *= T(0.25);
  C2 *= T(0.25);
  const T rG = rcp(Gf);
  const T Dd = absv(U) - U * U * rG;
  const T X = C1 * B1 + C2 * B2;
  const T sg = (ge0(U) && le0(U)) ? T(0) : (nonneg(U) ? T(1) : T(-1));  // sign(0) = 0
  aadd(Ub, ub * (sg * A - T(2) * U * rG * A - X * rG));
  const T Ab = ub * Dd;
  const T B1b = ub * (-U * C1 * rG), B2b = ub * (-U * C2 * rG);
  const T C1b = T(0.25) * ub * (-U * B1 * rG), C2b = T(0.25) * ub * (-U * B2 * rG);
  aadd(&Pb[R], Ab * (T(1) - A) * rd);
  aadd(&Pb[L], Ab * (T(-1) - A) * rd);
  T wp = B1b * (T(0.5) - B1) * rd1, wm = B1b * (T(-0.5) - B1) * rd1;
  aadd(&Pb[r1p], wp); aadd(&Pb[l1p], wp); aadd(&Pb[r1m], wm); aadd(&Pb[l1m], wm);
  wp = B2b * (T(0.5) - B2) * rd2;
  wm = B2b * (T(-0.5) - B2) * rd2;
  aadd(&Pb[r2p], wp); aadd(&Pb[l2p], wp); aadd(&Pb[r2m], wm); aadd(&Pb[l2m], wm);
  for (int q = 0; q < 4; ++q) {
    if (k1[q] >= 0) aadd(&c1b[k1[q]], C1b);
    if (k2[q] >= 0) aadd(&c2b[k2[q]], C2b);
  }
}

template <class T>
__global__ void rev_pseudo_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
                                  const T* __restrict__ cv, const T* __restrict__ cw,
                                  const T* __restrict__ G, const T* __restrict__ utb,
                                  const T* __restrict__ vtb, const T* __restrict__ wtb, T* Pb,
                                  T* ub, T* vb, T* wb) {
  Cell c = cell_of(g);
  if (!c.ok) return;
  const int i = c.i, j = c.j, k = c.k;
  const int ip = wrap_up(i, g.nx), im = wrap_dn(i, g.nx);
  const int jp = wrap_up(j, g.ny), jm = wrap_dn(j, g.ny);
  const int kp = clampk(k + 1, g.nz), km = clampk(k - 1, g.nz);
  auto A_ = [&](int a, int b, int d) { return at(g, a, b, d); };
  // a vertical face index, or -1 when the face is closed
  auto wf = [&](int a, int b, int d) -> int64_t {
    return (d < 0 || d >= g.nz - 1) ? -1 : at(g, a, b, d);
  };
  const int64_t q = A_(i, j, k);
  {  // x face (i+1/2): cross directions y (V) and z (W)
    const int64_t R = A_(ip, j, k);
    const int64_t k1[4] = {q, R, A_(i, jm, k), A_(ip, jm, k)};
    const int64_t k2[4] = {wf(i, j, k), wf(ip, j, k), wf(i, j, k - 1), wf(ip, j, k - 1)};
    rev_face(utb[q], P, q, R, A_(i, jp, k), A_(ip, jp, k), A_(i, jm, k), A_(ip, jm, k),
             A_(i, j, kp), A_(ip, j, kp), A_(i, j, km), A_(ip, j, km), cu[q],
             T(0.5) * (G[q] + G[R]), cv, k1, cw, k2, Pb, &ub[q], vb, wb);
  }
  {  // y face (j+1/2): cross directions x (U) and z (W)
    const int64_t R = A_(i, jp, k);
    const int64_t k1[4] = {q, R, A_(im, j, k), A_(im, jp, k)};
    const int64_t k2[4] = {wf(i, j, k), wf(i, jp, k), wf(i, j, k - 1), wf(i, jp, k - 1)};
    rev_face(vtb[q], P, q, R, A_(ip, j, k), A_(ip, jp, k), A_(im, j, k), A_(im, jp, k),
             A_(i, j, kp), A_(i, jp, kp), A_(i, j, km), A_(i, jp, km), cv[q],
             T(0.5) * (G[q] + G[R]), cu, k1, cw, k2, Pb, &vb[q], ub, wb);
  }
  if (k < g.nz - 1) {  // z face (k+1/2): cross directions x (U) and y (V)
    const int64_t R = q + g.pxy;
    const int64_t k1[4] = {q, R, A_(im, j, k), A_(im, j, k + 1)};
    const int64_t k2[4] = {q, R, A_(i, jm, k), A_(i, jm, k + 1)};
    rev_face(wtb[q], P, q, R, A_(ip, j, k), A_(ip, j, k + 1), A_(im, j, k), A_(im, j, k + 1),
             A_(i, jp, k), A_(i, jp, k + 1), A_(i, jm, k), A_(i, jm, k + 1), cw[q],
             T(0.5) * (G[q] + G[R]), cu, k1, cv, k2, Pb, &wb[q], ub, vb);
  }
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

}  // namespace adj
}  // namespace mpd
