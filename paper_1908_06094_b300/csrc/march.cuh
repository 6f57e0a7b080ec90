// march.cuh -- the antidiffusive pseudo-velocity faces, the corrective-pass
// stage of the MPDATA sequence of Listing 8 (velocity formula of
// Smolarkiewicz 1984, G-weighted as in Smolarkiewicz & Margolin 1998),
// organised for the B300's FP64 pipe: a k-marching tile kernel that hands
// every face's ingredients to an operation (the forward velocity here, the
// reverse-mode weights in adjoint.cuh).
//
// The B300 issues FP64 arithmetic at 2 lanes per SM per clock, so this
// stage, the costliest of the step, is bound by its count of FP64
// instructions, not by memory.  Two changes against the cell-parallel form
// (one thread computes the three faces of its cell from scratch, about 140
// FP64 instructions per cell) bring the FP64 forward to about 86:
//
//  1. Each face needs four ratios -- A, two B's and 1/G_face -- and the four
//     divisions (a reciprocal seed plus a refinement each) dominate.  They
//     are put over one common denominator:
//        Ut = [4(|U| Gs - 2U^2) N_A D_1 D_2 - U D_A (S1 N_1 D_2 + S2 N_2 D_1)]
//             / (4 Gs D_A D_1 D_2)
//     with Gs = G_L + G_R, N_A/D_A = A, N_1/D_1 = 2B_1, N_2/D_2 = 2B_2 and
//     S1, S2 the sums of the four cross-direction Courant numbers; in exact
//     arithmetic this is the same rational function as the per-ratio form.
//     U is then factored out of the numerator, |U| Gs - 2U^2 being
//     U (sgn(U) Gs - 2U) with the sign moved onto Gs as a bit: 17 FP64
//     instructions a face.
//     The denominators are >= epsilon for non-negative psi, so the product
//     stays in the normal range (it would overflow only for |psi| ~ 1e90).
//  2. Every psi pair sum S (psi_L + psi_R across a face) is used by five
//     faces (as D_A of its own face and as one of the four B sums of the
//     faces beside it), and every pair of Courant numbers by two.  A CTA
//     owns a TX x TY column tile and marches k: each thread forms the pair
//     sums of its own cell once per plane, keeps the ones its own faces need
//     at k-1, k, k+1 in registers, and publishes the ones its neighbours
//     need (i +- 1, j +- 1) in shared memory; a few warps fill the one-cell
//     ring around the tile.  Threads past a ragged domain edge take the
//     periodic image of their cell, so they supply exactly the ring values
//     the edge cells need.
//
// The corrective-pass options ride on the same march: |psi| is read in
// place of psi (signed fields), the infinite gauge is its own face
// operation (one reciprocal, no ratios), and the divergent-flow term adds
// -2 U dsum D_A D_1 D_2 to the common numerator, dsum = D_L + D_R formed
// from the Courant numbers two faces apart and the differences of the
// cross-direction pair sums the march already holds.
#pragma once
#include "grid.cuh"

namespace mpd {
namespace march {

constexpr int TX = 32, TY = 8, KC = 8;

// 4x exactly, by raising the exponent: x is a sum of two metric factors G,
// positive and normal, far from the top of the range.
__device__ __forceinline__ double times4(double x) {
  return __hiloint2double(__double2hiint(x) + (2 << 20), __double2loint(x));
}
__device__ __forceinline__ float times4(float x) { return x * 4.0f; }

// |x| with the sign of s (x >= 0): a sign-bit move on the high words.
__device__ __forceinline__ double sign_of(double x, double s) {
  return __hiloint2double(__double2hiint(x) | (__double2hiint(s) & (int)0x80000000),
                          __double2loint(x));
}

// The ingredients of one face: U its Courant number, gsum = G_L + G_R,
// pl, pr psi1 left and right, DA = S_own + eps, N1 = S(+1) - S(-1) and
// D1 = S(+1) + S(-1) + eps in the first cross direction, N2, D2 in the
// second, s1, s2 the sums of the four cross-direction Courant numbers
// (first, second).  N1/D1 = 2 B1 and N2/D2 = 2 B2.  dsum (the divergent-
// flow option only, else 0): D_L + D_R, the Courant-number divergences of
// the face's two cells.
template <class T>
struct FaceIn {
  T U, gsum, pl, pr, DA, N1, D1, N2, D2, s1, s2, dsum;
};

// Where the calling thread's cell sits: shared-memory row r = ty+1 and
// column c = tx+1 of the tile-plus-ring planes, its level k.
struct CellAt {
  int r, c, k;
  bool own;   // an interior cell (false: the periodic image past a ragged edge)
  bool kper;  // the grid is periodic in k
};

// Ops without shared accumulators.
struct NoAcc {};

// Forward, FP64: the common-denominator form (see the header comment),
//   Ut = U [4 (sgn(U) Gs - 2U) N_A D_1 D_2 - D_A (S1 N_1 D_2 + S2 N_2 D_1)]
//        / (4 Gs D_A D_1 D_2).
// DFL: with the divergent-flow term -(1/2) U dsum / Gs, which over the
// common denominator adds -2 dsum D_A D_1 D_2 to the bracket.
// FLUX: it also stores each face's donor flux of Ut, F(psi_L, psi_R, Ut)
// (psi signed: not with the signed-field option), in fx, fy, fz: the flux
// the limiter's in/out sums and limited fluxes are formed from.
template <bool DFL = false, bool FLUX = false>
struct PseudoMergedT {
  using Acc = NoAcc;
  struct Load {};
  static constexpr bool kAccum = false;
  __device__ __forceinline__ Load load(int64_t) const { return {}; }
  double *ut, *vt, *wt;
  double *fx = nullptr, *fy = nullptr, *fz = nullptr;
  __device__ __forceinline__ void face(int fam, int64_t q, const FaceIn<double>& f) const {
    const double g4 = times4(f.gsum);
    const double NA = f.pr - f.pl;
    const double t1 = fma(f.U, -8.0, sign_of(g4, f.U));  // 4 (sgn(U) Gs - 2U)
    const double D12 = f.D1 * f.D2;
    const double inner = fma(f.s1 * f.N1, f.D2, (f.s2 * f.N2) * f.D1);
    double num = fma(-f.DA, inner, D12 * (t1 * NA));
    const double dad = f.DA * D12;
    if constexpr (DFL) num = fma(-2.0 * f.dsum, dad, num);
    const double Ut = (f.U * num) * rcp(g4 * dad);
    (fam == 0 ? ut : fam == 1 ? vt : wt)[q] = Ut;
    if constexpr (FLUX) (fam == 0 ? fx : fam == 1 ? fy : fz)[q] = donor(f.pl, f.pr, Ut);
  }
  __device__ __forceinline__ void cell(int64_t q, const FaceIn<double>& x,
                                      const FaceIn<double>& y, const FaceIn<double>& z,
                                      bool top, CellAt, Load, Acc&) const {
    face(0, q, x);
    face(1, q, y);
    if (top) {
      wt[q] = 0.0;
      if constexpr (FLUX) fz[q] = 0.0;
    } else {
      face(2, q, z);
    }
  }
};
using PseudoMerged = PseudoMergedT<false>;

// Forward, FP64, infinite gauge: the limit of c times the pseudo-velocity
// of psi + c, whose ratios are cA -> (pr - pl)/2 and cB -> N/8:
//   Ft = (|U| - U^2/Gf)(pr - pl)/2 - U (s1 N1 + s2 N2) / (32 Gf),
// one reciprocal of Gs per face.
struct PseudoIGA {
  using Acc = NoAcc;
  struct Load {};
  static constexpr bool kAccum = false;
  __device__ __forceinline__ Load load(int64_t) const { return {}; }
  double *ut, *vt, *wt;
  __device__ __forceinline__ void face(int fam, int64_t q, const FaceIn<double>& f) const {
    const double q2 = 2.0 * f.U * rcp(f.gsum);                   // U / Gf
    const double diff = fabs(f.U) - f.U * q2;                     // |U| - U^2/Gf
    const double cross = 0.03125 * fma(f.s1, f.N1, f.s2 * f.N2);  // (s1 N1 + s2 N2)/32
    (fam == 0 ? ut : fam == 1 ? vt : wt)[q] = fma(diff, 0.5 * (f.pr - f.pl), -q2 * cross);
  }
  __device__ __forceinline__ void cell(int64_t q, const FaceIn<double>& fx,
                                      const FaceIn<double>& fy, const FaceIn<double>& fz,
                                      bool top, CellAt, Load, Acc&) const {
    face(0, q, fx);
    face(1, q, fy);
    if (top) wt[q] = 0.0;
    else face(2, q, fz);
  }
};

// One plane of published sums; row index r+1 holds tile row r (r = -1 ..
// TY), column index c+1 tile column c (c = -1 .. TX).
template <class T>
struct Plane {
  T sx[TY + 2][TX], ex[TY + 2][TX];          // S_x = psi(i) + psi(i+1), S_x + eps
  T sy[TY][TX + 2], ey[TY][TX + 2];          // S_y = psi(j) + psi(j+1), S_y + eps
  T sz[TY + 2][TX + 2], ez[TY + 2][TX + 2];  // S_z = psi(k) + psi(k+1), + eps
  T pvx[TY + 1][TX], pvz[TY + 1][TX];        // V(i)+V(i+1); V(k)+V(k+1)  rows -1 .. TY-1
  T puy[TY][TX + 1], puz[TY][TX + 1];        // U(j)+U(j+1); U(k)+U(k+1)  cols -1 .. TX-1
};

// CTAs per SM the registers are sized for.  (Loading each level one level
// ahead, which costs ~20 registers, was measured slower for the FP32
// reverse than the third CTA per SM it displaces: 178 vs 161 µs.)
template <class T, class Op> struct MarchMinB { static constexpr int v = 2; };
template <class Op> struct MarchMinB<float, Op> { static constexpr int v = 3; };

// Grid: (ceil(nx/TX), ceil(ny/TY), ceil(nz/kc)); block (TX, TY).  Calls
// op.cell(q, x, y, z, top, at, l, acc) with the ingredients of the x, y and
// z "+" faces of every interior cell q of its tile and k range, l = op.load(q)
// the op's own reads for the cell (top: the z
// face is the closed top face and its ingredients are meaningless).  An op
// with kAccum also owns shared accumulators (Op::Acc); it is called for
// every thread of the tile (at.own false past a ragged edge), and after the
// cells of level k and a barrier op.flush(acc, k, false, ...) writes out
// the accumulator levels no later cell of the CTA touches, after the last
// level op.flush(acc, k1-1, true, ...) the rest.
// OPT (kOpt* bits, forward ops only): ABS reads |psi| wherever psi enters
// (A and B of |psi|); DFL hands each face its dsum.
template <class T, class Op, int OPT = 0>
__global__ void __launch_bounds__(TX * TY, MarchMinB<T, Op>::v)
march_kernel(Geo g, const T* __restrict__ P, const T* __restrict__ cu,
             const T* __restrict__ cv, const T* __restrict__ cw, const T* __restrict__ G, Op op,
             int kc) {
  pdl_enter();
  constexpr bool kABS = (OPT & kOptABS) != 0, kDFL = (OPT & kOptDFL) != 0;
  auto lp = [&](int64_t a) { return kABS ? absv(P[a]) : P[a]; };
  // op is a per-thread copy: accumulating ops keep their flush positions in it
  // accumulating ops order the plane's reuse by their own barrier: one copy
  __shared__ Plane<T> sm[Op::kAccum ? 1 : 2];
  __shared__ typename Op::Acc acc;
  const T eps = Eps<T>::v, zero = T(0);
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const bool own = i0 + tx < g.nx && j0 + ty < g.ny;
  const int i = (i0 + tx) % g.nx, j = (j0 + ty) % g.ny;
  const int64_t o = at(g, i, j, 0), oi = at(g, wrap_up(i, g.nx), j, 0);
  const int64_t oj = at(g, i, wrap_up(j, g.ny), 0);
  // DFL: the cells at i-1 and j-1 (their Courant numbers close the
  // divergences of the faces' two cells)
  const int64_t oim = at(g, wrap_dn(i, g.nx), j, 0), ojm = at(g, i, wrap_dn(j, g.ny), 0);

  // ring task: rows j0-1 and j0+TY (threads 0 .. 2TX-1), columns i0-1 and
  // i0+TX (the next 2TY threads)
  int rkind = 0, rs = 0, rc = 0;
  int64_t ro = 0, rn = 0;
  if (t < 2 * TX) {
    rkind = 1;
    rc = t % TX;
    const bool up = t >= TX;
    const int ri = (i0 + rc) % g.nx;
    const int rj = up ? (j0 + TY) % g.ny : (j0 + g.ny - 1) % g.ny;
    rs = up ? TY + 1 : 0;
    ro = at(g, ri, rj, 0);
    rn = at(g, wrap_up(ri, g.nx), rj, 0);
  } else if (t < 2 * TX + 2 * TY) {
    rkind = 2;
    rs = (t - 2 * TX) % TY;
    const bool up = t >= 2 * TX + TY;
    const int rj = (j0 + rs) % g.ny;
    const int ri = up ? (i0 + TX) % g.nx : (i0 + g.nx - 1) % g.nx;
    rc = up ? TX + 1 : 0;
    ro = at(g, ri, rj, 0);
    rn = at(g, ri, wrap_up(rj, g.ny), 0);
  }

  const int64_t pxy = g.pxy;
  const int k0 = blockIdx.z * kc, k1 = min(k0 + kc, g.nz);
  if constexpr (Op::kAccum) {
    op.zero(acc, t);  // ordered by the first barrier
    op.setup(g, i0, j0, t);
  }
  // register queues: psi and pair sums at k (and k-1), W pairs at k-1/2
  T pc = lp(o + k0 * pxy), pi = lp(oi + k0 * pxy), pj = lp(oj + k0 * pxy);
  T sx = pc + pi, exx = sx + eps, sy = pc + pj, eyy = sy + eps;
  const int64_t ob = (int64_t)kadj(g, k0 - 1) * pxy;  // the level below the chunk
  T sxm = lp(o + ob) + lp(oi + ob), sym = lp(o + ob) + lp(oj + ob);
  T pwxm = zero, pwym = zero, wm = zero;  // wm: own W at the face below (DFL)
  if (zopen(g, k0 - 1)) {  // the face below the chunk
    pwxm = cw[o + ob] + cw[oi + ob];
    pwym = cw[o + ob] + cw[oj + ob];
    wm = cw[o + ob];
  }
  // Everything level k reads from memory (n: level k+1, clamped).
  struct In {
    T pcn, pin, pjn, uc, vc, wc, cvi, cuj, cwi, cwj, cun, cvn, gc, gi, gj, gn;
    T ra, rb, rcn, rv0, rv1, rvn;  // ring task: psi at k (two points), k+1; Courant
    T ui, uim, vj, vjm, wn;        // DFL: U at i+-1, V at j+-1, own W one face up
    typename Op::Load ol;
  };
  const T* rvel = rkind == 1 ? cv : cu;
  auto load = [&](int k) {
    const int64_t ok = k * pxy, on = (int64_t)kadj(g, k + 1) * pxy;
    In v;
    v.pcn = lp(o + on); v.pin = lp(oi + on); v.pjn = lp(oj + on);
    v.uc = cu[o + ok]; v.vc = cv[o + ok]; v.wc = cw[o + ok];
    v.cvi = cv[oi + ok]; v.cuj = cu[oj + ok]; v.cwi = cw[oi + ok]; v.cwj = cw[oj + ok];
    v.cun = cu[o + on]; v.cvn = cv[o + on];
    v.gc = G[o + ok]; v.gi = G[oi + ok]; v.gj = G[oj + ok]; v.gn = G[o + on];
    if (rkind) {
      v.ra = lp(ro + ok); v.rb = lp(rn + ok); v.rcn = lp(ro + on);
      v.rv0 = rvel[ro + ok]; v.rv1 = rvel[rn + ok]; v.rvn = rvel[ro + on];
    }
    if constexpr (kDFL) {
      v.ui = cu[oi + ok]; v.uim = cu[oim + ok];
      v.vj = cv[oj + ok]; v.vjm = cv[ojm + ok];
      v.wn = zopen(g, k + 1) ? cw[o + on] : zero;  // the face above level k+1
    } else {
      v.ui = v.uim = v.vj = v.vjm = v.wn = zero;
    }
    v.ol = op.load(o + ok);
    return v;
  };
  for (int k = k0; k < k1; ++k) {
    const int64_t ok = k * pxy;
    const bool top = !zopen(g, k);  // the face above k is closed (zero-flux top)
    const In in = load(k);
    const T pcn = in.pcn, pin = in.pin, pjn = in.pjn;
    const T sxn = pcn + pin, exn = sxn + eps, syn = pcn + pjn, eyn = syn + eps;
    const T uc = in.uc, vc = in.vc, wc = in.wc;
    const T pvx = vc + in.cvi, puy = uc + in.cuj;
    T sz = zero, ez = zero, puz = zero, pvz = zero, pwx = zero, pwy = zero;
    if (!top) {  // the face k+1/2 is open
      sz = pc + pcn;
      ez = sz + eps;
      puz = uc + in.cun;
      pvz = vc + in.cvn;
      pwx = wc + in.cwi;
      pwy = wc + in.cwj;
    }
    Plane<T>& s = sm[Op::kAccum ? 0 : (k & 1)];
    s.sx[ty + 1][tx] = sx;
    s.ex[ty + 1][tx] = exx;
    s.sy[ty][tx + 1] = sy;
    s.ey[ty][tx + 1] = eyy;
    s.sz[ty + 1][tx + 1] = sz;
    s.ez[ty + 1][tx + 1] = ez;
    s.pvx[ty + 1][tx] = pvx;
    s.pvz[ty + 1][tx] = pvz;
    s.puy[ty][tx + 1] = puy;
    s.puz[ty][tx + 1] = puz;
    if (rkind == 1) {  // row ring: S_x, S_z (+eps above), V pairs below
      const T rsx = in.ra + in.rb;
      const T rsz = top ? zero : in.ra + in.rcn;
      s.sx[rs][rc] = rsx;
      s.sz[rs][rc + 1] = rsz;
      if (rs == 0) {
        s.pvx[0][rc] = in.rv0 + in.rv1;
        s.pvz[0][rc] = top ? zero : in.rv0 + in.rvn;
      } else {
        s.ex[rs][rc] = rsx + eps;
        s.ez[rs][rc + 1] = rsz + eps;
      }
    } else if (rkind == 2) {  // column ring: S_y, S_z (+eps right), U pairs left
      const T rsy = in.ra + in.rb;
      const T rsz = top ? zero : in.ra + in.rcn;
      s.sy[rs][rc] = rsy;
      s.sz[rs + 1][rc] = rsz;
      if (rc == 0) {
        s.puy[rs][0] = in.rv0 + in.rv1;
        s.puz[rs][0] = top ? zero : in.rv0 + in.rvn;
      } else {
        s.ey[rs][rc] = rsy + eps;
        s.ez[rs + 1][rc] = rsz + eps;
      }
    }
    __syncthreads();
    if (own || Op::kAccum) {  // accumulating ops run whole warps (zero weights past the edge)
      const int64_t q = o + ok;
      // DFL: D_L + D_R per face: the own-direction Courant numbers two faces
      // apart, and the cross directions' pair sums differenced (the closed
      // faces' W are zero)
      T dx = zero, dy = zero, dz = zero;
      if constexpr (kDFL) {
        const T wo = top ? zero : wc;  // own W at face k+1/2
        dx = (in.ui - in.uim) + (s.pvx[ty + 1][tx] - s.pvx[ty][tx]) + (pwx - pwxm);
        dy = (in.vj - in.vjm) + (s.puy[ty][tx + 1] - s.puy[ty][tx]) + (pwy - pwym);
        dz = (in.wn - wm) + (s.puz[ty][tx + 1] - s.puz[ty][tx]) +
             (s.pvz[ty + 1][tx] - s.pvz[ty][tx]);
        wm = wo;
      }
      op.cell(q,
              FaceIn<T>{uc, in.gc + in.gi, pc, pi, exx, s.sx[ty + 2][tx] - s.sx[ty][tx],
                        s.ex[ty + 2][tx] + s.sx[ty][tx], sxn - sxm, exn + sxm,
                        s.pvx[ty + 1][tx] + s.pvx[ty][tx], pwx + pwxm, dx},
              FaceIn<T>{vc, in.gc + in.gj, pc, pj, eyy, s.sy[ty][tx + 2] - s.sy[ty][tx],
                        s.ey[ty][tx + 2] + s.sy[ty][tx], syn - sym, eyn + sym,
                        s.puy[ty][tx + 1] + s.puy[ty][tx], pwy + pwym, dy},
              FaceIn<T>{wc, in.gc + in.gn, pc, pcn, ez,
                        s.sz[ty + 1][tx + 2] - s.sz[ty + 1][tx],
                        s.ez[ty + 1][tx + 2] + s.sz[ty + 1][tx],
                        s.sz[ty + 2][tx + 1] - s.sz[ty][tx + 1],
                        s.ez[ty + 2][tx + 1] + s.sz[ty][tx + 1],
                        s.puz[ty][tx + 1] + s.puz[ty][tx], s.pvz[ty + 1][tx] + s.pvz[ty][tx],
                        dz},
              top, CellAt{ty + 1, tx + 1, k, own, g.kper != 0}, in.ol, acc);
    } else if constexpr (kDFL) {
      wm = top ? zero : in.wc;
    }
    if constexpr (Op::kAccum) {
      __syncthreads();
      op.flush(acc, k, false, g, i0, j0, k0, k1, t);
    }
    sxm = sx; sx = sxn; exx = exn;
    sym = sy; sy = syn; eyy = eyn;
    pwxm = pwx; pwym = pwy;
    pc = pcn; pi = pin; pj = pjn;
  }
  if constexpr (Op::kAccum) op.flush(acc, k1 - 1, true, g, i0, j0, k0, k1, t);
}

// Launch geometry of march_kernel.
inline dim3 march_grid(const Geo& g, int kc = KC) {
  return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + kc - 1) / kc);
}

}  // namespace march
}  // namespace mpd
