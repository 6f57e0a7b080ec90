// fusedx.cuh -- the one-kernel FP32 MPDATA step (iord = 2) with two
// adjacent columns per thread and Blackwell's packed FP32 arithmetic.
//
// The stages, their planes, the shared rings and the two barriers a level
// are those of the one-column kernel (fused2.cuh): per level t, A psi1 on
// plane t+2, B pseudo-velocities and C limiter bounds and betas on plane
// t+1, D limited face fluxes on plane t, E advance on plane t-1.  What
// changes is the unit of work: a thread owns the columns x and x+1 (x even)
// and carries each value of its two columns as one float2, whose additions,
// subtractions, products and fused multiply-adds are single f32x2
// instructions (add/sub/mul/fma.rn.f32x2).  Reciprocals, min/max and
// sign selects stay per lane.  So the stage guards, plane-slot and address
// arithmetic, loop control and queue shifts serve two columns, the
// arithmetic takes one instruction for two, and the shared and global
// loads of a row pair are 8-byte loads.
//
// Every operation of a lane is the explicitly rounded operation the
// one-column kernel performs, in the same order, so the two kernels give
// the same bits.  Neighbours one column to the side are (own.y, next) or
// (prev, own.x): one 4-byte shared load completes the shifted pair.
//
// Requirements (checked by the caller): FP32, even nx and halo (so every
// pair starts on an 8-byte boundary in device memory and a periodic wrap
// never separates the two columns), fewer than 2^31 elements a field,
// the i-j domain periodic (not a slab), no corrective-pass options.  Both
// vertical boundaries; with TAPE the step also writes the adjoint's tape.
#pragma once
#include <climits>
#include <type_traits>

#include "grid.cuh"

namespace mpd {
namespace fusedx {

using f2 = float2;

__device__ __forceinline__ f2 mk(float a, float b) { return make_float2(a, b); }

// packed FP32 arithmetic, round to nearest, each lane exactly the scalar op
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
// a * b + c with one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ f2 splat(float a) { return mk(a, a); }
__device__ __forceinline__ f2 rcp2(f2 a) { return mk(rcp(a.x), rcp(a.y)); }
__device__ __forceinline__ f2 pos2(f2 a) { return mk(pos(a.x), pos(a.y)); }
__device__ __forceinline__ f2 neg2(f2 a) { return mk(neg(a.x), neg(a.y)); }
__device__ __forceinline__ f2 abs2(f2 a) { return mk(absv(a.x), absv(a.y)); }

// donor-cell flux of each lane (the scalar donor: C times the upwind value)
__device__ __forceinline__ f2 donor2(f2 L, f2 R, f2 C) {
  return mul2(C, mk(nonneg(C.x) ? L.x : R.x, nonneg(C.y) ? L.y : R.y));
}
// The same with one scalar product a lane, for fluxes that a sum consumes
// directly: the code generator may fuse a packed product into the packed
// add or subtract that consumes it (one rounding instead of two), which the
// one-column kernel's explicitly rounded scalar product never allows.
__device__ __forceinline__ f2 donor2s(f2 L, f2 R, f2 C) {
  return mk(mul_rn(C.x, nonneg(C.x) ? L.x : R.x), mul_rn(C.y, nonneg(C.y) ? L.y : R.y));
}
// limited velocity of each lane (the scalar limit_face)
__device__ __forceinline__ f2 limit2(f2 C, f2 buL, f2 bdL, f2 buR, f2 bdR) {
  return mul2(mk(limit_factor(C.x, buL.x, bdL.x, buR.x, bdR.x),
                 limit_factor(C.y, buL.y, bdL.y, buR.y, bdR.y)),
              C);
}
// pseudo-velocity of each lane: the operations of pseudo_velocity (grid.cuh)
// with the sign carried by -1/Gf, so no lane needs a separate negation:
// U (-q) + |U| is -U q + |U| and (-q) cross is -(q cross), exactly.
__device__ __forceinline__ f2 pseudo2(f2 U, f2 gsum, f2 pl, f2 pr, f2 s1p, f2 s1m, f2 s2p,
                                      f2 s2m, f2 vsum, f2 wsum) {
  const f2 eps = splat(Eps<float>::v);
  const f2 rGn = mul2(splat(-2.0f), rcp2(gsum));                          // -1/Gf
  const f2 A = mul2(sub2(pr, pl), rcp2(add2(add2(pr, pl), eps)));
  const f2 B1 = mul2(sub2(s1p, s1m), rcp2(add2(add2(s1p, s1m), eps)));
  const f2 B2 = mul2(sub2(s2p, s2m), rcp2(add2(add2(s2p, s2m), eps)));
  const f2 qn = mul2(U, rGn);                                             // -U/Gf
  const f2 diff = fma2(U, qn, abs2(U));                                   // |U| - U^2/Gf
  const f2 cross = mul2(splat(0.125f), fma2(vsum, B1, mul2(wsum, B2)));
  return fma2(diff, A, mul2(qn, cross));
}
// the infinite-gauge pseudo-flux of each lane: the operations of
// pseudo_flux_iga (grid.cuh), the sign carried by -1/Gf as in pseudo2
__device__ __forceinline__ f2 pseudo_iga2(f2 U, f2 gsum, f2 pl, f2 pr, f2 s1p, f2 s1m, f2 s2p,
                                          f2 s2m, f2 vsum, f2 wsum) {
  const f2 rGn = mul2(splat(-2.0f), rcp2(gsum));                          // -1/Gf
  const f2 qn = mul2(U, rGn);
  const f2 diff = fma2(U, qn, abs2(U));                                   // |U| - U^2/Gf
  const f2 cross = mul2(splat(0.03125f), fma2(vsum, sub2(s1p, s1m), mul2(wsum, sub2(s2p, s2m))));
  return fma2(diff, mul2(splat(0.5f), sub2(pr, pl)), mul2(qn, cross));
}
// the divergent-flow term of each lane (divergent_flow_term, grid.cuh), its
// last product per lane: a sum consumes it
__device__ __forceinline__ f2 dft2(f2 U, f2 gsum, f2 dsum) {
  const f2 t = mul2(mul2(splat(-0.5f), U), dsum);
  return mk(mul_rn(t.x, rcp(gsum.x)), mul_rn(t.y, rcp(gsum.y)));
}
// the options' forms (free functions, no captures): |psi1| with ABS, the
// face's pseudo-velocity or infinite-gauge pseudo-flux, and the corrective
// flux of a face (the donor flux of its velocity, or in the infinite gauge
// the value itself)
template <bool ABS>
__device__ __forceinline__ f2 ap(f2 v) { return ABS ? abs2(v) : v; }
template <bool IGA>
__device__ __forceinline__ f2 pse(f2 C, f2 gsum, f2 pl, f2 pr, f2 s1p, f2 s1m, f2 s2p, f2 s2m,
                                  f2 c1, f2 c2) {
  if constexpr (IGA) return pseudo_iga2(C, gsum, pl, pr, s1p, s1m, s2p, s2m, c1, c2);
  else return pseudo2(C, gsum, pl, pr, s1p, s1m, s2p, s2m, c1, c2);
}
template <bool IGA>
__device__ __forceinline__ f2 cflux2(f2 L, f2 R, f2 C) {
  if constexpr (IGA) return C;
  else return donor2(L, R, C);
}
// the limiter bounds of each lane over its 14 values, folded in the order
// of the scalar bounds()
template <int N>
__device__ __forceinline__ void bounds2(const f2 (&v)[N], f2& hi, f2& lo) {
  float hx = v[0].x, lx = v[0].x, hy = v[0].y, ly = v[0].y;
#pragma unroll
  for (int q = 1; q < N; ++q) {
    hx = fmaxf(hx, v[q].x);
    lx = fminf(lx, v[q].x);
    hy = fmaxf(hy, v[q].y);
    ly = fminf(ly, v[q].y);
  }
  hi = mk(hx, hy);
  lo = mk(lx, ly);
}

// Shared planes: radius-2 planes (TX+4) x (TY+4) from column -2, radius-3
// planes (TX+8) x (TY+6) from column -4 (one unused column on each side, so
// that every pair starts on an even slot).  The rings and their depths are
// those of the one-column kernel.
template <int TX, int TY>
struct Layout {
  static constexpr int EX = TX + 4, EY = TY + 4, SN = EX * EY;
  static constexpr int RX = TX + 8, RY = TY + 6, RN = RX * RY;
  static constexpr int NRING = (TX + 6) * (TY + 6) - SN;  // radius-3 ring cells
  static constexpr int P0S = 0;             // psi^n, 4 planes, radius 3
  static constexpr int US = P0S + 4 * RN;   // U, 4 planes, radius 3
  static constexpr int VS = US + 4 * RN;    // V, 4 planes, radius 3
  static constexpr int WS = VS + 4 * RN;    // W, 4 faces, radius 2
  static constexpr int GS = WS + 4 * SN;    // G, 4 planes, radius 2
  static constexpr int P1S = GS + 4 * SN;   // psi1, 4 planes
  static constexpr int UTS = P1S + 4 * SN;  // Ut, 1 plane
  static constexpr int VTS = UTS + SN;      // Vt, 1 plane
  static constexpr int BUS = VTS + SN;      // beta-up, 2 planes
  static constexpr int BDS = BUS + 2 * SN;  // beta-down, 2 planes
  static constexpr int FXS = BDS + 2 * SN;  // x-face fluxes, 2 planes
  static constexpr int FYS = FXS + 2 * SN;  // y-face fluxes, 2 planes
  static constexpr int NVAL = FYS + 2 * SN;
  static constexpr size_t bytes = (size_t)NVAL * sizeof(float);
  static_assert(EX % 2 == 0 && RX % 2 == 0 && SN % 2 == 0 && RN % 2 == 0, "pair alignment");
};

// The pair (x, x+1) of thread tid, x even in [-2, TX], y in [-2, TY+1]:
// the tile's pairs first (TX/2 a row), then the pairs at x = -2 and x = TX
// of the tile's rows, rows -1 and TY, row -2 (stage B forms its y faces),
// row TY+1 (stage A only).  NC threads run stages C (rows -1 .. TY), NB
// stage B.
template <int TX, int TY>
struct PairMap {
  static_assert(TX % 2 == 0, "pairs of columns");
  static constexpr int NPX = (TX + 4) / 2;  // pairs a row
  static constexpr int NT = NPX * (TY + 4);
  static constexpr int NTILE = (TX / 2) * TY;
  static constexpr int NC = NPX * (TY + 2);
  static constexpr int NB = NC + NPX;
  static __device__ __forceinline__ void cell(int tid, int& x, int& y) {
    if (tid < NTILE) { x = 2 * (tid % (TX / 2)); y = tid / (TX / 2); return; }
    int r = tid - NTILE;
    if (r < 2 * TY) { x = r < TY ? -2 : TX; y = r < TY ? r : r - TY; return; }
    r -= 2 * TY;
    if (r < NPX) { x = 2 * r - 2; y = -1; return; }
    r -= NPX;
    if (r < NPX) { x = 2 * r - 2; y = TY; return; }
    r -= NPX;
    if (r < NPX) { x = 2 * r - 2; y = -2; return; }
    r -= NPX;
    x = 2 * r - 2;
    y = TY + 1;
  }
};

// TAPE: the step also writes the intermediates of its interior cells (the
// adjoint's tape), each a padded field like psi, tstride elements apart from
// tape (psi1): psi1, Ut, Vt, Wt, beta-up, beta-down at slots 0..5 and the
// limited Ul, Vl, Wl at slots 8..10 (slots 6 and 7 are FP64's reciprocals).
template <int TX, int TY, int MINB, bool LIMIT, bool KPER, bool TAPE = false, int OPT = 0>
__global__ void __launch_bounds__(PairMap<TX, TY>::NT, MINB)
step_kernel_x2(Geo g, int kchunk, const float* __restrict__ P0, const float* __restrict__ U,
               const float* __restrict__ V, const float* __restrict__ W,
               const float* __restrict__ G, float* __restrict__ out,
               float* __restrict__ tape, long long tstride) {
  pdl_enter();
  using L = Layout<TX, TY>;
  using Map = PairMap<TX, TY>;
  constexpr int EX = L::EX, RX = L::RX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x;
  const int nz = g.nz;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  const f2 zero2 = splat(0.0f), eps2 = splat(Eps<float>::v);

  int x, y;
  Map::cell(tid, x, y);
  const int s2 = (y + 2) * EX + (x + 2);  // radius-2 slot of the pair (even)
  const int s3 = (y + 3) * RX + (x + 4);  // radius-3 slot of the pair (even)
  const bool inB = tid < Map::NB, inC = tid < Map::NC;
  // stage D: the faces stage E reads (x faces of columns -1 .. TX-1 on the
  // tile's rows, y faces of the tile's columns on rows -1 .. TY-1)
  const bool inD = tid < Map::NTILE + TY ||
                   (tid >= Map::NTILE + 2 * TY && tid < Map::NTILE + 2 * TY + Map::NPX &&
                    x >= 0 && x < TX);
  // periodic wrap: nx even and x even, so the two columns of a pair are
  // adjacent in device memory wherever the pair falls
  auto wrapi = [&](int i) { return ((i % g.nx) + g.nx) % g.nx; };
  auto wrapj = [&](int j) { return ((j % g.ny) + g.ny) % g.ny; };
  const int col = wrapj(j0 + y) * (int)g.px + wrapi(i0 + x);
  const bool ringer = tid < L::NRING;
  int r3 = 0, rcol = 0;
  if (ringer) {  // the radius-3 ring, one cell a thread
    constexpr int RW = TX + 6;
    int rx, ry, r = tid;
    if (r < RW) { rx = r - 3; ry = -3; }
    else if ((r -= RW) < RW) { rx = r - 3; ry = TY + 2; }
    else if ((r -= RW) < L::EY) { rx = -3; ry = r - 2; }
    else { r -= L::EY; rx = TX + 2; ry = r - 2; }
    r3 = (ry + 3) * RX + (rx + 4);
    rcol = wrapj(j0 + ry) * (int)g.px + wrapi(i0 + rx);
  }
  const int pxy = (int)g.pxy;
  constexpr bool kper = KPER;
  auto clampk_ = [&](int k) {
    return kper ? ((k % nz) + nz) % nz : (k < 0 ? 0 : (k >= nz ? nz - 1 : k));
  };
  const int klo = kper ? INT_MIN / 2 : 0, khi = kper ? INT_MAX / 2 : nz - 1;
  auto zface = [&](int k) { return kper || (k >= 0 && k < nz - 1); };
  const int c0 = (int)g.off0 + col, rc0 = (int)g.off0 + rcol;
  auto ld2 = [&](const float* f, int off) {
    return *reinterpret_cast<const f2*>(f + c0 + off);
  };
  auto ldk = [&](const float* f, int k) { return ld2(f, clampk_(k) * pxy); };
  auto ldw = [&](int k) {
    if constexpr (KPER) return ld2(W, clampk_(k) * pxy);
    else return (k < 0 || k >= nz - 1) ? zero2 : ld2(W, k * pxy);
  };
  auto ldr = [&](const float* f, int k) { return f[rc0 + clampk_(k) * pxy]; };
  float* p0s = sm + L::P0S;
  float* us = sm + L::US;
  float* vs = sm + L::VS;
  float* ws = sm + L::WS;
  float* gs = sm + L::GS;
  float* p1s = sm + L::P1S;
  float* uts = sm + L::UTS;
  float* vts = sm + L::VTS;
  float* fxs = sm + L::FXS;
  float* fys = sm + L::FYS;
  auto at2 = [&](const float* p) { return *reinterpret_cast<const f2*>(p); };
  auto st2 = [&](float* p, f2 v) { *reinterpret_cast<f2*>(p) = v; };
  // psi1 of plane k: the pair's slot, and a scalar at offset o from it
  auto P1v = [&](int k, int o) -> float* { return p1s + (k & 3) * L::SN + s2 + o; };
  // corrective-pass options (kOpt* bits, as in the one-column kernel): ABS
  // forms A and B from |psi1| and trades beta-up and beta-down on a face
  // whose upwind psi1 is negative, IGA uses the infinite-gauge pseudo-fluxes
  // (which are the corrective fluxes), DFL adds the divergent-flow term
  constexpr bool kABS = (OPT & kOptABS) != 0, kIGA = (OPT & kOptIGA) != 0;
  constexpr bool kDFL = (OPT & kOptDFL) != 0;
  static_assert(!TAPE || OPT == 0, "the taped step has no options");
  (void)kDFL;

  // the tile's pairs write psi^(n+1): each lane inside the grid
  const bool inT = x >= 0 && x < TX && y >= 0 && y < TY;
  const int gi = i0 + x, gj = j0 + y;
  const bool wr0 = inT && gi < g.nx && gj < g.ny, wr1 = inT && gi + 1 < g.nx && gj < g.ny;
  const bool noimg = gi >= g.h && gi + 1 < g.nx - g.h && gj >= g.h && gj < g.ny - g.h;
  const bool whole = wr0 && wr1 && noimg;  // both lanes, one 8-byte store

  const int t0 = k0 - 5;
  f2 p0 = ldk(P0, t0), p1 = ldk(P0, t0 + 1), p2 = ldk(P0, t0 + 2), p3 = ldk(P0, t0 + 3);
  f2 pn = ldk(P0, t0 + 4);
  f2 u1 = ldk(U, t0 + 1), u2 = ldk(U, t0 + 2), un = ldk(U, t0 + 3);
  f2 v1 = ldk(V, t0 + 1), v2 = ldk(V, t0 + 2), vn = ldk(V, t0 + 3);
  f2 w0 = ldw(t0), w1 = ldw(t0 + 1), w2 = ldw(t0 + 2), wn = ldw(t0 + 3);
  f2 g1 = ldk(G, t0 + 1), g2 = ldk(G, t0 + 2), gn = ldk(G, t0 + 3);
  float rp = 0.0f, ru = 0.0f, rv = 0.0f;  // ring values of plane t+3
  if (ringer) { rp = ldr(P0, t0 + 3); ru = ldr(U, t0 + 3); rv = ldr(V, t0 + 3); }
  f2 q0 = zero2, q1 = zero2, q2 = zero2;  // psi1 at t, t+1, t+2
  f2 utA = zero2, vtA = zero2, utB = zero2, vtB = zero2;  // Ut, Vt at t, t+1
  f2 wtA = zero2, wtB = zero2;            // Wt at faces t+1/2, t+3/2
  f2 buA = zero2, bdA = zero2, buB = zero2, bdB = zero2;  // betas at t, t+1
  f2 c1z = zero2;  // stage C's last upper z flux
  f2 f1z = zero2;  // the donor flux through face t+3/2 (stage A's last "+" z face)
  f2 fzAA = zero2, fzA = zero2, fzB = zero2;  // vertical fluxes at faces t-3/2 .. t+1/2
  int l4 = clampk_(t0 + 4), l5 = clampk_(t0 + 5);

  // the planes the first level reads (the levels publish one plane ahead)
  {
    const int a = t0 + 2;
    st2(p0s + (a & 3) * L::RN + s3, p2);
    st2(us + (a & 3) * L::RN + s3, u2);
    st2(vs + (a & 3) * L::RN + s3, v2);
    if (ringer) {
      p0s[(a & 3) * L::RN + r3] = ldr(P0, a);
      us[(a & 3) * L::RN + r3] = ldr(U, a);
      vs[(a & 3) * L::RN + r3] = ldr(V, a);
    }
    st2(ws + ((t0 + 1) & 3) * L::SN + s2, w1);
    st2(gs + ((t0 + 1) & 3) * L::SN + s2, g1);
  }
  __syncthreads();
  // One level of the march; STEADY as in the one-column kernel.
  auto level = [&](const int t, auto steady) {
    constexpr bool S = decltype(steady)::value;
    // ---- publish plane t+3 of psi^n, U, V, face t+2 of W, plane t+2 of G --
    {
      const int a = t + 3;
      st2(p0s + (a & 3) * L::RN + s3, p3);
      st2(us + (a & 3) * L::RN + s3, un);
      st2(vs + (a & 3) * L::RN + s3, vn);
      if (ringer) {
        p0s[(a & 3) * L::RN + r3] = rp;
        us[(a & 3) * L::RN + r3] = ru;
        vs[(a & 3) * L::RN + r3] = rv;
      }
      st2(ws + ((t + 2) & 3) * L::SN + s2, w2);
      st2(gs + ((t + 2) & 3) * L::SN + s2, g2);
    }
    // loads one plane ahead
    const int o5 = (KPER ? l5 : (S ? t + 5 : clampk_(t + 5))) * pxy;
    const int o4 = (KPER || !S) ? (KPER ? l4 : clampk_(t + 4)) * pxy : o5 - pxy;
    const f2 pn_next = ld2(P0, o5);
    const f2 un_next = ld2(U, o4), vn_next = ld2(V, o4), gn_next = ld2(G, o4);
    const f2 wn_next = (S || zface(t + 4)) ? ld2(W, o4) : zero2;  // closed faces
    float rp_next = 0.0f, ru_next = 0.0f, rv_next = 0.0f;
    if (ringer) {
      rp_next = P0[rc0 + o4];
      ru_next = U[rc0 + o4];
      rv_next = V[rc0 + o4];
    }
    // ---- A: psi1 on plane a = t+2 ---------------------------------------
    const int a = t + 2;
    if (S || (a >= max(klo, k0 - 3) && a <= min(khi, k1 + 1))) {
      const float* pa = p0s + (a & 3) * L::RN + s3;
      const float* ua = us + (a & 3) * L::RN + s3;
      const float* va = vs + (a & 3) * L::RN + s3;
      const f2 fxp = donor2s(p2, mk(p2.y, pa[2]), u2);
      const f2 fxm = donor2s(mk(pa[-1], p2.x), p2, mk(ua[-1], u2.x));
      const f2 fyp = donor2s(p2, at2(pa + RX), v2);
      const f2 fym = donor2s(at2(pa - RX), p2, at2(va - RX));
      const f2 fzp = donor2s(p2, p3, w2);  // w2 = 0 on a zero-flux top face
      // the "-" z face is the previous level's "+" z face (the same operation
      // on the same values): stage A ran a level before every steady level
      const f2 fzm = S ? f1z : donor2s(p1, p2, w1);  // w1 = 0 on a zero-flux bottom face
      f1z = fzp;
      q2 = fma2(add2(add2(sub2(fxm, fxp), sub2(fym, fyp)), sub2(fzm, fzp)), rcp2(g2), p2);
      st2(P1v(a, 0), q2);
    }
    __syncthreads();
    // ---- B: pseudo-velocities on plane b = t+1 ---------------------------
    const int b = t + 1;
    const bool runB = inB && (S || (b >= max(klo, k0 - 2) && b <= min(khi, k1)));
    // psi1 of plane b around the pair, kept for stage C (the plane is not
    // written before C reads it)
    f2 pxm = zero2, pxp = zero2, pym = zero2, pyp = zero2;
    if (runB) {
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, klo);
      const f2 qp = (S || bp != b) ? q2 : q1;  // own psi1 at the clamped b+1
      const f2 qm = (S || bm != b) ? q0 : q1;  // own psi1 at the clamped b-1
      const float* pb1 = P1v(b, 0);
      const float* gb = gs + (b & 3) * L::SN + s2;
      const float* vb = vs + (b & 3) * L::RN + s3;
      const float* ub = us + (b & 3) * L::RN + s3;
      const float* wb = ws + (b & 3) * L::SN + s2;
      const float* wbm = ws + ((b - 1) & 3) * L::SN + s2;
      pyp = at2(pb1 + EX);                 // (x, x+1) at y+1
      pym = at2(pb1 - EX);                 // (x, x+1) at y-1
      pxp = mk(q1.y, pb1[2]);              // (x+1, x+2)
      pxm = mk(pb1[-1], q1.x);             // (x-1, x)
      if constexpr (OPT == 0) {  // the basic scheme (kept apart: its code as measured)
        // Every thread of B forms all three faces: row -2, which needs only
        // its y faces, forms x and z faces into a slot and a register nobody
        // reads, and the faces' arithmetic, with no branch between them,
        // interleaves (776 against 784 us a launch)
        {  // x faces
          const f2 s1p = add2(mk(pyp.y, pb1[EX + 2]), pyp);
          const f2 s1m = add2(mk(pym.y, pb1[-EX + 2]), pym);
          const f2 s2p = add2(mk(qp.y, P1v(bp, 2)[0]), qp);
          const f2 s2m = add2(mk(qm.y, P1v(bm, 2)[0]), qm);
          const f2 vm = at2(vb - RX);
          const f2 vsum = add2(add2(add2(v1, mk(v1.y, vb[2])), vm), mk(vm.y, vb[-RX + 2]));
          const f2 wsum = add2(add2(add2(w1, mk(w1.y, wb[2])), w0), mk(w0.y, wbm[2]));
          const f2 gsum = add2(g1, mk(g1.y, gb[2]));
          utB = pseudo2(u1, gsum, q1, pxp, s1p, s1m, s2p, s2m, vsum, wsum);
          st2(uts + s2, utB);
        }
        {  // y faces
          const f2 s1p = add2(mk(pyp.y, pb1[EX + 2]), pxp);
          const f2 s1m = add2(mk(pb1[EX - 1], pyp.x), pxm);
          const f2 s2p = add2(at2(P1v(bp, EX)), qp);
          const f2 s2m = add2(at2(P1v(bm, EX)), qm);
          const f2 up = at2(ub + RX);
          const f2 usum = add2(add2(add2(u1, up), mk(ub[-1], u1.x)), mk(ub[RX - 1], up.x));
          const f2 wsum = add2(add2(add2(w1, at2(wb + EX)), w0), at2(wbm + EX));
          const f2 gsum = add2(g1, at2(gb + EX));
          vtB = pseudo2(v1, gsum, q1, pyp, s1p, s1m, s2p, s2m, usum, wsum);
          st2(vts + s2, vtB);
        }
        {  // z faces
          f2 res = zero2;
          if (S || zface(b)) {  // a zero-flux top face is closed
            const float* pb2 = P1v(b + 1, 0);
            const float* ub1 = us + ((b + 1) & 3) * L::RN + s3;
            const float* vb1 = vs + ((b + 1) & 3) * L::RN + s3;
            const f2 s1p = add2(mk(q2.y, pb2[2]), pxp);
            const f2 s1m = add2(mk(pb2[-1], q2.x), pxm);
            const f2 s2p = add2(at2(pb2 + EX), pyp);
            const f2 s2m = add2(at2(pb2 - EX), pym);
            const f2 usum = add2(add2(add2(u1, u2), mk(ub[-1], u1.x)), mk(ub1[-1], u2.x));
            const f2 vsum = add2(add2(add2(v1, v2), at2(vb - RX)), at2(vb1 - RX));
            res = pseudo2(w1, add2(g1, g2), q1, q2, s1p, s1m, s2p, s2m, usum, vsum);
          }
          wtB = res;
        }
      } else {
        // Every thread of B forms all three faces: row -2, which needs only
        // its y faces, forms x and z faces into a slot and a register nobody
        // reads, and the faces' arithmetic, with no branch between them,
        // interleaves (776 against 784 us a launch)
        // DFL: the divergence of the Courant numbers of the pair's cells at
        // plane b (closed faces' W are 0 in the queue)
        const f2 dc = kDFL ? add2(add2(sub2(u1, mk(ub[-1], u1.x)), sub2(v1, at2(vb - RX))),
                                  sub2(w1, w0))
                           : zero2;
        {  // x faces
          const f2 s1p = add2(ap<kABS>(mk(pyp.y, pb1[EX + 2])), ap<kABS>(pyp));
          const f2 s1m = add2(ap<kABS>(mk(pym.y, pb1[-EX + 2])), ap<kABS>(pym));
          const f2 s2p = add2(ap<kABS>(mk(qp.y, P1v(bp, 2)[0])), ap<kABS>(qp));
          const f2 s2m = add2(ap<kABS>(mk(qm.y, P1v(bm, 2)[0])), ap<kABS>(qm));
          const f2 vm = at2(vb - RX);
          const f2 vsum = add2(add2(add2(v1, mk(v1.y, vb[2])), vm), mk(vm.y, vb[-RX + 2]));
          const f2 wsum = add2(add2(add2(w1, mk(w1.y, wb[2])), w0), mk(w0.y, wbm[2]));
          const f2 gsum = add2(g1, mk(g1.y, gb[2]));
          utB = pse<kIGA>(u1, gsum, ap<kABS>(q1), ap<kABS>(pxp), s1p, s1m, s2p, s2m, vsum, wsum);
          if constexpr (kDFL) {  // + the cells at x+1
            const f2 dr = add2(add2(sub2(mk(u1.y, ub[2]), u1), sub2(mk(v1.y, vb[2]), mk(vm.y, vb[-RX + 2]))),
                               sub2(mk(w1.y, wb[2]), mk(w0.y, wbm[2])));
            utB = add2(utB, dft2(u1, gsum, add2(dc, dr)));
          }
          st2(uts + s2, utB);
        }
        {  // y faces
          const f2 s1p = add2(ap<kABS>(mk(pyp.y, pb1[EX + 2])), ap<kABS>(pxp));
          const f2 s1m = add2(ap<kABS>(mk(pb1[EX - 1], pyp.x)), ap<kABS>(pxm));
          const f2 s2p = add2(ap<kABS>(at2(P1v(bp, EX))), ap<kABS>(qp));
          const f2 s2m = add2(ap<kABS>(at2(P1v(bm, EX))), ap<kABS>(qm));
          const f2 up = at2(ub + RX);
          const f2 usum = add2(add2(add2(u1, up), mk(ub[-1], u1.x)), mk(ub[RX - 1], up.x));
          const f2 wsum = add2(add2(add2(w1, at2(wb + EX)), w0), at2(wbm + EX));
          const f2 gsum = add2(g1, at2(gb + EX));
          vtB = pse<kIGA>(v1, gsum, ap<kABS>(q1), ap<kABS>(pyp), s1p, s1m, s2p, s2m, usum, wsum);
          if constexpr (kDFL) {  // + the cells at y+1
            const f2 dr = add2(add2(sub2(up, mk(ub[RX - 1], up.x)), sub2(at2(vb + RX), v1)),
                               sub2(at2(wb + EX), at2(wbm + EX)));
            vtB = add2(vtB, dft2(v1, gsum, add2(dc, dr)));
          }
          st2(vts + s2, vtB);
        }
        {  // z faces
          f2 res = zero2;
          if (S || zface(b)) {  // a zero-flux top face is closed
            const float* pb2 = P1v(b + 1, 0);
            const float* ub1 = us + ((b + 1) & 3) * L::RN + s3;
            const float* vb1 = vs + ((b + 1) & 3) * L::RN + s3;
            const f2 s1p = add2(ap<kABS>(mk(q2.y, pb2[2])), ap<kABS>(pxp));
            const f2 s1m = add2(ap<kABS>(mk(pb2[-1], q2.x)), ap<kABS>(pxm));
            const f2 s2p = add2(ap<kABS>(at2(pb2 + EX)), ap<kABS>(pyp));
            const f2 s2m = add2(ap<kABS>(at2(pb2 - EX)), ap<kABS>(pym));
            const f2 usum = add2(add2(add2(u1, u2), mk(ub[-1], u1.x)), mk(ub1[-1], u2.x));
            const f2 vsum = add2(add2(add2(v1, v2), at2(vb - RX)), at2(vb1 - RX));
            res = pse<kIGA>(w1, add2(g1, g2), ap<kABS>(q1), ap<kABS>(q2), s1p, s1m, s2p, s2m, usum, vsum);
            if constexpr (kDFL) {  // + the cells at plane b+1
              const f2 dr = add2(add2(sub2(u2, mk(ub1[-1], u2.x)), sub2(v2, at2(vb1 - RX))),
                                 sub2(w2, w1));
              res = add2(res, dft2(w1, add2(g1, g2), add2(dc, dr)));
            }
          }
          wtB = res;
        }
      }
    }
    __syncthreads();
    // ---- C: limiter bounds and betas on plane b = t+1 --------------------
    if (LIMIT && inC && (S || (b >= max(klo, k0 - 1) && b <= min(khi, k1)))) {  // tile + 1
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, klo);
      const f2 qp = (S || bp != b) ? q2 : q1, qm = (S || bm != b) ? q0 : q1;
      const float* pb = p0s + (b & 3) * L::RN + s3;
      const f2 vals[14] = {q1,  p1,  mk(pb[-1], p1.x), mk(p1.y, pb[2]), at2(pb - RX),
                           at2(pb + RX), p0, p2, pxm, pxp, pym, pyp, qm, qp};
      f2 hi, lo;
      bounds2(vals, hi, lo);
      const f2 fxp = cflux2<kIGA>(q1, pxp, utB);
      const f2 fxm = cflux2<kIGA>(pxm, q1, mk(uts[s2 - 1], utB.x));
      const f2 fyp = cflux2<kIGA>(q1, pyp, vtB);
      const f2 fym = cflux2<kIGA>(pym, q1, at2(vts + s2 - EX));
      const f2 fzp = cflux2<kIGA>(q1, qp, wtB);  // wtB = 0 on a zero-flux top face
      // the lower face's flux is the previous level's upper one (the same
      // operation on the same values): C ran a level before every steady level
      const f2 fzm = S ? c1z : cflux2<kIGA>(qm, q1, wtA);  // wtA = 0 on a zero-flux bottom face
      c1z = fzp;
      const f2 in = add2(add2(sub2(pos2(fxm), neg2(fxp)), sub2(pos2(fym), neg2(fyp))),
                         sub2(pos2(fzm), neg2(fzp)));
      const f2 ou = add2(add2(sub2(pos2(fxp), neg2(fxm)), sub2(pos2(fyp), neg2(fym))),
                         sub2(pos2(fzp), neg2(fzm)));
      const f2 ri = rcp2(add2(in, eps2)), ro = rcp2(add2(ou, eps2));
      buB = mul2(mul2(sub2(hi, q1), g1), ri);
      bdB = mul2(mul2(sub2(q1, lo), g1), ro);
      st2(sm + L::BUS + (b & 1) * L::SN + s2, buB);
      st2(sm + L::BDS + (b & 1) * L::SN + s2, bdB);
    }
    // ---- D: limited donor fluxes of plane t and face t+1/2 ---------------
    // (the betas of plane t were written at level t-1; no barrier after C)
    if (inD && (S || (t >= max(klo, k0 - 1) && t <= k1 - 1))) {
      const float* bu0 = sm + L::BUS + (t & 1) * L::SN + s2;
      const float* bd0 = sm + L::BDS + (t & 1) * L::SN + s2;
      const float* pt = P1v(t, 0);
      // the limited velocity of each lane; with ABS a face whose upwind psi1
      // is negative carries its flux against its velocity: beta-up and
      // beta-down trade places there
      auto lim = [&](f2 C, f2 pr, f2 buR, f2 bdR) {
        if constexpr (kABS) {
          auto lane = [&](float c, float q, float r, float bu, float bd, float bur, float bdr) {
            const bool sw = !ge0(ge0(c) ? q : r);
            return limit_factor(c, sw ? bd : bu, sw ? bu : bd, sw ? bdr : bur, sw ? bur : bdr);
          };
          return mul2(mk(lane(C.x, q0.x, pr.x, buA.x, bdA.x, buR.x, bdR.x),
                         lane(C.y, q0.y, pr.y, buA.y, bdA.y, buR.y, bdR.y)),
                      C);
        } else {
          return limit2(C, buA, bdA, buR, bdR);
        }
      };
      f2 u = utA, v = vtA, f = zero2, w = zero2;
      if constexpr (OPT == 0) {  // the basic scheme (kept apart: its code as measured)
        if (LIMIT) u = limit2(u, buA, bdA, mk(buA.y, bu0[2]), mk(bdA.y, bd0[2]));
        st2(fxs + (t & 1) * L::SN + s2, donor2(q0, mk(q0.y, pt[2]), u));
        if (LIMIT) v = limit2(v, buA, bdA, at2(bu0 + EX), at2(bd0 + EX));
        st2(fys + (t & 1) * L::SN + s2, donor2(q0, at2(pt + EX), v));
        if (S || zface(t)) {
          w = wtA;
          if (LIMIT) w = limit2(w, buA, bdA, buB, bdB);
          f = donor2(q0, q1, w);
        }
      } else {
        if (LIMIT) u = lim(u, mk(q0.y, pt[2]), mk(buA.y, bu0[2]), mk(bdA.y, bd0[2]));
        st2(fxs + (t & 1) * L::SN + s2, cflux2<kIGA>(q0, mk(q0.y, pt[2]), u));
        if (LIMIT) v = lim(v, at2(pt + EX), at2(bu0 + EX), at2(bd0 + EX));
        st2(fys + (t & 1) * L::SN + s2, cflux2<kIGA>(q0, at2(pt + EX), v));
        if (S || zface(t)) {
          w = wtA;
          if (LIMIT) w = lim(w, q1, buB, bdB);
          f = cflux2<kIGA>(q0, q1, w);
        }
      }
      fzB = f;
      if constexpr (TAPE) {
        if (t >= k0 && (wr0 || wr1)) {
          constexpr int NF = LIMIT ? 9 : 4;
          const f2 tv[9] = {q0, utA, vtA, wtA, buA, bdA, u, v, w};  // Wt, Wl: 0 on the top face
          float* tq = tape + c0 + t * pxy;
#pragma unroll
          for (int z = 0; z < NF; ++z) {
            float* d = tq + (long long)(z < 6 ? z : z + 2) * tstride;
            if (wr0 && wr1) {
              st2(d, tv[z]);
            } else {
              if (wr0) d[0] = tv[z].x;
              if (wr1) d[1] = tv[z].y;
            }
          }
        }
      }
    }
    // ---- E: advance and write psi^(n+1) on plane e = t-1 ------------------
    const int e = t - 1;
    if ((S || e >= k0) && (wr0 || wr1)) {
      const float* fx = fxs + (e & 1) * L::SN + s2;
      const float* fy = fys + (e & 1) * L::SN + s2;
      const f2 fzm = (S || zface(e - 1)) ? fzAA : zero2;
      const f2 fxo = at2(fx);
      const f2 nd = add2(add2(sub2(mk(fx[-1], fxo.x), fxo), sub2(at2(fy - EX), at2(fy))),
                         sub2(fzm, fzA));
      const f2 r = fma2(nd, rcp2(at2(gs + (e & 3) * L::SN + s2)), at2(P1v(e, 0)));
      if (S && !KPER && whole) {
        st2(out + c0 + e * pxy, r);  // both lanes, no periodic image
      } else {
        // each lane: one store, or the value and its periodic images in the
        // i-j halo and (bottom and top levels, or periodic k) the k halo
        auto put = [&](int lane, float val) {
          const int ii0 = gi + lane;
          const int ni = (ii0 < g.h) ? 1 : ((ii0 >= g.nx - g.h) ? -1 : 0);
          const int nj = (gj < g.h) ? 1 : ((gj >= g.ny - g.h) ? -1 : 0);
          if (ni == 0 && nj == 0 &&
              (KPER ? e >= g.h && e < nz - g.h : (S || (e > 0 && e < nz - 1)))) {
            out[c0 + lane + e * pxy] = val;
            return;
          }
          int ilo = (e == 0) ? -g.h : e, ihi = (e == nz - 1) ? nz - 1 + g.h : e;
          if constexpr (KPER) {
            ilo = e;
            while (ilo - nz >= -g.h) ilo -= nz;
            ihi = nz - 1 + g.h;
          }
          for (int kk = ilo; kk <= ihi; kk += kper ? nz : 1) {
            if (!kper && kk != e && kk >= 0 && kk < nz) continue;
            const int64_t pk = g.off0 + (int64_t)kk * g.pxy;
            for (int a2 = 0; a2 <= (ni != 0); ++a2) {
              const int ii = ii0 + a2 * ni * g.nx;
              for (int b2 = 0; b2 <= (nj != 0); ++b2) {
                const int jj = gj + b2 * nj * g.ny;
                out[pk + (int64_t)jj * g.px + ii] = val;
              }
            }
          }
        };
        if (wr0) put(0, r.x);
        if (wr1) put(1, r.y);
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
    if constexpr (KPER) { l4 = l5; l5 = l5 + 1 == nz ? 0 : l5 + 1; }
  };
  // steady levels as in the one-column kernel: zero-flux t in
  // [max(k0 + 1, 2), min(k1 - 1, nz - 6)], periodic k the chunk but its
  // first level; the last level, t = k1, runs stage E alone
  const int tS = KPER ? k0 + 1 : max(k0 + 1, 2), tE = KPER ? k1 - 1 : min(k1 - 1, nz - 6);
  int t = t0;
  for (; t < tS && t <= k1; ++t) level(t, std::false_type{});
  for (; t <= tE; ++t) level(t, std::true_type{});
  for (; t <= k1; ++t) level(t, std::false_type{});
}

}  // namespace fusedx
}  // namespace mpd
