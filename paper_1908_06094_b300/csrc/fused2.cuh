// fused2.cuh -- the one-kernel MPDATA step (iord = 2) with one thread per
// column.
//
// Per level t of the march, five stages run on planes t+2, t+1, t+1, t, t-1:
// A psi1 (donor pass), B pseudo-velocities, C limiter bounds and betas,
// D limited face fluxes, E advance and halo images.  A stage reads what an
// earlier level wrote, except B (psi1 of plane t+2, from A) and C (Ut, Vt of
// plane t+1, from B), so a level has two barriers: every shared ring holds
// enough planes that a level's writes never land in a slot the same level
// reads.  They are organised so that almost every instruction is arithmetic:
//   * the CTA has one thread per column of the tile + 2 ring, (TX+4)(TY+4)
//     threads; a thread keeps its own column's values (psi^n, U, V, W, G,
//     psi1, the pseudo-velocities, the betas, the vertical fluxes) in
//     register queues as it marches up in k, so vertical neighbours cost
//     nothing;
//   * each plane of psi^n, U, V, W, G is read from device memory once per CTA
//     (every thread loads its own column one plane ahead; threads 0..115
//     also load the radius-3 ring that the donor pass of the outer cells
//     needs) and published in shared memory, where horizontal neighbours are
//     read at compile-time offsets from the thread's own slot;
//   * the wrapped (periodic) column offsets are computed once per thread.
// Intermediates that neighbours need (psi1, Ut, Vt, betas, x/y fluxes) go to
// shared-memory rings; Wt and the vertical fluxes stay in registers.
#pragma once
#include <climits>
#include <type_traits>

#include "grid.cuh"

namespace mpd {
namespace fused2 {

template <class T, int TX, int TY>
struct Layout {
  static constexpr int EX = TX + 4, EY = TY + 4, SN = EX * EY;  // radius-2 planes
  static constexpr int RX = TX + 6, RY = TY + 6, RN = RX * RY;  // radius-3 planes
  static constexpr int NT = SN;                                 // threads per CTA
  static constexpr int NRING = RN - SN;                         // radius-3 ring cells
  // offsets (in elements of T)
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
  static constexpr size_t bytes = (size_t)NVAL * sizeof(T);
};

// Where a taped step also writes the intermediates of its own cells (the
// adjoint's tape): psi1, Ut, Vt, Wt, beta-up, beta-down, the limited Ul, Vl,
// Wl and, in FP64 only, the reciprocals 1/(in+eps), 1/(out+eps) (the FP32
// beta reverse re-forms them), all padded fields like psi.
template <class T>
struct TapeOut {
  T *p1, *ut, *vt, *wt, *bu, *bd, *ri, *ro, *ul, *vl, *wl;
};
// whether the tape keeps the limiter's reciprocals
template <class T> struct TapesReciprocals { static constexpr bool v = sizeof(T) == 8; };

// The column of thread tid in the (TX+4) x (TY+4) tile-plus-ring: the
// tile's TX*TY columns first, one tile row per TX threads (a warp a row for
// TX = 32), then the ring in the order of the stages that need it: the
// one-cell ring (stages B, C and D run on the tile and this ring), the
// cells of the second ring whose faces stage B must also form (column
// x = -2 and row y = -2: the "-" faces of the first ring's cells), and the
// rest of the second ring (stage A only).  So whole warps past a stage's
// region skip it.  NB = the threads stage B runs on, NC = those of C.
template <int TX, int TY>
struct TileMap {
  static constexpr int NC = (TX + 2) * (TY + 2);
  static constexpr int NB = NC + (TY + 2) + (TX + 2);
  static __device__ __forceinline__ void cell(int tid, int& x, int& y) {
    if (tid < TX * TY) { x = tid % TX; y = tid / TX; return; }
    int r = tid - TX * TY;
    if (r < TX + 2) { x = r - 1; y = -1; return; }      // row -1
    r -= TX + 2;
    if (r < TX + 2) { x = r - 1; y = TY; return; }      // row TY
    r -= TX + 2;
    if (r < TY) { x = -1; y = r; return; }              // column -1
    r -= TY;
    if (r < TY) { x = TX; y = r; return; }              // column TX
    r -= TY;
    if (r < TY + 2) { x = -2; y = r - 1; return; }      // column -2, rows -1 .. TY
    r -= TY + 2;
    if (r < TX + 2) { x = r - 1; y = -2; return; }      // row -2, columns -1 .. TX
    r -= TX + 2;
    if (r < TX + 4) { x = r - 2; y = TY + 1; return; }  // row TY+1
    r -= TX + 4;
    if (r < TY + 3) { x = TX + 1; y = r - 2; return; }  // column TX+1, rows -2 .. TY
    x = -2; y = -2;                                      // the last corner
  }
};

template <class T, int TX, int TY, bool LIMIT, bool TAPE = false, int UNROLL = 1,
          bool KPER = false, int OPT = 0, bool MAP = (UNROLL == 1), bool OPENIJ = false,
          bool I32 = false>
__device__ __forceinline__ void step_tile2(const Geo& g, int i0, int j0, int k0, int k1,
                                           const T* __restrict__ P0, const T* __restrict__ U,
                                           const T* __restrict__ V, const T* __restrict__ W,
                                           const T* __restrict__ G, T* __restrict__ out,
                                           unsigned char* smem_raw, TapeOut<T> tape = {}) {
  using L = Layout<T, TX, TY>;
  constexpr int EX = L::EX, RX = L::RX;
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int tid = threadIdx.x;
  const int nz = g.nz;
  const T zero = T(0), eps = Eps<T>::v;

  // own column: (x, y) in [-2, TX+1] x [-2, TY+1].  The single-domain
  // march (UNROLL = 1) orders its threads by TileMap and skips stages B, C,
  // D on the warps past their regions (FP32 512x512x128: 1.048 -> 1.030 ms,
  // periodic in k 1.081 -> 1.027 ms); the batch's unrolled march keeps one
  // thread per column in row-major order over the whole (TX+4)-wide plane
  // and runs B, C, D everywhere (the TileMap order made it 9.5 % slower).
  using Map = TileMap<TX, TY>;
  constexpr bool kMap = MAP;
  int x, y;
  if constexpr (kMap) {
    Map::cell(tid, x, y);
  } else {
    x = tid % EX - 2;
    y = tid / EX - 2;
  }
  const int s2 = (y + 2) * EX + (x + 2);      // radius-2 slot
  const int s3 = (y + 3) * RX + (x + 3);      // radius-3 slot
  const bool inB = !kMap || tid < Map::NB, inC = !kMap || tid < Map::NC;
  // stage B's faces: the x faces on the tile+1 and column x = -2, the y
  // faces on the tile+1 and row y = -2, the z faces on the tile+1
  const bool inBx = !kMap || tid < Map::NC + TY + 2;
  const bool inBy = !kMap || tid < Map::NC || (tid >= Map::NC + TY + 2 && tid < Map::NB);
  const bool inD = !kMap || (inC && x < TX && y < TY);  // the faces stage E reads
  // the column of a tile cell: wrapped (periodic domain) or, on a slab of a
  // decomposed domain, the cell itself, read from the exchanged halo (h >= 3
  // covers the radius-3 ring); cells of a partial last tile past the halo
  // are clamped into it -- they feed only columns past the interior, which
  // are never written
  // (OPENIJ: a compile-time variant, so the periodic instances carry none
  // of the slab's code)
  auto wrapi = [&](int i) {
    if constexpr (OPENIJ) return min(i, g.nx + g.h - 1);
    else return ((i % g.nx) + g.nx) % g.nx;
  };
  auto wrapj = [&](int j) {
    if constexpr (OPENIJ) return min(j, g.ny + g.h - 1);
    else return ((j % g.ny) + g.ny) % g.ny;
  };
  // element offsets: 32-bit when the padded field has fewer than 2^31
  // elements (I32: fewer registers and one-word address arithmetic)
  using Ix = std::conditional_t<I32, int, int64_t>;
  const Ix col = (Ix)wrapj(j0 + y) * (Ix)g.px + wrapi(i0 + x);
  // radius-3 ring cell of this thread (threads < NRING)
  const bool ringer = tid < L::NRING;
  int r3 = 0;
  Ix rcol = 0;
  if (ringer) {
    int rx, ry, r = tid;
    if (r < RX) { rx = r - 3; ry = -3; }
    else if ((r -= RX) < RX) { rx = r - 3; ry = TY + 2; }
    else if ((r -= RX) < L::EY) { rx = -3; ry = r - 2; }
    else { r -= L::EY; rx = TX + 2; ry = r - 2; }
    r3 = (ry + 3) * RX + (rx + 3);
    rcol = (Ix)wrapj(j0 + ry) * (Ix)g.px + wrapi(i0 + rx);
  }
  const Ix pxy = (Ix)g.pxy;
  constexpr bool kper = KPER;  // periodic in k (g.kper): a compile-time variant
  // the level of plane k: clamped (edge copy) or, periodic in k, wrapped
  // (any distance: the march runs up to 5 planes past the grid)
  auto clampk_ = [&](int k) {
    return kper ? ((k % nz) + nz) % nz : (k < 0 ? 0 : (k >= nz ? nz - 1 : k));
  };
  // the planes a stage runs on: the chunk's range widened by the stage's
  // depth, cut to the grid unless k is periodic (then every plane is real)
  const int klo = kper ? INT_MIN / 2 : 0, khi = kper ? INT_MAX / 2 : nz - 1;
  // the face above plane k carries flux
  auto zface = [&](int k) { return kper || (k >= 0 && k < nz - 1); };
  // per-thread column pointers (plane 0); plane k is + k*pxy (warp-uniform)
  const Ix c0 = (Ix)g.off0 + col, rc0 = (Ix)g.off0 + rcol;
  auto ld = [&](const T* f, int k, Ix c) { return f[c + (Ix)clampk_(k) * pxy]; };
  // vertical face value with the closed bottom and top faces
  auto ldw = [&](int k, Ix c) {
    if constexpr (KPER) return W[c + (Ix)clampk_(k) * pxy];
    else return (k < 0 || k >= nz - 1) ? zero : W[c + (Ix)k * pxy];
  };
  // shared-memory views
  T* p0s = sm + L::P0S;
  T* us = sm + L::US;
  T* vs = sm + L::VS;
  T* ws = sm + L::WS;
  T* gs = sm + L::GS;
  T* p1s = sm + L::P1S;
  T* uts = sm + L::UTS;
  T* vts = sm + L::VTS;
  T* fxs = sm + L::FXS;
  T* fys = sm + L::FYS;
  auto P1 = [&](int k, int o) -> T& { return p1s[(k & 3) * L::SN + s2 + o]; };
  // corrective-pass options (kOpt* bits): ABS forms A and B from |psi1|, IGA
  // uses the infinite-gauge pseudo-fluxes (which are the corrective fluxes),
  // DFL adds the divergent-flow term
  constexpr bool kABS = (OPT & kOptABS) != 0, kIGA = (OPT & kOptIGA) != 0;
  constexpr bool kDFL = (OPT & kOptDFL) != 0;
  auto ap = [&](T v) { return kABS ? absv(v) : v; };
  auto pseudo = [&](T C, T gsum, T pl, T pr, T s1p, T s1m, T s2p, T s2m, T c1, T c2) {
    if constexpr (kIGA) return pseudo_flux_iga(C, gsum, pl, pr, s1p, s1m, s2p, s2m, c1, c2);
    else return pseudo_velocity(C, gsum, pl, pr, s1p, s1m, s2p, s2m, c1, c2);
  };
  // the corrective flux of a face: the donor flux of its (limited) velocity,
  // or, in the infinite gauge, the value itself
  auto cflux = [&](T L_, T R_, T C) {
    if constexpr (kIGA) return C;
    else return donor(L_, R_, C);
  };

  // Stages B, C and D run on the columns whose results a later stage reads
  // (inB, inC, inD; see TileMap), with a few extra lanes in the warps that
  // straddle two regions (the unrolled march: on every column); the extra
  // lanes read neighbouring shared slots that
  // stay inside the shared allocation (the arrays are laid out so a
  // radius-1 step off the plane lands in the neighbouring array) and their
  // results are never read.
  const bool inT = x >= 0 && x < TX && y >= 0 && y < TY;
  const int gi = i0 + x, gj = j0 + y;
  const bool writes = inT && gi < g.nx && gj < g.ny;
  // the column's periodic images in the i/j halo (+1 / -1: one period up /
  // down, 0: none), formed once for the unrolled march (the batch's:
  // +2.4 % there); the single-domain march (UNROLL = 1) forms them per
  // level, where the registers they would hold across the march cost 3.7 %
  // the column has no periodic image in the i-j halo (the single-domain
  // march's steady levels store such a value with one store)
  const bool noimg = OPENIJ || (gi >= g.h && gi < g.nx - g.h && gj >= g.h && gj < g.ny - g.h);
  int niU = 0, njU = 0;
  if constexpr (UNROLL > 1) {
    niU = OPENIJ ? 0 : ((gi < g.h) ? 1 : ((gi >= g.nx - g.h) ? -1 : 0));
    njU = OPENIJ ? 0 : ((gj < g.h) ? 1 : ((gj >= g.ny - g.h) ? -1 : 0));
  }

  // The march starts 5 levels below the chunk (stages A..E are 5 levels
  // deep).  With UNROLL = 2 or 4 the start is rounded down to a multiple of
  // UNROLL and the levels run in groups of UNROLL, so the ring slot indices
  // (t & 1, t & 3) are constants of each unrolled copy; the extra levels at
  // the start are skipped by the stage guards.  Measured on the B300: the
  // single-domain kernel is fastest at 1 (1.10 ms, against 1.19 at 4 and
  // 1.29 at 2 on 512x512x128), the batch, with its many short chunks, at 4
  // (2.65e10 against 2.44e10 tracer-updates/s).
  // Under the zero-flux boundary no stage runs below plane 0, so the
  // unrolled march (the batch's items march whole columns from the bottom)
  // begins a chunk at the bottom at t = -2, where stage A reaches plane 0
  // (the planes below are edge copies the clamped loads supply): four
  // levels of loads and barriers fewer, +3.3 % tracer-updates/s.  (The
  // single-domain march measured 0.2 % slower with it and keeps k0 - 5.)
  static_assert(UNROLL == 1 || UNROLL == 2 || UNROLL == 4, "UNROLL: 1, 2 or 4");
  const int t0 =
      ((KPER || UNROLL == 1) ? k0 - 5 : max(k0 - 5, -2)) & ~(UNROLL - 1);
  // register queues of the own column (values at planes t..t+3 / faces t..t+2)
  T p0 = ld(P0, t0, c0), p1 = ld(P0, t0 + 1, c0), p2 = ld(P0, t0 + 2, c0);
  T p3 = ld(P0, t0 + 3, c0), pn = ld(P0, t0 + 4, c0);
  T u1 = ld(U, t0 + 1, c0), u2 = ld(U, t0 + 2, c0), un = ld(U, t0 + 3, c0);
  T v1 = ld(V, t0 + 1, c0), v2 = ld(V, t0 + 2, c0), vn = ld(V, t0 + 3, c0);
  T w0 = ldw(t0, c0), w1 = ldw(t0 + 1, c0), w2 = ldw(t0 + 2, c0), wn = ldw(t0 + 3, c0);
  T g0 = ld(G, t0, c0), g1 = ld(G, t0 + 1, c0), g2 = ld(G, t0 + 2, c0), gn = ld(G, t0 + 3, c0);
  T rp = zero, ru = zero, rv = zero;  // ring values of plane t+3
  if (ringer) { rp = ld(P0, t0 + 3, rc0); ru = ld(U, t0 + 3, rc0); rv = ld(V, t0 + 3, rc0); }
  T q0 = zero, q1 = zero, q2 = zero;     // psi1 at t, t+1, t+2
  T utA = zero, vtA = zero, utB = zero, vtB = zero;  // Ut, Vt at t, t+1
  T wtA = zero, wtB = zero;              // Wt at faces t+1/2, t+3/2
  T buA = zero, bdA = zero, buB = zero, bdB = zero;  // betas at t, t+1
  constexpr bool kTapeR = TAPE && TapesReciprocals<T>::v;
  T riA = zero, roA = zero, riB = zero, roB = zero;  // their 1/(in+eps), 1/(out+eps) (FP64 tape)
  T fzAA = zero, fzA = zero, fzB = zero;  // vertical fluxes at faces t-3/2, t-1/2, t+1/2
  T f1z = zero;  // the donor flux through face t+3/2 (stage A's last "+" z face)

  // periodic k: the wrapped levels of planes t+4, t+5, advanced by one
  // level per plane (no division in the loop)
  int l4 = clampk_(t0 + 4), l5 = clampk_(t0 + 5);

  // Each level publishes the planes the next level's first stage reads
  // (psi^n, U, V at t+3, W at face t+2, G at t+2), so a stage of level t
  // reads only what level t-1 or an earlier stage of level t wrote: the
  // slots of the planes published at level t are not read at level t.
  // The march starts with the planes its first level reads.
  __syncthreads();  // the shared memory may still be read by a previous tile
  {
    const int a = t0 + 2;
    p0s[(a & 3) * L::RN + s3] = p2;
    us[(a & 3) * L::RN + s3] = u2;
    vs[(a & 3) * L::RN + s3] = v2;
    if (ringer) {
      p0s[(a & 3) * L::RN + r3] = ld(P0, a, rc0);
      us[(a & 3) * L::RN + r3] = ld(U, a, rc0);
      vs[(a & 3) * L::RN + r3] = ld(V, a, rc0);
    }
    ws[((t0 + 1) & 3) * L::SN + s2] = w1;
    gs[((t0 + 1) & 3) * L::SN + s2] = g1;
  }
  __syncthreads();
  // One level of the march.  STEADY: a level inside the chunk where every
  // stage runs and no vertical neighbour is clamped or closed, so the
  // stages' plane guards and the boundary clamps are compile-time true.
  auto level = [&](const int t, auto steady) {
    constexpr bool S = decltype(steady)::value;
    // ---- publish plane t+3 of psi^n, U, V, face t+2 of W, plane t+2 of G --
    // (read from level t+1 on: no barrier before stage A)
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
    // loads one plane ahead (used from the next iteration on); the plane
    // offsets are the same for every thread
    // (steady levels, zero-flux: planes t+4 and t+5 are inside the grid and
    // the face t+4 is open)
    const Ix o5 = (Ix)(KPER ? l5 : (S ? t + 5 : clampk_(t + 5))) * pxy;
    const Ix o4 = (KPER || !S) ? (Ix)(KPER ? l4 : clampk_(t + 4)) * pxy : o5 - pxy;
    const T pn_next = P0[c0 + o5];
    const T un_next = U[c0 + o4], vn_next = V[c0 + o4], gn_next = G[c0 + o4];
    const T wn_next = (S || zface(t + 4)) ? W[c0 + o4] : zero;  // closed faces
    T rp_next = zero, ru_next = zero, rv_next = zero;
    if (ringer) {
      rp_next = P0[rc0 + o4];
      ru_next = U[rc0 + o4];
      rv_next = V[rc0 + o4];
    }
    // ---- A: psi1 on plane a = t+2 ---------------------------------------
    const int a = t + 2;
    if (S || (a >= max(klo, k0 - 3) && a <= min(khi, k1 + 1))) {
      const T* pa = p0s + (a & 3) * L::RN + s3;
      const T* ua = us + (a & 3) * L::RN + s3;
      const T* va = vs + (a & 3) * L::RN + s3;
      const T fxp = donor(p2, pa[1], u2);
      const T fxm = donor(pa[-1], p2, ua[-1]);
      const T fyp = donor(p2, pa[RX], v2);
      const T fym = donor(pa[-RX], p2, va[-RX]);
      const T fzp = donor(p2, p3, w2);  // w2 = 0 on a zero-flux top face
      // the "-" z face is the previous level's "+" z face (the same operation
      // on the same values): stage A ran a level before every steady level
      const T fzm = S ? f1z : donor(p1, p2, w1);  // w1 = 0 on a zero-flux bottom face
      f1z = fzp;
      // psi - div * (1/G), one rounding: the negated divergence is formed
      // exactly (every difference and sum negated) and fused in
      q2 = fma_rn((fxm - fxp) + (fym - fyp) + (fzm - fzp), rcp(g2), p2);
      P1(a, 0) = q2;
    }
    __syncthreads();
    // ---- B: pseudo-velocities on plane b = t+1 ---------------------------
    const int b = t + 1;
    const bool runB = inB && (S || (b >= max(klo, k0 - 2) && b <= min(khi, k1)));
    if (runB) {
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, klo);
      const T qp = (S || bp != b) ? q2 : q1;  // own psi1 at the clamped b+1
      const T qm = (S || bm != b) ? q0 : q1;  // own psi1 at the clamped b-1
      const T* gb = gs + (b & 3) * L::SN + s2;
      const T* vb = vs + (b & 3) * L::RN + s3;
      const T* ub = us + (b & 3) * L::RN + s3;
      const T* wb = ws + (b & 3) * L::SN + s2;
      const T* wbm = ws + ((b - 1) & 3) * L::SN + s2;
      // DFL: the divergence of the Courant numbers of the cell at plane b,
      // own column (closed faces' W are 0 in the queue)
      const T dc = kDFL ? (u1 - ub[-1]) + (v1 - vb[-RX]) + (w1 - w0) : zero;
      if (inBx) {  // x face (used on x in [-2, TX], y in [-1, TY])
        const T s1p = ap(P1(b, EX + 1)) + ap(P1(b, EX)), s1m = ap(P1(b, -EX + 1)) + ap(P1(b, -EX));
        const T s2p = ap(P1(bp, 1)) + ap(qp), s2m = ap(P1(bm, 1)) + ap(qm);
        const T vsum = v1 + vb[1] + vb[-RX] + vb[-RX + 1];
        const T wsum = w1 + wb[1] + w0 + wbm[1];
        const T gsum = g1 + gb[1];
        utB = pseudo(u1, gsum, ap(q1), ap(P1(b, 1)), s1p, s1m, s2p, s2m, vsum, wsum);
        if constexpr (kDFL) {  // + the cell at x+1
          const T dr = (ub[1] - u1) + (vb[1] - vb[-RX + 1]) + (wb[1] - wbm[1]);
          utB = add_rn(utB, divergent_flow_term(u1, gsum, dc + dr));
        }
        uts[s2] = utB;
      }
      if (inBy) {  // y face (used on x in [-1, TX], y in [-2, TY])
        const T s1p = ap(P1(b, EX + 1)) + ap(P1(b, 1)), s1m = ap(P1(b, EX - 1)) + ap(P1(b, -1));
        const T s2p = ap(P1(bp, EX)) + ap(qp), s2m = ap(P1(bm, EX)) + ap(qm);
        const T usum = u1 + ub[RX] + ub[-1] + ub[RX - 1];
        const T wsum = w1 + wb[EX] + w0 + wbm[EX];
        const T gsum = g1 + gb[EX];
        vtB = pseudo(v1, gsum, ap(q1), ap(P1(b, EX)), s1p, s1m, s2p, s2m, usum, wsum);
        if constexpr (kDFL) {  // + the cell at y+1
          const T dr = (ub[RX] - ub[RX - 1]) + (vb[RX] - v1) + (wb[EX] - wbm[EX]);
          vtB = add_rn(vtB, divergent_flow_term(v1, gsum, dc + dr));
        }
        vts[s2] = vtB;
      }
      if (inC) {  // z face (used on x in [-1, TX], y in [-1, TY])
        T res = zero;
        if (S || zface(b)) {  // a zero-flux top face is closed
          const T* ub1 = us + ((b + 1) & 3) * L::RN + s3;
          const T* vb1 = vs + ((b + 1) & 3) * L::RN + s3;
          const T s1p = ap(P1(b + 1, 1)) + ap(P1(b, 1)), s1m = ap(P1(b + 1, -1)) + ap(P1(b, -1));
          const T s2p = ap(P1(b + 1, EX)) + ap(P1(b, EX));
          const T s2m = ap(P1(b + 1, -EX)) + ap(P1(b, -EX));
          const T usum = u1 + u2 + ub[-1] + ub1[-1];
          const T vsum = v1 + v2 + vb[-RX] + vb1[-RX];
          res = pseudo(w1, g1 + g2, ap(q1), ap(q2), s1p, s1m, s2p, s2m, usum, vsum);
          if constexpr (kDFL) {  // + the cell at plane b+1
            const T dr = (u2 - ub1[-1]) + (v2 - vb1[-RX]) + (w2 - w1);
            res = add_rn(res, divergent_flow_term(w1, g1 + g2, dc + dr));
          }
        }
        wtB = res;
      }
    }
    __syncthreads();
    // ---- C: limiter bounds and betas on plane b = t+1 --------------------
    if (LIMIT && inC && (S || (b >= max(klo, k0 - 1) && b <= min(khi, k1)))) {  // tile + 1
      const int bp = S ? b + 1 : min(b + 1, khi), bm = S ? b - 1 : max(b - 1, klo);
      const T qp = (S || bp != b) ? q2 : q1, qm = (S || bm != b) ? q0 : q1;
      const T* pb = p0s + (b & 3) * L::RN + s3;
      const T pxm = P1(b, -1), pxp = P1(b, 1), pym = P1(b, -EX), pyp = P1(b, EX);
      const T vals[14] = {q1, p1, pb[-1], pb[1], pb[-RX], pb[RX], p0, p2,
                          pxm, pxp, pym, pyp, qm, qp};
      T hi, lo;
      bounds(vals, hi, lo);
      const T fxp = cflux(q1, pxp, utB);
      const T fxm = cflux(pxm, q1, uts[s2 - 1]);
      const T fyp = cflux(q1, pyp, vtB);
      const T fym = cflux(pym, q1, vts[s2 - EX]);
      const T fzp = cflux(q1, qp, wtB);  // wtB = 0 on a zero-flux top face
      const T fzm = cflux(qm, q1, wtA);  // wtA = 0 on a zero-flux bottom face
      const T in = (pos(fxm) - neg(fxp)) + (pos(fym) - neg(fyp)) + (pos(fzm) - neg(fzp));
      const T ou = (pos(fxp) - neg(fxm)) + (pos(fyp) - neg(fym)) + (pos(fzp) - neg(fzm));
      const T ri = rcp(in + eps), ro = rcp(ou + eps);
      buB = (hi - q1) * g1 * ri;
      bdB = (q1 - lo) * g1 * ro;
      if (kTapeR) { riB = ri; roB = ro; }
      sm[L::BUS + (b & 1) * L::SN + s2] = buB;
      sm[L::BDS + (b & 1) * L::SN + s2] = bdB;
    }
    // (no barrier: D reads the betas of plane t, written at level t-1, and
    // its own betas of plane t+1; C and D share no other slot)
    // ---- D: limited donor fluxes of plane t and face t+1/2 ---------------
    if (inD && (S || (t >= max(klo, k0 - 1) && t <= k1 - 1))) {
      const T* bu0 = sm + L::BUS + (t & 1) * L::SN + s2;
      const T* bd0 = sm + L::BDS + (t & 1) * L::SN + s2;
      // the limited velocity; with ABS a face whose upwind psi1 is negative
      // carries its flux against its velocity: beta-up and beta-down trade
      // places there
      auto lim = [&](T C, T pr, T buR, T bdR) {
        T uL = buA, dL = bdA, uR = buR, dR = bdR;
        if constexpr (kABS) {
          if (!ge0(ge0(C) ? q0 : pr)) {
            uL = bdA; dL = buA; uR = bdR; dR = buR;
          }
        }
        return limit_face(C, uL, dL, uR, dR);
      };
      T u = utA;  // used on x in [-1, TX-1], y in [0, TY-1]
      if (LIMIT) u = lim(u, P1(t, 1), bu0[1], bd0[1]);
      fxs[(t & 1) * L::SN + s2] = cflux(q0, P1(t, 1), u);
      T v = vtA;  // used on x in [0, TX-1], y in [-1, TY-1]
      if (LIMIT) v = lim(v, P1(t, EX), bu0[EX], bd0[EX]);
      fys[(t & 1) * L::SN + s2] = cflux(q0, P1(t, EX), v);
      T f = zero, w = zero;
      if (S || zface(t)) {
        w = wtA;
        if (LIMIT) w = lim(w, q1, buB, bdB);
        f = cflux(q0, q1, w);
      }
      fzB = f;
      if (TAPE && t >= k0 && writes) {
        const int64_t q = (int64_t)c0 + (int64_t)t * (int64_t)pxy;
        tape.p1[q] = q0;
        tape.ut[q] = utA;
        tape.vt[q] = vtA;
        tape.wt[q] = wtA;  // 0 on the top face
        if (LIMIT) {
          tape.bu[q] = buA;
          tape.bd[q] = bdA;
          if (kTapeR) {
            tape.ri[q] = riA;
            tape.ro[q] = roA;
          }
          tape.ul[q] = u;
          tape.vl[q] = v;
          tape.wl[q] = w;
        }
      }
    }
    // ---- E: advance and write psi^(n+1) on plane e = t-1 ------------------
    // (one level behind D: its fluxes were written before this level's
    // barriers, so no barrier separates D and E; psi1 and G of plane e come
    // from the thread's own shared slots)
    const int e = t - 1;
    if ((S || e >= k0) && writes) {
      const T* fx = fxs + (e & 1) * L::SN + s2;
      const T* fy = fys + (e & 1) * L::SN + s2;
      const T fzm = (S || zface(e - 1)) ? fzAA : zero;
      const T r = fma_rn((fx[-1] - fx[0]) + (fy[-EX] - fy[0]) + (fzm - fzA),
                         rcp(gs[(e & 3) * L::SN + s2]), P1(e, 0));
      // a steady level of a column without i-j images: one store
      if (S && !KPER && UNROLL == 1 && noimg) {
        out[c0 + (Ix)e * pxy] = r;
      } else {
      // the column's periodic images in the i-j halo (none on a slab: the
      // halo exchange fills a slab's halo)
      const int ni = UNROLL > 1 ? niU
                                : (OPENIJ ? 0 : ((gi < g.h) ? 1 : ((gi >= g.nx - g.h) ? -1 : 0)));
      const int nj = UNROLL > 1 ? njU
                                : (OPENIJ ? 0 : ((gj < g.h) ? 1 : ((gj >= g.ny - g.h) ? -1 : 0)));
      // the value and its periodic images in the halo
      auto images = [&]() {
        // the levels holding this value: e, and its k-halo images -- edge
        // copies of the bottom and top levels, or under periodic k the
        // levels e + m nz within [-h, nz + h)
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
            const int ii = gi + a2 * ni * g.nx;
            for (int b2 = 0; b2 <= (nj != 0); ++b2) {
              const int jj = gj + b2 * nj * g.ny;
              out[pk + (int64_t)jj * g.px + ii] = r;
            }
          }
        }
      };
      // a value without images takes a single store
      if (ni == 0 && nj == 0 &&
          (KPER ? e >= g.h && e < nz - g.h : (S || (e > 0 && e < nz - 1))))
        out[c0 + (Ix)e * pxy] = r;
      else
        images();
      }
    }
    // ---- shift the queues ------------------------------------------------
    p0 = p1; p1 = p2; p2 = p3; p3 = pn; pn = pn_next;
    u1 = u2; u2 = un; un = un_next;
    v1 = v2; v2 = vn; vn = vn_next;
    w0 = w1; w1 = w2; w2 = wn; wn = wn_next;
    g0 = g1; g1 = g2; g2 = gn; gn = gn_next;
    rp = rp_next; ru = ru_next; rv = rv_next;
    q0 = q1; q1 = q2;
    utA = utB; vtA = vtB; wtA = wtB;
    buA = buB; bdA = bdB;
    if (kTapeR) { riA = riB; roA = roB; }
    fzAA = fzA; fzA = fzB;
    if constexpr (KPER) { l4 = l5; l5 = l5 + 1 == nz ? 0 : l5 + 1; }
  };
  // The single-domain march runs its steady levels without guards (FP32
  // 512x512x128: 989 -> 945 us per launch); the batch's unrolled march
  // keeps every level guarded (its steady groups spilled at the register
  // cap and measured 6 % slower).
  if constexpr (UNROLL == 1) {
    // the levels where every guard holds: zero-flux, t in [max(k0 + 1, 2),
    // min(k1 - 1, nz - 6)] (stage E advances a plane of the chunk with an
    // open face below it, no stage reaches below plane 0 or the top two
    // planes, and the loads one plane ahead stay below the top); periodic
    // in k, the chunk but its first level.  The last level, t = k1, runs
    // stage E alone.
    const int tS = KPER ? k0 + 1 : max(k0 + 1, 2), tE = KPER ? k1 - 1 : min(k1 - 1, nz - 6);
    int t = t0;
    for (; t < tS && t <= k1; ++t) level(t, std::false_type{});
    for (; t <= tE; ++t) level(t, std::true_type{});
    for (; t <= k1; ++t) level(t, std::false_type{});
  } else {
    for (int tg = t0; tg <= k1; tg += UNROLL) {
#pragma unroll
      for (int u = 0; u < UNROLL; ++u) {
        const int t = tg + u;
        if (t > k1) break;  // uniform over the CTA
        level(t, std::false_type{});
      }
    }
  }
  // The next tile's march (the batch's items) starts with a barrier before
  // it publishes its first planes.
}

template <class T, int TX, int TY, int MINB, bool LIMIT, bool TAPE = false, bool KPER = false,
          int OPT = 0, int UNROLL = 1, bool OPENIJ = false, bool I32 = false>
__global__ void __launch_bounds__((TX + 4) * (TY + 4), MINB)
step_kernel2(Geo g, int kchunk, const T* __restrict__ P0, const T* __restrict__ U,
             const T* __restrict__ V, const T* __restrict__ W, const T* __restrict__ G,
             T* __restrict__ out, TapeOut<T> tape) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k0 = blockIdx.z * kchunk;
  step_tile2<T, TX, TY, LIMIT, TAPE, UNROLL, KPER, OPT, true, OPENIJ, I32>(g, blockIdx.x * TX, blockIdx.y * TY, k0,
                                              min(g.nz, k0 + kchunk), P0, U, V, W, G, out,
                                              smem_raw, tape);
}

}  // namespace fused2
}  // namespace mpd
