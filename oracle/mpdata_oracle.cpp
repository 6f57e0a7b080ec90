/*
 * MPDATA oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, loop-by-loop FP64 CPU statement of one MPDATA time step on a
 * structured, halo-padded 3D grid.  It exists to check the CUDA library; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header or constant with the CUDA path.
 *
 * Storage: every field is [nz+2h][ny+2h][nx+2h], i fastest.  U[k][j][i] is
 * the face i+1/2, V the face j+1/2, W the face k+1/2 (C-grid convention of
 * Sec. 3.1.4.1).  U, V, W are G-weighted Courant numbers.
 *
 * Where the paper fixes the arithmetic it is followed directly:
 *   - donor-cell (upwind) flux F(L,R,C) = max(C,0) L + min(C,0) R
 *     (Listings 4 and 5);
 *   - vertical flux with zero-flux top and bottom faces, i.e. the boundary
 *     factor pivbz = 0 (Listing 7);
 *   - flux divergence followed by the solution advance (Listings 8 and 9),
 *     with the metric/density G in the role of the density rho.
 * The paper defers the antidiffusive and non-oscillatory passes to another
 * document (Sec. 5), so they follow the published MPDATA literature: the
 * pseudo-velocity with A and B ratios (Smolarkiewicz 1984), the G-weighted
 * form (Smolarkiewicz & Margolin 1998) and the non-oscillatory limiter
 * (Smolarkiewicz & Grabowski 1990).  Step order:
 *   1. halo fill: periodic in i and j, edge copy in k; zero-flux W faces;
 *   2. donor-cell pass -> psi1;
 *   3. for m = 2..iord: pseudo-velocities from psi^(m-1); optional limiter
 *      (bounds over the 7-point stencil of psi^n and psi^(m-1), beta-up and
 *      beta-down, limited velocities); donor-cell pass with them;
 *   4. psi^(n+1) = psi^(iord).
 * epsilon = 1e-15 in every ratio.  Ties: max(a,b) = a if a >= b, min(a,b) = a
 * if a <= b, and |x| has derivative sign(x) with sign(0) = 0.
 *
 * Options of the corrective passes (bit flags, forward only; the paper does
 * not describe them, they follow the MPDATA literature):
 *   1 DFL  divergent-flow term added to the pseudo-velocities (Smolarkiewicz
 *          1984);
 *   2 ABS  signed fields: A and B are formed from |psi|, and the limiter
 *          takes its factors by the direction of the flux, not of the
 *          velocity (the two agree where psi >= 0);
 *   4 IGA  infinite gauge: the limit c -> infinity of the scheme applied to
 *          psi + c (Smolarkiewicz & Clark 1986): linear pseudo-fluxes that
 *          are themselves the corrective fluxes.
 *
 * The scalar type is a template parameter so that the same code, run on dual
 * numbers, gives the exact tangent-linear model used to pin the adjoint.
 */
#include <cmath>
#include <cstring>
#include <cstdint>
#include <algorithm>
#include <vector>

namespace {

const double EPS = 1e-15;

struct Grid {
  int nx, ny, nz, h;
  bool kper;        // periodic in k (else zero-flux top and bottom faces)
  long px, py, pz;  // padded extents
  Grid(int nx_, int ny_, int nz_, int h_, int kbc = 0)
      : nx(nx_), ny(ny_), nz(nz_), h(h_), kper(kbc == 1) {
    px = nx + 2L * h; py = ny + 2L * h; pz = nz + 2L * h;
  }
  // whether the vertical face above level k carries flux (the top face
  // k = nz-1 is closed unless k is periodic)
  bool zface(int k) const { return kper || k < nz - 1; }
  long size() const { return px * py * pz; }
  long at(int i, int j, int k) const { return ((k + h) * py + (j + h)) * px + (i + h); }
};

struct Opts {
  bool dfl, abs, iga;
  explicit Opts(int f = 0) : dfl(f & 1), abs(f & 2), iga(f & 4) {}
};

/* ---------------------------------------------------------------- scalars */

struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }

template <class T> inline T omax(T a, T b) { return val(a) >= val(b) ? a : b; }
template <class T> inline T omin(T a, T b) { return val(a) <= val(b) ? a : b; }
inline double oabs(double x) { return std::fabs(x); }
inline Dual oabs(Dual x) {
  return Dual(std::fabs(x.v), x.v > 0 ? x.d : (x.v < 0 ? -x.d : 0.0));
}

/* Donor-cell (upwind) flux through a face with left value L, right value R
   and face Courant number C (Listings 4/5). */
template <class T> inline T donor(T L, T R, T C) {
  return omax(C, T(0.0)) * L + omin(C, T(0.0)) * R;
}

/* ------------------------------------------------------------------ halos */

inline int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

/* Cell-centred fields (psi, G) and the horizontal face fields (U, V):
   periodic in i and j, corners included; the k halo copies the edge level
   (periodic k: the level nz away). */
template <class T> void fill_halo_periodic(T* f, const Grid& g) {
  for (int k = 0; k < g.nz; ++k) {
    for (int j = 0; j < g.ny; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i)
        if (i < 0 || i >= g.nx) f[g.at(i, j, k)] = f[g.at(wrap(i, g.nx), j, k)];
    for (int j = -g.h; j < g.ny + g.h; ++j)
      if (j < 0 || j >= g.ny)
        for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, wrap(j, g.ny), k)];
  }
  for (int k = -g.h; k < g.nz + g.h; ++k) {
    if (k >= 0 && k < g.nz) continue;
    int ks = g.kper ? wrap(k, g.nz) : (k < 0 ? 0 : g.nz - 1);
    for (int j = -g.h; j < g.ny + g.h; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = f[g.at(i, j, ks)];
  }
}

/* Vertical face fields (W, its pseudo-velocity): periodic in i and j; the
   bottom face (k = -1, i.e. -1/2) and the top face (k = nz-1, i.e. nz-1/2)
   carry no flux (pivbz = 0 in Listing 7), nor does anything beyond them. */
template <class T> void fill_halo_wface(T* f, const Grid& g) {
  fill_halo_periodic(f, g);
  if (g.kper) return;  // periodic k: every face is open, the halo wraps
  for (int k = -g.h; k < g.nz + g.h; ++k) {
    if (k >= 0 && k < g.nz - 1) continue;
    for (int j = -g.h; j < g.ny + g.h; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i) f[g.at(i, j, k)] = T(0.0);
  }
}

/* -------------------------------------------------------------- the stages */

/* Flux divergence and solution advance (Listings 8/9):
   out = P - (1/G) * sum_d [F(P_c, P_c+d, C_c+d/2) - F(P_c-d, P_c, C_c-d/2)]. */
template <class T>
void advance(const Grid& g, const T* P, const T* u, const T* v, const T* w, const T* G, T* out) {
  const long sx = 1, sy = g.px, sz = g.px * g.py;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        T fxp = donor(P[c], P[c + sx], u[c]);
        T fxm = donor(P[c - sx], P[c], u[c - sx]);
        T fyp = donor(P[c], P[c + sy], v[c]);
        T fym = donor(P[c - sy], P[c], v[c - sy]);
        T fzp = donor(P[c], P[c + sz], w[c]);
        T fzm = donor(P[c - sz], P[c], w[c - sz]);
        out[c] = P[c] - ((fxp - fxm) + (fyp - fym) + (fzp - fzm)) / G[c];
      }
}

/* Antidiffusive pseudo-velocity on the faces c+1/2 of every interior cell
   (Smolarkiewicz 1984, G-weighted as in Smolarkiewicz & Margolin 1998):

     Ut = (|U| - U^2/Gf) A - U (Vbar By + Wbar Bz) / Gf,
     A  = (P_R - P_L) / (P_R + P_L + eps),
     By = 1/2 (P_R,j+1 + P_L,j+1 - P_R,j-1 - P_L,j-1)
              / (P_R,j+1 + P_L,j+1 + P_R,j-1 + P_L,j-1 + eps),
     Vbar = 1/4 (V at the four j-faces around the face),  Gf = (G_L + G_R)/2,

   and the same with the directions cycled for Vt and Wt.  Wt on the top
   face is zero. */
template <class T>
void pseudo_velocity(const Grid& g, const T* P, const T* u, const T* v, const T* w, const T* G,
                     T* ut, T* vt, T* wt) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  const T eps(EPS), half(0.5), quarter(0.25);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        {  // x face between c and c+X
          long L = c, R = c + X;
          T U = u[c];
          T Gf = half * (G[L] + G[R]);
          T A = (P[R] - P[L]) / (P[R] + P[L] + eps);
          T By = half * (P[R + Y] + P[L + Y] - P[R - Y] - P[L - Y]) /
                 (P[R + Y] + P[L + Y] + P[R - Y] + P[L - Y] + eps);
          T Bz = half * (P[R + Z] + P[L + Z] - P[R - Z] - P[L - Z]) /
                 (P[R + Z] + P[L + Z] + P[R - Z] + P[L - Z] + eps);
          T Vb = quarter * (v[L] + v[R] + v[L - Y] + v[R - Y]);
          T Wb = quarter * (w[L] + w[R] + w[L - Z] + w[R - Z]);
          ut[c] = (oabs(U) - U * U / Gf) * A - U * (Vb * By + Wb * Bz) / Gf;
        }
        {  // y face between c and c+Y
          long L = c, R = c + Y;
          T V = v[c];
          T Gf = half * (G[L] + G[R]);
          T A = (P[R] - P[L]) / (P[R] + P[L] + eps);
          T Bx = half * (P[R + X] + P[L + X] - P[R - X] - P[L - X]) /
                 (P[R + X] + P[L + X] + P[R - X] + P[L - X] + eps);
          T Bz = half * (P[R + Z] + P[L + Z] - P[R - Z] - P[L - Z]) /
                 (P[R + Z] + P[L + Z] + P[R - Z] + P[L - Z] + eps);
          T Ub = quarter * (u[L] + u[R] + u[L - X] + u[R - X]);
          T Wb = quarter * (w[L] + w[R] + w[L - Z] + w[R - Z]);
          vt[c] = (oabs(V) - V * V / Gf) * A - V * (Ub * Bx + Wb * Bz) / Gf;
        }
        if (g.zface(k)) {  // z face between c and c+Z (open faces only)
          long L = c, R = c + Z;
          T W = w[c];
          T Gf = half * (G[L] + G[R]);
          T A = (P[R] - P[L]) / (P[R] + P[L] + eps);
          T Bx = half * (P[R + X] + P[L + X] - P[R - X] - P[L - X]) /
                 (P[R + X] + P[L + X] + P[R - X] + P[L - X] + eps);
          T By = half * (P[R + Y] + P[L + Y] - P[R - Y] - P[L - Y]) /
                 (P[R + Y] + P[L + Y] + P[R - Y] + P[L - Y] + eps);
          T Ub = quarter * (u[L] + u[R] + u[L - X] + u[R - X]);
          T Vb = quarter * (v[L] + v[R] + v[L - Y] + v[R - Y]);
          wt[c] = (oabs(W) - W * W / Gf) * A - W * (Ub * Bx + Vb * By) / Gf;
        } else {
          wt[c] = T(0.0);
        }
      }
}

/* Infinite-gauge pseudo-fluxes (option IGA).  For psi + c the pseudo-velocity
   of a face behaves as 1/c and its donor flux tends, as c grows, to c times
   it; that limit replaces both the pseudo-velocity and its flux:
     Ft = (|U| - U^2/Gf) (P_R - P_L)/2 - U (Vbar Ny + Wbar Nz) / Gf,
     Ny = (P_R,j+1 + P_L,j+1 - P_R,j-1 - P_L,j-1)/8,
   i.e. c A -> (P_R - P_L)/2 and c B -> (numerator of B)/8, the denominators
   P_R + P_L + eps and the four-point sum + eps being 2c and 4c in the limit.
   Vbar, Wbar and Gf as in pseudo_velocity.  Ft on a closed top face is 0. */
template <class T>
void pseudo_flux_iga(const Grid& g, const T* P, const T* u, const T* v, const T* w, const T* G,
                     T* fu, T* fv, T* fw) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  const T half(0.5), quarter(0.25), eighth(0.125);
  // one face: right cell at c + d; cross directions e1, e2 with their face
  // Courant fields c1, c2
  auto face = [&](long c, long d, long e1, long e2, T C, const T* c1, const T* c2) {
    const long L = c, R = c + d;
    const T Gf = half * (G[L] + G[R]);
    const T dA = half * (P[R] - P[L]);
    const T n1 = eighth * (P[R + e1] + P[L + e1] - P[R - e1] - P[L - e1]);
    const T n2 = eighth * (P[R + e2] + P[L + e2] - P[R - e2] - P[L - e2]);
    const T m1 = quarter * (c1[L] + c1[R] + c1[L - e1] + c1[R - e1]);
    const T m2 = quarter * (c2[L] + c2[R] + c2[L - e2] + c2[R - e2]);
    return (oabs(C) - C * C / Gf) * dA - C * (m1 * n1 + m2 * n2) / Gf;
  };
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        fu[c] = face(c, X, Y, Z, u[c], v, w);
        fv[c] = face(c, Y, X, Z, v[c], u, w);
        fw[c] = g.zface(k) ? face(c, Z, X, Y, w[c], u, v) : T(0.0);
      }
}

/* Divergent-flow term (option DFL; Smolarkiewicz 1984).  In a divergent flow
   the donor-cell scheme's first-order error has a further part, which the
   pseudo-velocity cancels with -1/2 U (dt div v): with the divergence of the
   G-weighted Courant numbers of a cell,
     D_c = (U_c - U_c-X) + (V_c - V_c-Y) + (W_c - W_c-Z),
   averaged over the face's two cells and divided by the face's G,
     Ut += -(1/4) U (D_L + D_R) / Gf,
   and the same for Vt and Wt (the closed faces' W are 0 in the halo). */
template <class T>
void add_divergent_flow_term(const Grid& g, const T* u, const T* v, const T* w, const T* G,
                             T* ut, T* vt, T* wt) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  const T half(0.5), quarter(0.25);
  auto D = [&](long c) { return (u[c] - u[c - X]) + (v[c] - v[c - Y]) + (w[c] - w[c - Z]); };
  auto term = [&](long L, long R, T C) {
    return -quarter * C * (D(L) + D(R)) / (half * (G[L] + G[R]));
  };
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        ut[c] = ut[c] + term(c, c + X, u[c]);
        vt[c] = vt[c] + term(c, c + Y, v[c]);
        if (g.zface(k)) wt[c] = wt[c] + term(c, c + Z, w[c]);
      }
}

/* Flux divergence and advance with the face fluxes given (the infinite-gauge
   corrective pass, whose pseudo-fluxes are fluxes already):
   out = P - (1/G) sum_d [F_c+d/2 - F_c-d/2]. */
template <class T>
void advance_fluxes(const Grid& g, const T* P, const T* fu, const T* fv, const T* fw, const T* G,
                    T* out) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        out[c] = P[c] - ((fu[c] - fu[c - X]) + (fv[c] - fv[c - Y]) + (fw[c] - fw[c - Z])) / G[c];
      }
}

/* Non-oscillatory limiter (Smolarkiewicz & Grabowski 1990), G-weighted.
   Bounds over the 7-point stencil of both psi^n (P0) and psi^(m-1) (P);
   unlimited antidiffusive fluxes f = F(P_L, P_R, Ut); incoming and outgoing
   flux sums; beta-up = (max - P) G / (in + eps), beta-down =
   (P - min) G / (out + eps); output: betas (halo-filled) in bu, bd.  With
   `unit` (infinite gauge) the face values ut, vt, wt are the fluxes. */
template <class T>
void limiter_betas(const Grid& g, const T* P0, const T* P, const T* ut, const T* vt, const T* wt,
                   const T* G, T* mx, T* mn, T* bu, T* bd, bool unit = false) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  const T eps(EPS), zero(0.0);
  const long nb[6] = {-X, X, -Y, Y, -Z, Z};
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        T hi = P0[c], lo = P0[c];
        hi = omax(hi, P[c]);
        lo = omin(lo, P[c]);
        for (int q = 0; q < 6; ++q) {
          hi = omax(hi, P0[c + nb[q]]);
          hi = omax(hi, P[c + nb[q]]);
          lo = omin(lo, P0[c + nb[q]]);
          lo = omin(lo, P[c + nb[q]]);
        }
        mx[c] = hi;
        mn[c] = lo;
        // fluxes through the six faces: the "+" faces and the "-" faces
        auto fl = [&](T L, T R, T C) { return unit ? C : donor(L, R, C); };
        T fxp = fl(P[c], P[c + X], ut[c]);
        T fxm = fl(P[c - X], P[c], ut[c - X]);
        T fyp = fl(P[c], P[c + Y], vt[c]);
        T fym = fl(P[c - Y], P[c], vt[c - Y]);
        T fzp = fl(P[c], P[c + Z], wt[c]);
        T fzm = fl(P[c - Z], P[c], wt[c - Z]);
        T in = (omax(fxm, zero) - omin(fxp, zero)) + (omax(fym, zero) - omin(fyp, zero)) +
               (omax(fzm, zero) - omin(fzp, zero));
        T out = (omax(fxp, zero) - omin(fxm, zero)) + (omax(fyp, zero) - omin(fym, zero)) +
                (omax(fzp, zero) - omin(fzm, zero));
        bu[c] = (hi - P[c]) * G[c] / (in + eps);
        bd[c] = (P[c] - lo) * G[c] / (out + eps);
      }
  fill_halo_periodic(bu, g);
  fill_halo_periodic(bd, g);
}

/* Limited velocity on the face between L and R:
   min(1, bd_L, bu_R) max(Ut,0) + min(1, bu_L, bd_R) min(Ut,0). */
template <class T> inline T limit_face(T Ut, T buL, T bdL, T buR, T bdR) {
  const T one(1.0), zero(0.0);
  T cpos = omin(omin(one, bdL), buR);
  T cneg = omin(omin(one, buL), bdR);
  return cpos * omax(Ut, zero) + cneg * omin(Ut, zero);
}

/* With `sgn` (signed fields, P = psi^(m-1)) a face whose upwind value is
   negative carries its flux against its velocity: beta-up and beta-down
   trade places there, which limits the flux by its own direction. */
template <class T>
void limit_velocities(const Grid& g, const T* ut, const T* vt, const T* wt, const T* bu,
                      const T* bd, T* ul, T* vl, T* wl, const T* P = nullptr, bool sgn = false) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  auto lim = [&](T Ut, long L, long R) {
    const bool flip = sgn && val(val(Ut) >= 0.0 ? P[L] : P[R]) < 0.0;
    return flip ? limit_face(Ut, bd[L], bu[L], bd[R], bu[R])
                : limit_face(Ut, bu[L], bd[L], bu[R], bd[R]);
  };
#pragma omp parallel for schedule(static)
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        ul[c] = lim(ut[c], c, c + X);
        vl[c] = lim(vt[c], c, c + Y);
        wl[c] = g.zface(k) ? lim(wt[c], c, c + Z) : T(0.0);
      }
}

/* Intermediates of the last corrective pass, for staged comparisons. */
struct Stages {
  double *psi1, *ut, *vt, *wt, *mx, *mn, *bu, *bd, *ul, *vl, *wl;
};

template <class T> void copy_out(double* dst, const std::vector<T>& src) {
  if (!dst) return;
  for (size_t q = 0; q < src.size(); ++q) dst[q] = val(src[q]);
}

/* One MPDATA step.  Inputs are read at their interior points only. */
template <class T>
void mpdata_step(const Grid& g, int iord, int nonosc, const T* psi_in, const T* Uin,
                 const T* Vin, const T* Win, const T* Gin, T* psi_out, const Stages* st,
                 Opts o = Opts()) {
  const long n = g.size();
  std::vector<T> P0(n), P(n), Pn(n), U(n), V(n), W(n), G(n), Pa(o.abs ? n : 0);
  std::vector<T> ut(n), vt(n), wt(n), ul(n), vl(n), wl(n), mx(n), mn(n), bu(n), bd(n);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        P0[c] = psi_in[c]; U[c] = Uin[c]; V[c] = Vin[c]; W[c] = Win[c]; G[c] = Gin[c];
      }
  // 1. halos and the zero-flux vertical boundary
  fill_halo_periodic(P0.data(), g);
  fill_halo_periodic(U.data(), g);
  fill_halo_periodic(V.data(), g);
  fill_halo_periodic(G.data(), g);
  fill_halo_wface(W.data(), g);
  // 2. donor-cell pass
  advance(g, P0.data(), U.data(), V.data(), W.data(), G.data(), P.data());
  fill_halo_periodic(P.data(), g);
  if (st) copy_out(st->psi1, P);
  // 3. corrective passes
  const T *cu = U.data(), *cv = V.data(), *cw = W.data();
  for (int m = 2; m <= iord; ++m) {
    if (o.iga) {
      pseudo_flux_iga(g, P.data(), cu, cv, cw, G.data(), ut.data(), vt.data(), wt.data());
    } else if (o.abs) {  // A and B of |psi^(m-1)|
      for (long q = 0; q < n; ++q) Pa[q] = oabs(P[q]);
      pseudo_velocity(g, Pa.data(), cu, cv, cw, G.data(), ut.data(), vt.data(), wt.data());
    } else {
      pseudo_velocity(g, P.data(), cu, cv, cw, G.data(), ut.data(), vt.data(), wt.data());
    }
    if (o.dfl) add_divergent_flow_term(g, cu, cv, cw, G.data(), ut.data(), vt.data(), wt.data());
    fill_halo_periodic(ut.data(), g);
    fill_halo_periodic(vt.data(), g);
    fill_halo_wface(wt.data(), g);
    if (nonosc) {
      limiter_betas(g, P0.data(), P.data(), ut.data(), vt.data(), wt.data(), G.data(), mx.data(),
                    mn.data(), bu.data(), bd.data(), o.iga);
      limit_velocities(g, ut.data(), vt.data(), wt.data(), bu.data(), bd.data(), ul.data(),
                       vl.data(), wl.data(), P.data(), o.abs && !o.iga);
    } else {
      std::copy(ut.begin(), ut.end(), ul.begin());
      std::copy(vt.begin(), vt.end(), vl.begin());
      std::copy(wt.begin(), wt.end(), wl.begin());
    }
    fill_halo_periodic(ul.data(), g);
    fill_halo_periodic(vl.data(), g);
    fill_halo_wface(wl.data(), g);
    if (o.iga)
      advance_fluxes(g, P.data(), ul.data(), vl.data(), wl.data(), G.data(), Pn.data());
    else
      advance(g, P.data(), ul.data(), vl.data(), wl.data(), G.data(), Pn.data());
    fill_halo_periodic(Pn.data(), g);
    if (st && m == iord) {
      copy_out(st->ut, ut); copy_out(st->vt, vt); copy_out(st->wt, wt);
      copy_out(st->mx, mx); copy_out(st->mn, mn); copy_out(st->bu, bu); copy_out(st->bd, bd);
      copy_out(st->ul, ul); copy_out(st->vl, vl); copy_out(st->wl, wl);
    }
    P.swap(Pn);
    // the next pass (iord >= 3) takes the limited velocities of this one
    cu = ul.data(); cv = vl.data(); cw = wl.data();
  }
  for (long q = 0; q < n; ++q) psi_out[q] = P[q];
}


/* ========================================================= adjoint (reverse) */

/* Reverse of fill_halo_periodic: every halo value was a copy of an interior
   (or, in k, an edge-plane) value, so its adjoint is added to that source
   and cleared; done in the reverse order of the forward fill. */
void rev_halo_periodic(double* a, const Grid& g) {
  for (int k = -g.h; k < g.nz + g.h; ++k) {
    if (k >= 0 && k < g.nz) continue;
    int ks = g.kper ? wrap(k, g.nz) : (k < 0 ? 0 : g.nz - 1);
    for (int j = -g.h; j < g.ny + g.h; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i) {
        a[g.at(i, j, ks)] += a[g.at(i, j, k)];
        a[g.at(i, j, k)] = 0.0;
      }
  }
  for (int k = 0; k < g.nz; ++k) {
    for (int j = -g.h; j < g.ny + g.h; ++j)
      if (j < 0 || j >= g.ny)
        for (int i = -g.h; i < g.nx + g.h; ++i) {
          a[g.at(i, wrap(j, g.ny), k)] += a[g.at(i, j, k)];
          a[g.at(i, j, k)] = 0.0;
        }
    for (int j = 0; j < g.ny; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i)
        if (i < 0 || i >= g.nx) {
          a[g.at(wrap(i, g.nx), j, k)] += a[g.at(i, j, k)];
          a[g.at(i, j, k)] = 0.0;
        }
  }
}

/* Reverse of fill_halo_wface: the closed faces were overwritten with zero,
   so their adjoints are dropped; the rest is the periodic reverse. */
void rev_halo_wface(double* a, const Grid& g) {
  for (int k = -g.h; k < g.nz + g.h && !g.kper; ++k) {
    if (k >= 0 && k < g.nz - 1) continue;
    for (int j = -g.h; j < g.ny + g.h; ++j)
      for (int i = -g.h; i < g.nx + g.h; ++i) a[g.at(i, j, k)] = 0.0;
  }
  rev_halo_periodic(a, g);
}

/* Reverse of F(L,R,C) = max(C,0) L + min(C,0) R with adjoint fb: the branch
   rules of omax/omin (a tie at C = 0 takes C on both sides). */
inline void rev_donor(double fb, double L, double R, double C, double* Lb, double* Rb,
                      double* Cb) {
  *Lb += fb * (C >= 0 ? C : 0.0);
  *Rb += fb * (C <= 0 ? C : 0.0);
  *Cb += fb * ((C >= 0 ? L : 0.0) + (C <= 0 ? R : 0.0));
}

/* Reverse of advance: out = P - (1/G) sum_d [F_+ - F_-], for the adjoint
   ob of out at the interior points; accumulates into Pb and the velocity
   adjoints (padded arrays, halo entries included). */
void rev_advance(const Grid& g, const double* P, const double* u, const double* v,
                 const double* w, const double* G, const double* ob, double* Pb, double* ub,
                 double* vb, double* wb) {
  const long D[3] = {1, g.px, g.px * g.py};
  const double* vel[3] = {u, v, w};
  double* velb[3] = {ub, vb, wb};
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        double a = ob[c];
        Pb[c] += a;
        double s = -a / G[c];
        for (int d = 0; d < 3; ++d) {
          rev_donor(s, P[c], P[c + D[d]], vel[d][c], &Pb[c], &Pb[c + D[d]], &velb[d][c]);
          rev_donor(-s, P[c - D[d]], P[c], vel[d][c - D[d]], &Pb[c - D[d]], &Pb[c],
                    &velb[d][c - D[d]]);
        }
      }
}

/* Reverse of the pseudo-velocity of one face.  L, R: the two cells;
   Y1/Y2: the strides of the two cross directions; cv1, cv2 the Courant
   fields of those directions, with their own "minus" strides M1, M2 (the
   cross averages take the faces at L, R, L-M, R-M). */
inline void rev_face_pseudo(double ub, const double* P, long L, long R, long Y1, long Y2,
                            double U, double Gf, const double* c1, const double* c2, long M1,
                            long M2, double* Pb, double* Ub, double* c1b, double* c2b) {
  const double eps = EPS;
  double n = P[R] - P[L], d = P[R] + P[L] + eps, A = n / d;
  double n1 = 0.5 * (P[R + Y1] + P[L + Y1] - P[R - Y1] - P[L - Y1]);
  double d1 = P[R + Y1] + P[L + Y1] + P[R - Y1] + P[L - Y1] + eps;
  double B1 = n1 / d1;
  double n2 = 0.5 * (P[R + Y2] + P[L + Y2] - P[R - Y2] - P[L - Y2]);
  double d2 = P[R + Y2] + P[L + Y2] + P[R - Y2] + P[L - Y2] + eps;
  double B2 = n2 / d2;
  double C1 = 0.25 * (c1[L] + c1[R] + c1[L - M1] + c1[R - M1]);
  double C2 = 0.25 * (c2[L] + c2[R] + c2[L - M2] + c2[R - M2]);
  double Dd = oabs(U) - U * U / Gf;
  double X = C1 * B1 + C2 * B2;
  double sg = U > 0 ? 1.0 : (U < 0 ? -1.0 : 0.0);
  *Ub += ub * (sg * A - 2.0 * U / Gf * A - X / Gf);
  double Ab = ub * Dd;
  double B1b = ub * (-U * C1 / Gf), B2b = ub * (-U * C2 / Gf);
  double C1b = ub * (-U * B1 / Gf), C2b = ub * (-U * B2 / Gf);
  Pb[R] += Ab * (1.0 - A) / d;
  Pb[L] += Ab * (-1.0 - A) / d;
  double wp = B1b * (0.5 - B1) / d1, wm = B1b * (-0.5 - B1) / d1;
  Pb[R + Y1] += wp; Pb[L + Y1] += wp; Pb[R - Y1] += wm; Pb[L - Y1] += wm;
  wp = B2b * (0.5 - B2) / d2; wm = B2b * (-0.5 - B2) / d2;
  Pb[R + Y2] += wp; Pb[L + Y2] += wp; Pb[R - Y2] += wm; Pb[L - Y2] += wm;
  c1b[L] += 0.25 * C1b; c1b[R] += 0.25 * C1b; c1b[L - M1] += 0.25 * C1b; c1b[R - M1] += 0.25 * C1b;
  c2b[L] += 0.25 * C2b; c2b[R] += 0.25 * C2b; c2b[L - M2] += 0.25 * C2b; c2b[R - M2] += 0.25 * C2b;
}

void rev_pseudo(const Grid& g, const double* P, const double* u, const double* v, const double* w,
                const double* G, const double* utb, const double* vtb, const double* wtb,
                double* Pb, double* ub, double* vb, double* wb) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        rev_face_pseudo(utb[c], P, c, c + X, Y, Z, u[c], 0.5 * (G[c] + G[c + X]), v, w, Y, Z,
                        Pb, &ub[c], vb, wb);
        rev_face_pseudo(vtb[c], P, c, c + Y, X, Z, v[c], 0.5 * (G[c] + G[c + Y]), u, w, X, Z,
                        Pb, &vb[c], ub, wb);
        if (g.zface(k))
          rev_face_pseudo(wtb[c], P, c, c + Z, X, Y, w[c], 0.5 * (G[c] + G[c + Z]), u, v, X, Y,
                          Pb, &wb[c], ub, vb);
      }
}

/* Reverse of limit_face: routes the adjoint of the limited velocity to Ut and
   to the betas that won the two min(1, ., .) folds (tie: the earlier one). */
inline void rev_limit_face(double lb, double Ut, double buL, double bdL, double buR, double bdR,
                           double* Utb, double* buLb, double* bdLb, double* buRb, double* bdRb) {
  double m1 = (1.0 <= bdL) ? 1.0 : bdL;
  bool p_is_bdL = !(1.0 <= bdL);
  double cpos = (m1 <= buR) ? m1 : buR;
  bool p_first = (m1 <= buR);
  double n1 = (1.0 <= buL) ? 1.0 : buL;
  bool n_is_buL = !(1.0 <= buL);
  double cneg = (n1 <= bdR) ? n1 : bdR;
  bool n_first = (n1 <= bdR);
  *Utb += lb * ((Ut >= 0 ? cpos : 0.0) + (Ut <= 0 ? cneg : 0.0));
  double cpb = lb * (Ut >= 0 ? Ut : 0.0), cnb = lb * (Ut <= 0 ? Ut : 0.0);
  if (p_first) { if (p_is_bdL) *bdLb += cpb; } else { *buRb += cpb; }
  if (n_first) { if (n_is_buL) *buLb += cnb; } else { *bdRb += cnb; }
}

void rev_limit(const Grid& g, const double* ut, const double* vt, const double* wt,
               const double* bu, const double* bd, const double* ulb, const double* vlb,
               const double* wlb, double* utb, double* vtb, double* wtb, double* bub,
               double* bdb) {
  const long D[3] = {1, g.px, g.px * g.py};
  const double* vt3[3] = {ut, vt, wt};
  const double* lb3[3] = {ulb, vlb, wlb};
  double* tb3[3] = {utb, vtb, wtb};
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        for (int d = 0; d < 3; ++d) {
          if (d == 2 && !g.zface(k)) continue;  // closed top face: constant
          long r = c + D[d];
          rev_limit_face(lb3[d][c], vt3[d][c], bu[c], bd[c], bu[r], bd[r], &tb3[d][c], &bub[c],
                         &bdb[c], &bub[r], &bdb[r]);
        }
      }
}

/* Reverse of limiter_betas for the adjoints bub, bdb of the betas. */
void rev_beta(const Grid& g, const double* P0, const double* P, const double* ut,
              const double* vt, const double* wt, const double* G, const double* bub,
              const double* bdb, double* P0b, double* Pb, double* utb, double* vtb, double* wtb) {
  const long X = 1, Y = g.px, Z = g.px * g.py;
  const long nb[6] = {-X, X, -Y, Y, -Z, Z};
  const long D[3] = {X, Y, Z};
  const double* vt3[3] = {ut, vt, wt};
  double* tb3[3] = {utb, vtb, wtb};
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        // bounds, remembering which element won each fold (same order as forward)
        double hi = P0[c], lo = P0[c];
        double* hip = &P0b[c];
        double* lop = &P0b[c];
        if (!(hi >= P[c])) { hi = P[c]; hip = &Pb[c]; }
        if (!(lo <= P[c])) { lo = P[c]; lop = &Pb[c]; }
        for (int q = 0; q < 6; ++q) {
          long n = c + nb[q];
          if (!(hi >= P0[n])) { hi = P0[n]; hip = &P0b[n]; }
          if (!(hi >= P[n])) { hi = P[n]; hip = &Pb[n]; }
          if (!(lo <= P0[n])) { lo = P0[n]; lop = &P0b[n]; }
          if (!(lo <= P[n])) { lo = P[n]; lop = &Pb[n]; }
        }
        double fp[3], fm[3];
        for (int d = 0; d < 3; ++d) {
          fp[d] = donor(P[c], P[c + D[d]], vt3[d][c]);
          fm[d] = donor(P[c - D[d]], P[c], vt3[d][c - D[d]]);
        }
        double in = (omax(fm[0], 0.0) - omin(fp[0], 0.0)) + (omax(fm[1], 0.0) - omin(fp[1], 0.0)) +
                    (omax(fm[2], 0.0) - omin(fp[2], 0.0));
        double out = (omax(fp[0], 0.0) - omin(fm[0], 0.0)) + (omax(fp[1], 0.0) - omin(fm[1], 0.0)) +
                     (omax(fp[2], 0.0) - omin(fm[2], 0.0));
        double din = in + EPS, dout = out + EPS;
        double bu = (hi - P[c]) * G[c] / din, bd = (P[c] - lo) * G[c] / dout;
        double ab = bub[c], db = bdb[c];
        *hip += ab * G[c] / din;
        Pb[c] -= ab * G[c] / din;
        double inb = -ab * bu / din;
        Pb[c] += db * G[c] / dout;
        *lop -= db * G[c] / dout;
        double outb = -db * bd / dout;
        for (int d = 0; d < 3; ++d) {
          // top/bottom closed faces carry constant zero fluxes
          bool has_p = !(d == 2 && !g.zface(k)), has_m = !(d == 2 && !g.kper && k == 0);
          double fpb = -inb * (fp[d] <= 0 ? 1.0 : 0.0) + outb * (fp[d] >= 0 ? 1.0 : 0.0);
          double fmb = inb * (fm[d] >= 0 ? 1.0 : 0.0) - outb * (fm[d] <= 0 ? 1.0 : 0.0);
          if (has_p) rev_donor(fpb, P[c], P[c + D[d]], vt3[d][c], &Pb[c], &Pb[c + D[d]], &tb3[d][c]);
          if (has_m)
            rev_donor(fmb, P[c - D[d]], P[c], vt3[d][c - D[d]], &Pb[c - D[d]], &Pb[c],
                      &tb3[d][c - D[d]]);
        }
      }
}

/* One adjoint step: psib holds the adjoint of psi^(n+1) at interior points
   on entry and that of psi^n on exit; ubar, vbar, wbar are incremented. */
void adjoint_step(const Grid& g, int iord, int nonosc, const double* psi_in, const double* Uin,
                  const double* Vin, const double* Win, const double* Gin, double* psib,
                  double* ubar, double* vbar, double* wbar) {
  const long n = g.size();
  // forward, keeping the input state and the intermediates of every
  // corrective pass m = 2..iord (pass m at index m-2)
  std::vector<double> P0(n), U(n), V(n), W(n), G(n);
  for (long q = 0; q < n; ++q) { P0[q] = psi_in[q]; U[q] = Uin[q]; V[q] = Vin[q]; W[q] = Win[q]; G[q] = Gin[q]; }
  fill_halo_periodic(P0.data(), g);
  fill_halo_periodic(U.data(), g);
  fill_halo_periodic(V.data(), g);
  fill_halo_periodic(G.data(), g);
  fill_halo_wface(W.data(), g);
  struct Pass {
    std::vector<double> P, ut, vt, wt, bu, bd, ul, vl, wl;  // P: the pass's input state
  };
  std::vector<Pass> pass(iord >= 2 ? iord - 1 : 0);
  std::vector<double> cur(n), nxt(n);
  advance(g, P0.data(), U.data(), V.data(), W.data(), G.data(), cur.data());
  fill_halo_periodic(cur.data(), g);
  const double *cu = U.data(), *cv = V.data(), *cw = W.data();
  for (int m = 2; m <= iord; ++m) {
    Pass& p = pass[m - 2];
    p.P = cur;
    for (auto* f : {&p.ut, &p.vt, &p.wt, &p.bu, &p.bd, &p.ul, &p.vl, &p.wl}) f->assign(n, 0.0);
    pseudo_velocity(g, p.P.data(), cu, cv, cw, G.data(), p.ut.data(), p.vt.data(), p.wt.data());
    fill_halo_periodic(p.ut.data(), g);
    fill_halo_periodic(p.vt.data(), g);
    fill_halo_wface(p.wt.data(), g);
    if (nonosc) {
      std::vector<double> mx(n), mn(n);
      limiter_betas(g, P0.data(), p.P.data(), p.ut.data(), p.vt.data(), p.wt.data(), G.data(),
                    mx.data(), mn.data(), p.bu.data(), p.bd.data());
      limit_velocities(g, p.ut.data(), p.vt.data(), p.wt.data(), p.bu.data(), p.bd.data(),
                       p.ul.data(), p.vl.data(), p.wl.data());
    } else {
      p.ul = p.ut;
      p.vl = p.vt;
      p.wl = p.wt;
    }
    fill_halo_periodic(p.ul.data(), g);
    fill_halo_periodic(p.vl.data(), g);
    fill_halo_wface(p.wl.data(), g);
    advance(g, p.P.data(), p.ul.data(), p.vl.data(), p.wl.data(), G.data(), nxt.data());
    fill_halo_periodic(nxt.data(), g);
    cur.swap(nxt);
    cu = p.ul.data(); cv = p.vl.data(); cw = p.wl.data();
  }

  // reverse, pass by pass from the last; ob is the adjoint of the pass's
  // output state, carry that of its limited velocities coming from the pass
  // above (whose input velocities they were)
  std::vector<double> P0b(n, 0.0), Ub(n, 0.0), Vb(n, 0.0), Wb(n, 0.0);
  std::vector<double> ob(n, 0.0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) ob[g.at(i, j, k)] = psib[g.at(i, j, k)];
  std::vector<double> cuu(n, 0.0), cvv(n, 0.0), cww(n, 0.0);  // the carry
  for (int m = iord; m >= 2; --m) {
    Pass& p = pass[m - 2];
    std::vector<double> Pb(n, 0.0);
    std::vector<double> ulb = cuu, vlb = cvv, wlb = cww;
    rev_advance(g, p.P.data(), p.ul.data(), p.vl.data(), p.wl.data(), G.data(), ob.data(),
                Pb.data(), ulb.data(), vlb.data(), wlb.data());
    rev_halo_periodic(ulb.data(), g);
    rev_halo_periodic(vlb.data(), g);
    rev_halo_wface(wlb.data(), g);
    std::vector<double> utb(n, 0.0), vtb(n, 0.0), wtb(n, 0.0);
    if (nonosc) {
      std::vector<double> bub(n, 0.0), bdb(n, 0.0);
      rev_limit(g, p.ut.data(), p.vt.data(), p.wt.data(), p.bu.data(), p.bd.data(), ulb.data(),
                vlb.data(), wlb.data(), utb.data(), vtb.data(), wtb.data(), bub.data(),
                bdb.data());
      rev_halo_periodic(bub.data(), g);
      rev_halo_periodic(bdb.data(), g);
      rev_beta(g, P0.data(), p.P.data(), p.ut.data(), p.vt.data(), p.wt.data(), G.data(),
               bub.data(), bdb.data(), P0b.data(), Pb.data(), utb.data(), vtb.data(),
               wtb.data());
      rev_halo_periodic(utb.data(), g);
      rev_halo_periodic(vtb.data(), g);
      rev_halo_wface(wtb.data(), g);
    } else {
      utb = ulb;
      vtb = vlb;
      wtb = wlb;
    }
    // the pass's input velocities: U, V, W for the first corrective pass,
    // else the limited velocities of the pass below
    const bool first = m == 2;
    const Pass* below = first ? nullptr : &pass[m - 3];
    std::vector<double> tu(n, 0.0), tv(n, 0.0), tw(n, 0.0);
    rev_pseudo(g, p.P.data(), first ? U.data() : below->ul.data(),
               first ? V.data() : below->vl.data(), first ? W.data() : below->wl.data(),
               G.data(), utb.data(), vtb.data(), wtb.data(), Pb.data(),
               first ? Ub.data() : tu.data(), first ? Vb.data() : tv.data(),
               first ? Wb.data() : tw.data());
    if (!first) {
      rev_halo_periodic(tu.data(), g);
      rev_halo_periodic(tv.data(), g);
      rev_halo_wface(tw.data(), g);
      cuu.swap(tu); cvv.swap(tv); cww.swap(tw);
    }
    rev_halo_periodic(Pb.data(), g);  // the pass's input state had its halo filled
    ob.swap(Pb);
  }
  rev_advance(g, P0.data(), U.data(), V.data(), W.data(), G.data(), ob.data(), P0b.data(),
              Ub.data(), Vb.data(), Wb.data());
  rev_halo_periodic(P0b.data(), g);
  rev_halo_periodic(Ub.data(), g);
  rev_halo_periodic(Vb.data(), g);
  rev_halo_wface(Wb.data(), g);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        long c = g.at(i, j, k);
        psib[c] = P0b[c];
        ubar[c] += Ub[c];
        vbar[c] += Vb[c];
        wbar[c] += Wb[c];
      }
}

/* ============================================ edge-based flux stages (Sec. 5)

   The subset of MPDATA that Listings 5, 7, 8 and 9 show, on a mesh given by
   connectivity tables (indirect addressing):
     1. upwind flux on every edge e and level k (Listings 4/5):
          flux = max(0, vn) pD(first node) + min(0, vn) pD(second node);
     2. upwind flux through the vertical faces of every node (Listing 7):
          face k (1 <= k <= nz-1, between levels k-1 and k)
          fluz_k = max(0, W_k) pD_{k-1} + min(0, W_k) pD_k,
          and the boundary faces fluz_0 = pivbz fluz_1, fluz_nz = pivbz fluz_{nz-1};
     3. flux divergence over the node's dual cell (compute_fluxdiv, Listing 8):
          divVD = (sum_j sign_j flux(edge_j) + fluz_{k+1} - fluz_k) / vol;
     4. advance (advance_solution, Listing 8): pD = pD - divVD / rho.
   The paper names steps 3 and 4 without their bodies; these are the plain
   finite-volume divergence (sign +1 where the node is the edge's first node,
   the edge's flux leaving it) and the density-weighted update.
   Fields are level-major: node field [k][n], edge field [k][e], vertical
   faces [k][n] for k = 0..nz. */

struct EdgeMesh {
  long N, E;
  int nz;
  const long* e2n;     // [E][2]
  const long* n2e;     // [N][6]
  const double* sgn;   // [N][6]
};

void edge_upwind_flux(const EdgeMesh& m, const double* pD, const double* vn, double* flux) {
#pragma omp parallel for schedule(static)
  for (long e = 0; e < m.E; ++e) {
    const long ip1 = m.e2n[2 * e], ip2 = m.e2n[2 * e + 1];
    for (int k = 0; k < m.nz; ++k) {
      const double v = vn[k * m.E + e];
      const double zpos = std::max(0.0, v), zneg = std::min(0.0, v);
      flux[k * m.E + e] = pD[k * m.N + ip1] * zpos + pD[k * m.N + ip2] * zneg;
    }
  }
}

void edge_upwind_fluz(const EdgeMesh& m, const double* pD, const double* W, double pivbz,
                      double* fluz) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < m.N; ++n) {
    for (int k = 1; k < m.nz; ++k) {
      const double w = W[k * m.N + n];
      fluz[k * m.N + n] = std::max(0.0, w) * pD[(k - 1) * m.N + n] +
                          std::min(0.0, w) * pD[k * m.N + n];
    }
    fluz[n] = pivbz * fluz[m.N + n];
    fluz[m.nz * m.N + n] = pivbz * fluz[(m.nz - 1) * m.N + n];
  }
}

void edge_fluxdiv(const EdgeMesh& m, const double* flux, const double* fluz, const double* vol,
                  double* div) {
#pragma omp parallel for schedule(static)
  for (long n = 0; n < m.N; ++n)
    for (int k = 0; k < m.nz; ++k) {
      double s = 0.0;
      for (int j = 0; j < 6; ++j) s += m.sgn[6 * n + j] * flux[k * m.E + m.n2e[6 * n + j]];
      s += fluz[(k + 1) * m.N + n] - fluz[k * m.N + n];
      div[k * m.N + n] = s / vol[n];
    }
}

void edge_advance(const EdgeMesh& m, double* pD, const double* div, const double* rho) {
#pragma omp parallel for schedule(static)
  for (long q = 0; q < m.N * m.nz; ++q) pD[q] = pD[q] - div[q] / rho[q];
}

}  // namespace

/* =============================================================== C ABI */

extern "C" {

int orc_version() { return 1; }

/* Every entry point takes the vertical boundary kbc: 0 zero-flux (closed
   top and bottom faces, k halo an edge copy), 1 periodic in k.
   Halo fill.  kind 0: cell/horizontal-face field (periodic i-j, k copy);
   kind 1: vertical-face field (periodic i-j, zero boundary faces). */
void orc_fill_halo(int nx, int ny, int nz, int h, int kbc, int kind, double* f) {
  Grid g(nx, ny, nz, h, kbc);
  if (kind == 1) fill_halo_wface(f, g); else fill_halo_periodic(f, g);
}

/* nsteps MPDATA steps; psi_out gets the padded result with its halo filled.
   The optional stage pointers (may be null) receive the intermediates of the
   last corrective pass of the last step.  opts: the option flags (DFL 1,
   ABS 2, IGA 4). */
void orc_run(int nx, int ny, int nz, int h, int kbc, int iord, int nonosc, int opts, int nsteps,
             const double* psi_in, const double* U, const double* V, const double* W,
             const double* G, double* psi_out, double* psi1, double* ut, double* vt, double* wt,
             double* mx, double* mn, double* bu, double* bd, double* ul, double* vl, double* wl) {
  Grid g(nx, ny, nz, h, kbc);
  Stages st{psi1, ut, vt, wt, mx, mn, bu, bd, ul, vl, wl};
  std::vector<double> cur(psi_in, psi_in + g.size()), nxt(g.size());
  for (int s = 0; s < nsteps; ++s) {
    mpdata_step<double>(g, iord, nonosc, cur.data(), U, V, W, G, nxt.data(),
                        s == nsteps - 1 ? &st : nullptr, Opts(opts));
    cur.swap(nxt);
  }
  std::memcpy(psi_out, cur.data(), sizeof(double) * g.size());
}

/* Pseudo-velocities of a given field P with Courant fields U, V, W. */
void orc_pseudo_velocity(int nx, int ny, int nz, int h, int kbc, const double* Pin, const double* Uin,
                         const double* Vin, const double* Win, const double* Gin, double* ut,
                         double* vt, double* wt) {
  Grid g(nx, ny, nz, h, kbc);
  long n = g.size();
  std::vector<double> P(Pin, Pin + n), U(Uin, Uin + n), V(Vin, Vin + n), W(Win, Win + n),
      G(Gin, Gin + n);
  fill_halo_periodic(P.data(), g);
  fill_halo_periodic(U.data(), g);
  fill_halo_periodic(V.data(), g);
  fill_halo_periodic(G.data(), g);
  fill_halo_wface(W.data(), g);
  pseudo_velocity(g, P.data(), U.data(), V.data(), W.data(), G.data(), ut, vt, wt);
}

/* Mass sum_interior psi * G, summed in (k, j, i) order. */
double orc_mass(int nx, int ny, int nz, int h, const double* psi, const double* G) {
  Grid g(nx, ny, nz, h);
  double s = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) s += psi[g.at(i, j, k)] * G[g.at(i, j, k)];
  return s;
}

/* Tangent-linear model of nsteps steps (dual numbers through the forward
   code): returns psi_out and its directional derivative dpsi_out along
   (dpsi, dU, dV, dW).  G is held fixed. */
void orc_tlm(int nx, int ny, int nz, int h, int kbc, int iord, int nonosc, int nsteps, const double* psi,
             const double* U, const double* V, const double* W, const double* G,
             const double* dpsi, const double* dU, const double* dV, const double* dW,
             double* psi_out, double* dpsi_out) {
  Grid g(nx, ny, nz, h, kbc);
  long n = g.size();
  std::vector<Dual> p(n), u(n), v(n), w(n), gg(n), o(n);
  for (long q = 0; q < n; ++q) {
    p[q] = Dual(psi[q], dpsi[q]);
    u[q] = Dual(U[q], dU[q]);
    v[q] = Dual(V[q], dV[q]);
    w[q] = Dual(W[q], dW[q]);
    gg[q] = Dual(G[q], 0.0);
  }
  for (int s = 0; s < nsteps; ++s) {
    mpdata_step<Dual>(g, iord, nonosc, p.data(), u.data(), v.data(), w.data(), gg.data(),
                      o.data(), nullptr);
    p.swap(o);
  }
  for (long q = 0; q < n; ++q) { psi_out[q] = p[q].v; dpsi_out[q] = p[q].d; }
}

/* Adjoint of nsteps steps (iord 1 or 2): psib holds dJ/dpsi at step nsteps
   (interior) on entry and dJ/dpsi at step 0 on exit; ubar, vbar, wbar are
   incremented by dJ/dU, dJ/dV, dJ/dW.  The forward states are recomputed
   from psi (all stored; the oracle is for small grids).  G is held fixed. */
void orc_adjoint(int nx, int ny, int nz, int h, int kbc, int iord, int nonosc, int nsteps,
                 const double* psi, const double* U, const double* V, const double* W,
                 const double* G, double* psib, double* ubar, double* vbar, double* wbar) {
  Grid g(nx, ny, nz, h, kbc);
  long n = g.size();
  std::vector<std::vector<double>> states(nsteps > 0 ? nsteps : 1, std::vector<double>(n));
  std::vector<double> cur(psi, psi + n);
  for (int s = 0; s < nsteps; ++s) {
    states[s] = cur;
    std::vector<double> nxt(n);
    mpdata_step<double>(g, iord, nonosc, cur.data(), U, V, W, G, nxt.data(), nullptr);
    cur.swap(nxt);
  }
  for (int s = nsteps - 1; s >= 0; --s)
    adjoint_step(g, iord, nonosc, states[s].data(), U, V, W, G, psib, ubar, vbar, wbar);
}

/* nsteps applications of the edge-based flux stages (Listings 5, 7, 8):
   pD (level-major [nz][N]) is advanced in place.  W has nz+1 faces; its
   faces 0 and nz are never read. */
void orc_edge_run(long N, long E, int nz, int nsteps, const long* e2n, const long* n2e,
                  const double* sgn, const double* vn, const double* W, const double* rho,
                  const double* vol, double pivbz, double* pD) {
  EdgeMesh m{N, E, nz, e2n, n2e, sgn};
  std::vector<double> flux(E * nz), fluz(N * (nz + 1)), div(N * nz);
  for (int s = 0; s < nsteps; ++s) {
    edge_upwind_flux(m, pD, vn, flux.data());
    edge_upwind_fluz(m, pD, W, pivbz, fluz.data());
    edge_fluxdiv(m, flux.data(), fluz.data(), vol, div.data());
    edge_advance(m, pD, div.data(), rho);
  }
}

/* The cell-neighbour reduction of Table 1 (the on_cells operation of
   Fig. 5): for every cell s and level k, B = fac * (A at its three
   neighbours, summed in table order).  t: neighbour table [3][ncells]
   (any numbering); A, B: [nz][ncells]. */
void orc_cells_sum(long ncells, int nz, const int* t, const double* A, double fac, double* B) {
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (long s = 0; s < ncells; ++s) {
      const double* a = A + k * ncells;
      B[k * ncells + s] = (a[t[s]] + a[t[ncells + s]] + a[t[2 * ncells + s]]) * fac;
    }
}

}  // extern "C"
