// grid.cuh -- index geometry of the halo-padded fields and the boundary rules.
//
// Every field is [nz+2h][ny+2h][nx+2h], i fastest.  The step kernels never
// read a halo: periodic neighbours in i and j are taken by wrapping the
// interior index; in k (zero-flux boundary) the neighbours of psi by
// clamping (edge copy) and the vertical faces k = -1/2 and k = nz-1/2 are
// closed (the boundary factor pivbz = 0 of Listing 7), or (periodic k) by
// wrapping with every face open.  What the caller leaves in the halos never
// matters.
#pragma once
#include <cstdint>

namespace mpd {

struct Geo {
  int nx, ny, nz, h;
  int kper;      // 1: periodic in k; 0: closed (zero-flux) bottom and top faces
  int openij;    // 1: the grid is one slab of a decomposed domain: i-j neighbours
                 //    past the interior are read from the halo (filled by the
                 //    halo exchange) and no periodic images are written;
                 // 0: periodic in i and j (the whole domain)
  int64_t px;    // padded row length (elements)
  int64_t pxy;   // padded plane size (elements)
  int64_t off0;  // offset of interior point (0,0,0)
  int64_t total; // padded field size (elements)
};

inline Geo make_geo(int nx, int ny, int nz, int h, int kper = 0) {
  Geo g;
  g.nx = nx; g.ny = ny; g.nz = nz; g.h = h; g.kper = kper; g.openij = 0;
  g.px = nx + 2 * (int64_t)h;
  g.pxy = g.px * (ny + 2 * (int64_t)h);
  g.off0 = h * g.pxy + h * g.px + h;
  g.total = g.pxy * (nz + 2 * (int64_t)h);
  return g;
}

__host__ __device__ __forceinline__ int64_t at(const Geo& g, int i, int j, int k) {
  return g.off0 + (int64_t)k * g.pxy + (int64_t)j * g.px + i;
}
__device__ __forceinline__ int wrap_up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
__device__ __forceinline__ int wrap_dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }
__device__ __forceinline__ int clampk(int k, int nz) { return k < 0 ? 0 : (k >= nz ? nz - 1 : k); }
// The level of a vertical neighbour k (-1 <= k <= nz): wrapped when k is
// periodic, else clamped (the edge copy of psi).
__device__ __forceinline__ int kadj(const Geo& g, int k) {
  if (g.kper) return k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
  return k < 0 ? 0 : (k >= g.nz ? g.nz - 1 : k);
}
// Whether the vertical face above level k (k = -1: the bottom face) carries
// flux: all do when k is periodic, else the bottom and top faces are closed.
__device__ __forceinline__ bool zopen(const Geo& g, int k) {
  return g.kper || (k >= 0 && k < g.nz - 1);
}

template <class T> struct Eps;
template <> struct Eps<double> { static constexpr double v = 1e-15; };
template <> struct Eps<float> { static constexpr float v = 1e-15f; };

// Explicitly rounded multiply and fused multiply-add: the compiler never
// re-contracts these, so one formula evaluated at two places in the code (a
// face flux seen from its left and from its right cell) gives the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// Sign tests on the bit pattern (integer pipe): on the B300 the FP64 pipe
// issues 2 lanes per SM per clock, so compares and min/max of doubles are
// kept off it.  nonneg(x) is true for +0 and positive x.
__device__ __forceinline__ bool nonneg(double x) { return __double2hiint(x) >= 0; }
__device__ __forceinline__ bool nonneg(float x) { return __float_as_int(x) >= 0; }

// The bit pattern of a double through an opaque move, so that integer tests
// on it stay integer: a plain bit cast lets the compiler turn a test such as
// (bits & 0x7fff...) == 0 back into an FP64 compare.
__device__ __forceinline__ long long dbits(double x) {
  long long b;
  asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
  return b;
}

__device__ __forceinline__ long long okey(double x);
__device__ __forceinline__ long long okey0(double x);
// x >= 0 and x <= 0 with IEEE semantics (both hold for +0 and -0).
__device__ __forceinline__ bool ge0(double x) {
  const long long b = dbits(x);
  return b >= 0 || (b & 0x7fffffffffffffffLL) == 0;
}
__device__ __forceinline__ bool le0(double x) {
  const long long b = dbits(x);
  return b < 0 || b == 0;
}
__device__ __forceinline__ bool ge0(float x) { return x >= 0.0f; }
__device__ __forceinline__ bool le0(float x) { return x <= 0.0f; }
// a >= b and a <= b for doubles through the order keys (IEEE semantics for
// finite values, +0 == -0); floats compare directly.
__device__ __forceinline__ bool geq(double a, double b) { return okey0(a) >= okey0(b); }
__device__ __forceinline__ bool leq(double a, double b) { return okey0(a) <= okey0(b); }
__device__ __forceinline__ bool geq(float a, float b) { return a >= b; }
__device__ __forceinline__ bool leq(float a, float b) { return a <= b; }

// [x]+ and [x]- of the donor-cell split (FP32: one min/max instruction; FP64:
// a sign-bit select, off the FP64 pipe).
__device__ __forceinline__ double pos(double x) { return nonneg(x) ? x : 0.0; }
__device__ __forceinline__ double neg(double x) { return nonneg(x) ? 0.0 : x; }
__device__ __forceinline__ float pos(float x) { return fmaxf(x, 0.0f); }
__device__ __forceinline__ float neg(float x) { return fminf(x, 0.0f); }
__device__ __forceinline__ double absv(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ float absv(float x) { return fabsf(x); }

// Donor-cell (upwind) flux through a face: left value L, right value R,
// face Courant number C (Listings 4/5): max(C,0) L + min(C,0) R, which is
// C*L for C >= 0 and C*R otherwise (one product, the same rounded value).
template <class T>
__device__ __forceinline__ T donor(T L, T R, T C) {
  return mul_rn(C, nonneg(C) ? L : R);
}

// min/max.  FP32 uses the hardware min/max (integer-rate pipe).  FP64 maps
// each double to an int64 key with the same order (sign-magnitude ->
// two's complement: flip the magnitude bits of negatives) and compares keys.
__device__ __forceinline__ long long okey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);  // -0 sorts just below +0
}
// The same order with -0 and +0 equal (IEEE ties), for branch decisions
// that must match IEEE comparisons exactly (the adjoint's tie rules).
__device__ __forceinline__ long long okey0(double x) {
  const long long b = dbits(x);
  return b >= 0 ? b : -(b & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double kdecode(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ double vmax(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ double vmin(double a, double b) { return okey(a) <= okey(b) ? a : b; }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
// Largest and smallest of n values (the limiter bounds).  FP64 folds on the
// order keys (one key per value, integer compares), FP32 on min/max.
template <int N>
__device__ __forceinline__ void bounds(const double (&v)[N], double& hi, double& lo) {
  long long kh = okey(v[0]), kl = kh;
#pragma unroll
  for (int q = 1; q < N; ++q) {
    const long long k = okey(v[q]);
    kh = k > kh ? k : kh;
    kl = k < kl ? k : kl;
  }
  hi = kdecode(kh);
  lo = kdecode(kl);
}
template <int N>
__device__ __forceinline__ void bounds(const float (&v)[N], float& hi, float& lo) {
  hi = v[0];
  lo = v[0];
#pragma unroll
  for (int q = 1; q < N; ++q) {
    hi = fmaxf(hi, v[q]);
    lo = fminf(lo, v[q]);
  }
}

// min of non-negative values (limiter factors): raw bit patterns order them.
__device__ __forceinline__ double nmin(double a, double b) {
  return dbits(a) <= dbits(b) ? a : b;
}
__device__ __forceinline__ float nmin(float a, float b) { return fminf(a, b); }

// Reciprocal of a positive normal number.  FP32: the hardware approximation
// (rcp.approx, about 1 ulp).  FP64: the hardware seed r (relative error
// e = 1 - b r, |e| < 2^-19) refined by one third-order step of the series
// 1/b = r / (1 - e) = r (1 + e + e^2 + ...): r <- r + r (e + e^2), whose
// truncation error e^3 < 2^-57 is below the final rounding; three FMAs,
// against four for two Newton steps.  a*rcp(b) is within ~2 ulp of a/b.
// Used for every ratio of the scheme: A, B, beta, 1/G and 1/G_face, whose
// denominators are >= epsilon > 0 or G > 0.
__device__ __forceinline__ float rcp(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
__device__ __forceinline__ double rcp(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  const double e = fma(-b, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// Programmatic dependent launch.  A kernel launched with programmatic
// stream serialization may be scheduled while the kernel before it in the
// stream is still running; it first waits until that kernel has completed
// and its writes are visible, then lets the next kernel of the stream be
// scheduled the same way.  This hides the launch latency between the small
// kernels of a step.  Launched without the attribute, the wait returns at
// once and the trigger does nothing.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host: launch kernel k, which begins with pdl_enter(), with programmatic
// stream serialization.  A launch error is reported as for <<<...>>>: by
// cudaGetLastError.
template <class... P, class... A>
inline void launch_pdl(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       A&&... a) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<A>(a)...);
}

// Limited velocity on a face (non-oscillatory option):
// min(1, bd_L, bu_R) [Ut]+ + min(1, bu_L, bd_R) [Ut]-; the betas are >= 0,
// and only one of the two parts is non-zero.  The factor is selected before
// the one product (selecting between two products costs the FP64 pipe a
// second multiply).
template <class T>
__device__ __forceinline__ T limit_factor(T Ut, T buL, T bdL, T buR, T bdR) {
  const bool up = nonneg(Ut);
  return nmin(nmin(T(1), up ? bdL : buL), up ? buR : bdR);
}
template <class T>
__device__ __forceinline__ T limit_face(T Ut, T buL, T bdL, T buR, T bdR) {
  return mul_rn(limit_factor(Ut, buL, bdL, buR, bdR), Ut);
}

// Antidiffusive pseudo-velocity on one face from its ingredients:
//   U       face Courant number;           gsum  G_L + G_R (G_face = gsum/2)
//   pl, pr  psi1 left and right;           s1p, s1m  sums of the two psi1
//           values one row/level above and below in the first cross direction
//   s2p, s2m  the same in the second cross direction
//   vsum, wsum  sums of the four cross-direction Courant numbers around the face
// Ut = (|U| - U^2/Gf) A - U (Vbar B1 + Wbar B2)/Gf with A = (pr-pl)/(pr+pl+eps),
// B = (1/2)(s+ - s-)/(s+ + s- + eps), Vbar = vsum/4 (Smolarkiewicz 1984,
// G-weighted as in Smolarkiewicz & Margolin 1998).  The factors 1/2 and 1/4
// are applied as one exact 1/8 scaling.  Every operation is explicitly
// rounded (no contraction left to the compiler), so the two-lane form of
// the FP32 step (fusedx.cuh) evaluates the same sequence and gives the same
// bits.
template <class T>
__device__ __forceinline__ T pseudo_velocity(T U, T gsum, T pl, T pr, T s1p, T s1m, T s2p,
                                             T s2m, T vsum, T wsum) {
  const T eps = Eps<T>::v;
  const T rG = mul_rn(T(2), rcp(gsum));                                   // 1/Gf
  const T A = mul_rn(sub_rn(pr, pl), rcp(add_rn(add_rn(pr, pl), eps)));
  const T B1 = mul_rn(sub_rn(s1p, s1m), rcp(add_rn(add_rn(s1p, s1m), eps)));  // 2 B1
  const T B2 = mul_rn(sub_rn(s2p, s2m), rcp(add_rn(add_rn(s2p, s2m), eps)));  // 2 B2
  const T q = mul_rn(U, rG);
  const T diff = fma_rn(-U, q, absv(U));                                  // |U| - U^2/Gf
  const T cross = mul_rn(T(0.125), fma_rn(vsum, B1, mul_rn(wsum, B2)));   // Vbar B1 + Wbar B2
  return fma_rn(diff, A, -mul_rn(q, cross));
}

// Corrective-pass options (bit flags; the MPDATA literature's variants).
enum : int { kOptDFL = 1, kOptABS = 2, kOptIGA = 4 };

// Infinite-gauge pseudo-flux of one face (option IGA), the same ingredients
// as pseudo_velocity: the limit c -> infinity of c times the pseudo-velocity
// of psi + c (Smolarkiewicz & Clark 1986), where cA -> (pr - pl)/2 and
// cB -> (s+ - s-)/8:
//   Ft = (|U| - U^2/Gf) (pr - pl)/2 - U (vsum (s1p - s1m) + wsum (s2p - s2m)) / (32 Gf).
// Ft is itself the corrective flux of the face.
// Explicitly rounded, like pseudo_velocity.
template <class T>
__device__ __forceinline__ T pseudo_flux_iga(T U, T gsum, T pl, T pr, T s1p, T s1m, T s2p,
                                             T s2m, T vsum, T wsum) {
  const T rG = mul_rn(T(2), rcp(gsum));                // 1/Gf
  const T q = mul_rn(U, rG);
  const T diff = fma_rn(-U, q, absv(U));               // |U| - U^2/Gf
  const T cross = mul_rn(T(0.03125), fma_rn(vsum, sub_rn(s1p, s1m),
                                            mul_rn(wsum, sub_rn(s2p, s2m))));
  return fma_rn(diff, mul_rn(T(0.5), sub_rn(pr, pl)), -mul_rn(q, cross));
}

// Divergent-flow term of one face (option DFL; Smolarkiewicz 1984): with
// dsum = D_L + D_R, the divergences of the G-weighted Courant numbers of
// the face's two cells,  -(1/4) U dsum / Gf.  Explicitly rounded; a caller
// adds it with add_rn (no contraction of its last product into the sum).
template <class T>
__device__ __forceinline__ T divergent_flow_term(T U, T gsum, T dsum) {
  return mul_rn(mul_rn(mul_rn(T(-0.5), U), dsum), rcp(gsum));
}

}  // namespace mpd
