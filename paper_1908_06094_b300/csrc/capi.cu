// capi.cu -- the C ABI of libmpdata_b300.so (declared in include/mpdata.h):
// the context, host-side argument checks, and the per-step launch sequence.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>

#include "../../include/mpdata.h"
#include "grid.cuh"
#include "mass.cuh"
#include "staged.cuh"
#include "march.cuh"
#include "exchange.cuh"
#include "fused2.cuh"
#include "fusedx.cuh"
#include "adjoint.cuh"

using mpd::Geo;

struct mpdata_ctx {
  Geo g;
  int iord, nonosc, dtype, kbc, variant, device;
  int opts;  // corrective-pass options (MPDATA_OPT_* bits)
  size_t esize;
  cudaStream_t stream;
  // scratch of one step (one allocation)
  void* scratch;
  void *psi1, *psi2, *fx, *fy, *fz, *ut, *vt, *wt, *bu, *bd, *ul, *vl, *wl;
  void* rg;  // 1/G, shared by the advances of one FP64 staged step (iord >= 2)
  double* part;
  // fused kernel launch shape (chosen in init)
  int fused_ok, nchunks, kchunk;
  // the two-column FP32 kernel's launch shape (x2_ok: it runs the untaped
  // FP32 step)
  int x2_ok, x2_nchunks, x2_kchunk;
  // the FP64 one-level grid of at most 128 x 128 columns runs its plain
  // step on 8 x small_ty tiles (0: not)
  int small_ty;
  // the last staged step wrote the halo of its output itself
  bool halo_done;
  // level-chunk lengths of the k-marching kernels (0: not chosen yet)
  int kc_fwd, kc_rev;
  // the adjoint's accumulators (psi^n-bar, beta adjoints) are known to be
  // zero: every reverse step leaves them so (its readers clear them)
  bool adj_zero;
  // device copies for the HOST-buffer call (allocated on its first use)
  void* hbuf;
  // the pipelined HOST-buffer calls (created on their first use): two sets
  // of five device fields, a host-to-device and a device-to-host stream, and
  // per set the events in-copied, stepped, out-copied
  void* pbuf;
  cudaStream_t ps_in, ps_out;
  cudaEvent_t pe_in[2], pe_step[2], pe_out[2];
  int pslot;
  bool pused[2];
  // adjoint scratch (allocated on the first adjoint call)
  void* adjbuf;
  void* a_out;  // the recomputed psi^(n+1) of mpdata_adjoint_step
  // instrumentation
  long long launches;
  bool prof_on;
  int prof_n, prof_cap;
  cudaEvent_t* prof_ev;
  int* prof_stage;
  char err[256];
};

namespace {

int cuda_fail(mpdata_ctx* c, cudaError_t e, const char* where) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s: %s", where, cudaGetErrorString(e));
  return MPDATA_ECUDA;
}

int fail(mpdata_ctx* c, int code, const char* what) {
  if (c) std::snprintf(c->err, sizeof(c->err), "%s", what);
  return code;
}

#define MPD_CHECK_LAUNCH(c, where)                      \
  do {                                                  \
    cudaError_t e_ = cudaGetLastError();                \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

// Every kernel launch goes through MPD_LAUNCH: it is counted, and timed with
// a pair of events on the context's stream while profiling is enabled.
void prof_begin(mpdata_ctx* c) {
  if (c->prof_on && c->prof_n < c->prof_cap) cudaEventRecord(c->prof_ev[2 * c->prof_n], c->stream);
}
void prof_end(mpdata_ctx* c, int stage) {
  ++c->launches;
  if (c->prof_on && c->prof_n < c->prof_cap) {
    cudaEventRecord(c->prof_ev[2 * c->prof_n + 1], c->stream);
    c->prof_stage[c->prof_n++] = stage;
  }
}
#define MPD_LAUNCH(c, stage, ...) \
  do {                            \
    prof_begin(c);                \
    __VA_ARGS__;                  \
    prof_end(c, stage);           \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

dim3 cell_grid(const Geo& g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }
const dim3 kCellBlock(32, 8, 1);

// Grid of the halo kernels: one thread per halo cell (with the interior
// top level of a WFACE fill).
dim3 halo_grid(const Geo& g) {
  const int64_t plane = g.px * (int64_t)(g.ny + 2 * g.h);
  const int64_t n = (2 * g.h + 1) * plane + (int64_t)g.nz * 2 * g.h * (g.px + g.ny);
  return dim3((unsigned)((n + 255) / 256));
}

template <class T>
int halo_launch(mpdata_ctx* c, T* f, int kind) {
  MPD_LAUNCH(c, MPDATA_STAGE_HALO,
             mpd::launch_pdl(mpd::halo_kernel<T>, halo_grid(c->g), 256, 0, c->stream, c->g, f,
                             kind));
  MPD_CHECK_LAUNCH(c, "halo_kernel");
  return MPDATA_OK;
}

// Level-chunk length of a k-marching kernel; a CTA costs about (its levels
// + 2 start-up levels).  A kernel bound by the SM's FP64 pipe shares it
// among the CTAs resident on an SM, so its time goes as (CTAs per SM) x
// (levels + 2); a latency-bound one runs its resident CTAs side by side, so
// its time goes as (waves of resident CTAs) x (levels + 2).  Take the
// cheapest length.  (For the FP32 pseudo-velocity reverse on 256x256x64 the
// wave model ranks the measured chunk lengths 13 < 8 < 11, 22 < 16 < 32.)
template <class K>
int march_chunk(mpdata_ctx* c, K kernel, bool pipe_bound) {
  namespace M = mpd::march;
  const Geo& g = c->g;
  int occ = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, M::TX * M::TY, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaGetLastError();
  if (occ < 1 || sms < 1) return M::KC;
  const long tiles = (long)((g.nx + M::TX - 1) / M::TX) * ((g.ny + M::TY - 1) / M::TY);
  const long slots = pipe_bound ? sms : (long)occ * sms;
  int best = g.nz;
  double best_cost = 1e300;
  for (int kc = 1; kc <= g.nz; ++kc) {
    const long n = (g.nz + kc - 1) / kc;
    const long waves = (tiles * n + slots - 1) / slots;
    const double cost = (double)waves * (kc + 2);
    if (cost < best_cost - 1e-9) { best_cost = cost; best = kc; }
  }
  return best;
}

// The pseudo-velocity stage: FP64 on the k-marching common-denominator
// kernel (bound by FP64 instruction count), FP32 on the cell-parallel one.
// FLUX (FP64 without the signed-field or infinite-gauge options): also
// store the donor fluxes of the pseudo-velocities in fx, fy, fz.
template <class T, int OPT = 0, bool FLUX = false>
void pseudo_launch(mpdata_ctx* c, const T* P, const T* U, const T* V, const T* W, const T* G,
                   T* ut, T* vt, T* wt, T* fx = nullptr, T* fy = nullptr, T* fz = nullptr) {
  const Geo& g = c->g;
  if constexpr (std::is_same<T, double>::value) {
    // FP64: the k-marching kernel, with the options' terms (IGA: its own
    // face operation; ABS, DFL: flags of the common-denominator one)
    namespace M = mpd::march;
    constexpr bool kIGA = (OPT & mpd::kOptIGA) != 0, kDFL = (OPT & mpd::kOptDFL) != 0;
    static_assert(!FLUX || (OPT & (mpd::kOptABS | mpd::kOptIGA)) == 0, "FLUX: signed psi only");
    using Op = std::conditional_t<kIGA, M::PseudoIGA, M::PseudoMergedT<kDFL, FLUX>>;
    Op op{ut, vt, wt};
    if constexpr (FLUX) {
      op.fx = fx;
      op.fy = fy;
      op.fz = fz;
    }
    auto kern = M::march_kernel<double, Op, OPT>;
    if (!c->kc_fwd) c->kc_fwd = march_chunk(c, M::march_kernel<double, M::PseudoMerged>, true);
    MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
               mpd::launch_pdl(kern, M::march_grid(g, c->kc_fwd), dim3(M::TX, M::TY), 0, c->stream,
                               g, P, U, V, W, G, op, c->kc_fwd));
  } else if constexpr (OPT != 0) {  // FP32 staged with options: cell-parallel kernel
    MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
               mpd::launch_pdl(mpd::staged::pseudo_kernel<T, OPT>, cell_grid(g), kCellBlock, 0,
                               c->stream, g, P, U, V, W, G, ut, vt, wt));
  } else {
    MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
               mpd::launch_pdl(mpd::staged::pseudo_kernel<T>, cell_grid(g), kCellBlock, 0,
                               c->stream, g, P, U, V, W, G, ut, vt, wt));
  }
}

// One MPDATA step, staged organisation (one kernel per stage).
// psi_out may equal psi_in: psi_in is last read (by the limiter) before the
// final advance writes psi_out.  OPT: the corrective-pass options.
template <class T, int OPT>
int step_staged_opt(mpdata_ctx* c, const T* psi_in, T* psi_out, const T* U, const T* V,
                    const T* W, const T* G) {
  constexpr bool kUnit = (OPT & mpd::kOptIGA) != 0;  // pseudo-fluxes are the fluxes
  // FP64 without the signed-field or infinite-gauge options: the pseudo-
  // velocity stage also stores the donor fluxes of the pseudo-velocities in
  // fx, fy, fz (the donor pass's fluxes are dead by then); the beta stage
  // reads them as its fluxes and the limiter scales them in place
  constexpr bool kFin =
      std::is_same<T, double>::value && (OPT & (mpd::kOptABS | mpd::kOptIGA)) == 0;
  using namespace mpd::staged;
  const Geo& g = c->g;
  const dim3 grid = cell_grid(g);
  cudaStream_t s = c->stream;
  c->halo_done = false;
  const T* psi = psi_in;
  T *fx = (T*)c->fx, *fy = (T*)c->fy, *fz = (T*)c->fz;
  // FP64: the donor fluxes' kernel (bound by memory) stores 1/G for all the
  // advances of the step (bound by the FP64 pipe)
  T* rg = (T*)c->rg;
  // pass 1: donor cell
  T* cur = c->iord == 1 ? psi_out : (T*)c->psi1;
  if (rg) {
    MPD_LAUNCH(c, MPDATA_STAGE_DONOR,
               (mpd::launch_pdl(flux_kernel<T, true>, grid, kCellBlock, 0, s, g, psi, U, V, W, fx,
                                fy, fz, G, rg)));
    MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
               (mpd::launch_pdl(advance_kernel<T, 2>, grid, kCellBlock, 0, s, g, psi, fx, fy, fz, G,
                                cur, rg)));
  } else {
    MPD_LAUNCH(c, MPDATA_STAGE_DONOR,
               mpd::launch_pdl(flux_kernel<T>, grid, kCellBlock, 0, s, g, psi, U, V, W, fx, fy, fz,
                               nullptr, nullptr));
    MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
               mpd::launch_pdl(advance_kernel<T>, grid, kCellBlock, 0, s, g, psi, fx, fy, fz, G,
                               cur, nullptr));
  }
  MPD_CHECK_LAUNCH(c, "donor pass");
  // corrective passes
  const T *cu = U, *cv = V, *cw = W;
  T* setA[3] = {(T*)c->ut, (T*)c->vt, (T*)c->wt};
  T* setB[3] = {(T*)c->ul, (T*)c->vl, (T*)c->wl};
  for (int m = 2; m <= c->iord; ++m) {
    T** tset = (cu == setA[0]) ? setB : setA;  // unlimited pseudo-velocities
    T** lset = (tset == setA) ? setB : setA;   // limited ones (next pass's input)
    const bool more = m < c->iord;
    pseudo_launch<T, OPT, kFin>(c, cur, cu, cv, cw, G, tset[0], tset[1], tset[2], fx, fy, fz);
    const T *ffx = fx, *ffy = fy, *ffz = fz;  // the pass's face fluxes
    T* dest = !more ? psi_out : (cur == (T*)c->psi1 ? (T*)c->psi2 : (T*)c->psi1);
    if (c->nonosc) {
      const T* bf[3] = {kFin ? fx : tset[0], kFin ? fy : tset[1], kFin ? fz : tset[2]};
      MPD_LAUNCH(c, MPDATA_STAGE_BETA,
                 (mpd::launch_pdl(beta_kernel<T, kUnit || kFin>, grid, kCellBlock, 0, s, g, psi,
                                  cur, bf[0], bf[1], bf[2], G, (T*)c->bu, (T*)c->bd, nullptr,
                                  nullptr)));
      if (kFin && !more && rg) {  // the last pass: limited fluxes and advance in one
        // with the halo images of psi^(n+1) where one image a side covers
        // the halo and the k halo's images fall on the bottom and top levels
        // only (no separate halo fill then; a grid of one or a few levels,
        // whose every cell would write 2h images, keeps the fill kernel)
        const bool img = g.nx >= 2 * g.h && g.ny >= 2 * g.h && g.nz > 2 * g.h;
        if (img)
          MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
                     (mpd::launch_pdl(limadvance_kernel<T, true>, grid, kCellBlock, 0, s, g, cur,
                                      tset[0], tset[1], tset[2], (T*)c->bu, (T*)c->bd, fx, fy, fz,
                                      rg, dest)));
        else
          MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
                     (mpd::launch_pdl(limadvance_kernel<T, false>, grid, kCellBlock, 0, s, g, cur,
                                      tset[0], tset[1], tset[2], (T*)c->bu, (T*)c->bd, fx, fy, fz,
                                      rg, dest)));
        c->halo_done = img;
        MPD_CHECK_LAUNCH(c, "corrective pass");
        cur = dest;
        continue;  // the last pass: nothing carries over
      }
      MPD_LAUNCH(c, MPDATA_STAGE_LIMIT,
                 (mpd::launch_pdl(limflux_kernel<T, OPT, kFin>, grid, kCellBlock, 0, s, g, cur,
                                  tset[0], tset[1], tset[2], (T*)c->bu, (T*)c->bd, fx, fy, fz,
                                  more ? lset[0] : nullptr, more ? lset[1] : nullptr,
                                  more ? lset[2] : nullptr)));
    } else if (kUnit) {  // the unlimited pseudo-fluxes themselves
      ffx = tset[0]; ffy = tset[1]; ffz = tset[2];
    } else if (kFin) {  // fx, fy, fz hold the pass's fluxes already
    } else {
      MPD_LAUNCH(c, MPDATA_STAGE_LIMIT,
                 mpd::launch_pdl(flux_kernel<T>, grid, kCellBlock, 0, s, g, cur, tset[0], tset[1],
                                 tset[2], fx, fy, fz, nullptr, nullptr));
    }
    if (rg) {
      MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
                 (mpd::launch_pdl(advance_kernel<T, 2>, grid, kCellBlock, 0, s, g, cur, ffx, ffy,
                                  ffz, G, dest, rg)));
    } else {
      MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
                 mpd::launch_pdl(advance_kernel<T>, grid, kCellBlock, 0, s, g, cur, ffx, ffy, ffz,
                                 G, dest, nullptr));
    }
    MPD_CHECK_LAUNCH(c, "corrective pass");
    cur = dest;
    T** vset = c->nonosc ? lset : tset;
    cu = vset[0]; cv = vset[1]; cw = vset[2];
  }
  return MPDATA_OK;
}

template <class T>
int step_staged(mpdata_ctx* c, const T* psi_in, T* psi_out, const T* U, const T* V,
                const T* W, const T* G) {
  using namespace mpd;
  switch (c->opts) {
    case 0: return step_staged_opt<T, 0>(c, psi_in, psi_out, U, V, W, G);
    case kOptDFL: return step_staged_opt<T, kOptDFL>(c, psi_in, psi_out, U, V, W, G);
    case kOptABS: return step_staged_opt<T, kOptABS>(c, psi_in, psi_out, U, V, W, G);
    case kOptDFL | kOptABS:
      return step_staged_opt<T, kOptDFL | kOptABS>(c, psi_in, psi_out, U, V, W, G);
    case kOptIGA: return step_staged_opt<T, kOptIGA>(c, psi_in, psi_out, U, V, W, G);
    default: return fail(c, MPDATA_EINVAL, "unsupported option set");
  }
}

// Tile shape of the fused kernel (one thread per column of the tile + 2
// ring: (TX+4)(TY+4) threads); MINB: CTAs per SM the registers are sized for.
template <class T> struct FusedShape;
template <> struct FusedShape<double> { static constexpr int TX = 32, TY = 8, MINB = 1; };
template <> struct FusedShape<float> { static constexpr int TX = 32, TY = 16, MINB = 1; };

template <class T, bool LIMIT, bool TAPE = false, bool KPER = false, bool I32 = false>
auto fused_kernel_ptr() {
  using F = FusedShape<T>;
  return mpd::fused2::step_kernel2<T, F::TX, F::TY, F::MINB, LIMIT, TAPE, KPER, 0, 1, false, I32>;
}

// the slab instance (MPDATA_IJ_HALO: neighbours from the exchanged halo)
template <class T, bool LIMIT, bool KPER>
auto fused_slab_ptr() {
  using F = FusedShape<T>;
  return mpd::fused2::step_kernel2<T, F::TX, F::TY, F::MINB, LIMIT, false, KPER, 0, 1, true>;
}

template <class T, bool LIMIT, bool KPER, int OPT>
auto fused_opt_ptr() {
  using F = FusedShape<T>;
  return mpd::fused2::step_kernel2<T, F::TX, F::TY, F::MINB, LIMIT, false, KPER, OPT>;
}

// FP32 instances with corrective-pass options (FP64 runs options on the
// staged kernels); the basic instance for opts == 0.
template <bool LIMIT, bool KPER>
auto fused_opt_pick(int opts) {
  using namespace mpd;
  switch (opts) {
    case kOptDFL: return fused_opt_ptr<float, LIMIT, KPER, kOptDFL>();
    case kOptABS: return fused_opt_ptr<float, LIMIT, KPER, kOptABS>();
    case kOptDFL | kOptABS: return fused_opt_ptr<float, LIMIT, KPER, kOptDFL | kOptABS>();
    case kOptIGA: return fused_opt_ptr<float, LIMIT, KPER, kOptIGA>();
    default: return fused_opt_ptr<float, LIMIT, KPER, 0>();
  }
}

// The instance for the context's limiter, vertical boundary and options.
template <class T, bool TAPE>
auto fused_pick(const mpdata_ctx* c) {
  if constexpr (!TAPE) {
    if (c->g.openij) {  // a slab (no options, no tape)
      if (c->g.kper)
        return c->nonosc ? fused_slab_ptr<T, true, true>() : fused_slab_ptr<T, false, true>();
      return c->nonosc ? fused_slab_ptr<T, true, false>() : fused_slab_ptr<T, false, false>();
    }
  }
  if constexpr (std::is_same<T, float>::value && !TAPE) {
    if (c->opts) {
      if (c->g.kper)
        return c->nonosc ? fused_opt_pick<true, true>(c->opts) : fused_opt_pick<false, true>(c->opts);
      return c->nonosc ? fused_opt_pick<true, false>(c->opts) : fused_opt_pick<false, false>(c->opts);
    }
  }
  // fields of fewer than 2^31 elements take the 32-bit-offset instances
  if (!TAPE && c->g.total < ((int64_t)1 << 31)) {
    if (c->g.kper)
      return c->nonosc ? fused_kernel_ptr<T, true, TAPE, true, true>()
                       : fused_kernel_ptr<T, false, TAPE, true, true>();
    return c->nonosc ? fused_kernel_ptr<T, true, TAPE, false, true>()
                     : fused_kernel_ptr<T, false, TAPE, false, true>();
  }
  if (c->g.kper)
    return c->nonosc ? fused_kernel_ptr<T, true, TAPE, true>() : fused_kernel_ptr<T, false, TAPE, true>();
  return c->nonosc ? fused_kernel_ptr<T, true, TAPE>() : fused_kernel_ptr<T, false, TAPE>();
}

template <class T>
size_t fused_smem() {
  using F = FusedShape<T>;
  return mpd::fused2::Layout<T, F::TX, F::TY>::bytes;
}

template <class T>
constexpr int fused_threads() {
  using F = FusedShape<T>;
  return (F::TX + 4) * (F::TY + 4);
}

// Split k into chunks when there are too few column tiles to load every
// SM: an SM's time ~ (CTAs it runs) x (levels per chunk + the ~4 extra
// planes each chunk recomputes at its start); take the cheapest split.
// Returns the chunk count; *kchunk its length.
int pick_chunks(const Geo& g, long ctas, int sms, int* kchunk) {
  long best_n = 1;
  double best_cost = 1e300;
  for (long n = 1; n <= g.nz; ++n) {
    const long kc = (g.nz + n - 1) / n;
    const long nn = (g.nz + kc - 1) / kc;
    const long per_sm = (ctas * nn + sms - 1) / sms;
    const double cost = (double)per_sm * (kc + 4);
    if (cost < best_cost - 1e-9) { best_cost = cost; best_n = nn; }
  }
  *kchunk = (int)((g.nz + best_n - 1) / best_n);
  return (g.nz + *kchunk - 1) / *kchunk;
}

// The FP64 step of a small one-level grid (at most 128 x 128 columns): the
// one-kernel step on 8 x TY tiles.  FP64 issues 2 lanes an SM a clock, so a
// step of a few thousand cells is bound by how many SMs share its FP64 work:
// the staged kernels' 32 x 8 blocks, or 32 x 8 tiles, cover 16-64 SMs of a
// 64 x 64 to 128 x 128 grid, 8 x 8 tiles 64-256, 8 x 4 tiles 128-512 (their
// ring recompute included).  Per step at 64 x 64: 8 x 4 tiles 11.8 us, 8 x 8
// 12.4-13.3, staged kernels 18.1, 32 x 8 tiles 23.2; at 128 x 128: 8 x 8
// tiles 17.7-19.3, 8 x 4 21.5, staged 19.2; 256 x 256 runs faster staged
// (42 against 62).  So 8 x 4 tiles up to 64 x 64 columns, 8 x 8 up to
// 128 x 128.
template <int TY, bool LIMIT, bool KPER>
auto fused_small_ptr() {
  return mpd::fused2::step_kernel2<double, 8, TY, 1, LIMIT, false, KPER, 0, 1, false, true>;
}
template <int TY>
auto fused_small_pick(const mpdata_ctx* c) {
  if (c->g.kper)
    return c->nonosc ? fused_small_ptr<TY, true, true>() : fused_small_ptr<TY, false, true>();
  return c->nonosc ? fused_small_ptr<TY, true, false>() : fused_small_ptr<TY, false, false>();
}
template <int TY>
constexpr size_t fused_small_smem() {
  return mpd::fused2::Layout<double, 8, TY>::bytes;
}
template <int TY>
bool fused_small_attr(const mpdata_ctx* c) {
  if (cudaFuncSetAttribute(fused_small_pick<TY>(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fused_small_smem<TY>()) == cudaSuccess)
    return true;
  cudaGetLastError();
  return false;
}
void fused_small_setup(mpdata_ctx* c) {
  const Geo& g = c->g;
  c->small_ty = 0;
  const int64_t cols = (int64_t)g.nx * g.ny;
  if (c->dtype != MPDATA_F64 || !c->fused_ok || g.openij || g.nz != 1 || cols > 128 * 128)
    return;
  if (cols <= 64 * 64) c->small_ty = fused_small_attr<4>(c) ? 4 : 0;
  else c->small_ty = fused_small_attr<8>(c) ? 8 : 0;
}
template <int TY>
int fused_small_launch(mpdata_ctx* c, const double* in, double* out, const double* U,
                       const double* V, const double* W, const double* G) {
  const Geo& g = c->g;
  const dim3 gs((g.nx + 7) / 8, (g.ny + TY - 1) / TY, 1);
  MPD_LAUNCH(c, MPDATA_STAGE_FUSED,
             mpd::launch_pdl(fused_small_pick<TY>(c), gs, 12 * (TY + 4), fused_small_smem<TY>(),
                             c->stream, g, g.nz, in, U, V, W, G, out,
                             mpd::fused2::TapeOut<double>{}));
  MPD_CHECK_LAUNCH(c, "fused step kernel");
  return MPDATA_OK;
}

// The two-column FP32 step (fusedx.cuh): its tile (32 x 24 columns, 504
// threads of two columns, up to 128 registers) and instances.
struct FusedX { static constexpr int TX = 32, TY = 24, MINB = 1; };
template <bool LIMIT, bool KPER, bool TAPE, int OPT = 0>
auto fusedx_ptr() {
  return mpd::fusedx::step_kernel_x2<FusedX::TX, FusedX::TY, FusedX::MINB, LIMIT, KPER, TAPE,
                                     OPT>;
}
// the option instances (with the limiter; the taped step has no options)
template <bool KPER>
auto fusedx_opt_pick(int opts) {
  using namespace mpd;
  switch (opts) {
    case kOptDFL: return fusedx_ptr<true, KPER, false, kOptDFL>();
    case kOptABS: return fusedx_ptr<true, KPER, false, kOptABS>();
    case kOptDFL | kOptABS: return fusedx_ptr<true, KPER, false, kOptDFL | kOptABS>();
    default: return fusedx_ptr<true, KPER, false, kOptIGA>();
  }
}
template <bool TAPE = false>
auto fusedx_pick(const mpdata_ctx* c) {
  if constexpr (!TAPE) {
    if (c->opts) return c->g.kper ? fusedx_opt_pick<true>(c->opts) : fusedx_opt_pick<false>(c->opts);
  }
  if (c->g.kper)
    return c->nonosc ? fusedx_ptr<true, true, TAPE>() : fusedx_ptr<false, true, TAPE>();
  return c->nonosc ? fusedx_ptr<true, false, TAPE>() : fusedx_ptr<false, false, TAPE>();
}
constexpr int fusedx_threads() { return mpd::fusedx::PairMap<FusedX::TX, FusedX::TY>::NT; }
constexpr size_t fusedx_smem() { return mpd::fusedx::Layout<FusedX::TX, FusedX::TY>::bytes; }

// Whether the two-column kernel can run this context's step (plain or
// taped): FP32, no options or options with the limiter, the periodic i-j
// domain, pairs of columns on 8-byte
// boundaries (even nx and halo: even row length and interior offset) and
// 32-bit offsets.
void fusedx_setup(mpdata_ctx* c) {
  const Geo& g = c->g;
  c->x2_ok = 0;
  if (c->dtype != MPDATA_F32 || (c->opts != 0 && !c->nonosc) || g.openij || g.nx % 2 != 0 ||
      g.h % 2 != 0 || g.total >= ((int64_t)1 << 31))
    return;
  auto k = fusedx_pick(c);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fusedx_smem()) != cudaSuccess ||
      cudaFuncSetAttribute(fusedx_pick<true>(c), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)fusedx_smem()) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int occ = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, fusedx_threads(), fusedx_smem());
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaGetLastError();
  if (occ < 1) return;
  const long ctas = (long)((g.nx + FusedX::TX - 1) / FusedX::TX) * ((g.ny + FusedX::TY - 1) / FusedX::TY);
  c->x2_nchunks = pick_chunks(g, ctas, sms, &c->x2_kchunk);
  c->x2_ok = 1;
}

// Pick the k-chunking so that the grid covers the GPU about twice.
template <class T>
int fused_setup(mpdata_ctx* c) {
  using F = FusedShape<T>;
  const Geo& g = c->g;
  c->fused_ok = 0;
  c->x2_ok = 0;
  c->small_ty = 0;
  // the periodic images a column writes need nx, ny >= 2h; a slab writes
  // none and needs only an interior as wide as the strips it sends
  const int minw = g.openij ? g.h : 2 * g.h;
  if (c->iord != 2 || g.nx < minw || g.ny < minw) return MPDATA_OK;
  const size_t bytes = fused_smem<T>();
  auto kplain = fused_pick<T, false>(c);
  auto ktape = fused_pick<T, true>(c);
  const int ib = (int)bytes;
  if (cudaFuncSetAttribute(kplain, cudaFuncAttributeMaxDynamicSharedMemorySize, ib) != cudaSuccess ||
      cudaFuncSetAttribute(ktape, cudaFuncAttributeMaxDynamicSharedMemorySize, ib) != cudaSuccess) {
    cudaGetLastError();
    return MPDATA_OK;  // not eligible on this device: the staged kernels run
  }
  int occ = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kplain, fused_threads<T>(), bytes);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  cudaGetLastError();
  if (occ < 1) return MPDATA_OK;
  const long ctas = (long)((g.nx + F::TX - 1) / F::TX) * ((g.ny + F::TY - 1) / F::TY);
  c->nchunks = pick_chunks(g, ctas, sms, &c->kchunk);
  c->fused_ok = 1;
  fusedx_setup(c);
  fused_small_setup(c);
  return MPDATA_OK;
}

// One fused step; with tape != nullptr it also writes the step's
// intermediates of every interior cell (a taped step).
template <class T>
int fused_launch(mpdata_ctx* c, const T* in, T* out, const T* U, const T* V, const T* W,
                 const T* G, const mpd::fused2::TapeOut<T>* tape = nullptr) {
  using F = FusedShape<T>;
  const Geo& g = c->g;
  if constexpr (std::is_same<T, float>::value) {
    // the two-column kernel (the same bits) reads and writes 8-byte pairs:
    // every field must start on an 8-byte boundary
    auto al8 = [](const void* p) { return ((uintptr_t)p & 7) == 0; };
    // (the taped step: its fields tstride elements apart from psi1, each on
    // an 8-byte boundary)
    const long long tstride = tape ? (long long)(tape->ut - tape->p1) : 0;
    if (c->x2_ok && (c->opts == 0 || (!tape && c->nonosc)) && !g.openij && al8(in) &&
        al8(out) && al8(U) &&
        al8(V) && al8(W) && al8(G) && (!tape || (al8(tape->p1) && tstride % 2 == 0))) {
      dim3 gx((g.nx + FusedX::TX - 1) / FusedX::TX, (g.ny + FusedX::TY - 1) / FusedX::TY,
              c->x2_nchunks);
      if (tape) {
        auto kx = fusedx_pick<true>(c);
        MPD_LAUNCH(c, MPDATA_STAGE_FUSED,
                   mpd::launch_pdl(kx, gx, fusedx_threads(), fusedx_smem(), c->stream, g,
                                   c->x2_kchunk, in, U, V, W, G, out, tape->p1, tstride));
      } else {
        auto kx = fusedx_pick(c);
        MPD_LAUNCH(c, MPDATA_STAGE_FUSED,
                   mpd::launch_pdl(kx, gx, fusedx_threads(), fusedx_smem(), c->stream, g,
                                   c->x2_kchunk, in, U, V, W, G, out, nullptr, 0));
      }
      MPD_CHECK_LAUNCH(c, "fused step kernel");
      return MPDATA_OK;
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    if (c->small_ty && !tape && c->opts == 0)  // a small one-level grid: 8 x TY tiles
      return c->small_ty == 4 ? fused_small_launch<4>(c, in, out, U, V, W, G)
                              : fused_small_launch<8>(c, in, out, U, V, W, G);
  }
  dim3 grid((g.nx + F::TX - 1) / F::TX, (g.ny + F::TY - 1) / F::TY, c->nchunks);
  const size_t bytes = fused_smem<T>();
  const mpd::fused2::TapeOut<T> tp = tape ? *tape : mpd::fused2::TapeOut<T>{};
  auto go = [&](auto kern) {
    MPD_LAUNCH(c, MPDATA_STAGE_FUSED,
               mpd::launch_pdl(kern, grid, fused_threads<T>(), bytes, c->stream, g, c->kchunk, in,
                               U, V, W, G, out, tp));
  };
  if (tape) go(fused_pick<T, true>(c));
  else go(fused_pick<T, false>(c));
  MPD_CHECK_LAUNCH(c, "fused step kernel");
  return MPDATA_OK;
}

bool use_fused(const mpdata_ctx* c) {
  // a slab of a decomposed domain always runs the one-kernel step (its one
  // halo exchange per step feeds exactly that kernel's radius-3 reads)
  if (c->g.openij) return c->fused_ok != 0;
  // options run fused in FP32 only (FP64 takes the staged kernels)
  if (!c->fused_ok || (c->opts != 0 && c->dtype != MPDATA_F32)) return false;
  if (c->variant == MPDATA_AUTO) return c->dtype == MPDATA_F32;
  return c->variant == MPDATA_FUSED;
}
// The plain step of a small one-level FP64 grid runs fused on 8 x 8 tiles
// unless the staged kernels are asked for.
bool use_fused_plain(const mpdata_ctx* c) {
  return use_fused(c) || (c->small_ty && c->opts == 0 && c->variant != MPDATA_STAGED);
}

// One step psi_in -> psi_out (distinct buffers), halo of psi_out filled.
template <class T>
int step_out(mpdata_ctx* c, const T* in, T* out, const T* U, const T* V, const T* W,
             const T* G) {
  if (use_fused_plain(c)) return fused_launch<T>(c, in, out, U, V, W, G);
  int rc = step_staged<T>(c, in, out, U, V, W, G);
  if (rc) return rc;
  if (c->halo_done) return MPDATA_OK;  // the last pass wrote the halo images
  return halo_launch<T>(c, out, MPDATA_HALO_CELL);
}

template <class T>
int step_n(mpdata_ctx* c, T* psi, const T* U, const T* V, const T* W, const T* G, int nsteps) {
  if (nsteps == 0) return MPDATA_OK;
  if (!use_fused_plain(c)) {
    for (int s = 0; s < nsteps; ++s) {
      int rc = step_staged<T>(c, psi, psi, U, V, W, G);
      if (rc) return rc;
    }
    return halo_launch<T>(c, psi, MPDATA_HALO_CELL);
  }
  // the fused kernel cannot work in place: alternate with the scratch field
  T* scratch = (T*)c->psi1;
  const T* src = psi;
  for (int s = 0; s < nsteps; ++s) {
    T* dst = (src == psi) ? scratch : psi;
    int rc = fused_launch<T>(c, src, dst, U, V, W, G);
    if (rc) return rc;
    src = dst;
  }
  if (src != psi) {  // the copy back: a kernel, so that it too overlaps its launch
    const int64_t n = c->g.total;
    const bool vec = (((uintptr_t)src | (uintptr_t)psi) & 15) == 0;
    const int64_t items = vec ? n / (16 / (int64_t)sizeof(T)) + 1 : n;
    const unsigned blocks = (unsigned)std::min<int64_t>((items + 255) / 256, 148 * 8);
    MPD_LAUNCH(c, MPDATA_STAGE_FUSED,
               mpd::launch_pdl(mpd::copy_kernel<T>, blocks, 256, 0, c->stream, src, psi,
                               n, vec));
    MPD_CHECK_LAUNCH(c, "copy-back");
  }
  return MPDATA_OK;
}

template <class T>
int mass_launch(mpdata_ctx* c, const T* psi, const T* G, double* out) {
  MPD_LAUNCH(c, MPDATA_STAGE_MASS,
             mpd::mass_partial_launch<T>(c->g, psi, G, c->part, c->stream, true));
  MPD_LAUNCH(c, MPDATA_STAGE_MASS,
             mpd::launch_pdl(mpd::mass_final_kernel, 1, 1024, 0, c->stream, c->part,
                             mpd::MASS_BLOCKS, out));
  MPD_CHECK_LAUNCH(c, "mass kernels");
  return MPDATA_OK;
}

// ------------------------------------------------------------- adjoint --

// A step's tape: one block per corrective pass m = 2..iord (one block for
// iord 1, unused): the pass's input state psi^(m-1), Ut, Vt, Wt,
// beta-up, beta-down, 1/(in+eps), 1/(out+eps), Ul, Vl, Wl.
constexpr int kTapeFields = 11;
int tape_passes(const mpdata_ctx* c) { return c->iord >= 2 ? c->iord - 1 : 1; }

// The adjoint scratch: psi1-bar (two, one per alternate pass), psi^n-bar,
// the pseudo-velocity adjoints, the carried limited-velocity adjoints
// (iord >= 3), the beta adjoints, the FP64 pseudo-velocity weights, the
// tape of mpdata_adjoint_step and its recomputed psi^(n+1).
enum {
  kAdjP1b = 0, kAdjP0b = 1, kAdjUtb = 2, kAdjCarry = 5, kAdjBub = 8, kAdjBdb = 9,
  kAdjP1b2 = 10, kAdjWts = 11, kAdjTape = 35
};

size_t field_pad(const mpdata_ctx* c) {
  return ((size_t)c->g.total * c->esize + 255) & ~(size_t)255;
}

size_t adj_fields(const mpdata_ctx* c) {
  return kAdjTape + (size_t)kTapeFields * tape_passes(c) + 1;
}

int adjoint_scratch(mpdata_ctx* c) {
  if (c->adjbuf) return MPDATA_OK;
  if (cudaMalloc(&c->adjbuf, adj_fields(c) * field_pad(c)) != cudaSuccess) {
    cudaGetLastError();
    c->adjbuf = nullptr;
    return MPDATA_ENOMEM;
  }
  c->a_out = (char*)c->adjbuf + (adj_fields(c) - 1) * field_pad(c);
  return MPDATA_OK;
}

// The block of corrective pass m (m = 2..iord) of the tape at base.
template <class T>
struct Tape {
  T *p1, *ut, *vt, *wt, *bu, *bd, *ri, *ro, *ul, *vl, *wl;
};

template <class T>
Tape<T> tape_view(const mpdata_ctx* c, const void* base, int m = 2) {
  const size_t f = field_pad(c);
  char* p = (char*)base + (size_t)(m - 2) * kTapeFields * f;
  Tape<T> t;
  T** slots[kTapeFields] = {&t.p1, &t.ut, &t.vt, &t.wt, &t.bu, &t.bd,
                            &t.ri, &t.ro, &t.ul, &t.vl, &t.wl};
  for (int q = 0; q < kTapeFields; ++q) *slots[q] = (T*)(p + q * f);
  return t;
}

template <class T>
int halo_fold_launch(mpdata_ctx* c, T* f) {
  const dim3 hg = halo_grid(c->g);
  MPD_LAUNCH(c, MPDATA_STAGE_HALO, mpd::launch_pdl(mpd::halo_fold_kernel<T>, hg, 256, 0, c->stream,
                                                   c->g, f));
  MPD_LAUNCH(c, MPDATA_STAGE_HALO, mpd::launch_pdl(mpd::halo_zero_kernel<T>, hg, 256, 0, c->stream,
                                                   c->g, f));
  MPD_CHECK_LAUNCH(c, "halo adjoint fold");
  return MPDATA_OK;
}

// One forward step psi_in -> psi_out that keeps its intermediates in the
// tape at base: the fused kernel where the plain step would run it (iord
// 2), else the staged kernels, pass by pass.
template <class T>
int step_tape(mpdata_ctx* c, const T* psi, T* out, const T* U, const T* V, const T* W,
              const T* G, const void* base) {
  using namespace mpd::staged;
  if (use_fused(c)) {  // the fused step writes the tape and the output's halo itself
    const Tape<T> tp = tape_view<T>(c, base);
    const mpd::fused2::TapeOut<T> to{tp.p1, tp.ut, tp.vt, tp.wt, tp.bu, tp.bd,
                                     tp.ri, tp.ro, tp.ul, tp.vl, tp.wl};
    return fused_launch<T>(c, psi, out, U, V, W, G, &to);
  }
  const Geo& g = c->g;
  const dim3 grid = cell_grid(g);
  cudaStream_t s = c->stream;
  T *fx = (T*)c->fx, *fy = (T*)c->fy, *fz = (T*)c->fz;
  MPD_LAUNCH(c, MPDATA_STAGE_DONOR, mpd::launch_pdl(flux_kernel<T>, grid, kCellBlock, 0, s, g, psi,
                                                    U, V, W, fx, fy, fz, nullptr, nullptr));
  if (c->iord == 1) {
    MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE, mpd::launch_pdl(advance_kernel<T>, grid, kCellBlock, 0, s,
                                                        g, psi, fx, fy, fz, G, out, nullptr));
  } else {
    MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
               mpd::launch_pdl(advance_kernel<T>, grid, kCellBlock, 0, s, g, psi, fx, fy, fz, G,
                               tape_view<T>(c, base, 2).p1, nullptr));
    const T *cu = U, *cv = V, *cw = W;  // the pass's input velocities
    // FP64: the pseudo-velocity stage stores the donor fluxes too, as in
    // the plain staged step (the same kernels, so the same bits)
    constexpr bool kFin = std::is_same<T, double>::value;
    for (int m = 2; m <= c->iord; ++m) {
      const Tape<T> tp = tape_view<T>(c, base, m);
      T* dest = m == c->iord ? out : tape_view<T>(c, base, m + 1).p1;
      pseudo_launch<T, 0, kFin>(c, tp.p1, cu, cv, cw, G, tp.ut, tp.vt, tp.wt, fx, fy, fz);
      if (c->nonosc) {
        const T* bf[3] = {kFin ? fx : tp.ut, kFin ? fy : tp.vt, kFin ? fz : tp.wt};
        MPD_LAUNCH(c, MPDATA_STAGE_BETA,
                   (mpd::launch_pdl(beta_kernel<T, kFin>, grid, kCellBlock, 0, s, g, psi, tp.p1,
                                    bf[0], bf[1], bf[2], G, tp.bu, tp.bd, tp.ri, tp.ro)));
        MPD_LAUNCH(c, MPDATA_STAGE_LIMIT,
                   (mpd::launch_pdl(limflux_kernel<T, 0, kFin>, grid, kCellBlock, 0, s, g, tp.p1,
                                    tp.ut, tp.vt, tp.wt, tp.bu, tp.bd, fx, fy, fz, tp.ul, tp.vl,
                                    tp.wl)));
        cu = tp.ul; cv = tp.vl; cw = tp.wl;
      } else {
        if (!kFin)
          MPD_LAUNCH(c, MPDATA_STAGE_LIMIT,
                     mpd::launch_pdl(flux_kernel<T>, grid, kCellBlock, 0, s, g, tp.p1, tp.ut, tp.vt,
                                     tp.wt, fx, fy, fz, nullptr, nullptr));
        cu = tp.ut; cv = tp.vt; cw = tp.wt;
      }
      MPD_LAUNCH(c, MPDATA_STAGE_ADVANCE,
                 mpd::launch_pdl(advance_kernel<T>, grid, kCellBlock, 0, s, g, tp.p1, fx, fy, fz, G,
                                 dest, nullptr));
    }
  }
  MPD_CHECK_LAUNCH(c, "taped forward step");
  return halo_launch<T>(c, out, MPDATA_HALO_CELL);
}

// The reverse kernels of one step, from its tape: the corrective passes in
// reverse order, then the donor pass.  Pass m's pseudo-velocity reverse
// gives the adjoint of its input velocities: U, V, W (into ub, vb, wb) for
// m = 2, else the limited velocities of pass m-1, carried to that pass's
// advance reverse.
template <class T>
int adjoint_tape(mpdata_ctx* c, const void* tape, const T* psi, const T* U, const T* V,
                 const T* W, const T* G, T* psib, T* ub, T* vb, T* wb) {
  using namespace mpd::adj;
  int rc = adjoint_scratch(c);
  if (rc) return rc;
  const Geo& g = c->g;
  const dim3 grid = cell_grid(g);
  cudaStream_t s = c->stream;
  const size_t f = field_pad(c);
  char* base = (char*)c->adjbuf;
  auto field = [&](int q) { return (T*)(base + (size_t)q * f); };
  T *p0b = field(kAdjP0b), *utb = field(kAdjUtb), *vtb = field(kAdjUtb + 1);
  T* wtb = field(kAdjUtb + 2);
  T *cub = field(kAdjCarry), *cvb = field(kAdjCarry + 1), *cwb = field(kAdjCarry + 2);
  T *bub = field(kAdjBub), *bdb = field(kAdjBdb);
  T* pbuf[2] = {field(kAdjP1b), field(kAdjP1b2)};  // psi^(m-1)-bar, alternating
  T* wts = field(kAdjWts);                         // 24 weight fields, g.total apart
  const size_t fb = (size_t)g.total * sizeof(T);
  // The gather-form advance reverses store their outputs; only the fields
  // that atomic scatters reach first must start at zero: p0b (beta-bound
  // adjoints, then the donor reverse adds) and the beta adjoints.  Their
  // only readers (the donor reverse, the beta reverse) clear them again, so
  // they are cleared here only on the first step or after a failed one.
  if (c->iord >= 2 && !c->adj_zero) {
    T* zero_list[3] = {p0b, bub, bdb};
    for (int q = 0; q < 3; ++q) {
      cudaError_t e = cudaMemsetAsync(zero_list[q], 0, fb, s);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint clear");
    }
  }
  c->adj_zero = false;
  // gather-form advance reverse: FP32 forms s = ob/G on the fly, FP64 reads
  // it from a pre-pass (wts is free while the advance reverses run)
  constexpr bool kPreS = std::is_same<T, double>::value;
  T* sf = wts;
  auto adv = [&](int stage, const T* P, const T* cu_, const T* cv_, const T* cw_, const T* ob,
                 T* Pin, T* Pb, auto out, auto add_p) {
    constexpr bool kAddP = decltype(add_p)::value;
    if (kPreS)
      MPD_LAUNCH(c, stage, mpd::launch_pdl(rev_scale_kernel<T>, grid, kCellBlock, 0, s, g, ob, G,
                                           sf));
    MPD_LAUNCH(c, stage,
               (mpd::launch_pdl(rev_advance_gather_kernel<T, kAddP, kPreS, decltype(out)>, grid,
                                kCellBlock, 0, s, g, P, cu_, cv_, cw_, G, ob, sf, Pin, Pb, out)));
  };
  using Store = std::false_type;
  using Add = std::true_type;
  if (c->iord == 1) {
    adv(MPDATA_STAGE_ADVANCE, psi, U, V, W, psib, nullptr, p0b,
        VelOut<T, true>{ub, vb, wb, nullptr, nullptr, nullptr}, Store{});
  } else {
    const T* ob = psib;  // adjoint of the pass's output state
    for (int m = c->iord; m >= 2; --m) {
      const Tape<T> tp = tape_view<T>(c, tape, m);
      T* Pb = pbuf[(c->iord - m) & 1];
      // adjoint of this pass's limited velocities from the pass above
      const bool carried = m < c->iord;
      const T *au = carried ? cub : nullptr, *av = carried ? cvb : nullptr;
      const T* aw = carried ? cwb : nullptr;
      if (c->nonosc) {  // the limiter reverse rides on the final advance reverse
        adv(MPDATA_STAGE_ADVANCE, tp.p1, tp.ul, tp.vl, tp.wl, ob, nullptr, Pb,
            LimitOut<T>{tp.ut, tp.vt, tp.wt, tp.bu, tp.bd, utb, vtb, wtb, bub, bdb, au, av, aw},
            Store{});
        MPD_LAUNCH(c, MPDATA_STAGE_BETA, mpd::launch_pdl(rev_beta_kernel<T>, grid, kCellBlock, 0, s,
                                                         g, psi, tp.p1, tp.ut, tp.vt, tp.wt, G,
                                                         tp.bu, tp.bd, tp.ri, tp.ro, bub, bdb, p0b,
                                                         Pb, utb, vtb, wtb));
      } else {
        adv(MPDATA_STAGE_ADVANCE, tp.p1, tp.ut, tp.vt, tp.wt, ob, nullptr, Pb,
            VelOut<T, false>{utb, vtb, wtb, au, av, aw}, Store{});
      }
      // the pass's input velocities and where their adjoints go
      const bool first = m == 2;
      const Tape<T> below = tape_view<T>(c, tape, first ? 2 : m - 1);
      const T* iu = first ? U : (c->nonosc ? below.ul : below.ut);
      const T* iv = first ? V : (c->nonosc ? below.vl : below.vt);
      const T* iw = first ? W : (c->nonosc ? below.wl : below.wt);
      T *tu = first ? ub : cub, *tv = first ? vb : cvb, *tw = first ? wb : cwb;
      if (!first) {  // the carry was read above: clear it for the pass below
        T* carry[3] = {cub, cvb, cwb};
        for (int q = 0; q < 3; ++q) {
          cudaError_t e = cudaMemsetAsync(carry[q], 0, fb, s);
          if (e != cudaSuccess) return cuda_fail(c, e, "adjoint carry clear");
        }
      }
      namespace M = mpd::march;
      if constexpr (std::is_same<T, float>::value) {
        // one pass, shared accumulators
        auto kern = M::march_kernel<T, RevPseudoAcc<T>>;
        if (!c->kc_rev) c->kc_rev = march_chunk(c, kern, false);
        const RevPseudoAcc<T> op{utb, vtb, wtb, Pb, tu, tv, tw};
        MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
                   mpd::launch_pdl(kern, M::march_grid(g, c->kc_rev), dim3(M::TX, M::TY), 0, s, g,
                                   tp.p1, iu, iv, iw, G, op, c->kc_rev));
      } else {
        auto kern = M::march_kernel<T, RevPseudo<T>>;
        if (!c->kc_rev) c->kc_rev = march_chunk(c, kern, true);
        const RevPseudo<T> op{utb, vtb, wtb, wts, g.total, tu, tv, tw};
        MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
                   mpd::launch_pdl(kern, M::march_grid(g, c->kc_rev), dim3(M::TX, M::TY), 0, s, g,
                                   tp.p1, iu, iv, iw, G, op, c->kc_rev));
        MPD_LAUNCH(c, MPDATA_STAGE_PSEUDO,
                   mpd::launch_pdl(rev_pg_kernel<T>, grid, kCellBlock, 0, s, g, wts, Pb, tu, tv,
                                   tw));
      }
      ob = Pb;
    }
    // psib (read last by the final advance reverse) takes the result
    // directly; p0b is cleared as it is read
    adv(MPDATA_STAGE_DONOR, psi, U, V, W, ob, p0b, psib,
        VelOut<T, true>{ub, vb, wb, nullptr, nullptr, nullptr}, Add{});
  }
  if (c->iord == 1) {  // there the reverse read psib while writing p0b
    cudaError_t e = cudaMemcpyAsync(psib, p0b, fb, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint result copy");
  } else {  // psib's interior holds the result; its halo is cleared
    MPD_LAUNCH(c, MPDATA_STAGE_HALO,
               mpd::launch_pdl(mpd::halo_zero_kernel<T>, halo_grid(g), 256, 0, s, g, psib));
  }
  MPD_CHECK_LAUNCH(c, "adjoint reverse kernels");
  c->adj_zero = true;
  return MPDATA_OK;
}

// One adjoint step with its own forward recompute (into the internal tape).
template <class T>
int adjoint_step(mpdata_ctx* c, const T* psi, const T* U, const T* V, const T* W, const T* G,
                 T* psib, T* ub, T* vb, T* wb) {
  int rc = adjoint_scratch(c);
  if (rc) return rc;
  const void* tape = (char*)c->adjbuf + (size_t)kAdjTape * field_pad(c);
  // the recomputed psi^(n+1) goes to the context's second psi scratch
  T* out = (T*)c->a_out;
  if ((rc = step_tape<T>(c, psi, out, U, V, W, G, tape))) return rc;
  return adjoint_tape<T>(c, tape, psi, U, V, W, G, psib, ub, vb, wb);
}

int check_fields(const void* const* ptrs, int n) {
  for (int q = 0; q < n; ++q) {
    if (!ptrs[q]) return MPDATA_EINVAL;
    if (!aligned16(ptrs[q])) return MPDATA_EALIGN;
  }
  return MPDATA_OK;
}

// One halo strip of a slab: field -> buffer (pack) or buffer -> field.
template <class T, bool UNPACK>
int strip_launch(mpdata_ctx* c, const void* src, void* dst, int face) {
  const mpd::xch::Strip st = mpd::xch::strip(c->g, face, UNPACK);
  if (st.n == 0) return MPDATA_OK;
  const int64_t want = (st.n + 255) / 256;
  const int blocks = (int)(want < 148 * 8 ? want : 148 * 8);
  MPD_LAUNCH(c, MPDATA_STAGE_EXCHANGE,
             (mpd::xch::strip_kernel<T, UNPACK><<<blocks, 256, 0, c->stream>>>(
                 c->g, st, (const T*)src, (T*)dst)));
  MPD_CHECK_LAUNCH(c, "halo strip kernel");
  return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* mpdata_strerror(int code) {
  switch (code) {
    case MPDATA_OK: return "ok";
    case MPDATA_EINVAL: return "invalid argument (size, option or null pointer)";
    case MPDATA_ENOMEM: return "device allocation failed";
    case MPDATA_ECUDA: return "CUDA runtime error";
    case MPDATA_EALIGN: return "field pointer not 16-byte aligned";
    case MPDATA_EDEVICE: return "no usable CUDA device";
    case MPDATA_ERANGE: return "size beyond the documented maximum";
    default: return "unknown status";
  }
}

const char* mpdata_last_error_string(mpdata_ctx* c) { return c ? c->err : ""; }

int mpdata_init(mpdata_ctx** out, int nx, int ny, int nz, int halo, int iord, int nonosc,
                int dtype, int k_bc, void* stream) {
  if (!out) return MPDATA_EINVAL;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || halo < 1 || iord < 1 || iord > 8) return MPDATA_EINVAL;
  if (iord >= 2 && halo < 2) return MPDATA_EINVAL;
  if (nonosc != 0 && nonosc != 1) return MPDATA_EINVAL;
  if (dtype != MPDATA_F64 && dtype != MPDATA_F32) return MPDATA_EINVAL;
  if (k_bc != MPDATA_K_ZEROFLUX && k_bc != MPDATA_K_PERIODIC) return MPDATA_EINVAL;
  if (nz > 65535) return MPDATA_ERANGE;
  // padded extents must fit the 32-bit index arithmetic of a row/plane
  if ((int64_t)(nx + 2 * halo) * (ny + 2 * halo) > (int64_t)1 << 31) return MPDATA_ERANGE;
  // the mass reduction counts interior rows (j, k) in 32 bits
  if ((int64_t)ny * nz > MPDATA_MASS_MAX_ROWS) return MPDATA_ERANGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MPDATA_EDEVICE;
  mpdata_ctx* c = new (std::nothrow) mpdata_ctx();
  if (!c) return MPDATA_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->g = mpd::make_geo(nx, ny, nz, halo, k_bc == MPDATA_K_PERIODIC ? 1 : 0);
  c->iord = iord;
  c->nonosc = nonosc;
  c->dtype = dtype;
  c->kbc = k_bc;
  c->variant = MPDATA_AUTO;
  c->device = dev;
  c->esize = dtype == MPDATA_F64 ? 8 : 4;
  c->stream = (cudaStream_t)stream;
  const size_t fbytes = ((size_t)c->g.total * c->esize + 255) & ~(size_t)255;
  const int nfields = iord >= 2 ? (iord >= 3 ? 13 : 9) : 3;
  const int nrg = (dtype == MPDATA_F64 && iord >= 2) ? 1 : 0;
  const size_t bytes = fbytes * (nfields + nrg) + sizeof(double) * mpd::MASS_BLOCKS;
  if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MPDATA_ENOMEM;
  }
  char* p = (char*)c->scratch;
  void** slots[13] = {&c->fx, &c->fy, &c->fz, &c->psi1, &c->ut, &c->vt, &c->wt, &c->bu,
                      &c->bd, &c->psi2, &c->ul, &c->vl, &c->wl};
  for (int q = 0; q < nfields; ++q) *slots[q] = p + q * fbytes;
  c->rg = nrg ? p + nfields * fbytes : nullptr;
  c->part = (double*)(p + (nfields + nrg) * fbytes);
  if (dtype == MPDATA_F64) fused_setup<double>(c); else fused_setup<float>(c);
  *out = c;
  return MPDATA_OK;
}

int mpdata_set_stream(mpdata_ctx* c, void* stream) {
  if (!c) return MPDATA_EINVAL;
  c->stream = (cudaStream_t)stream;
  return MPDATA_OK;
}

int mpdata_set_variant(mpdata_ctx* c, int variant) {
  if (!c || variant < MPDATA_FUSED || variant > MPDATA_AUTO) return MPDATA_EINVAL;
  c->variant = variant;
  return MPDATA_OK;
}

int mpdata_set_options(mpdata_ctx* c, int opts) {
  if (!c) return MPDATA_EINVAL;
  const int all = MPDATA_OPT_DFL | MPDATA_OPT_ABS | MPDATA_OPT_IGA;
  if (opts & ~all) return fail(c, MPDATA_EINVAL, "unknown option bits");
  if (opts && c->g.openij) return fail(c, MPDATA_EINVAL, "a slab takes no option");
  if ((opts & MPDATA_OPT_IGA) && (opts & (MPDATA_OPT_DFL | MPDATA_OPT_ABS)))
    return fail(c, MPDATA_EINVAL, "the infinite gauge takes no other option");
  if ((opts & MPDATA_OPT_IGA) && c->iord > 2)
    return fail(c, MPDATA_EINVAL, "the infinite gauge is defined for iord <= 2");
  const int prev = c->opts;
  c->opts = opts;
  if (c->dtype == MPDATA_F32 && c->fused_ok) {  // the option instance's shared memory
    const int ib = (int)fused_smem<float>();
    if (cudaFuncSetAttribute(fused_pick<float, false>(c),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, ib) != cudaSuccess) {
      cudaGetLastError();
      c->opts = prev;
      return fail(c, MPDATA_ECUDA, "fused kernel attribute");
    }
    fusedx_setup(c);  // the two-column kernel's instance for these options
  }
  return MPDATA_OK;
}

int mpdata_get_options(mpdata_ctx* c, int* opts) {
  if (!c || !opts) return MPDATA_EINVAL;
  *opts = c->opts;
  return MPDATA_OK;
}

int mpdata_step(mpdata_ctx* c, void* psi, const void* u, const void* v, const void* w,
                const void* g, int nsteps) {
  if (!c || nsteps < 0) return MPDATA_EINVAL;
  if (c->g.openij && !c->fused_ok) return fail(c, MPDATA_EINVAL, "slab without its step kernel");
  const void* f[5] = {psi, u, v, w, g};
  int rc = check_fields(f, 5);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64)
    return step_n<double>(c, (double*)psi, (const double*)u, (const double*)v,
                          (const double*)w, (const double*)g, nsteps);
  return step_n<float>(c, (float*)psi, (const float*)u, (const float*)v, (const float*)w,
                       (const float*)g, nsteps);
}

int mpdata_step_out(mpdata_ctx* c, const void* psi_in, void* psi_out, const void* u,
                    const void* v, const void* w, const void* g) {
  if (!c) return MPDATA_EINVAL;
  if (c->g.openij && !c->fused_ok) return fail(c, MPDATA_EINVAL, "slab without its step kernel");
  const void* f[6] = {psi_in, psi_out, u, v, w, g};
  int rc = check_fields(f, 6);
  if (rc) return rc;
  if (psi_in == psi_out) return MPDATA_EINVAL;
  if (c->dtype == MPDATA_F64)
    return step_out<double>(c, (const double*)psi_in, (double*)psi_out, (const double*)u,
                            (const double*)v, (const double*)w, (const double*)g);
  return step_out<float>(c, (const float*)psi_in, (float*)psi_out, (const float*)u,
                         (const float*)v, (const float*)w, (const float*)g);
}

int mpdata_step_host(mpdata_ctx* c, void* psi_h, const void* u_h, const void* v_h,
                     const void* w_h, const void* g_h, int nsteps) {
  if (!c || nsteps < 0 || !psi_h || !u_h || !v_h || !w_h || !g_h) return MPDATA_EINVAL;
  const size_t fbytes = (size_t)c->g.total * c->esize;
  const size_t fpad = (fbytes + 255) & ~(size_t)255;
  if (!c->hbuf) {
    if (cudaMalloc(&c->hbuf, 5 * fpad) != cudaSuccess) {
      cudaGetLastError();
      c->hbuf = nullptr;
      return MPDATA_ENOMEM;
    }
  }
  char* d = (char*)c->hbuf;
  const void* src[5] = {psi_h, u_h, v_h, w_h, g_h};
  for (int q = 0; q < 5; ++q) {
    cudaError_t e = cudaMemcpyAsync(d + q * fpad, src[q], fbytes, cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  }
  int rc = mpdata_step(c, d, d + fpad, d + 2 * fpad, d + 3 * fpad, d + 4 * fpad, nsteps);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(psi_h, d, fbytes, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  return MPDATA_OK;
}

namespace {
// A 3D copy between a field's interior in padded device storage and a host
// array of the interior alone (nx*ny*nz, i fastest): rows of nx elements,
// the padded side at its row and plane pitches.
cudaError_t interior_copy(const mpdata_ctx* c, void* dev_field, void* host, bool to_device,
                          cudaStream_t s) {
  const Geo& g = c->g;
  const size_t es = c->esize;
  char* origin = (char*)dev_field + (size_t)g.off0 * es;
  cudaMemcpy3DParms p = {};
  cudaPitchedPtr dev = make_cudaPitchedPtr(origin, (size_t)g.px * es, (size_t)g.nx,
                                           (size_t)(g.pxy / g.px));
  cudaPitchedPtr hst = make_cudaPitchedPtr(host, (size_t)g.nx * es, (size_t)g.nx, (size_t)g.ny);
  p.srcPtr = to_device ? hst : dev;
  p.dstPtr = to_device ? dev : hst;
  p.extent = make_cudaExtent((size_t)g.nx * es, (size_t)g.ny, (size_t)g.nz);
  p.kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
  return cudaMemcpy3DAsync(&p, s);
}

// The pipelined host-buffer steps, with padded host fields or, interior,
// with host arrays of the interior alone.
int host_async(mpdata_ctx* c, const void* psi_in_h, void* psi_out_h, const void* u_h,
               const void* v_h, const void* w_h, const void* g_h, int nsteps, bool interior) {
  if (!c || nsteps < 0 || !psi_in_h || !psi_out_h || !u_h || !v_h || !w_h || !g_h)
    return MPDATA_EINVAL;
  if (interior && c->g.openij)
    return fail(c, MPDATA_EINVAL, "a slab takes its halo from the halo exchange");
  const size_t fbytes = (size_t)c->g.total * c->esize;
  const size_t fpad = (fbytes + 255) & ~(size_t)255;
  cudaError_t e;
  if (!c->pbuf) {
    if (cudaMalloc(&c->pbuf, 10 * fpad) != cudaSuccess) {
      cudaGetLastError();
      c->pbuf = nullptr;
      return MPDATA_ENOMEM;
    }
    bool ok = cudaStreamCreateWithFlags(&c->ps_in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->ps_out, cudaStreamNonBlocking) == cudaSuccess;
    for (int q = 0; q < 2 && ok; ++q)
      ok = cudaEventCreateWithFlags(&c->pe_in[q], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->pe_step[q], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->pe_out[q], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {  // undo the partial set-up, so that a later call starts afresh
      e = cudaGetLastError();
      for (int q = 0; q < 2; ++q) {
        if (c->pe_in[q]) cudaEventDestroy(c->pe_in[q]);
        if (c->pe_step[q]) cudaEventDestroy(c->pe_step[q]);
        if (c->pe_out[q]) cudaEventDestroy(c->pe_out[q]);
        c->pe_in[q] = c->pe_step[q] = c->pe_out[q] = nullptr;
      }
      if (c->ps_in) cudaStreamDestroy(c->ps_in);
      if (c->ps_out) cudaStreamDestroy(c->ps_out);
      c->ps_in = c->ps_out = nullptr;
      cudaFree(c->pbuf);
      c->pbuf = nullptr;
      return cuda_fail(c, e, "pipeline streams");
    }
    c->pslot = 0;
    c->pused[0] = c->pused[1] = false;
  }
  const int b = c->pslot;
  char* d = (char*)c->pbuf + (size_t)b * 5 * fpad;
  // the set's previous problem must have been copied back before its
  // fields are overwritten
  if (c->pused[b] && (e = cudaStreamWaitEvent(c->ps_in, c->pe_out[b], 0)) != cudaSuccess)
    return cuda_fail(c, e, "pipeline wait");
  const void* src[5] = {psi_in_h, u_h, v_h, w_h, g_h};
  // (interior: the step reads no input halo, so only the interior crosses)
  for (int q = 0; q < 5; ++q) {
    e = interior ? interior_copy(c, d + q * fpad, const_cast<void*>(src[q]), true, c->ps_in)
                 : cudaMemcpyAsync(d + q * fpad, src[q], fbytes, cudaMemcpyHostToDevice, c->ps_in);
    if (e != cudaSuccess) return cuda_fail(c, e, "host-to-device copy");
  }
  if ((e = cudaEventRecord(c->pe_in[b], c->ps_in)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(c->stream, c->pe_in[b], 0)) != cudaSuccess)
    return cuda_fail(c, e, "pipeline events");
  int rc = mpdata_step(c, d, d + fpad, d + 2 * fpad, d + 3 * fpad, d + 4 * fpad, nsteps);
  if (rc) return rc;
  if ((e = cudaEventRecord(c->pe_step[b], c->stream)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(c->ps_out, c->pe_step[b], 0)) != cudaSuccess)
    return cuda_fail(c, e, "pipeline events");
  e = interior ? interior_copy(c, d, psi_out_h, false, c->ps_out)
               : cudaMemcpyAsync(psi_out_h, d, fbytes, cudaMemcpyDeviceToHost, c->ps_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "device-to-host copy");
  if ((e = cudaEventRecord(c->pe_out[b], c->ps_out)) != cudaSuccess)
    return cuda_fail(c, e, "pipeline events");
  c->pused[b] = true;
  c->pslot = b ^ 1;
  return MPDATA_OK;
}
}  // namespace

int mpdata_step_host_async(mpdata_ctx* c, const void* psi_in_h, void* psi_out_h, const void* u_h,
                           const void* v_h, const void* w_h, const void* g_h, int nsteps) {
  return host_async(c, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps, false);
}

int mpdata_step_host_interior_async(mpdata_ctx* c, const void* psi_in_h, void* psi_out_h,
                                    const void* u_h, const void* v_h, const void* w_h,
                                    const void* g_h, int nsteps) {
  return host_async(c, psi_in_h, psi_out_h, u_h, v_h, w_h, g_h, nsteps, true);
}

int mpdata_host_wait(mpdata_ctx* c) {
  if (!c) return MPDATA_EINVAL;
  if (!c->pbuf) return MPDATA_OK;
  cudaError_t e = cudaStreamSynchronize(c->ps_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "pipeline synchronize");
  return MPDATA_OK;
}

int mpdata_fill_halo(mpdata_ctx* c, void* field, int kind) {
  if (!c || (kind != MPDATA_HALO_CELL && kind != MPDATA_HALO_WFACE)) return MPDATA_EINVAL;
  if (c->g.openij) return fail(c, MPDATA_EINVAL, "a slab's halo comes from the halo exchange");
  const void* f[1] = {field};
  int rc = check_fields(f, 1);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64) return halo_launch<double>(c, (double*)field, kind);
  return halo_launch<float>(c, (float*)field, kind);
}

int mpdata_mass(mpdata_ctx* c, const void* psi, const void* g, double* out_dev) {
  if (!c || !out_dev) return MPDATA_EINVAL;
  const void* f[2] = {psi, g};
  int rc = check_fields(f, 2);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64)
    return mass_launch<double>(c, (const double*)psi, (const double*)g, out_dev);
  return mass_launch<float>(c, (const float*)psi, (const float*)g, out_dev);
}

long long mpdata_launch_count(mpdata_ctx* c) { return c ? c->launches : -1; }

int mpdata_profile(mpdata_ctx* c, int enable) {
  if (!c) return MPDATA_EINVAL;
  if (enable && !c->prof_ev) {
    const int cap = 8192;
    c->prof_ev = new (std::nothrow) cudaEvent_t[2 * cap];
    c->prof_stage = new (std::nothrow) int[cap];
    if (!c->prof_ev || !c->prof_stage) return MPDATA_ENOMEM;
    for (int q = 0; q < 2 * cap; ++q) {
      cudaError_t e = cudaEventCreate(&c->prof_ev[q]);
      if (e != cudaSuccess) {
        for (int r = 0; r < q; ++r) cudaEventDestroy(c->prof_ev[r]);
        delete[] c->prof_ev;
        c->prof_ev = nullptr;
        return cuda_fail(c, e, "cudaEventCreate");
      }
    }
    c->prof_cap = cap;
  }
  if (enable) c->prof_n = 0;
  c->prof_on = enable != 0;
  return MPDATA_OK;
}

int mpdata_profile_read(mpdata_ctx* c, int stage, double* ms, int* launches) {
  if (!c || !ms || !launches || stage < 0 || stage >= MPDATA_NSTAGES) return MPDATA_EINVAL;
  *ms = 0.0;
  *launches = 0;
  if (!c->prof_ev) return MPDATA_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  for (int q = 0; q < c->prof_n; ++q) {
    if (c->prof_stage[q] != stage) continue;
    float t = 0.f;
    e = cudaEventElapsedTime(&t, c->prof_ev[2 * q], c->prof_ev[2 * q + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
    *ms += t;
    ++*launches;
  }
  return MPDATA_OK;
}

int mpdata_adjoint_step(mpdata_ctx* c, const void* psi_n, const void* u, const void* v,
                        const void* w, const void* g, void* psi_bar, void* u_bar, void* v_bar,
                        void* w_bar) {
  if (!c) return MPDATA_EINVAL;
  if (c->g.openij) return fail(c, MPDATA_EINVAL, "a slab has no adjoint");
  if (c->opts) return fail(c, MPDATA_EINVAL, "options have no adjoint");
  const void* f[9] = {psi_n, u, v, w, g, psi_bar, u_bar, v_bar, w_bar};
  int rc = check_fields(f, 9);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64)
    return adjoint_step<double>(c, (const double*)psi_n, (const double*)u, (const double*)v,
                                (const double*)w, (const double*)g, (double*)psi_bar,
                                (double*)u_bar, (double*)v_bar, (double*)w_bar);
  return adjoint_step<float>(c, (const float*)psi_n, (const float*)u, (const float*)v,
                             (const float*)w, (const float*)g, (float*)psi_bar, (float*)u_bar,
                             (float*)v_bar, (float*)w_bar);
}

int mpdata_tape_bytes(mpdata_ctx* c, size_t* bytes) {
  if (!c || !bytes) return MPDATA_EINVAL;
  *bytes = (size_t)kTapeFields * tape_passes(c) * field_pad(c);
  return MPDATA_OK;
}

int mpdata_step_tape(mpdata_ctx* c, const void* psi_in, void* psi_out, const void* u,
                     const void* v, const void* w, const void* g, void* tape) {
  if (!c) return MPDATA_EINVAL;
  if (c->g.openij) return fail(c, MPDATA_EINVAL, "a slab has no adjoint");
  if (c->opts) return fail(c, MPDATA_EINVAL, "options have no adjoint");
  const void* f[7] = {psi_in, psi_out, u, v, w, g, tape};
  int rc = check_fields(f, 7);
  if (rc) return rc;
  if (psi_in == psi_out) return MPDATA_EINVAL;
  if (c->dtype == MPDATA_F64)
    return step_tape<double>(c, (const double*)psi_in, (double*)psi_out, (const double*)u,
                             (const double*)v, (const double*)w, (const double*)g, tape);
  return step_tape<float>(c, (const float*)psi_in, (float*)psi_out, (const float*)u,
                          (const float*)v, (const float*)w, (const float*)g, tape);
}

int mpdata_adjoint_step_tape(mpdata_ctx* c, const void* tape, const void* psi_n, const void* u,
                             const void* v, const void* w, const void* g, void* psi_bar,
                             void* u_bar, void* v_bar, void* w_bar) {
  if (!c) return MPDATA_EINVAL;
  if (c->g.openij) return fail(c, MPDATA_EINVAL, "a slab has no adjoint");
  if (c->opts) return fail(c, MPDATA_EINVAL, "options have no adjoint");
  const void* f[10] = {tape, psi_n, u, v, w, g, psi_bar, u_bar, v_bar, w_bar};
  int rc = check_fields(f, 10);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64)
    return adjoint_tape<double>(c, tape, (const double*)psi_n,
                                (const double*)u, (const double*)v, (const double*)w,
                                (const double*)g, (double*)psi_bar, (double*)u_bar,
                                (double*)v_bar, (double*)w_bar);
  return adjoint_tape<float>(c, tape, (const float*)psi_n,
                             (const float*)u, (const float*)v, (const float*)w, (const float*)g,
                             (float*)psi_bar, (float*)u_bar, (float*)v_bar, (float*)w_bar);
}

int mpdata_fold_halo_adjoint(mpdata_ctx* c, void* field) {
  if (!c) return MPDATA_EINVAL;
  if (c->g.openij) return fail(c, MPDATA_EINVAL, "a slab has no adjoint");
  const void* f[1] = {field};
  int rc = check_fields(f, 1);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64) return halo_fold_launch<double>(c, (double*)field);
  return halo_fold_launch<float>(c, (float*)field);
}

int mpdata_set_ij_boundary(mpdata_ctx* c, int mode) {
  if (!c || (mode != MPDATA_IJ_PERIODIC && mode != MPDATA_IJ_HALO)) return MPDATA_EINVAL;
  if (mode == MPDATA_IJ_HALO) {
    if (c->iord != 2) return fail(c, MPDATA_EINVAL, "a slab runs the one-kernel step: iord 2");
    if (c->g.h < 3) return fail(c, MPDATA_EINVAL, "a slab needs a halo of at least 3");
    if (c->opts) return fail(c, MPDATA_EINVAL, "a slab takes no option");
    if (c->g.nx < c->g.h || c->g.ny < c->g.h)
      return fail(c, MPDATA_EINVAL, "a slab must be at least as wide as its halo");
  }
  const int prev = c->g.openij;
  c->g.openij = mode == MPDATA_IJ_HALO ? 1 : 0;
  if (c->dtype == MPDATA_F64) fused_setup<double>(c); else fused_setup<float>(c);
  if (c->g.openij && !c->fused_ok) {
    c->g.openij = prev;
    if (c->dtype == MPDATA_F64) fused_setup<double>(c); else fused_setup<float>(c);
    return fail(c, MPDATA_ECUDA, "the one-kernel step cannot run on this device");
  }
  return MPDATA_OK;
}

int mpdata_halo_strip_elems(mpdata_ctx* c, int face, long long* n) {
  if (!c || !n || face < 0 || face > 3) return MPDATA_EINVAL;
  *n = (long long)mpd::xch::strip(c->g, face, false).n;
  return MPDATA_OK;
}


int mpdata_halo_pack(mpdata_ctx* c, const void* field, int face, void* buf) {
  if (!c || face < 0 || face > 3) return MPDATA_EINVAL;
  const void* f[2] = {field, buf};
  int rc = check_fields(f, 2);
  if (rc) return rc;
  if (c->dtype == MPDATA_F64) return strip_launch<double, false>(c, field, buf, face);
  return strip_launch<float, false>(c, field, buf, face);
}

int mpdata_halo_unpack(mpdata_ctx* c, const void* buf, int face, void* field) {
  if (!c || face < 0 || face > 3) return MPDATA_EINVAL;
  const void* f[2] = {buf, field};
  int rc = check_fields(f, 2);
  if (rc) return rc;
  if (buf == field) return MPDATA_EINVAL;
  if (c->dtype == MPDATA_F64) return strip_launch<double, true>(c, buf, field, face);
  return strip_launch<float, true>(c, buf, field, face);
}

void mpdata_destroy(mpdata_ctx* c) {
  if (!c) return;
  if (c->adjbuf) cudaFree(c->adjbuf);
  if (c->prof_ev) {
    for (int q = 0; q < 2 * c->prof_cap; ++q) cudaEventDestroy(c->prof_ev[q]);
    delete[] c->prof_ev;
    delete[] c->prof_stage;
  }
  if (c->scratch) cudaFree(c->scratch);
  if (c->hbuf) cudaFree(c->hbuf);
  if (c->pbuf) {
    cudaStreamSynchronize(c->ps_out);
    for (int q = 0; q < 2; ++q) {
      if (c->pe_in[q]) cudaEventDestroy(c->pe_in[q]);
      if (c->pe_step[q]) cudaEventDestroy(c->pe_step[q]);
      if (c->pe_out[q]) cudaEventDestroy(c->pe_out[q]);
    }
    if (c->ps_in) cudaStreamDestroy(c->ps_in);
    if (c->ps_out) cudaStreamDestroy(c->ps_out);
    cudaFree(c->pbuf);
  }
  delete c;
}

}  // extern "C"
