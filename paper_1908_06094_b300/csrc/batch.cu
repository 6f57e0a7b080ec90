// batch.cu -- many independent MPDATA problems in one persistent launch.
//
// A batch holds domains of different sizes, each with several tracers that
// share the domain's Courant fields and metric.  One step of every tracer of
// every domain is one launch of a persistent kernel: SMs x occupancy CTAs
// pull work items (domain, column tile, level chunk, tracer) from an atomic
// counter until the list is exhausted, and run the fused step on each item.
// Items of the same tile and chunk are consecutive for all tracers, so the
// CTAs working on them at the same time read the shared U, V, W, G columns
// through L2 once rather than once per tracer; uneven domain sizes are
// balanced by the queue.  The launch (counter reset + kernel) is captured in
// a CUDA graph per ping-pong direction and replayed.
//
// The tile shape (one of the compiled instances below) and the chunk length
// are chosen by mpdata_batch_autotune, which times every combination.
#include <cuda_runtime.h>

#include <climits>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mpdata.h"
#include "fused2.cuh"
#include "fusedt.cuh"
#include "grid.cuh"

using mpd::Geo;

namespace {

struct BDom {
  Geo g;
  const void* pa;
  void* pb;
  const void *u, *v, *w, *gm;
  long long item0;   // first work item of this domain
  long long tstride; // elements between consecutive tracers
  int ntr, tx, ty, nch, kchunk;
  int nit;           // items of one tile and chunk: ntr, or (ntr + 1) / 2 tracer pairs
};

__device__ __forceinline__ int find_domain(const BDom* __restrict__ d, int nd, long long item) {
  int lo = 0, hi = nd - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T, int TX, int TY, int NT, int MINB, bool LIMIT>
__global__ void __launch_bounds__((TX + 4) * (TY + 4), MINB)
batch_kernel(const BDom* __restrict__ dom, int nd, long long nitems, int* counter, int dir) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long it = s_item;
    if (it >= nitems) break;
    const int d = find_domain(dom, nd, it);
    const BDom& b = dom[d];
    long long r = it - b.item0;
    const int tr = (int)(r % b.ntr);
    r /= b.ntr;
    const int ch = (int)(r % b.nch);
    const int tile = (int)(r / b.nch);
    const int tx = tile % b.tx, ty = tile / b.tx;
    const T* src = (const T*)(dir == 0 ? b.pa : (const void*)b.pb) + tr * b.tstride;
    T* dst = (T*)(dir == 0 ? b.pb : (void*)b.pa) + tr * b.tstride;
    const int k0 = ch * b.kchunk;
    // FP32: levels in groups of 4 (constant ring slots), faster for the
    // batch's short chunks though not for one long domain (measured);
    // FP64 stays at 1, where the larger body spills
    mpd::fused2::step_tile2<T, TX, TY, LIMIT, false, sizeof(T) == 4 ? 4 : 1>(
        b.g, tx * TX, ty * TY, k0, min(b.g.nz, k0 + b.kchunk), src, (const T*)b.u,
        (const T*)b.v, (const T*)b.w, (const T*)b.gm, dst, smem_raw);
    // step_tile2 begins with a barrier, so s_item is not rewritten before all
    // threads have read it
  }
}

// The same for tracer pairs (FP32, fusedt.cuh): an item is a tile and chunk
// of two tracers of one domain.
template <int TX, int TY, int MINB, bool LIMIT>
__global__ void __launch_bounds__((TX + 4) * (TY + 4), MINB)
batch_kernel_t2(const BDom* __restrict__ dom, int nd, long long nitems, int* counter, int dir) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long it = s_item;
    if (it >= nitems) break;
    const int d = find_domain(dom, nd, it);
    const BDom& b = dom[d];
    long long r = it - b.item0;
    const int tp = (int)(r % b.nit);
    r /= b.nit;
    const int ch = (int)(r % b.nch);
    const int tile = (int)(r / b.nch);
    const int tx = tile % b.tx, ty = tile / b.tx;
    const int ta = 2 * tp, tb = min(2 * tp + 1, b.ntr - 1);
    const float* src = (const float*)(dir == 0 ? b.pa : (const void*)b.pb);
    float* dst = (float*)(dir == 0 ? b.pb : (void*)b.pa);
    const int k0 = ch * b.kchunk;
    mpd::fusedt::step_tile_t2<TX, TY, LIMIT>(
        b.g, tx * TX, ty * TY, k0, min(b.g.nz, k0 + b.kchunk), src + ta * b.tstride,
        src + tb * b.tstride, (const float*)b.u, (const float*)b.v, (const float*)b.w,
        (const float*)b.gm, dst + ta * b.tstride, dst + tb * b.tstride, ta != tb, smem_raw);
    // step_tile_t2 begins with a barrier (s_item is read before it)
  }
}

// Compiled tile shapes the autotuner chooses from.
struct Shape {
  int tx, ty, nt;
  int pair;  // items of two tracers (FP32)
};
// one thread per column of the tile + 2 ring: nt = (tx+4)(ty+4)
constexpr Shape kShapes32[] = {{32, 16, 720, 0}, {64, 8, 816, 0}, {32, 8, 432, 0},
                               {16, 16, 400, 0}, {32, 8, 432, 1},  {32, 12, 576, 1}};
constexpr Shape kShapes64[] = {{32, 8, 432, 0}, {16, 16, 400, 0}, {16, 8, 240, 0}};
constexpr int kNShapes32 = 6, kNShapes64 = 3;

template <class T, int S> struct ShapeOf;
#define MPD_SHAPE(TT, S, X, Y, N, P) \
  template <> struct ShapeOf<TT, S> {  \
    static constexpr int TX = X, TY = Y, NT = N; \
    static constexpr bool PAIR = P;    \
  };
MPD_SHAPE(float, 0, 32, 16, 720, false)
MPD_SHAPE(float, 1, 64, 8, 816, false)
MPD_SHAPE(float, 2, 32, 8, 432, false)
MPD_SHAPE(float, 3, 16, 16, 400, false)
MPD_SHAPE(float, 4, 32, 8, 432, true)
MPD_SHAPE(float, 5, 32, 12, 576, true)
MPD_SHAPE(double, 0, 32, 8, 432, false)
MPD_SHAPE(double, 1, 16, 16, 400, false)
MPD_SHAPE(double, 2, 16, 8, 240, false)
#undef MPD_SHAPE

}  // namespace

struct mpdata_batch {
  int nd, nonosc, dtype, device, sms;
  cudaStream_t stream;
  std::vector<mpdata_domain_desc> host;
  BDom* d_dom;
  int* d_counter;
  long long nitems;
  int shape, kchunk_levels, grid;
  size_t smem;
  const void* kern;
  cudaGraphExec_t exec[2];
  long long launches;
  char err[256];
};

namespace {

int bfail(mpdata_batch* b, cudaError_t e, const char* where) {
  if (b) std::snprintf(b->err, sizeof(b->err), "%s: %s", where, cudaGetErrorString(e));
  cudaGetLastError();
  return MPDATA_ECUDA;
}

template <class T, int S, bool LIMIT>
const void* kernel_ptr() {
  using Sh = ShapeOf<T, S>;
  constexpr int MINB = 1;
  if constexpr (Sh::PAIR)
    return reinterpret_cast<const void*>(&batch_kernel_t2<Sh::TX, Sh::TY, MINB, LIMIT>);
  else
    return reinterpret_cast<const void*>(&batch_kernel<T, Sh::TX, Sh::TY, Sh::NT, MINB, LIMIT>);
}

template <class T, int S>
size_t smem_of() {
  using Sh = ShapeOf<T, S>;
  if constexpr (Sh::PAIR) return mpd::fusedt::Layout<Sh::TX, Sh::TY>::bytes;
  else return mpd::fused2::Layout<T, Sh::TX, Sh::TY>::bytes;
}

template <class T>
void shape_info(int s, bool limit, const void** k, size_t* smem, int* nt, int* tx, int* ty) {
  if constexpr (sizeof(T) == 4) {
    switch (s) {
      case 0: *k = limit ? kernel_ptr<T, 0, true>() : kernel_ptr<T, 0, false>(); *smem = smem_of<T, 0>(); break;
      case 1: *k = limit ? kernel_ptr<T, 1, true>() : kernel_ptr<T, 1, false>(); *smem = smem_of<T, 1>(); break;
      case 2: *k = limit ? kernel_ptr<T, 2, true>() : kernel_ptr<T, 2, false>(); *smem = smem_of<T, 2>(); break;
      case 3: *k = limit ? kernel_ptr<T, 3, true>() : kernel_ptr<T, 3, false>(); *smem = smem_of<T, 3>(); break;
      case 4: *k = limit ? kernel_ptr<T, 4, true>() : kernel_ptr<T, 4, false>(); *smem = smem_of<T, 4>(); break;
      default: *k = limit ? kernel_ptr<T, 5, true>() : kernel_ptr<T, 5, false>(); *smem = smem_of<T, 5>(); break;
    }
    *nt = kShapes32[s].nt; *tx = kShapes32[s].tx; *ty = kShapes32[s].ty;
  } else {
    switch (s) {
      case 0: *k = limit ? kernel_ptr<T, 0, true>() : kernel_ptr<T, 0, false>(); *smem = smem_of<T, 0>(); break;
      case 1: *k = limit ? kernel_ptr<T, 1, true>() : kernel_ptr<T, 1, false>(); *smem = smem_of<T, 1>(); break;
      default: *k = limit ? kernel_ptr<T, 2, true>() : kernel_ptr<T, 2, false>(); *smem = smem_of<T, 2>(); break;
    }
    *nt = kShapes64[s].nt; *tx = kShapes64[s].tx; *ty = kShapes64[s].ty;
  }
}

int nshapes(int dtype) { return dtype == MPDATA_F64 ? kNShapes64 : kNShapes32; }

void drop_graphs(mpdata_batch* b) {
  for (int q = 0; q < 2; ++q)
    if (b->exec[q]) { cudaGraphExecDestroy(b->exec[q]); b->exec[q] = nullptr; }
}

// Build the descriptor table for the current shape and chunk length.
int configure(mpdata_batch* b, int shape, int kchunk_levels) {
  if (shape < 0 || shape >= nshapes(b->dtype) || kchunk_levels < 0) return MPDATA_EINVAL;
  const void* k = nullptr;
  size_t smem = 0;
  int nt = 0, tx = 0, ty = 0;
  if (b->dtype == MPDATA_F64) shape_info<double>(shape, b->nonosc, &k, &smem, &nt, &tx, &ty);
  else shape_info<float>(shape, b->nonosc, &k, &smem, &nt, &tx, &ty);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return bfail(b, e, "cudaFuncSetAttribute");
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nt, smem);
  if (e != cudaSuccess || occ < 1) return bfail(b, e, "occupancy");
  std::vector<BDom> tab(b->nd);
  const bool pair = b->dtype == MPDATA_F32 && kShapes32[shape].pair;
  long long item = 0;
  for (int d = 0; d < b->nd; ++d) {
    const mpdata_domain_desc& h = b->host[d];
    BDom& t = tab[d];
    t.g = mpd::make_geo(h.nx, h.ny, h.nz, h.halo);
    t.pa = h.psi_a; t.pb = h.psi_b;
    t.u = h.u; t.v = h.v; t.w = h.w; t.gm = h.g;
    t.tstride = t.g.total;
    t.ntr = h.ntracers;
    t.tx = (h.nx + tx - 1) / tx;
    t.ty = (h.ny + ty - 1) / ty;
    t.kchunk = kchunk_levels > 0 && kchunk_levels < h.nz ? kchunk_levels : h.nz;
    t.nch = (h.nz + t.kchunk - 1) / t.kchunk;
    t.nit = pair ? (t.ntr + 1) / 2 : t.ntr;
    // tracer pairs address a field with 32-bit offsets
    if (pair && t.g.total >= ((int64_t)1 << 31)) return MPDATA_ERANGE;
    t.item0 = item;
    item += (long long)t.tx * t.ty * t.nch * t.nit;
  }
  // the work counter is a 32-bit int that every CTA bumps once past the
  // last item before it exits, so it climbs to nitems + grid - 1
  const long long want = (long long)b->sms * occ;
  if (item > (long long)INT_MAX - want) return MPDATA_ERANGE;
  e = cudaMemcpy(b->d_dom, tab.data(), sizeof(BDom) * b->nd, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(b, e, "descriptor upload");
  drop_graphs(b);
  b->nitems = item;
  b->shape = shape;
  b->kchunk_levels = kchunk_levels;
  b->kern = k;
  b->smem = smem;
  b->grid = (int)(want < item ? want : (item > 0 ? item : 1));
  return MPDATA_OK;
}

int launch_once(mpdata_batch* b, int dir) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
  if (e != cudaSuccess) return bfail(b, e, "counter reset");
  int nd = b->nd;
  long long nitems = b->nitems;
  BDom* dom = b->d_dom;
  int* counter = b->d_counter;
  void* args[] = {&dom, &nd, &nitems, &counter, &dir};
  e = cudaLaunchKernel(b->kern, dim3(b->grid), dim3(b->dtype == MPDATA_F64
                                                        ? kShapes64[b->shape].nt
                                                        : kShapes32[b->shape].nt),
                       args, b->smem, b->stream);
  if (e != cudaSuccess) return bfail(b, e, "batch kernel launch");
  ++b->launches;
  return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_batch_init(mpdata_batch** out, const mpdata_domain_desc* doms, int ndomains,
                      int nonoscillatory, int dtype, void* stream) {
  if (!out) return MPDATA_EINVAL;
  *out = nullptr;
  if (!doms || ndomains < 1 || (nonoscillatory != 0 && nonoscillatory != 1)) return MPDATA_EINVAL;
  if (dtype != MPDATA_F64 && dtype != MPDATA_F32) return MPDATA_EINVAL;
  for (int d = 0; d < ndomains; ++d) {
    const mpdata_domain_desc& h = doms[d];
    if (h.nx < 1 || h.ny < 1 || h.nz < 1 || h.halo < 2 || h.ntracers < 1) return MPDATA_EINVAL;
    if (h.nx < 2 * h.halo || h.ny < 2 * h.halo) return MPDATA_EINVAL;
    if ((int64_t)(h.nx + 2 * h.halo) * (h.ny + 2 * h.halo) > (int64_t)1 << 31) return MPDATA_ERANGE;
    const void* p[6] = {h.psi_a, h.psi_b, h.u, h.v, h.w, h.g};
    for (int q = 0; q < 6; ++q) {
      if (!p[q]) return MPDATA_EINVAL;
      if (reinterpret_cast<uintptr_t>(p[q]) & 15u) return MPDATA_EALIGN;
    }
    if (h.psi_a == h.psi_b) return MPDATA_EINVAL;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MPDATA_EDEVICE; }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  mpdata_batch* b = new (std::nothrow) mpdata_batch();
  if (!b) return MPDATA_ENOMEM;
  b->nd = ndomains;
  b->nonosc = nonoscillatory;
  b->dtype = dtype;
  b->device = dev;
  b->sms = sms > 0 ? sms : 148;
  b->stream = (cudaStream_t)stream;
  b->host.assign(doms, doms + ndomains);
  b->exec[0] = b->exec[1] = nullptr;
  if (cudaMalloc(&b->d_dom, sizeof(BDom) * ndomains) != cudaSuccess ||
      cudaMalloc(&b->d_counter, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (b->d_dom) cudaFree(b->d_dom);
    delete b;
    return MPDATA_ENOMEM;
  }
  int rc = configure(b, 0, 0);
  if (rc) {
    cudaFree(b->d_dom);
    cudaFree(b->d_counter);
    delete b;
    return rc;
  }
  *out = b;
  return MPDATA_OK;
}

int mpdata_batch_step(mpdata_batch* b, int direction, int use_graph) {
  if (!b || (direction != 0 && direction != 1)) return MPDATA_EINVAL;
  if (!use_graph) return launch_once(b, direction);
  if (b->stream == nullptr) return MPDATA_EINVAL;  // capture needs a non-default stream
  if (!b->exec[direction]) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, e, "begin capture");
    int rc = launch_once(b, direction);
    e = cudaStreamEndCapture(b->stream, &graph);
    if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e != cudaSuccess) return bfail(b, e, "end capture");
    e = cudaGraphInstantiate(&b->exec[direction], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { b->exec[direction] = nullptr; return bfail(b, e, "graph instantiate"); }
    --b->launches;  // the captured launch did not run
  }
  cudaError_t e = cudaGraphLaunch(b->exec[direction], b->stream);
  if (e != cudaSuccess) return bfail(b, e, "graph launch");
  ++b->launches;
  return MPDATA_OK;
}

int mpdata_batch_set_config(mpdata_batch* b, int shape, int kchunk_levels) {
  if (!b) return MPDATA_EINVAL;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, e, "stream synchronize");
  return configure(b, shape, kchunk_levels);
}

int mpdata_batch_get_config(mpdata_batch* b, int* shape, int* kchunk_levels, int* tile_x,
                            int* tile_y, int* threads, long long* items) {
  if (!b) return MPDATA_EINVAL;
  const Shape& s = b->dtype == MPDATA_F64 ? kShapes64[b->shape] : kShapes32[b->shape];
  if (shape) *shape = b->shape;
  if (kchunk_levels) *kchunk_levels = b->kchunk_levels;
  if (tile_x) *tile_x = s.tx;
  if (tile_y) *tile_y = s.ty;
  if (threads) *threads = s.nt;
  if (items) *items = b->nitems;
  return MPDATA_OK;
}

int mpdata_batch_autotune(mpdata_batch* b, int reps, double* best_ms) {
  if (!b || reps < 1) return MPDATA_EINVAL;
  const int chunks[4] = {0, 32, 16, 8};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return MPDATA_ECUDA;
  }
  double best = 1e300;
  int bs = 0, bk = 0;
  int rc = MPDATA_OK;
  for (int s = 0; s < nshapes(b->dtype) && rc == MPDATA_OK; ++s)
    for (int c = 0; c < 4 && rc == MPDATA_OK; ++c) {
      if ((rc = mpdata_batch_set_config(b, s, chunks[c]))) {
        if (rc == MPDATA_ERANGE) { rc = MPDATA_OK; break; }  // not for this batch's sizes
        break;
      }
      if ((rc = launch_once(b, 0))) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < reps && rc == MPDATA_OK; ++r) rc = launch_once(b, r & 1);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = bfail(b, cudaGetLastError(), "autotune"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / reps < best) { best = ms / reps; bs = s; bk = chunks[c]; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (best_ms) *best_ms = best;
  return mpdata_batch_set_config(b, bs, bk);
}

long long mpdata_batch_launch_count(mpdata_batch* b) { return b ? b->launches : -1; }

const char* mpdata_batch_last_error_string(mpdata_batch* b) { return b ? b->err : ""; }

void mpdata_batch_destroy(mpdata_batch* b) {
  if (!b) return;
  drop_graphs(b);
  cudaFree(b->d_dom);
  cudaFree(b->d_counter);
  delete b;
}

}  // extern "C"
