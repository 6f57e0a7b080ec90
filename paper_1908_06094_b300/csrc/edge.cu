// edge.cu -- C ABI of the edge-based flux stages on a structured triangular
// patch (see edge.cuh and include/mpdata.h, "Edge-based flux stages").
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>

#include "../../include/mpdata.h"
#include "edge.cuh"

struct mpdata_edge {
  mpd::edge::Patch p;
  int dtype, variant;
  int width;  // nodes per thread of the fused kernel (1, or 4: FP32, nc % 4 == 0)
  double pivbz;
  size_t esize;
  cudaStream_t stream;
  void* scratch;           // staged organisation: flux, fluz, divVD
  void *flux, *fluz, *div;
  long long launches;
  char err[256];
};

namespace {

int edge_fail(mpdata_edge* e, int code, const char* what, cudaError_t ce = cudaSuccess) {
  if (e) {
    if (ce != cudaSuccess)
      std::snprintf(e->err, sizeof(e->err), "%s: %s", what, cudaGetErrorString(ce));
    else
      std::snprintf(e->err, sizeof(e->err), "%s", what);
  }
  return code;
}

bool al16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

dim3 node_grid(const mpd::edge::Patch& p, int levels) {
  using namespace mpd::edge;
  return dim3((p.nc + BX - 1) / BX, (p.nr + BY - 1) / BY, levels);
}

// The fused kernel's default width: four nodes per thread where the rows
// are 16-byte vectors (FP32, nc a multiple of 4), else one.
int auto_width(const mpd::edge::Patch& p, int dtype) {
  return (dtype == MPDATA_F32 && p.nc % 4 == 0) ? 4 : 1;
}

template <class T>
int edge_step(mpdata_edge* e, const T* pD, T* out, const T* vn, const T* W, const T* rho,
              const T* vol) {
  using namespace mpd::edge;
  const Patch& p = e->p;
  const dim3 blk(BX, BY);
  const T pv = (T)e->pivbz;
  cudaStream_t s = e->stream;
  if (e->variant != MPDATA_STAGED) {
    bool vec = false;
    if constexpr (std::is_same<T, float>::value) {
      if (e->width == 4) {
        const dim3 g((p.nc / 4 + BX4 - 1) / BX4, (p.nr + BY - 1) / BY, p.nz);
        edge_fused4_kernel<<<g, dim3(BX4, BY), 0, s>>>(p, pD, vn, W, rho, vol, pv, out);
        vec = true;
      }
    }
    if (!vec)
      edge_fused_kernel<T><<<node_grid(p, p.nz), blk, 0, s>>>(p, pD, vn, W, rho, vol, pv, out);
    e->launches += 1;
  } else {
    T *flux = (T*)e->flux, *fluz = (T*)e->fluz, *div = (T*)e->div;
    edge_flux_kernel<T><<<node_grid(p, p.nz), blk, 0, s>>>(p, pD, vn, flux);
    edge_fluz_kernel<T><<<node_grid(p, p.nz + 1), blk, 0, s>>>(p, pD, W, pv, fluz);
    edge_fluxdiv_kernel<T><<<node_grid(p, p.nz), blk, 0, s>>>(p, flux, fluz, vol, div);
    edge_advance_kernel<T><<<node_grid(p, p.nz), blk, 0, s>>>(p, pD, div, rho, out);
    e->launches += 4;
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return edge_fail(e, MPDATA_ECUDA, "edge step", ce);
  return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_edge_init(mpdata_edge** out, int nr, int nc, int nz, int dtype, double pivbz,
                     void* stream) {
  if (!out) return MPDATA_EINVAL;
  *out = nullptr;
  if (nr < 1 || nc < 1 || nz < 2) return MPDATA_EINVAL;
  if (dtype != MPDATA_F64 && dtype != MPDATA_F32) return MPDATA_EINVAL;
  if (!std::isfinite(pivbz)) return MPDATA_EINVAL;
  if (nz + 1 > 65535 || (nr + mpd::edge::BY - 1) / mpd::edge::BY > 65535) return MPDATA_ERANGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MPDATA_EDEVICE;
  }
  mpdata_edge* e = new (std::nothrow) mpdata_edge();
  if (!e) return MPDATA_ENOMEM;
  std::memset(e, 0, sizeof(*e));
  e->p = mpd::edge::make_patch(nr, nc, nz);
  e->dtype = dtype;
  e->variant = MPDATA_AUTO;
  e->width = auto_width(e->p, dtype);
  e->pivbz = pivbz;
  e->esize = dtype == MPDATA_F64 ? 8 : 4;
  e->stream = (cudaStream_t)stream;
  // staged scratch: flux 3 nz planes, fluz nz+1 planes, divVD nz planes
  const size_t plane = (size_t)e->p.plane * e->esize;
  const size_t fb = (3 * (size_t)nz) * plane, zb = (size_t)(nz + 1) * plane, db = (size_t)nz * plane;
  auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
  cudaError_t ce = cudaMalloc(&e->scratch, up256(fb) + up256(zb) + up256(db));
  if (ce != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return MPDATA_ENOMEM;
  }
  char* base = (char*)e->scratch;
  e->flux = base;
  e->fluz = base + up256(fb);
  e->div = base + up256(fb) + up256(zb);
  *out = e;
  return MPDATA_OK;
}

int mpdata_edge_set_stream(mpdata_edge* e, void* stream) {
  if (!e) return MPDATA_EINVAL;
  e->stream = (cudaStream_t)stream;
  return MPDATA_OK;
}

int mpdata_edge_set_variant(mpdata_edge* e, int variant) {
  if (!e || variant < MPDATA_FUSED || variant > MPDATA_AUTO) return MPDATA_EINVAL;
  e->variant = variant;
  return MPDATA_OK;
}

int mpdata_edge_step(mpdata_edge* e, const void* pD_in, void* pD_out, const void* vn,
                     const void* wn, const void* rho, const void* vol) {
  if (!e) return MPDATA_EINVAL;
  const void* f[6] = {pD_in, pD_out, vn, wn, rho, vol};
  for (const void* q : f)
    if (!q) return edge_fail(e, MPDATA_EINVAL, "null field pointer");
  for (const void* q : f)
    if (!al16(q)) return edge_fail(e, MPDATA_EALIGN, "field pointer not 16-byte aligned");
  if (pD_in == pD_out) return edge_fail(e, MPDATA_EINVAL, "pD_in and pD_out must differ");
  if (e->dtype == MPDATA_F64)
    return edge_step<double>(e, (const double*)pD_in, (double*)pD_out, (const double*)vn,
                             (const double*)wn, (const double*)rho, (const double*)vol);
  return edge_step<float>(e, (const float*)pD_in, (float*)pD_out, (const float*)vn,
                          (const float*)wn, (const float*)rho, (const float*)vol);
}

int mpdata_edge_set_width(mpdata_edge* e, int width) {
  if (!e) return MPDATA_EINVAL;
  if (width == 0) {
    e->width = auto_width(e->p, e->dtype);
  } else if (width == 1) {
    e->width = 1;
  } else if (width == 4 && e->dtype == MPDATA_F32 && e->p.nc % 4 == 0) {
    e->width = 4;
  } else {
    return edge_fail(e, MPDATA_EINVAL, "width 4 needs FP32 and nc a multiple of 4");
  }
  return MPDATA_OK;
}

int mpdata_edge_get_width(mpdata_edge* e, int* width) {
  if (!e || !width) return MPDATA_EINVAL;
  *width = e->width;
  return MPDATA_OK;
}

long long mpdata_edge_launch_count(mpdata_edge* e) { return e ? e->launches : -1; }

const char* mpdata_edge_last_error_string(mpdata_edge* e) { return e ? e->err : ""; }

void mpdata_edge_destroy(mpdata_edge* e) {
  if (!e) return;
  if (e->scratch) cudaFree(e->scratch);
  delete e;
}

}  // extern "C"
