// cells.cu -- C ABI of the cell-neighbour reduction (see cells.cuh and
// include/mpdata.h, "Cell-neighbour reduction").
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/mpdata.h"
#include "cells.cuh"

struct mpdata_cells {
  int64_t ncells;
  int nz, nr, nc, dtype, kc;
  int* table;  // device [3][ncells], or null: structured direct access
  cudaStream_t stream;
  long long launches;
  char err[256];
};

namespace {

int cells_fail(mpdata_cells* c, int code, const char* what, cudaError_t ce = cudaSuccess) {
  if (c) {
    if (ce != cudaSuccess)
      std::snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(ce));
    else
      std::snprintf(c->err, sizeof(c->err), "%s", what);
  }
  return code;
}

// Levels per thread: enough CTAs for about 8 per SM on 148 SMs.
int pick_kc(int64_t ncells, int nz) {
  const int64_t blocks = (ncells + mpd::cells::kThreads - 1) / mpd::cells::kThreads;
  int64_t chunks = (8 * 148 + blocks - 1) / blocks;
  if (chunks < 1) chunks = 1;
  if (chunks > nz) chunks = nz;
  return (int)((nz + chunks - 1) / chunks);
}

template <class T>
int cells_sum(mpdata_cells* c, const T* A, T* B, T fac) {
  using namespace mpd::cells;
  const dim3 grid((unsigned)((c->ncells + kThreads - 1) / kThreads),
                  (unsigned)((c->nz + c->kc - 1) / c->kc));
  if (c->table)
    cells_sum_table_kernel<T><<<grid, kThreads, 0, c->stream>>>(c->ncells, c->nz, c->kc,
                                                                c->table, A, B, fac);
  else
    cells_sum_direct_kernel<T><<<grid, kThreads, 0, c->stream>>>(c->nr, c->nc, c->nz, c->kc,
                                                                 A, B, fac);
  c->launches += 1;
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cells_fail(c, MPDATA_ECUDA, "cells sum", ce);
  return MPDATA_OK;
}

}  // namespace

extern "C" {

int mpdata_cells_init(mpdata_cells** out, long long ncells, int nz, int dtype, const int* table,
                      int nr, int nc, void* stream) {
  if (!out) return MPDATA_EINVAL;
  *out = nullptr;
  if (ncells < 1 || nz < 1) return MPDATA_EINVAL;
  if (dtype != MPDATA_F64 && dtype != MPDATA_F32) return MPDATA_EINVAL;
  if (ncells > (1LL << 31) - 1 || (ncells + 255) / 256 > 2147483647LL || nz > 65535 * 64)
    return MPDATA_ERANGE;
  if (!table && (nr < 1 || nc < 1 || 2LL * nr * nc != ncells)) return MPDATA_EINVAL;
  if (table) {  // every neighbour must be a cell of the mesh
    for (long long q = 0; q < 3 * ncells; ++q)
      if (table[q] < 0 || table[q] >= ncells) return MPDATA_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MPDATA_EDEVICE;
  }
  mpdata_cells* c = new (std::nothrow) mpdata_cells();
  if (!c) return MPDATA_ENOMEM;
  std::memset(c, 0, sizeof(*c));
  c->ncells = ncells;
  c->nz = nz;
  c->nr = nr;
  c->nc = nc;
  c->dtype = dtype;
  c->kc = pick_kc(ncells, nz);
  if ((nz + c->kc - 1) / c->kc > 65535) c->kc = (nz + 65534) / 65535;
  c->stream = (cudaStream_t)stream;
  if (table) {
    const size_t bytes = 3 * (size_t)ncells * sizeof(int);
    cudaError_t ce = cudaMalloc(&c->table, bytes);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->table, table, bytes, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      if (c->table) cudaFree(c->table);
      delete c;
      return MPDATA_ENOMEM;
    }
  }
  *out = c;
  return MPDATA_OK;
}

int mpdata_cells_set_stream(mpdata_cells* c, void* stream) {
  if (!c) return MPDATA_EINVAL;
  c->stream = (cudaStream_t)stream;
  return MPDATA_OK;
}

int mpdata_cells_sum(mpdata_cells* c, const void* A, void* B, double fac) {
  if (!c) return MPDATA_EINVAL;
  if (!A || !B) return cells_fail(c, MPDATA_EINVAL, "null field pointer");
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u)
    return cells_fail(c, MPDATA_EALIGN, "field pointer not 16-byte aligned");
  if (A == B) return cells_fail(c, MPDATA_EINVAL, "A and B must differ");
  if (c->dtype == MPDATA_F64) return cells_sum<double>(c, (const double*)A, (double*)B, fac);
  return cells_sum<float>(c, (const float*)A, (float*)B, (float)fac);
}

long long mpdata_cells_launch_count(mpdata_cells* c) { return c ? c->launches : -1; }

const char* mpdata_cells_last_error_string(mpdata_cells* c) { return c ? c->err : ""; }

void mpdata_cells_destroy(mpdata_cells* c) {
  if (!c) return;
  if (c->table) cudaFree(c->table);
  delete c;
}

}  // extern "C"
