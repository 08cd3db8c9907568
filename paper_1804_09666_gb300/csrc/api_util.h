// api_util.h -- host-side validation and workspace carving for the C entry points.
#pragma once
#include <cstddef>
#include <cstdint>
#include <initializer_list>
#include <cuda_runtime.h>

#include "band.h"
#include "common.cuh"

namespace band {

// Bump allocator over the caller's workspace (p == nullptr: size computation only).
struct Carve {
  char* p;
  size_t used;
  explicit Carve(void* base) : p(static_cast<char*>(base)), used(0) {}
  void* take(size_t bytes) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return p ? p + off : nullptr;
  }
  size_t size() const { return (used + 255) & ~size_t(255); }
};

inline size_t dtype_size(int32_t dt) { return dt == BAND_F32 ? 4 : 8; }

// Alignment the kernels rely on.  Element arrays are read and written as whole elements
// (8 bytes FP64, 4 FP32; 4-byte statuses, 8-byte offsets and system ids).  Workspaces
// and factor buffers are carved at 256-byte offsets from their base, and parts of them
// are read as 16-byte vectors, so the base must sit on a 256-byte boundary (as
// cudaMalloc's allocations do).  A pointer that breaks this would fault on the GPU; the
// entry points reject it instead.
constexpr size_t kWsAlign = 256;
inline bool aligned_to(const void* p, size_t a) { return ((uintptr_t)p & (a - 1)) == 0; }
// the caller's workspace: present, on a kWsAlign boundary, at least `need` bytes
inline bool ws_fits(const void* ws, size_t ws_bytes, size_t need) {
  return ws && aligned_to(ws, kWsAlign) && ws_bytes >= need;
}
// every given pointer (NULL counts as aligned) on an `a`-byte boundary
inline bool aligned_all(size_t a, std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (!aligned_to(p, a)) return false;
  return true;
}
// the five diagonals (any may be NULL), f and x in `dtype`, and the int32 statuses
inline bool arrays_aligned(int32_t dtype, const void* const diag[5], const void* f,
                           const void* x, const int32_t* status) {
  const size_t s = dtype_size(dtype);
  if (diag)
    for (int q = 0; q < 5; ++q)
      if (!aligned_to(diag[q], s)) return false;
  return aligned_all(s, {f, x}) && aligned_to(status, 4);
}
inline bool ragged(const band_desc* d) { return d->offsets != nullptr; }

// Rows of one scratch array: interleaved by system for uniform batches (S x n with S
// = nsys rounded up to a warp), packed like the data for ragged batches.
// Ragged batches with an id list (a size bucket) keep their scratch interleaved by
// position in the list, rows up to n (the bucket's largest size).
inline int64_t spill_rows(const band_desc* d) {
  return (ragged(d) && !d->systems) ? d->total_rows : round_up(d->nsys, kWarp) * d->n;
}
inline Spill spill_of(const band_desc* d) {
  Spill w;
  w.S = round_up(d->nsys, kWarp);
  w.offsets = d->systems ? nullptr : d->offsets;
  return w;
}
inline Layout layout_of(const band_desc* d) {
  Layout L;
  L.nsys = d->nsys;
  L.n = d->n;
  L.ss = d->sys_stride;
  L.es = d->elem_stride;
  L.offsets = d->offsets;
  L.hbw = d->hbw;
  L.ids = d->systems;
  L.extent = ragged(d) ? d->total_rows
                       : (d->n - 1) * d->elem_stride + (d->nsys - 1) * d->sys_stride + 1;
  L.half_bw = d->half_bw;
  return L;
}

// Structural checks of a descriptor (values only; device arrays are not read).
inline bool desc_ok(const band_desc* d) {
  if (!d) return false;
  if (d->dtype != BAND_F64 && d->dtype != BAND_F32) return false;
  if (d->nsys < 0 || d->n < 1) return false;
  if (!d->hbw && d->half_bw != 1 && d->half_bw != 2) return false;
  if (d->schedule < BAND_SCHED_AUTO || d->schedule > BAND_SCHED_GRID) return false;
  if (d->chunks != 0 && (d->schedule != BAND_SCHED_PARTITIONED || d->chunks < 4 ||
                         d->chunks > 256 || (d->chunks & (d->chunks - 1)) != 0))
    return false;
  if (d->systems && !d->offsets) return false;     // id lists select from a ragged packing
  if (!aligned_all(8, {d->offsets, d->systems})) return false;   // device int64 arrays
  if (ragged(d)) {
    if (d->total_rows < 0) return false;
  } else {
    if (d->elem_stride < 1 || d->sys_stride < 1) return false;
    // systems must not overlap: one stride has to span the other's whole extent
    const bool inner_rows = d->nsys <= 1 || d->elem_stride * (d->n - 1) < d->sys_stride;
    const bool inner_sys = d->n <= 1 || d->sys_stride * (d->nsys - 1) < d->elem_stride;
    if (!inner_rows && !inner_sys) return false;
  }
  return true;
}

// Can any system of the batch be pentadiagonal?
inline bool may_be_pd(const band_desc* d) { return d->hbw != nullptr || d->half_bw == 2; }

// kmode for the kernels: 1 TD, 2 PD, 0 per system from hbw; -1 if inconsistent.
inline int kmode_for(const band_desc* d, int32_t method) {
  const int m = method;
  if (m == BAND_NTDM || m == BAND_STDM) return (d->hbw == nullptr && d->half_bw == 1) ? 1 : -1;
  if (m == BAND_NPDM || m == BAND_SPDM) return (d->hbw == nullptr && d->half_bw == 2) ? 2 : -1;
  if (m == BAND_AUTO_NUMERIC || m == BAND_AUTO_SYMBOLIC) return d->hbw ? 0 : d->half_bw;
  return -1;
}
inline bool is_symbolic(int32_t m) {
  return m == BAND_STDM || m == BAND_SPDM || m == BAND_AUTO_SYMBOLIC;
}

inline band_status cuda_status(cudaError_t e) { return e == cudaSuccess ? BAND_OK : BAND_ERR_CUDA; }

}  // namespace band
