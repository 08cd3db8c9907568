// batch_kernel.cuh -- the kernel of band_solve_batch (batch.cu), a template on the warps
// per block so that the autotuner can choose the block size: batch.cu instantiates two
// warps per block, batch_w1.cu and batch_w4.cu one and four (one translation unit each,
// compiled in parallel).
#pragma once
#include <cstdint>

#include "api_util.h"
#include "kernels.h"
#include "partition.cuh"
#include "sip_impl.cuh"
#include "sweeps.cuh"

namespace band {

enum : int32_t { kDirect64 = 0, kDirect32 = 1, kSip = 2 };

struct BatchItem {
  int32_t kind;
  int16_t kmode;     // 1 TD, 2 PD, 0 per system
  int8_t two_sided;  // two threads (lanes l, l ^ 16) per system
  int8_t parts;      // partitioned: lanes per system (32 / parts systems a warp), or 0
  int64_t task0;     // first warp of this problem
  union {
    DirectArgs<double> d64;
    DirectArgs<float> d32;
    SipArgs sip;
  } u;
};

struct BatchTable {
  int32_t count;
  int32_t stage_bytes;   // staging ring bytes per warp (0: none)
  int64_t total;     // warp tasks
  BatchItem it[BAND_MAX_BATCH];
};

template <typename T>
__device__ __forceinline__ void run_direct(const DirectArgs<T>& p, int kmode, int64_t t,
                                           void* stage) {
  if (t >= p.L.nsys) return;
  const int K = kmode ? kmode : p.L.kband(p.L.sys(t));
  if (K == 1) direct_one<T, 1>(p, t, stage);
  else direct_one<T, 2>(p, t, stage);
}

// Scratch rows a partitioned task's backward sweeps load together inside this kernel.
// Four, as in the single-problem kernel: under this kernel's 128 registers they spill a
// little more than two (184 B against 124 B), yet the 65536-system ragged batch took
// 4.56 ms against 4.68 ms with two.
constexpr int kBatchPartRows = 4;

template <typename T>
__device__ __forceinline__ void run_partition(const DirectArgs<T>& p, int kmode, int parts,
                                              int64_t warp, void* stage) {
  T* st = static_cast<T*>(stage);    // the warp's staging area (stage_bytes_per_warp<T>)
  if (kmode == 1) {
    switch (parts) {
      case 8: partition_one<T, 1, 8, kBatchPartRows>(p, warp, st); break;
      case 16: partition_one<T, 1, 16, kBatchPartRows>(p, warp, st); break;
      default: partition_one<T, 1, 32, kBatchPartRows>(p, warp, st); break;
    }
  } else {
    switch (parts) {
      case 8: partition_one<T, 2, 8, kBatchPartRows>(p, warp, st); break;
      case 16: partition_one<T, 2, 16, kBatchPartRows>(p, warp, st); break;
      default: partition_one<T, 2, 32, kBatchPartRows>(p, warp, st); break;
    }
  }
}

// One warp task: 32 systems of one problem (16 two-sided, 32 / P partitioned).  Blocks are
// handed out by the hardware scheduler as earlier ones finish, in task order, and the
// host orders the problems heaviest first.  (A persistent loop over a task counter was
// tried: keeping every task variant's state live across the loop doubled the kernel's
// registers, 126 -> 255, and halved the resident warps.)
// Warps per block of k_batch.  Small blocks let the hardware spread the heaviest-first
// tasks over all SMs instead of packing four per SM (measured on the 30-solve ADI step:
// 1, 2 and 4 warps give 5.00, 4.96 and 5.19 ms); 128 registers allow 16 warps per SM.

// Part: the table may hold partitioned tasks.  Without them compiled in the kernel fits
// its 128 registers without spilling (60 / 464 B of spill stores / loads with them),
// which measured 29.4-29.6 -> 30.6 G unknowns/s on the 30-solve ADI step; the launch
// takes that variant whenever no problem of the table is partitioned.
template <int W, bool Part>
__global__ void __launch_bounds__(32 * W, 16 / W) k_batch(const __grid_constant__ BatchTable t) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  void* stage = t.stage_bytes ? stage_mem + (threadIdx.x >> 5) * t.stage_bytes : nullptr;
  const int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (task >= t.total) return;
  int j = 0;
  while (j + 1 < t.count && t.it[j + 1].task0 <= task) ++j;
  const BatchItem& b = t.it[j];
  if (Part && b.parts) {
    const int64_t w = task - b.task0;
    if (b.kind == kDirect64) run_partition<double>(b.u.d64, b.kmode, b.parts, w, stage);
    else run_partition<float>(b.u.d32, b.kmode, b.parts, w, stage);
    return;
  }
  if (b.two_sided) {         // 16 systems per warp
    const int64_t t2 = (task - b.task0) * 16 + (threadIdx.x & 15);
    if (b.kind == kDirect64) {
      if (b.kmode == 1) twisted_one<double, 1>(b.u.d64, t2, t2 < b.u.d64.L.nsys, stage);
      else twisted_one<double, 2>(b.u.d64, t2, t2 < b.u.d64.L.nsys, stage);
    } else {
      if (b.kmode == 1) twisted_one<float, 1>(b.u.d32, t2, t2 < b.u.d32.L.nsys, stage);
      else twisted_one<float, 2>(b.u.d32, t2, t2 < b.u.d32.L.nsys, stage);
    }
    return;
  }
  const int64_t s = (task - b.task0) * kWarp + (threadIdx.x & (kWarp - 1));
  if (b.kind == kDirect64) run_direct<double>(b.u.d64, b.kmode, s, stage);
  else if (b.kind == kDirect32) run_direct<float>(b.u.d32, b.kmode, s, stage);
  else if (s < b.u.sip.L.nsys) sip_literal(b.u.sip, s, stage);
}


// Launches k_batch<W, Part> over `warps` warp tasks (smem: W staging areas).
template <int W>
cudaError_t launch_batch_w(const BatchTable& t, int64_t warps, cudaStream_t st) {
  const size_t smem = (size_t)W * (size_t)t.stage_bytes;
  const unsigned grid = (unsigned)((warps + W - 1) / W);
  bool part = false;
  for (int32_t j = 0; j < t.count; ++j) part = part || t.it[j].parts != 0;
  if (part) k_batch<W, true><<<grid, 32 * W, smem, st>>>(t);
  else k_batch<W, false><<<grid, 32 * W, smem, st>>>(t);
  return cudaGetLastError();
}
cudaError_t launch_batch(const BatchTable& t, int64_t warps, int w, cudaStream_t st);

}  // namespace band
