// batch.cu -- band_solve_batch: several independent problems in one launch.
//
// The ADI step of the paper solves N systems per grid line and direction
// (Veneva & Ayriyan, Sec. 1); the solves of one step are independent.  One 2048 x 2048
// sweep has only 2048 systems, 64 warps for 152 SMs, while the FP64 units of a
// GB300 SM need at least four resident warps.  Here the problems of a step share one
// kernel: every warp takes consecutive systems of one problem (32 on one thread each,
// 16 on the two-sided schedule, 32 / P partitioned; the sweeps of sweeps.cuh,
// partition.cuh and sip_impl.cuh), so the launch holds the warps of all of them.  The
// problem table travels as a __grid_constant__ kernel parameter; nothing is
// allocated.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "api_util.h"
#include "batch_kernel.cuh"
#include "kernels.h"
#include "partition.cuh"
#include "sip_impl.cuh"
#include "sweeps.cuh"
#include "symbolic.cuh"

namespace band {

// k_batch with two warps per block here; one and four in batch_w1.cu, batch_w4.cu
template cudaError_t launch_batch_w<2>(const BatchTable&, int64_t, cudaStream_t);
cudaError_t launch_batch_w1(const BatchTable& t, int64_t warps, cudaStream_t st);
cudaError_t launch_batch_w4(const BatchTable& t, int64_t warps, cudaStream_t st);
cudaError_t launch_batch(const BatchTable& t, int64_t warps, int w, cudaStream_t st) {
  if (w == 1) return launch_batch_w1(t, warps, st);
  if (w == 4) return launch_batch_w4(t, warps, st);
  return launch_batch_w<2>(t, warps, st);
}

// Warps per block of k_batch on each device: two unless the autotuner (runtime.cu) has
// measured another to be faster.
static std::atomic<int> g_batch_warps[64];
int batch_warps(int dev) {
  const int w = (dev >= 0 && dev < 64) ? g_batch_warps[dev].load(std::memory_order_relaxed) : 0;
  return w ? w : 2;
}
void set_batch_warps(int dev, int w) {
  if (dev >= 0 && dev < 64 && (w == 1 || w == 2 || w == 4))
    g_batch_warps[dev].store(w, std::memory_order_relaxed);
}

namespace {

struct TailTable {
  int32_t count;
  int32_t pad;
  int64_t smem_rows;     // rows of a system the dynamic shared memory holds
  SipArgs it[BAND_MAX_BATCH];
};

struct SymItem {
  SymArgs a;
  int64_t slot0;
};

struct SymTable {
  int32_t count;
  int32_t pad;
  int64_t total;     // warps (slots)
  SymItem it[BAND_MAX_BATCH];
};

// the symbolic fix-ups of all problems: warp g serves slot g - slot0 of its problem
constexpr int kSymWarps = 4;
__global__ void __launch_bounds__(32 * kSymWarps) k_symbolic_batch(const __grid_constant__ SymTable t) {
  __shared__ lser::dd stage[kSymWarps][128];
  const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (g >= t.total) return;
  int j = 0;
  while (j + 1 < t.count && t.it[j + 1].slot0 <= g) ++j;
  const SymArgs& p = t.it[j].a;
  const int64_t slot = g - t.it[j].slot0;
  const unsigned long long count = *p.fix_count;
  const lser::SlotView sv = lser::slot_view(p, slot);
  for (unsigned long long item = slot; item < count; item += p.nslots)
    lser::symbolic_warp(p, p.fix_list[item], sv, stage[threadIdx.x >> 5]);
}

// the deferred residual and decision of the SIP problems (blockIdx.y: the problem)
__global__ void __launch_bounds__(256, 4) k_sip_resid_batch(const __grid_constant__ TailTable t) {
  sip_resid_cell(t.it[blockIdx.y], (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void __launch_bounds__(256) k_sip_decide_batch(const __grid_constant__ TailTable t) {
  const SipArgs& p = t.it[blockIdx.y];
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < p.L.nsys) sip_decide_one(p, s);
}

__global__ void __launch_bounds__(kTailThreads) k_sip_tail_batch(const __grid_constant__ TailTable t) {
  __shared__ Aff sh[kTailThreads];
  __shared__ double red[kTailThreads / 32];
  extern __shared__ double tail_smem[];
  // the tail lists of all problems as one list, dealt out round-robin over the blocks
  // (a few systems per problem would otherwise queue on the same few blocks)
  unsigned long long total = 0;
  for (int j = 0; j < t.count; ++j) total += *t.it[j].tail_count;
  for (unsigned long long g = blockIdx.x; g < total; g += gridDim.x) {
    int j = 0;
    unsigned long long it = g;
    for (unsigned long long c = *t.it[0].tail_count; it >= c; c = *t.it[j].tail_count) {
      it -= c;
      ++j;
    }
    const SipArgs& p = t.it[j];
    sip_tail_block(p, p.tail_list[it], p.tail_rn[it], sh, red, tail_smem, t.smem_rows);
  }
}

}  // namespace
}  // namespace band

using namespace band;

// Relative cost of one warp task of a problem: rows on its longest dependent chain times
// the work per row (SIP's first update and residual ~2.5x a PD sweep, TD ~0.6x, FP32
// ~0.5x; a partitioned chunk row ~2.3x, plus the interface solve).  Tasks are handed out
// heaviest problem first.
static double task_cost(const band_problem& q) {
  const band_desc* d = q.desc;
  double rows = (double)d->n;
  double w = 1.0;
  if (q.op == BAND_OP_SIP) {
    w = 2.5;
  } else {
    const bool td = d->hbw == nullptr && d->half_bw == 1;
    w = td ? 0.6 : 1.0;
    if (d->dtype == BAND_F32) w *= 0.5;
    if (kmode_for(d, q.method) > 0) {
      const bool alias = q.x == q.f && !is_symbolic(q.method);
      const int P = choose_parts(d, 32);
      if (P) rows = rows / P * 2.3 + 8.0 * P;
      else if (choose_two_sided(d, alias)) rows *= 0.5;
    }
  }
  return rows * w;
}

extern "C" band_status band_solve_batch(const band_problem* in, int32_t count, void* stream) {
  if (count < 0 || count > BAND_MAX_BATCH || (count > 0 && !in)) return BAND_ERR_ARG;
  for (int32_t i = 0; i < count; ++i)
    if (!in[i].desc || !desc_ok(in[i].desc)) return BAND_ERR_ARG;
  // heaviest problems first; among equal costs the numeric methods before the symbolic
  // ones (a stable order otherwise; results do not depend on it).  Measured on the
  // 30-solve ADI step: the TD problems with STDM before NTDM 4.54 ms, with NTDM first
  // 4.14 ms (the same instructions and DRAM bytes; the tail differs).
  int32_t order[BAND_MAX_BATCH];
  for (int32_t i = 0; i < count; ++i) order[i] = i;
  auto symbolic_of = [&](int32_t x) {
    return in[x].op == BAND_OP_SOLVE && is_symbolic(in[x].method) ? 1 : 0;
  };
  std::stable_sort(order, order + count, [&](int32_t x, int32_t y) {
    const double cx = task_cost(in[x]), cy = task_cost(in[y]);
    if (cx != cy) return cx > cy;
    return symbolic_of(x) < symbolic_of(y);
  });
  band_problem probs[BAND_MAX_BATCH];
  for (int32_t i = 0; i < count; ++i) probs[i] = in[order[i]];
  static_assert(sizeof(BatchTable) < 32000, "kernel parameter table too large");
  static_assert(sizeof(TailTable) < 32000, "kernel parameter table too large");
  BatchTable t;
  SymTable sym;
  TailTable tail;
  std::memset(&t, 0, sizeof t);
  std::memset(&sym, 0, sizeof sym);
  std::memset(&tail, 0, sizeof tail);
  void* counters[BAND_MAX_BATCH];
  int ncounters = 0;
  void* pend_clear[BAND_MAX_BATCH];     // SIP: per-system max|r| and pending flags
  size_t pend_bytes[BAND_MAX_BATCH];
  int npend = 0;
  int64_t warps = 0, slots = 0;
  for (int32_t i = 0; i < count; ++i) {
    const band_problem& q = probs[i];
    if (q.desc->nsys == 0) {
      if (q.op != BAND_OP_SOLVE && q.op != BAND_OP_SIP) return BAND_ERR_ARG;
      continue;
    }
    BatchItem& b = t.it[t.count];
    if (q.op == BAND_OP_SOLVE) {
      DirectReq r;
      const band_status v = make_direct(q.desc, q.method, q.diag, q.f, q.x, q.sys_status, q.ws,
                                        q.ws_bytes, &r, 32);
      if (v != BAND_OK) return v;
      b.kmode = (int16_t)r.kmode;
      b.two_sided = r.two_sided ? 1 : 0;
      // four chunks run in band_solve alone: in this kernel their task's code costs
      // every other task spill space (128-register cap: 72 / 608 B against 60 / 464 B of
      // spill stores / loads, the ADI step 4.1 -> 4.3 ms)
      if (r.parts == 4) return BAND_ERR_ARG;
      b.parts = (int8_t)r.parts;
      // Uniform contiguous problems read through L1 here: next to the batch's other
      // tasks that measured faster than granule staging (ADI step 4.85 vs 5.16 ms);
      // ragged buckets keep it (65536 systems: 10.7 -> 8.7 ms).
      if (!q.desc->offsets) r.d64.gran = r.d32.gran = 0;
      if (q.desc->dtype == BAND_F64) {
        b.kind = kDirect64;
        b.u.d64 = r.d64;
        t.stage_bytes = std::max(t.stage_bytes, stage_bytes_per_warp<double>());
      } else {
        b.kind = kDirect32;
        b.u.d32 = r.d32;
        t.stage_bytes = std::max(t.stage_bytes, stage_bytes_per_warp<float>());
      }
      if (r.symbolic) {
        counters[ncounters++] = r.sym.fix_count_mut;
        SymItem& si = sym.it[sym.count++];
        si.a = r.sym.args;
        si.slot0 = slots;
        slots += r.sym.args.nslots;
      }
    } else if (q.op == BAND_OP_SIP) {
      SipArgs sa;
      const band_status v = make_sip(q.desc, q.diag, q.f, q.x, q.tol, q.max_it, 0, q.iters,
                                     q.resid, q.sys_status, q.ws, q.ws_bytes, &sa, nullptr);
      if (v != BAND_OK) return v;
      // SIP runs one thread per system here: the two-sided first update needs more
      // registers than the other tasks of this kernel (180 against 128) and measured
      // slower in it (ADI step 4.42 -> 6.9 ms)
      sa.two_sided = 0;
      t.stage_bytes = std::max(t.stage_bytes, stage_bytes_per_warp<double>());
      b.kind = kSip;
      b.kmode = 2;
      b.two_sided = 0;
      b.parts = 0;
      b.u.sip = sa;
      counters[ncounters++] = sa.tail_count;
      pend_clear[npend] = sa.rn_sys;
      pend_bytes[npend++] = (size_t)((char*)(sa.pend + q.desc->nsys) - (char*)sa.rn_sys);
      tail.it[tail.count++] = sa;
    } else {
      return BAND_ERR_ARG;
    }
    b.task0 = warps;
    if (b.parts) {
      const int per = kWarp / b.parts;
      warps += (q.desc->nsys + per - 1) / per;
    } else {
      warps += b.two_sided ? (q.desc->nsys + 15) / 16 : (q.desc->nsys + kWarp - 1) / kWarp;
    }
    ++t.count;
  }
  t.total = warps;
  sym.total = slots;
  if (warps == 0) return BAND_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < ncounters; ++i)
    if (cudaMemsetAsync(counters[i], 0, sizeof(unsigned long long), st) != cudaSuccess)
      return BAND_ERR_CUDA;
  for (int i = 0; i < npend; ++i)
    if (cudaMemsetAsync(pend_clear[i], 0, pend_bytes[i], st) != cudaSuccess) return BAND_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return BAND_ERR_CUDA;
  if (launch_batch(t, warps, batch_warps(dev), st) != cudaSuccess) return BAND_ERR_CUDA;
  if (sym.count > 0 && slots > 0) {
    k_symbolic_batch<<<(unsigned)((slots + kSymWarps - 1) / kSymWarps), 32 * kSymWarps, 0, st>>>(sym);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  }
  if (tail.count > 0) {
    int64_t cells = 0, nmax = 0;
    for (int j = 0; j < tail.count; ++j) {
      const Layout& L = tail.it[j].L;
      cells = std::max(cells, resid_cells(L));
      nmax = std::max(nmax, L.nsys);
    }
    k_sip_resid_batch<<<dim3((unsigned)((cells + 255) / 256), (unsigned)tail.count), 256, 0, st>>>(tail);
    k_sip_decide_batch<<<dim3((unsigned)((nmax + 255) / 256), (unsigned)tail.count), 256, 0, st>>>(tail);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t n_max = 0;
    for (int j = 0; j < tail.count; ++j) n_max = std::max(n_max, tail.it[j].L.n);
    const size_t smem = tail_smem_bytes(n_max);
    tail.smem_rows = tail_smem_rows(smem);
    if (tail_prepare((const void*)k_sip_tail_batch) != cudaSuccess) return BAND_ERR_CUDA;
    k_sip_tail_batch<<<(unsigned)(nsm > 0 ? nsm : 1), kTailThreads, smem, st>>>(tail);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  }
  return BAND_OK;
}
