// api.cu -- C entry points for the direct solvers (band_solve, band_factor) and the
// shared utilities of libband.  See include/band.h for the contract of each call.
#include <cstdint>
#include <cstring>

#include "api_util.h"
#include "kernels.h"

using namespace band;

namespace band {

// Workspace of band_solve.  Numeric methods: alpha and beta rows.  Symbolic methods:
// alpha, beta and z rows, the flagged-system counter and list, and the Laurent-series
// rows of min(nsys, kFixSlots) flagged systems redone at a time (the last region, so
// that a larger workspace holds more of them; see fix_slots).
// The partitioned schedule adds the rows of z (always: f stays intact until a failed
// system has been redone) and of the coupling columns' z, all chunk-major.
SolveWs carve_solve(const band_desc* d, int32_t method, void* base, size_t* bytes) {
  Carve c(base);
  SolveWs w{};
  const bool part = d->schedule == BAND_SCHED_PARTITIONED && kmode_for(d, method) > 0;
  const int64_t r0 = spill_rows(d);
  const int64_t pr = part ? part_rows_bound(d) : 0;
  const size_t rows = (size_t)(r0 > pr ? r0 : pr) * dtype_size(d->dtype);
  w.al = c.take(rows);
  w.be = c.take(rows);
  if (part) {
    w.zs = c.take(rows);
    w.zv1 = c.take((size_t)pr * dtype_size(d->dtype));
    if (may_be_pd(d)) w.zv2 = c.take((size_t)pr * dtype_size(d->dtype));
  }
  if (is_symbolic(method)) {
    if (!w.zs) w.zs = c.take(rows);
    w.count = c.take(sizeof(unsigned long long));
    w.list = c.take(sizeof(int64_t) * (size_t)(d->nsys > 0 ? d->nsys : 1));
    w.nslots = d->nsys < kFixSlots ? d->nsys : kFixSlots;
    w.slots = c.take((size_t)w.nslots * symbolic_slot_bytes(d->n));
  }
  *bytes = c.size();
  return w;
}

// Fix-up slots a workspace of ws_bytes holds: the stated ones plus as many more as fit
// behind them, at most min(nsys, kFixSlotsMax).
int64_t fix_slots(const band_desc* d, const SolveWs& w, size_t need, size_t ws_bytes) {
  int64_t n = w.nslots;
  if (ws_bytes > need) n += (int64_t)((ws_bytes - need) / symbolic_slot_bytes(d->n));
  const int64_t cap = d->nsys < kFixSlotsMax ? d->nsys : kFixSlotsMax;
  return n < cap ? n : cap;
}

struct FactorBuf {
  void *gam, *rmu, *al, *be;
};
static FactorBuf carve_factors(const band_desc* d, const void* base, size_t* bytes) {
  Carve c(const_cast<void*>(base));
  const size_t rows = (size_t)spill_rows(d) * dtype_size(d->dtype);
  FactorBuf fb;
  fb.gam = c.take(rows);
  fb.rmu = c.take(rows);
  fb.al = c.take(rows);
  fb.be = c.take(rows);
  *bytes = c.size();
  return fb;
}

size_t factor_bytes(const band_desc* d) {
  size_t b = 0;
  carve_factors(d, nullptr, &b);
  return b;
}
FactorPtrs factor_ptrs(const band_desc* d, const void* factors) {
  size_t b = 0;
  FactorBuf fb = carve_factors(d, factors, &b);
  return FactorPtrs{fb.gam, fb.rmu, fb.al, fb.be};
}

// The automatic schedule.  Measured on GB300 with the staging ring in both schedules,
// the two-sided sweep is faster than one thread per system for the uniform batches with
// n >= 32 that were tried (n = 128 .. 8192, 1024 .. 131072 systems, FP64 and FP32,
// interleaved and contiguous; from parity at 32768 x 512 to 1.9x at 2048 x 2048), also
// inside a batched launch of 30 such problems, with one exception (65536 x 1024 FP64:
// 2.14 ms against 1.95 ms); below n = 32 the interface solve is a large share of the
// work.  band_autotune replaces the rule by measurement.
bool choose_two_sided(const band_desc* d, bool alias) {
  if (d->schedule == BAND_SCHED_THREAD || d->schedule == BAND_SCHED_PARTITIONED) return false;
  if (d->schedule == BAND_SCHED_TWO_SIDED) return true;
  if ((d->offsets && !d->systems) || alias) return false;   // whole ragged packings: thread
  return d->n >= 32;
}

// The automatic schedule of a single problem.  A small batch of long systems (fewer than
// 32 per SM, n >= 256: the two-sided schedule would leave under two warps per SM) is
// bound by its chains, not by the FP64 pipes, and P lanes per system shorten them
// P / 2-fold for about twice the arithmetic per row.  Measured on GB300 (FP64 NPDM,
// ms, two-sided against partitioned with the library's chunk count): 2048 x 2048
// 0.83 / 0.45, 256 x 8192 3.11 / 0.36, 64 x 65536 24.9 / 1.01; above the line
// two-sided stays ahead (7280 x 6000: 2.84 / 3.78, 16384 x 4096: 2.12 / 5.07).
// A chunk restarts the elimination at its first row, and on rows that are not
// diagonally dominant it can meet a pivot far below NPDM's (the pivot guard of
// partition.cuh); such a system is listed, and a second launch of the AUTO sweep
// (two-sided, or one thread when x aliases f) solves the listed systems again from f,
// which the partitioned sweep leaves intact.  With the redo inside the partitioned
// kernel, on one lane, the indefinite r = 2 ADI rows took 2.3-3.5 ms against 0.85-0.96
// two-sided.  Numeric methods only (a symbolic system that meets a small chunk pivot
// goes to the series pass, ~24 us a row); uniform batches of one bandwidth.
namespace {

bool auto_part(const band_desc* d, int32_t method) {
  if (d->schedule != BAND_SCHED_AUTO || d->offsets || d->n < 256 || is_symbolic(method) ||
      kmode_for(d, method) <= 0)
    return false;
  static int nsm_cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  int nsm = dev < 64 ? nsm_cache[dev] : 0;
  if (nsm == 0) {
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      return false;
    if (dev < 64) nsm_cache[dev] = nsm;
  }
  return d->nsys < (int64_t)32 * nsm;
}

band_desc partitioned_of(const band_desc* d) {
  band_desc r = *d;
  r.schedule = BAND_SCHED_PARTITIONED;
  r.chunks = 0;
  return r;
}

// Byte offset of the redo counter behind the partitioned workspace; the list follows
// 256 bytes later.
size_t redo_offset(const band_desc* dp, int32_t method) {
  size_t need = 0;
  carve_solve(dp, method, nullptr, &need);
  return (size_t)round_up((int64_t)need, 256);
}

cudaError_t launch_req(const DirectReq& r, int32_t dtype, cudaStream_t st) {
  if (r.parts)
    return dtype == BAND_F64 ? launch_partition<double>(r.d64, r.kmode, r.parts, st)
                             : launch_partition<float>(r.d32, r.kmode, r.parts, st);
  if (r.two_sided)
    return dtype == BAND_F64 ? launch_twisted<double>(r.d64, r.kmode, st)
                             : launch_twisted<float>(r.d32, r.kmode, st);
  return dtype == BAND_F64 ? launch_direct<double>(r.d64, r.kmode, st)
                           : launch_direct<float>(r.d32, r.kmode, st);
}

}  // namespace

size_t single_solve_bytes(const band_desc* d, int32_t method) {
  size_t plain = 0;
  carve_solve(d, method, nullptr, &plain);
  if (!auto_part(d, method)) return plain;
  const band_desc dp = partitioned_of(d);
  const size_t part = redo_offset(&dp, method) + 256 + (size_t)d->nsys * sizeof(int64_t);
  return part > plain ? part : plain;
}

band_status run_single(const band_desc* desc, int32_t method, const void* const diag[5],
                       const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                       cudaStream_t st, const int32_t* skip) {
  if (auto_part(desc, method)) {
    if (!ws_fits(ws, ws_bytes, single_solve_bytes(desc, method))) return BAND_ERR_WORKSPACE;
    const band_desc dp = partitioned_of(desc);
    // both sweeps carve alpha and beta from the workspace's start (the partitioned
    // carve extends the plain one); the second launch runs after the first is done
    DirectReq rp, ra;
    band_status v = make_direct(&dp, method, diag, f, x, sys_status, ws, ws_bytes, &rp, 256);
    if (v != BAND_OK) return v;
    v = make_direct(desc, method, diag, f, x, sys_status, ws, ws_bytes, &ra, 256);
    if (v != BAND_OK) return v;
    rp.d64.skip = rp.d32.skip = ra.d64.skip = ra.d32.skip = skip;
    char* base = static_cast<char*>(ws) + redo_offset(&dp, method);
    auto* count = reinterpret_cast<unsigned long long*>(base);
    auto* list = reinterpret_cast<int64_t*>(base + 256);
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess)
      return BAND_ERR_CUDA;
    rp.d64.redo_list = rp.d32.redo_list = list;
    rp.d64.redo_count = rp.d32.redo_count = count;
    if (launch_req(rp, desc->dtype, st) != cudaSuccess) return BAND_ERR_CUDA;
    ra.d64.L.ids = ra.d32.L.ids = list;          // position t: the t-th listed system
    ra.d64.nsys_dev = ra.d32.nsys_dev = count;
    return cuda_status(launch_req(ra, desc->dtype, st));
  }
  DirectReq r;
  const band_status v = make_direct(desc, method, diag, f, x, sys_status, ws, ws_bytes, &r, 256);
  if (v != BAND_OK) return v;
  r.d64.skip = r.d32.skip = skip;
  if (r.symbolic && cudaMemsetAsync(r.sym.fix_count_mut, 0, sizeof(unsigned long long), st) !=
                        cudaSuccess)
    return BAND_ERR_CUDA;
  if (launch_req(r, desc->dtype, st) != cudaSuccess) return BAND_ERR_CUDA;
  if (r.symbolic) return cuda_status(launch_symbolic_fixup(r.sym.args, st));
  return BAND_OK;
}

// Slots per chunk row of the partitioned scratch: nsys rounded up to the systems of a
// warp (32 / P for P <= 32, one system per block beyond).
int64_t part_np(int64_t nsys, int parts) { return parts >= 32 ? nsys : round_up(nsys, 32 / parts); }

// Chunk-major rows of one partitioned scratch array: ceil(n / P) rows of P chunks for
// part_np systems; desc->chunks == 0 takes the largest over the chunk counts.
int64_t part_rows_bound(const band_desc* d) {
  int64_t best = 0;
  for (int P = 4; P <= 256; P *= 2) {
    if (d->chunks && P != d->chunks) continue;
    const int64_t r = (d->n + P - 1) / P * P * part_np(d->nsys, P);
    if (r > best) best = r;
  }
  return best;
}

// Lanes per system on the partitioned schedule (0: another schedule).  chunks == 0: the
// P in {8, 16, .., max_parts} (chunks of 8 rows or more) with the least estimated time
//   warps(P) * (n / P * c_row + (P / 2 + 2) * c_if) / min(1, warps(P) / (8 warps x SMs)),
// warps(P) = nsys * P / 32: the FP64 instructions of the launch (a chunk row costs
// c_row = 32 (PD) / 14 (TD); the interface, eliminated from both ends, c_if = 60 / 25
// per chunk on its longer half, plus the meeting), slowed down while too few warps are
// resident to keep the FP64 pipes busy.  Measured on GB300 (FP64 NPDM, ms):
// 2048 x 2048 0.53 / 0.45 / 0.75 at P = 8 / 16 / 32 (chosen: 16); 256 x 8192 0.55 /
// 0.36 / 0.38 at P = 32 / 64 / 128 (chosen: 128); 64 x 65536 1.17 / 1.01 at P = 128 /
// 256 (chosen: 256); 7280 x 6000 3.77 / 3.07 at P = 8 / 16 (chosen: 8, the model's
// worst miss; band_autotune measures instead).
int choose_parts(const band_desc* d, int max_parts) {
  if (d->schedule != BAND_SCHED_PARTITIONED) return 0;
  if (d->chunks) return d->chunks < max_parts ? d->chunks : max_parts;
  static int nsm_cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  int nsm = dev < 64 ? nsm_cache[dev] : 0;
  if (nsm == 0) {
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 1;
    if (dev < 64) nsm_cache[dev] = nsm;
  }
  const bool td = d->hbw == nullptr && d->half_bw == 1;
  const double c_row = td ? 14.0 : 32.0, c_if = td ? 25.0 : 60.0;
  const double sat = 8.0 * nsm;
  int best = 8;
  double best_t = -1.0;
  for (int P = 8; P <= max_parts; P *= 2) {
    if (P > 8 && d->n < (int64_t)8 * P) break;
    const double warps = (double)d->nsys * P / 32.0;
    const double eff = warps < sat ? warps / sat : 1.0;
    const double t =
        warps * ((double)d->n / P * c_row + (P / 2 + 2) * c_if) / (eff > 0 ? eff : 1e-9);
    if (best_t < 0 || t < best_t) { best_t = t; best = P; }
  }
  return best;
}

band_status make_direct(const band_desc* desc, int32_t method, const void* const diag[5],
                        const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                        DirectReq* r, int max_parts) {
  if (!desc_ok(desc) || desc->schedule == BAND_SCHED_GRID) return BAND_ERR_ARG;
  const int kmode = kmode_for(desc, method);
  if (kmode < 0) return BAND_ERR_ARG;
  if (is_symbolic(method) && desc->dtype != BAND_F64) return BAND_ERR_ARG;
  if (!diag || !f || !x || !diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc) && kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  if (!arrays_aligned(desc->dtype, diag, f, x, sys_status)) return BAND_ERR_ARG;
  size_t need = 0;
  carve_solve(desc, method, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const SolveWs w = carve_solve(desc, method, ws, &need);
  const Layout L = layout_of(desc);
  const Spill W = spill_of(desc);
  r->kmode = kmode;
  r->symbolic = is_symbolic(method);
  r->two_ok = kmode != 0;
  r->alias = x == f && !r->symbolic;   // symbolic methods keep f until the backward sweep
  r->two_sided = r->two_ok && choose_two_sided(desc, r->alias);
  r->parts = r->two_ok ? choose_parts(desc, max_parts) : 0;
  r->d64 = DirectArgs<double>{L, W,
                              (const double*)diag[0], (const double*)diag[1],
                              (const double*)diag[2], (const double*)diag[3],
                              (const double*)diag[4], (const double*)f, (double*)x,
                              (double*)w.al, (double*)w.be, (double*)w.zs, sys_status,
                              (unsigned long long*)w.count, (int64_t*)w.list};
  r->d32 = DirectArgs<float>{L, W,
                             (const float*)diag[0], (const float*)diag[1], (const float*)diag[2],
                             (const float*)diag[3], (const float*)diag[4], (const float*)f,
                             (float*)x, (float*)w.al, (float*)w.be, nullptr, sys_status,
                             nullptr, nullptr};
  // contiguous rows (each lane its own system) are staged in 16-byte granules when
  // every array the sweep reads is 16-byte aligned
  {
    auto al16 = [](const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; };
    const bool contig = desc->offsets ? true : (desc->elem_stride == 1 && desc->sys_stride != 1);
    const bool aligned = al16(diag[1]) && al16(diag[2]) && al16(diag[3]) && al16(f) &&
                         (kmode == 1 || (diag[0] && diag[4] && al16(diag[0]) && al16(diag[4])));
    r->d64.gran = r->d32.gran = (contig && aligned) ? 1 : 0;
  }
  if (r->parts) {
    const int64_t np = part_np(desc->nsys, r->parts);
    r->d64.zs = (double*)w.zs;
    r->d64.zv1 = (double*)w.zv1;
    r->d64.zv2 = (double*)w.zv2;
    r->d64.part_np = np;
    r->d32.zs = (float*)w.zs;
    r->d32.zv1 = (float*)w.zv1;
    r->d32.zv2 = (float*)w.zv2;
    r->d32.part_np = np;
  }
  if (!r->symbolic) {
    if (!r->parts) r->d64.zs = nullptr;
    r->d64.fix_count = nullptr;
    r->d64.fix_list = nullptr;
  } else {
    r->sym.fix_count_mut = w.count;
    SymArgs& sa = r->sym.args;
    sa = SymArgs{};
    sa.L = L;
    sa.a = (const double*)diag[0];
    sa.b = (const double*)diag[1];
    sa.c = (const double*)diag[2];
    sa.d = (const double*)diag[3];
    sa.e = (const double*)diag[4];
    sa.f = (const double*)f;
    sa.x = (double*)x;
    sa.status = sys_status;
    sa.fix_count = (const unsigned long long*)w.count;
    sa.fix_list = (const int64_t*)w.list;
    sa.slot_mem = w.slots;
    sa.nslots = fix_slots(desc, w, need, ws_bytes);
    sa.nmax = desc->n;
  }
  return BAND_OK;
}

}  // namespace band

extern "C" {

size_t band_workspace_size(const band_desc* desc, int32_t op, int32_t method, int32_t sip_width) {
  if (op == BAND_OP_ADI) return adi_workspace_bytes(desc);   // a grid, checked there
  if (!desc_ok(desc)) return 0;
  size_t bytes = 0;
  switch (op) {
    case BAND_OP_SOLVE:
      if (method == BAND_MNPDM) return mnpdm_workspace_bytes(desc);
      if (desc->schedule == BAND_SCHED_GRID) return grid_workspace_bytes(desc);
      return single_solve_bytes(desc, method);
    case BAND_OP_FACTOR: return factor_bytes(desc);
    case BAND_OP_SIP: return sip_workspace_bytes(desc, sip_width);
    case BAND_OP_REFINE: return refine_workspace_bytes(desc);
    case BAND_OP_ADJOINT: return adjoint_workspace_bytes(desc);
    case BAND_OP_DET: return det_workspace_bytes(desc);
    case BAND_OP_SIP2D: return sip2d_workspace_bytes(desc);
    default: return 0;
  }
}

band_status band_solve(const band_desc* desc, int32_t method, const void* factors,
                       const void* const diag[5], const void* f, void* x, int32_t* sys_status,
                       void* ws, size_t ws_bytes, void* stream) {
  if (!desc_ok(desc)) return BAND_ERR_ARG;
  if (desc->nsys > 0) {
    if (!arrays_aligned(desc->dtype, diag, f, x, sys_status)) return BAND_ERR_ARG;
    if (!aligned_to(factors, kWsAlign)) return BAND_ERR_WORKSPACE;
  }
  if (method == BAND_MNPDM) {
    if (factors) return BAND_ERR_ARG;
    if (desc->nsys == 0) return BAND_OK;
    return mnpdm_solve(desc, diag, f, x, sys_status, ws, ws_bytes, static_cast<cudaStream_t>(stream));
  }
  const int kmode = kmode_for(desc, method);
  if (kmode < 0) return BAND_ERR_ARG;
  if (is_symbolic(method) && (desc->dtype != BAND_F64 || factors)) return BAND_ERR_ARG;
  if (factors && desc->systems) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;   // nothing to do (empty arrays may be NULL)
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (factors) {
    if (!diag || !f || !x || !diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
    if (may_be_pd(desc) && kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
    const Layout L = layout_of(desc);
    const Spill W = spill_of(desc);
    const FactorPtrs fp = factor_ptrs(desc, factors);
    if (desc->dtype == BAND_F64) {
      FactoredArgs<double> p{L, W, (const double*)diag[0], (const double*)fp.gam,
                             (const double*)fp.rmu, (const double*)fp.al, (const double*)fp.be,
                             (const double*)f, (double*)x, sys_status};
      return cuda_status(launch_fsolve<double>(p, kmode, st));
    }
    FactoredArgs<float> p{L, W, (const float*)diag[0], (const float*)fp.gam,
                          (const float*)fp.rmu, (const float*)fp.al, (const float*)fp.be,
                          (const float*)f, (float*)x, sys_status};
    return cuda_status(launch_fsolve<float>(p, kmode, st));
  }
  if (desc->schedule == BAND_SCHED_GRID) return grid_solve(desc, method, diag, f, x, sys_status, ws, ws_bytes, st);
  return run_single(desc, method, diag, f, x, sys_status, ws, ws_bytes, st);
}

band_status band_factor(const band_desc* desc, int32_t method, const void* const diag[5],
                        void* factors, size_t factors_bytes, int32_t* sys_status, void* stream) {
  if (!desc_ok(desc) || desc->systems) return BAND_ERR_ARG;
  const int kmode = kmode_for(desc, method);
  if (kmode < 0 || is_symbolic(method)) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !factors) return BAND_ERR_ARG;
  if (!diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc) && kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  if (!arrays_aligned(desc->dtype, diag, nullptr, nullptr, sys_status)) return BAND_ERR_ARG;
  if (!aligned_to(factors, kWsAlign) || factors_bytes < factor_bytes(desc)) return BAND_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const FactorPtrs fp = factor_ptrs(desc, factors);
  const Layout L = layout_of(desc);
  const Spill W = spill_of(desc);
  if (desc->dtype == BAND_F64) {
    FactorArgs<double> p{L, W, (const double*)diag[0], (const double*)diag[1],
                         (const double*)diag[2], (const double*)diag[3], (const double*)diag[4],
                         (double*)fp.gam, (double*)fp.rmu, (double*)fp.al, (double*)fp.be,
                         sys_status};
    return cuda_status(launch_factor<double>(p, kmode, st));
  }
  FactorArgs<float> p{L, W, (const float*)diag[0], (const float*)diag[1], (const float*)diag[2],
                      (const float*)diag[3], (const float*)diag[4], (float*)fp.gam,
                      (float*)fp.rmu, (float*)fp.al, (float*)fp.be, sys_status};
  return cuda_status(launch_factor<float>(p, kmode, st));
}

const char* band_status_str(int32_t s) {
  switch (s) {
    case BAND_OK: return "BAND_OK";
    case BAND_ERR_ARG: return "BAND_ERR_ARG";
    case BAND_ERR_CUDA: return "BAND_ERR_CUDA";
    case BAND_ERR_ZERO_PIVOT: return "BAND_ERR_ZERO_PIVOT";
    case BAND_ERR_SINGULAR: return "BAND_ERR_SINGULAR";
    case BAND_ERR_NONFINITE: return "BAND_ERR_NONFINITE";
    case BAND_ERR_NOT_CONVERGED: return "BAND_ERR_NOT_CONVERGED";
    case BAND_ERR_SYMBOLIC_RANGE: return "BAND_ERR_SYMBOLIC_RANGE";
    case BAND_ERR_INTERNAL: return "BAND_ERR_INTERNAL";
    case BAND_ERR_WORKSPACE: return "BAND_ERR_WORKSPACE";
    default: return "BAND_UNKNOWN_STATUS";
  }
}

const char* band_version(void) { return "libband 0.1 (sm_103a)"; }

}  // extern "C"
