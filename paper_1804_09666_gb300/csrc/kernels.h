// kernels.h -- argument blocks and launchers of the libband kernels (internal).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace band {

// Symbolic fix-up: flagged systems redone at a time, one warp each.  The workspace that
// band_workspace_size() states holds kFixSlots of them (one per SM of a GB300); a larger
// workspace holds more, up to kFixSlotsMax (two warps per SM sub-partition).
constexpr int64_t kFixSlots = 152;
constexpr int64_t kFixSlotsMax = 1216;

template <typename T>
struct DirectArgs {
  Layout L;
  Spill W;
  const T *a, *b, *c, *d, *e, *f;
  T* x;
  T *al, *be, *zs;                 // workspace rows (zs: symbolic methods only)
  int32_t* status;
  unsigned long long* fix_count;   // symbolic methods: flagged-system counter and list
  int64_t* fix_list;
  int32_t gran;                    // contiguous rows staged in 16-byte granules (GranRing)
  const int32_t* skip;             // per system id, or null: nonzero = leave the system alone
  // partitioned schedule: forward rows of the coupling columns (chunk-major, like al,
  // be and zs then) and the slots per chunk row (nsys rounded up to 32 / chunks)
  T *zv1, *zv2;
  int64_t part_np;
  // partitioned schedule: a system whose elimination fails is appended to redo_list
  // (position in the batch; redo_count counts them) for a follow-up launch, instead of
  // being redone in the kernel by one lane (null: in the kernel)
  int64_t* redo_list;
  unsigned long long* redo_count;
  // thread / two-sided sweeps: positions at or beyond *nsys_dev are left alone (the
  // follow-up launch over a redo list; null: L.nsys alone bounds them)
  const unsigned long long* nsys_dev;
};

template <typename T>
struct FactorArgs {
  Layout L;
  Spill W;
  const T *a, *b, *c, *d, *e;
  T *gam, *rmu, *al, *be;
  int32_t* status;
};

template <typename T>
struct FactoredArgs {
  Layout L;
  Spill W;
  const T* a;
  const T *gam, *rmu, *al, *be;
  const T* f;
  T* x;
  int32_t* status;
};

struct SymArgs {
  Layout L;
  const double *a, *b, *c, *d, *e, *f;
  double* x;
  int32_t* status;
  const unsigned long long* fix_count;
  const int64_t* fix_list;
  void* slot_mem;
  int64_t nslots, nmax;
  double* det_mant;       // optional per-system determinant (mantissa, base-2 exponent)
  long long* det_exp;
  int32_t det_only;       // determinant only: no z, no backward sweep, x untouched
};

template <typename T> cudaError_t launch_direct(const DirectArgs<T>&, int kmode, cudaStream_t);
template <typename T> cudaError_t launch_twisted(const DirectArgs<T>&, int kmode, cudaStream_t);
template <typename T>
cudaError_t launch_partition(const DirectArgs<T>&, int kmode, int parts, cudaStream_t);
template <typename T> cudaError_t launch_factor(const FactorArgs<T>&, int kmode, cudaStream_t);
template <typename T> cudaError_t launch_fsolve(const FactoredArgs<T>&, int kmode, cudaStream_t);
cudaError_t launch_symbolic_fixup(const SymArgs&, cudaStream_t);
size_t symbolic_slot_bytes(int64_t nmax);

// Workspace of band_solve (see api.cu).
struct SolveWs {
  void *al, *be, *zs, *count, *list, *slots, *zv1, *zv2;
  int64_t nslots;
};
SolveWs carve_solve(const band_desc* d, int32_t method, void* base, size_t* bytes);

// A validated fused direct solve: kernel arguments for both element types and, for
// symbolic methods, the fix-up arguments and the counter to clear before the sweep.
struct DirectReq {
  int kmode;
  bool symbolic;
  bool two_ok;          // the two-sided and partitioned schedules apply (one bandwidth)
  bool two_sided;       // schedule: two threads per system
  int parts;            // schedule: partitioned, lanes (chunks) per system; 0 = not
  bool alias;           // x is f
  DirectArgs<double> d64;
  DirectArgs<float> d32;
  struct {
    void* fix_count_mut;
    SymArgs args;
  } sym;
};
// max_parts: the most lanes per system the caller's kernels run (256 for band_solve's
// own launch, 32 inside band_solve_batch, whose tasks are single warps).
band_status make_direct(const band_desc* desc, int32_t method, const void* const diag[5],
                        const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                        DirectReq* r, int max_parts);
bool choose_two_sided(const band_desc* d, bool alias);
// A single-problem direct solve (band_solve, band_solve_static, the transposed solve of
// band_adjoint) with everything band_solve does after its argument checks, on the
// workspace single_solve_bytes sizes (defined in api.cu).  On BAND_SCHED_AUTO a small
// batch of long NTDM / NPDM systems runs partitioned, and the systems whose partitioned
// elimination fails are solved again by the AUTO sweep in a second launch.  Batched
// launches keep their own rule: there the other problems fill the GPU.
size_t single_solve_bytes(const band_desc* d, int32_t method);
// skip (may be null): per system id, nonzero = leave the system alone (DirectArgs::skip).
band_status run_single(const band_desc* desc, int32_t method, const void* const diag[5],
                       const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                       cudaStream_t st, const int32_t* skip = nullptr);
int choose_parts(const band_desc* d, int max_parts);
// Warps per block of band_solve_batch's kernel on device `dev` (1, 2 or 4; 2 unless the
// autotuner chose otherwise; defined in batch.cu).
int batch_warps(int dev);
void set_batch_warps(int dev, int w);
// Lets `kernel` launch with more than 48 KiB of dynamic shared memory (the attribute is
// set once per kernel and device; defined in sip.cu).
cudaError_t tail_prepare(const void* kernel);
int64_t part_rows_bound(const band_desc* d);

// host-side helpers shared by the entry points (defined in api.cu and the feature files)
struct FactorPtrs {
  void *gam, *rmu, *al, *be;
};
size_t factor_bytes(const band_desc* d);
FactorPtrs factor_ptrs(const band_desc* d, const void* factors);
size_t sip_workspace_bytes(const band_desc* d, int32_t width);
size_t refine_workspace_bytes(const band_desc* d);
size_t adjoint_workspace_bytes(const band_desc* d);
size_t det_workspace_bytes(const band_desc* d);
size_t adi_workspace_bytes(const band_desc* grid);
size_t sip2d_workspace_bytes(const band_desc* d);
// MNPDM (mnpdm.cu): band_solve's path and workspace for BAND_MNPDM
size_t mnpdm_workspace_bytes(const band_desc* d);
band_status mnpdm_solve(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                        int32_t* sys_status, void* ws, size_t ws_bytes, cudaStream_t st);
// the grid schedule (grid.cu): band_solve's path and workspace for BAND_SCHED_GRID
size_t grid_workspace_bytes(const band_desc* d);
int64_t grid_chunks(const band_desc* d);
band_status grid_solve(const band_desc* desc, int32_t method, const void* const diag[5],
                       const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                       cudaStream_t st);
}  // namespace band
