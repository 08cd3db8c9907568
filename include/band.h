/*
 * band.h -- C ABI of libband: batched tridiagonal / pentadiagonal solvers on one
 * NVIDIA GB300 (sm_103a).
 *
 * Methods (Veneva & Ayriyan, "Performance Analysis of Effective Methods for Solving
 * Band Matrix SLAEs after Parabolic Nonlinear PDEs", arXiv:1804.09666):
 *   NTDM / NPDM  LU-based direct solvers without pivoting for tridiagonal (TD) and
 *                pentadiagonal (PD) systems (Sec. 1; cost 9N+2 and 19N-29, Table 7).
 *   STDM / SPDM  the symbolic variants: a pivot that is exactly zero is replaced by a
 *                symbol t and the solution is evaluated at the limit t -> 0, so only
 *                nonsingularity is required (Sec. 1; O(N) determinant, Sec. 3.2
 *                Remark 1).
 *   SIP          the Stone method with ILU(0) (Sec. 2, Algorithm 1), optionally with
 *                Hotelling-Bodewig inverses in place of the substitutions (Remark of
 *                Sec. 2; Eq. (1) of the Appendix).
 * In the paper's ADI time step (Sec. 1) the systems of one sweep, one per grid line,
 * do not depend on one another; every call here solves a batch of such systems.
 *
 * Storage.  A system of n rows is given by five row-aligned diagonals
 *   a[i] = A[i][i-2], b[i] = A[i][i-1], c[i] = A[i][i], d[i] = A[i][i+1], e[i] = A[i][i+2]
 * (TD systems use b, c, d; a and e may be NULL).  Slots outside the matrix
 * (a[0], a[1], b[0], d[n-1], e[n-2], e[n-1]) must be readable but never enter the
 * arithmetic (they may hold NaN).  Right-hand side f, solution x.
 * Element i of system s of every array lives at
 *   s * sys_stride + i * elem_stride          (uniform batches, offsets == NULL), or
 *   offsets[s] + i                             (ragged batches, offsets != NULL),
 * counted in elements of the array's type.  Interleaved (sys_stride 1, elem_stride
 * >= nsys) gives coalesced access and is the fast layout; contiguous systems
 * (elem_stride 1, sys_stride >= n) and any other stride pair are accepted.
 *
 * Ownership and asynchrony.  Every pointer except `desc` and the host-side arrays
 * named as such is a device pointer owned by the caller.  The library allocates no
 * device memory: scratch comes from the caller's workspace, whose size
 * band_workspace_size() gives (a multiple of 256 bytes).  All calls enqueue work on
 * `stream` (a cudaStream_t; NULL = the legacy default stream) and return without
 * waiting.  Inputs are never modified; x may alias f.
 *
 * Alignment.  Every element array starts on a boundary of its element size (8 bytes
 * for FP64 and int64 arrays, 4 for FP32 and int32); workspaces and factor buffers
 * start on a 256-byte boundary (as cudaMalloc's allocations do).  A call given a
 * pointer off its boundary returns BAND_ERR_ARG (BAND_ERR_WORKSPACE for a workspace
 * or factor buffer) and launches nothing.
 *
 * Errors.  The return value reports argument, workspace and launch errors only.
 * Numerical outcomes are written per system to the device array sys_status
 * (band_status values; NULL = not wanted).
 */
#ifndef BAND_H
#define BAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BAND_OK = 0,
  BAND_ERR_ARG = 1,             /* invalid argument (return value) */
  BAND_ERR_CUDA = 2,            /* CUDA launch or runtime error (return value) */
  BAND_ERR_ZERO_PIVOT = 3,      /* per system: NTDM/NPDM met a pivot that is exactly 0 */
  BAND_ERR_SINGULAR = 4,        /* per system: the determinant's limit is 0 (STDM/SPDM) */
  BAND_ERR_NONFINITE = 5,       /* per system: Inf or NaN in the result */
  BAND_ERR_NOT_CONVERGED = 6,   /* per system: SIP / refinement / HB reached its cap */
  BAND_ERR_SYMBOLIC_RANGE = 7,  /* per system: the Laurent window of the symbolic path ran out */
  BAND_ERR_INTERNAL = 8,        /* per system: a kernel-side consistency check failed */
  BAND_ERR_WORKSPACE = 9        /* workspace missing, misaligned or smaller than band_workspace_size() */
} band_status;

typedef enum {
  BAND_NTDM = 0,   /* numeric TD (requires half_bw 1) */
  BAND_NPDM = 1,   /* numeric PD (requires half_bw 2) */
  BAND_STDM = 2,   /* symbolic TD */
  BAND_SPDM = 3,   /* symbolic PD */
  BAND_AUTO_NUMERIC = 4,   /* NTDM or NPDM per system by its half bandwidth (ragged mixes) */
  BAND_AUTO_SYMBOLIC = 5,  /* STDM or SPDM per system by its half bandwidth */
  BAND_MNPDM = 6           /* PD systems whose outer diagonals are mostly zero: the outer
                              entries eliminated, then NTDM (band_solve only; see there) */
} band_method;

typedef enum { BAND_F64 = 0, BAND_F32 = 1 } band_dtype;

typedef struct {
  int32_t half_bw;        /* 1 = tridiagonal, 2 = pentadiagonal (default when hbw is NULL) */
  int32_t dtype;          /* band_dtype of the diagonals, f and x */
  int64_t nsys;           /* number of independent systems, >= 0 */
  int64_t n;              /* uniform: rows per system (>= 1); ragged: an upper bound on
                             every system's rows (>= 1) */
  int64_t sys_stride;     /* uniform: elements between row i of systems s and s+1 */
  int64_t elem_stride;    /* uniform: elements between rows i and i+1 of one system */
  const int64_t* offsets; /* ragged: device array of nsys+1 nondecreasing row offsets
                             (system s = rows offsets[s] .. offsets[s+1]-1); else NULL */
  const int8_t* hbw;      /* device array of per-system half bandwidths (1 or 2), or NULL */
  int64_t total_rows;     /* ragged: offsets[nsys] (the host's copy); uniform: ignored */
  int32_t schedule;       /* band_schedule for NTDM/NPDM solves (BAND_SCHED_AUTO = 0) */
  int32_t chunks;         /* BAND_SCHED_PARTITIONED: lanes (row chunks) per system, 4, 8,
                             16, 32 (lanes of a warp) or 64, 128, 256 (a block of 2, 4, 8
                             warps per system); 0 = chosen from nsys and n (8 or more).
                             band_solve_batch rejects 4.  Otherwise 0. */
  /* Ragged batches only, else NULL: device array of nsys system ids.  The batch is then
   * the systems ids[0 .. nsys-1] of the packing that offsets (and hbw) describe, and
   * every per-system output (sys_status, iters, resid) is indexed by the id.  A solve
   * over a subset (a size bucket, see band_plan_ragged) writes only its systems' rows of
   * x.  Accepted by band_solve (without factors), band_solve_batch and band_sip with
   * width 0 (which then needs sys_status); the other calls return BAND_ERR_ARG. */
  const int64_t* systems;
} band_desc;

/* How the fused direct sweep (NTDM/NPDM, and the numeric sweep of STDM/SPDM) maps onto
 * threads; solves with stored factors, per-system bandwidths and the symbolic fix-up
 * always take one thread per system.
 * BAND_SCHED_THREAD: one thread per system runs the whole recurrence of Sec. 1.
 * BAND_SCHED_TWO_SIDED: two threads per system.  One eliminates rows 0 .. m-1 top-down
 *   (m = ceil(n/2); NPDM's own operations on those rows), the other rows n-1 .. m
 *   bottom-up (the same recurrence on the row- and column-reversed system, i.e. the UL
 *   factorisation of that block); they meet in a 4x4 (PD) / 2x2 (TD) interface system
 *   solved with partial pivoting, then back-substitute their halves.  Each dependent
 *   chain is half as long and the launch has twice the threads.  A zero pivot in either
 *   half, or a singular interface system, sends an STDM/SPDM system to the symbolic
 *   fix-up (as a zero pivot of the one-thread sweep does); for NTDM/NPDM it makes the
 *   first thread redo the system with NPDM alone, so BAND_ERR_ZERO_PIVOT still means that
 *   NPDM's order meets an exactly zero pivot -- except when x aliases f (f is then
 *   already overwritten), where it means a zero pivot of the two-sided elimination.  A
 *   system that NPDM's order would fail on in its lower half may be solved (status OK).
 *   Systems with fewer than 4 (PD) / 2 (TD) rows are solved by one thread.  Needs one
 *   half bandwidth for the batch.
 * BAND_SCHED_PARTITIONED: P = desc->chunks lanes per system: 32 / P systems a warp for
 *   P <= 32, one system per block of P / 32 warps beyond (band_solve only; inside
 *   band_solve_batch, whose tasks are single warps, P > 32 runs as P = 32).  Lane k
 *   eliminates rows [k n / P, (k+1) n / P) (about) with NPDM's recurrence, carrying the
 *   columns through which the chunk couples to its neighbours' boundary rows (the SPIKE
 *   partition); the chunks' boundary rows form a block-tridiagonal system of P blocks
 *   of 4 (PD) / 2 (TD) unknowns, eliminated from both ends by two lanes (a 2x2 (PD) /
 *   1x1 (TD) pivot block per chunk, partial pivoting) that meet in a 4x4 / 2x2 system;
 *   then every lane back-substitutes its chunk.  About 2.3x (PD) / 1.8x (TD) NPDM's
 *   arithmetic per row, for a dependent chain of n / P rows: for batches with too few systems to
 *   fill the GPU, and for the longest systems of a ragged batch.  A zero pivot in a
 *   chunk or a singular interface block sends an STDM/SPDM system to the symbolic fix-up
 *   and makes the first lane redo an NTDM/NPDM system with NPDM alone (BAND_ERR_ZERO_PIVOT
 *   means that NPDM's order meets an exactly zero pivot, also when x aliases f).
 *   Systems with fewer than 8 P rows are solved by one lane.  Needs one half bandwidth
 *   for the batch; any layout, ragged packings included.  Workspace: five (PD) / four
 *   (TD) scratch arrays of ceil(n / P) * P rows for nsys rounded up to 32 / P systems
 *   (the largest over P when chunks is 0).
 *   Accuracy: a chunk restarts NPDM's recurrence at its first row and the interface has
 *   no pivoting across blocks, so on matrices that are not diagonally dominant either
 *   can meet pivots far smaller than NPDM's; a pivot 2^-17 (FP64) / 2^-10 (FP32) below
 *   its row's largest entry, or an interface block as close to singular, is handled
 *   like a zero pivot (the system is redone as above).  On dominant matrices no system
 *   is redone.  Chunk counts are 8 ... 256 (4 is not offered).
 * BAND_SCHED_GRID: one system, or a few, over the whole GPU (the paper's single
 *   systems of up to 10^8 rows, Table 3 and Table 5).  band_solve only, NTDM / NPDM,
 *   uniform layouts, no stored factors, desc->chunks 0; the library cuts every system
 *   into P chunks of at least 64 rows so that the batch fills one wave of 16 warps per
 *   SM (P = 77824 / nsys on a GB300, fewer for short systems; one chunk below 128
 *   rows).  Lane c eliminates chunk c as the partitioned schedule does and writes its
 *   boundary rows' block row of the reduced system L_c y_{c-1} + y_c + U_c y_{c+1} = g_c
 *   (y_c: the chunk's top and bottom 2 (PD) / 1 (TD) unknowns); block cyclic reduction
 *   solves that system in ceil(log2 P) launches each way (2K x 2K blocks, partial
 *   pivoting inside each block); every lane then back-substitutes its chunk.  About
 *   2.4x NPDM's arithmetic per row plus the reduction's ~500 operations per chunk; x may
 *   alias f.  A chunk pivot 2^-17 (FP64) / 2^-10 (FP32) below its row's largest entry,
 *   or a reduction block as close to singular, ends the system with
 *   BAND_ERR_ZERO_PIVOT (this schedule's elimination order met a pivot it cannot use;
 *   another schedule may solve it); on diagonally dominant systems that does not
 *   happen.  Workspace: five (PD) / four (TD) arrays of ceil(n / P) * P * nsys rows plus
 *   ~450 B per chunk.  Other calls return BAND_ERR_ARG for this schedule.
 * BAND_SCHED_AUTO: in band_solve, band_solve_static and band_adjoint, an NTDM / NPDM
 *   solve of a uniform batch of one bandwidth with n >= 256 and fewer than 32 systems
 *   per SM of the GPU (the two-sided schedule would leave fewer than two warps per SM)
 *   runs PARTITIONED, with the chunk count chosen as for chunks == 0; a system whose
 *   partitioned elimination fails (a chunk pivot the guard rejects, possible on rows
 *   that are not diagonally dominant) is solved again, from f, by a second launch on
 *   the schedule described next, and band_workspace_size covers both.  Otherwise, and
 *   always inside band_solve_batch (where the other problems fill the GPU): TWO_SIDED
 *   for uniform-bandwidth solves with n >= 32
 *   that are not a whole ragged packing (ragged id lists, i.e. size buckets, qualify)
 *   and, for NTDM/NPDM, whose x does not alias f; THREAD otherwise.  band_autotune
 *   replaces the rule by measurement. */
typedef enum {
  BAND_SCHED_AUTO = 0,
  BAND_SCHED_THREAD = 1,
  BAND_SCHED_TWO_SIDED = 2,
  BAND_SCHED_PARTITIONED = 3,
  BAND_SCHED_GRID = 4
} band_schedule;

/* Bytes of workspace that the operation `op` needs for `desc` (0 = none).  op is one
 * of the BAND_OP_* values; `method` as for the call it serves (ignored where n/a). */
enum {
  BAND_OP_SOLVE = 0,      /* band_solve */
  BAND_OP_FACTOR = 1,     /* band_factor: returns the size of the factor buffer */
  BAND_OP_SIP = 2,        /* band_sip (uses sip_width) */
  BAND_OP_REFINE = 3,     /* band_refine_solve */
  BAND_OP_ADJOINT = 4,    /* band_adjoint */
  BAND_OP_DET = 5,        /* band_det */
  BAND_OP_ADI = 6,        /* band_adi_step (desc describes the grid, see there) */
  BAND_OP_SIP2D = 7       /* band_sip2d */
};
size_t band_workspace_size(const band_desc* desc, int32_t op, int32_t method, int32_t sip_width);

/* Solve A x = f for every system (NTDM/NPDM fused factor + solve, or STDM/SPDM:
 * the same sweep with an exact zero-pivot test, after which only the flagged
 * systems are redone in truncated Laurent arithmetic in t and evaluated at t -> 0;
 * their determinant limit decides BAND_ERR_SINGULAR).
 * The symbolic fix-up runs one warp per flagged system; its series carry
 * double-double coefficients of t^-15 .. t^3, and a system that runs out of that
 * window is redone with t^-15 .. t^16 (BAND_ERR_SYMBOLIC_RANGE beyond).  A coefficient
 * that comes out below 2^-80 of the magnitude of the terms it was summed from is taken
 * as exactly zero (rounding residue of an exact cancellation).  The workspace holds
 * the series rows of min(nsys, 152) flagged systems at a time (one per SM of a GB300;
 * 1584 * n bytes each); a larger workspace lets more of them run at once, up to
 * min(nsys, 1216).
 * diag[5] = {a, b, c, d, e} device pointers (a, e unused and may be NULL for TD).
 * factors: NULL for the fused path, or a buffer filled by band_factor() for the same
 * desc and diagonals (then only NTDM/NPDM).  ws: device workspace of ws_bytes >=
 * band_workspace_size(desc, BAND_OP_SOLVE, method, 0). */
band_status band_solve(const band_desc* desc, int32_t method, const void* factors,
                       const void* const diag[5], const void* f, void* x,
                       int32_t* sys_status, void* ws, size_t ws_bytes, void* stream);

/* One time step of a nonlinear parabolic PDE by the alternating direction implicit
 * method, the setting of the paper's band solves (Sec. 1: an ADI step solves N
 * independent TD or PD systems per direction):
 *   u_t = u_xx + u_yy + lambda u (1 - u) + s(x, y)  on the unit square, u = 0 on the
 *   boundary, n x n interior points, h = 1 / (n + 1), u[y * n + x] (row-major, device).
 * Second differences: the 3-point stencil (1, -2, 1) / h^2 (grid->half_bw 1: TD systems,
 * NTDM) or the fourth-order 5-point stencil (-1, 16, -30, 16, -1) / (12 h^2) (half_bw 2:
 * PD systems, NPDM) whose point beyond the boundary is the odd reflection of the first
 * interior point; the nonlinear term and s stay on the right-hand side, evaluated at
 * the latest values.  One Peaceman-Rachford step, theta = tau / 2:
 *   (I - theta D_x) u* = u + theta (D_y u + g(u) + s),   then
 *   (I - theta D_y) u  = u* + theta (D_x u* + g(u*) + s),   g(u) = lambda u (1 - u):
 * n row systems (contiguous), then n column systems (interleaved), each solved by
 * band_solve on the automatic schedule.  grid: half_bw 1 or 2, dtype BAND_F64,
 * nsys = n = the grid size (n >= 3), hbw / offsets NULL, schedule 0, chunks 0 (strides
 * ignored).
 * source: n * n values or NULL (s = 0).  u is updated in place.  sys_status (may be
 * NULL): 2n entries, the row systems' statuses then the column systems'.  ws:
 * band_workspace_size(grid, BAND_OP_ADI, 0, 0) bytes.  Asynchronous on `stream` (the
 * right-hand sides, the constant diagonals and the solves are kernels only), so that a
 * caller can capture a number of steps in one CUDA graph. */
band_status band_adi_step(const band_desc* grid, double tau, double lambda, const double* source,
                          double* u, int32_t* sys_status, void* ws, size_t ws_bytes,
                          void* stream);

/* Stone's method (Sec. 2, Algorithm 1) on a batch of two-dimensional five-point
 * systems, where ILU(0) drops the fill that the pattern creates (on the PD band it is
 * the exact LU and Algorithm 1 stops after one update).  System s is an nx x ny grid,
 * unknown k = y nx + x (desc->n = nx * ny, uniform layout, FP64); row k of the matrix
 * holds diag[0][k] at column k - nx, diag[1][k] at k - 1, diag[2][k] at k, diag[3][k]
 * at k + 1, diag[4][k] at k + nx (entries that would leave the grid are read but never
 * used).  ILU(0) with L's and U's entries on A's pattern, then from x^0 = 0 updates
 * LU x^{j+1} = (LU - A) x^j + f until max|f - A x| < tol (status OK) or max_it updates
 * (BAND_ERR_NOT_CONVERGED); a zero ILU(0) pivot is BAND_ERR_ZERO_PIVOT.  One warp per
 * system when nx <= 32 (lane x takes column x; the substitutions run on anti-diagonal
 * wavefronts), one thread per system otherwise; the same operations per unknown either
 * way (desc->schedule AUTO, chunks 0).  The warp kernel reads each system's elements
 * consecutively: a batch with elem_stride != 1 is copied system-major into the
 * workspace (the diagonals, f and x; 7 nsys n doubles more workspace), solved there and
 * x copied back, with the same bits as a contiguous batch.  A system whose ILU(0)
 * fails keeps the caller's x.  x must not alias f; iters, resid (per system) may be
 * NULL.  ws: band_workspace_size(desc, BAND_OP_SIP2D, 0, 0). */
band_status band_sip2d(const band_desc* desc, int64_t nx, const void* const diag[5],
                       const double* f, double* x, double tol, int32_t max_it, int32_t* iters,
                       double* resid, int32_t* sys_status, void* ws, size_t ws_bytes,
                       void* stream);

/* band_solve with method BAND_MNPDM (Sec. 1: the PD method that takes the sparsity of the
 * outer diagonals into account; Sec. 3.2 Remark 2: the Gaussian elimination that turns the
 * PD matrix into a TD one costs 16 operations per row with both outer entries nonzero):
 * bottom-up, every nonzero e_i is eliminated with row i+1; top-down, every nonzero a_i
 * with row i-1; NTDM then solves the TD system.  For PD batches (half_bw 2, no hbw, no id
 * list), any layout, FP64 or FP32, factors NULL; x may alias f.  desc->schedule AUTO on a
 * uniform batch: the eliminations run one thread per row (a chain of consecutive rows
 * with outer entries by the thread of its first row), the TD system goes to the
 * workspace laid out like the input and is solved as band_solve's NTDM on its automatic
 * schedule; THREAD, or a ragged packing: one thread per system for all three sweeps.  A zero divisor of the elimination (the superdiagonal of
 * row i+1, or the subdiagonal of row i-1, as they stand then) or a zero NTDM pivot gives
 * BAND_ERR_ZERO_PIVOT.  No pivoting: meant for K << n rows with outer entries (on fully
 * pentadiagonal matrices its multipliers are ratios of off-diagonal entries and it loses
 * accuracy that NPDM keeps).  Workspace: band_workspace_size(desc, BAND_OP_SOLVE,
 * BAND_MNPDM, 0): on AUTO four arrays of the input's span, nsys flags and NTDM's
 * workspace; on THREAD five arrays of nsys rounded up to 32 times n elements. */

/* LU factors of NTDM/NPDM (gamma, 1/mu, alpha, beta per row; opaque layout) into
 * `factors`, a device buffer of band_workspace_size(desc, BAND_OP_FACTOR, method, 0)
 * bytes, for repeated band_solve() calls and for band_adjoint(). */
band_status band_factor(const band_desc* desc, int32_t method, const void* const diag[5],
                        void* factors, size_t factors_bytes, int32_t* sys_status, void* stream);

/* SIP / Stone method (Algorithm 1) on PD systems (TD: a = e = 0 is used), FP64 only.
 * width == 0: Algorithm 1 as printed, with the exact substitutions of the ILU(0)
 * factors; width > 0: Hotelling-Bodewig inverses of L and U kept to `width`
 * diagonals (at most 8), iterated from X_0 = diag^{-1} until
 * max|X_{k+1}-X_k| <= hb_tol max|X_k| or hb_max_it, and the update
 * x += U~^{-1} L~^{-1} (f - A x).  Stops per system when max|f - A x| < tol or after
 * max_it updates; with width == 0 also when an update from the second on does not
 * lower max|f - A x| (exact ILU(0) factors leave K = LU - A at the rounding level, so
 * the residual has reached its floor; status NOT_CONVERGED).  iters (int32[nsys]) and
 * resid (double[nsys], max |f - A x|) may be NULL.  x must not alias f.
 * desc->schedule (band_schedule) applies to width == 0: on BAND_SCHED_TWO_SIDED (and
 * AUTO for n >= 32, non-ragged) the first update x^1 = (LU)^{-1} f runs with two
 * threads per system, the lower half of the exact ILU(0) = LU factorisation taken
 * bottom-up (equal in exact arithmetic; the residual and the stop test are
 * Algorithm 1's); later updates use the top-down factors, rebuilt for the lower half.
 * As for the direct sweeps, a system whose top-down order meets a zero pivot only in
 * its lower half may then be solved in one update (status OK). */
band_status band_sip(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                     double tol, int32_t max_it, int32_t width, int32_t hb_max_it, double hb_tol,
                     int32_t* iters, double* resid, int32_t* sys_status, void* ws, size_t ws_bytes,
                     void* stream);

/* One batched launch over several independent problems (at most BAND_MAX_BATCH).
 * The ADI step solves N systems per grid line and direction (Sec. 1); its solves are
 * independent, so they share one kernel launch in which every warp takes consecutive
 * systems of one problem (32 on one thread each, 16 two-sided, 32 / P partitioned with
 * P <= 32; a larger desc->chunks runs as P = 32), filling the GPU even when each problem
 * alone has too few systems.
 * op = BAND_OP_SOLVE: method as for band_solve (fused, no stored factors; STDM/SPDM
 *   systems with a zero pivot go through one batched symbolic fix-up launch).
 * op = BAND_OP_SIP: Algorithm 1 with exact substitutions (width 0) on FP64 PD
 *   systems, with tol and max_it as for band_sip; iters / resid may be NULL.  One
 *   thread per system whatever desc->schedule says.
 * Each problem brings its own workspace of band_workspace_size(desc, op, method, 0)
 * bytes.  Argument checks as for the single calls; the first failing problem's code
 * is returned and nothing is launched. */
#define BAND_MAX_BATCH 64
typedef struct {
  int32_t op;                /* BAND_OP_SOLVE or BAND_OP_SIP */
  int32_t method;            /* band_method (BAND_OP_SOLVE) */
  const band_desc* desc;     /* host pointer */
  const void* diag[5];
  const void* f;
  void* x;
  int32_t* sys_status;
  void* ws;
  size_t ws_bytes;
  double tol;                /* BAND_OP_SIP */
  int32_t max_it;            /* BAND_OP_SIP */
  int32_t* iters;            /* BAND_OP_SIP, may be NULL */
  double* resid;             /* BAND_OP_SIP, may be NULL */
} band_problem;
band_status band_solve_batch(const band_problem* problems, int32_t count, void* stream);

/* Mixed precision: PD/TD systems stored in FP32 (desc->dtype = BAND_F32 describes
 * diag32), right-hand side and solution in FP64 with the same strides.  FP32 NPDM/NTDM
 * solve, then refinement steps r = f - A x (A = the FP64 values of the FP32 diagonals),
 * delta = s * solve32(r / s) with s a power of two near max|f| 2^-20, x += delta,
 * until max|delta| <= rel_stop * max|x| or max_steps steps.  steps (int32[nsys]) may be
 * NULL.  The FP32 solves run on desc32->schedule (and chunks) as band_solve's would
 * (not BAND_SCHED_GRID).
 * band_refine_solve forms the residual and the update in FP64 (fused multiply-adds on
 * the caller's FP64 x; x must not alias f).  band_refine_solve_ex with
 * flags = BAND_REFINE_PAIRS keeps x, f, the residual and the update as pairs of FP32
 * numbers with error-free transformations instead (about 2^-48 relative; no FP64
 * arithmetic until x is assembled at the end; x may alias f); flags = 0 is
 * band_refine_solve. */
#define BAND_REFINE_PAIRS 1
band_status band_refine_solve(const band_desc* desc32, const void* const diag32[5],
                              const double* f, double* x, double rel_stop, int32_t max_steps,
                              int32_t* steps, int32_t* sys_status, void* ws, size_t ws_bytes,
                              void* stream);
band_status band_refine_solve_ex(const band_desc* desc32, const void* const diag32[5],
                                 const double* f, double* x, double rel_stop, int32_t max_steps,
                                 int32_t flags, int32_t* steps, int32_t* sys_status, void* ws,
                                 size_t ws_bytes, void* stream);

/* Adjoint of x = A^{-1} f for a loss L with dL/dx = w (FP64, NTDM/NPDM factorisation):
 * lambda = A^{-T} w by the transposed sweeps of the LU factors, then
 * grad_f = lambda, grad_a[i] = -lambda_i x_{i-2}, grad_b[i] = -lambda_i x_{i-1},
 * grad_c[i] = -lambda_i x_i, grad_d[i] = -lambda_i x_{i+1}, grad_e[i] = -lambda_i x_{i+2}
 * (out-of-matrix slots receive 0; TD: grad_a, grad_e may be NULL).  factors: NULL to
 * refactor from diag, or band_factor()'s buffer.  Without factors on a uniform layout,
 * A^T (row-aligned diagonals e_{i-2}, d_{i-1}, c_i, b_{i+1}, a_{i+2}) is formed in the
 * workspace and solved as a band system on desc->schedule (as band_solve; the same
 * lambda in exact arithmetic, with ZERO_PIVOT referring to A^T's elimination order);
 * with factors, or on a ragged layout, by the transposed sweeps of the LU factors. */
band_status band_adjoint(const band_desc* desc, int32_t method, const void* factors,
                         const void* const diag[5], const void* x, const void* w,
                         void* const grad_diag[5], void* grad_f, int32_t* sys_status,
                         void* ws, size_t ws_bytes, void* stream);

/* Determinant of every system in O(n) (Sec. 3.2, Remark 1: the symbolic algorithm
 * yields det A as the limit of the product of its pivots), FP64 only.
 * desc->half_bw (or desc->hbw per system) gives the bandwidth; the schedule fields are
 * ignored; id lists (desc->systems) are not accepted.  diag as for band_solve.
 * Output per system s: det A = det_mant[s] * 2^det_exp[s], with 0.5 <= |det_mant[s]| < 1
 * (device arrays of nsys entries), and sys_status[s] (required):
 *   BAND_OK              the product of the pivots of the NPDM / NTDM factorisation, or,
 *                        for a system whose factorisation meets a pivot that is exactly
 *                        zero, the limit t -> 0 of the product of the pivots of the
 *                        symbolic factorisation (zero pivots replaced by t, as STDM /
 *                        SPDM do), i.e. the product of the pivots' leading coefficients;
 *   BAND_ERR_SINGULAR    that limit is 0 (det_mant = 0, det_exp = 0);
 *   BAND_ERR_SYMBOLIC_RANGE  the Laurent window ran out (det_mant = 0);
 *   BAND_ERR_NONFINITE   an Inf or NaN entered the product.
 * Accuracy: the rounding of n pivots, about n ulps relative, more where the pivots
 * grow (no pivoting).  ws: band_workspace_size(desc, BAND_OP_DET, 0, 0) bytes. */
band_status band_det(const band_desc* desc, const void* const diag[5], double* det_mant,
                     int64_t* det_exp, int32_t* sys_status, void* ws, size_t ws_bytes,
                     void* stream);

/* NTDM / NPDM solve for callers that cannot allocate device memory (the paper has
 * no counterpart).  Some callers cannot allocate where they solve: code that must not
 * block on cudaMalloc's device-wide synchronisation, hosts that own every byte of
 * device memory through their own pool, or C callers without an allocator.  This call
 * is band_solve (method BAND_NTDM, BAND_NPDM or BAND_AUTO_NUMERIC, factors NULL, no id
 * list) without the workspace argument: its scratch rows come from an array of
 * BAND_STATIC_SCRATCH_BYTES that the library places in device memory on every GPU
 * that loads it, held until the process exits.  The first call on a device looks up
 * that array's device address (once per device, with that device current; again after
 * a cudaDeviceReset); make that first call before any stream capture.  desc->schedule
 * applies as for band_solve (not BAND_SCHED_GRID).  A batch whose workspace,
 * band_workspace_size(desc, BAND_OP_SOLVE, method, 0) for the same desc (the rule for
 * every layout and schedule), exceeds the array returns BAND_ERR_WORKSPACE; other
 * methods return BAND_ERR_ARG.  The array is shared by every call and keeps the last
 * call's contents (nothing in it needs to start at zero): calls whose kernels overlap
 * on one GPU race on it and must be serialised by the caller.  No device memory is
 * allocated. */
#define BAND_STATIC_SCRATCH_BYTES ((size_t)32 << 20)
band_status band_solve_static(const band_desc* desc, int32_t method, const void* const diag[5],
                              const void* f, void* x, int32_t* sys_status, void* stream);

/* ---------------------------------------------------------------- batch runtime
 * A ragged batch of thousands of systems of uneven size and mixed bandwidth runs best
 * as size buckets: systems of one half bandwidth whose sizes lie within a factor of two,
 * each bucket one problem of a band_solve_batch launch (id list: band_desc.systems).
 * Host-side planning, no device work. */
typedef struct {
  int64_t first;      /* first position of the bucket in `order` */
  int64_t count;      /* systems in the bucket */
  int64_t n_max;      /* largest system size in the bucket */
  int32_t half_bw;    /* 1 (TD) or 2 (PD) */
  int32_t pad;
} band_bucket;

/* Sort the nsys systems of a ragged packing by (half bandwidth, floor(log2 n), n
 * descending) and cut them into buckets of one half bandwidth and one power-of-two
 * size range.  offsets (nsys + 1 entries) and hbw (nsys entries, or NULL: half_bw for
 * every system) are HOST arrays.  Writes order[0 .. nsys-1] (system ids, bucket by
 * bucket) and the buckets; returns their number, or -1 on bad arguments (a size < 1, a
 * bandwidth other than 1 or 2) or when more than max_buckets would be needed. */
int32_t band_plan_ragged(const int64_t* offsets, const int8_t* hbw, int32_t half_bw, int64_t nsys,
                         int64_t* order, band_bucket* buckets, int32_t max_buckets);

/* Autotuner of the schedules (band_schedule) of a band_solve_batch list.  Problems it
 * may decide: fused direct solves of one half bandwidth whose desc->schedule is
 * BAND_SCHED_AUTO; the others keep their desc->schedule and desc->chunks.
 * 1. Each such problem is timed alone as a band_solve_batch launch on the thread and
 *    two-sided schedules (one warm-up, then the best of `reps` runs; CUDA events on
 *    `stream`) and gets the faster.  These decisions are cached for the process per
 *    (dtype, method, half bandwidth, ceil(log2 n), ceil(log2 nsys), layout, x aliasing
 *    f), so later calls reuse them without timing.
 * 2. With flags & BAND_TUNE_JOINT: the whole list is timed as one launch, and the
 *    problems (n >= 64, largest n first) are moved in turn to BAND_SCHED_PARTITIONED
 *    with 8, 16 or 32 chunks (those that leave chunks of 16 rows or more); a move is
 *    kept when it shortens the launch by 2 % or more.  A pass over the problems not yet
 *    moved ends after two problems in a row gain nothing; passes repeat (at most four)
 *    until one moves nothing, since a move can pay only once a longer chain elsewhere
 *    has been cut.  Only problems whose ws_bytes cover the partitioned
 *    schedule's workspace (band_workspace_size with schedule BAND_SCHED_PARTITIONED)
 *    and whose every row is diagonally dominant (|c| >= |a| + |b| + |d| + |e|, checked
 *    on the device) are tried: on other matrices a chunk's block can be far worse
 *    conditioned than the whole matrix.  Not cached: the result depends on the whole
 *    list.  Then the list, on the schedules chosen, is timed with 1, 2 and 4 warps per
 *    block of band_solve_batch's kernel, and the fastest becomes this device's block
 *    size for every later band_solve_batch call of the process (2 before any tuning).
 * Persistence: the decisions of step 1 and the block size are appended as JSON lines
 *   {"gpu": "<device name>", "cc": "<major>.<minor>", "cuda": <runtime version>,
 *    "kind": "schedule", "key": [dtype, method, half_bw, ceil log2 n, ceil log2 nsys,
 *    layout, x aliases f], "value": <band_schedule>}
 *   {"gpu": ..., "cuda": ..., "kind": "batch_warps", "value": <1, 2 or 4>}
 * to the file named by the environment variable BAND_TUNE_CACHE (unset:
 * $HOME/.cache/libband/tune.jsonl; empty: no file), and the lines of this GPU and CUDA
 * version are read back by the first band_autotune call of a process on each device
 * (later lines win), so a new process skips the timings already made.  A file that
 * cannot be read or written is ignored.
 * Writes schedules[i] and, if chunks is not NULL, chunks[i] (the desc fields to set).
 * The trial runs solve the problems (outputs are overwritten).  Synchronises the
 * stream; do not call while it is being captured.  Returns BAND_ERR_ARG (also for
 * unknown flags) / BAND_ERR_CUDA / the solve's error. */
#define BAND_TUNE_JOINT 1
band_status band_autotune(const band_problem* probs, int32_t count, int32_t reps, int32_t flags,
                          int32_t* schedules, int32_t* chunks, void* stream);

/* The warps per block (1, 2 or 4) that band_solve_batch launches with on CUDA device
 * `device`, or -1 for a device number outside 0..63.  No CUDA call. */
int32_t band_batch_warps(int32_t device);

/* Forget the autotuner's in-process decisions (all devices) and restore the default
 * block size; the persisted file is left as it is and is read again by the next
 * band_autotune call. */
void band_autotune_reset(void);

/* Diagnostic (the paper has no counterpart): measures this GPU's FP64 fused
 * multiply-add rate in FMA/s with a short register-only kernel on `stream` and waits
 * for it.  scratch: device buffer of at least 8 * 256 * 8 * (SM count) bytes.
 * Returns a negative value on error.  The FP64 recurrences are bounded by this rate. */
double band_fp64_fma_rate(void* scratch, size_t scratch_bytes, void* stream);

/* Human-readable name of a status code (static string). */
const char* band_status_str(int32_t status);

/* Library version string (static). */
const char* band_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BAND_H */
