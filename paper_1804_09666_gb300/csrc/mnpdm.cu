// mnpdm.cu -- MNPDM: the PD method that takes the sparsity of the outer diagonals into
// account (Veneva & Ayriyan, arXiv:1804.09666, Sec. 1), for pentadiagonal systems
// whose rows mostly have a_i = e_i = 0.  A Gaussian elimination turns the PD matrix
// into a TD one at 16 operations per row that carries both outer entries (Sec. 3.2,
// Remark 2); NTDM then solves the TD system.  Reading of the elimination (the paper
// prints neither its steps nor their order): bottom-up, every nonzero e_i (column
// i+2) is eliminated with row i+1, which by then has no entry beyond column i+2,
//   m = e_i / D_{i+1};  B_i -= m a_{i+1};  C_i -= m B_{i+1};  D_i -= m C_{i+1};  F_i -= m F_{i+1};
// then top-down every nonzero a_i (column i-2) with row i-1, by then tridiagonal,
//   m = a_i / B_{i-1};  B_i -= m C_{i-1};  C_i -= m D_{i-1};  F_i -= m F_{i-1},
// with (B, C, D, F) a row's sub-, main and superdiagonal entries and right-hand side as
// they stand.
//
// Uniform batches on the automatic schedule: the eliminations touch only the rows with
// nonzero outer entries and the rows of a chain of such rows (consecutive rows with
// e != 0, or with a != 0) depend only on each other, so both run one thread per row:
//  1. every row with e_i = 0 copies (b, c, d, f) into the workspace's (B, C, D, F);
//     the bottom row of each chain of e != 0 rows (its row i+1 has e = 0 and is the
//     pivot row as it stands) eliminates the chain upwards and writes its rows;
//  2. the top row of each chain of a != 0 rows eliminates it downwards in place;
//  3. the tridiagonal system (B, C, D, F), laid out like the input, goes to band_solve's
//     NTDM on its automatic schedule (two-sided, or partitioned for a small batch),
//     skipping the systems whose elimination met a zero divisor.
// NTDM then carries the per-row work: 8 FP64 instructions a row against NPDM's 14.
// Ragged packings and the thread schedule: one thread per system, three sweeps:
//  1. bottom-up: the e eliminations.  Only rows with e_i != 0 are changed, and only
//     their (B, C, D, F) are written to the workspace; the sweep reads e and, at those
//     rows, the rows involved, so with K << n it reads little more than e.
//  2. top-down: each row as it stands after sweep 1, its a elimination, and NTDM's
//     forward recurrence (mu_i = C_i - B_i alpha_{i-1}, alpha_i = D_i / mu_i,
//     z_i = (F_i - B_i z_{i-1}) / mu_i, the reciprocal taken once); alpha to the
//     workspace, z to x.
//  3. bottom-up: x_i = z_i - alpha_i x_{i+1}.
// A zero divisor of the elimination or a zero pivot of NTDM is BAND_ERR_ZERO_PIVOT.
// Elimination divisions are IEEE divisions (rare rows); NTDM's reciprocals rcp.
#include <cstdint>

#include "api_util.h"
#include "common.cuh"
#include "kernels.h"

namespace band {

namespace {

template <typename T>
struct MnpdmArgs {
  Layout L;
  Spill W;
  const T *a, *b, *c, *d, *e, *f;
  T* x;
  T *Bm, *Cm, *Dm, *Fm;    // rows changed by sweep 1, interleaved by system like alpha
  T* al;
  int32_t* status;
};

// Loads of one row of a system (the raw entries sweep 2 may need; e decides whether
// sweep 1 changed the row).
template <typename T>
struct MRow {
  T a, b, c, d, e, f;
};
template <typename T>
__device__ __forceinline__ MRow<T> mload(const MnpdmArgs<T>& p, int64_t q) {
  return MRow<T>{ldro(p.a + q), ldro(p.b + q), ldro(p.c + q), ldro(p.d + q), ldro(p.e + q), p.f[q]};
}

template <typename T>
__global__ void __launch_bounds__(32 * SweepWarps<T>::value) k_mnpdm(const MnpdmArgs<T> p) {
  extern __shared__ __align__(16) unsigned char stage_mem[];
  void* stage = stage_mem + (threadIdx.x >> 5) * stage_bytes_per_warp<T>();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.L.nsys) return;
  const int64_t s = p.L.sys(t);
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(t), ws = p.W.stride();
  bool fail = false;
  constexpr int kB = 8;     // rows whose loads are issued together
  // ---- sweep 1 (bottom-up): (B1, C1, D1, F1) = row i+1 as it stands
  {
    T B1 = 0, C1 = 0, D1 = 0, F1 = 0;
    bool have1 = false;   // row i+1's values are in registers (changed rows always are)
    for (int64_t top = n - 3; top >= 0 && !fail; top -= kB) {
      T ev[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) ev[u] = top - u >= 0 ? ldro(p.e + q0 + (top - u) * es) : T(0);
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int64_t i = top - u;
        if (i < 0 || fail) break;
        const int64_t q = q0 + i * es;
        const T ei = ev[u];
        if (is_zero(ei)) {
          have1 = false;
          continue;
        }
        const int64_t q1 = q + es;
        if (!have1) {       // row i+1 unchanged: its own entries
          B1 = ldro(p.b + q1);
          C1 = ldro(p.c + q1);
          D1 = ldro(p.d + q1);
          F1 = ldro(p.f + q1);
        }
        if (is_zero(D1)) {
          fail = true;
          break;
        }
        const T m = ei / D1;
        const T a1 = i + 1 >= 2 ? ldro(p.a + q1) : T(0);
        const T Bi = i >= 1 ? fma(-m, a1, ldro(p.b + q)) : T(0);
        const T Ci = fma(-m, B1, ldro(p.c + q));
        const T Di = fma(-m, C1, ldro(p.d + q));
        const T Fi = fma(-m, F1, p.f[q]);
        const int64_t w = w0 + i * ws;
        p.Bm[w] = Bi;
        p.Cm[w] = Ci;
        p.Dm[w] = Di;
        p.Fm[w] = Fi;
        B1 = Bi; C1 = Ci; D1 = Di; F1 = Fi;
        have1 = true;
      }
    }
  }
  // ---- sweep 2 (top-down): the a eliminations and NTDM's forward recurrence.  Raw rows
  // of interleaved systems come through the warp's shared-memory ring (cp.async,
  // StageDepth rows ahead, as in the NPDM sweeps); other layouts two rows ahead in
  // registers.
  T Bp = 0, Cp = 0, Dp = 0, Fp = 0;    // row i-1 as it stands (tridiagonal)
  T al1 = 0, z1 = 0;
  auto step = [&](int64_t i, const MRow<T>& r0) -> bool {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * ws;
    const bool changed = i + 2 < n && !is_zero(r0.e);
    T B, C, D, F;
    if (changed) {
      B = p.Bm[w]; C = p.Cm[w]; D = p.Dm[w]; F = p.Fm[w];
    } else {
      B = i >= 1 ? r0.b : T(0);
      C = r0.c;
      D = i + 1 < n ? r0.d : T(0);
      F = r0.f;
    }
    if (i >= 2 && !is_zero(r0.a)) {
      if (is_zero(Bp)) return false;
      const T m = r0.a / Bp;
      B = fma(-m, Cp, B);
      C = fma(-m, Dp, C);
      F = fma(-m, Fp, F);
    }
    Bp = B; Cp = C; Dp = D; Fp = F;
    const T mu = fma(-al1, B, C);
    if (is_zero(mu)) return false;
    const T r = rcp<T>(mu);
    const T alv = D * r;
    const T zv = fma(-z1, B, F) * r;
    p.al[w] = alv;
    p.x[q] = zv;
    al1 = alv;
    z1 = zv;
    return true;
  };
  if (!fail && stage && !p.L.offsets && p.L.ss == 1) {
    constexpr int Dp_ = StageDepth<T>::value;
    const RowRing<T, 6, Dp_> ring{static_cast<T*>(stage), (int)(threadIdx.x & 31)};
    const T* src[6] = {p.a, p.b, p.c, p.d, p.e, p.f};
#pragma unroll
    for (int j = 0; j < Dp_ - 1; ++j) {
      if (j < n) ring.issue(j, src, q0 + j * es);
      else ring.skip();
    }
    for (int64_t i = 0; i < n; ++i) {
      const int64_t ip = i + Dp_ - 1;
      if (ip < n) ring.issue((int)(ip & (Dp_ - 1)), src, q0 + ip * es);
      else ring.skip();
      cp_async_wait<Dp_ - 1>();
      const int slot = (int)(i & (Dp_ - 1));
      const MRow<T> r0{ring.get(slot, 0), ring.get(slot, 1), ring.get(slot, 2),
                       ring.get(slot, 3), ring.get(slot, 4), ring.get(slot, 5)};
      if (!step(i, r0)) {
        fail = true;
        break;
      }
    }
    cp_async_wait<0>();
  } else if (!fail) {
    MRow<T> r0{}, r1{};
    if (n > 0) r0 = mload(p, q0);
    if (n > 1) r1 = mload(p, q0 + es);
    for (int64_t i = 0; i < n; ++i) {
      MRow<T> r2{};
      if (i + 2 < n) r2 = mload(p, q0 + (i + 2) * es);
      if (!step(i, r0)) {
        fail = true;
        break;
      }
      r0 = r1;
      r1 = r2;
    }
  }
  if (fail) {
    set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
    return;
  }
  // ---- sweep 3 (bottom-up): back-substitution, loads in blocks of kB rows
  T x1 = 0;
  bool bad = false;
  for (int64_t top = n - 1; top >= 0; top -= kB) {
    T av[kB], zv[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      av[u] = zv[u] = T(0);
      if (top - u >= 0) {
        av[u] = p.al[w0 + (top - u) * ws];
        zv[u] = p.x[q0 + (top - u) * es];
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int64_t i = top - u;
      if (i < 0) break;
      const T xi = fma(-av[u], x1, zv[u]);
      p.x[q0 + i * es] = xi;
      bad |= not_finite(xi);
      x1 = xi;
    }
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

// ---- the row-parallel path (uniform batches)
template <typename T>
struct MnRows {
  Layout L;
  const T *a, *b, *c, *d, *e, *f;
  T *B, *C, *D, *F;     // the tridiagonal system, at the input's indices
  int32_t* skip;        // per system: an elimination met a zero divisor
  int32_t* status;
};

// (i, s) of the idx-th element of a uniform batch, the unit-stride index running first
__device__ __forceinline__ void mn_elem(const Layout& L, int64_t idx, int64_t& i, int64_t& s) {
  if (L.ss == 1) { s = idx % L.nsys; i = idx / L.nsys; }
  else { i = idx % L.n; s = idx / L.n; }
}

template <typename T>
__device__ __forceinline__ void mn_fail(const MnRows<T>& p, int64_t s) {
  p.skip[s] = 1;
  set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
}

// step 1: copies, and the e chains bottom-up
template <typename T>
__global__ void __launch_bounds__(256) k_mnpdm_e(const MnRows<T> p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.L.nsys * p.L.n) return;
  int64_t i, s;
  mn_elem(p.L, idx, i, s);
  const int64_t n = p.L.n, es = p.L.es, q0 = s * p.L.ss, q = q0 + i * es;
  const T ei = i + 2 < n ? ldro(p.e + q) : T(0);
  if (is_zero(ei)) {
    p.B[q] = i >= 1 ? ldro(p.b + q) : T(0);
    p.C[q] = ldro(p.c + q);
    p.D[q] = i + 1 < n ? ldro(p.d + q) : T(0);
    p.F[q] = p.f[q];
    return;
  }
  if (i + 3 < n && !is_zero(ldro(p.e + q + es))) return;   // not the chain's bottom
  // row i+1 (e = 0): the pivot row as it stands
  const int64_t q1 = q + es;
  T B1 = ldro(p.b + q1), C1 = ldro(p.c + q1), D1 = ldro(p.d + q1), F1 = p.f[q1];
  for (int64_t r = i;; --r) {
    const int64_t qr = q0 + r * es;
    if (is_zero(D1)) {
      mn_fail(p, s);
      return;
    }
    const T m = ldro(p.e + qr) / D1;
    const T a1 = r + 1 >= 2 ? ldro(p.a + qr + es) : T(0);
    const T Bi = r >= 1 ? fma(-m, a1, ldro(p.b + qr)) : T(0);
    const T Ci = fma(-m, B1, ldro(p.c + qr));
    const T Di = fma(-m, C1, ldro(p.d + qr));
    const T Fi = fma(-m, F1, p.f[qr]);
    p.B[qr] = Bi;
    p.C[qr] = Ci;
    p.D[qr] = Di;
    p.F[qr] = Fi;
    B1 = Bi; C1 = Ci; D1 = Di; F1 = Fi;
    if (r == 0 || is_zero(ldro(p.e + qr - es))) break;   // row r-1: its own thread's copy
  }
}

// step 2: the a chains top-down, in place
template <typename T>
__global__ void __launch_bounds__(256) k_mnpdm_a(const MnRows<T> p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.L.nsys * p.L.n) return;
  int64_t i, s;
  mn_elem(p.L, idx, i, s);
  const int64_t n = p.L.n, es = p.L.es, q0 = s * p.L.ss, q = q0 + i * es;
  if (i < 2 || is_zero(ldro(p.a + q)) || p.skip[s]) return;
  if (i - 1 >= 2 && !is_zero(ldro(p.a + q - es))) return;  // not the chain's top
  // row i-1 (a = 0): the pivot row as step 1 left it
  const int64_t qp = q - es;
  T Bp = p.B[qp], Cp = p.C[qp], Dp = p.D[qp], Fp = p.F[qp];
  for (int64_t r = i;; ++r) {
    const int64_t qr = q0 + r * es;
    if (is_zero(Bp)) {
      mn_fail(p, s);
      return;
    }
    const T m = ldro(p.a + qr) / Bp;
    const T B = fma(-m, Cp, p.B[qr]);
    const T C = fma(-m, Dp, p.C[qr]);
    const T F = fma(-m, Fp, p.F[qr]);
    const T D = p.D[qr];
    p.B[qr] = B;
    p.C[qr] = C;
    p.F[qr] = F;
    Bp = B; Cp = C; Dp = D; Fp = F;
    if (r + 1 >= n || is_zero(ldro(p.a + qr + es))) break;
  }
}

// Elements one strided array of a uniform batch spans.
int64_t mn_span(const band_desc* d) {
  return (d->n - 1) * d->elem_stride + (d->nsys - 1) * d->sys_stride + 1;
}

band_desc mn_td(const band_desc* d) {
  band_desc t = *d;
  t.half_bw = 1;
  t.schedule = BAND_SCHED_AUTO;
  t.chunks = 0;
  return t;
}

struct MnRowWs {
  void *B, *C, *D, *F;
  int32_t* skip;
  void* solve;
  size_t solve_bytes;
};
MnRowWs carve_mn_rows(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  MnRowWs w;
  const size_t arr = (size_t)mn_span(d) * dtype_size(d->dtype);
  w.B = c.take(arr);
  w.C = c.take(arr);
  w.D = c.take(arr);
  w.F = c.take(arr);
  w.skip = (int32_t*)c.take((size_t)d->nsys * sizeof(int32_t));
  const band_desc td = mn_td(d);
  w.solve_bytes = single_solve_bytes(&td, BAND_NTDM);
  w.solve = c.take(w.solve_bytes);
  *bytes = c.size();
  return w;
}

bool mn_rows_path(const band_desc* d) {
  return d->schedule == BAND_SCHED_AUTO && !d->offsets && d->nsys > 0 && d->n > 0;
}

template <typename T>
band_status mn_rows_solve(const band_desc* desc, const void* const diag[5], const void* f,
                          void* x, int32_t* sys_status, const MnRowWs& w, cudaStream_t st) {
  MnRows<T> p{layout_of(desc), (const T*)diag[0], (const T*)diag[1], (const T*)diag[2],
              (const T*)diag[3], (const T*)diag[4], (const T*)f, (T*)w.B, (T*)w.C, (T*)w.D,
              (T*)w.F, w.skip, sys_status};
  if (cudaMemsetAsync(w.skip, 0, (size_t)desc->nsys * sizeof(int32_t), st) != cudaSuccess)
    return BAND_ERR_CUDA;
  const int64_t total = desc->nsys * desc->n;
  const unsigned grid = (unsigned)((total + 255) / 256);
  k_mnpdm_e<T><<<grid, 256, 0, st>>>(p);
  k_mnpdm_a<T><<<grid, 256, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  const band_desc td = mn_td(desc);
  const void* dtd[5] = {nullptr, w.B, w.C, w.D, nullptr};
  return run_single(&td, BAND_NTDM, dtd, w.F, x, sys_status, w.solve, w.solve_bytes, st, w.skip);
}

struct MnpdmWs {
  void *B, *C, *D, *F, *al;
};
MnpdmWs carve_mnpdm(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  const size_t rows = (size_t)spill_rows(d) * dtype_size(d->dtype);
  MnpdmWs w;
  w.B = c.take(rows);
  w.C = c.take(rows);
  w.D = c.take(rows);
  w.F = c.take(rows);
  w.al = c.take(rows);
  *bytes = c.size();
  return w;
}

}  // namespace

size_t mnpdm_workspace_bytes(const band_desc* d) {
  size_t b = 0;
  if (mn_rows_path(d)) carve_mn_rows(d, nullptr, &b);
  else carve_mnpdm(d, nullptr, &b);
  return b;
}

// band_solve with method BAND_MNPDM: PD batches (half_bw 2, no per-system bandwidths);
// uniform batches on the automatic schedule row-parallel, the rest one thread per
// system.
band_status mnpdm_solve(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                        int32_t* sys_status, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (desc->hbw || desc->half_bw != 2 || desc->systems) return BAND_ERR_ARG;
  if (desc->schedule != BAND_SCHED_AUTO && desc->schedule != BAND_SCHED_THREAD) return BAND_ERR_ARG;
  if (!diag || !f || !x || !diag[0] || !diag[1] || !diag[2] || !diag[3] || !diag[4])
    return BAND_ERR_ARG;
  size_t need = 0;
  if (mn_rows_path(desc)) {
    carve_mn_rows(desc, nullptr, &need);
    if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
    const MnRowWs rw = carve_mn_rows(desc, ws, &need);
    return desc->dtype == BAND_F64
               ? mn_rows_solve<double>(desc, diag, f, x, sys_status, rw, st)
               : mn_rows_solve<float>(desc, diag, f, x, sys_status, rw, st);
  }
  carve_mnpdm(desc, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const MnpdmWs w = carve_mnpdm(desc, ws, &need);
  const Layout L = layout_of(desc);
  const Spill W = spill_of(desc);
  if (desc->dtype == BAND_F64) {
    const int tb = 32 * SweepWarps<double>::value;
    const unsigned grid = (unsigned)((desc->nsys + tb - 1) / tb);
    const size_t smem = (size_t)SweepWarps<double>::value * stage_bytes_per_warp<double>();
    MnpdmArgs<double> p{L, W, (const double*)diag[0], (const double*)diag[1],
                        (const double*)diag[2], (const double*)diag[3], (const double*)diag[4],
                        (const double*)f, (double*)x, (double*)w.B, (double*)w.C, (double*)w.D,
                        (double*)w.F, (double*)w.al, sys_status};
    k_mnpdm<double><<<grid, tb, smem, st>>>(p);
  } else {
    const int tb = 32 * SweepWarps<float>::value;
    const unsigned grid = (unsigned)((desc->nsys + tb - 1) / tb);
    const size_t smem = (size_t)SweepWarps<float>::value * stage_bytes_per_warp<float>();
    MnpdmArgs<float> p{L, W, (const float*)diag[0], (const float*)diag[1], (const float*)diag[2],
                       (const float*)diag[3], (const float*)diag[4], (const float*)f, (float*)x,
                       (float*)w.B, (float*)w.C, (float*)w.D, (float*)w.F, (float*)w.al,
                       sys_status};
    k_mnpdm<float><<<grid, tb, smem, st>>>(p);
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace band
