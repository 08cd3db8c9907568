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
// they stand.  One thread per system, three sweeps:
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
  carve_mnpdm(d, nullptr, &b);
  return b;
}

// band_solve with method BAND_MNPDM: PD batches (half_bw 2, no per-system bandwidths),
// any layout, one thread per system whatever desc->schedule (thread or auto) says.
band_status mnpdm_solve(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                        int32_t* sys_status, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (desc->hbw || desc->half_bw != 2 || desc->systems) return BAND_ERR_ARG;
  if (desc->schedule != BAND_SCHED_AUTO && desc->schedule != BAND_SCHED_THREAD) return BAND_ERR_ARG;
  if (!diag || !f || !x || !diag[0] || !diag[1] || !diag[2] || !diag[3] || !diag[4])
    return BAND_ERR_ARG;
  size_t need = 0;
  carve_mnpdm(desc, nullptr, &need);
  if (!ws || ws_bytes < need) return BAND_ERR_WORKSPACE;
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
