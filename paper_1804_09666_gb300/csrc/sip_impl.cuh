// sip_impl.cuh -- device code of SIP / the Stone method (Veneva & Ayriyan,
// arXiv:1804.09666, Sec. 2, Algorithm 1): ILU(0), Algorithm 1 with exact substitutions,
// and the Hotelling-Bodewig correction form (Remark of Sec. 2).  One thread per system,
// FP64.  Shared by the band_sip kernels and the batched kernel.
//
// ILU(0) on the pentadiagonal pattern, row-wise: for k = i-2, i-1 in the pattern,
// l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for j > k in the pattern of row i.  For
// this pattern nothing is dropped, so L (unit; l2 = L[i][i-2], l1 = L[i][i-1]) and
// U (u0 = U[i][i], u1 = U[i][i+1], u2 = U[i][i+2] = e_i) are the exact LU factors.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace band {

constexpr int kMaxWidth = 8;

// Workspace rows of band_sip: ILU(0) factors, substitution scratch, the second iterate
// buffer, the HB inverses and their ping-pong partners, and a status scratch.
struct SipWs {
  double *l2, *l1, *u0, *ru0, *u1, *y, *xb;
  double* X[2 * kMaxWidth];  // XL then XU
  double* T[2 * kMaxWidth];  // ping-pong partners
  int32_t* st;               // status scratch when the caller passes none
  unsigned long long* tail_count;   // systems needing more than one update
  int64_t* tail_list;
  double* tail_rn;
  int32_t* pend;                    // deferred residual: pending systems and their max|r|
  unsigned long long* rn_sys;
};
SipWs carve_sip(const band_desc* d, int32_t width, void* base, size_t* bytes);

struct SipArgs {
  Layout L;
  Spill W;
  const double *a, *b, *c, *d, *e, *f;
  double* x;           // result (also one of the two iterate buffers)
  double* xb;          // second iterate buffer (workspace, spill layout)
  double* y;           // substitution scratch (workspace, spill layout)
  double *l2, *l1, *u0, *ru0, *u1;   // ILU(0) factor rows (workspace)
  int w;
  const double* XL[kMaxWidth];
  const double* XU[kMaxWidth];
  double tol;
  int max_it;
  int32_t *iters, *status;
  double* resid;
  // systems whose first update leaves max|r| >= tol go to a tail list, finished by a
  // block-cooperative kernel (null: finish them in the same thread)
  unsigned long long* tail_count;
  int64_t* tail_list;
  double* tail_rn;     // per tail-list entry: max|r| after the first update (-1: none yet)
  // the first update ran on the two-sided schedule (sip_two_sided): rows (n+1)/2 .. n-1
  // of ru0, u1 hold the mirrored factors and the tail rebuilds them first
  int32_t two_sided;
  // Deferred residual (when pend is set): the first update's sweeps leave x^1 and mark
  // the system pending; an elementwise pass forms max|f - A x^1| (rn_sys, bits of a
  // double >= 0) and a per-system pass takes Algorithm 1's decision.  Both indexed by
  // position in the batch.
  int32_t* pend;
  unsigned long long* rn_sys;
};

struct Row {
  double a, b, c, d, e, f;
};
__device__ __forceinline__ Row load_row(const SipArgs& p, int64_t q, int64_t i, int64_t n) {
  Row r;
  r.a = (i >= 2) ? ldro(p.a + q) : 0.0;
  r.b = (i >= 1) ? ldro(p.b + q) : 0.0;
  r.c = ldro(p.c + q);
  r.d = (i + 1 < n) ? ldro(p.d + q) : 0.0;
  r.e = (i + 2 < n) ? ldro(p.e + q) : 0.0;
  r.f = p.f[q];
  return r;
}

// HB variant: x <- x + U~^{-1} (L~^{-1} (f - A x)) in one sweep per iteration.  The
// sweep computes r = f - A x_old (and its norm), y = L~^{-1} r with a lag of 0 and
// x_new = x_old + U~^{-1} y with a lag of w-1 rows.  When max|r| < tol the update
// just computed is discarded: the answer is x_old with k updates (Algorithm 1's
// stop test on the residual of the current iterate).
__device__ inline void sip_hb(const SipArgs& p, int64_t s) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  const int w = p.w;
  // iterate buffers: element i of buffer 0 is x[q0 + i*es], of buffer 1 xb[w0 + i*ws]
  for (int64_t i = 0; i < n; ++i) p.x[q0 + i * es] = 0.0;
  int cur = 0;
  int k = 0;
  double rn = 0.0;
  int32_t st = BAND_ERR_NOT_CONVERGED;
  for (;;) {
    auto xold = [&](int64_t i) -> double {
      return cur == 0 ? p.x[q0 + i * es] : p.xb[w0 + i * ws];
    };
    auto xnew_store = [&](int64_t i, double v) {
      if (cur == 0) p.xb[w0 + i * ws] = v;
      else p.x[q0 + i * es] = v;
    };
    double rr[kMaxWidth], yr[kMaxWidth];
    for (int j = 0; j < kMaxWidth; ++j) { rr[j] = 0.0; yr[j] = 0.0; }
    double xm2 = 0, xm1 = 0, x0 = xold(0), xp1 = n > 1 ? xold(1) : 0.0;
    rn = 0.0;
    bool nan_seen = false;
    for (int64_t t = 0; t < n + w - 1; ++t) {
      if (t < n) {
        const int64_t q = q0 + t * es, wi = w0 + t * ws;
        const Row A = load_row(p, q, t, n);
        const double xp2 = (t + 2 < n) ? xold(t + 2) : 0.0;
        double ax = A.c * x0;
        ax = fma(A.a, xm2, ax);
        ax = fma(A.b, xm1, ax);
        ax = fma(A.d, xp1, ax);
        ax = fma(A.e, xp2, ax);
        const double r = A.f - ax;
        nan_seen |= (r != r);
        rn = fmax(rn, fabs(r));
        for (int j = w - 1; j > 0; --j) rr[j] = rr[j - 1];
        rr[0] = r;
        double yv = 0.0;
        for (int j = 0; j < w; ++j) yv = fma(p.XL[j][wi], rr[j], yv);
        for (int j = w - 1; j > 0; --j) yr[j] = yr[j - 1];
        yr[0] = yv;
        xm2 = xm1; xm1 = x0; x0 = xp1; xp1 = xp2;
      } else {
        for (int j = w - 1; j > 0; --j) yr[j] = yr[j - 1];
        yr[0] = 0.0;
      }
      const int64_t i = t - (w - 1);  // row whose U~^{-1} y is complete
      if (i >= 0) {
        const int64_t wi = w0 + i * ws;
        double acc = 0.0;
        for (int j = 0; j < w; ++j) acc = fma(p.XU[j][wi], yr[w - 1 - j], acc);
        xnew_store(i, xold(i) + acc);
      }
    }
    if (nan_seen || !isfinite(rn)) { rn = NAN; st = BAND_ERR_NONFINITE; break; }
    if (rn < p.tol) { st = BAND_OK; break; }
    if (k >= p.max_it) break;
    ++k;
    cur ^= 1;
  }
  if (cur == 1) {  // the answer sits in the workspace buffer
    for (int64_t i = 0; i < n; ++i) p.x[q0 + i * es] = p.xb[w0 + i * ws];
  }
  if (p.iters) p.iters[s] = k;
  if (p.resid) p.resid[s] = rn;
  set_status(p.status, s, st);
}


// ILU(0) of one system into the factor rows l2, l1, u0, 1/u0, u1.  Returns false on a
// zero pivot.
__device__ inline bool ilu0_into(const SipArgs& p, int64_t s) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  double ru0_1 = 0, u1_1 = 0, e_1 = 0, ru0_2 = 0, u1_2 = 0, e_2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t w = w0 + i * ws;
    const Row A = load_row(p, q0 + i * es, i, n);
    double l2 = A.a, l1 = A.b, u0 = A.c, u1 = A.d;
    if (i >= 2) {
      l2 = l2 * ru0_2;
      l1 = fma(-l2, u1_2, l1);
      u0 = fma(-l2, e_2, u0);
    }
    if (i >= 1) {
      l1 = l1 * ru0_1;
      u0 = fma(-l1, u1_1, u0);
      u1 = fma(-l1, e_1, u1);
    }
    if (u0 == 0.0) return false;
    const double r = rcp64(u0);
    p.l2[w] = l2;
    p.l1[w] = l1;
    p.u0[w] = u0;
    p.ru0[w] = r;
    p.u1[w] = u1;
    ru0_2 = ru0_1; u1_2 = u1_1; e_2 = e_1;
    ru0_1 = r; u1_1 = u1; e_1 = A.e;
  }
  return true;
}

// Algorithm 1 with exact substitutions.  x^0 = 0 makes K x^0 = 0, so the first update
// is x^1 = U^{-1} L^{-1} f: one forward sweep does ILU(0) and L y = f together (only
// 1/u0, u1 and y are kept), one backward sweep does U x = y.  The residual of x^1 and
// the stop / continue decision are separate passes (sip_resid_cell, sip_decide_one);
// systems that need more updates go to the block-cooperative tail.
__device__ inline void sip_literal(const SipArgs& p, int64_t t, void* stage) {
  const int64_t s = p.L.sys(t);     // t: position in the batch, s: the system id

  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(t), ws = p.W.stride();
  double ru0_1 = 0, u1_1 = 0, e_1 = 0, ru0_2 = 0, u1_2 = 0, e_2 = 0;
  double y1 = 0, y2 = 0, rn = 0.0;
  // row i of the forward sweep (ILU(0) with L y = f); false on a zero pivot
  auto row = [&](int64_t i, const Row& r) -> bool {
    const int64_t w = w0 + i * ws;
    double l2 = r.a, l1 = r.b, u0 = r.c, u1 = r.d;
    if (i >= 2) {
      l2 = l2 * ru0_2;
      l1 = fma(-l2, u1_2, l1);
      u0 = fma(-l2, e_2, u0);
    }
    if (i >= 1) {
      l1 = l1 * ru0_1;
      u0 = fma(-l1, u1_1, u0);
      u1 = fma(-l1, e_1, u1);
    }
    if (is_zero(u0)) return false;
    const double rr = rcp64(u0);
    const double yv = fma(-l2, y2, fma(-l1, y1, r.f));
    p.ru0[w] = rr;
    p.u1[w] = u1;
    p.y[w] = yv;
    rn = max_abs(rn, r.f);               // r^0 = f - A x^0 = f (a NaN f wins the max)
    y2 = y1; y1 = yv;
    ru0_2 = ru0_1; u1_2 = u1_1; e_2 = e_1;
    ru0_1 = rr; u1_1 = u1; e_1 = r.e;
    return true;
  };
  bool zero = false;
  if (stage && !p.L.offsets && p.L.ss == 1) {
    // interleaved systems: rows staged through the warp's shared-memory ring ahead of
    // the recurrence (as the direct sweeps do), so its chain does not wait on memory
    constexpr int D = StageDepth<double>::value;
    const RowRing<double, 6, D> ring{static_cast<double*>(stage), (int)(threadIdx.x & 31)};
    const double* src[6] = {p.a, p.b, p.c, p.d, p.e, p.f};
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      if (j < n) ring.issue(j, src, q0 + j * es);
      else ring.skip();
    }
    for (int64_t i = 0; i < n; ++i) {
      const int64_t ip = i + D - 1;
      if (ip < n) ring.issue((int)(ip & (D - 1)), src, q0 + ip * es);
      else ring.skip();
      cp_async_wait<D - 1>();
      const int slot = (int)(i & (D - 1));
      Row r;
      r.a = (i >= 2) ? ring.get(slot, 0) : 0.0;
      r.b = (i >= 1) ? ring.get(slot, 1) : 0.0;
      r.c = ring.get(slot, 2);
      r.d = (i + 1 < n) ? ring.get(slot, 3) : 0.0;
      r.e = (i + 2 < n) ? ring.get(slot, 4) : 0.0;
      r.f = ring.get(slot, 5);
      if (!row(i, r)) {
        zero = true;
        break;
      }
    }
    cp_async_wait<0>();
  } else {
    Row r0 = load_row(p, q0, 0, n), r1, r2;
    if (n > 1) r1 = load_row(p, q0 + es, 1, n);
    for (int64_t i = 0; i < n; ++i) {
      if (i + 2 < n) r2 = load_row(p, q0 + (i + 2) * es, i + 2, n);
      if (!row(i, r0)) {
        zero = true;
        break;
      }
      r0 = r1;
      r1 = r2;
    }
  }
  if (zero) {
    if (p.iters) p.iters[s] = 0;
    if (p.resid) p.resid[s] = NAN;
    set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
    return;
  }
  if (rn < p.tol || p.max_it < 1 || !isfinite(rn)) {   // no update: x = x^0 = 0
    for (int64_t i = 0; i < n; ++i) p.x[q0 + i * es] = 0.0;
    if (p.iters) p.iters[s] = 0;
    if (p.resid) p.resid[s] = rn;
    set_status(p.status, s,
               !isfinite(rn) ? BAND_ERR_NONFINITE
                             : (rn < p.tol ? BAND_OK : BAND_ERR_NOT_CONVERGED));
    return;
  }
  // U x = y; the residual pass and Algorithm 1's decision come after (pend)
  constexpr int kB = 8;
  double x1 = 0, x2 = 0;
  for (int64_t top = n - 1; top >= 0; top -= kB) {
    double yv[kB], uv[kB], rv[kB], ev[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int64_t i = top - j;
      yv[j] = uv[j] = rv[j] = ev[j] = 0.0;
      if (i >= 0) {
        const int64_t w = w0 + i * ws;
        ev[j] = (i + 2 < n) ? ldro(p.e + q0 + i * es) : 0.0;
        yv[j] = p.y[w];
        uv[j] = p.u1[w];
        rv[j] = p.ru0[w];
      }
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const int64_t i = top - j;
      if (i < 0) break;
      const double xi = fma(-ev[j], x2, fma(-uv[j], x1, yv[j])) * rv[j];
      p.x[q0 + i * es] = xi;
      x2 = x1;
      x1 = xi;
    }
  }
  p.pend[t] = 1;
}

// ---------------------------------------------------------------------------
// Algorithm 1's first update on the two-sided schedule (lanes l and l ^ 16 of a warp
// share system s).  x^1 = (LU)^{-1} f with the exact ILU(0) = LU factors: the top lane
// runs sip_literal's forward sweep (ILU(0) row by row with L y = f) on rows 0 .. m-1,
// the bottom lane the same sweep on the reversed system (rows n-1 .. m, diagonals
// (a, b, c, d, e) read as (e, d, c, b, a)), i.e. the UL factorisation of that block.
// Their last two rows, normalised (x_i + alpha x_{i+-1} + beta x_{i+-2} = z), form the
// same 4x4 interface system as the two-sided direct sweep; then each lane
// back-substitutes its half.  x^1 equals sip_literal's in exact arithmetic; the
// residual and the decision are the same separate passes.  A zero pivot in either
// half, a singular interface system or n < 4 hands the system to the tail kernel from
// x^0 = 0 (tail_rn = -1), which factors it top-down and runs Algorithm 1 from its
// first update.
__device__ inline void sip_two_sided(const SipArgs& p, int64_t t, bool active) {
  const int64_t s = active ? p.L.sys(t) : 0;   // t: position in the batch, s: system id

  const int lane = (int)(threadIdx.x & 31);
  const bool bottom = lane >= 16;
  const unsigned full = 0xffffffffu;
  const int64_t n = active ? p.L.rows(s) : 0;
  const bool split = n >= 4;
  const int64_t m = (n + 1) / 2;
  const int64_t q0 = active ? p.L.base(s) : 0, es = active ? p.L.stride() : 0;
  const int64_t w0 = active ? p.W.base(t) : 0, ws = active ? p.W.stride() : 0;
  const int64_t rows = (!active || !split) ? 0 : (bottom ? n - m : m);
  const int dir = bottom ? -1 : 1;
  const int64_t first = bottom ? n - 1 : 0;
  // ---- forward: ILU(0) of this lane's block with L y = f (register prefetch)
  double ru0_1 = 0, u1_1 = 0, e_1 = 0, ru0_2 = 0, u1_2 = 0, e_2 = 0;
  double y1 = 0, y2 = 0, rn0 = 0.0;
  bool zero = false;
  {
    auto load = [&](int64_t j) -> Row {            // j-th row of this lane's sweep
      const int64_t i = first + dir * j;
      Row r = load_row(p, q0 + i * es, i, n);
      if (bottom) {                                // reversed system
        const double ta = r.a, tb = r.b;
        r.a = r.e; r.b = r.d; r.d = tb; r.e = ta;
      }
      return r;
    };
    Row r0{}, r1{}, r2{};
    if (rows > 0) r0 = load(0);
    if (rows > 1) r1 = load(1);
    for (int64_t j = 0; j < rows; ++j) {
      if (j + 2 < rows) r2 = load(j + 2);
      const int64_t w = w0 + (first + dir * j) * ws;
      double l2 = r0.a, l1 = r0.b, u0 = r0.c, u1 = r0.d;
      if (j >= 2) {
        l2 = l2 * ru0_2;
        l1 = fma(-l2, u1_2, l1);
        u0 = fma(-l2, e_2, u0);
      }
      if (j >= 1) {
        l1 = l1 * ru0_1;
        u0 = fma(-l1, u1_1, u0);
        u1 = fma(-l1, e_1, u1);
      }
      if (is_zero(u0)) { zero = true; break; }
      const double r = rcp64(u0);
      const double yv = fma(-l2, y2, fma(-l1, y1, r0.f));
      p.ru0[w] = r;
      p.u1[w] = u1;
      p.y[w] = yv;
      rn0 = max_abs(rn0, r0.f);          // r^0 = f - A x^0 = f
      y2 = y1; y1 = yv;
      ru0_2 = ru0_1; u1_2 = u1_1; e_2 = e_1;
      ru0_1 = r; u1_1 = u1; e_1 = r0.e;
      r0 = r1;
      r1 = r2;
    }
  }
  // ---- exchange (every lane reaches every shuffle)
  const double o_rn0 = __shfl_xor_sync(full, rn0, 16);
  const bool o_zero = __shfl_xor_sync(full, (int)zero, 16) != 0;
  // normalised last two rows: row "1" is the last one eliminated, row "2" the one before
  const double al1 = u1_1 * ru0_1, be1 = e_1 * ru0_1, z1 = y1 * ru0_1;
  const double al2 = u1_2 * ru0_2, be2 = e_2 * ru0_2, z2 = y2 * ru0_2;
  const double o_al1 = __shfl_xor_sync(full, al1, 16), o_al2 = __shfl_xor_sync(full, al2, 16);
  const double o_be1 = __shfl_xor_sync(full, be1, 16), o_be2 = __shfl_xor_sync(full, be2, 16);
  const double o_z1 = __shfl_xor_sync(full, z1, 16), o_z2 = __shfl_xor_sync(full, z2, 16);
  __syncwarp();
  rn0 = max_abs(rn0, o_rn0);
  bool fail = split && (zero || o_zero);
  const bool stop0 = split && !fail && (rn0 < p.tol || p.max_it < 1 || !isfinite(rn0));
  double xm2 = 0, xm1 = 0, xm0 = 0, xp1 = 0;      // x_{m-2} .. x_{m+1}
  if (active && split && !fail && !stop0) {
    const double tal2 = bottom ? o_al2 : al2, tbe2 = bottom ? o_be2 : be2, tz2 = bottom ? o_z2 : z2;
    const double tal1 = bottom ? o_al1 : al1, tbe1 = bottom ? o_be1 : be1, tz1 = bottom ? o_z1 : z1;
    const double bal2 = bottom ? al2 : o_al2, bbe2 = bottom ? be2 : o_be2, bz2 = bottom ? z2 : o_z2;
    const double bal1 = bottom ? al1 : o_al1, bbe1 = bottom ? be1 : o_be1, bz1 = bottom ? z1 : o_z1;
    double M[4][5];
    M[0][0] = 1;    M[0][1] = tal2; M[0][2] = tbe2; M[0][3] = 0;    M[0][4] = tz2;
    M[1][0] = 0;    M[1][1] = 1;    M[1][2] = tal1; M[1][3] = tbe1; M[1][4] = tz1;
    M[2][0] = bbe1; M[2][1] = bal1; M[2][2] = 1;    M[2][3] = 0;    M[2][4] = bz1;
    M[3][0] = 0;    M[3][1] = bbe2; M[3][2] = bal2; M[3][3] = 1;    M[3][4] = bz2;
    if (solve_small<double, 4>(M)) {
      xm2 = M[0][4]; xm1 = M[1][4]; xm0 = M[2][4]; xp1 = M[3][4];
    } else {
      fail = true;         // both lanes hold the same M, so both see this
    }
  }
  // ---- back-substitution of this lane's half with the residual of its own rows.
  // Walk top: i = m-3 down to -2, bottom: i = m+2 up to n+1 (x_i = 0 outside the matrix),
  // with x_{m-2} .. x_{m+1} known; the residual of row jr = i + 2 (top) or i - 2
  // (bottom) is taken once x_{jr-2} .. x_{jr+2} are known.  n1 .. n4 hold the previous
  // four x's in walk order.
  if (active && split && !fail && !stop0) {
    // back-substitution only: the residual pass and the decision come after
    const int64_t start = bottom ? m + 2 : m - 3;
    const int64_t cnt = bottom ? n - m - 2 : m - 2;
    const int bdir = bottom ? 1 : -1;
    const double* pe = bottom ? p.a : p.e;
    double x1 = bottom ? xp1 : xm2, x2 = bottom ? xm0 : xm1;
    constexpr int kB = 8;
    for (int64_t k0 = 0; k0 < cnt; k0 += kB) {
      double yv[kB], uv[kB], rv[kB], ev[kB];
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        yv[j] = uv[j] = rv[j] = ev[j] = 0.0;
        if (k0 + j < cnt) {
          const int64_t i = start + bdir * (k0 + j);
          const int64_t w = w0 + i * ws;
          const bool has_e = bottom ? (i >= 2) : (i + 2 < n);
          ev[j] = has_e ? ldro(pe + q0 + i * es) : 0.0;
          yv[j] = p.y[w];
          uv[j] = p.u1[w];
          rv[j] = p.ru0[w];
        }
      }
#pragma unroll
      for (int j = 0; j < kB; ++j) {
        if (k0 + j >= cnt) break;
        const int64_t i = start + bdir * (k0 + j);
        const double xi = fma(-ev[j], x2, fma(-uv[j], x1, yv[j])) * rv[j];
        p.x[q0 + i * es] = xi;
        x2 = x1;
        x1 = xi;
      }
    }
    if (!bottom) {
      p.x[q0 + (m - 2) * es] = xm2;
      p.x[q0 + (m - 1) * es] = xm1;
    } else {
      p.x[q0 + m * es] = xm0;
      p.x[q0 + (m + 1) * es] = xp1;
    }
  }
  if (!active || bottom) return;
  if (!split || fail) {          // the tail kernel starts this system from x^0 = 0
    const unsigned long long k = atomicAdd(p.tail_count, 1ull);
    p.tail_list[k] = t;
    p.tail_rn[k] = -1.0;
    return;
  }
  if (stop0) {                   // no update: x = x^0 = 0
    for (int64_t i = 0; i < n; ++i) p.x[q0 + i * es] = 0.0;
    if (p.iters) p.iters[s] = 0;
    if (p.resid) p.resid[s] = rn0;
    set_status(p.status, s,
               !isfinite(rn0) ? BAND_ERR_NONFINITE : (rn0 < p.tol ? BAND_OK : BAND_ERR_NOT_CONVERGED));
    return;
  }
  p.pend[t] = 1;                 // the residual pass and the decision come after
}

// ---------------------------------------------------------------------------
// Deferred residual of the first update: r = f - A x^1 over a cell of rows of the t-th
// system (the expression and order of sip_literal's inline residual), its max|r| into
// rn_sys[t]; then Algorithm 1's decision per system.
// Cells: where consecutive systems sit at consecutive addresses (interleaved), a cell
// is kResChunk rows and consecutive threads take consecutive systems; where each
// system's rows are consecutive (contiguous, ragged), a cell is kResRows rows and
// consecutive threads take consecutive cells of one system, so a warp reads
// 32 x kResRows consecutive rows of every array.
// ---------------------------------------------------------------------------
constexpr int kResChunk = 32;
constexpr int kResRows = 4;

__host__ __device__ inline bool resid_rows_fastest(const Layout& L) {
  return L.offsets != nullptr || (L.es == 1 && L.ss != 1);
}
__host__ __device__ inline int64_t resid_cells(const Layout& L) {
  const int64_t rows = resid_rows_fastest(L) ? kResRows : kResChunk;
  return L.nsys * ((L.n + rows - 1) / rows);
}

// max|f - A x| over rows i0 .. i1-1 of the t-th system (bits of a double >= 0)
__device__ inline double sip_resid_rows(const SipArgs& p, int64_t t, int64_t i0, int64_t i1) {
  const int64_t s = p.L.sys(t);
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  if (i1 > n) i1 = n;
  if (i0 >= i1) return 0.0;
  auto X = [&](int64_t j) -> double { return (j >= 0 && j < n) ? p.x[q0 + j * es] : 0.0; };
  double xm2 = X(i0 - 2), xm1 = X(i0 - 1), x0 = X(i0), xp1 = X(i0 + 1);
  double rn = 0.0;
  constexpr int kB = 1;
  for (int64_t ib = i0; ib < i1; ib += kB) {
    Row A[kB];
    double xv[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int64_t i = ib + u;
      A[u] = Row{0, 0, 0, 0, 0, 0};
      xv[u] = 0.0;
      if (i < i1) {
        A[u] = load_row(p, q0 + i * es, i, n);
        xv[u] = X(i + 2);
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      if (ib + u >= i1) break;
      const double xp2 = xv[u];
      double ax = A[u].c * x0;
      ax = fma(A[u].a, xm2, ax);
      ax = fma(A[u].b, xm1, ax);
      ax = fma(A[u].d, xp1, ax);
      ax = fma(A[u].e, xp2, ax);
      rn = max_abs(rn, A[u].f - ax);      // a NaN wins the max
      xm2 = xm1; xm1 = x0; x0 = xp1; xp1 = xp2;
    }
  }
  return rn;
}

// Cell idx of the residual pass (idx may lie past the last cell).  Every thread of the
// warp calls it: in the rows-fastest mapping a warp whose cells all belong to one
// system combines its maxima by shuffles before the one atomic.
__device__ inline void sip_resid_cell(const SipArgs& p, int64_t idx) {
  const bool rows_fastest = resid_rows_fastest(p.L);
  const int64_t rows = rows_fastest ? kResRows : kResChunk;
  const int64_t nch = (p.L.n + rows - 1) / rows;
  const bool valid = idx < p.L.nsys * nch;
  const int64_t t = !valid ? -1 : (rows_fastest ? idx / nch : idx % p.L.nsys);
  const int64_t c = !valid ? 0 : (rows_fastest ? idx % nch : idx / p.L.nsys);
  unsigned long long v = 0ull;
  if (valid && p.pend[t])
    v = (unsigned long long)__double_as_longlong(sip_resid_rows(p, t, c * rows, c * rows + rows));
  if (rows_fastest) {
    const unsigned full = 0xffffffffu;
    const int64_t t0 = __shfl_sync(full, t, 0);
    if (__all_sync(full, t < 0 || t == t0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(full, v, o);
        v = v > w ? v : w;
      }
      if ((threadIdx.x & 31) == 0 && v) atomicMax(p.rn_sys + t0, v);
      return;
    }
  }
  if (v) atomicMax(p.rn_sys + t, v);
}

__device__ inline void sip_decide_one(const SipArgs& p, int64_t t) {
  if (!p.pend[t]) return;
  p.pend[t] = 0;
  const int64_t s = p.L.sys(t);
  const double rn = __longlong_as_double((long long)p.rn_sys[t]);
  p.rn_sys[t] = 0ull;
  if (rn < p.tol || p.max_it <= 1 || !isfinite(rn)) {
    if (p.iters) p.iters[s] = 1;
    if (p.resid) p.resid[s] = rn;
    set_status(p.status, s,
               !isfinite(rn) ? BAND_ERR_NONFINITE
                             : (rn < p.tol ? BAND_OK : BAND_ERR_NOT_CONVERGED));
    return;
  }
  const unsigned long long k = atomicAdd(p.tail_count, 1ull);   // more updates: the tail
  p.tail_list[k] = t;
  p.tail_rn[k] = rn;
}

// ---------------------------------------------------------------------------
// Tail: further Algorithm 1 updates of one system by a whole thread block.  With the
// ILU(0) factors known every step is either a stencil over rows (K x + f, f - A x) or
// a second-order linear recurrence (L y = rhs, U x = y), so thread t takes a chunk of
// consecutive rows and the recurrences run as a scan of affine maps over the chunks:
// each chunk computes, from a zero state, its particular solution and the responses to
// the two unit states; a block-wide scan composes these maps in sweep order; each
// chunk then reruns from its true starting state.  The arithmetic is the same as the
// sequential substitutions up to the order of rounding.
// ---------------------------------------------------------------------------
constexpr int kTailThreads = 256;

// Affine map of the 2-state (v_{t-1}, v_{t-2}) -> (v_t, v_{t-1}) over a chunk:
// out = M in + c, M = [[m00, m01], [m10, m11]].
struct Aff {
  double m00, m01, m10, m11, c0, c1;
};
__device__ __forceinline__ Aff aff_after(const Aff& b, const Aff& a) {   // b o a
  Aff r;
  r.m00 = fma(b.m00, a.m00, b.m01 * a.m10);
  r.m01 = fma(b.m00, a.m01, b.m01 * a.m11);
  r.m10 = fma(b.m10, a.m00, b.m11 * a.m10);
  r.m11 = fma(b.m10, a.m01, b.m11 * a.m11);
  r.c0 = fma(b.m00, a.c0, fma(b.m01, a.c1, b.c0));
  r.c1 = fma(b.m10, a.c0, fma(b.m11, a.c1, b.c1));
  return r;
}

// v_i = r_i - c1_i v_{i-dir} - c2_i v_{i-2 dir} over rows 0..n-1 (dir = +1 forward,
// -1 backward), chunks [t m, (t+1) m) per thread; coef(i, r, c1, c2); out(i, v).
template <class Coef, class Out>
__device__ inline void block_recurrence2(int64_t n, int dir, Coef coef, Out out, Aff* sh) {
  const int t = threadIdx.x, P = blockDim.x;
  const int64_t m = (n + P - 1) / P;
  const int64_t lo = min(n, (int64_t)t * m), hi = min(n, lo + m);
  const int pos = dir > 0 ? t : P - 1 - t;     // chunk position in sweep order
  // pass 1: particular (p) and unit responses (h: state (1,0), g: state (0,1))
  double p1 = 0, p2 = 0, h1 = 1, h2 = 0, g1 = 0, g2 = 1;
  for (int64_t k = 0; k < hi - lo; ++k) {
    const int64_t i = dir > 0 ? lo + k : hi - 1 - k;
    double r, c1, c2;
    coef(i, r, c1, c2);
    const double np = fma(-c2, p2, fma(-c1, p1, r));
    const double nh = fma(-c2, h2, -c1 * h1);
    const double ng = fma(-c2, g2, -c1 * g1);
    p2 = p1; p1 = np; h2 = h1; h1 = nh; g2 = g1; g1 = ng;
  }
  Aff mine{h1, g1, h2, g2, p1, p2};
  __syncthreads();
  sh[pos] = mine;
  __syncthreads();
  for (int off = 1; off < P; off <<= 1) {      // inclusive scan: S_pos = map_pos o S_{pos-1}
    Aff prev{};
    const bool take = pos >= off;
    if (take) prev = sh[pos - off];
    __syncthreads();
    if (take) {
      mine = aff_after(mine, prev);
      sh[pos] = mine;
    }
    __syncthreads();
  }
  double s1 = 0, s2 = 0;                       // state entering this chunk
  if (pos > 0) { s1 = sh[pos - 1].c0; s2 = sh[pos - 1].c1; }
  __syncthreads();
  for (int64_t k = 0; k < hi - lo; ++k) {
    const int64_t i = dir > 0 ? lo + k : hi - 1 - k;
    double r, c1, c2;
    coef(i, r, c1, c2);
    const double v = fma(-c2, s2, fma(-c1, s1, r));
    out(i, v);
    s2 = s1; s1 = v;
  }
}

__device__ inline double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// One system as the tail sees it: each array with its own stride (the system's rows in
// global memory, or a copy of the whole system in shared memory with stride 1).
struct TailSys {
  const double *a, *b, *c, *d, *e, *f;
  int64_t sa;                  // stride of a..f
  double* x;
  int64_t sx;
  double *ru0, *u1;
  double* y;
  int64_t sw;                  // stride of ru0, u1, y
  int64_t n;
  __device__ __forceinline__ Row row(int64_t i) const {
    Row r;
    const int64_t q = i * sa;
    r.a = (i >= 2) ? a[q] : 0.0;
    r.b = (i >= 1) ? b[q] : 0.0;
    r.c = c[q];
    r.d = (i + 1 < n) ? d[q] : 0.0;
    r.e = (i + 2 < n) ? e[q] : 0.0;
    r.f = f[q];
    return r;
  }
};

// ILU(0) entries l2_i, l1_i, u0_i of row i recomputed from A and the stored 1/u0, u1 of
// rows i-1, i-2: the same operations in the same order as the first sweep, so the
// values are bitwise those of the sequential factorisation.
struct IluRow {
  double l2, l1, u0;
};
__device__ __forceinline__ IluRow ilu_row(const TailSys& S, int64_t i) {
  const Row A = S.row(i);
  double l2 = A.a, l1 = A.b, u0 = A.c;
  if (i >= 2) {
    const int64_t w2 = (i - 2) * S.sw;
    const double e2 = S.e[(i - 2) * S.sa];   // i - 2 + 2 < n holds
    l2 = l2 * S.ru0[w2];
    l1 = fma(-l2, S.u1[w2], l1);
    u0 = fma(-l2, e2, u0);
  }
  if (i >= 1) {
    const int64_t w1 = (i - 1) * S.sw;
    l1 = l1 * S.ru0[w1];
    u0 = fma(-l1, S.u1[w1], u0);
  }
  return IluRow{l2, l1, u0};
}

// Rows from .. n-1 of the top-down ILU(0) factors (1/u0, u1), continuing from the stored
// rows from-2, from-1: the operations of sip_literal's forward sweep in its order, so the
// values are bitwise the sequential ones.  One thread.  Returns false on a zero pivot.
__device__ inline bool ilu_rebuild(const TailSys& S, int64_t from) {
  const int64_t n = S.n;
  double ru0_2 = 0, u1_2 = 0, e_2 = 0, ru0_1 = 0, u1_1 = 0, e_1 = 0;
  if (from >= 2) {
    ru0_2 = S.ru0[(from - 2) * S.sw];
    u1_2 = S.u1[(from - 2) * S.sw];
    e_2 = S.row(from - 2).e;
  }
  if (from >= 1) {
    ru0_1 = S.ru0[(from - 1) * S.sw];
    u1_1 = S.u1[(from - 1) * S.sw];
    e_1 = S.row(from - 1).e;
  }
  for (int64_t i = from; i < n; ++i) {
    const Row A = S.row(i);
    double l2 = A.a, l1 = A.b, u0 = A.c, u1 = A.d;
    if (i >= 2) {
      l2 = l2 * ru0_2;
      l1 = fma(-l2, u1_2, l1);
      u0 = fma(-l2, e_2, u0);
    }
    if (i >= 1) {
      l1 = l1 * ru0_1;
      u0 = fma(-l1, u1_1, u0);
      u1 = fma(-l1, e_1, u1);
    }
    if (is_zero(u0)) return false;
    const double r = rcp64(u0);
    S.ru0[i * S.sw] = r;
    S.u1[i * S.sw] = u1;
    ru0_2 = ru0_1; u1_2 = u1_1; e_2 = e_1;
    ru0_1 = r; u1_1 = u1; e_1 = A.e;
  }
  return true;
}

// One system by the whole block, continuing Algorithm 1 from k = 1 and max|r| = rn.
// Returns (to every thread) k and the final max|r|; thread 0 writes iters, resid and
// the status.
__device__ inline void sip_tail_run(const SipArgs& p, int64_t s, const TailSys& S, double rn,
                                    Aff* sh, double* red) {
  const int64_t n = S.n;
  const int P = blockDim.x;
  const int64_t m = (n + P - 1) / P;
  const int64_t lo = min(n, (int64_t)threadIdx.x * m), hi = min(n, lo + m);
  auto X = [&](int64_t i) -> double { return (i >= 0 && i < n) ? S.x[i * S.sx] : 0.0; };
  auto U1 = [&](int64_t i) -> double { return (i >= 0 && i < n) ? S.u1[i * S.sw] : 0.0; };
  auto U0 = [&](int64_t i) -> double { return (i >= 0 && i < n) ? ilu_row(S, i).u0 : 0.0; };
  int k = 1;
  const bool scratch = rn < 0.0;      // start from x^0 = 0 (no factors stored yet)
  if (scratch || (p.two_sided && n >= 4)) {
    // the top-down factors of every row (from scratch) or of the lower half, which the
    // two-sided first update left mirrored (one thread, sip_literal's operations)
    __shared__ int ok;
    if (threadIdx.x == 0) ok = ilu_rebuild(S, scratch ? 0 : (n + 1) / 2) ? 1 : 0;
    __syncthreads();
    const bool good = ok != 0;
    __syncthreads();
    if (!good) {      // the top-down order meets a zero pivot: as sip_literal reports it
      if (threadIdx.x == 0) {
        if (p.iters) p.iters[s] = 0;
        if (p.resid) p.resid[s] = NAN;
        set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
      }
      __syncthreads();
      return;
    }
  }
  if (scratch) {      // x^0 = 0, r^0 = f
    double loc = 0.0;
    bool nan_seen = false;
    for (int64_t i = lo; i < hi; ++i) {
      S.x[i * S.sx] = 0.0;
      const double fi = S.f[i * S.sa];
      nan_seen |= (fi != fi);
      loc = fmax(loc, fabs(fi));
    }
    rn = block_max(nan_seen ? INFINITY : loc, red);
    k = 0;
  }
  double prev = INFINITY;
  bool nonfinite = !isfinite(rn);
  for (;;) {
    if (rn < p.tol || k >= p.max_it || nonfinite) break;
    if (k >= 2 && !(rn < prev)) break;
    prev = rn;
    // rhs = K x + f with K = LU - A on the own rows (K[i][i+2] = 0)
    for (int64_t i = lo; i < hi; ++i) {
      const Row A = S.row(i);
      const IluRow R = ilu_row(S, i);
      const double l2 = R.l2, l1 = R.l1, u0 = R.u0;
      const double u1 = (i + 1 < n) ? U1(i) : 0.0;
      const double u0m2 = U0(i - 2), u1m2 = U1(i - 2), u0m1 = U0(i - 1);
      const double u1m1 = U1(i - 1);
      const double em2 = (i >= 2 && i < n) ? S.e[(i - 2) * S.sa] : 0.0;
      const double em1 = (i >= 1 && i + 1 < n) ? S.e[(i - 1) * S.sa] : 0.0;
      const double ka = l2 * u0m2 - A.a;
      const double kb = fma(l2, u1m2, l1 * u0m1) - A.b;
      const double kc = fma(l2, em2, fma(l1, u1m1, u0)) - A.c;
      const double kd = fma(l1, em1, u1) - A.d;
      double rhs = fma(kc, X(i), A.f);
      rhs = fma(ka, X(i - 2), rhs);
      rhs = fma(kb, X(i - 1), rhs);
      rhs = fma(kd, X(i + 1), rhs);
      S.y[i * S.sw] = rhs;
    }
    __syncthreads();
    // L y = rhs (unit lower: y_i = rhs_i - l1_i y_{i-1} - l2_i y_{i-2})
    block_recurrence2(
        n, +1,
        [&](int64_t i, double& r, double& c1, double& c2) {
          const IluRow R = ilu_row(S, i);
          r = S.y[i * S.sw];
          c1 = i >= 1 ? R.l1 : 0.0;
          c2 = i >= 2 ? R.l2 : 0.0;
        },
        [&](int64_t i, double v) { S.y[i * S.sw] = v; }, sh);
    __syncthreads();
    // U x = y: x_i = (y_i - u1_i x_{i+1} - e_i x_{i+2}) / u0_i
    block_recurrence2(
        n, -1,
        [&](int64_t i, double& r, double& c1, double& c2) {
          const double ru = S.ru0[i * S.sw];
          r = S.y[i * S.sw] * ru;
          c1 = (i + 1 < n) ? S.u1[i * S.sw] * ru : 0.0;
          c2 = (i + 2 < n) ? S.e[i * S.sa] * ru : 0.0;
        },
        [&](int64_t i, double v) { S.x[i * S.sx] = v; }, sh);
    __syncthreads();
    // r = f - A x
    double loc = 0.0;
    bool nan_seen = false;
    for (int64_t i = lo; i < hi; ++i) {
      const Row A = S.row(i);
      double ax = A.c * X(i);
      ax = fma(A.a, X(i - 2), ax);
      ax = fma(A.b, X(i - 1), ax);
      ax = fma(A.d, X(i + 1), ax);
      ax = fma(A.e, X(i + 2), ax);
      const double r = A.f - ax;
      nan_seen |= (r != r);
      loc = fmax(loc, fabs(r));
    }
    rn = block_max(nan_seen ? INFINITY : loc, red);
    nonfinite = !isfinite(rn);
    ++k;
  }
  if (threadIdx.x == 0) {
    if (p.iters) p.iters[s] = k;
    if (p.resid) p.resid[s] = nonfinite ? NAN : rn;
    set_status(p.status, s,
               nonfinite ? BAND_ERR_NONFINITE : (rn < p.tol ? BAND_OK : BAND_ERR_NOT_CONVERGED));
  }
  __syncthreads();
}

// Shared-memory bytes per row of a system held whole by the tail: a..f, x, 1/u0, u1, y.
constexpr int kTailSmemArrays = 10;

// System s of p continued by the block.  When the system has at most smem_rows rows, all
// its arrays are first copied into `smem` (kTailSmemArrays * smem_rows doubles), the
// updates run there and x is copied back; otherwise they run on global memory.  Same
// operations in the same order either way.
__device__ inline void sip_tail_block(const SipArgs& p, int64_t t, double rn, Aff* sh, double* red,
                                      double* smem, int64_t smem_rows) {
  const int64_t s = p.L.sys(t);     // t: position in the batch, s: the system id

  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(t), ws = p.W.stride();
  if (n <= smem_rows) {
    double* sa = smem;
    double* sb = sa + n;
    double* sc = sb + n;
    double* sd = sc + n;
    double* se = sd + n;
    double* sf = se + n;
    double* sx = sf + n;
    double* sr = sx + n;
    double* su = sr + n;
    double* sy = su + n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int64_t q = q0 + i * es, w = w0 + i * ws;
      sa[i] = ldro(p.a + q);
      sb[i] = ldro(p.b + q);
      sc[i] = ldro(p.c + q);
      sd[i] = ldro(p.d + q);
      se[i] = ldro(p.e + q);
      sf[i] = p.f[q];
      sx[i] = p.x[q];
      sr[i] = p.ru0[w];
      su[i] = p.u1[w];
    }
    __syncthreads();
    const TailSys S{sa, sb, sc, sd, se, sf, 1, sx, 1, sr, su, sy, 1, n};
    sip_tail_run(p, s, S, rn, sh, red);
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p.x[q0 + i * es] = sx[i];
    __syncthreads();
  } else {
    const TailSys S{p.a + q0, p.b + q0, p.c + q0, p.d + q0, p.e + q0, p.f + q0, es,
                    p.x + q0, es, p.ru0 + w0, p.u1 + w0, p.y + w0, ws, n};
    sip_tail_run(p, s, S, rn, sh, red);
  }
}

// Largest dynamic shared memory of a tail block: 200 KiB (2560 rows), next to the
// block's static scan buffers, within the 227 KiB an sm_103a block may opt in to.
constexpr size_t kTailSmemMax = (size_t)200 << 10;
size_t tail_smem_bytes(int64_t n_max);
cudaError_t tail_prepare(const void* kernel);

// Rows a tail block can hold in shared memory (dynamic bytes `bytes`).
__host__ __device__ inline int64_t tail_smem_rows(size_t bytes) {
  return (int64_t)(bytes / (sizeof(double) * kTailSmemArrays));
}

struct SipArgs;
cudaError_t launch_sip_tail(const SipArgs& p, int64_t nsys, cudaStream_t st);
band_status make_sip(const band_desc* desc, const void* const diag[5], const void* f, void* x,
                     double tol, int32_t max_it, int32_t width, int32_t* iters, double* resid,
                     int32_t* sys_status, void* ws, size_t ws_bytes, SipArgs* sa, SipWs* wout);

}  // namespace band
