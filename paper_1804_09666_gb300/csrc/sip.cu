// sip.cu -- SIP / the Stone method (Veneva & Ayriyan, arXiv:1804.09666, Sec. 2,
// Algorithm 1) with ILU(0) and, optionally, Hotelling-Bodewig band inverses in place
// of the forward/backward substitutions (Remark of Sec. 2; Eq. (1), Appendix).
// One thread per system; FP64.
//
// ILU(0) on the pentadiagonal pattern, row-wise: for k = i-2, i-1 in the pattern,
// l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for j > k in the pattern of row i.  For
// this pattern nothing is dropped, so L (unit; l2 = L[i][i-2], l1 = L[i][i-1]) and
// U (u0 = U[i][i], u1 = U[i][i+1], u2 = U[i][i+2] = e_i) are the exact LU factors.
#include "api_util.h"
#include "kernels.h"

namespace band {
namespace {

constexpr int kMaxWidth = 8;

struct IluArgs {
  Layout L;
  Spill W;
  const double *a, *b, *c, *d, *e;
  double *l2, *l1, *u0, *ru0, *u1;
  int32_t* status;
};

__global__ void __launch_bounds__(128) k_ilu0(const IluArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  // rows i-1 and i-2 of U: u0, 1/u0, u1, u2
  double ru0_1 = 0, u1_1 = 0, u2_1 = 0, ru0_2 = 0, u1_2 = 0, u2_2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es, w = w0 + i * ws;
    double w0v = (i >= 2) ? ldro(p.a + q) : 0.0;
    double w1v = (i >= 1) ? ldro(p.b + q) : 0.0;
    double w2v = ldro(p.c + q);
    double w3v = (i + 1 < n) ? ldro(p.d + q) : 0.0;
    const double w4v = (i + 2 < n) ? ldro(p.e + q) : 0.0;
    if (i >= 2) {
      w0v = w0v * ru0_2;
      w1v = fma(-w0v, u1_2, w1v);
      w2v = fma(-w0v, u2_2, w2v);
    }
    if (i >= 1) {
      w1v = w1v * ru0_1;
      w2v = fma(-w1v, u1_1, w2v);
      w3v = fma(-w1v, u2_1, w3v);
    }
    if (w2v == 0.0) {
      set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
      return;
    }
    const double r = rcp64(w2v);
    p.l2[w] = w0v;
    p.l1[w] = w1v;
    p.u0[w] = w2v;
    p.ru0[w] = r;
    p.u1[w] = w3v;
    ru0_2 = ru0_1; u1_2 = u1_1; u2_2 = u2_1;
    ru0_1 = r; u1_1 = w3v; u2_1 = w4v;
  }
  set_status(p.status, s, BAND_OK);
}

// Band Hotelling-Bodewig, X_{k+1} = X_k (2I - M X_k), X_0 = diag(M)^{-1}, X kept to
// w diagonals.  Written along a sweep index t (t = i for L, t = n-1-i for U) so that
// both factors look lower triangular: X_j[t] = X[t][t-j], and M's entries along the
// sweep are m0 (diagonal; 1 for L), m1 (one step back), m2 (two steps back).  With
// P = M X:  Pr_j[t] = sum_{o<=min(2,j)} M_o[t] X_{j-o}[t-o], and
//   Xnew_j[t] = 2 X_j[t] - sum_{k=0..j} X_k[t] Pr_{j-k}[t-k].
struct HbArgs {
  Layout L;
  Spill W;
  int w, upper, max_it;
  double tol;
  const double *m0, *m1, *m2;   // L: (nullptr, l1, l2); U: (u0, u1, e-from-input)
  const double* e_in;           // U's second superdiagonal is e itself (input layout)
  double* X[kMaxWidth];         // result
  double* Y[kMaxWidth];         // ping-pong partner
  int32_t* status;
  int32_t* hb_iters;
};

__global__ void __launch_bounds__(64) k_hb(const HbArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (p.status && p.status[s] != BAND_OK) return;
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  const int w = p.w;
  auto row_of = [&](int64_t t) { return p.upper ? n - 1 - t : t; };
  auto Mo = [&](int o, int64_t t) -> double {  // M entry o steps back along the sweep
    const int64_t i = row_of(t);
    const int64_t wi = w0 + i * ws;
    if (o == 0) return p.upper ? p.m0[wi] : 1.0;
    if (o == 1) return p.m1[wi];
    return p.upper ? ldro(p.e_in + q0 + i * es) : p.m2[wi];
  };
  double* const* cur = p.Y;
  double* const* nxt = p.X;
  // X_0 = diag(M)^{-1} into `cur`
  for (int64_t t = 0; t < n; ++t) {
    const int64_t wi = w0 + row_of(t) * ws;
    cur[0][wi] = 1.0 / Mo(0, t);
    for (int j = 1; j < w; ++j) cur[j][wi] = 0.0;
  }
  int it = 0;
  int32_t st = BAND_ERR_NOT_CONVERGED;
  while (it < p.max_it) {
    double xr[3][kMaxWidth];          // X rows t, t-1, t-2 (ring by t % 3)
    double pr[kMaxWidth][kMaxWidth];  // Pr rows t .. t-w+1 (ring by t % w)
    for (int r = 0; r < 3; ++r)
      for (int j = 0; j < kMaxWidth; ++j) xr[r][j] = 0.0;
    for (int r = 0; r < kMaxWidth; ++r)
      for (int j = 0; j < kMaxWidth; ++j) pr[r][j] = 0.0;
    double dmax = 0.0, xmax = 0.0;
    bool nan_seen = false;
    for (int64_t t = 0; t < n; ++t) {
      const int64_t wi = w0 + row_of(t) * ws;
      const int r0 = (int)(t % 3), r1 = (int)((t + 2) % 3), r2 = (int)((t + 1) % 3);
      for (int j = 0; j < w; ++j) xr[r0][j] = cur[j][wi];
      const double mm0 = Mo(0, t);
      const double mm1 = t >= 1 ? Mo(1, t) : 0.0;
      const double mm2 = t >= 2 ? Mo(2, t) : 0.0;
      const int pt = (int)(t % w);
      for (int j = 0; j < w; ++j) {
        double v = mm0 * xr[r0][j];
        if (j >= 1 && t >= 1) v = fma(mm1, xr[r1][j - 1], v);
        if (j >= 2 && t >= 2) v = fma(mm2, xr[r2][j - 2], v);
        pr[pt][j] = v;
      }
      for (int j = 0; j < w; ++j) {
        double acc = 2.0 * xr[r0][j];
        for (int k = 0; k <= j; ++k) {
          if (t - k < 0) break;
          const int pk = (int)((t - k) % w);
          acc = fma(-xr[r0][k], pr[pk][j - k], acc);
        }
        const double old = xr[r0][j];
        nxt[j][wi] = acc;
        const double dd = fabs(acc - old);
        nan_seen |= (acc != acc);
        dmax = fmax(dmax, dd);
        xmax = fmax(xmax, fabs(old));
      }
    }
    ++it;
    double* const* tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (nan_seen || !isfinite(dmax)) { st = BAND_ERR_NONFINITE; break; }
    if (dmax <= p.tol * xmax) { st = BAND_OK; break; }
  }
  // the result must end in X
  if (cur != p.X) {
    for (int64_t t = 0; t < n; ++t) {
      const int64_t wi = w0 + row_of(t) * ws;
      for (int j = 0; j < w; ++j) p.X[j][wi] = cur[j][wi];
    }
  }
  if (p.hb_iters) p.hb_iters[s] = it;
  // a capped HB iteration still gives usable approximate inverses; SIP decides
  if (st == BAND_ERR_NONFINITE) set_status(p.status, s, st);
}

struct SipArgs {
  Layout L;
  Spill W;
  const double *a, *b, *c, *d, *e, *f;
  double* x;           // result (also one of the two iterate buffers)
  double* xb;          // second iterate buffer (workspace, spill layout)
  double* y;           // substitution scratch (workspace, spill layout)
  const double *l2, *l1, *u0, *ru0, *u1;
  int w;
  const double* XL[kMaxWidth];
  const double* XU[kMaxWidth];
  double tol;
  int max_it;
  int32_t *iters, *status;
  double* resid;
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

// Algorithm 1 as printed: rhs = K x + f, L y = rhs, U x = y, r = f - A x, until
// max|r| < tol or max_it updates, or until an update from the second on fails to
// lower max|r| (the rounding floor of exact ILU(0) factors; NOT_CONVERGED).
__device__ void sip_literal(const SipArgs& p, int64_t s) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  double rn = 0.0;
  for (int64_t i = 0; i < n; ++i) {  // x^0 = 0, r^0 = f
    const int64_t q = q0 + i * es;
    rn = fmax(rn, fabs(p.f[q]));
    p.x[q] = 0.0;
  }
  int k = 0;
  double prev = INFINITY;
  for (;;) {
    if (rn < p.tol || k >= p.max_it || !isfinite(rn)) break;
    // K = LU - A holds only rounding errors: an update (from the second on) that does
    // not lower the residual means its rounding floor is reached
    if (k >= 2 && !(rn < prev)) break;
    prev = rn;
    // forward: rhs_i = sum_j K[i][j] x_j + f_i, y_i = rhs_i - l1_i y_{i-1} - l2_i y_{i-2}
    double y1 = 0, y2 = 0;
    double u0m1 = 0, u1m1 = 0, u0m2 = 0, u1m2 = 0, em1 = 0, em2 = 0;
    double xm2 = 0, xm1 = 0, x0 = p.x[q0], xp1 = n > 1 ? p.x[q0 + es] : 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t q = q0 + i * es, wi = w0 + i * ws;
      const Row A = load_row(p, q, i, n);
      const double l2 = (i >= 2) ? p.l2[wi] : 0.0, l1 = (i >= 1) ? p.l1[wi] : 0.0;
      const double u0 = p.u0[wi], u1 = (i + 1 < n) ? p.u1[wi] : 0.0;
      // K = LU - A on this row (K[i][i+2] = u2 - e = 0)
      const double ka = l2 * u0m2 - A.a;
      const double kb = fma(l2, u1m2, l1 * u0m1) - A.b;
      const double kc = fma(l2, em2, fma(l1, u1m1, u0)) - A.c;
      const double kd = fma(l1, em1, u1) - A.d;
      double rhs = fma(kc, x0, A.f);
      rhs = fma(ka, xm2, rhs);
      rhs = fma(kb, xm1, rhs);
      rhs = fma(kd, xp1, rhs);
      const double yv = fma(-l2, y2, fma(-l1, y1, rhs));
      p.y[wi] = yv;
      y2 = y1; y1 = yv;
      u0m2 = u0m1; u1m2 = u1m1; em2 = em1;
      u0m1 = u0; u1m1 = u1; em1 = A.e;
      xm2 = xm1; xm1 = x0; x0 = xp1;
      xp1 = (i + 2 < n) ? p.x[q + 2 * es] : 0.0;
    }
    // backward: x_i = (y_i - u1_i x_{i+1} - e_i x_{i+2}) / u0_i, with the residual of
    // row i+2 once x_i .. x_{i+4} are new
    double n1 = 0, n2 = 0, n3 = 0, n4 = 0;  // new x_{i+1} .. x_{i+4}
    rn = 0.0;
    bool nan_seen = false;
    for (int64_t i = n - 1; i >= -2; --i) {
      double xi = 0.0;
      if (i >= 0) {
        const int64_t q = q0 + i * es, wi = w0 + i * ws;
        const double u1 = (i + 1 < n) ? p.u1[wi] : 0.0;
        const double ei = (i + 2 < n) ? ldro(p.e + q) : 0.0;
        xi = fma(-ei, n2, fma(-u1, n1, p.y[wi])) * p.ru0[wi];
        p.x[q] = xi;
      }
      const int64_t j = i + 2;  // residual row
      if (j >= 0 && j < n) {
        const Row A = load_row(p, q0 + j * es, j, n);
        double ax = A.c * n2;
        ax = fma(A.a, xi, ax);
        ax = fma(A.b, n1, ax);
        ax = fma(A.d, n3, ax);
        ax = fma(A.e, n4, ax);
        const double r = A.f - ax;
        nan_seen |= (r != r);
        rn = fmax(rn, fabs(r));
      }
      n4 = n3; n3 = n2; n2 = n1; n1 = xi;
    }
    if (nan_seen) rn = NAN;
    ++k;
  }
  if (p.iters) p.iters[s] = k;
  if (p.resid) p.resid[s] = rn;
  set_status(p.status, s,
             !isfinite(rn) ? BAND_ERR_NONFINITE : (rn < p.tol ? BAND_OK : BAND_ERR_NOT_CONVERGED));
}

// HB variant: x <- x + U~^{-1} (L~^{-1} (f - A x)) in one sweep per iteration.  The
// sweep computes r = f - A x_old (and its norm), y = L~^{-1} r with a lag of 0 and
// x_new = x_old + U~^{-1} y with a lag of w-1 rows.  When max|r| < tol the update
// just computed is discarded: the answer is x_old with k updates (Algorithm 1's
// stop test on the residual of the current iterate).
__device__ void sip_hb(const SipArgs& p, int64_t s) {
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

__global__ void __launch_bounds__(64) k_sip(const SipArgs p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (p.status && p.status[s] != BAND_OK) {  // ILU(0) or HB failed for this system
    if (p.iters) p.iters[s] = 0;
    if (p.resid) p.resid[s] = NAN;
    return;
  }
  if (p.w == 0) sip_literal(p, s);
  else sip_hb(p, s);
}

struct SipWs {
  double *l2, *l1, *u0, *ru0, *u1, *y, *xb;
  double* X[2 * kMaxWidth];  // XL then XU
  double* T[2 * kMaxWidth];  // ping-pong partners
  int32_t* st;               // status scratch when the caller passes none
};

SipWs carve_sip(const band_desc* d, int32_t width, void* base, size_t* bytes) {
  Carve c(base);
  SipWs w{};
  const size_t rows = (size_t)spill_rows(d) * sizeof(double);
  w.l2 = (double*)c.take(rows);
  w.l1 = (double*)c.take(rows);
  w.u0 = (double*)c.take(rows);
  w.ru0 = (double*)c.take(rows);
  w.u1 = (double*)c.take(rows);
  w.y = (double*)c.take(rows);
  w.xb = (double*)c.take(rows);
  for (int j = 0; j < 2 * width; ++j) w.X[j] = (double*)c.take(rows);
  for (int j = 0; j < 2 * width; ++j) w.T[j] = (double*)c.take(rows);
  w.st = (int32_t*)c.take(sizeof(int32_t) * (size_t)(d->nsys > 0 ? d->nsys : 1));
  *bytes = c.size();
  return w;
}

}  // namespace

size_t sip_workspace_bytes(const band_desc* d, int32_t width) {
  if (width < 0 || width > kMaxWidth) return 0;
  size_t b = 0;
  carve_sip(d, width, nullptr, &b);
  return b;
}

}  // namespace band

using namespace band;

extern "C" band_status band_sip(const band_desc* desc, const void* const diag[5], const void* f,
                                void* x, double tol, int32_t max_it, int32_t width,
                                int32_t hb_max_it, double hb_tol, int32_t* iters, double* resid,
                                int32_t* sys_status, void* ws, size_t ws_bytes, void* stream) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64) return BAND_ERR_ARG;
  if (width < 0 || width > kMaxWidth || max_it < 0 || hb_max_it < 0) return BAND_ERR_ARG;
  if (!(tol >= 0.0) || !(hb_tol >= 0.0)) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !f || !x) return BAND_ERR_ARG;
  if (!diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc) && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  if (width < 0 || width > kMaxWidth || max_it < 0 || hb_max_it < 0) return BAND_ERR_ARG;
  if (!(tol >= 0.0) || !(hb_tol >= 0.0)) return BAND_ERR_ARG;
  // TD systems are treated as PD with a = e = 0; that needs a and e arrays.
  if (!diag[0] || !diag[4]) return BAND_ERR_ARG;
  size_t need = 0;
  carve_sip(desc, width, nullptr, &need);
  if (!ws || ws_bytes < need) return BAND_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const SipWs w = carve_sip(desc, width, ws, &need);
  int32_t* status = sys_status ? sys_status : w.st;
  const Layout L = layout_of(desc);
  const Spill W = spill_of(desc);
  const double* A[5] = {(const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
                        (const double*)diag[3], (const double*)diag[4]};
  const unsigned g128 = (unsigned)((desc->nsys + 127) / 128);
  const unsigned g64 = (unsigned)((desc->nsys + 63) / 64);
  IluArgs ia{L, W, A[0], A[1], A[2], A[3], A[4], w.l2, w.l1, w.u0, w.ru0, w.u1, status};
  k_ilu0<<<g128, 128, 0, st>>>(ia);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  SipArgs sa{};
  sa.L = L;
  sa.W = W;
  sa.a = A[0]; sa.b = A[1]; sa.c = A[2]; sa.d = A[3]; sa.e = A[4];
  sa.f = (const double*)f;
  sa.x = (double*)x;
  sa.xb = w.xb;
  sa.y = w.y;
  sa.l2 = w.l2; sa.l1 = w.l1; sa.u0 = w.u0; sa.ru0 = w.ru0; sa.u1 = w.u1;
  sa.w = width;
  sa.tol = tol;
  sa.max_it = max_it;
  sa.iters = iters;
  sa.status = status;
  sa.resid = resid;
  if (width > 0) {
    for (int upper = 0; upper < 2; ++upper) {
      HbArgs h{};
      h.L = L;
      h.W = W;
      h.w = width;
      h.upper = upper;
      h.max_it = hb_max_it;
      h.tol = hb_tol;
      h.m0 = upper ? w.u0 : nullptr;
      h.m1 = upper ? w.u1 : w.l1;
      h.m2 = upper ? nullptr : w.l2;
      h.e_in = A[4];
      for (int j = 0; j < width; ++j) {
        h.X[j] = w.X[upper * width + j];
        h.Y[j] = w.T[upper * width + j];
      }
      h.status = status;
      h.hb_iters = nullptr;
      k_hb<<<g64, 64, 0, st>>>(h);
      if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    }
    for (int j = 0; j < width; ++j) {
      sa.XL[j] = w.X[j];
      sa.XU[j] = w.X[width + j];
    }
  }
  k_sip<<<g64, 64, 0, st>>>(sa);
  return cuda_status(cudaGetLastError());
}
