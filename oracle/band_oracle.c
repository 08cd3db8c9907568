/*
 * band_oracle.c -- plain, slow, FP64 CPU oracle for the batched band solvers
 * (the Laurent-series pass of the symbolic methods carries double-double
 * coefficients; see R3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library; it is
 * not part of the product.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or constant with the CUDA path.
 *
 * Source: M. Veneva, A. Ayriyan, "Performance Analysis of Effective Methods for
 * Solving Band Matrix SLAEs after Parabolic Nonlinear PDEs" (arXiv:1804.09666).
 * The paper names the methods but prints the recurrences of NPDM/NTDM/SPDM/STDM
 * only by reference (Sec. 1), so the recurrences below are LU factorisation
 * without pivoting written from its definition; NPDM's operation count is pinned
 * to the paper's 19N-29 (Table 7).
 *
 * Storage (row-aligned diagonals, one system, contiguous, length n):
 *   a[i] = A[i][i-2], b[i] = A[i][i-1], c[i] = A[i][i], d[i] = A[i][i+1], e[i] = A[i][i+2].
 *   Slots outside the matrix (a[0], a[1], b[0], d[n-1], e[n-2], e[n-1]) are never read
 *   into the arithmetic.  Tridiagonal routines use b, c, d only.  Right-hand side f,
 *   solution x.
 *
 * Every routine allocates its own scratch with malloc and returns an ORC_* status.
 * Compiled with -O2 -ffp-contract=off so that every operation is rounded on its own.
 *
 * parity unpinned: the NTDM count (the paper's 9N+2 in Table 7 is not reproduced
 * by R1, which performs 8N-7) and the SIP count (31N-36 per iteration, Table 7)
 * are recorded by the counters below but pin nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* Status codes of the oracle (its own numbering; the tests map them by name). */
enum {
  ORC_OK = 0,
  ORC_ARG = 1,
  ORC_ZERO_PIVOT = 3,
  ORC_SINGULAR = 4,
  ORC_NONFINITE = 5,
  ORC_NOT_CONVERGED = 6,
  ORC_SYMBOLIC_RANGE = 7,
  ORC_NOMEM = 10
};

/* ------------------------------------------------------------------------- */
/* Operation counting (Table 7).  A NULL counter disables counting.           */
/* ------------------------------------------------------------------------- */
#define CNT(ops) do { if (ops) ++*(ops); } while (0)
static inline double op_add(double x, double y, long long* ops) { CNT(ops); return x + y; }
static inline double op_sub(double x, double y, long long* ops) { CNT(ops); return x - y; }
static inline double op_mul(double x, double y, long long* ops) { CNT(ops); return x * y; }
static inline double op_div(double x, double y, long long* ops) { CNT(ops); return x / y; }

static int all_finite(int64_t n, const double* x) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* ------------------------------------------------------------------------- */
/* R1 -- NTDM: LU of a tridiagonal matrix without pivoting, U unit (Sec. 1;   */
/* the Thomas method of Sec. 4).                                              */
/*   mu_0 = c_0, alpha_0 = d_0/mu_0, z_0 = f_0/mu_0                           */
/*   mu_i = c_i - b_i alpha_{i-1};  alpha_i = d_i/mu_i;  z_i = (f_i - b_i z_{i-1})/mu_i */
/*   x_{n-1} = z_{n-1};  x_i = z_i - alpha_i x_{i+1}                           */
/* ------------------------------------------------------------------------- */
int orc_ntdm(int64_t n, const double* b, const double* c, const double* d,
             const double* f, double* x, long long* ops) {
  if (n < 1) return ORC_ARG;
  double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  if (!alpha || !z) { free(alpha); free(z); return ORC_NOMEM; }
  int st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    double mu = c[i];
    if (i >= 1) mu = op_sub(mu, op_mul(b[i], alpha[i - 1], ops), ops);
    if (mu == 0.0) { st = ORC_ZERO_PIVOT; break; }
    if (i <= n - 2) alpha[i] = op_div(d[i], mu, ops);
    double zi = f[i];
    if (i >= 1) zi = op_sub(zi, op_mul(b[i], z[i - 1], ops), ops);
    z[i] = op_div(zi, mu, ops);
  }
  if (st == ORC_OK) {
    x[n - 1] = z[n - 1];
    for (int64_t i = n - 2; i >= 0; --i)
      x[i] = op_sub(z[i], op_mul(alpha[i], x[i + 1], ops), ops);
    if (!all_finite(n, x)) st = ORC_NONFINITE;
  } else {
    for (int64_t i = 0; i < n; ++i) x[i] = NAN;
  }
  free(alpha); free(z);
  return st;
}

/* ------------------------------------------------------------------------- */
/* R2 -- NPDM: LU of a pentadiagonal matrix without pivoting (Sec. 1, ref. to */
/* the PD algorithm; cost 19N-29, Table 7).  L has diagonals (a_i, gamma_i,   */
/* mu_i), U is unit upper with (alpha_i, beta_i).  Terms that reach outside   */
/* the matrix are skipped, not multiplied by zero, so the operation count is  */
/* exactly the paper's.                                                       */
/*   gamma_i = b_i - alpha_{i-2} a_i                                          */
/*   mu_i    = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i                     */
/*   alpha_i = (d_i - beta_{i-1} gamma_i) / mu_i                              */
/*   beta_i  = e_i / mu_i                                                     */
/*   z_i     = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i                   */
/*   x_{n-1} = z_{n-1}; x_{n-2} = z_{n-2} - alpha_{n-2} x_{n-1};              */
/*   x_i = z_i - alpha_i x_{i+1} - beta_i x_{i+2}                             */
/* If `fac` is not NULL it receives gamma, mu, alpha, beta (4 arrays of n).   */
/* ------------------------------------------------------------------------- */
int orc_npdm(int64_t n, const double* a, const double* b, const double* c,
             const double* d, const double* e, const double* f, double* x,
             double* fac, long long* ops) {
  if (n < 1) return ORC_ARG;
  double* gam = (double*)calloc((size_t)n, sizeof(double));
  double* mu = (double*)calloc((size_t)n, sizeof(double));
  double* alpha = (double*)calloc((size_t)n, sizeof(double));
  double* beta = (double*)calloc((size_t)n, sizeof(double));
  double* z = (double*)calloc((size_t)n, sizeof(double));
  if (!gam || !mu || !alpha || !beta || !z) {
    free(gam); free(mu); free(alpha); free(beta); free(z);
    return ORC_NOMEM;
  }
  int st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    double g = 0.0;
    if (i >= 1) g = b[i];
    if (i >= 2) g = op_sub(b[i], op_mul(alpha[i - 2], a[i], ops), ops);
    gam[i] = g;
    double m = c[i];
    if (i >= 2) m = op_sub(m, op_mul(beta[i - 2], a[i], ops), ops);
    if (i >= 1) m = op_sub(m, op_mul(alpha[i - 1], g, ops), ops);
    mu[i] = m;
    if (m == 0.0) { st = ORC_ZERO_PIVOT; break; }
    if (i <= n - 2) {
      double num = d[i];
      if (i >= 1) num = op_sub(num, op_mul(beta[i - 1], g, ops), ops);
      alpha[i] = op_div(num, m, ops);
    }
    if (i <= n - 3) beta[i] = op_div(e[i], m, ops);
    double zi = f[i];
    if (i >= 2) zi = op_sub(zi, op_mul(z[i - 2], a[i], ops), ops);
    if (i >= 1) zi = op_sub(zi, op_mul(z[i - 1], g, ops), ops);
    z[i] = op_div(zi, m, ops);
  }
  if (st == ORC_OK) {
    x[n - 1] = z[n - 1];
    if (n >= 2) x[n - 2] = op_sub(z[n - 2], op_mul(alpha[n - 2], x[n - 1], ops), ops);
    for (int64_t i = n - 3; i >= 0; --i) {
      double xi = op_sub(z[i], op_mul(alpha[i], x[i + 1], ops), ops);
      x[i] = op_sub(xi, op_mul(beta[i], x[i + 2], ops), ops);
    }
    if (!all_finite(n, x)) st = ORC_NONFINITE;
  } else {
    for (int64_t i = 0; i < n; ++i) x[i] = NAN;
  }
  if (fac) {
    memcpy(fac, gam, sizeof(double) * (size_t)n);
    memcpy(fac + n, mu, sizeof(double) * (size_t)n);
    memcpy(fac + 2 * n, alpha, sizeof(double) * (size_t)n);
    memcpy(fac + 3 * n, beta, sizeof(double) * (size_t)n);
  }
  free(gam); free(mu); free(alpha); free(beta); free(z);
  return st;
}

/* The same R2 recurrence in single precision (used by the refinement R7). */
static int npdm_f32(int64_t n, const float* a, const float* b, const float* c,
                    const float* d, const float* e, const float* f, float* x,
                    float* w /* 4n scratch */) {
  float* alpha = w;
  float* beta = w + n;
  float* z = w + 2 * n;
  for (int64_t i = 0; i < n; ++i) {
    float g = 0.0f;
    if (i >= 1) g = b[i];
    if (i >= 2) g = b[i] - alpha[i - 2] * a[i];
    float m = c[i];
    if (i >= 2) m = m - beta[i - 2] * a[i];
    if (i >= 1) m = m - alpha[i - 1] * g;
    if (m == 0.0f) return ORC_ZERO_PIVOT;
    alpha[i] = 0.0f;
    beta[i] = 0.0f;
    if (i <= n - 2) {
      float num = d[i];
      if (i >= 1) num = num - beta[i - 1] * g;
      alpha[i] = num / m;
    }
    if (i <= n - 3) beta[i] = e[i] / m;
    float zi = f[i];
    if (i >= 2) zi = zi - z[i - 2] * a[i];
    if (i >= 1) zi = zi - z[i - 1] * g;
    z[i] = zi / m;
  }
  x[n - 1] = z[n - 1];
  if (n >= 2) x[n - 2] = z[n - 2] - alpha[n - 2] * x[n - 1];
  for (int64_t i = n - 3; i >= 0; --i)
    x[i] = (z[i] - alpha[i] * x[i + 1]) - beta[i] * x[i + 2];
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return ORC_NONFINITE;
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R0 -- banded Gaussian elimination with partial (row) pivoting: the truth   */
/* x = A^{-1} f that SPDM/STDM reach exactly and SIP within its tolerance.    */
/* Half bandwidth k (1 = TD, 2 = PD).  Column band storage: entry (i, j) of   */
/* the working matrix lives at W[(kv + i - j) + j*ld], kv = 2k (row swaps     */
/* widen U to 2k superdiagonals), ld = 3k+1.  det receives det(A) (may be    */
/* NULL); it is 0 when a column has no nonzero pivot candidate.              */
/* ------------------------------------------------------------------------- */
int orc_gepp_band(int64_t n, int k, const double* a, const double* b, const double* c,
                  const double* d, const double* e, const double* f, double* x, double* det) {
  if (n < 1 || (k != 1 && k != 2)) return ORC_ARG;
  const int kl = k, kv = 2 * k, ld = 3 * k + 1;
  double* W = (double*)calloc((size_t)ld * (size_t)n, sizeof(double));
  if (!W) return ORC_NOMEM;
#define WIJ(i, j) W[(size_t)(kv + (i) - (j)) + (size_t)(j) * (size_t)ld]
  for (int64_t i = 0; i < n; ++i) {
    WIJ(i, i) = c[i];
    if (i >= 1) WIJ(i, i - 1) = b[i];
    if (i + 1 < n) WIJ(i, i + 1) = d[i];
    if (k == 2) {
      if (i >= 2) WIJ(i, i - 2) = a[i];
      if (i + 2 < n) WIJ(i, i + 2) = e[i];
    }
    x[i] = f[i];
  }
  double dt = 1.0;
  int singular = 0;
  for (int64_t j = 0; j < n; ++j) {
    int64_t last = j + kl < n - 1 ? j + kl : n - 1;
    int64_t p = j;
    double best = fabs(WIJ(j, j));
    for (int64_t i = j + 1; i <= last; ++i)
      if (fabs(WIJ(i, j)) > best) { best = fabs(WIJ(i, j)); p = i; }
    if (best == 0.0) { singular = 1; dt = 0.0; continue; }
    int64_t cend = j + kv < n - 1 ? j + kv : n - 1;
    if (p != j) {
      for (int64_t cc = j; cc <= cend; ++cc) {
        double t = WIJ(j, cc); WIJ(j, cc) = WIJ(p, cc); WIJ(p, cc) = t;
      }
      double t = x[j]; x[j] = x[p]; x[p] = t;
      dt = -dt;
    }
    dt *= WIJ(j, j);
    for (int64_t i = j + 1; i <= last; ++i) {
      double l = WIJ(i, j) / WIJ(j, j);
      WIJ(i, j) = l;
      for (int64_t cc = j + 1; cc <= cend; ++cc) WIJ(i, cc) -= l * WIJ(j, cc);
      x[i] -= l * x[j];
    }
  }
  if (det) *det = dt;
  if (singular) {
    for (int64_t i = 0; i < n; ++i) x[i] = NAN;
    free(W);
    return ORC_SINGULAR;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    int64_t cend = i + kv < n - 1 ? i + kv : n - 1;
    double s = x[i];
    for (int64_t cc = i + 1; cc <= cend; ++cc) s -= WIJ(i, cc) * x[cc];
    x[i] = s / WIJ(i, i);
  }
#undef WIJ
  free(W);
  return all_finite(n, x) ? ORC_OK : ORC_NONFINITE;
}

/* ------------------------------------------------------------------------- */
/* R2m -- MNPDM (Sec. 1: the PD method that takes the sparsity of the outer   */
/* diagonals into account; Sec. 3.2 Remark 2: a Gaussian elimination turns   */
/* the PD matrix into a TD one at 16 operations per row that carries nonzero  */
/* outer entries), then R1 on the TD system.  The paper prints neither the    */
/* elimination nor its order; reading: first, bottom-up, every nonzero e_i    */
/* (column i+2) is eliminated with row i+1, which by then has no entry beyond */
/* column i+2:                                                                */
/*   m = e_i / D_{i+1};  B_i -= m a_{i+1};  C_i -= m B_{i+1};                  */
/*   D_i -= m C_{i+1};  F_i -= m F_{i+1}          (1 + 8 operations);          */
/* then, top-down, every nonzero a_i (column i-2) with row i-1, which by then */
/* is tridiagonal:                                                            */
/*   m = a_i / B_{i-1};  B_i -= m C_{i-1};  C_i -= m D_{i-1};                   */
/*   F_i -= m F_{i-1}                              (1 + 6 operations),         */
/* where (B, C, D, F) are the row's sub-, main and superdiagonal entries and  */
/* right-hand side as they stand.  A row with both outer entries nonzero costs */
/* 16 operations, a row 0 with only e (no column i-1) 7, a row with only a 7.  */
/* A zero divisor (D_{i+1} or B_{i-1}) is ZERO_PIVOT, as is a zero pivot of   */
/* R1 on the result.                                                          */
/* ------------------------------------------------------------------------- */
int orc_mnpdm(int64_t n, const double* a, const double* b, const double* c, const double* d,
              const double* e, const double* f, double* x, long long* ops) {
  if (n < 1) return ORC_ARG;
  double* B = (double*)malloc(sizeof(double) * (size_t)n);
  double* C = (double*)malloc(sizeof(double) * (size_t)n);
  double* D = (double*)malloc(sizeof(double) * (size_t)n);
  double* F = (double*)malloc(sizeof(double) * (size_t)n);
  if (!B || !C || !D || !F) { free(B); free(C); free(D); free(F); return ORC_NOMEM; }
  int st = ORC_OK;
  for (int64_t i = n - 1; i >= 0; --i) {
    B[i] = i >= 1 ? b[i] : 0.0;
    C[i] = c[i];
    D[i] = i + 1 < n ? d[i] : 0.0;
    F[i] = f[i];
    if (i + 2 < n && e[i] != 0.0) {
      if (D[i + 1] == 0.0) { st = ORC_ZERO_PIVOT; break; }
      double m = op_div(e[i], D[i + 1], ops);
      if (i >= 1) B[i] = op_sub(B[i], op_mul(m, i + 1 >= 2 ? a[i + 1] : 0.0, ops), ops);
      C[i] = op_sub(C[i], op_mul(m, B[i + 1], ops), ops);
      D[i] = op_sub(D[i], op_mul(m, C[i + 1], ops), ops);
      F[i] = op_sub(F[i], op_mul(m, F[i + 1], ops), ops);
    }
  }
  for (int64_t i = 2; st == ORC_OK && i < n; ++i) {
    if (a[i] == 0.0) continue;
    if (B[i - 1] == 0.0) { st = ORC_ZERO_PIVOT; break; }
    double m = op_div(a[i], B[i - 1], ops);
    B[i] = op_sub(B[i], op_mul(m, C[i - 1], ops), ops);
    C[i] = op_sub(C[i], op_mul(m, D[i - 1], ops), ops);
    F[i] = op_sub(F[i], op_mul(m, F[i - 1], ops), ops);
  }
  if (st == ORC_OK) st = orc_ntdm(n, B, C, D, F, x, ops);
  else for (int64_t i = 0; i < n; ++i) x[i] = NAN;
  free(B); free(C); free(D); free(F);
  return st;
}

/* ------------------------------------------------------------------------- */
/* R3 -- SPDM / STDM: the R2 / R1 recurrences in which a pivot that is zero   */
/* is replaced by a symbol t; every later quantity becomes a function of t    */
/* and the solution is its limit t -> 0 (Sec. 1: the symbolic methods "only   */
/* require nonsingularity").  Replacing mu_i by t is the exact LU of          */
/* A(t) = A + t * sum_{flagged j} e_j e_j^T, so x(t) -> A^{-1} f.             */
/*                                                                            */
/* A system without a zero pivot never meets the symbol: its SPDM / STDM is   */
/* R2 / R1 itself (R1 is R2 with a = e = 0, operation for operation), and     */
/* det A is the product of R2's pivots.  A system whose R2 pass meets an      */
/* exactly zero pivot is solved again in truncated Laurent series in t.       */
/*                                                                            */
/* Series arithmetic.  Coefficient of t^k at q[k + LP], k in [-LP, LP]; the   */
/* series is known for exponents k < hi (hi <= LP + 1; a plain number has hi  */
/* = LP + 1).  Coefficients are double-double numbers (below), and a          */
/* coefficient formed as a sum of terms (a sum or difference of two series,   */
/* a coefficient of a product, the numerator of a quotient's coefficient)    */
/* whose result lies below 2^-80 of the sum of the terms' magnitudes is set   */
/* to zero: in exact arithmetic it is zero, and what double-double leaves of  */
/* it is rounding residue (~2^-104 of the terms per operation), which would   */
/* otherwise pass for a nonzero leading coefficient.  Readings (the paper is  */
/* silent):                                                                   */
/*  - a zero pivot of the R2 pass is an exact IEEE zero, or a pivot within    */
/*    rounding residue of zero (residue_pivot below); in the series pass one  */
/*    symbol stands for every pivot whose known coefficients are all zero;    */
/*  - x(t) is analytic at t = 0 when A is nonsingular, so the negative-power */
/*    coefficients of each x_i are rounding residue and are dropped;          */
/*  - det A = lim prod mu_i(t): with V = sum of the valuations of the mu_i,   */
/*    V > 0 means det A = 0 (SINGULAR), V = 0 gives the product of the        */
/*    leading coefficients (Sec. 3.2, Remark 1: the O(N) determinant), V < 0 */
/*    cannot happen in exact arithmetic and is reported as SYMBOLIC_RANGE;   */
/*  - a pole deeper than t^-LP, or an x_i whose t^0 coefficient is not known,*/
/*    is SYMBOLIC_RANGE.                                                      */
/* ------------------------------------------------------------------------- */

/* Double-double numbers hi + lo with |lo| <= ulp(hi) / 2 (Dekker, "A floating- */
/* point technique for extending the available precision", 1971).  The exact  */
/* error of a rounded sum comes from Knuth's two-sum, that of a rounded        */
/* product from one fused multiply-add; sum, product and quotient are then     */
/* accurate to about 2^-104 relative.                                          */
typedef struct { double hi, lo; } dd;

static dd dd_of(double v) { dd r = {v, 0.0}; return r; }
/* s + e = a + b exactly (any a, b) */
static dd two_sum(double a, double b) {
  double s = a + b;
  double bv = s - a;
  double av = s - bv;
  dd r = {s, (a - av) + (b - bv)};
  return r;
}
/* s + e = a + b exactly, when |a| >= |b| or a == 0 */
static dd quick_two_sum(double a, double b) {
  double s = a + b;
  dd r = {s, b - (s - a)};
  return r;
}
static dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd x) { dd r = {-x.hi, -x.lo}; return r; }
static dd dd_mul(dd x, dd y) {
  double p = x.hi * y.hi;
  double e = fma(x.hi, y.hi, -p);             /* p + e = x.hi * y.hi exactly */
  e += x.hi * y.lo + x.lo * y.hi;
  return quick_two_sum(p, e);
}
/* x / y by three quotient digits, each correcting the remainder */
static dd dd_div(dd x, dd y) {
  double q1 = x.hi / y.hi;
  dd r = dd_add(x, dd_neg(dd_mul(y, dd_of(q1))));
  double q2 = r.hi / y.hi;
  r = dd_add(r, dd_neg(dd_mul(y, dd_of(q2))));
  double q3 = r.hi / y.hi;
  return dd_add(quick_two_sum(q1, q2), dd_of(q3));
}
static int dd_is_zero(dd x) { return x.hi == 0.0; }
#define DD_RESIDUE 0x1p-80
/* v, or zero when it is rounding residue of terms of total magnitude mag */
static dd dd_flush(dd v, double mag) {
  if (fabs(v.hi) <= DD_RESIDUE * mag) return dd_of(0.0);
  return v;
}

#define LP 16
#define LW (2 * LP + 1)
typedef struct { dd q[LW]; int hi; } lser;

static lser ls_const(double v) {
  lser s; memset(&s, 0, sizeof s); s.q[LP] = dd_of(v); s.hi = LP + 1; return s;
}
static lser ls_symbol(void) {
  lser s; memset(&s, 0, sizeof s); s.q[LP + 1] = dd_of(1.0); s.hi = LP + 1; return s;
}
/* lowest exponent with a known nonzero coefficient, or LP + 1 if none */
static int ls_val(const lser* s) {
  for (int k = -LP; k < s->hi && k <= LP; ++k)
    if (!dd_is_zero(s->q[k + LP])) return k;
  return LP + 1;
}
static int imin(int x, int y) { return x < y ? x : y; }

static lser ls_addsub(const lser* x, const lser* y, double sign) {
  lser r; memset(&r, 0, sizeof r);
  r.hi = imin(x->hi, y->hi);
  for (int k = -LP; k < r.hi && k <= LP; ++k) {
    dd u = x->q[k + LP], v = y->q[k + LP];
    if (sign < 0) v = dd_neg(v);
    r.q[k + LP] = dd_flush(dd_add(u, v), fabs(u.hi) + fabs(v.hi));
  }
  return r;
}
/* a series with no known nonzero coefficient is O(t^hi) */
static int ls_veff(const lser* s) { int v = ls_val(s); return v <= LP ? v : s->hi; }

/* product; known below min(vx + hi_y, vy + hi_x), so every kept coefficient is complete */
static lser ls_mul(const lser* x, const lser* y, int* err) {
  lser r; memset(&r, 0, sizeof r);
  double mag[LW] = {0};
  int vx = ls_veff(x), vy = ls_veff(y);
  r.hi = imin(LP + 1, imin(vx + y->hi, vy + x->hi));
  for (int i = -LP; i < x->hi && i <= LP; ++i)
    for (int j = -LP; j < y->hi && j <= LP; ++j) {
      if (dd_is_zero(x->q[i + LP]) || dd_is_zero(y->q[j + LP])) continue;
      int k = i + j;
      if (k >= r.hi) continue;
      if (k < -LP) { *err = 1; continue; }
      dd p = dd_mul(x->q[i + LP], y->q[j + LP]);
      r.q[k + LP] = dd_add(r.q[k + LP], p);
      mag[k + LP] += fabs(p.hi);
    }
  for (int k = 0; k < LW; ++k) r.q[k] = dd_flush(r.q[k], mag[k]);
  return r;
}
/* quotient by long division; relative precision is the smaller of the two */
static lser ls_div(const lser* x, const lser* y, int* err) {
  lser r; memset(&r, 0, sizeof r);
  int vy = ls_val(y);
  if (vy > LP) { *err = 1; r.hi = -LP; return r; }   /* divisor not known to be nonzero */
  int vx = ls_val(x);
  if (vx > LP) { r.hi = imin(LP + 1, x->hi - vy); return r; }
  int v = vx - vy;
  int rel = imin(x->hi - vx, y->hi - vy);
  r.hi = imin(LP + 1, v + rel);
  if (v < -LP) { *err = 1; return r; }
  /* c_k = (x_{k+vy} - sum_{j>=1} y_{vy+j} c_{k-j}) / y_{vy} */
  for (int k = v; k < r.hi; ++k) {
    dd s = x->q[k + vy + LP];
    double mag = fabs(s.hi);
    for (int j = 1; k - j >= v; ++j) {
      dd p = dd_mul(y->q[vy + j + LP], r.q[k - j + LP]);
      s = dd_add(s, dd_neg(p));
      mag += fabs(p.hi);
    }
    r.q[k + LP] = dd_div(dd_flush(s, mag), y->q[vy + LP]);
  }
  return r;
}
static lser ls_sub_mul(const lser* acc, const lser* p, const lser* q, int* err) {
  lser m = ls_mul(p, q, err);
  return ls_addsub(acc, &m, -1.0);
}

typedef struct { int V; double mant; long long ex; } detacc;
static void det_push(detacc* D, int v, double lead) {
  D->V += v;
  int e2;
  double m = frexp(lead, &e2);
  D->mant *= m; D->ex += e2;
  int e3; D->mant = frexp(D->mant, &e3); D->ex += e3;
}

/* The series pass over a system whose R2 pass met a zero pivot. */
static int symbolic_series(int64_t n, int k, const double* a, const double* b, const double* c,
                           const double* d, const double* e, const double* f, double* x,
                           detacc* D, int* nflag) {
  lser* alpha = (lser*)calloc((size_t)n, sizeof(lser));
  lser* beta = (lser*)calloc((size_t)n, sizeof(lser));
  lser* z = (lser*)calloc((size_t)n, sizeof(lser));
  lser* xs = (lser*)calloc((size_t)n, sizeof(lser));
  if (!alpha || !beta || !z || !xs) { free(alpha); free(beta); free(z); free(xs); return ORC_NOMEM; }
  int err = 0, flags = 0;
  for (int64_t i = 0; i < n; ++i) {
    lser ai = ls_const((k == 2 && i >= 2) ? a[i] : 0.0);
    lser g = ls_const(0.0);
    if (i >= 1) g = ls_const(b[i]);
    if (k == 2 && i >= 2) g = ls_sub_mul(&g, &alpha[i - 2], &ai, &err);
    lser m = ls_const(c[i]);
    if (k == 2 && i >= 2) m = ls_sub_mul(&m, &beta[i - 2], &ai, &err);
    if (i >= 1) m = ls_sub_mul(&m, &alpha[i - 1], &g, &err);
    if (ls_val(&m) > LP) { m = ls_symbol(); ++flags; }      /* zero pivot -> t */
    int v = ls_val(&m);
    det_push(D, v, m.q[v + LP].hi);
    alpha[i] = ls_const(0.0);
    beta[i] = ls_const(0.0);
    if (i <= n - 2) {
      lser num = ls_const(d[i]);
      if (k == 2 && i >= 1) num = ls_sub_mul(&num, &beta[i - 1], &g, &err);
      alpha[i] = ls_div(&num, &m, &err);
    }
    if (k == 2 && i <= n - 3) {
      lser ei = ls_const(e[i]);
      beta[i] = ls_div(&ei, &m, &err);
    }
    lser zi = ls_const(f[i]);
    if (k == 2 && i >= 2) zi = ls_sub_mul(&zi, &z[i - 2], &ai, &err);
    if (i >= 1) zi = ls_sub_mul(&zi, &z[i - 1], &g, &err);
    z[i] = ls_div(&zi, &m, &err);
  }
  /* back substitution; keep only the non-negative powers of every x_i */
  for (int64_t i = n - 1; i >= 0; --i) {
    lser xi = z[i];
    if (i + 1 < n) xi = ls_sub_mul(&xi, &alpha[i], &xs[i + 1], &err);
    if (k == 2 && i + 2 < n) xi = ls_sub_mul(&xi, &beta[i], &xs[i + 2], &err);
    for (int kk = -LP; kk < 0; ++kk) xi.q[kk + LP] = dd_of(0.0);
    if (xi.hi <= 0) err = 1;
    xs[i] = xi;
    x[i] = xi.q[LP].hi;
  }
  *nflag = flags;
  free(alpha); free(beta); free(z); free(xs);
  if (D->V > 0) return ORC_SINGULAR;
  if (err || D->V < 0) return ORC_SYMBOLIC_RANGE;
  return all_finite(n, x) ? ORC_OK : ORC_NONFINITE;
}

/* Does R2's pass hold a pivot that double arithmetic cannot tell from zero?   */
/* mu_i = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i, with gamma_i = b_i -      */
/* alpha_{i-2} a_i.  When |mu_i| lies 2^40 or more below the largest quantity  */
/* that entered it -- the row's entries a_i, b_i, c_i, the products           */
/* beta_{i-2} a_i and alpha_{i-1} gamma_i, and the terms of alpha_{i-1}       */
/* gamma_i with gamma_i expanded (alpha_{i-1} b_i, alpha_{i-1} alpha_{i-2}     */
/* a_i, which catch a cancellation inside gamma_i) -- an exact zero and the    */
/* rounding residue of one cannot be told apart in double arithmetic, so the   */
/* system goes to the series pass, whose double-double arithmetic decides      */
/* (reading; Sec. 1 asks only for a nonsingular matrix).  A pivot that is      */
/* merely small gets the same, exact-to-double-double, treatment there.        */
/* fac = R2's (gamma, mu, alpha, beta).                                        */
#define PIVOT_RESIDUE 0x1p-40
static double dmax(double x, double y) { return x > y ? x : y; }
static int residue_pivot(int64_t n, const double* a, const double* b, const double* c,
                         const double* fac) {
  const double* gam = fac;
  const double* mu = fac + n;
  const double* alpha = fac + 2 * n;
  const double* beta = fac + 3 * n;
  for (int64_t i = 0; i < n; ++i) {
    double ai = i >= 2 ? a[i] : 0.0, bi = i >= 1 ? b[i] : 0.0;
    double al1 = i >= 1 ? alpha[i - 1] : 0.0, al2 = i >= 2 ? alpha[i - 2] : 0.0;
    double be2 = i >= 2 ? beta[i - 2] : 0.0;
    double big = dmax(dmax(fabs(ai), fabs(bi)), fabs(c[i]));
    big = dmax(big, dmax(fabs(be2 * ai), fabs(al1 * gam[i])));
    big = dmax(big, dmax(fabs(al1 * bi), fabs(al1 * al2 * ai)));
    if (fabs(mu[i]) <= PIVOT_RESIDUE * big) return 1;
  }
  return 0;
}

/* Symbolic PD (k = 2) or TD (k = 1) solve.  det_out (may be NULL) receives   */
/* det(A) as mant * 2^ex (ex in *det_ex); *nflag the number of zero pivots.  */
int orc_symbolic(int64_t n, int k, const double* a, const double* b, const double* c,
                 const double* d, const double* e, const double* f, double* x,
                 double* det_mant, long long* det_ex, int* nflag) {
  if (n < 1 || (k != 1 && k != 2)) return ORC_ARG;
  double* fac = (double*)malloc(4 * (size_t)n * sizeof(double));
  double* zero = k == 1 ? (double*)calloc((size_t)n, sizeof(double)) : NULL;
  if (!fac || (k == 1 && !zero)) { free(fac); free(zero); return ORC_NOMEM; }
  const double* pa = k == 2 ? a : zero;
  const double* pe = k == 2 ? e : zero;
  detacc D = {0, 1.0, 0};
  int flags = 0;
  int st = orc_npdm(n, pa, b, c, d, pe, f, x, fac, NULL);
  if (st == ORC_OK && residue_pivot(n, pa, b, c, fac)) st = ORC_ZERO_PIVOT;
  if (st == ORC_ZERO_PIVOT) {
    st = symbolic_series(n, k, pa, b, c, d, pe, f, x, &D, &flags);
  } else {
    for (int64_t i = 0; i < n; ++i) det_push(&D, 0, fac[n + i]);    /* R2's mu_i */
  }
  free(fac); free(zero);
  if (nflag) *nflag = flags;
  if (det_mant) *det_mant = D.V == 0 ? D.mant : 0.0;
  if (det_ex) *det_ex = D.V == 0 ? D.ex : 0;
  return st;
}

/* ------------------------------------------------------------------------- */
/* R4 -- ILU(0) on the pentadiagonal pattern (Sec. 2), in the row-wise        */
/* (IKJ) form of incomplete Gaussian elimination: for row i and each k < i in */
/* the pattern, l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for every j > k    */
/* that is in the pattern of row i (entries outside the pattern are dropped). */
/* For a pentadiagonal pattern no update ever falls outside it, which is why */
/* the paper notes that LU is again pentadiagonal.  Output: L unit lower with */
/* l2 = L[i][i-2], l1 = L[i][i-1]; U with u0 = U[i][i], u1 = U[i][i+1],       */
/* u2 = U[i][i+2].                                                            */
/* ------------------------------------------------------------------------- */
int orc_ilu0(int64_t n, const double* a, const double* b, const double* c, const double* d,
             const double* e, double* l2, double* l1, double* u0, double* u1, double* u2) {
  if (n < 1) return ORC_ARG;
  for (int64_t i = 0; i < n; ++i) {
    /* row i of the working matrix, columns i-2 .. i+2 */
    double w[5];
    w[0] = i >= 2 ? a[i] : 0.0;
    w[1] = i >= 1 ? b[i] : 0.0;
    w[2] = c[i];
    w[3] = i + 1 < n ? d[i] : 0.0;
    w[4] = i + 2 < n ? e[i] : 0.0;
    /* k = i-2: pattern of row i-2 to the right of its diagonal is {i-1, i} */
    if (i >= 2) {
      if (u0[i - 2] == 0.0) return ORC_ZERO_PIVOT;
      w[0] = w[0] / u0[i - 2];
      w[1] = w[1] - w[0] * u1[i - 2];
      w[2] = w[2] - w[0] * u2[i - 2];
    }
    /* k = i-1: pattern of row i-1 to the right of its diagonal is {i, i+1} */
    if (i >= 1) {
      if (u0[i - 1] == 0.0) return ORC_ZERO_PIVOT;
      w[1] = w[1] / u0[i - 1];
      w[2] = w[2] - w[1] * u1[i - 1];
      w[3] = w[3] - w[1] * u2[i - 1];
    }
    l2[i] = w[0]; l1[i] = w[1]; u0[i] = w[2]; u1[i] = w[3]; u2[i] = w[4];
    if (u0[i] == 0.0) return ORC_ZERO_PIVOT;
  }
  return ORC_OK;
}

/* K = LU - A on the five diagonals: the remainder of the splitting A = LU - K */
/* that Algorithm 1 iterates on.                                              */
void orc_lu_minus_a(int64_t n, const double* l2, const double* l1, const double* u0,
                    const double* u1, const double* u2, const double* a, const double* b,
                    const double* c, const double* d, const double* e,
                    double* ka, double* kb, double* kc, double* kd, double* ke) {
  for (int64_t i = 0; i < n; ++i) {
    /* (LU)[i][j] = sum_m L[i][m] U[m][j], L[i][i] = 1 */
    double lu_a = 0.0, lu_b = 0.0, lu_c = 0.0, lu_d = 0.0, lu_e = 0.0;
    if (i >= 2) { lu_a += l2[i] * u0[i - 2]; lu_b += l2[i] * u1[i - 2]; lu_c += l2[i] * u2[i - 2]; }
    if (i >= 1) { lu_b += l1[i] * u0[i - 1]; lu_c += l1[i] * u1[i - 1]; lu_d += l1[i] * u2[i - 1]; }
    lu_c += u0[i]; lu_d += u1[i]; lu_e += u2[i];
    ka[i] = i >= 2 ? lu_a - a[i] : 0.0;
    kb[i] = i >= 1 ? lu_b - b[i] : 0.0;
    kc[i] = lu_c - c[i];
    kd[i] = i + 1 < n ? lu_d - d[i] : 0.0;
    ke[i] = i + 2 < n ? lu_e - e[i] : 0.0;
  }
}

/* ------------------------------------------------------------------------- */
/* R5 -- Hotelling-Bodewig inverse iteration, Eq. (1) of the Appendix:        */
/*   X_{k+1} = X_k (2I - M X_k),  X_0 = diag(M)^{-1}                          */
/* in the band ("array") form: X is kept to w diagonals, lower (M = L, unit   */
/* lower with l1, l2) or upper (M = U with u0, u1, u2).  Storage: X[j*n + i]  */
/* = X[i][i-j] (lower) or X[i][i+j] (upper), j = 0..w-1.  The product         */
/* P = M X_k is formed first, then X_{k+1} = X_k (2I - P) is truncated to w  */
/* diagonals.  Stops when max|X_{k+1} - X_k| <= tol * max|X_k| or after       */
/* max_it iterations; *iters receives the number of iterations done.         */
/* Dense helpers index the band through these two accessors.                 */
/* ------------------------------------------------------------------------- */
static double band_get(const double* X, int64_t n, int w, int lower, int64_t i, int64_t j) {
  if (i < 0 || j < 0 || i >= n || j >= n) return 0.0;
  int64_t off = lower ? i - j : j - i;
  if (off < 0 || off >= w) return 0.0;
  return X[off * n + i];
}
static double mat_get(int lower, int64_t n, const double* m0, const double* m1,
                      const double* m2, int64_t i, int64_t j) {
  /* lower: L[i][i]=1, L[i][i-1]=m1[i], L[i][i-2]=m2[i]; upper: U[i][i]=m0[i], U[i][i+1]=m1[i], U[i][i+2]=m2[i] */
  if (i < 0 || j < 0 || i >= n || j >= n) return 0.0;
  int64_t off = lower ? i - j : j - i;
  if (off == 0) return lower ? 1.0 : m0[i];
  if (off == 1) return m1[i];
  if (off == 2) return m2[i];
  return 0.0;
}

int orc_hb(int64_t n, int w, int lower, const double* m0, const double* m1, const double* m2,
           double* X, int max_it, double tol, int* iters) {
  if (n < 1 || w < 1) return ORC_ARG;
  int wp = w + 2;                       /* bandwidth of P = M X */
  double* Xn = (double*)calloc((size_t)w * (size_t)n, sizeof(double));
  double* P = (double*)calloc((size_t)wp * (size_t)n, sizeof(double));
  if (!Xn || !P) { free(Xn); free(P); return ORC_NOMEM; }
  memset(X, 0, sizeof(double) * (size_t)w * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    double dg = lower ? 1.0 : m0[i];
    if (dg == 0.0) { free(Xn); free(P); return ORC_ZERO_PIVOT; }
    X[i] = 1.0 / dg;                    /* X_0 = diag(M)^{-1} */
  }
  int it = 0, st = ORC_NOT_CONVERGED;
  while (it < max_it) {
    /* P = M X */
    for (int64_t i = 0; i < n; ++i)
      for (int jo = 0; jo < wp; ++jo) {
        int64_t j = lower ? i - jo : i + jo;
        double s = 0.0;
        for (int mo = 0; mo <= 2; ++mo) {
          int64_t m = lower ? i - mo : i + mo;
          s += mat_get(lower, n, m0, m1, m2, i, m) * band_get(X, n, w, lower, m, j);
        }
        P[jo * n + i] = s;
      }
    /* X_{k+1} = X (2I - P), kept to w diagonals */
    double dmax = 0.0, xmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int jo = 0; jo < w; ++jo) {
        int64_t j = lower ? i - jo : i + jo;
        double s = 0.0;
        for (int mo = 0; mo < w; ++mo) {
          int64_t m = lower ? i - mo : i + mo;
          double y = (m == j ? 2.0 : 0.0) - band_get(P, n, wp, lower, m, j);
          s += band_get(X, n, w, lower, i, m) * y;
        }
        Xn[jo * n + i] = s;
        double old = X[jo * n + i];
        if (fabs(s - old) > dmax) dmax = fabs(s - old);
        if (fabs(old) > xmax) xmax = fabs(old);
      }
    memcpy(X, Xn, sizeof(double) * (size_t)w * (size_t)n);
    ++it;
    if (!(dmax == dmax) || !isfinite(dmax)) { st = ORC_NONFINITE; break; }
    if (dmax <= tol * xmax) { st = ORC_OK; break; }
  }
  *iters = it;
  free(Xn); free(P);
  return st;
}

/* y = M r for a band inverse X stored as in orc_hb */
static void band_apply(const double* X, int64_t n, int w, int lower, const double* r, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int jo = 0; jo < w; ++jo) {
      int64_t j = lower ? i - jo : i + jo;
      if (j < 0 || j >= n) continue;
      s += X[jo * n + i] * r[j];
    }
    y[i] = s;
  }
}

/* r = f - A x (pentadiagonal); returns max |r_i|, or NaN if any r_i is NaN */
static double residual_pd(int64_t n, const double* a, const double* b, const double* c,
                          const double* d, const double* e, const double* f, const double* x,
                          double* r, long long* ops) {
  double m = 0.0;
  int nan_seen = 0;
  for (int64_t i = 0; i < n; ++i) {
    double s = op_mul(c[i], x[i], ops);
    if (i >= 2) s = op_add(s, op_mul(a[i], x[i - 2], ops), ops);
    if (i >= 1) s = op_add(s, op_mul(b[i], x[i - 1], ops), ops);
    if (i + 1 < n) s = op_add(s, op_mul(d[i], x[i + 1], ops), ops);
    if (i + 2 < n) s = op_add(s, op_mul(e[i], x[i + 2], ops), ops);
    r[i] = op_sub(f[i], s, ops);
    if (isnan(r[i])) nan_seen = 1;
    else if (fabs(r[i]) > m) m = fabs(r[i]);
  }
  return nan_seen ? NAN : m;
}

/* ------------------------------------------------------------------------- */
/* R6 -- SIP / the Stone method, Algorithm 1 (Sec. 2).                       */
/* hb_width == 0: the stationary iteration of the splitting A = LU - K with   */
/*   the ILU(0) factors: from x^0 = 0, every update solves LU x^{k+1} =       */
/*   K x^k + f by the two substitutions, and the iteration stops once the     */
/*   residual f - A x has max-norm below tol (Algorithm 1's steps, in its     */
/*   order).                                                                  */
/* hb_width  > 0: the Remark of Sec. 2 -- L^{-1}, U^{-1} from Hotelling-     */
/*   Bodewig (R5, w = hb_width) replace the two substitutions; with inexact  */
/*   inverses the update is written in correction form                        */
/*   x <- x + U~^{-1} L~^{-1} (f - A x), identical to Algorithm 1 when the    */
/*   inverses are exact (reading).                                            */
/* The loop also stops after max_it updates (NOT_CONVERGED), and, for          */
/* hb_width == 0, once an update (from the second on) fails to lower max|r|:    */
/* with exact ILU(0) factors K = LU - A holds only rounding errors, so the      */
/* residual has reached its rounding floor (NOT_CONVERGED; reading).            */
/* *iters gets k,                                                               */
/* *resid the final max |r_i|.  hb_iters (may be NULL) gets the HB counts for */
/* L and U.                                                                   */
/* ------------------------------------------------------------------------- */
int orc_sip(int64_t n, const double* a, const double* b, const double* c, const double* d,
            const double* e, const double* f, double* x, double tol, int max_it, int hb_width,
            int hb_max_it, double hb_tol, int* iters, double* resid, int* hb_iters,
            long long* ops) {
  if (n < 1 || max_it < 0 || hb_width < 0) return ORC_ARG;
  size_t N = (size_t)n;
  int w = hb_width;
  double* l2 = (double*)calloc(N, sizeof(double));
  double* l1 = (double*)calloc(N, sizeof(double));
  double* u0 = (double*)calloc(N, sizeof(double));
  double* u1 = (double*)calloc(N, sizeof(double));
  double* u2 = (double*)calloc(N, sizeof(double));
  double* K = (double*)calloc(5 * N, sizeof(double));
  double* r = (double*)calloc(N, sizeof(double));
  double* y = (double*)calloc(N, sizeof(double));
  double* XL = w > 0 ? (double*)calloc((size_t)w * N, sizeof(double)) : NULL;
  double* XU = w > 0 ? (double*)calloc((size_t)w * N, sizeof(double)) : NULL;
  int st = ORC_OK;
  if (!l2 || !l1 || !u0 || !u1 || !u2 || !K || !r || !y || (w > 0 && (!XL || !XU))) {
    st = ORC_NOMEM; goto done;
  }
  st = orc_ilu0(n, a, b, c, d, e, l2, l1, u0, u1, u2);
  if (st != ORC_OK) goto done;
  if (w == 0) {
    orc_lu_minus_a(n, l2, l1, u0, u1, u2, a, b, c, d, e, K, K + N, K + 2 * N, K + 3 * N, K + 4 * N);
  } else {
    int itl = 0, itu = 0;
    int s1 = orc_hb(n, w, 1, NULL, l1, l2, XL, hb_max_it, hb_tol, &itl);
    int s2 = orc_hb(n, w, 0, u0, u1, u2, XU, hb_max_it, hb_tol, &itu);
    if (hb_iters) { hb_iters[0] = itl; hb_iters[1] = itu; }
    if (s1 == ORC_NONFINITE || s2 == ORC_NONFINITE) { st = ORC_NONFINITE; goto done; }
    if (s1 == ORC_ZERO_PIVOT || s2 == ORC_ZERO_PIVOT) { st = ORC_ZERO_PIVOT; goto done; }
  }
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  int k = 0;
  double rn = residual_pd(n, a, b, c, d, e, f, x, r, ops);
  double prev = INFINITY;
  while (!(rn < tol)) {
    if (k >= max_it || !isfinite(rn)) break;
    /* Algorithm 1 with exact substitutions: K = LU - A is rounding-level, so an update
       that does not lower the residual means the rounding floor is reached (reading) */
    if (w == 0 && k >= 2 && !(rn < prev)) break;
    prev = rn;
    if (w == 0) {
      /* rhs = K x + f, into y */
      const double *ka = K, *kb = K + N, *kc = K + 2 * N, *kd = K + 3 * N, *ke = K + 4 * N;
      for (int64_t i = 0; i < n; ++i) {
        double s = op_mul(kc[i], x[i], ops);
        if (i >= 2) s = op_add(s, op_mul(ka[i], x[i - 2], ops), ops);
        if (i >= 1) s = op_add(s, op_mul(kb[i], x[i - 1], ops), ops);
        if (i + 1 < n) s = op_add(s, op_mul(kd[i], x[i + 1], ops), ops);
        if (i + 2 < n) s = op_add(s, op_mul(ke[i], x[i + 2], ops), ops);
        y[i] = op_add(s, f[i], ops);
      }
      /* solve L y = rhs (unit lower), in place */
      for (int64_t i = 0; i < n; ++i) {
        if (i >= 1) y[i] = op_sub(y[i], op_mul(l1[i], y[i - 1], ops), ops);
        if (i >= 2) y[i] = op_sub(y[i], op_mul(l2[i], y[i - 2], ops), ops);
      }
      /* solve U x = y */
      for (int64_t i = n - 1; i >= 0; --i) {
        double s = y[i];
        if (i + 1 < n) s = op_sub(s, op_mul(u1[i], x[i + 1], ops), ops);
        if (i + 2 < n) s = op_sub(s, op_mul(u2[i], x[i + 2], ops), ops);
        x[i] = op_div(s, u0[i], ops);
      }
    } else {
      band_apply(XL, n, w, 1, r, y);
      band_apply(XU, n, w, 0, y, r);
      for (int64_t i = 0; i < n; ++i) x[i] += r[i];
    }
    ++k;
    rn = residual_pd(n, a, b, c, d, e, f, x, r, ops);
  }
  *iters = k;
  *resid = rn;
  if (!isfinite(rn)) st = ORC_NONFINITE;
  else if (!(rn < tol)) st = ORC_NOT_CONVERGED;
done:
  free(l2); free(l1); free(u0); free(u1); free(u2); free(K); free(r); free(y); free(XL); free(XU);
  return st;
}

/* ------------------------------------------------------------------------- */
/* R6b -- SIP on a two-dimensional five-point matrix (Sec. 2: Stone's method,    */
/* whose ILU(0) drops the fill-in that a two-dimensional pattern creates).       */
/* Unknown k = y nx + x of an nx x ny grid; row k holds s_k at column k - nx,    */
/* w_k at k - 1, c_k at k, e_k at k + 1, t_k at k + nx (entries leaving the grid */
/* are not part of the matrix).  ILU(0) keeps L's and U's entries on A's         */
/* pattern: L unit lower with ls (column k - nx) and lw (k - 1), U with uc (k),   */
/* ue (k + 1), ut (k + nx), fixed row by row so that (LU)_{kj} = A_{kj} on the   */
/* pattern:                                                                     */
/*   ls_k = s_k / uc_{k-nx},  lw_k = w_k / uc_{k-1},                             */
/*   uc_k = c_k - ls_k ut_{k-nx} - lw_k ue_{k-1},  ue_k = e_k,  ut_k = t_k;       */
/* the products ls_k ue_{k-nx} (column k - nx + 1) and lw_k ut_{k-1} (column      */
/* k + nx - 1) fall outside the pattern and are dropped: they are K = LU - A.    */
/* Algorithm 1 then iterates LU x^{j+1} = K x^j + f from x^0 = 0 until          */
/* max|f - A x| < tol, or max_it updates (NOT_CONVERGED).                        */
/* ------------------------------------------------------------------------- */
static int in_grid(int64_t nx, int64_t ny, int64_t k, int dx, int dy) {
  int64_t x = k % nx + dx, y = k / nx + dy;
  return x >= 0 && x < nx && y >= 0 && y < ny;
}

int orc_sip2d(int64_t nx, int64_t ny, const double* s, const double* w, const double* c,
              const double* e, const double* t, const double* f, double* x, double tol,
              int max_it, int* iters, double* resid) {
  if (nx < 1 || ny < 1 || max_it < 0) return ORC_ARG;
  int64_t N = nx * ny;
  double* ls = (double*)calloc((size_t)N, sizeof(double));
  double* lw = (double*)calloc((size_t)N, sizeof(double));
  double* uc = (double*)calloc((size_t)N, sizeof(double));
  double* y = (double*)calloc((size_t)N, sizeof(double));
  if (!ls || !lw || !uc || !y) { free(ls); free(lw); free(uc); free(y); return ORC_NOMEM; }
  int st = ORC_OK;
  /* entries of A on the grid (zero where the neighbour leaves it) */
#define AS(k) (in_grid(nx, ny, k, 0, -1) ? s[k] : 0.0)
#define AW(k) (in_grid(nx, ny, k, -1, 0) ? w[k] : 0.0)
#define AE(k) (in_grid(nx, ny, k, 1, 0) ? e[k] : 0.0)
#define AT(k) (in_grid(nx, ny, k, 0, 1) ? t[k] : 0.0)
  for (int64_t k = 0; k < N; ++k) {
    double v = c[k];
    if (in_grid(nx, ny, k, 0, -1)) { ls[k] = AS(k) / uc[k - nx]; v -= ls[k] * AT(k - nx); }
    if (in_grid(nx, ny, k, -1, 0)) { lw[k] = AW(k) / uc[k - 1]; v -= lw[k] * AE(k - 1); }
    uc[k] = v;
    if (v == 0.0) { st = ORC_ZERO_PIVOT; break; }
  }
  int it = 0;
  double rn = INFINITY;
  if (st == ORC_OK) {
    for (int64_t k = 0; k < N; ++k) x[k] = 0.0;
    for (;;) {
      /* r = f - A x, max |r| */
      rn = 0.0;
      for (int64_t k = 0; k < N; ++k) {
        double ax = c[k] * x[k];
        if (in_grid(nx, ny, k, 0, -1)) ax += AS(k) * x[k - nx];
        if (in_grid(nx, ny, k, -1, 0)) ax += AW(k) * x[k - 1];
        if (in_grid(nx, ny, k, 1, 0)) ax += AE(k) * x[k + 1];
        if (in_grid(nx, ny, k, 0, 1)) ax += AT(k) * x[k + nx];
        double r = f[k] - ax;
        if (!(fabs(r) <= rn)) rn = fabs(r);
      }
      if (rn < tol || it >= max_it || !isfinite(rn)) break;
      /* K x + f, then L y = K x + f, then U x = y */
      for (int64_t k = 0; k < N; ++k) {
        double v = f[k];
        if (in_grid(nx, ny, k, 1, -1)) v += ls[k] * AE(k - nx) * x[k - nx + 1];
        if (in_grid(nx, ny, k, -1, 1)) v += lw[k] * AT(k - 1) * x[k + nx - 1];
        y[k] = v;
      }
      for (int64_t k = 0; k < N; ++k) {
        if (in_grid(nx, ny, k, 0, -1)) y[k] -= ls[k] * y[k - nx];
        if (in_grid(nx, ny, k, -1, 0)) y[k] -= lw[k] * y[k - 1];
      }
      for (int64_t k = N - 1; k >= 0; --k) {
        double v = y[k];
        if (in_grid(nx, ny, k, 1, 0)) v -= AE(k) * x[k + 1];
        if (in_grid(nx, ny, k, 0, 1)) v -= AT(k) * x[k + nx];
        x[k] = v / uc[k];
      }
      ++it;
    }
#undef AS
#undef AW
#undef AE
#undef AT
    if (!isfinite(rn)) st = ORC_NONFINITE;
    else if (!(rn < tol)) st = ORC_NOT_CONVERGED;
  }
  if (iters) *iters = it;
  if (resid) *resid = rn;
  free(ls); free(lw); free(uc); free(y);
  return st;
}

/* The ILU(0) factors of R6b alone (for the pins): ls, lw, uc (ue = e, ut = t). */
int orc_ilu0_2d(int64_t nx, int64_t ny, const double* s, const double* w, const double* c,
                const double* e, const double* t, double* ls, double* lw, double* uc) {
  if (nx < 1 || ny < 1) return ORC_ARG;
  int64_t N = nx * ny;
  for (int64_t k = 0; k < N; ++k) {
    double v = c[k];
    ls[k] = lw[k] = 0.0;
    if (in_grid(nx, ny, k, 0, -1)) {
      ls[k] = s[k] / uc[k - nx];
      v -= ls[k] * t[k - nx];
    }
    if (in_grid(nx, ny, k, -1, 0)) {
      lw[k] = w[k] / uc[k - 1];
      v -= lw[k] * e[k - 1];
    }
    uc[k] = v;
    if (v == 0.0) return ORC_ZERO_PIVOT;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* R7 -- mixed precision: FP32 R2 solve, then iterative refinement            */
/*   r = f - A x (FP64, A = the FP64 values of the FP32 diagonals),           */
/*   s = max|r|, delta = s * solve32(r / s), x += delta (FP64),               */
/* until max|delta| <= rel_stop * max|x| or max_steps corrections.  *steps    */
/* receives the number of corrections applied.                                */
/* ------------------------------------------------------------------------- */
int orc_refine(int64_t n, const float* a, const float* b, const float* c, const float* d,
               const float* e, const double* f, double* x, double rel_stop, int max_steps,
               int* steps) {
  if (n < 1) return ORC_ARG;
  size_t N = (size_t)n;
  double* A64 = (double*)malloc(5 * N * sizeof(double));
  double* r = (double*)malloc(N * sizeof(double));
  float* r32 = (float*)malloc(N * sizeof(float));
  float* x32 = (float*)malloc(N * sizeof(float));
  float* w32 = (float*)malloc(4 * N * sizeof(float));
  int st = ORC_OK, k = 0;
  if (!A64 || !r || !r32 || !x32 || !w32) { st = ORC_NOMEM; goto done; }
  for (size_t i = 0; i < N; ++i) {
    A64[i] = a[i]; A64[N + i] = b[i]; A64[2 * N + i] = c[i]; A64[3 * N + i] = d[i]; A64[4 * N + i] = e[i];
    r32[i] = (float)f[i];
  }
  st = npdm_f32(n, a, b, c, d, e, r32, x32, w32);
  if (st != ORC_OK) goto done;
  for (size_t i = 0; i < N; ++i) x[i] = x32[i];
  while (k < max_steps) {
    double s = residual_pd(n, A64, A64 + N, A64 + 2 * N, A64 + 3 * N, A64 + 4 * N, f, x, r, NULL);
    if (!isfinite(s)) { st = ORC_NONFINITE; break; }
    if (s == 0.0) break;
    for (size_t i = 0; i < N; ++i) r32[i] = (float)(r[i] / s);
    st = npdm_f32(n, a, b, c, d, e, r32, x32, w32);
    if (st != ORC_OK) break;
    double dmax = 0.0, xmax = 0.0;
    for (size_t i = 0; i < N; ++i) {
      double dl = s * (double)x32[i];
      x[i] += dl;
      if (fabs(dl) > dmax) dmax = fabs(dl);
    }
    for (size_t i = 0; i < N; ++i) if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
    ++k;
    if (dmax <= rel_stop * xmax) break;
  }
  if (st == ORC_OK && !all_finite(n, x)) st = ORC_NONFINITE;
done:
  if (steps) *steps = k;
  free(A64); free(r); free(r32); free(x32); free(w32);
  return st;
}

/* ------------------------------------------------------------------------- */
/* R8 -- adjoint of x = A^{-1} f for a loss L(x) with dL/dx = w:               */
/*   A^T lambda = w (R0 on A^T), dL/df = lambda, dL/dA[i][j] = -lambda_i x_j, */
/* so on the row-aligned diagonals: ga_i = -lambda_i x_{i-2},                 */
/* gb_i = -lambda_i x_{i-1}, gc_i = -lambda_i x_i, gd_i = -lambda_i x_{i+1},  */
/* ge_i = -lambda_i x_{i+2}; out-of-matrix slots get 0.  A^T's diagonals in  */
/* the same naming: a'_i = e_{i-2}, b'_i = d_{i-1}, c'_i = c_i,               */
/* d'_i = b_{i+1}, e'_i = a_{i+2}.  k = 1 (TD) fills only gb, gc, gd.         */
/* ------------------------------------------------------------------------- */
int orc_adjoint(int64_t n, int k, const double* a, const double* b, const double* c,
                const double* d, const double* e, const double* x, const double* w,
                double* ga, double* gb, double* gc, double* gd, double* ge, double* gf) {
  if (n < 1 || (k != 1 && k != 2)) return ORC_ARG;
  size_t N = (size_t)n;
  double* T = (double*)calloc(5 * N, sizeof(double));
  if (!T) return ORC_NOMEM;
  double *ta = T, *tb = T + N, *tc = T + 2 * N, *td = T + 3 * N, *te = T + 4 * N;
  for (int64_t i = 0; i < n; ++i) {
    tc[i] = c[i];
    if (i >= 1) tb[i] = d[i - 1];
    if (i + 1 < n) td[i] = b[i + 1];
    if (k == 2 && i >= 2) ta[i] = e[i - 2];
    if (k == 2 && i + 2 < n) te[i] = a[i + 2];
  }
  int st = orc_gepp_band(n, k, ta, tb, tc, td, te, w, gf, NULL);
  for (int64_t i = 0; i < n; ++i) {
    double l = gf[i];
    ga[i] = (k == 2 && i >= 2) ? -l * x[i - 2] : 0.0;
    gb[i] = i >= 1 ? -l * x[i - 1] : 0.0;
    gc[i] = -l * x[i];
    gd[i] = i + 1 < n ? -l * x[i + 1] : 0.0;
    ge[i] = (k == 2 && i + 2 < n) ? -l * x[i + 2] : 0.0;
  }
  free(T);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Condition estimate kappa_1(A) = ||A||_1 ||A^{-1}||_1 with Hager's method    */
/* (as refined by Higham): x = (1/n, ..., 1/n); repeat y = A^{-1} x,           */
/* xi = sign(y), z = A^{-T} xi; stop when max|z_j| <= z^T x, else x = e_j with */
/* j = argmax |z_j|; ||A^{-1}||_1 >= ||y||_1 is the estimate.  Solves use R0.  */
/* Used only to scale the parity tolerance of ill-conditioned systems.        */
/* ------------------------------------------------------------------------- */
double orc_cond1(int64_t n, int k, const double* a, const double* b, const double* c,
                 const double* d, const double* e) {
  size_t N = (size_t)n;
  double* T = (double*)calloc(5 * N, sizeof(double));
  double* x = (double*)malloc(N * sizeof(double));
  double* y = (double*)malloc(N * sizeof(double));
  double* z = (double*)malloc(N * sizeof(double));
  if (!T || !x || !y || !z) { free(T); free(x); free(y); free(z); return -1.0; }
  double *ta = T, *tb = T + N, *tc = T + 2 * N, *td = T + 3 * N, *te = T + 4 * N;
  double anorm = 0.0;     /* ||A||_1 = max column sum */
  for (int64_t j = 0; j < n; ++j) {
    double s = fabs(c[j]);
    if (j + 1 < n) s += fabs(b[j + 1]);
    if (j >= 1) s += fabs(d[j - 1]);
    if (k == 2 && j + 2 < n) s += fabs(a[j + 2]);
    if (k == 2 && j >= 2) s += fabs(e[j - 2]);
    if (s > anorm) anorm = s;
    tc[j] = c[j];
    if (j >= 1) tb[j] = d[j - 1];
    if (j + 1 < n) td[j] = b[j + 1];
    if (k == 2 && j >= 2) ta[j] = e[j - 2];
    if (k == 2 && j + 2 < n) te[j] = a[j + 2];
  }
  for (int64_t i = 0; i < n; ++i) x[i] = 1.0 / (double)n;
  double est = 0.0;
  for (int it = 0; it < 5; ++it) {
    if (orc_gepp_band(n, k, a, b, c, d, e, x, y, NULL) != ORC_OK) { est = INFINITY; break; }
    double s1 = 0.0;
    for (int64_t i = 0; i < n; ++i) { s1 += fabs(y[i]); y[i] = y[i] >= 0.0 ? 1.0 : -1.0; }
    est = s1;
    if (orc_gepp_band(n, k, ta, tb, tc, td, te, y, z, NULL) != ORC_OK) { est = INFINITY; break; }
    int64_t jm = 0;
    double zx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      zx += z[i] * x[i];
      if (fabs(z[i]) > fabs(z[jm])) jm = i;
    }
    if (fabs(z[jm]) <= zx) break;
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    x[jm] = 1.0;
  }
  free(T); free(x); free(y); free(z);
  return anorm * est;
}

/* ------------------------------------------------------------------------- */
/* Batch driver: loops over independent systems (Sec. 1: the N systems of a */
/* sweep share no data, so any order is valid), gathering each system        */
/* into contiguous scratch.  Element i of system s of array p lives at        */
/* p[off_s + i * elem_stride] with off_s = offsets ? offsets[s] : s*sys_stride*/
/* and length n_s = offsets ? offsets[s+1]-offsets[s] : n.  Per-system half   */
/* bandwidth: hbw ? hbw[s] : k.  Systems are split statically over nthreads  */
/* POSIX threads.                                                             */
/* method: 0 NTDM/NPDM (by bandwidth), 1 STDM/SPDM, 2 GEPP-band (truth),      */
/*         3 SIP.                                                              */
/* ------------------------------------------------------------------------- */
typedef struct {
  int method, k;
  int64_t nsys, n, sys_stride, elem_stride;
  const int64_t* offsets;
  const int8_t* hbw;
  const double *a, *b, *c, *d, *e, *f;
  double* x;
  int32_t* status;
  double tol; int max_it, hb_width, hb_max_it; double hb_tol;
  int32_t* iters; double* resid;
  int64_t s0, s1;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* J = (batch_job*)arg;
  int64_t nmax = J->n;
  if (J->offsets)
    for (int64_t s = J->s0; s < J->s1; ++s)
      if (J->offsets[s + 1] - J->offsets[s] > nmax) nmax = J->offsets[s + 1] - J->offsets[s];
  size_t N = (size_t)(nmax > 0 ? nmax : 1);
  double* buf = (double*)malloc(7 * N * sizeof(double));
  if (!buf) {
    for (int64_t s = J->s0; s < J->s1; ++s) J->status[s] = ORC_NOMEM;
    return NULL;
  }
  double *A = buf, *B = buf + N, *C = buf + 2 * N, *D = buf + 3 * N, *E = buf + 4 * N,
         *F = buf + 5 * N, *X = buf + 6 * N;
  for (int64_t s = J->s0; s < J->s1; ++s) {
    int64_t off = J->offsets ? J->offsets[s] : s * J->sys_stride;
    int64_t n = J->offsets ? J->offsets[s + 1] - J->offsets[s] : J->n;
    int k = J->hbw ? J->hbw[s] : J->k;
    for (int64_t i = 0; i < n; ++i) {
      int64_t p = off + i * J->elem_stride;
      A[i] = J->a ? J->a[p] : 0.0;
      B[i] = J->b[p]; C[i] = J->c[p]; D[i] = J->d[p];
      E[i] = J->e ? J->e[p] : 0.0;
      F[i] = J->f[p];
    }
    int st;
    if (J->method == 0)
      st = k == 1 ? orc_ntdm(n, B, C, D, F, X, NULL) : orc_npdm(n, A, B, C, D, E, F, X, NULL, NULL);
    else if (J->method == 1)
      st = orc_symbolic(n, k, A, B, C, D, E, F, X, NULL, NULL, NULL);
    else if (J->method == 2)
      st = orc_gepp_band(n, k, A, B, C, D, E, F, X, NULL);
    else {
      int it = 0; double rs = 0.0;
      st = orc_sip(n, A, B, C, D, E, F, X, J->tol, J->max_it, J->hb_width, J->hb_max_it,
                   J->hb_tol, &it, &rs, NULL, NULL);
      if (J->iters) J->iters[s] = it;
      if (J->resid) J->resid[s] = rs;
    }
    J->status[s] = st;
    for (int64_t i = 0; i < n; ++i) J->x[off + i * J->elem_stride] = X[i];
  }
  free(buf);
  return NULL;
}

int orc_batch(int method, int k, int64_t nsys, int64_t n, int64_t sys_stride, int64_t elem_stride,
              const int64_t* offsets, const int8_t* hbw, const double* a, const double* b,
              const double* c, const double* d, const double* e, const double* f, double* x,
              int32_t* status, double tol, int max_it, int hb_width, int hb_max_it, double hb_tol,
              int32_t* iters, double* resid, int nthreads) {
  if (nsys < 0 || nthreads < 1) return ORC_ARG;
  if (nthreads > 256) nthreads = 256;
  if (nthreads > nsys) nthreads = nsys > 0 ? (int)nsys : 1;
  batch_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    batch_job J = {method, k, nsys, n, sys_stride, elem_stride, offsets, hbw, a, b, c, d, e, f, x,
                   status, tol, max_it, hb_width, hb_max_it, hb_tol, iters, resid,
                   nsys * t / nthreads, nsys * (t + 1) / nthreads};
    jobs[t] = J;
  }
  if (nthreads == 1) { batch_worker(&jobs[0]); return ORC_OK; }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  return ORC_OK;
}
