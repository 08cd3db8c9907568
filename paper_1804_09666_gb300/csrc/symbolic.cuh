// symbolic.cuh -- the STDM / SPDM fix-up: a system whose numeric sweep met a pivot
// that is exactly zero is solved again in truncated Laurent series in one symbol t
// (Veneva & Ayriyan, arXiv:1804.09666, Sec. 1: the symbolic methods need only a
// nonsingular matrix; Sec. 3.2 Remark 1: the determinant in O(N)).
//
// Replacing a zero pivot mu_j by t is replacing c_j by c_j + t (plus terms of higher
// order in t), so the sweep is the exact LU factorisation of a matrix A(t) -> A, and
// x(t) = A(t)^{-1} f -> A^{-1} f as t -> 0 whenever A is nonsingular.
//
// One warp per system.  Lane l holds the coefficient of t^(l - kZ) of a series, so a
// series spans t^-15 .. t^16, and every coefficient is a double-double number
// (Dekker 1971: an unevaluated sum hi + lo, sums by Knuth's two-sum, products by one
// fused multiply-add).  A series is known for exponents below `hi` (warp-uniform);
// `v` and `top` are its lowest and highest nonzero known exponents.  A coefficient
// formed as a sum of terms whose result lies below 2^-80 of the terms' total
// magnitude is set to zero: in exact arithmetic it is zero, and what double-double
// leaves of it is rounding residue (~2^-104 of the terms), which would otherwise pass
// for a nonzero leading coefficient.
//
// Readings (the paper is silent on the arithmetic of its symbolic methods):
//  * one symbol stands for every pivot whose known coefficients are all zero, and
//    that pivot becomes exactly t; a pivot whose t^0 coefficient is not known
//    (hi < 1) cannot be decided and ends the attempt (SYMBOLIC_RANGE);
//  * x(t) is analytic at t = 0 for nonsingular A, so the negative powers of every x_i
//    are rounding residue and are cleared; x_i is its t^0 coefficient;
//  * det A = lim prod mu_i(t): V = sum of the pivots' valuations; V > 0 -> det A = 0
//    (SINGULAR), V = 0 -> the product of the leading coefficients, V < 0 is impossible
//    in exact arithmetic (SYMBOLIC_RANGE);
//  * a pole deeper than t^-15, or an x_i whose t^0 coefficient is not known, is
//    SYMBOLIC_RANGE.
// The positive extent E of the window is chosen per attempt: a first pass keeps
// t^-15 .. t^3 (enough for a single zero pivot: its x needs t^1, and on PD rows the
// known range loses two orders through the pole rows' products), and a system that
// runs out of window there is solved again with t^16.  Truncation changes only
// which coefficients are known, never their values, so the first pass can end in
// SYMBOLIC_RANGE where the second does not, but not in a different result.
#pragma once
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace band {
namespace lser {

constexpr int kZ = 15;                 // lane l: coefficient of t^(l - kZ)
constexpr int kMaxE = 31 - kZ;         // 16: the highest exponent a lane holds
constexpr int kNone = 1 << 20;         // valuation of a series without a nonzero coefficient
constexpr unsigned kAll = 0xffffffffu;
constexpr double kResidue = 0x1p-80;

struct dd {
  double h, l;
};

// s + err = a + b exactly (Knuth)
__device__ __forceinline__ dd two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bv = __dsub_rn(s, a);
  const double av = __dsub_rn(s, bv);
  return dd{s, __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv))};
}
// the same when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  return dd{s, __dsub_rn(b, __dsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.h, -x.l}; }
__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.h, y.h);
  const dd t = two_sum(x.l, y.l);
  s = fast_two_sum(s.h, __dadd_rn(s.l, t.h));
  return fast_two_sum(s.h, __dadd_rn(s.l, t.l));
}
__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  const double p = __dmul_rn(x.h, y.h);
  double e = fma(x.h, y.h, -p);
  e = fma(x.h, y.l, e);
  e = fma(x.l, y.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mul_d(dd x, double s) {
  const double p = __dmul_rn(x.h, s);
  double e = fma(x.h, s, -p);
  e = fma(x.l, s, e);
  return fast_two_sum(p, e);
}
// 1 / y: a double quotient refined by one Newton step carried in double-double,
// r = r0 + r0 (1 - y r0), which squares the relative error of r0 (~2^-53).
__device__ __forceinline__ dd dd_recip(dd y) {
  const double r0 = 1.0 / y.h;
  const dd res = dd_add(dd{1.0, 0.0}, dd_neg(dd_mul_d(y, r0)));
  return fast_two_sum(r0, __dmul_rn(r0, res.h));
}
__device__ __forceinline__ bool dd_zero(dd x) { return x.h == 0.0; }

// A running sum of products in the compensated form of Ogita, Rump and Oishi
// ("Accurate sum and dot product", 2005): s collects the rounded terms exactly through
// two-sum, c their errors; mag the terms' total magnitude for the residue test.
struct Acc {
  double s, c, mag;
};
__device__ __forceinline__ Acc acc_of(dd x) { return Acc{x.h, x.l, fabs(x.h)}; }
// acc += sign * x * y
__device__ __forceinline__ void acc_fma(Acc& a, dd x, dd y, double sign) {
  const double p = __dmul_rn(x.h, y.h);
  double pe = fma(x.h, y.h, -p);
  pe = fma(x.h, y.l, pe);
  pe = fma(x.l, y.h, pe);
  const dd t = two_sum(a.s, sign * p);
  a.s = t.h;
  a.c = __dadd_rn(a.c, fma(sign, pe, t.l));
  a.mag = __dadd_rn(a.mag, fabs(p));
}
__device__ __forceinline__ dd acc_value(const Acc& a) {
  const dd v = two_sum(a.s, a.c);
  if (fabs(v.h) <= kResidue * a.mag) return dd{0.0, 0.0};
  return v;
}

// One series, one coefficient per lane; hi, v, top are the same in every lane.
struct Ser {
  dd q;
  int hi, v, top;
};

__device__ __forceinline__ int lane_exp() { return (int)(threadIdx.x & 31) - kZ; }

// v and top from the known nonzero coefficients
__device__ __forceinline__ void set_meta(Ser& s) {
  const int e = lane_exp();
  if (e >= s.hi) s.q = dd{0.0, 0.0};
  const unsigned m = __ballot_sync(kAll, !dd_zero(s.q));
  s.v = m ? (__ffs((int)m) - 1 - kZ) : kNone;
  s.top = m ? (31 - __clz((int)m) - kZ) : -kNone;
}
__device__ __forceinline__ int veff(const Ser& s) { return s.v != kNone ? s.v : s.hi; }

__device__ __forceinline__ Ser constant(double x, int E) {
  Ser r;
  r.q = dd{lane_exp() == 0 ? x : 0.0, 0.0};
  r.hi = E + 1;
  const bool nz = x != 0.0;   // NaN counts as nonzero
  r.v = nz ? 0 : kNone;
  r.top = nz ? 0 : -kNone;
  return r;
}
__device__ __forceinline__ Ser symbol(int E) {
  Ser r;
  r.q = dd{lane_exp() == 1 ? 1.0 : 0.0, 0.0};
  r.hi = E + 1;
  r.v = 1;
  r.top = 1;
  return r;
}

// x - y
__device__ __forceinline__ Ser sub(const Ser& x, const Ser& y) {
  Ser r;
  r.hi = min(x.hi, y.hi);
  const dd d = dd_add(x.q, dd_neg(y.q));
  r.q = fabs(d.h) <= kResidue * (fabs(x.q.h) + fabs(y.q.h)) ? dd{0.0, 0.0} : d;
  set_meta(r);
  return r;
}

// x - y * s for a plain number s (a series known to t^E): the product is known below
// min(E + 1, veff(y) + E + 1, veff(s) + y.hi)
__device__ __forceinline__ Ser sub_scaled(const Ser& x, const Ser& y, double s, int E) {
  const int vs = (s != 0.0) ? 0 : E + 1;
  Ser p;
  p.hi = min(E + 1, min(veff(y) + E + 1, vs + y.hi));
  p.q = dd_mul_d(y.q, s);
  set_meta(p);
  return sub(x, p);
}

// x * y; known below min(veff(x) + y.hi, veff(y) + x.hi), so every kept coefficient
// has all its terms.  sx, sy: this warp's staging rows (32 coefficients each).
__device__ __forceinline__ Ser mul(const Ser& x, const Ser& y, int E, bool& err, dd* sx, dd* sy) {
  Ser r;
  r.hi = min(E + 1, min(veff(x) + y.hi, veff(y) + x.hi));
  r.q = dd{0.0, 0.0};
  if (x.v == kNone || y.v == kNone) {
    set_meta(r);
    return r;
  }
  if (x.v + y.v < -kZ) err = true;        // a pole deeper than the window
  const int lane = (int)(threadIdx.x & 31), e = lane - kZ;
  // the loop runs over the operand with fewer nonzero coefficients
  const bool swap = (x.top - x.v) > (y.top - y.v);
  const Ser& u = swap ? y : x;
  const Ser& w = swap ? x : y;
  sx[lane] = u.q;
  sy[lane] = w.q;
  __syncwarp();
  Acc a{0.0, 0.0, 0.0};
  const bool live = e < r.hi;
  for (int i = u.v; i <= u.top; ++i) {
    const int j = e - i;
    if (live && j >= w.v && j <= w.top) acc_fma(a, sx[i + kZ], sy[j + kZ], 1.0);
  }
  __syncwarp();
  r.q = live ? acc_value(a) : dd{0.0, 0.0};
  set_meta(r);
  return r;
}

// The quotients n_k / m (k = 1, 2, 3; a numerator with use_k false is skipped) by long
// division: with vm = m.v, the quotient's coefficient of t^k is
//   (n_{k+vm} - sum_{j>=1} m_{vm+j} c_{k-j}) / m_vm,
// known below v + min(n.hi - n.v, m.hi - vm) (v = n.v - vm).  The three divisions share
// the divisor and run interleaved; every finished coefficient is broadcast and pushed
// into the sums of the higher ones.  A divisor with one nonzero coefficient (m.top =
// vm, e.g. a constant) pushes nothing, so c_k = n_{k+vm} / m_vm is zero beyond n.top:
// those steps are skipped (their coefficients stay the exact zeros they would get).
// sm, s1, s2, s3: staging rows.
__device__ __forceinline__ void div3(const Ser* num, const bool* use, const Ser& m, Ser* out,
                                     int E, bool& err, dd* sm, dd* s1, dd* s2, dd* s3) {
  const int lane = (int)(threadIdx.x & 31), e = lane - kZ;
  dd* sn[3] = {s1, s2, s3};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[k].q = dd{0.0, 0.0};
    out[k].hi = E + 1;
  }
  if (m.v == kNone) {      // the divisor is not known to be nonzero
    err = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      out[k].hi = -kZ;
      set_meta(out[k]);
    }
    return;
  }
  const int vm = m.v;
  sm[lane] = m.q;
#pragma unroll
  for (int k = 0; k < 3; ++k) sn[k][lane] = num[k].q;
  __syncwarp();
  const dd inv = dd_recip(sm[vm + kZ]);
  int v[3], hi[3], lim[3];
  bool act[3];
  Acc acc[3];
  int steps = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    act[k] = false;
    v[k] = 0;
    lim[k] = 0;
    hi[k] = E + 1;
    acc[k] = Acc{0.0, 0.0, 0.0};
    if (!use[k]) continue;
    if (num[k].v == kNone) {
      hi[k] = min(E + 1, num[k].hi - vm);
      continue;
    }
    v[k] = num[k].v - vm;
    hi[k] = min(E + 1, v[k] + min(num[k].hi - num[k].v, m.hi - vm));
    if (v[k] < -kZ) {
      err = true;
      continue;
    }
    act[k] = true;
    if (e >= v[k] && e < hi[k]) acc[k] = acc_of(sn[k][e + vm + kZ]);
    lim[k] = hi[k] - v[k];
    if (m.top == vm) lim[k] = min(lim[k], num[k].top - num[k].v + 1);
    steps = max(steps, lim[k]);
  }
  for (int st = 0; st < steps; ++st) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!act[k] || st >= lim[k]) continue;
      const int ek = v[k] + st;                  // the exponent finished in this step
      const dd mine = dd_mul(acc_value(acc[k]), inv);
      dd c;
      c.h = __shfl_sync(kAll, mine.h, ek + kZ);
      c.l = __shfl_sync(kAll, mine.l, ek + kZ);
      if (e == ek) out[k].q = c;
      const int j = e - ek;
      if (j >= 1 && e < hi[k] && vm + j <= m.top) acc_fma(acc[k], sm[vm + j + kZ], c, -1.0);
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    out[k].hi = hi[k];
    set_meta(out[k]);
  }
}

// Series rows of one flagged system in the slot memory: 3 kinds (alpha, beta, z) x
// nmax rows x 32 coefficients, then 3 x nmax (hi, v, top) records.
struct SlotView {
  dd* coef;
  int4* meta;
  int64_t nmax;
  __device__ __forceinline__ void put(int kind, int64_t i, const Ser& s) const {
    coef[((int64_t)kind * nmax + i) * 32 + (threadIdx.x & 31)] = s.q;
    if ((threadIdx.x & 31) == 0) meta[(int64_t)kind * nmax + i] = make_int4(s.hi, s.v, s.top, 0);
  }
  __device__ __forceinline__ Ser get(int kind, int64_t i) const {
    Ser s;
    s.q = coef[((int64_t)kind * nmax + i) * 32 + (threadIdx.x & 31)];
    const int4 m = meta[(int64_t)kind * nmax + i];
    s.hi = m.x;
    s.v = m.y;
    s.top = m.z;
    return s;
  }
};

__host__ __device__ constexpr size_t slot_bytes(int64_t nmax) {
  return (size_t)3 * (size_t)nmax * (32 * sizeof(dd) + sizeof(int4));
}

// slot `slot` of the fix-up's series memory
__device__ __forceinline__ SlotView slot_view(const SymArgs& p, int64_t slot) {
  unsigned char* base = static_cast<unsigned char*>(p.slot_mem) + slot * slot_bytes(p.nmax);
  return SlotView{reinterpret_cast<dd*>(base),
                  reinterpret_cast<int4*>(base + (size_t)3 * p.nmax * 32 * sizeof(dd)), p.nmax};
}

struct Outcome {
  int32_t status;
  int V;
  double mant;
  long long ex;
};

// One attempt with positive extent E on system s (rows n, half bandwidth K).
__device__ inline Outcome solve_attempt(const SymArgs& p, int64_t s, int E, const SlotView& sv,
                                        dd* stage) {
  const int64_t n = p.L.rows(s);
  const int K = p.L.kband(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const bool want_x = !p.det_only;
  dd *s0 = stage, *s1 = stage + 32, *s2 = stage + 64, *s3 = stage + 96;
  bool err = false;
  Outcome o{BAND_OK, 0, 1.0, 0};
  Ser al1 = constant(0.0, E), al2 = al1, be1 = al1, be2 = al1, z1 = al1, z2 = al1;
  for (int64_t i = 0; i < n && !err; ++i) {
    const int64_t q = q0 + i * es;
    const double ai = (K == 2 && i >= 2) ? p.a[q] : 0.0;
    Ser g = constant(i >= 1 ? p.b[q] : 0.0, E);
    if (K == 2 && i >= 2) g = sub_scaled(g, al2, ai, E);
    Ser m = constant(p.c[q], E);
    if (K == 2 && i >= 2) m = sub_scaled(m, be2, ai, E);
    if (i >= 1) m = sub(m, mul(al1, g, E, err, s0, s1));
    if (m.v == kNone) {
      if (m.hi < 1) err = true;         // its t^0 coefficient is unknown
      m = symbol(E);
    }
    {
      const double lead = __shfl_sync(kAll, m.q.h, (m.v + kZ) & 31);
      o.V += m.v;
      int e2;
      o.mant *= frexp(lead, &e2);
      o.ex += e2;
      int e3;
      o.mant = frexp(o.mant, &e3);
      o.ex += e3;
    }
    Ser num[3];
    bool use[3];
    num[0] = constant(0.0, E);
    use[0] = i + 1 < n;
    if (use[0]) {
      num[0] = constant(p.d[q], E);
      if (K == 2 && i >= 1) num[0] = sub(num[0], mul(be1, g, E, err, s0, s1));
    }
    use[1] = K == 2 && i + 2 < n;
    num[1] = constant(use[1] ? p.e[q] : 0.0, E);
    use[2] = want_x;
    num[2] = constant(0.0, E);
    if (want_x) {
      num[2] = constant(p.f[q], E);
      if (K == 2 && i >= 2) num[2] = sub_scaled(num[2], z2, ai, E);
      if (i >= 1) num[2] = sub(num[2], mul(z1, g, E, err, s0, s1));
    }
    Ser r[3];
    div3(num, use, m, r, E, err, s0, s1, s2, s3);
    if (!use[0]) r[0] = constant(0.0, E);
    if (!use[1]) r[1] = constant(0.0, E);
    if (want_x) {
      sv.put(0, i, r[0]);
      sv.put(1, i, r[1]);
      sv.put(2, i, r[2]);
    }
    al2 = al1; al1 = r[0];
    be2 = be1; be1 = r[1];
    z2 = z1; z1 = r[2];
  }
  if (!err && want_x) {
    __syncwarp();
    Ser x1 = constant(0.0, E), x2 = x1;
    bool bad = false;
    for (int64_t i = n - 1; i >= 0 && !err; --i) {
      Ser xi = sv.get(2, i);
      if (i + 1 < n) xi = sub(xi, mul(sv.get(0, i), x1, E, err, s0, s1));
      if (K == 2 && i + 2 < n) xi = sub(xi, mul(sv.get(1, i), x2, E, err, s0, s1));
      if (lane_exp() < 0) xi.q = dd{0.0, 0.0};
      set_meta(xi);
      if (xi.hi <= 0) err = true;
      const double xv = __shfl_sync(kAll, xi.q.h, kZ);
      if ((threadIdx.x & 31) == 0) p.x[q0 + i * es] = xv;
      bad |= !isfinite(xv);
      x2 = x1;
      x1 = xi;
    }
    if (bad) o.status = BAND_ERR_NONFINITE;
  }
  // An attempt that ran out of window stops at that row, so its V is a partial sum and
  // says nothing about the determinant: it ends in SYMBOLIC_RANGE (and the wider
  // window is tried).
  if (err || o.V < 0) o.status = BAND_ERR_SYMBOLIC_RANGE;
  else if (o.V > 0) o.status = BAND_ERR_SINGULAR;
  return o;
}

// The fix-up of the batch's t-th system by one warp: a pass with t^3, and one with
// t^16 if that ran out of window.
constexpr int kFirstE = 3;
__device__ inline void symbolic_warp(const SymArgs& p, int64_t t, const SlotView& sv, dd* stage) {
  const int64_t s = p.L.sys(t);
  Outcome o = solve_attempt(p, s, kFirstE, sv, stage);
  if (o.status == BAND_ERR_SYMBOLIC_RANGE) o = solve_attempt(p, s, kMaxE, sv, stage);
  if ((threadIdx.x & 31) == 0) {
    set_status(p.status, s, o.status);
    if (p.det_mant) {
      const bool ok = o.status == BAND_OK || o.status == BAND_ERR_NONFINITE;
      p.det_mant[s] = ok && o.V == 0 ? o.mant : 0.0;
      p.det_exp[s] = ok && o.V == 0 ? o.ex : 0;
    }
  }
}

}  // namespace lser
}  // namespace band
