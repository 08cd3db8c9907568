// direct.cu -- NTDM / NPDM (LU without pivoting) and STDM / SPDM (symbolic zero
// pivots) for batches of independent band systems, one thread per system.
//
// Veneva & Ayriyan, arXiv:1804.09666: the direct numerical methods NPDM/NTDM and
// the symbolic methods SPDM/STDM (Sec. 1; costs in Table 7).  The PD recurrence,
// with U unit upper and every quantity with a negative index zero:
//   gamma_i = b_i - alpha_{i-2} a_i
//   mu_i    = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i
//   alpha_i = (d_i - beta_{i-1} gamma_i) / mu_i,   beta_i = e_i / mu_i
//   z_i     = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i
//   x_i     = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
// (TD: a = e = 0).  Each mu_i is inverted once and used by multiplication.  The
// forward sweep keeps alpha, beta in the workspace (interleaved by system) and z in
// x (numeric methods) or in the workspace too (symbolic methods, so that a system
// handed to the fix-up pass still has an intact f when x aliases f); the backward
// sweep writes x.
#include "common.cuh"
#include "kernels.h"

namespace band {

// ---------------------------------------------------------------------------
// fused factor + solve
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void direct_one(const DirectArgs<T>& p, int64_t s) {
  const int64_t n = p.L.rows(s);
  if (n <= 0) {
    set_status(p.status, s, BAND_OK);
    return;
  }
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), wst = p.W.stride();
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
  bool zero = false;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T bi = ldro(p.b + q);
    const T ci = ldro(p.c + q);
    T di = ldro(p.d + q);
    const T fi = p.f[q];
    bi = (i >= 1) ? bi : T(0);
    di = (i + 1 < n) ? di : T(0);
    if (K == 2) {
      T ai = ldro(p.a + q), ei = ldro(p.e + q);
      ai = (i >= 2) ? ai : T(0);
      ei = (i + 2 < n) ? ei : T(0);
      const T g = fma(-al2, ai, bi);
      const T m = fma(-al1, g, fma(-be2, ai, ci));
      if (m == T(0)) { zero = true; break; }
      const T r = rcp<T>(m);
      const T alv = fma(-be1, g, di) * r;
      const T bev = ei * r;
      const T zv = fma(-z1, g, fma(-z2, ai, fi)) * r;
      p.al[w] = alv;
      p.be[w] = bev;
      if (p.zs) p.zs[w] = zv; else p.x[q] = zv;
      al2 = al1; al1 = alv; be2 = be1; be1 = bev; z2 = z1; z1 = zv;
    } else {
      const T m = fma(-al1, bi, ci);
      if (m == T(0)) { zero = true; break; }
      const T r = rcp<T>(m);
      const T alv = di * r;
      const T zv = fma(-z1, bi, fi) * r;
      p.al[w] = alv;
      if (p.zs) p.zs[w] = zv; else p.x[q] = zv;
      al1 = alv; z1 = zv;
    }
  }
  if (zero) {
    if (p.fix_list) {  // symbolic method: hand the system to the fix-up pass
      const unsigned long long k = atomicAdd(p.fix_count, 1ull);
      p.fix_list[k] = s;
    } else {
      set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
    }
    return;
  }
  T x1 = 0, x2 = 0;
  bool bad = false;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T xi = fma(-p.al[w], x1, p.zs ? p.zs[w] : p.x[q]);
    if (K == 2) xi = fma(-p.be[w], x2, xi);
    p.x[q] = xi;
    bad |= !finite(xi);
    x2 = x1;
    x1 = xi;
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) k_direct(const DirectArgs<T> p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (K == 0) {
    if (p.L.kband(s) == 1) direct_one<T, 1>(p, s);
    else direct_one<T, 2>(p, s);
  } else {
    direct_one<T, K>(p, s);
  }
}

template <typename T>
cudaError_t launch_direct(const DirectArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 128;
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_direct<T, 1><<<grid, tb, 0, st>>>(p);
  else if (kmode == 2) k_direct<T, 2><<<grid, tb, 0, st>>>(p);
  else k_direct<T, 0><<<grid, tb, 0, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_direct<double>(const DirectArgs<double>&, int, cudaStream_t);
template cudaError_t launch_direct<float>(const DirectArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// factorisation only: gamma, 1/mu, alpha, beta per row (interleaved like the spill)
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void factor_one(const FactorArgs<T>& p, int64_t s) {
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), wst = p.W.stride();
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T bi = ldro(p.b + q);
    const T ci = ldro(p.c + q);
    T di = ldro(p.d + q);
    bi = (i >= 1) ? bi : T(0);
    di = (i + 1 < n) ? di : T(0);
    T ai = 0, ei = 0;
    if (K == 2) {
      ai = ldro(p.a + q);
      ei = ldro(p.e + q);
      ai = (i >= 2) ? ai : T(0);
      ei = (i + 2 < n) ? ei : T(0);
    }
    const T g = fma(-al2, ai, bi);
    const T m = fma(-al1, g, fma(-be2, ai, ci));
    if (m == T(0)) {
      set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
      return;
    }
    const T r = rcp<T>(m);
    const T alv = fma(-be1, g, di) * r;
    const T bev = ei * r;
    p.gam[w] = g;
    p.rmu[w] = r;
    p.al[w] = alv;
    p.be[w] = bev;
    al2 = al1; al1 = alv; be2 = be1; be1 = bev;
  }
  set_status(p.status, s, BAND_OK);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) k_factor(const FactorArgs<T> p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (K == 0) {
    if (p.L.kband(s) == 1) factor_one<T, 1>(p, s);
    else factor_one<T, 2>(p, s);
  } else {
    factor_one<T, K>(p, s);
  }
}

template <typename T>
cudaError_t launch_factor(const FactorArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 128;
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_factor<T, 1><<<grid, tb, 0, st>>>(p);
  else if (kmode == 2) k_factor<T, 2><<<grid, tb, 0, st>>>(p);
  else k_factor<T, 0><<<grid, tb, 0, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_factor<double>(const FactorArgs<double>&, int, cudaStream_t);
template cudaError_t launch_factor<float>(const FactorArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// solve with stored factors: z_i = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i,
// x_i = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void fsolve_one(const FactoredArgs<T>& p, int64_t s) {
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), wst = p.W.stride();
  T z1 = 0, z2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T zz = p.f[q];
    if (K == 2) {
      T ai = ldro(p.a + q);
      ai = (i >= 2) ? ai : T(0);
      zz = fma(-z2, ai, zz);
    }
    const T zv = fma(-z1, ldro(p.gam + w), zz) * ldro(p.rmu + w);
    p.x[q] = zv;
    z2 = z1;
    z1 = zv;
  }
  T x1 = 0, x2 = 0;
  bool bad = false;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t q = q0 + i * es;
    const int64_t w = w0 + i * wst;
    T xi = fma(-ldro(p.al + w), x1, p.x[q]);
    if (K == 2) xi = fma(-ldro(p.be + w), x2, xi);
    p.x[q] = xi;
    bad |= !finite(xi);
    x2 = x1;
    x1 = xi;
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

template <typename T, int K>
__global__ void __launch_bounds__(128) k_fsolve(const FactoredArgs<T> p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  if (K == 0) {
    if (p.L.kband(s) == 1) fsolve_one<T, 1>(p, s);
    else fsolve_one<T, 2>(p, s);
  } else {
    fsolve_one<T, K>(p, s);
  }
}

template <typename T>
cudaError_t launch_fsolve(const FactoredArgs<T>& p, int kmode, cudaStream_t st) {
  if (p.L.nsys == 0) return cudaSuccess;
  const int tb = 128;
  const unsigned grid = (unsigned)((p.L.nsys + tb - 1) / tb);
  if (kmode == 1) k_fsolve<T, 1><<<grid, tb, 0, st>>>(p);
  else if (kmode == 2) k_fsolve<T, 2><<<grid, tb, 0, st>>>(p);
  else k_fsolve<T, 0><<<grid, tb, 0, st>>>(p);
  return cudaGetLastError();
}
template cudaError_t launch_fsolve<double>(const FactoredArgs<double>&, int, cudaStream_t);
template cudaError_t launch_fsolve<float>(const FactoredArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// STDM / SPDM fix-up: the systems whose sweep met an exact zero pivot are redone in
// truncated Laurent arithmetic in one symbol t (every zero pivot becomes t, i.e.
// c_i -> c_i + t, so the sweep is the exact LU of A(t) = A + t sum e_i e_i^T and
// x(t) -> A^{-1} f as t -> 0 when A is nonsingular).  A series holds the
// coefficients of t^-SP .. t^SP and is known for exponents below `hi`.
//   * a pivot with no known nonzero coefficient is a zero pivot and becomes t;
//   * det A = lim prod mu_i(t): V = sum of the pivots' valuations; V > 0 -> det 0
//     (SINGULAR), V = 0 -> product of the leading coefficients, V < 0 impossible in
//     exact arithmetic (SYMBOLIC_RANGE);
//   * x(t) is analytic at 0 for nonsingular A, so the negative powers of each x_i are
//     rounding residue and are cleared; x_i = its t^0 coefficient;
//   * a pole deeper than t^-SP, or an x_i whose t^0 term is unknown, is SYMBOLIC_RANGE.
// ---------------------------------------------------------------------------
struct Ser {
  double q[kSerWidth];
  int hi;
  int pad;
};
constexpr int SP = kSerPole;

__device__ inline Ser ser_const(double v) {
  Ser r;
#pragma unroll
  for (int k = 0; k < kSerWidth; ++k) r.q[k] = 0.0;
  r.q[SP] = v;
  r.hi = SP + 1;
  r.pad = 0;
  return r;
}
__device__ inline Ser ser_symbol() {
  Ser r = ser_const(0.0);
  r.q[SP + 1] = 1.0;
  return r;
}
__device__ inline int ser_val(const Ser& s) {
  for (int k = -SP; k < s.hi && k <= SP; ++k)
    if (s.q[k + SP] != 0.0) return k;
  return SP + 1;
}
__device__ inline int ser_veff(const Ser& s) {
  const int v = ser_val(s);
  return v <= SP ? v : s.hi;
}
__device__ inline Ser ser_sub(const Ser& x, const Ser& y) {
  Ser r = ser_const(0.0);
  r.hi = min(x.hi, y.hi);
  for (int k = -SP; k < r.hi && k <= SP; ++k) r.q[k + SP] = x.q[k + SP] - y.q[k + SP];
  return r;
}
__device__ inline Ser ser_mul(const Ser& x, const Ser& y, bool& err) {
  Ser r = ser_const(0.0);
  const int vx = ser_veff(x), vy = ser_veff(y);
  r.hi = min(SP + 1, min(vx + y.hi, vy + x.hi));
  for (int i = -SP; i < x.hi && i <= SP; ++i) {
    const double xv = x.q[i + SP];
    if (xv == 0.0) continue;
    for (int j = -SP; j < y.hi && j <= SP; ++j) {
      const double pv = xv * y.q[j + SP];
      if (pv == 0.0) continue;
      const int k = i + j;
      if (k >= r.hi) continue;
      if (k < -SP) { err = true; continue; }
      r.q[k + SP] += pv;
    }
  }
  return r;
}
__device__ inline Ser ser_div(const Ser& x, const Ser& y, bool& err) {
  Ser r = ser_const(0.0);
  const int vy = ser_val(y);
  if (vy > SP) { err = true; r.hi = -SP; return r; }
  const int vx = ser_val(x);
  if (vx > SP) { r.hi = min(SP + 1, x.hi - vy); return r; }
  const int v = vx - vy;
  r.hi = min(SP + 1, v + min(x.hi - vx, y.hi - vy));
  if (v < -SP) { err = true; return r; }
  const double inv = 1.0 / y.q[vy + SP];
  for (int k = v; k < r.hi; ++k) {
    double acc = x.q[k + vy + SP];
    for (int j = 1; k - j >= v; ++j) acc -= y.q[vy + j + SP] * r.q[k - j + SP];
    r.q[k + SP] = acc * inv;
  }
  return r;
}

__global__ void __launch_bounds__(64) k_symbolic_fixup(const SymArgs p) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= p.nslots) return;
  const unsigned long long count = *p.fix_count;
  Ser* mem = reinterpret_cast<Ser*>(p.slot_mem) + slot * 3 * p.nmax;
  for (unsigned long long item = slot; item < count; item += p.nslots) {
    const int64_t s = p.fix_list[item];
    const int64_t n = p.L.rows(s);
    const int K = p.L.kband(s);
    const int64_t q0 = p.L.base(s), es = p.L.stride();
    Ser* AL = mem;
    Ser* BE = mem + p.nmax;
    Ser* Z = mem + 2 * p.nmax;
    bool err = false;
    int V = 0;
    double dmant = 1.0;
    long long dexp = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t q = q0 + i * es;
      const Ser ai = ser_const((K == 2 && i >= 2) ? p.a[q] : 0.0);
      Ser g = ser_const(i >= 1 ? p.b[q] : 0.0);
      if (K == 2 && i >= 2) g = ser_sub(g, ser_mul(AL[i - 2], ai, err));
      Ser m = ser_const(p.c[q]);
      if (K == 2 && i >= 2) m = ser_sub(m, ser_mul(BE[i - 2], ai, err));
      if (i >= 1) m = ser_sub(m, ser_mul(AL[i - 1], g, err));
      if (ser_val(m) > SP) m = ser_symbol();
      {
        const int v = ser_val(m);
        V += v;
        int e2;
        dmant *= frexp(m.q[v + SP], &e2);
        dexp += e2;
        int e3;
        dmant = frexp(dmant, &e3);
        dexp += e3;
      }
      Ser al = ser_const(0.0), be = ser_const(0.0);
      if (i + 1 < n) {
        Ser num = ser_const(p.d[q]);
        if (K == 2 && i >= 1) num = ser_sub(num, ser_mul(BE[i - 1], g, err));
        al = ser_div(num, m, err);
      }
      if (K == 2 && i + 2 < n) be = ser_div(ser_const(p.e[q]), m, err);
      Ser zz = ser_const(p.f[q]);
      if (K == 2 && i >= 2) zz = ser_sub(zz, ser_mul(Z[i - 2], ai, err));
      if (i >= 1) zz = ser_sub(zz, ser_mul(Z[i - 1], g, err));
      AL[i] = al;
      BE[i] = be;
      Z[i] = ser_div(zz, m, err);
    }
    Ser x1 = ser_const(0.0), x2 = ser_const(0.0);
    bool bad = false;
    for (int64_t i = n - 1; i >= 0; --i) {
      Ser xi = Z[i];
      if (i + 1 < n) xi = ser_sub(xi, ser_mul(AL[i], x1, err));
      if (K == 2 && i + 2 < n) xi = ser_sub(xi, ser_mul(BE[i], x2, err));
      for (int k = 0; k < SP; ++k) xi.q[k] = 0.0;
      if (xi.hi <= 0) err = true;
      const double xv = xi.q[SP];
      p.x[q0 + i * es] = xv;
      bad |= !isfinite(xv);
      x2 = x1;
      x1 = xi;
    }
    int32_t st = BAND_OK;
    if (V > 0) st = BAND_ERR_SINGULAR;
    else if (err || V < 0) st = BAND_ERR_SYMBOLIC_RANGE;
    else if (bad) st = BAND_ERR_NONFINITE;
    set_status(p.status, s, st);
    if (p.det_mant) {
      p.det_mant[s] = (V == 0) ? dmant : 0.0;
      p.det_exp[s] = (V == 0) ? dexp : 0;
    }
  }
}

cudaError_t launch_symbolic_fixup(const SymArgs& p, cudaStream_t st) {
  if (p.nslots <= 0) return cudaSuccess;
  const int tb = 64;
  k_symbolic_fixup<<<(unsigned)((p.nslots + tb - 1) / tb), tb, 0, st>>>(p);
  return cudaGetLastError();
}

size_t symbolic_slot_bytes(int64_t nmax) { return (size_t)3 * (size_t)nmax * sizeof(Ser); }

}  // namespace band
