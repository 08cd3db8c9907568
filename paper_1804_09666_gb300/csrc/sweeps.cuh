// sweeps.cuh -- per-system sweeps shared by the single-problem and batched kernels.
//
// NTDM / NPDM (Veneva & Ayriyan, arXiv:1804.09666, Sec. 1; Table 7), with U unit upper
// and every quantity with a negative index zero:
//   gamma_i = b_i - alpha_{i-2} a_i
//   mu_i    = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i
//   alpha_i = (d_i - beta_{i-1} gamma_i) / mu_i,   beta_i = e_i / mu_i
//   z_i     = (f_i - z_{i-2} a_i - z_{i-1} gamma_i) / mu_i
//   x_i     = z_i - alpha_i x_{i+1} - beta_i x_{i+2}
// (TD: a = e = 0).  Each mu_i is inverted once (rcp) and used by multiplication.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace band {

template <typename T>
struct RowIn {
  T a, b, c, d, e, f;
};

// Loads of row i of one system; out-of-matrix slots are read but masked later.
template <typename T, int K>
__device__ __forceinline__ void load_in(const DirectArgs<T>& p, int64_t q, RowIn<T>& r) {
  r.b = ldro(p.b + q);
  r.c = ldro(p.c + q);
  r.d = ldro(p.d + q);
  r.f = p.f[q];
  if (K == 2) {
    r.a = ldro(p.a + q);
    r.e = ldro(p.e + q);
  } else {
    r.a = T(0);
    r.e = T(0);
  }
}

// Symbolic methods (STDM / SPDM): a pivot that double arithmetic cannot tell from zero
// goes to the series pass like an exact zero; the series pass, in double-double, decides
// whether it is one.  mu_i = c_i - beta_{i-2} a_i - alpha_{i-1} gamma_i (gamma_i = b_i -
// alpha_{i-2} a_i) is such a pivot when its binary exponent lies 40 or more below that of
// the largest quantity that entered it: a_i, b_i, c_i, beta_{i-2} a_i, alpha_{i-1} gamma_i
// and, for a cancellation inside gamma_i, alpha_{i-1} b_i and alpha_{i-1} alpha_{i-2} a_i (a
// product's exponent taken as the sum of its factors').  On integer-valued systems with
// exact zero pivots, fused multiply-adds leave the rounding error of alpha in place of an
// exact zero far more often than separately rounded operations do.  Integer operations
// only (the FP64 pipe is the scarce unit); TD passes a_i = alpha_{i-2} = beta_{i-2} = 0.
constexpr int kResidueBits = 40;
template <typename T>
__device__ __forceinline__ bool residue_pivot(T, T, T, T, T, T, T, T) { return false; }
template <>
__device__ __forceinline__ bool residue_pivot<double>(double m, double ai, double bi, double ci,
                                                      double al1, double al2, double be2,
                                                      double g) {
  const int ea1 = expo_of(al1) - 1023, ea = expo_of(ai);
  int big = max(max(expo_of(bi), expo_of(ci)), ea);
  big = max(big, ea1 + max(expo_of(g), expo_of(bi)));
  big = max(big, max(expo_of(be2) - 1023 + ea, ea1 + expo_of(al2) - 1023 + ea));
  return expo_of(m) + kResidueBits <= big;
}

// One row of the NPDM / NTDM forward recurrence.  Returns false on a zero pivot (for the
// symbolic methods also on a pivot within rounding residue of zero, residue_pivot).
template <typename T, int K>
__device__ __forceinline__ bool forward_row(const DirectArgs<T>& p, int64_t i, int64_t n,
                                            int64_t q, int64_t w, T ai, T bi, T ci, T di, T ei,
                                            T fi, T& al1, T& al2, T& be1, T& be2, T& z1, T& z2) {
  bi = (i >= 1) ? bi : T(0);
  di = (i + 1 < n) ? di : T(0);
  if (K == 2) {
    ai = (i >= 2) ? ai : T(0);
    ei = (i + 2 < n) ? ei : T(0);
    const T g = fma(-al2, ai, bi);
    const T m = fma(-al1, g, fma(-be2, ai, ci));
    if (is_zero(m)) return false;
    if (p.fix_list && residue_pivot<T>(m, ai, bi, ci, al1, al2, be2, g)) return false;
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
    if (is_zero(m)) return false;
    if (p.fix_list && residue_pivot<T>(m, T(0), bi, ci, al1, T(0), T(0), bi)) return false;
    const T r = rcp<T>(m);
    const T alv = di * r;
    const T zv = fma(-z1, bi, fi) * r;
    p.al[w] = alv;
    if (p.zs) p.zs[w] = zv; else p.x[q] = zv;
    al1 = alv; z1 = zv;
  }
  return true;
}

// One system, one thread: forward sweep (factor + z), then backward sweep (x).  The
// rows of the forward sweep are staged through this warp's shared-memory ring
// (`stage`, stage_bytes_per_warp<T>() bytes) StageDepth<T> rows ahead of their use, so the
// memory latency overlaps the recurrence.  alpha, beta go to the workspace rows; z goes
// to x (numeric methods) or to the workspace (symbolic methods, keeping f intact when
// x aliases f).
template <typename T, int K>
__device__ __forceinline__ void direct_one(const DirectArgs<T>& p, int64_t t, void* stage) {
  const int64_t s = p.L.sys(t);     // t: position in the batch, s: the system id
  if (p.skip && p.skip[s]) return;

  const int64_t n = p.L.rows(s);
  if (n <= 0) {
    set_status(p.status, s, BAND_OK);
    return;
  }
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(t), wst = p.W.stride();
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
  bool zero = false;
  // Interleaved systems (consecutive lanes read consecutive addresses) are staged through
  // the warp's shared-memory ring; other layouts prefetch two rows into registers and
  // lean on L1 for the sectors they share across rows.
  if (stage && !p.L.offsets && p.L.ss == 1) {
    constexpr int D = StageDepth<T>::value;
    constexpr int NA = K == 2 ? 6 : 4;     // arrays staged: (a,) b, c, d, (e,) f
    const RowRing<T, NA, D> ring{static_cast<T*>(stage), (int)(threadIdx.x & 31)};
    const T* src[NA];
    if (K == 2) {
      src[0] = p.a; src[1] = p.b; src[2] = p.c; src[3] = p.d; src[4] = p.e; src[5] = p.f;
    } else {
      src[0] = p.b; src[1] = p.c; src[2] = p.d; src[3] = p.f;
    }
    constexpr int IB = K == 2 ? 1 : 0, IC = IB + 1, ID = IB + 2, IF = NA - 1;
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
      const T ai = K == 2 ? ring.get(slot, 0) : T(0);
      const T ei = K == 2 ? ring.get(slot, 4) : T(0);
      if (!forward_row<T, K>(p, i, n, q0 + i * es, w0 + i * wst, ai, ring.get(slot, IB),
                             ring.get(slot, IC), ring.get(slot, ID), ei, ring.get(slot, IF),
                             al1, al2, be1, be2, z1, z2)) {
        zero = true;
        break;
      }
    }
    cp_async_wait<0>();
  } else {
    RowIn<T> r0, r1, r2;
    load_in<T, K>(p, q0, r0);
    if (n > 1) load_in<T, K>(p, q0 + es, r1);
    for (int64_t i = 0; i < n; ++i) {
      if (i + 2 < n) load_in<T, K>(p, q0 + (i + 2) * es, r2);
      if (!forward_row<T, K>(p, i, n, q0 + i * es, w0 + i * wst, r0.a, r0.b, r0.c, r0.d, r0.e,
                             r0.f, al1, al2, be1, be2, z1, z2)) {
        zero = true;
        break;
      }
      r0 = r1;
      r1 = r2;
    }
  }
  if (zero) {
    if (p.fix_list) {  // symbolic method: hand the system to the fix-up pass
      const unsigned long long k = atomicAdd(p.fix_count, 1ull);
      p.fix_list[k] = t;
    } else {
      set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
    }
    return;
  }
  // backward sweep: its rows carry little arithmetic, so their spill values are loaded
  // in blocks of kBack rows, one memory latency per block
  constexpr int kBack = 8;
  const T* zsrc = p.zs;
  T x1 = 0, x2 = 0;
  bool bad = false;
  for (int64_t top = n - 1; top >= 0; top -= kBack) {
    T av[kBack], bv[kBack], zv[kBack];
#pragma unroll
    for (int j = 0; j < kBack; ++j) {
      const int64_t i = top - j;
      av[j] = bv[j] = zv[j] = T(0);
      if (i >= 0) {
        const int64_t w = w0 + i * wst;
        av[j] = p.al[w];
        if (K == 2) bv[j] = p.be[w];
        zv[j] = zsrc ? zsrc[w] : p.x[q0 + i * es];
      }
    }
#pragma unroll
    for (int j = 0; j < kBack; ++j) {
      const int64_t i = top - j;
      if (i >= 0) {
        T xi = fma(-av[j], x1, zv[j]);
        if (K == 2) xi = fma(-bv[j], x2, xi);
        p.x[q0 + i * es] = xi;
        bad |= not_finite(xi);
        x2 = x1;
        x1 = xi;
      }
    }
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

// The rare path of the two-sided schedule, kept out of line so that it costs its
// caller no registers.
template <typename T, int K>
__device__ __noinline__ void direct_redo(const DirectArgs<T>& p, int64_t t) {

  direct_one<T, K>(p, t, nullptr);
}

// ---------------------------------------------------------------------------
// Two-sided schedule (two lanes per system, lanes l and l ^ 16 of a warp).  The top
// lane runs the NPDM/NTDM recurrence on rows 0 .. m-1 (exactly NPDM's operations on
// those rows); the bottom lane runs the same recurrence on the reversed system, from
// row n-1 up to row m, where row i's diagonals (a, b, c, d, e) read as (e, d, c, b, a)
// -- the UL factorisation of the bottom block.  Their last two eliminated rows
//   top:     x_i + alpha_i x_{i+1} + beta_i x_{i+2} = z_i          (i = m-2, m-1)
//   bottom:  x_i + alpha'_i x_{i-1} + beta'_i x_{i-2} = z'_i       (i = m, m+1)
// are four equations in x_{m-2} .. x_{m+1} only (two in x_{m-1}, x_m for TD), solved
// by both lanes with partial pivoting after exchanging them by shuffles; then each
// lane back-substitutes its half.  Every chain of dependent rows is half as long and
// the launch has twice the threads; the arithmetic is NPDM's apart from the mirrored
// bottom block and the small interface solve.  Needs n >= 4 (PD) or n >= 2 (TD); a
// system with fewer rows is solved by the top lane alone.  For STDM / SPDM, z goes to
// the workspace (f stays intact) and a system with a zero pivot goes to the fix-up.
// ---------------------------------------------------------------------------
template <typename T, int K>
__device__ __forceinline__ void twisted_one(const DirectArgs<T>& p, int64_t t, bool active,
                                            void* stage) {
  const int64_t s = active ? p.L.sys(t) : 0;   // t: position in the batch, s: system id
  if (active && p.skip && p.skip[s]) active = false;   // every lane still reaches the shuffles

  const int lane = (int)(threadIdx.x & 31);
  const bool bottom = lane >= 16;
  const int64_t n = active ? p.L.rows(s) : 0;
  const bool split = n >= (K == 2 ? 4 : 2);
  const int64_t m = (n + 1) / 2;                       // top rows 0 .. m-1
  const int64_t q0 = active ? p.L.base(s) : 0, es = active ? p.L.stride() : 0;
  const int64_t w0 = active ? p.W.base(t) : 0, wst = active ? p.W.stride() : 0;
  // ---- elimination of this lane's block (the mirrored recurrence for the bottom)
  const int64_t rows = !active ? 0 : (!split ? (bottom ? 0 : n) : (bottom ? n - m : m));
  const int dir = bottom ? -1 : 1;
  const int64_t first = bottom ? n - 1 : 0;
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
  bool zero = false;
  if (stage && !p.L.offsets && p.L.ss == 1) {
    // interleaved systems: rows staged through the warp's shared-memory ring as in
    // direct_one; each lane copies the rows of its own sweep
    constexpr int D = StageDepth<T>::value;
    constexpr int NA = K == 2 ? 6 : 4;
    const RowRing<T, NA, D> ring{static_cast<T*>(stage), (int)(threadIdx.x & 31)};
    const T* src[NA];
    if (K == 2) {
      src[0] = p.a; src[1] = p.b; src[2] = p.c; src[3] = p.d; src[4] = p.e; src[5] = p.f;
    } else {
      src[0] = p.b; src[1] = p.c; src[2] = p.d; src[3] = p.f;
    }
    constexpr int IB = K == 2 ? 1 : 0, IC = IB + 1, ID = IB + 2, IF = NA - 1;
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      if (j < rows) ring.issue(j, src, q0 + (first + dir * j) * es);
      else ring.skip();
    }
    for (int64_t j = 0; j < rows; ++j) {
      const int64_t jp = j + D - 1;
      if (jp < rows) ring.issue((int)(jp & (D - 1)), src, q0 + (first + dir * jp) * es);
      else ring.skip();
      cp_async_wait<D - 1>();
      const int slot = (int)(j & (D - 1));
      T ai = K == 2 ? ring.get(slot, 0) : T(0);
      T bi = ring.get(slot, IB);
      T di = ring.get(slot, ID);
      T ei = K == 2 ? ring.get(slot, 4) : T(0);
      if (bottom) {                                  // reversed system
        const T ta = ai, tb = bi;
        ai = ei; bi = di; di = tb; ei = ta;
      }
      const int64_t i = first + dir * j;
      if (!forward_row<T, K>(p, j, n, q0 + i * es, w0 + i * wst, ai, bi, ring.get(slot, IC), di,
                             ei, ring.get(slot, IF), al1, al2, be1, be2, z1, z2)) {
        zero = true;
        break;
      }
    }
    cp_async_wait<0>();
  } else if (stage && p.gran) {
    // each lane walks its own contiguous system: 16-byte granules staged ahead
    constexpr int D = GranDepth<T>::value;
    constexpr int NA = K == 2 ? 6 : 4;
    constexpr int E = GranRing<T, NA, D>::E;
    const GranRing<T, NA, D> ring{static_cast<T*>(stage), (int)(threadIdx.x & 31)};
    const T* src[NA];
    if (K == 2) {
      src[0] = p.a; src[1] = p.b; src[2] = p.c; src[3] = p.d; src[4] = p.e; src[5] = p.f;
    } else {
      src[0] = p.b; src[1] = p.c; src[2] = p.d; src[3] = p.f;
    }
    constexpr int IB = K == 2 ? 1 : 0, IC = IB + 1, ID = IB + 2, IF = NA - 1;
    // element of row j of this sweep: e0 + dir * j (stride 1); its granule e / E
    const int64_t e0 = q0 + first;
    const int64_t g0 = e0 / E;
    const int64_t ng = rows > 0 ? (dir > 0 ? (e0 + rows - 1) / E - g0 + 1 : g0 - (e0 - rows + 1) / E + 1) : 0;
#pragma unroll
    for (int k = 0; k < D - 1; ++k) {
      if (k < ng) ring.issue(k, src, g0 + dir * k, p.L.extent);
      else cp_async_commit();
    }
    int64_t gk = -1;                       // visit index of the granule of row j
    for (int64_t j = 0; j < rows; ++j) {
      const int64_t e = e0 + dir * j;
      const int off = (int)(e % E);
      if (j == 0 || off == (dir > 0 ? 0 : E - 1)) {     // entering the next granule
        ++gk;
        const int64_t kn = gk + D - 1;
        if (kn < ng) ring.issue((int)(kn & (D - 1)), src, g0 + dir * kn, p.L.extent);
        else cp_async_commit();
        cp_async_wait<D - 1>();
      }
      const int slot = (int)(gk & (D - 1));
      T ai = K == 2 ? ring.get(slot, 0, off) : T(0);
      T bi = ring.get(slot, IB, off);
      T di = ring.get(slot, ID, off);
      T ei = K == 2 ? ring.get(slot, 4, off) : T(0);
      if (bottom) {                                  // reversed system
        const T ta = ai, tb = bi;
        ai = ei; bi = di; di = tb; ei = ta;
      }
      const int64_t i = first + dir * j;
      if (!forward_row<T, K>(p, j, n, q0 + i * es, w0 + i * wst, ai, bi, ring.get(slot, IC, off),
                             di, ei, ring.get(slot, IF, off), al1, al2, be1, be2, z1, z2)) {
        zero = true;
        break;
      }
    }
    cp_async_wait<0>();
  } else {
    RowIn<T> r0, r1, r2;
    auto load = [&](int64_t j, RowIn<T>& r) {       // j-th row of this lane's sweep
      const int64_t i = first + dir * j;
      load_in<T, K>(p, q0 + i * es, r);
      if (bottom) {                                  // reversed system: (a,b,c,d,e) -> (e,d,c,b,a)
        const T ta = r.a, tb = r.b;
        r.a = r.e; r.b = r.d; r.d = tb; r.e = ta;
      }
    };
    if (rows > 0) load(0, r0);
    if (rows > 1) load(1, r1);
    for (int64_t j = 0; j < rows; ++j) {
      if (j + 2 < rows) load(j + 2, r2);
      const int64_t i = first + dir * j;
      // masks of the (reversed) system of n rows are NPDM's masks at position j
      if (!forward_row<T, K>(p, j, n, q0 + i * es, w0 + i * wst, r0.a, r0.b, r0.c, r0.d, r0.e,
                             r0.f, al1, al2, be1, be2, z1, z2)) {
        zero = true;
        break;
      }
      r0 = r1;
      r1 = r2;
    }
  }
  // ---- interface: exchange the last two eliminated rows of each half.  Every lane of
  // the warp reaches both exchanges (no return in between).
  const unsigned full = 0xffffffffu;
  const T o_al1 = __shfl_xor_sync(full, al1, 16), o_al2 = __shfl_xor_sync(full, al2, 16);
  const T o_be1 = __shfl_xor_sync(full, be1, 16), o_be2 = __shfl_xor_sync(full, be2, 16);
  const T o_z1 = __shfl_xor_sync(full, z1, 16), o_z2 = __shfl_xor_sync(full, z2, 16);
  const bool o_zero = __shfl_xor_sync(full, (int)zero, 16) != 0;
  __syncwarp();           // the halves' stores are visible to the whole warp from here
  bool fail = zero || (split && o_zero);
  // nx1, nx2: the solved neighbours of the first row this lane back-substitutes
  // (top: x_{i+1}, x_{i+2}; bottom: x_{i-1}, x_{i-2})
  T nx1 = 0, nx2 = 0;
  if (active && split && !fail) {
    // top rows m-2 (al2, be2, z2) and m-1 (al1, be1, z1); bottom rows m+1 and m
    const T tal2 = bottom ? o_al2 : al2, tbe2 = bottom ? o_be2 : be2, tz2 = bottom ? o_z2 : z2;
    const T tal1 = bottom ? o_al1 : al1, tbe1 = bottom ? o_be1 : be1, tz1 = bottom ? o_z1 : z1;
    const T bal2 = bottom ? al2 : o_al2, bbe2 = bottom ? be2 : o_be2, bz2 = bottom ? z2 : o_z2;
    const T bal1 = bottom ? al1 : o_al1, bbe1 = bottom ? be1 : o_be1, bz1 = bottom ? z1 : o_z1;
    T M[4][5];
    if (K == 2) {   // unknowns x_{m-2}, x_{m-1}, x_m, x_{m+1}
      M[0][0] = 1;    M[0][1] = tal2; M[0][2] = tbe2; M[0][3] = 0;    M[0][4] = tz2;
      M[1][0] = 0;    M[1][1] = 1;    M[1][2] = tal1; M[1][3] = tbe1; M[1][4] = tz1;
      M[2][0] = bbe1; M[2][1] = bal1; M[2][2] = 1;    M[2][3] = 0;    M[2][4] = bz1;
      M[3][0] = 0;    M[3][1] = bbe2; M[3][2] = bal2; M[3][3] = 1;    M[3][4] = bz2;
    } else {        // unknowns x_{m-1}, x_m (right-hand side in column 2)
      M[0][0] = 1;    M[0][1] = tal1; M[0][2] = tz1;
      M[1][0] = bal1; M[1][1] = 1;    M[1][2] = bz1;
    }
    // symbolic methods: an interface pivot within rounding residue of zero counts as
    // zero (the system goes to the series pass, as for residue_pivot)
    if (!solve_small<T, K == 2 ? 4 : 2>(M, p.fix_list ? kResidueBits : 0)) {
      fail = true;
    } else if (K == 2) {
      const T xm2 = M[0][4], xm1 = M[1][4], xm0 = M[2][4], xp1 = M[3][4];
      if (!bottom) {
        p.x[q0 + (m - 2) * es] = xm2;
        p.x[q0 + (m - 1) * es] = xm1;
        nx1 = xm2; nx2 = xm1;            // row m-3 needs x_{m-2}, x_{m-1}
      } else {
        p.x[q0 + m * es] = xm0;
        p.x[q0 + (m + 1) * es] = xp1;
        nx1 = xp1; nx2 = xm0;            // row m+2 needs x_{m+1}, x_m
      }
    } else {
      const T xm1 = M[0][2], xm0 = M[1][2];
      if (!bottom) { p.x[q0 + (m - 1) * es] = xm1; nx1 = xm1; }
      else { p.x[q0 + m * es] = xm0; nx1 = xm0; }
    }
  }
  // ---- back-substitution of this lane's block, away from the interface
  int64_t cnt = 0, start = 0;
  if (active && !fail) {
    if (!split) { cnt = bottom ? 0 : n; start = n - 1; }
    else if (K == 2) { cnt = bottom ? n - m - 2 : m - 2; start = bottom ? m + 2 : m - 3; }
    else { cnt = bottom ? n - m - 1 : m - 1; start = bottom ? m + 1 : m - 2; }
  }
  const int bdir = bottom ? 1 : -1;
  bool bad = (active && split && !fail) && (not_finite(nx1) || not_finite(nx2));
  // blocks of kBack rows: their spill values are loaded together, one latency a block
  constexpr int kBack = 8;
  for (int64_t k0 = 0; k0 < cnt; k0 += kBack) {
    T av[kBack], bv[kBack], zv[kBack];
#pragma unroll
    for (int j = 0; j < kBack; ++j) {
      av[j] = bv[j] = zv[j] = T(0);
      if (k0 + j < cnt) {
        const int64_t i = start + bdir * (k0 + j);
        const int64_t w = w0 + i * wst;
        av[j] = p.al[w];
        if (K == 2) bv[j] = p.be[w];
        zv[j] = p.zs ? p.zs[w] : p.x[q0 + i * es];
      }
    }
#pragma unroll
    for (int j = 0; j < kBack; ++j) {
      if (k0 + j < cnt) {
        const int64_t i = start + bdir * (k0 + j);
        T xi = fma(-av[j], nx1, zv[j]);
        if (K == 2) xi = fma(-bv[j], nx2, xi);
        p.x[q0 + i * es] = xi;
        bad |= not_finite(xi);
        nx2 = nx1;
        nx1 = xi;
      }
    }
  }
  // A zero pivot in either half or a singular interface.  Symbolic methods hand the
  // system to the fix-up pass (which starts again from f).  Numeric methods: the top
  // lane redoes the system with NPDM in one thread (f is still intact unless x aliases
  // it), so ZERO_PIVOT is reported exactly when NPDM's own order meets one.
  const bool to_fix = active && !bottom && fail && p.fix_list;
  if (to_fix) {
    const unsigned long long k = atomicAdd(p.fix_count, 1ull);
    p.fix_list[k] = t;
  }
  const bool redo = active && !bottom && split && fail && !p.fix_list && (const T*)p.x != p.f;
  if (redo) direct_redo<T, K>(p, t);
  const bool o_bad = __shfl_xor_sync(full, (int)bad, 16) != 0;
  if (active && !bottom && !redo && !to_fix)
    set_status(p.status, s, fail ? BAND_ERR_ZERO_PIVOT
                                 : ((bad || (split && o_bad)) ? BAND_ERR_NONFINITE : BAND_OK));
}

}  // namespace band
