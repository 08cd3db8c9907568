// partition.cuh -- the partitioned schedule: P lanes per system, lane k eliminating
// chunk k of P consecutive row blocks of its system.  P = 8, 16 or 32 lanes of a warp
// (32 / P systems per warp), or P = 64, 128 or 256: a block of P / 32 warps per system.
//
// Chunk k (rows s0 .. s0+L-1, block A_k of the matrix) couples to the K unknowns just
// above it, u_k = (x_{s0-K} .. x_{s0-1}), through the a, b entries of its first rows
// (the columns B_k), and to the K just below it, v_k = (x_{s0+L} .. x_{s0+L+K-1}),
// through the d, e entries of its last rows (C_k).  Hence
//   x_k = g_k - V_k u_k - W_k v_k,   g = A_k^{-1} f_k,  V = A_k^{-1} B_k,  W = A_k^{-1} C_k.
// Each lane factors its block with the NPDM / NTDM recurrence of Sec. 1 (U unit upper),
// carrying f and B's K columns through the forward sweep (C's columns have entries in
// the last K rows only, so their forward values are formed at the end).  A first
// backward sweep over the five (three for TD) columns keeps only their top and bottom K
// rows: with y_k = (top K rows, bottom K rows) of chunk k, these give the
// block-tridiagonal interface system
//   y_k + L_k y_{k-1} + U_k y_{k+1} = (g_top, g_bottom)_k,
//   L_k y_{k-1} = V_k (bottom K rows of y_{k-1}),   U_k y_{k+1} = W_k (top K rows of y_{k+1}),
// which two lanes solve by block elimination from both ends, meeting in the middle; the
// blocks' structure leaves one K x K solve (partial pivoting) per chunk.  Then each lane
// back-substitutes its chunk once more, with z - z_V u_k - z_W v_k in place of z: x_k.
// Arithmetic per row: about 2.3x NPDM (PD) and 1.8x NTDM (TD); the dependent chain of a
// system is n / P rows long instead of n (one thread) or n / 2 (two-sided).
//
// Scratch (alpha, beta, z of f, z of B's columns) is chunk-major: row j of chunk k of
// the batch's t-th system at ((j * np + t) * P + k), np = nsys rounded up to 32 / P, so
// the lanes of a warp touch consecutive elements.  z of f goes to the zs rows, so f
// stays intact (also when x aliases f) for a redo or the symbolic fix-up.
//
// A chunk may meet a zero (or, see TinyPivot, a tiny) pivot where NPDM's order does
// not, and the interface elimination may meet a singular block: an STDM / SPDM system
// then goes to the symbolic fix-up, and an NTDM / NPDM system is redone by its first
// lane with NPDM alone (so BAND_ERR_ZERO_PIVOT keeps its meaning).  Systems with fewer than 8 P rows are solved by
// their first lane with NPDM.
#pragma once
#include "common.cuh"
#include "kernels.h"
#include "sweeps.cuh"

namespace band {

constexpr int kPartMinRowsPerChunk = 8;

// Pivot guard.  A chunk restarts the recurrence at its first row, so on matrices that
// are not diagonally dominant it can meet pivots far smaller than NPDM's on the whole
// system; the multipliers then grow and the chunk's solution loses accuracy.  (On the
// indefinite PD ADI rows at r = 2, a plain FP64 emulation shows the error tracking the
// smallest chunk pivot: 5e-10 at a pivot 1.3e-7 times its row's largest entry, 1e-11 at
// 5e-6, NPDM's own 1e-12 above 1e-5, with every chunk block's condition number ~2.6e3.)
// A pivot whose binary exponent lies TinyPivot<T> or more below that of its row's
// largest entry is handled like a zero pivot: the system is redone by NPDM in one lane
// (or by the symbolic fix-up).  Exponents are compared with integer operations.
template <typename T> struct TinyPivot;
template <> struct TinyPivot<double> { static constexpr int value = 17; };   // < ~7.6e-6
template <> struct TinyPivot<float> { static constexpr int value = 10; };    // < ~9.8e-4

// The same guard for the interface's K x K pivot blocks: A (= I - X) counts as singular
// when |det A| lies TinyPivot<T> binary orders per row below max(1, max |A_ij|)^K.  The
// block elimination has no pivoting across blocks, so on indefinite matrices it can
// meet such a block where the whole interface system is regular.
template <typename T, int K>
__device__ __forceinline__ bool near_singular(const T (&A)[K][K]) {
  const int one = expo_of(T(1));
  int s = one;
#pragma unroll
  for (int r = 0; r < K; ++r)
#pragma unroll
    for (int c = 0; c < K; ++c) s = max(s, expo_of(A[r][c]));
  const T det = K == 1 ? A[0][0] : fma(A[0][0], A[K - 1][K - 1], -A[0][K - 1] * A[K - 1][0]);
  if (is_zero(det)) return true;
  // exponents: det ~ 2^(e - one), scale^K ~ 2^(K (s - one))
  return (expo_of(det) - one) + K * TinyPivot<T>::value <= K * (s - one);
}

// Values of T per lane in the interface exchange: y's right-hand side (2K) and the
// 2K rows of V's and W's K columns.
template <int K>
__host__ __device__ constexpr int part_words() { return 2 * K + 4 * K * K; }

template <typename T>
__host__ __device__ constexpr int part_xch_bytes() { return 32 * part_words<2>() * (int)sizeof(T); }
static_assert(part_xch_bytes<double>() <= stage_bytes_per_warp<double>(),
              "the interface exchange lives in the warp's staging area");
static_assert(part_xch_bytes<float>() <= stage_bytes_per_warp<float>(),
              "the interface exchange lives in the warp's staging area");

template <int P>
__device__ __forceinline__ int64_t part_idx(int64_t j, int64_t t, int64_t np, int k) {
  return (j * np + t) * P + k;
}

// Solves M X = R in place (R becomes X) for NB unknowns and NR columns with partial
// pivoting; false on a zero pivot.  Row exchanges are selects (M stays in registers).
template <typename T, int NB, int NR>
__device__ __forceinline__ bool block_solve(T (&M)[NB][NB], T (&R)[NB][NR]) {
  T inv[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    int piv = c;
    T big = fabs(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < NB; ++r)
      if (fabs(M[r][c]) > big) { big = fabs(M[r][c]); piv = r; }
#pragma unroll
    for (int r = c + 1; r < NB; ++r) {
      const bool sw = (r == piv);
#pragma unroll
      for (int k = c; k < NB; ++k) {
        const T u = M[c][k], v = M[r][k];
        M[c][k] = sw ? v : u;
        M[r][k] = sw ? u : v;
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const T u = R[c][k], v = R[r][k];
        R[c][k] = sw ? v : u;
        R[r][k] = sw ? u : v;
      }
    }
    if (is_zero(M[c][c])) return false;
    inv[c] = rcp<T>(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < NB; ++r) {
      const T l = M[r][c] * inv[c];
#pragma unroll
      for (int k = c + 1; k < NB; ++k) M[r][k] = fma(-l, M[c][k], M[r][k]);
#pragma unroll
      for (int k = 0; k < NR; ++k) R[r][k] = fma(-l, R[c][k], R[r][k]);
    }
  }
#pragma unroll
  for (int c = NB - 1; c >= 0; --c) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      T v = R[c][k];
#pragma unroll
      for (int m = c + 1; m < NB; ++m) v = fma(-M[c][m], R[m][k], v);
      R[c][k] = v * inv[c];
    }
  }
  return true;
}

// NPDM / NTDM on one system by one lane, scratch in the chunk-major layout (the redo of
// a failed partitioned system, and systems too short to cut).  On a zero pivot: the
// fix-up list (symbolic methods) or BAND_ERR_ZERO_PIVOT.
template <typename T, int K, int P>
__device__ __noinline__ void part_serial(const DirectArgs<T>& p, int64_t t) {
  const int64_t s = p.L.sys(t);
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const int64_t np = p.part_np;
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    RowIn<T> r;
    load_in<T, K>(p, q, r);
    if (!forward_row<T, K>(p, i, n, q, part_idx<P>(i / P, t, np, (int)(i % P)), r.a, r.b, r.c,
                           r.d, r.e, r.f, al1, al2, be1, be2, z1, z2)) {
      if (p.fix_list) {
        const unsigned long long c = atomicAdd(p.fix_count, 1ull);
        p.fix_list[c] = t;
      } else {
        set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
      }
      return;
    }
  }
  T x1 = 0, x2 = 0;
  bool bad = false;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t q = q0 + i * es;
    const int64_t w = part_idx<P>(i / P, t, np, (int)(i % P));
    T xi = fma(-p.al[w], x1, p.zs ? p.zs[w] : p.x[q]);
    if (K == 2) xi = fma(-p.be[w], x2, xi);
    p.x[q] = xi;
    bad |= not_finite(xi);
    x2 = x1;
    x1 = xi;
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

// The lanes that share one system: P of a warp's lanes (P <= 32), or a whole block of
// P / 32 warps.  any(): some lane of the group holds v.  Every lane of the warp (block)
// calls sync() and any().
struct WarpGroup {
  unsigned mask;     // the group's lanes
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool any(bool v) const {
    return (__ballot_sync(0xffffffffu, v) & mask) != 0;
  }
};
struct BlockGroup {
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool v) const { return __syncthreads_or(v) != 0; }
};

// ---------------------------------------------------------------------------
// The interface system y_k + L_k y_{k-1} + U_k y_{k+1} = g_k over a system's P chunks
// (exchange slots xch: per chunk g, V's and W's K columns; y_k = (top K, bottom K rows)).
// Block elimination from both ends: with D_k = I - L_k Cp_{k-1} (D_0 = I),
// hp_k = D_k^{-1} (g_k - L_k hp_{k-1}) and Cp_k = D_k^{-1} U_k top-down over chunks
// 0 .. P/2-1.  U_k acts on the top K rows of y_{k+1} and L_k on the bottom K rows of
// y_{k-1}, so only Cp's first K columns are nonzero and D_k = [[I - X_top, 0],
// [-X_bottom, I]] with X = V_k (bottom K rows of Cp_{k-1}): a K x K solve (partial
// pivoting) for the top rows, then Y_bottom = R_bottom + X_bottom Y_top.  Bottom-up over
// chunks P-1 .. P/2 the same step applies to the mirrored system: y's halves swapped
// (slot r read as (r + K) mod 2K) and the roles of V and W exchanged.  hp overwrites
// slots [0, NB) of a chunk and Cp's column c slots [NB (1 + c), NB (2 + c)), in the
// pass's own row order.  Returns false on a singular K x K pivot block.
template <typename T, int K, int P>
__device__ __forceinline__ bool part_eliminate(T* xch, bool up) {
  constexpr int NB = 2 * K;
  constexpr int PW = part_words<K>();
  const int rot = up ? K : 0;                       // slot of row r: (r + rot) mod NB
  const int offP = up ? 2 * NB : NB;                // coupling to the chunk done before
  const int offN = up ? NB : 2 * NB;                // coupling to the chunk done after
  auto row = [&](int r) { return (r + rot) & (NB - 1); };
  for (int q = 0; q < P / 2; ++q) {
    const int kk = up ? P - 1 - q : q;
    T* e = xch + kk * PW;
    T R[NB][K + 1];        // columns: the coupling to the next chunk, then g
    T X[NB][K];
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      R[r][K] = e[row(r)];
      R[r][0] = e[offN + row(r)];
      if (K == 2) R[r][K - 1] = e[offN + 2 * NB + row(r)];
#pragma unroll
      for (int c = 0; c < K; ++c) X[r][c] = T(0);
    }
    if (q > 0) {
      const T* ep = up ? e + PW : e - PW;
#pragma unroll
      for (int r = 0; r < NB; ++r) {
        T vr[K];
        vr[0] = e[offP + row(r)];
        if (K == 2) vr[K - 1] = e[offP + 2 * NB + row(r)];
#pragma unroll
        for (int m = 0; m < K; ++m) {
#pragma unroll
          for (int c = 0; c < K; ++c) X[r][c] = fma(vr[m], ep[NB * (1 + c) + row(K + m)], X[r][c]);
          R[r][K] = fma(-vr[m], ep[row(K + m)], R[r][K]);
        }
      }
    }
    T A[K][K], Rt[K][K + 1];
#pragma unroll
    for (int r = 0; r < K; ++r) {
#pragma unroll
      for (int c = 0; c < K; ++c) A[r][c] = (r == c ? T(1) : T(0)) - X[r][c];
#pragma unroll
      for (int c = 0; c <= K; ++c) Rt[r][c] = R[r][c];
    }
    if (near_singular<T, K>(A) || !block_solve<T, K, K + 1>(A, Rt)) return false;
#pragma unroll
    for (int c = 0; c <= K; ++c) {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        T v = R[K + r][c];
#pragma unroll
        for (int m = 0; m < K; ++m) v = fma(X[K + r][m], Rt[m][c], v);
        R[K + r][c] = v;
        R[r][c] = Rt[r][c];
      }
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      e[row(r)] = R[r][K];
#pragma unroll
      for (int c = 0; c < K; ++c) e[NB * (1 + c) + row(r)] = R[r][c];
    }
  }
  return true;
}

// Where the passes meet: chunk m-1 = P/2-1 gives y_{m-1} = hp - Cp (top K rows of y_m),
// chunk m (bottom-up) y_m = hp' - Cp' (bottom K rows of y_{m-1}).  With u = bottom
// rows of y_{m-1} and v = top rows of y_m: [[I, Cp_bottom], [Cp'_top, I]] (u, v) =
// (hp_bottom, hp'_top), solved with partial pivoting; then both chunks' y (natural row
// order: chunk m's mirrored row r is y's row (r + K) mod NB, in that slot).  False if
// singular.
template <typename T, int K, int P>
__device__ __forceinline__ bool part_meet(T* xch) {
  constexpr int NB = 2 * K;
  constexpr int PW = part_words<K>();
  constexpr int m = P / 2;
  T* a = xch + (m - 1) * PW;       // top-down, natural row order
  T* b = xch + m * PW;             // bottom-up: row r in slot (r + K) mod NB
  T M[4][5];
#pragma unroll
  for (int r = 0; r < K; ++r) {
#pragma unroll
    for (int c = 0; c < K; ++c) {
      M[r][c] = r == c ? T(1) : T(0);
      M[r][K + c] = a[NB * (1 + c) + K + r];            // Cp_{m-1}, bottom row r, column c
      M[K + r][c] = b[NB * (1 + c) + r];                // Cp'_m, its row K + r = top row r
      M[K + r][K + c] = r == c ? T(1) : T(0);
    }
    M[r][NB] = a[K + r];
    M[K + r][NB] = b[r];
  }
  {   // the meeting system is singular exactly when I - Cp'_top Cp_bottom is
    T S[K][K];
#pragma unroll
    for (int r = 0; r < K; ++r)
#pragma unroll
      for (int c = 0; c < K; ++c) {
        T v = r == c ? T(1) : T(0);
#pragma unroll
        for (int q = 0; q < K; ++q) v = fma(-M[K + r][q], M[q][K + c], v);
        S[r][c] = v;
      }
    if (near_singular<T, K>(S)) return false;
  }
  if (!solve_small<T, NB>(M)) return false;
  T u[K], v[K];
#pragma unroll
  for (int c = 0; c < K; ++c) {
    u[c] = M[c][NB];
    v[c] = M[K + c][NB];
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    T ya = a[r], yb = b[r];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      ya = fma(-a[NB * (1 + c) + r], v[c], ya);
      yb = fma(-b[NB * (1 + c) + r], u[c], yb);
    }
    a[r] = ya;
    b[r] = yb;
  }
  return true;
}

// Back-substitution of one pass's half, away from the meeting point: top-down chunks
// P/2-2 .. 0 (y_k = hp_k - Cp_k (top rows of y_{k+1})) or bottom-up chunks P/2+1 .. P-1
// (the mirrored step).  The mirrored row r sits in slot (r + K) mod NB, which is where
// y's row (r + K) mod NB belongs: y ends in natural order in both halves.
template <typename T, int K, int P>
__device__ __forceinline__ void part_backsub(T* xch, bool up) {
  constexpr int NB = 2 * K;
  constexpr int PW = part_words<K>();
  const int rot = up ? K : 0;
  for (int q = P / 2 - 2; q >= 0; --q) {
    const int kk = up ? P - 1 - q : q;
    T* e = xch + kk * PW;
    const T* en = up ? e - PW : e + PW;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int sr = (r + rot) & (NB - 1);
      T v = e[sr];
#pragma unroll
      for (int c = 0; c < K; ++c) v = fma(-e[NB * (1 + c) + sr], en[(c + rot) & (NB - 1)], v);
      e[sr] = v;
    }
  }
}

// The batch's t-th system, chunk k of P, by one lane of its group.  ring: this warp's
// staging area (stage_bytes_per_warp<T>() bytes of shared memory) for the forward
// sweep's row ring; xch: the group's exchange area, P * part_words<K>() values of T
// (it may overlap the group's rings: the group synchronises after the forward sweep).
// KB: rows whose scratch the backward sweeps load together (registers against memory
// latency).
template <typename T, int K, int P, int KB, class Grp>
__device__ __forceinline__ void partition_sys(const DirectArgs<T>& p, int64_t t, int k, int lane,
                                              T* ring_area, T* xch, const Grp& grp) {
  constexpr int NB = 2 * K;
  constexpr int PW = part_words<K>();
  bool active = t < p.L.nsys;
  const int64_t s = active ? p.L.sys(t) : 0;
  if (active && p.skip && p.skip[s]) active = false;
  const int64_t n = active ? p.L.rows(s) : 0;
  // 0: nothing, 1: the first lane alone (short system), 2: partitioned
  const int mode = !active ? 0 : (n < (int64_t)kPartMinRowsPerChunk * P ? 1 : 2);
  const int64_t q0 = active ? p.L.base(s) : 0, es = active ? p.L.stride() : 0;
  const int64_t L0 = n / P, rem = n % P;
  const int64_t s0 = k * L0 + (k < rem ? k : rem);
  const int64_t L = mode == 2 ? L0 + (k < rem ? 1 : 0) : 0;
  const int64_t np = p.part_np;
  T* const zsf = p.zs;        // z of f (set for this schedule; x if null)

  // ---- forward: the chunk's LU with f and B's columns
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0;
  T zf1 = 0, zf2 = 0, zv11 = 0, zv12 = 0, zv21 = 0, zv22 = 0;
  T gl = 0, rcl = 0, rcl2 = 0, el2 = 0, dl = 0, el = 0;   // last rows, for C's columns
  bool zero = false;
  {
    // rows staged through the warp's shared-memory ring, StageDepth rows ahead; each
    // lane copies (and later reads) only its own slots
    constexpr int D = StageDepth<T>::value;
    constexpr int NA = K == 2 ? 6 : 4;     // arrays staged: (a,) b, c, d, (e,) f
    constexpr int IB = K == 2 ? 1 : 0, IC = IB + 1, ID = IB + 2, IF = NA - 1;
    const RowRing<T, NA, D> ring{ring_area, lane};
    const T* src[NA];
    if (K == 2) {
      src[0] = p.a; src[1] = p.b; src[2] = p.c; src[3] = p.d; src[4] = p.e; src[5] = p.f;
    } else {
      src[0] = p.b; src[1] = p.c; src[2] = p.d; src[3] = p.f;
    }
#pragma unroll
    for (int j = 0; j < D - 1; ++j) {
      if (j < L) ring.issue(j, src, q0 + (s0 + j) * es);
      else ring.skip();
    }
    for (int64_t j = 0; j < L; ++j) {
      const int64_t i = s0 + j;
      const int64_t jp = j + D - 1;
      if (jp < L) ring.issue((int)(jp & (D - 1)), src, q0 + (s0 + jp) * es);
      else ring.skip();
      cp_async_wait<D - 1>();
      const int slot = (int)(j & (D - 1));
      // the matrix's masks, then the chunk's own block
      const T ag = (K == 2 && i >= 2) ? ring.get(slot, 0) : T(0);
      const T bg = (i >= 1) ? ring.get(slot, IB) : T(0);
      const T dg = (i + 1 < n) ? ring.get(slot, ID) : T(0);
      const T eg = (K == 2 && i + 2 < n) ? ring.get(slot, 4) : T(0);
      const T cc = ring.get(slot, IC), ff = ring.get(slot, IF);
      const T aa = (j >= 2) ? ag : T(0);
      const T bb = (j >= 1) ? bg : T(0);
      const T dd = (j + 1 < L) ? dg : T(0);
      const T ee = (j + 2 < L) ? eg : T(0);
      // B's columns (unknowns x_{s0-K} ..): row 0 holds a (x_{s0-2}) and b (x_{s0-1}),
      // row 1 a (x_{s0-1}); TD: row 0 holds b
      T rv1 = 0, rv2 = 0;
      if (K == 2) {
        rv1 = j == 0 ? ag : T(0);
        rv2 = j == 0 ? bg : (j == 1 ? ag : T(0));
      } else {
        rv1 = j == 0 ? bg : T(0);
      }
      T g, m;
      if (K == 2) {
        g = fma(-al2, aa, bb);
        m = fma(-al1, g, fma(-be2, aa, cc));
      } else {
        g = bb;
        m = fma(-al1, g, cc);
      }
      {
        int ex = expo_of(cc);
        ex = max(ex, max(expo_of(bg), expo_of(dg)));
        if (K == 2) ex = max(ex, max(expo_of(ag), expo_of(eg)));
        if (is_zero(m) || expo_of(m) + TinyPivot<T>::value <= ex) { zero = true; break; }
      }
      const T rc = rcp<T>(m);
      const T alv = (K == 2 ? fma(-be1, g, dd) : dd) * rc;
      const int64_t w = part_idx<P>(j, t, np, k);
      p.al[w] = alv;
      T zf, zv1;
      if (K == 2) {
        const T bev = ee * rc;
        p.be[w] = bev;
        zf = fma(-zf1, g, fma(-zf2, aa, ff)) * rc;
        zv1 = fma(-zv11, g, fma(-zv12, aa, rv1)) * rc;
        const T zv2 = fma(-zv21, g, fma(-zv22, aa, rv2)) * rc;
        p.zv2[w] = zv2;
        zv22 = zv21; zv21 = zv2;
        be2 = be1; be1 = bev;
      } else {
        zf = fma(-zf1, g, ff) * rc;
        zv1 = fma(-zv11, g, rv1) * rc;
      }
      if (zsf) zsf[w] = zf; else p.x[q0 + i * es] = zf;
      p.zv1[w] = zv1;
      al2 = al1; al1 = alv;
      zf2 = zf1; zf1 = zf; zv12 = zv11; zv11 = zv1;
      rcl2 = rcl; rcl = rc; gl = g; el2 = el; el = eg; dl = dg;
    }
    cp_async_wait<0>();
  }
  grp.sync();     // the rings' slots become the exchange area below
  // forward values of C's columns (nonzero only in the last K rows).  PD: column 1
  // (x_{s0+L}) has e at row L-2 and d at row L-1, column 2 (x_{s0+L+1}) e at row L-1.
  T zw1_2 = 0, zw1_1 = 0, zw2_1 = 0;     // zw<column>_<rows from the end>
  if (!zero && L > 0) {
    if (K == 2) {
      zw1_2 = el2 * rcl2;
      zw1_1 = fma(-zw1_2, gl, dl) * rcl;
      zw2_1 = el * rcl;
    } else {
      zw1_1 = dl * rcl;
    }
  }
  // ---- first backward sweep: top and bottom K rows of g, V, W, written to this lane's
  // exchange slots (y-slot of row j: top rows 0 .. K-1 -> 0 .. K-1, bottom rows
  // L-K .. L-1 -> K .. 2K-1; columns g, V1, W1, V2, W2 at offsets 0, NB, 2NB, 3NB, 4NB)
  T* const my = xch + k * PW;
  if (!zero && L > 0) {
    T xf1 = 0, xf2 = 0, xv11 = 0, xv12 = 0, xv21 = 0, xv22 = 0;
    T xw11 = 0, xw12 = 0, xw21 = 0, xw22 = 0;
    // rows in blocks of kB: the block's scratch values are loaded together (one memory
    // latency a block)
    constexpr int kB = KB;
    for (int64_t top = L - 1; top >= 0; top -= kB) {
      T av[kB], bv[kB], fv[kB], v1[kB], v2[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        av[u] = bv[u] = fv[u] = v1[u] = v2[u] = T(0);
        const int64_t j = top - u;
        if (j >= 0) {
          const int64_t w = part_idx<P>(j, t, np, k);
          av[u] = p.al[w];
          fv[u] = zsf ? zsf[w] : p.x[q0 + (s0 + j) * es];
          v1[u] = p.zv1[w];
          if (K == 2) {
            bv[u] = p.be[w];
            v2[u] = p.zv2[w];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int64_t j = top - u;
        if (j < 0) break;
        const T a = av[u];
        // forward values of W's columns at this row
        const T zw1 = j == L - 1 ? zw1_1 : (K == 2 && j == L - 2 ? zw1_2 : T(0));
        T xf = fma(-a, xf1, fv[u]);
        T xv1 = fma(-a, xv11, v1[u]);
        T xw1 = fma(-a, xw11, zw1);
        T xv2 = 0, xw2 = 0;
        if (K == 2) {
          const T b = bv[u];
          const T zw2 = j == L - 1 ? zw2_1 : T(0);
          xf = fma(-b, xf2, xf);
          xv1 = fma(-b, xv12, xv1);
          xw1 = fma(-b, xw12, xw1);
          xv2 = fma(-b, xv22, fma(-a, xv21, v2[u]));
          xw2 = fma(-b, xw22, fma(-a, xw21, zw2));
          xv22 = xv21; xv21 = xv2; xw22 = xw21; xw21 = xw2;
        }
        if (j >= L - K) {                  // a bottom row
          const int slot = K + (int)(j - (L - K));
          my[slot] = xf;
          my[NB + slot] = xv1;
          my[2 * NB + slot] = xw1;
          if (K == 2) {
            my[3 * NB + slot] = xv2;
            my[4 * NB + slot] = xw2;
          }
        }
        xf2 = xf1; xf1 = xf; xv12 = xv11; xv11 = xv1; xw12 = xw11; xw11 = xw1;
      }
    }
    // the top rows: the sweep's last values (row 0 in *1, row 1 in *2)
    my[0] = xf1;
    my[NB] = xv11;
    my[2 * NB] = xw11;
    if (K == 2) {
      my[1] = xf2;
      my[NB + 1] = xv12;
      my[2 * NB + 1] = xw12;
      my[3 * NB] = xv21;
      my[3 * NB + 1] = xv22;
      my[4 * NB] = xw21;
      my[4 * NB + 1] = xw22;
    }
  } else {
#pragma unroll
    for (int c = 0; c < PW; ++c) my[c] = T(0);
  }
  const bool gzero = grp.any(zero);
  grp.sync();
  bool fail = gzero;
  // the interface: chunks 0 .. P/2-1 eliminated top-down by chunk 0's lane, chunks
  // P-1 .. P/2 bottom-up by chunk P-1's lane, at the same time; they meet in a 2K x 2K
  // system, then each back-substitutes its half
  const bool ilane = mode == 2 && (k == 0 || k == P - 1);
  bool ifail = false;
  // (every lane of the warp or block must reach grp.any: no short-circuit around it)
  if (ilane && !fail) ifail = !part_eliminate<T, K, P>(xch, k != 0);
  const bool elim_fail = grp.any(ifail);
  fail = fail || elim_fail;
  grp.sync();
  if (mode == 2 && k == 0 && !fail) ifail = !part_meet<T, K, P>(xch);
  const bool meet_fail = grp.any(ifail);
  fail = fail || meet_fail;
  grp.sync();
  if (ilane && !fail) part_backsub<T, K, P>(xch, k != 0);
  grp.sync();
  // ---- redo (short systems, failed eliminations) by the first lane, or the second
  // backward sweep with z - z_V u - z_W v
  if (k == 0 && (mode == 1 || (mode == 2 && fail))) {
    if (mode == 2 && p.fix_list) {
      const unsigned long long c = atomicAdd(p.fix_count, 1ull);
      p.fix_list[c] = t;
    } else if (mode == 2 && p.redo_list) {      // solved again by a follow-up launch
      const unsigned long long c = atomicAdd(p.redo_count, 1ull);
      p.redo_list[c] = t;
    } else {
      part_serial<T, K, P>(p, t);
    }
  }
  const bool back = mode == 2 && !fail;
  bool bad = false;
  if (back) {
    T u[K], v[K];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      u[m] = k > 0 ? xch[(k - 1) * PW + K + m] : T(0);
      v[m] = k + 1 < P ? xch[(k + 1) * PW + m] : T(0);
    }
    T x1 = 0, x2 = 0;
    constexpr int kB = KB;
    for (int64_t top = L - 1; top >= 0; top -= kB) {
      T av[kB], bv[kB], fv[kB], v1[kB], v2[kB];
#pragma unroll
      for (int e = 0; e < kB; ++e) {
        av[e] = bv[e] = fv[e] = v1[e] = v2[e] = T(0);
        const int64_t j = top - e;
        if (j >= 0) {
          const int64_t w = part_idx<P>(j, t, np, k);
          av[e] = p.al[w];
          fv[e] = zsf ? zsf[w] : p.x[q0 + (s0 + j) * es];
          v1[e] = p.zv1[w];
          if (K == 2) {
            bv[e] = p.be[w];
            v2[e] = p.zv2[w];
          }
        }
      }
#pragma unroll
      for (int e = 0; e < kB; ++e) {
        const int64_t j = top - e;
        if (j < 0) break;
        T z = fma(-v1[e], u[0], fv[e]);
        if (K == 2) z = fma(-v2[e], u[K - 1], z);
        if (j == L - 1) {
          z = fma(-zw1_1, v[0], z);
          if (K == 2) z = fma(-zw2_1, v[K - 1], z);
        } else if (K == 2 && j == L - 2) {
          z = fma(-zw1_2, v[0], z);
        }
        T xi = fma(-av[e], x1, z);
        if (K == 2) xi = fma(-bv[e], x2, xi);
        p.x[q0 + (s0 + j) * es] = xi;
        bad |= not_finite(xi);
        x2 = x1;
        x1 = xi;
      }
    }
  }
  const bool gbad = grp.any(bad);
  if (back && k == 0) set_status(p.status, s, gbad ? BAND_ERR_NONFINITE : BAND_OK);
}

// The warp's 32 / P systems (P <= 32), positions t = warp * (32 / P) + (lane / P).
// stage: the warp's staging area (stage_bytes_per_warp<T>() bytes of shared memory):
// the forward sweep's row ring, then the interface exchange.
template <typename T, int K, int P, int KB = 4>
__device__ __forceinline__ void partition_one(const DirectArgs<T>& p, int64_t warp, T* stage) {
  static_assert(P <= 32, "a warp holds at most 32 chunks");
  const int lane = (int)(threadIdx.x & 31);
  const int g = lane / P, k = lane % P;
  const WarpGroup grp{P == 32 ? 0xffffffffu : (((1u << (P & 31)) - 1u) << (g * P))};
  partition_sys<T, K, P, KB>(p, warp * (32 / P) + g, k, lane, stage,
                             stage + g * P * part_words<K>(), grp);
}

// One system per block of W warps: P = 32 W chunks, the batch's blockIdx.x-th system.
// smem: W staging areas of stage_bytes_per_warp<T>() bytes (the rings, then the
// exchange of all P chunks).
template <typename T, int K, int W>
__device__ __forceinline__ void partition_block(const DirectArgs<T>& p, unsigned char* smem) {
  constexpr int P = 32 * W;
  static_assert(P * part_words<K>() * (int)sizeof(T) <= W * stage_bytes_per_warp<T>(),
                "the block's exchange fits its staging areas");
  const int k = (int)threadIdx.x;
  T* ring = reinterpret_cast<T*>(smem + (k >> 5) * stage_bytes_per_warp<T>());
  const BlockGroup grp{};
  partition_sys<T, K, P, 4>(p, (int64_t)blockIdx.x, k, k & 31, ring, reinterpret_cast<T*>(smem),
                            grp);
}

}  // namespace band
