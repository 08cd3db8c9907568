// grid.cu -- the grid schedule (BAND_SCHED_GRID): one system, or a few, over the whole
// GPU.  The paper times single systems of up to N = 10^8 rows (Table 3 and Table 5:
// NPDM, MNPDM, NTDM), which one thread, two or even a block of 256 lanes leave mostly
// idle on a GPU.
//
// Each system is cut into P chunks of about n / P consecutive rows, one lane each, with
// P chosen so that the launch fills every SM (one wave of 16 warps per SM).
//  1. k_grid_chunks: lane c eliminates its chunk A_c with the NPDM / NTDM recurrence
//     of Sec. 1 (U unit upper), carrying f and the K columns B_c that couple the chunk
//     to the K unknowns above it, then back-substitutes g = A_c^{-1} f, V = A_c^{-1} B_c
//     and W = A_c^{-1} C_c (C_c: the columns coupling it to the K unknowns below it)
//     and keeps only their top K and bottom K rows.  With y_c = (top K, bottom K rows
//     of chunk c) the chunks' boundary unknowns satisfy the block-tridiagonal system
//       L_c y_{c-1} + y_c + U_c y_{c+1} = g_c,
//     L_c = V's rows on the bottom K entries of y_{c-1}, U_c = W's rows on the top K of
//     y_{c+1} (the partition of the partitioned schedule, with one chunk per lane of
//     the whole grid instead of a warp or a block).
//  2. Block cyclic reduction of that system, one launch per level: at level s the
//     blocks c = 0 mod 2s eliminate their neighbours c - s and c + s,
//       D_c -= L_c D_l^{-1} U_l + U_c D_r^{-1} L_r,  g_c -= L_c D_l^{-1} g_l + U_c D_r^{-1} g_r,
//       L_c <- -L_c D_l^{-1} L_l,  U_c <- -U_c D_r^{-1} U_r,
//     (2K x 2K blocks, each D solved with partial pivoting), until block 0 is alone;
//     then y_0 = D_0^{-1} g_0 and, level by level downwards, y_j = D_j^{-1} (g_j - L_j
//     y_{j-s} - U_j y_{j+s}) for the blocks eliminated at that level.
//  3. k_grid_back: every lane back-substitutes its chunk once more with
//     z - z_V u_c - z_W v_c (u_c = bottom K of y_{c-1}, v_c = top K of y_{c+1}): x.
// In exact arithmetic the result is A^{-1} f.  Neither the chunks nor the reduction
// pivot across blocks, so as for the partitioned schedule a chunk pivot 2^-17 (FP64) /
// 2^-10 (FP32) below its row's largest entry, or a reduction block as close to
// singular, marks the system BAND_ERR_ZERO_PIVOT ("this schedule's elimination order
// met a pivot it cannot use"); another schedule can solve it.  On diagonally dominant
// systems that never happens.
#include <cstdint>

#include "api_util.h"
#include "kernels.h"
#include "sweeps.cuh"

namespace band {

namespace {

template <typename T> struct GridTiny;
template <> struct GridTiny<double> { static constexpr int value = 17; };
template <> struct GridTiny<float> { static constexpr int value = 10; };

// Per chunk: the block row of the reduced system (D, L, U: NB x NB, g: NB) and the
// forward values of C's columns at the chunk's last rows (3), in one record.
template <int K>
__host__ __device__ constexpr int rec_words() {
  return 3 * (2 * K) * (2 * K) + 2 * K + 3;
}

template <typename T>
struct GridArgs {
  Layout L;
  const T *a, *b, *c, *d, *e, *f;
  T* x;
  T *al, *be, *zf, *zv1, *zv2;   // chunk-major scratch rows: row j of chunk g at j * C + g
  T* rec;                        // C records of rec_words<K>()
  T* y;                          // C x 2K solved boundary unknowns
  int32_t* flags;                // per system: bit 0 failed elimination, bit 1 non-finite
  int32_t* status;
  int64_t P;                     // chunks per system
  int64_t C;                     // chunks in all: nsys * P
};

template <typename T, int K>
__device__ __forceinline__ T* rec_D(const GridArgs<T>& p, int64_t g) { return p.rec + g * rec_words<K>(); }
template <typename T, int K>
__device__ __forceinline__ T* rec_L(const GridArgs<T>& p, int64_t g) {
  return p.rec + g * rec_words<K>() + (2 * K) * (2 * K);
}
template <typename T, int K>
__device__ __forceinline__ T* rec_U(const GridArgs<T>& p, int64_t g) {
  return p.rec + g * rec_words<K>() + 2 * (2 * K) * (2 * K);
}
template <typename T, int K>
__device__ __forceinline__ T* rec_g(const GridArgs<T>& p, int64_t g) {
  return p.rec + g * rec_words<K>() + 3 * (2 * K) * (2 * K);
}
template <typename T, int K>
__device__ __forceinline__ T* rec_zw(const GridArgs<T>& p, int64_t g) {
  return p.rec + g * rec_words<K>() + 3 * (2 * K) * (2 * K) + 2 * K;
}

__device__ __forceinline__ void set_flag(int32_t* flags, int64_t s, int32_t bit) {
  atomicOr(flags + s, bit);
}

// rows [s0, s0 + len) of chunk k of a system of n rows split into P chunks
__host__ __device__ __forceinline__ void chunk_rows(int64_t n, int64_t P, int64_t k, int64_t& s0,
                                                    int64_t& len) {
  const int64_t L0 = n / P, rem = n % P;
  s0 = k * L0 + (k < rem ? k : rem);
  len = L0 + (k < rem ? 1 : 0);
}

// ---------------------------------------------------------------- phase 1
template <typename T, int K>
__global__ void __launch_bounds__(64, 8) k_grid_chunks(const GridArgs<T> p) {
  constexpr int NB = 2 * K;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.C) return;
  const int64_t t = g / p.P, k = g % p.P;
  const int64_t s = p.L.sys(t);
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  int64_t s0, L;
  chunk_rows(n, p.P, k, s0, L);
  const int64_t C = p.C;
  T al1 = 0, al2 = 0, be1 = 0, be2 = 0;
  T zf1 = 0, zf2 = 0, zv11 = 0, zv12 = 0, zv21 = 0, zv22 = 0;
  T gl = 0, rcl = 0, rcl2 = 0, el2 = 0, dl = 0, el = 0;   // the last rows, for C's columns
  bool zero = false;
  // rows of the chunk, two ahead in registers
  auto load = [&](int64_t i, T& av, T& bv, T& cv, T& dv, T& ev, T& fv) {
    const int64_t q = q0 + i * es;
    av = K == 2 ? ldro(p.a + q) : T(0);
    bv = ldro(p.b + q);
    cv = ldro(p.c + q);
    dv = ldro(p.d + q);
    ev = K == 2 ? ldro(p.e + q) : T(0);
    fv = ldro(p.f + q);
  };
  T ra0 = 0, rb0 = 0, rc0 = 0, rd0 = 0, re0 = 0, rf0 = 0;
  T ra1 = 0, rb1 = 0, rc1 = 0, rd1 = 0, re1 = 0, rf1 = 0;
  if (L > 0) load(s0, ra0, rb0, rc0, rd0, re0, rf0);
  if (L > 1) load(s0 + 1, ra1, rb1, rc1, rd1, re1, rf1);
  for (int64_t j = 0; j < L; ++j) {
    const int64_t i = s0 + j;
    T ra2 = 0, rb2 = 0, rc2 = 0, rd2 = 0, re2 = 0, rf2 = 0;
    if (j + 2 < L) load(i + 2, ra2, rb2, rc2, rd2, re2, rf2);
    // the matrix's masks, then the chunk's own block
    const T ag = (K == 2 && i >= 2) ? ra0 : T(0);
    const T bg = (i >= 1) ? rb0 : T(0);
    const T dg = (i + 1 < n) ? rd0 : T(0);
    const T eg = (K == 2 && i + 2 < n) ? re0 : T(0);
    const T cc = rc0, ff = rf0;
    const T aa = (j >= 2) ? ag : T(0);
    const T bb = (j >= 1) ? bg : T(0);
    const T dd = (j + 1 < L) ? dg : T(0);
    const T ee = (j + 2 < L) ? eg : T(0);
    // B's columns (x_{s0-K} ..): PD row 0 holds a (x_{s0-2}) and b (x_{s0-1}), row 1
    // a (x_{s0-1}); TD row 0 holds b
    T rv1, rv2 = 0;
    if (K == 2) {
      rv1 = j == 0 ? ag : T(0);
      rv2 = j == 0 ? bg : (j == 1 ? ag : T(0));
    } else {
      rv1 = j == 0 ? bg : T(0);
    }
    T gm, m;
    if (K == 2) {
      gm = fma(-al2, aa, bb);
      m = fma(-al1, gm, fma(-be2, aa, cc));
    } else {
      gm = bb;
      m = fma(-al1, gm, cc);
    }
    {
      int ex = max(expo_of(cc), max(expo_of(bg), expo_of(dg)));
      if (K == 2) ex = max(ex, max(expo_of(ag), expo_of(eg)));
      if (is_zero(m) || expo_of(m) + GridTiny<T>::value <= ex) {
        zero = true;
        break;
      }
    }
    const T rc = rcp<T>(m);
    const T alv = (K == 2 ? fma(-be1, gm, dd) : dd) * rc;
    const int64_t w = j * C + g;
    p.al[w] = alv;
    T zf, zv1;
    if (K == 2) {
      const T bev = ee * rc;
      p.be[w] = bev;
      zf = fma(-zf1, gm, fma(-zf2, aa, ff)) * rc;
      zv1 = fma(-zv11, gm, fma(-zv12, aa, rv1)) * rc;
      const T zv2 = fma(-zv21, gm, fma(-zv22, aa, rv2)) * rc;
      p.zv2[w] = zv2;
      zv22 = zv21; zv21 = zv2;
      be2 = be1; be1 = bev;
    } else {
      zf = fma(-zf1, gm, ff) * rc;
      zv1 = fma(-zv11, gm, rv1) * rc;
    }
    p.zf[w] = zf;
    p.zv1[w] = zv1;
    al2 = al1; al1 = alv;
    zf2 = zf1; zf1 = zf; zv12 = zv11; zv11 = zv1;
    rcl2 = rcl; rcl = rc; gl = gm; el2 = el; el = eg; dl = dg;
    ra0 = ra1; rb0 = rb1; rc0 = rc1; rd0 = rd1; re0 = re1; rf0 = rf1;
    ra1 = ra2; rb1 = rb2; rc1 = rc2; rd1 = rd2; re1 = re2; rf1 = rf2;
  }
  // (a chunk of fewer than K rows occurs only when one chunk is the whole system, and
  // then no boundary unknowns are needed)
  if (zero || (p.P > 1 && L < K)) {
    set_flag(p.flags, s, 1);
    return;
  }
  // forward values of C's columns (nonzero only in the last K rows).  PD: column 1
  // (x_{s0+L}) has e at row L-2 and d at row L-1, column 2 (x_{s0+L+1}) e at row L-1.
  T zw1_2 = 0, zw1_1, zw2_1 = 0;
  if (K == 2) {
    zw1_2 = el2 * rcl2;
    zw1_1 = fma(-zw1_2, gl, dl) * rcl;
    zw2_1 = el * rcl;
  } else {
    zw1_1 = dl * rcl;
  }
  // first backward sweep: the top and bottom K rows of g, V (columns 1, 2) and W
  T gy[NB], vy[K][NB], wy[K][NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    gy[r] = T(0);
#pragma unroll
    for (int m = 0; m < K; ++m) vy[m][r] = wy[m][r] = T(0);
  }
  T xf1 = 0, xf2 = 0, xv11 = 0, xv12 = 0, xv21 = 0, xv22 = 0;
  T xw11 = 0, xw12 = 0, xw21 = 0, xw22 = 0;
  constexpr int kB = 4;
  for (int64_t top = L - 1; top >= 0; top -= kB) {
    T av[kB], bv[kB], fv[kB], v1[kB], v2[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      av[u] = bv[u] = fv[u] = v1[u] = v2[u] = T(0);
      const int64_t j = top - u;
      if (j >= 0) {
        const int64_t w = j * C + g;
        av[u] = p.al[w];
        fv[u] = p.zf[w];
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
      if (j >= L - K) {                 // a bottom row: slot K + (j - (L - K))
        const int slot = K + (int)(j - (L - K));
#pragma unroll
        for (int r = K; r < NB; ++r)
          if (r == slot) {
            gy[r] = xf;
            vy[0][r] = xv1;
            wy[0][r] = xw1;
            if (K == 2) {
              vy[K - 1][r] = xv2;
              wy[K - 1][r] = xw2;
            }
          }
      }
      xf2 = xf1; xf1 = xf; xv12 = xv11; xv11 = xv1; xw12 = xw11; xw11 = xw1;
    }
  }
  // the top rows: the sweep's last values (row 0 in *1, row 1 in *2)
  gy[0] = xf1;
  vy[0][0] = xv11;
  wy[0][0] = xw11;
  if (K == 2) {
    gy[1] = xf2;
    vy[0][1] = xv12;
    wy[0][1] = xw12;
    vy[1][0] = xv21;
    vy[1][1] = xv22;
    wy[1][0] = xw21;
    wy[1][1] = xw22;
  }
  // the block row: D = I, L's columns K.. (bottom entries of y_{c-1}) = V's columns,
  // U's columns 0 .. K-1 (top entries of y_{c+1}) = W's columns; the first and last
  // chunks have no neighbour there
  T* D = rec_D<T, K>(p, g);
  T* Lm = rec_L<T, K>(p, g);
  T* Um = rec_U<T, K>(p, g);
#pragma unroll
  for (int r = 0; r < NB; ++r) {
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      D[r * NB + c] = r == c ? T(1) : T(0);
      Lm[r * NB + c] = (k > 0 && c >= K) ? vy[c - K][r] : T(0);
      Um[r * NB + c] = (k + 1 < p.P && c < K) ? wy[c][r] : T(0);
    }
    rec_g<T, K>(p, g)[r] = gy[r];
  }
  T* zw = rec_zw<T, K>(p, g);
  zw[0] = zw1_1;
  zw[1] = zw1_2;
  zw[2] = zw2_1;
}

// ---------------------------------------------------------------- phase 2
// Solves M X = R for NB unknowns and NR right-hand columns with partial pivoting.
// False on a zero pivot or one GridTiny binary orders below M's largest entry.
template <typename T, int NB, int NR>
__device__ __forceinline__ bool small_solve(T (&M)[NB][NB], T (&R)[NB][NR]) {
  int top = 0;
#pragma unroll
  for (int r = 0; r < NB; ++r)
#pragma unroll
    for (int c = 0; c < NB; ++c) top = max(top, expo_of(M[r][c]));
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    int piv = c;
    T big = fabs(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < NB; ++r)
      if (fabs(M[r][c]) > big) {
        big = fabs(M[r][c]);
        piv = r;
      }
#pragma unroll
    for (int r = c + 1; r < NB; ++r) {
      const bool sw = r == piv;
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const T u = M[c][q], v = M[r][q];
        M[c][q] = sw ? v : u;
        M[r][q] = sw ? u : v;
      }
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const T u = R[c][q], v = R[r][q];
        R[c][q] = sw ? v : u;
        R[r][q] = sw ? u : v;
      }
    }
    if (is_zero(M[c][c]) || expo_of(M[c][c]) + GridTiny<T>::value <= top) return false;
    const T inv = T(1) / M[c][c];
#pragma unroll
    for (int r = c + 1; r < NB; ++r) {
      const T l = M[r][c] * inv;
#pragma unroll
      for (int q = c; q < NB; ++q) M[r][q] = fma(-l, M[c][q], M[r][q]);
#pragma unroll
      for (int q = 0; q < NR; ++q) R[r][q] = fma(-l, R[c][q], R[r][q]);
    }
  }
#pragma unroll
  for (int c = NB - 1; c >= 0; --c) {
    const T inv = T(1) / M[c][c];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      T v = R[c][q];
#pragma unroll
      for (int m = c + 1; m < NB; ++m) v = fma(-M[c][m], R[m][q], v);
      R[c][q] = v * inv;
    }
  }
  return true;
}

// Level s of the reduction: block c = 2 s i (of its system) eliminates c - s and c + s.
template <typename T, int K>
__global__ void __launch_bounds__(128) k_grid_reduce(const GridArgs<T> p, int64_t s) {
  constexpr int NB = 2 * K;
  const int64_t per = (p.P + 2 * s - 1) / (2 * s);          // kept blocks per system
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= per * p.L.nsys) return;
  const int64_t t = id / per, c = (id % per) * 2 * s;
  const int64_t g = t * p.P + c;
  const int64_t sys = p.L.sys(t);
  if (p.flags[sys] & 1) return;
  T Dc[NB][NB], Lc[NB][NB], Uc[NB][NB], gc[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      Dc[r][q] = rec_D<T, K>(p, g)[r * NB + q];
      Lc[r][q] = rec_L<T, K>(p, g)[r * NB + q];
      Uc[r][q] = rec_U<T, K>(p, g)[r * NB + q];
    }
    gc[r] = rec_g<T, K>(p, g)[r];
  }
  bool ok = true;
  for (int side = 0; side < 2 && ok; ++side) {
    const int64_t nb = side == 0 ? c - s : c + s;
    if (nb < 0 || nb >= p.P) {
      // no neighbour: nothing couples to it any more
      if (side == 0) {
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
          for (int q = 0; q < NB; ++q) Lc[r][q] = T(0);
      } else {
#pragma unroll
        for (int r = 0; r < NB; ++r)
#pragma unroll
          for (int q = 0; q < NB; ++q) Uc[r][q] = T(0);
      }
      continue;
    }
    const int64_t gn = t * p.P + nb;
    T M[NB][NB], R[NB][2 * NB + 1];     // D_n^{-1} [L_n | U_n | g_n]
#pragma unroll
    for (int r = 0; r < NB; ++r) {
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        M[r][q] = rec_D<T, K>(p, gn)[r * NB + q];
        R[r][q] = rec_L<T, K>(p, gn)[r * NB + q];
        R[r][NB + q] = rec_U<T, K>(p, gn)[r * NB + q];
      }
      R[r][2 * NB] = rec_g<T, K>(p, gn)[r];
    }
    if (!small_solve<T, NB, 2 * NB + 1>(M, R)) {
      ok = false;
      break;
    }
    // C = the coupling to the neighbour (L_c on the left, U_c on the right)
    T Cc[NB][NB];
#pragma unroll
    for (int r = 0; r < NB; ++r)
#pragma unroll
      for (int q = 0; q < NB; ++q) Cc[r][q] = side == 0 ? Lc[r][q] : Uc[r][q];
    // D_c -= C Y (left: Y = D_l^{-1} U_l; right: X = D_r^{-1} L_r), g_c -= C h, and the
    // new outer coupling -C (D_n^{-1} L_n on the left, D_n^{-1} U_n on the right)
    const int inner = side == 0 ? NB : 0, outer = side == 0 ? 0 : NB;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        T dsum = Dc[r][q], osum = T(0);
#pragma unroll
        for (int m = 0; m < NB; ++m) {
          dsum = fma(-Cc[r][m], R[m][inner + q], dsum);
          osum = fma(-Cc[r][m], R[m][outer + q], osum);
        }
        Dc[r][q] = dsum;
        if (side == 0) Lc[r][q] = osum;
        else Uc[r][q] = osum;
      }
      T gsum = gc[r];
#pragma unroll
      for (int m = 0; m < NB; ++m) gsum = fma(-Cc[r][m], R[m][2 * NB], gsum);
      gc[r] = gsum;
    }
  }
  if (!ok) {
    set_flag(p.flags, sys, 1);
    return;
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) {
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      rec_D<T, K>(p, g)[r * NB + q] = Dc[r][q];
      rec_L<T, K>(p, g)[r * NB + q] = Lc[r][q];
      rec_U<T, K>(p, g)[r * NB + q] = Uc[r][q];
    }
    rec_g<T, K>(p, g)[r] = gc[r];
  }
}

// Back-substitution of level s (s = 0: block 0 of every system, whose reduced block row
// couples to nothing): y_j = D_j^{-1} (g_j - L_j y_{j-s} - U_j y_{j+s}), j = s mod 2s.
template <typename T, int K>
__global__ void __launch_bounds__(128) k_grid_expand(const GridArgs<T> p, int64_t s) {
  constexpr int NB = 2 * K;
  const int64_t per = s == 0 ? 1 : (p.P + s) / (2 * s);       // blocks j = s, 3s, .. < P
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= per * p.L.nsys) return;
  const int64_t t = id / per;
  const int64_t j = s == 0 ? 0 : s + (id % per) * 2 * s;
  if (j >= p.P) return;
  const int64_t g = t * p.P + j;
  if (p.flags[p.L.sys(t)] & 1) return;
  T M[NB][NB], R[NB][1];
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    T v = rec_g<T, K>(p, g)[r];
    if (s > 0) {
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        v = fma(-rec_L<T, K>(p, g)[r * NB + q], p.y[(g - s) * NB + q], v);
        if (j + s < p.P) v = fma(-rec_U<T, K>(p, g)[r * NB + q], p.y[(g + s) * NB + q], v);
      }
    }
    R[r][0] = v;
#pragma unroll
    for (int q = 0; q < NB; ++q) M[r][q] = rec_D<T, K>(p, g)[r * NB + q];
  }
  if (!small_solve<T, NB, 1>(M, R)) {
    set_flag(p.flags, p.L.sys(t), 1);
    return;
  }
#pragma unroll
  for (int r = 0; r < NB; ++r) p.y[g * NB + r] = R[r][0];
}

// ---------------------------------------------------------------- phase 3
template <typename T, int K>
__global__ void __launch_bounds__(64, 8) k_grid_back(const GridArgs<T> p) {
  constexpr int NB = 2 * K;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= p.C) return;
  const int64_t t = g / p.P, k = g % p.P;
  const int64_t s = p.L.sys(t);
  if (p.flags[s] & 1) return;
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  int64_t s0, L;
  chunk_rows(n, p.P, k, s0, L);
  const int64_t C = p.C;
  T u[K], v[K];
#pragma unroll
  for (int m = 0; m < K; ++m) {
    u[m] = k > 0 ? p.y[(g - 1) * NB + K + m] : T(0);
    v[m] = k + 1 < p.P ? p.y[(g + 1) * NB + m] : T(0);
  }
  const T* zw = rec_zw<T, K>(p, g);
  const T zw1_1 = zw[0], zw1_2 = zw[1], zw2_1 = zw[2];
  T x1 = 0, x2 = 0;
  bool bad = false;
  constexpr int kB = 4;
  for (int64_t top = L - 1; top >= 0; top -= kB) {
    T av[kB], bv[kB], fv[kB], v1[kB], v2[kB];
#pragma unroll
    for (int e = 0; e < kB; ++e) {
      av[e] = bv[e] = fv[e] = v1[e] = v2[e] = T(0);
      const int64_t j = top - e;
      if (j >= 0) {
        const int64_t w = j * C + g;
        av[e] = p.al[w];
        fv[e] = p.zf[w];
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
  if (bad) set_flag(p.flags, s, 2);
}

template <typename T>
__global__ void __launch_bounds__(128) k_grid_status(const GridArgs<T> p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.L.nsys) return;
  const int64_t s = p.L.sys(t);
  const int32_t f = p.flags[s];
  set_status(p.status, s, (f & 1) ? BAND_ERR_ZERO_PIVOT : ((f & 2) ? BAND_ERR_NONFINITE : BAND_OK));
}

// Chunks per system: one wave of 16 warps per SM over the whole batch, chunks of at
// least kGridMinRows rows (one chunk for a system shorter than two of them).
constexpr int64_t kGridMinRows = 64;

}  // namespace

int64_t grid_chunks(const band_desc* d) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 152;
  const int64_t lanes = (int64_t)nsm * 16 * 32;
  const int64_t nsys = d->nsys > 0 ? d->nsys : 1;
  int64_t P = lanes / nsys;
  const int64_t cap = d->n / kGridMinRows;
  if (P > cap) P = cap;
  if (P < 1) P = 1;
  return P;
}

// Workspace: five (PD) / four (TD) chunk-major scratch arrays of ceil(n / P) * C rows,
// the C records and boundary unknowns, and the per-system flags.
struct GridWs {
  void *al, *be, *zf, *zv1, *zv2, *rec, *y, *flags;
};
static GridWs carve_grid(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  GridWs w{};
  const int64_t P = grid_chunks(d);
  const int64_t C = P * d->nsys;
  const int64_t Lmax = (d->n + P - 1) / P;
  const size_t es = dtype_size(d->dtype);
  const size_t rows = (size_t)Lmax * (size_t)C * es;
  const bool pd = d->half_bw == 2;
  w.al = c.take(rows);
  w.zf = c.take(rows);
  w.zv1 = c.take(rows);
  if (pd) {
    w.be = c.take(rows);
    w.zv2 = c.take(rows);
  }
  w.rec = c.take((size_t)C * (size_t)(pd ? rec_words<2>() : rec_words<1>()) * es);
  w.y = c.take((size_t)C * (size_t)(pd ? 4 : 2) * es);
  w.flags = c.take(sizeof(int32_t) * (size_t)(d->nsys > 0 ? d->nsys : 1));
  *bytes = c.size();
  return w;
}

size_t grid_workspace_bytes(const band_desc* d) {
  size_t b = 0;
  carve_grid(d, nullptr, &b);
  return b;
}

template <typename T, int K>
static cudaError_t run_grid(const GridArgs<T>& p, cudaStream_t st) {
  const unsigned g1 = (unsigned)((p.C + 63) / 64);
  k_grid_chunks<T, K><<<g1, 64, 0, st>>>(p);
  int64_t top = 1;
  for (int64_t s = 1; s < p.P; s *= 2) {
    const int64_t th = (p.P + 2 * s - 1) / (2 * s) * p.L.nsys;
    k_grid_reduce<T, K><<<(unsigned)((th + 127) / 128), 128, 0, st>>>(p, s);
    top = s;
  }
  k_grid_expand<T, K><<<(unsigned)((p.L.nsys + 127) / 128), 128, 0, st>>>(p, 0);
  for (int64_t s = top; s >= 1; s /= 2) {
    const int64_t th = (p.P + s) / (2 * s) * p.L.nsys;
    k_grid_expand<T, K><<<(unsigned)((th + 127) / 128), 128, 0, st>>>(p, s);
  }
  k_grid_back<T, K><<<g1, 64, 0, st>>>(p);
  k_grid_status<T><<<(unsigned)((p.L.nsys + 127) / 128), 128, 0, st>>>(p);
  return cudaGetLastError();
}

// band_solve on the grid schedule (uniform layouts, NTDM / NPDM, no stored factors).
band_status grid_solve(const band_desc* desc, int32_t method, const void* const diag[5],
                       const void* f, void* x, int32_t* sys_status, void* ws, size_t ws_bytes,
                       cudaStream_t st) {
  const int kmode = kmode_for(desc, method);
  if (kmode != 1 && kmode != 2) return BAND_ERR_ARG;
  if (is_symbolic(method) || desc->offsets || desc->chunks) return BAND_ERR_ARG;
  if (!diag || !f || !x || !diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (kmode == 2 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  size_t need = 0;
  carve_grid(desc, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const GridWs w = carve_grid(desc, ws, &need);
  if (cudaMemsetAsync(w.flags, 0, sizeof(int32_t) * (size_t)desc->nsys, st) != cudaSuccess)
    return BAND_ERR_CUDA;
  const int64_t P = grid_chunks(desc);
  const Layout L = layout_of(desc);
  cudaError_t e;
  if (desc->dtype == BAND_F64) {
    GridArgs<double> p{L, (const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
                       (const double*)diag[3], (const double*)diag[4], (const double*)f,
                       (double*)x, (double*)w.al, (double*)w.be, (double*)w.zf, (double*)w.zv1,
                       (double*)w.zv2, (double*)w.rec, (double*)w.y, (int32_t*)w.flags,
                       sys_status, P, P * desc->nsys};
    e = kmode == 2 ? run_grid<double, 2>(p, st) : run_grid<double, 1>(p, st);
  } else {
    GridArgs<float> p{L, (const float*)diag[0], (const float*)diag[1], (const float*)diag[2],
                      (const float*)diag[3], (const float*)diag[4], (const float*)f, (float*)x,
                      (float*)w.al, (float*)w.be, (float*)w.zf, (float*)w.zv1, (float*)w.zv2,
                      (float*)w.rec, (float*)w.y, (int32_t*)w.flags, sys_status, P,
                      P * desc->nsys};
    e = kmode == 2 ? run_grid<float, 2>(p, st) : run_grid<float, 1>(p, st);
  }
  return cuda_status(e);
}

}  // namespace band
