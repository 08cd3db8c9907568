// common.cuh -- device helpers shared by the libband kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "band.h"

namespace band {

constexpr int kWarp = 32;

__host__ __device__ inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Where the rows of one system live.  Uniform batches: element i of system s at
// s*sys_stride + i*elem_stride.  Ragged batches (n == 0): offsets[s] + i.
struct Layout {
  int64_t nsys, n, ss, es;
  const int64_t* offsets;
  const int8_t* hbw;
  const int64_t* ids;     // ragged subsets: the batch's s-th system is ids[s]
  int64_t extent;         // elements one array spans (the last valid index + 1)
  int32_t half_bw;
  // id of the batch's s-th system (the index of every per-system array)
  __device__ __forceinline__ int64_t sys(int64_t s) const { return ids ? ids[s] : s; }
  __device__ __forceinline__ int64_t base(int64_t s) const { return offsets ? offsets[s] : s * ss; }
  __device__ __forceinline__ int64_t rows(int64_t s) const {
    return offsets ? offsets[s + 1] - offsets[s] : n;
  }
  __device__ __forceinline__ int64_t stride() const { return offsets ? 1 : es; }
  __device__ __forceinline__ int kband(int64_t s) const { return hbw ? (int)hbw[s] : half_bw; }
};

// Scratch rows of one system: interleaved (row i of the batch's t-th system at i*S + t,
// S = nsys rounded up to a warp) for uniform batches and for ragged batches with an id
// list, packed like the data (offsets[t]) for other ragged batches.
struct Spill {
  int64_t S;
  const int64_t* offsets;
  __device__ __forceinline__ int64_t base(int64_t s) const { return offsets ? offsets[s] : s; }
  __device__ __forceinline__ int64_t stride() const { return offsets ? 1 : S; }
};

// ---------------------------------------------------------------- reciprocals
// 1/m in FP64 from an FP32 seed refined by the Newton-Raphson iteration for the
// reciprocal in its third-order form (the truncated series r0 (1 + e + e^2) of
// 1/m = r0 / (1 - e), as in Markstein's division and reciprocal sequences).
// The seed: the double's exponent is rebased into float range with integer ops (the
// leading 20 mantissa bits are kept), rcp.approx.f32 gives ~22 correct bits, and the
// result is rebased back.  With e = 1 - m r0 (|e| < 2^-19), one step
// r = r0 + r0 (e + e^2) leaves a relative error of order e^3 < 2^-57 before the final
// rounding, so the result is within one ulp of the correctly rounded 1/m
// (tests/test_gpu_rcp64.py checks that against IEEE division).  Outside the exponent window where the
// rebasing is valid (|m| roughly in [2^-120, 2^120]) and for 0, Inf and NaN the
// division is used instead.
__device__ __forceinline__ double rcp64(double m) {
  const unsigned hi = (unsigned)__double2hiint(m);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex - 903u > 240u) return 1.0 / m;
  const unsigned fb = (hi & 0x80000000u) | (((hi & 0x7fffffffu) - (896u << 20)) << 3);
  float r0f;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"(__uint_as_float(fb)));
  const unsigned rb = __float_as_uint(r0f);
  const unsigned rh = (rb & 0x80000000u) | (((rb & 0x7fffffffu) >> 3) + (896u << 20));
  const double r0 = __hiloint2double((int)rh, (int)(rb << 29));
  const double e = fma(-m, r0, 1.0);
  return fma(r0, fma(e, e, e), r0);
}

__device__ __forceinline__ float rcp32(float m) { return __frcp_rn(m); }

template <typename T>
__device__ __forceinline__ T rcp(T m);
template <>
__device__ __forceinline__ double rcp<double>(double m) { return rcp64(m); }
template <>
__device__ __forceinline__ float rcp<float>(float m) { return rcp32(m); }

// Tests on doubles done on their bit patterns with integer instructions: the FP64 pipe
// of GB300 is the scarce unit of these kernels, so comparisons stay off it.
__device__ __forceinline__ bool is_zero(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float v) { return v == 0.0f; }
__device__ __forceinline__ bool not_finite(double v) {
  return ((unsigned)__double2hiint(v) & 0x7ff00000u) == 0x7ff00000u;
}
__device__ __forceinline__ bool not_finite(float v) { return !isfinite(v); }
// max(acc, |v|) for acc >= 0 by integer comparison of the bit patterns (NaN wins).
__device__ __forceinline__ double max_abs(double acc, double v) {
  const long long a = __double_as_longlong(acc);
  const long long b = __double_as_longlong(v) & 0x7fffffffffffffffLL;
  return __longlong_as_double(a > b ? a : b);
}

template <typename T>
__device__ __forceinline__ bool finite(T v) { return !not_finite(v); }

// read-only global load (the diagonals are never written by any kernel)
template <typename T>
__device__ __forceinline__ T ldro(const T* p) { return __ldg(p); }

__device__ __forceinline__ void set_status(int32_t* st, int64_t s, int32_t v) {
  if (st) st[s] = v;
}

// Biased binary exponent of a value (0 for zero, all ones for Inf / NaN), by integer
// operations.
__device__ __forceinline__ int expo_of(double v) {
  return (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu);
}
__device__ __forceinline__ int expo_of(float v) { return (int)((__float_as_uint(v) >> 23) & 0xffu); }

// Gaussian elimination with partial pivoting on an NU x NU system (augmented column
// NU), fully unrolled: row exchanges are selects, so M stays in registers.  Returns
// false on a zero pivot, and with guard > 0 also on a pivot whose binary exponent lies
// guard or more below that of the largest coefficient of M.
template <typename T, int NU>
__device__ __forceinline__ bool solve_small(T (&M)[4][5], int guard = 0) {
  int top = 0;
  if (guard > 0) {
#pragma unroll
    for (int r = 0; r < NU; ++r)
#pragma unroll
      for (int k = 0; k < NU; ++k) top = max(top, expo_of(M[r][k]));
  }
#pragma unroll
  for (int c = 0; c < NU; ++c) {
    int piv = c;
    T big = fabs(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < NU; ++r)
      if (fabs(M[r][c]) > big) { big = fabs(M[r][c]); piv = r; }
#pragma unroll
    for (int r = c + 1; r < NU; ++r) {
      const bool sw = (r == piv);
#pragma unroll
      for (int k = c; k <= NU; ++k) {
        const T u = M[c][k], v = M[r][k];
        M[c][k] = sw ? v : u;
        M[r][k] = sw ? u : v;
      }
    }
    if (is_zero(M[c][c])) return false;
    if (guard > 0 && expo_of(M[c][c]) + guard <= top) return false;
    const T inv = T(1) / M[c][c];
#pragma unroll
    for (int r = c + 1; r < NU; ++r) {
      const T l = M[r][c] * inv;
#pragma unroll
      for (int k = c; k <= NU; ++k) M[r][k] = fma(-l, M[c][k], M[r][k]);
    }
  }
#pragma unroll
  for (int c = NU - 1; c >= 0; --c) {
    T v = M[c][NU];
#pragma unroll
    for (int k = c + 1; k < NU; ++k) v = fma(-M[c][k], M[k][NU], v);
    M[c][NU] = v / M[c][c];
  }
  return true;
}

// ------------------------------------------------------------- async staging
// Each lane copies its own element of a row into shared memory with cp.async (LDGSTS)
// and later waits for the copy group of that row: rows are fetched kStage rows ahead
// without holding registers.  A lane only ever reads what it copied itself, so no
// barrier is involved.
__device__ __forceinline__ void cp_async_elem(void* smem, const double* g) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_elem(void* smem, const float* g) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// 16-byte copy global -> shared that bypasses L1 (cp.async.cg); both addresses 16-byte
// aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* g) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}

// Rows staged per warp: an FP64 row carries ~14 FP64 instructions (>1000 cycles with
// several warps per sub-partition), so 4 rows cover the memory latency; an FP32 row is
// cheap, so 16.  Row-ring bytes per warp for six arrays: 6 KiB (FP64) and 12 KiB (FP32);
// a warp's staging area is the larger of that and the granule ring.
template <typename T> struct StageDepth;
template <> struct StageDepth<double> { static constexpr int value = 4; };
template <> struct StageDepth<float> { static constexpr int value = 16; };
constexpr int kStageArrays = 6;
// Granules staged ahead (GranRing, below): 2 x 2 FP64 rows and 4 x 4 FP32 rows, the
// same shared memory as the row ring (a larger FP64 ring shrinks the L1 that the other
// tasks of a batched launch read through: measured 4.85 -> 7.2 ms on the ADI step).
template <typename T> struct GranDepth;
template <> struct GranDepth<double> { static constexpr int value = 2; };
template <> struct GranDepth<float> { static constexpr int value = 4; };
template <typename T>
__host__ __device__ constexpr int stage_bytes_per_warp() {
  return StageDepth<T>::value * kStageArrays * 32 * (int)sizeof(T) >
                 GranDepth<T>::value * kStageArrays * 32 * 16
             ? StageDepth<T>::value * kStageArrays * 32 * (int)sizeof(T)
             : GranDepth<T>::value * kStageArrays * 32 * 16;
}
// Warps per block of the single-problem sweeps (k_direct, k_twisted).  Measured on
// GB300: FP64 gains from one warp per block (the hardware spreads the warps over more
// SMs: 2048 x 2048 two-sided NPDM 0.84 -> 0.81 ms, 16384 x 4096 2.31 -> 2.10 ms); FP32
// with its deeper staging ring keeps four (16384 x 4096 two-sided 0.86 ms vs 0.96).
template <typename T> struct SweepWarps;
template <> struct SweepWarps<double> { static constexpr int value = 1; };
template <> struct SweepWarps<float> { static constexpr int value = 4; };
// Resident warps per SM the sweeps are compiled for (128 registers a thread).  Large
// batches then fit in fewer waves: k_twisted<double> at its free 152 registers held 13
// warps per SM, so 32768 PD systems of n = 2048 (2048 warps) needed a second, almost
// empty wave and took 3.08 ms against 2.07 ms on one thread per system.
constexpr int kSweepWarpsPerSm = 16;

// Staging of rows that each lane reads from its own contiguous system (contiguous and
// ragged layouts): 16-byte granules (2 FP64 / 4 FP32 rows) of every array, D granules
// ahead of the sweep, copied with cp.async.cg into a per-lane ring.  A warp touches 32
// lines per row there; through L1 those lines are evicted by the other warps' before
// their next row, so the rows go around L1.  A granule that would reach past the
// arrays' last element (`extent`) is copied element by element.
template <typename T, int NA, int D>
struct GranRing {
  static constexpr int E = 16 / (int)sizeof(T);
  T* sm;     // D x NA x 32 granules
  int lane;
  __device__ __forceinline__ T* at(int slot, int a) const {
    return sm + ((((slot * NA + a) << 5) + lane) * E);
  }
  __device__ __forceinline__ void issue(int slot, const T* const* src, int64_t g,
                                        int64_t extent) const {
    const int64_t e = g * E;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      if (e + E <= extent) {
        cp_async16(at(slot, a), src[a] + e);
      } else {
        for (int k = 0; k < E; ++k)
          if (e + k < extent) cp_async_elem(at(slot, a) + k, src[a] + e + k);
      }
    }
    cp_async_commit();
  }
  __device__ __forceinline__ T get(int slot, int a, int off) const { return at(slot, a)[off]; }
  static constexpr int bytes() { return D * NA * 32 * 16; }
};

// Ring of D rows x NA arrays x 32 lanes for one warp.
template <typename T, int NA, int D>
struct RowRing {
  T* sm;
  int lane;
  __device__ __forceinline__ T* at(int slot, int a) const { return sm + ((slot * NA + a) << 5) + lane; }
  __device__ __forceinline__ void issue(int slot, const T* const* src, int64_t q) const {
#pragma unroll
    for (int a = 0; a < NA; ++a) cp_async_elem(at(slot, a), src[a] + q);
    cp_async_commit();
  }
  __device__ __forceinline__ void skip() const { cp_async_commit(); }
  __device__ __forceinline__ T get(int slot, int a) const { return *at(slot, a); }
};

}  // namespace band
