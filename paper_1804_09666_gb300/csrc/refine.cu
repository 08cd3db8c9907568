// refine.cu -- FP32 factor/solve with iterative refinement to FP64 accuracy.
//
// The systems are stored in FP32; the right-hand side and the solution are FP64.
//   x_1 = solve32(f)                    (f rounded to FP32)
//   step k >= 1:  r = f - A x_k         (A = the exact values of the FP32 diagonals)
//                 x_{k+1} = x_k + 2^e solve32(2^-e r)
// until max|x_{k+1} - x_k| <= rel_stop max|x_{k+1}| or max_steps steps.
// solve32 is NPDM / NTDM (Veneva & Ayriyan, Sec. 1) in single precision, run by the
// library's sweep kernels on the schedule the descriptor asks for (two-sided by
// default); 2^e is a power of two fixed per system from max|f| (exact scaling that
// keeps the FP32 right-hand side in range).
//
// Each step is made of passes that the GPU runs at full width:
//   update    x += 2^e delta (elementwise), with max|2^e delta| and max|x| per system
//   decide    per system: stop (converged, non-finite, zero pivot, cap) or go on
//   residual  r = f - A x (a five-point stencil, elementwise), written as 2^-e r in FP32
//   solve     delta = solve32(2^-e r) for the systems still going
// x, f, the residual and the update are kept in one of two forms:
//  * FP64 (the default): x in the caller's FP64 array, r = f - A x with FP64 fused
//    multiply-adds (A widened exactly from FP32 by integer operations), x += 2^e delta
//    with one FP64 fused multiply-add;
//  * FP32 pairs (BAND_REFINE_PAIRS): GB300 runs FP64 at 1/64 of the FP32 rate, so x, f,
//    the residual and the update are pairs of FP32 numbers handled with error-free
//    transformations (TwoProd with an FMA, TwoSum): about 2^-48 relative accuracy,
//    ample for the 1e-10 target; f is split into a pair once (integer bit operations),
//    x is assembled in FP64 once, at the end.
#include <cuda_runtime.h>

#include "api_util.h"
#include "kernels.h"

namespace band {
namespace {

// ------------------------------------------------------------- FP32 pairs
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return F2{s, e};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = a * b;
  return F2{p, fmaf(a, b, -p)};
}

// float -> double exactly, with integer operations for normal numbers.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)f;   // zero, subnormal, Inf, NaN
  const unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
  return __hiloint2double((int)hi, (int)(u << 29));
}

// double -> (h, l): h is v cut to 24 significant bits, l the float nearest v - h, so
// h + l = v to 2^-48 relative; integer operations for |v| in [2^-100, 2^100].
__device__ __forceinline__ F2 split(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned ex = (unsigned)(b >> 52) & 0x7ffu;
  if (ex - 923u > 200u) {                 // outside the window: FP64 conversions
    const float h = __double2float_rz(v);
    return F2{h, __double2float_rn(v - (double)h)};
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned hb = sign | ((ex - 896u) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rem = (unsigned)(b & 0x1fffffffu);               // the 29 low bits
  // rem * 2^(ex - 1075) = (rem * 2^-29) * 2^(ex - 1046), both factors normal floats
  const float scale = __uint_as_float((ex - 1046u + 127u) << 23);
  const float l = __uint2float_rn(rem) * 0x1p-29f * scale;
  return F2{__uint_as_float(hb), sign ? -l : l};
}

// s = s - a * x for an FP32 coefficient a and a pair x.
__device__ __forceinline__ void sub_prod(F2& s, float a, const F2& x) {
  const F2 p = two_prod(a, x.h);
  const F2 t = two_sum(s.h, -p.h);
  s.h = t.h;
  s.l = s.l + t.l - p.l - a * x.l;
}

// 2^k as a float (k clamped to the normal range)
__device__ __forceinline__ float pow2f(int k) {
  k = k < -126 ? -126 : (k > 127 ? 127 : k);
  return __uint_as_float((unsigned)(k + 127) << 23);
}

// ------------------------------------------------------------ refinement state
struct RefState {
  Layout L;
  const float *a, *b, *c, *d, *e;
  const double* f;
  double* x;
  float* r32;                    // 2^-e r (the correction solve's right-hand side)
  float* d32;                    // delta (the correction solve's solution)
  float *xh, *xl;                // x as a pair of floats (x = xh + xl to ~2^-48)
  float *fh, *fl;                // f as a pair of floats
  int32_t* done;                 // per system: refinement finished
  int32_t* sst;                  // per system: status of the last FP32 solve
  int32_t* fexp;                 // per system: e
  unsigned int* xmax;            // per system: max|x| (bit pattern of a float >= 0)
  unsigned int* dmax;            // per system: max|2^e delta| (bit pattern of a float >= 0)
  unsigned int* rmax;            // per system: max|r| (float bits; NaN and Inf on top)
  unsigned long long* fmax;      // per system: max|f|
  int32_t *steps, *status;
  double rel_stop;
  int max_steps;
  int fp64;                      // 1: x, r and the update in FP64; 0: FP32 pairs
};

constexpr int kChunk = 32;       // rows per thread in the elementwise passes

// Thread t of an elementwise pass: system (the fastest index, for coalescing on
// interleaved data) and chunk of kChunk rows.
__device__ __forceinline__ bool chunk_of(const Layout& L, int64_t t, int64_t& s, int64_t& i0,
                                         int64_t& i1) {
  const int64_t nch = (L.n + kChunk - 1) / kChunk;
  if (t >= L.nsys * nch) return false;
  s = t % L.nsys;
  const int64_t c = t / L.nsys;
  const int64_t n = L.rows(s);
  i0 = c * kChunk;
  i1 = i0 + kChunk < n ? i0 + kChunk : n;
  return i0 < n;
}

// The elementwise passes load kBatch rows before using any of them, so that a thread
// has several loads of each array in flight (one at a time, the passes ran at 40 % of
// HBM bandwidth, bound by memory latency).  x and f are kept as float pairs in the
// workspace during the iteration; x is assembled in FP64 once at the end.
#ifndef REF_BATCH
#define REF_BATCH 2
#endif
#ifndef REF_MINB
#define REF_MINB 4
#endif
constexpr int kBatch = REF_BATCH;

// Pass 0: the first right-hand side f rounded to FP32, f as a pair; max|f| per system.
__global__ void __launch_bounds__(256) k_ref_start(const RefState p) {
  int64_t s, i0, i1;
  if (!chunk_of(p.L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, s, i0, i1)) return;
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  double m = 0.0;
  for (int64_t ib = i0; ib < i1; ib += kBatch) {
    double fv[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) fv[u] = (ib + u < i1) ? p.f[q0 + (ib + u) * es] : 0.0;
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      if (ib + u < i1) {
        const int64_t q = q0 + (ib + u) * es;
        p.r32[q] = __double2float_rn(fv[u]);
        if (!p.fp64) {
          const F2 fp = split(fv[u]);
          p.fh[q] = fp.h;
          p.fl[q] = fp.l;
        }
        m = max_abs(m, fv[u]);
      }
    }
  }
  atomicMax(p.fmax + s, (unsigned long long)__double_as_longlong(m));
}

// x += 2^e delta (first: x = delta, the unscaled first solve), with the maxima.
__global__ void __launch_bounds__(256, REF_MINB) k_ref_update(const RefState p, int first) {
  int64_t s, i0, i1;
  if (!chunk_of(p.L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, s, i0, i1)) return;
  if (p.done[s]) return;
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  const float up = pow2f(p.fexp[s]);
  float dm = 0.0f, xm = 0.0f;
  bool nan_d = false, nan_x = false;
  if (p.fp64) {
    const double up64 = (double)up;
    for (int64_t ib = i0; ib < i1; ib += kBatch) {
      float dv[kBatch];
      double xv[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const bool in = ib + u < i1;
        const int64_t q = q0 + (ib + u) * es;
        dv[u] = in ? p.d32[q] : 0.0f;
        xv[u] = (in && !first) ? p.x[q] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (ib + u >= i1) break;
        const int64_t q = q0 + (ib + u) * es;
        double xn;
        if (first) {
          xn = f2d(dv[u]);
        } else {
          const float dd = dv[u] * up;                // exact: a power of two
          nan_d |= (dd != dd);
          dm = fmaxf(dm, fabsf(dd));
          xn = fma(f2d(dv[u]), up64, xv[u]);
        }
        p.x[q] = xn;
        const float xf = (float)xn;
        nan_x |= !isfinite(xf);
        xm = fmaxf(xm, fabsf(xf));
      }
    }
  } else {
    for (int64_t ib = i0; ib < i1; ib += kBatch) {
      float dv[kBatch], hv[kBatch], lv[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const bool in = ib + u < i1;
        const int64_t q = q0 + (ib + u) * es;
        dv[u] = in ? p.d32[q] : 0.0f;
        hv[u] = (in && !first) ? p.xh[q] : 0.0f;
        lv[u] = (in && !first) ? p.xl[q] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if (ib + u >= i1) break;
        const int64_t q = q0 + (ib + u) * es;
        F2 xn;
        if (first) {
          xn = F2{dv[u], 0.0f};
        } else {
          const float dd = dv[u] * up;                  // exact: a power of two
          nan_d |= (dd != dd);
          dm = fmaxf(dm, fabsf(dd));
          const F2 t1 = two_sum(hv[u], dd);
          xn = two_sum(t1.h, t1.l + lv[u]);
        }
        p.xh[q] = xn.h;
        p.xl[q] = xn.l;
        nan_x |= !isfinite(xn.h);
        xm = fmaxf(xm, fabsf(xn.h));
      }
    }
  }
  // a NaN wins the max (its bits order above every finite float and Inf)
  if (!first) atomicMax(p.dmax + s, nan_d ? 0x7fc00000u : __float_as_uint(dm));
  atomicMax(p.xmax + s, nan_x ? 0x7fc00000u : __float_as_uint(xm));
}

// r = f - A x in FP64 (A widened exactly from FP32); 2^-e r to r32.
template <int K>
__device__ __forceinline__ void residual_rows64(const RefState& p, int64_t s, int64_t i0,
                                                int64_t i1) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const double down = (double)pow2f(-p.fexp[s]);
  float rm = 0.0f;
  bool nan_r = false;
  auto X = [&](int64_t j) -> double { return (j >= 0 && j < n) ? p.x[q0 + j * es] : 0.0; };
  double w0 = X(i0 - 2), w1 = X(i0 - 1), w2 = X(i0), w3 = X(i0 + 1);   // x_{i-2} .. x_{i+1}
  for (int64_t ib = i0; ib < i1; ib += kBatch) {
    double xv[kBatch], fv[kBatch];
    float av[kBatch], bv[kBatch], cv[kBatch], dv[kBatch], ev[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = ib + u;
      const bool in = i < i1;
      const int64_t q = q0 + (in ? i : i0) * es;
      xv[u] = in ? X(i + 2) : 0.0;
      fv[u] = in ? p.f[q] : 0.0;
      cv[u] = in ? ldro(p.c + q) : 0.0f;
      bv[u] = (in && i >= 1) ? ldro(p.b + q) : 0.0f;
      dv[u] = (in && i + 1 < n) ? ldro(p.d + q) : 0.0f;
      av[u] = (K == 2 && in && i >= 2) ? ldro(p.a + q) : 0.0f;
      ev[u] = (K == 2 && in && i + 2 < n) ? ldro(p.e + q) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = ib + u;
      if (i >= i1) break;
      const double w4 = xv[u];                        // x_{i+2}
      double r = fma(-f2d(cv[u]), w2, fv[u]);
      r = fma(-f2d(bv[u]), w1, r);
      r = fma(-f2d(dv[u]), w3, r);
      if (K == 2) {
        r = fma(-f2d(av[u]), w0, r);
        r = fma(-f2d(ev[u]), w4, r);
      }
      const float rv = (float)(r * down);
      p.r32[q0 + i * es] = rv;
      const float ra = (float)fabs(r);
      nan_r |= (ra != ra);
      rm = fmaxf(rm, ra);
      w0 = w1; w1 = w2; w2 = w3; w3 = w4;
    }
  }
  atomicMax(p.rmax + s, nan_r ? 0x7fc00000u : __float_as_uint(rm));
}

// r = f - A x in FP32 pairs (A exact in FP32); 2^-e r to r32.
template <int K>
__device__ __forceinline__ void residual_rows(const RefState& p, int64_t s, int64_t i0,
                                              int64_t i1) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const float down = pow2f(-p.fexp[s]);
  float rm = 0.0f;
  bool nan_r = false;
  auto X = [&](int64_t j) -> F2 {
    return (j >= 0 && j < n) ? F2{p.xh[q0 + j * es], p.xl[q0 + j * es]} : F2{0.0f, 0.0f};
  };
  F2 w0 = X(i0 - 2), w1 = X(i0 - 1), w2 = X(i0), w3 = X(i0 + 1);   // x_{i-2} .. x_{i+1}
  for (int64_t ib = i0; ib < i1; ib += kBatch) {
    F2 xv[kBatch], fv[kBatch];
    float av[kBatch], bv[kBatch], cv[kBatch], dv[kBatch], ev[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = ib + u;
      const bool in = i < i1;
      const int64_t q = q0 + (in ? i : i0) * es;
      xv[u] = in ? X(i + 2) : F2{0.0f, 0.0f};
      fv[u] = in ? F2{p.fh[q], p.fl[q]} : F2{0.0f, 0.0f};
      cv[u] = in ? ldro(p.c + q) : 0.0f;
      bv[u] = (in && i >= 1) ? ldro(p.b + q) : 0.0f;
      dv[u] = (in && i + 1 < n) ? ldro(p.d + q) : 0.0f;
      av[u] = (K == 2 && in && i >= 2) ? ldro(p.a + q) : 0.0f;
      ev[u] = (K == 2 && in && i + 2 < n) ? ldro(p.e + q) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int64_t i = ib + u;
      if (i >= i1) break;
      const F2 w4 = xv[u];                            // x_{i+2}
      F2 r = fv[u];
      sub_prod(r, cv[u], w2);
      sub_prod(r, bv[u], w1);
      sub_prod(r, dv[u], w3);
      if (K == 2) {
        sub_prod(r, av[u], w0);
        sub_prod(r, ev[u], w4);
      }
      const float rv = r.h + r.l;
      p.r32[q0 + i * es] = rv * down;
      nan_r |= (rv != rv);
      rm = fmaxf(rm, fabsf(rv));
      w0 = w1; w1 = w2; w2 = w3; w3 = w4;
    }
  }
  atomicMax(p.rmax + s, nan_r ? 0x7fc00000u : __float_as_uint(rm));
}

// x in FP64 from its pair, for every system, at the end.
__global__ void __launch_bounds__(256) k_ref_finish(const RefState p) {
  int64_t s, i0, i1;
  if (p.fp64) return;                 // x is FP64 throughout
  if (!chunk_of(p.L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, s, i0, i1)) return;
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  for (int64_t ib = i0; ib < i1; ib += kBatch) {
    float hv[kBatch], lv[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const bool in = ib + u < i1;
      const int64_t q = q0 + (ib + u) * es;
      hv[u] = in ? p.xh[q] : 0.0f;
      lv[u] = in ? p.xl[q] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (ib + u < i1) p.x[q0 + (ib + u) * es] = f2d(hv[u]) + f2d(lv[u]);
  }
}

__global__ void __launch_bounds__(256, REF_MINB) k_ref_residual(const RefState p, int kmode) {
  int64_t s, i0, i1;
  if (!chunk_of(p.L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, s, i0, i1)) return;
  if (p.done[s]) return;
  const int K = kmode ? kmode : p.L.kband(s);
  if (p.fp64) {
    if (K == 1) residual_rows64<1>(p, s, i0, i1);
    else residual_rows64<2>(p, s, i0, i1);
  } else {
    if (K == 1) residual_rows<1>(p, s, i0, i1);
    else residual_rows<2>(p, s, i0, i1);
  }
}

// After step k's update (k corrections applied, k >= 0): stop or go on, and clear the
// maxima for the next step.  rmax is that of the residual the k-th correction was
// solved from (k >= 1): zero means the previous x solved the system exactly (the
// correction is then 0 and the step converged anyway).  One thread per system.
__global__ void __launch_bounds__(256) k_ref_decide(const RefState p, int k) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys || p.done[s]) return;
  int32_t st = -1;                              // -1: go on
  const float xm = __uint_as_float(p.xmax[s]);
  const float dm = __uint_as_float(p.dmax[s]);
  const float rm = __uint_as_float(p.rmax[s]);
  if (p.sst[s] != BAND_OK) st = p.sst[s];                       // the last solve failed
  else if (!isfinite(xm) || !(dm == dm) || !(rm == rm) || isinf(rm)) st = BAND_ERR_NONFINITE;
  else if (k >= 1 && (double)dm <= p.rel_stop * (double)xm) st = BAND_OK;   // converged
  else if (k >= p.max_steps) st = BAND_OK;                       // the cap
  if (st >= 0) {
    p.done[s] = 1;
    if (p.steps) p.steps[s] = p.sst[s] != BAND_OK ? (k > 0 ? k - 1 : 0) : k;
    set_status(p.status, s, st);
  }
  p.xmax[s] = 0u;
  p.dmax[s] = 0u;
  p.rmax[s] = 0u;
}

__global__ void __launch_bounds__(256) k_ref_init(const RefState p) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  const double fm = __longlong_as_double((long long)p.fmax[s]);
  // 2^e ~ max|f| 2^-20: the scaled residuals stay far inside FP32's range
  const int ex = (int)((unsigned)(__double_as_longlong(fm) >> 52) & 0x7ffu) - 1023;
  p.fexp[s] = ex - 20;
}

// ----------------------------------------------------------------- workspace
struct RefWs {
  float *r32, *d32, *xh, *xl, *fh, *fl;
  int32_t *done, *sst, *fexp;
  unsigned long long* fmax;
  unsigned int *xmax, *dmax, *rmax;
  void* solve;
  size_t solve_bytes;
};
RefWs carve_refine(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  RefWs w{};
  const size_t span = (size_t)layout_of(d).extent;
  const size_t ns = (size_t)(d->nsys > 0 ? d->nsys : 1);
  w.r32 = (float*)c.take(span * sizeof(float));
  w.d32 = (float*)c.take(span * sizeof(float));
  w.xh = (float*)c.take(span * sizeof(float));
  w.xl = (float*)c.take(span * sizeof(float));
  w.fh = (float*)c.take(span * sizeof(float));
  w.fl = (float*)c.take(span * sizeof(float));
  w.done = (int32_t*)c.take(ns * sizeof(int32_t));
  w.sst = (int32_t*)c.take(ns * sizeof(int32_t));
  w.fexp = (int32_t*)c.take(ns * sizeof(int32_t));
  w.fmax = (unsigned long long*)c.take(ns * sizeof(unsigned long long));
  w.xmax = (unsigned int*)c.take(ns * sizeof(unsigned int));
  w.dmax = (unsigned int*)c.take(ns * sizeof(unsigned int));
  w.rmax = (unsigned int*)c.take(ns * sizeof(unsigned int));
  size_t sb = 0;
  carve_solve(d, d->hbw ? BAND_AUTO_NUMERIC : (d->half_bw == 1 ? BAND_NTDM : BAND_NPDM), nullptr,
              &sb);
  w.solve = c.take(sb);
  w.solve_bytes = sb;
  *bytes = c.size();
  return w;
}

}  // namespace

size_t refine_workspace_bytes(const band_desc* d) {
  size_t b = 0;
  carve_refine(d, nullptr, &b);
  return b;
}

}  // namespace band

using namespace band;

extern "C" band_status band_refine_solve_ex(const band_desc* desc32, const void* const diag32[5],
                                            const double* f, double* x, double rel_stop,
                                            int32_t max_steps, int32_t flags, int32_t* steps,
                                            int32_t* sys_status, void* ws, size_t ws_bytes,
                                            void* stream) {
  if (!desc_ok(desc32) || desc32->dtype != BAND_F32 || desc32->systems) return BAND_ERR_ARG;
  if (desc32->schedule == BAND_SCHED_GRID) return BAND_ERR_ARG;
  if (flags & ~BAND_REFINE_PAIRS) return BAND_ERR_ARG;
  // the FP64 form updates x in place while later residuals still read f
  if (!(flags & BAND_REFINE_PAIRS) && (const void*)x == (const void*)f) return BAND_ERR_ARG;
  if (max_steps < 0 || !(rel_stop >= 0.0)) return BAND_ERR_ARG;
  if (desc32->nsys == 0) return BAND_OK;
  if (!diag32 || !f || !x) return BAND_ERR_ARG;
  if (!diag32[1] || !diag32[2] || !diag32[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc32) && (!diag32[0] || !diag32[4])) return BAND_ERR_ARG;
  if (!arrays_aligned(BAND_F32, diag32, nullptr, nullptr, sys_status) ||
      !aligned_all(8, {f, x}) || !aligned_all(4, {steps}))
    return BAND_ERR_ARG;
  size_t need = 0;
  carve_refine(desc32, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const RefWs w = carve_refine(desc32, ws, &need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int kmode = desc32->hbw ? 0 : desc32->half_bw;
  const int32_t method = kmode == 0 ? BAND_AUTO_NUMERIC : (kmode == 1 ? BAND_NTDM : BAND_NPDM);
  RefState p{};
  p.L = layout_of(desc32);
  p.a = (const float*)diag32[0]; p.b = (const float*)diag32[1]; p.c = (const float*)diag32[2];
  p.d = (const float*)diag32[3]; p.e = (const float*)diag32[4];
  p.f = f;
  p.x = x;
  p.r32 = w.r32; p.d32 = w.d32;
  p.xh = w.xh; p.xl = w.xl; p.fh = w.fh; p.fl = w.fl;
  p.done = w.done; p.sst = w.sst; p.fexp = w.fexp;
  p.xmax = w.xmax; p.dmax = w.dmax; p.rmax = w.rmax; p.fmax = w.fmax;
  p.steps = steps;
  p.status = sys_status;
  p.rel_stop = rel_stop;
  p.max_steps = max_steps;
  p.fp64 = (flags & BAND_REFINE_PAIRS) ? 0 : 1;
  const size_t ns = (size_t)desc32->nsys;
  // done, sst, fexp, then the maxima are contiguous from w.done on: clear them at once
  if (cudaMemsetAsync(w.done, 0, (size_t)((char*)w.rmax - (char*)w.done) + ns * sizeof(unsigned),
                      st) != cudaSuccess)
    return BAND_ERR_CUDA;
  // the correction solve: A32 d32 = r32, on the schedule the descriptor asks for
  DirectReq req;
  const band_status v = make_direct(desc32, method, diag32, w.r32, w.d32, w.sst, w.solve,
                                    w.solve_bytes, &req, 256);
  if (v != BAND_OK) return v;
  req.d32.skip = w.done;
  auto solve = [&]() -> cudaError_t {
    if (req.parts) return launch_partition<float>(req.d32, req.kmode, req.parts, st);
    return req.two_sided ? launch_twisted<float>(req.d32, req.kmode, st)
                         : launch_direct<float>(req.d32, req.kmode, st);
  };
  const int64_t nch = (desc32->n + kChunk - 1) / kChunk;
  const unsigned g_elem = (unsigned)((desc32->nsys * nch + 255) / 256);
  const unsigned g_sys = (unsigned)((desc32->nsys + 255) / 256);
  k_ref_start<<<g_elem, 256, 0, st>>>(p);
  k_ref_init<<<g_sys, 256, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess || solve() != cudaSuccess) return BAND_ERR_CUDA;
  // step k: apply the k-th solution (k = 0: x = delta), decide, and for the systems
  // that go on the residual and the next solve
  for (int k = 0; k <= max_steps; ++k) {
    k_ref_update<<<g_elem, 256, 0, st>>>(p, k == 0 ? 1 : 0);
    k_ref_decide<<<g_sys, 256, 0, st>>>(p, k);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    if (k == max_steps) break;
    k_ref_residual<<<g_elem, 256, 0, st>>>(p, kmode);
    if (cudaGetLastError() != cudaSuccess || solve() != cudaSuccess) return BAND_ERR_CUDA;
  }
  k_ref_finish<<<g_elem, 256, 0, st>>>(p);
  return cuda_status(cudaGetLastError());
}

extern "C" band_status band_refine_solve(const band_desc* desc32, const void* const diag32[5],
                                         const double* f, double* x, double rel_stop,
                                         int32_t max_steps, int32_t* steps, int32_t* sys_status,
                                         void* ws, size_t ws_bytes, void* stream) {
  return band_refine_solve_ex(desc32, diag32, f, x, rel_stop, max_steps, 0, steps, sys_status,
                              ws, ws_bytes, stream);
}
