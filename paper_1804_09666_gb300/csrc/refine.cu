// refine.cu -- FP32 factor/solve with iterative refinement to FP64 accuracy.
//
// The systems are stored in FP32; the right-hand side and the solution are FP64.
//   x_0 = solve32(f)
//   per step:  r = f - A x  (A = the exact values of the FP32 diagonals)
//              delta = 2^e solve32(2^-e r),  x = x + delta
// until max|delta| <= rel_stop max|x| or max_steps steps.  solve32 is the NPDM / NTDM
// recurrence (Veneva & Ayriyan, Sec. 1) in single precision; its factors (gamma, 1/mu,
// alpha, beta) are computed once and reused by every correction.  2^e is a power of two
// fixed per system from max|f| (exact scaling that keeps the FP32 right-hand side in
// range).
//
// GB300 runs FP64 at 1/64 of the FP32 rate, and one warp alone on a sub-partition
// issues one FP64 instruction per 64 cycles, so a residual in FP64 arithmetic would
// cost as much as the whole FP64 solve.  The residual and the update are therefore
// computed with pairs of FP32 numbers and error-free transformations (TwoProd with an
// FMA, TwoSum), giving about 2^-48 relative accuracy: ample for the 1e-10 target
// (refinement converges to the limit set by the residual's accuracy times kappa).
// Doubles are split into, and rebuilt from, such pairs with integer bit operations;
// one FP64 addition per row and step assembles the stored x.
//
// Passes over the rows (one thread per system):
//   F0  forward: factor + z = L^{-1} f                      (writes the factor rows, z)
//   B   backward: x = U^{-1} z (first time) or x += 2^e U^{-1} z (corrections), and the
//       residual of row i+2 once x_i .. x_{i+4} are final  (writes x, r)
//   F   forward: z = L^{-1} (2^-e r) through the stored factors
// then B, F, B, ... until the stop test.
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

// ------------------------------------------------------------------- rows
struct RefArgs {
  Layout L;
  Spill W;
  const float *a, *b, *c, *d, *e;
  const double* f;
  double* x;
  float *fa, *fb, *fg, *fr, *z, *r;   // factor rows, z and scaled residual (workspace)
  double rel_stop;
  int max_steps;
  int32_t *steps, *status;
};

// Row sources: either a cp.async ring (interleaved systems) or plain loads.
template <int NF, int ND, int D>
struct Ring2 {
  float* fs;     // D x NF x 32 floats
  double* ds;    // D x ND x 32 doubles
  int lane;
  __device__ __forceinline__ void issue(int slot, const float* const* fsrc, int64_t fq,
                                        const double* const* dsrc, int64_t dq) const {
#pragma unroll
    for (int a = 0; a < NF; ++a) cp_async_elem(fs + ((slot * NF + a) << 5) + lane, fsrc[a] + fq);
#pragma unroll
    for (int a = 0; a < ND; ++a) cp_async_elem(ds + ((slot * ND + a) << 5) + lane, dsrc[a] + dq);
    cp_async_commit();
  }
  __device__ __forceinline__ float getf(int slot, int a) const { return fs[((slot * NF + a) << 5) + lane]; }
  __device__ __forceinline__ double getd(int slot, int a) const { return ds[((slot * ND + a) << 5) + lane]; }
  static constexpr int bytes() { return D * 32 * (4 * NF + 8 * ND); }
};

constexpr int kRefWarps = 4;
constexpr int kDepthF0 = 16, kDepthB = 8, kDepthF = 16;
// ring bytes per warp of the passes (the largest sets the kernel's shared memory)
constexpr int kBytesF0 = Ring2<5, 1, kDepthF0>::bytes();     // a..e, f
constexpr int kBytesB = Ring2<8, 2, kDepthB>::bytes();       // a..e, alpha, beta, z, f, x
constexpr int kBytesF = Ring2<4, 0, kDepthF>::bytes();       // r, a, gamma, 1/mu
constexpr int kRefRingBytes =
    kBytesF0 > kBytesB ? (kBytesF0 > kBytesF ? kBytesF0 : kBytesF) : (kBytesB > kBytesF ? kBytesB : kBytesF);

template <int K, bool RING>
__device__ void refine_one(const RefArgs& p, int64_t s, unsigned char* stage) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  const int lane = threadIdx.x & 31;
  // TD systems may come without a and e: their loads read c instead (values unused)
  const float* pa = K == 2 ? p.a : p.c;
  const float* pe = K == 2 ? p.e : p.c;
  const float* A5[5] = {pa, p.b, p.c, p.d, pe};

  // ---- F0: FP32 factorisation and z = L^{-1} f ------------------------------
  double fmax = 0.0;
  bool zero = false;
  {
    constexpr int D = kDepthF0;
    const Ring2<5, 1, D> ring{reinterpret_cast<float*>(stage),
                              reinterpret_cast<double*>(stage + D * 32 * 4 * 5), lane};
    const double* F1[1] = {p.f};
    if (RING) {
#pragma unroll
      for (int j = 0; j < D - 1; ++j) {
        if (j < n) ring.issue(j, A5, q0 + j * es, F1, q0 + j * es);
        else cp_async_commit();
      }
    }
    float al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t q = q0 + i * es, w = w0 + i * ws;
      float av, bv, cv, dv, ev;
      double fv;
      if (RING) {
        const int64_t ip = i + D - 1;
        if (ip < n) ring.issue((int)(ip & (D - 1)), A5, q0 + ip * es, F1, q0 + ip * es);
        else cp_async_commit();
        cp_async_wait<D - 1>();
        const int sl = (int)(i & (D - 1));
        av = ring.getf(sl, 0); bv = ring.getf(sl, 1); cv = ring.getf(sl, 2);
        dv = ring.getf(sl, 3); ev = ring.getf(sl, 4); fv = ring.getd(sl, 0);
      } else {
        av = K == 2 ? ldro(pa + q) : 0.0f; bv = ldro(p.b + q); cv = ldro(p.c + q);
        dv = ldro(p.d + q); ev = K == 2 ? ldro(pe + q) : 0.0f; fv = p.f[q];
      }
      const float ai = (K == 2 && i >= 2) ? av : 0.0f;
      const float bi = (i >= 1) ? bv : 0.0f;
      const float di = (i + 1 < n) ? dv : 0.0f;
      const float ei = (K == 2 && i + 2 < n) ? ev : 0.0f;
      const float g = fmaf(-al2, ai, bi);
      const float m = fmaf(-al1, g, fmaf(-be2, ai, cv));
      if (m == 0.0f) { zero = true; break; }
      const float rr = __frcp_rn(m);
      const float alv = fmaf(-be1, g, di) * rr;
      const float bev = ei * rr;
      const float zv = fmaf(-z1, g, fmaf(-z2, ai, __double2float_rn(fv))) * rr;
      p.fa[w] = alv; p.fb[w] = bev; p.fg[w] = g; p.fr[w] = rr; p.z[w] = zv;
      fmax = max_abs(fmax, fv);
      al2 = al1; al1 = alv; be2 = be1; be1 = bev; z2 = z1; z1 = zv;
    }
    if (RING) cp_async_wait<0>();
  }
  if (zero) {
    if (p.steps) p.steps[s] = 0;
    set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
    return;
  }
  // residual scale 2^e with 2^e ~ max|f| 2^-20 (exact power of two)
  int fexp = ((int)((unsigned)(__double_as_longlong(fmax) >> 52) & 0x7ffu)) - 1023;
  const int escale = fexp - 20;
  const float up = pow2f(escale), down = pow2f(-escale);

  int k = 0;
  int32_t st = BAND_OK;
  // pass 0 is x_0 = U^{-1} z; pass m >= 1 applies correction m; at most max_steps + 1
  for (int pass = 0; pass <= p.max_steps; ++pass) {
    // ---- B: backward substitution (+ update), then the residual of the new x -----
    const bool first = (pass == 0);
    float dmaxf = 0.0f;
    double xmax = 0.0;
    bool bad = false;
    {
      constexpr int D = kDepthB;
      const Ring2<8, 2, D> ring{reinterpret_cast<float*>(stage),
                                reinterpret_cast<double*>(stage + D * 32 * 4 * 8), lane};
      // row t of the sweep is matrix row i = n-1-t; its residual row is i+2
      const float* FS[8] = {pa, p.b, p.c, p.d, pe, p.fa, p.fb, p.z};
      const double* DS[2] = {p.f, p.x};
      auto issue_row = [&](int slot, int64_t i) {
        // A row and f of residual row i+2 (clamped inside), spill and x of row i
        const int64_t j = i + 2 < n ? i + 2 : n - 1;
        const int64_t qj = q0 + j * es, wi = w0 + (i < 0 ? 0 : i) * ws, qi = q0 + (i < 0 ? 0 : i) * es;
#pragma unroll
        for (int a = 0; a < 5; ++a) cp_async_elem(ring.fs + ((slot * 8 + a) << 5) + lane, FS[a] + qj);
#pragma unroll
        for (int a = 5; a < 8; ++a) cp_async_elem(ring.fs + ((slot * 8 + a) << 5) + lane, FS[a] + wi);
        cp_async_elem(ring.ds + ((slot * 2 + 0) << 5) + lane, DS[0] + qj);
        cp_async_elem(ring.ds + ((slot * 2 + 1) << 5) + lane, DS[1] + qi);
        cp_async_commit();
      };
      const int64_t T = n + 2;          // t = 0 .. n+1 covers rows i = n-1 .. -2
      if (RING) {
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
          if (j < T) issue_row(j, n - 1 - j);
          else cp_async_commit();
        }
      }
      float d1 = 0, d2 = 0;               // delta (or x_0) of rows i+1, i+2
      F2 x1{0, 0}, x2{0, 0}, x3{0, 0}, x4{0, 0};   // new x of rows i+1 .. i+4
      for (int64_t t = 0; t < T; ++t) {
        const int64_t i = n - 1 - t;
        float A[5], av, bv2, zv;
        double fj, xo;
        if (RING) {
          const int64_t tp = t + D - 1;
          if (tp < T) issue_row((int)(tp & (D - 1)), n - 1 - tp);
          else cp_async_commit();
          cp_async_wait<D - 1>();
          const int sl = (int)(t & (D - 1));
#pragma unroll
          for (int a = 0; a < 5; ++a) A[a] = ring.getf(sl, a);
          av = ring.getf(sl, 5); bv2 = ring.getf(sl, 6); zv = ring.getf(sl, 7);
          fj = ring.getd(sl, 0); xo = ring.getd(sl, 1);
        } else {
          const int64_t j = i + 2 < n ? i + 2 : n - 1;
          const int64_t qj = q0 + j * es, wi = w0 + (i < 0 ? 0 : i) * ws;
          const int64_t qi = q0 + (i < 0 ? 0 : i) * es;
#pragma unroll
          for (int a = 0; a < 5; ++a) A[a] = (K == 1 && (a == 0 || a == 4)) ? 0.0f : ldro(A5[a] + qj);
          av = p.fa[wi]; bv2 = p.fb[wi]; zv = p.z[wi];
          fj = p.f[qj]; xo = p.x[qi];
        }
        F2 xn{0, 0};
        if (i >= 0) {
          float dv = fmaf(-av, d1, zv);
          if (K == 2) dv = fmaf(-bv2, d2, dv);
          d2 = d1;
          d1 = dv;
          if (first) {
            xn = F2{dv, 0.0f};
          } else {
            const float dd = dv * up;                 // the correction in x's units
            dmaxf = fmaxf(dmaxf, fabsf(dd));
            const F2 xs = split(xo);
            const F2 t1 = two_sum(xs.h, dd);
            const F2 t2 = two_sum(t1.h, t1.l + xs.l);
            xn = t2;
          }
          const double xv = f2d(xn.h) + f2d(xn.l);
          p.x[q0 + i * es] = xv;
          bad |= not_finite(xv);
          xmax = max_abs(xmax, xv);
        }
        // residual of row j = i + 2: x_{j-2} = xn (row i), x_{j-1} = x1, x_j = x2,
        // x_{j+1} = x3, x_{j+2} = x4
        const int64_t j = i + 2;
        if (j >= 0 && j < n) {
          F2 sres = split(fj);
          sub_prod(sres, A[2], x2);
          if (j >= 1) sub_prod(sres, A[1], x1);
          if (j + 1 < n) sub_prod(sres, A[3], x3);
          if (K == 2) {
            if (j >= 2) sub_prod(sres, A[0], xn);
            if (j + 2 < n) sub_prod(sres, A[4], x4);
          }
          p.r[w0 + j * ws] = (sres.h + sres.l) * down;
        }
        x4 = x3; x3 = x2; x2 = x1; x1 = xn;
      }
      if (RING) cp_async_wait<0>();
    }
    if (bad) { st = BAND_ERR_NONFINITE; break; }
    if (!first) {
      k = pass;
      if ((double)dmaxf <= p.rel_stop * xmax) break;
    }
    if (pass >= p.max_steps) break;
    // ---- F: z = L^{-1} (2^-e r) with the stored factors -----------------------------
    {
      constexpr int D = kDepthF;
      const Ring2<4, 0, D> ring{reinterpret_cast<float*>(stage), nullptr, lane};
      const float* FS[4] = {p.r, pa, p.fg, p.fr};
      auto issue_row = [&](int slot, int64_t i) {
        const int64_t wi = w0 + i * ws, qi = q0 + i * es;
        cp_async_elem(ring.fs + ((slot * 4 + 0) << 5) + lane, FS[0] + wi);
        cp_async_elem(ring.fs + ((slot * 4 + 1) << 5) + lane, FS[1] + qi);
        cp_async_elem(ring.fs + ((slot * 4 + 2) << 5) + lane, FS[2] + wi);
        cp_async_elem(ring.fs + ((slot * 4 + 3) << 5) + lane, FS[3] + wi);
        cp_async_commit();
      };
      if (RING) {
#pragma unroll
        for (int j = 0; j < D - 1; ++j) {
          if (j < n) issue_row(j, j);
          else cp_async_commit();
        }
      }
      float z1 = 0, z2 = 0;
      for (int64_t i = 0; i < n; ++i) {
        float rv, av, gv, rr;
        if (RING) {
          const int64_t ip = i + D - 1;
          if (ip < n) issue_row((int)(ip & (D - 1)), ip);
          else cp_async_commit();
          cp_async_wait<D - 1>();
          const int sl = (int)(i & (D - 1));
          rv = ring.getf(sl, 0); av = ring.getf(sl, 1); gv = ring.getf(sl, 2); rr = ring.getf(sl, 3);
        } else {
          const int64_t wi = w0 + i * ws;
          rv = p.r[wi]; av = K == 2 ? ldro(pa + q0 + i * es) : 0.0f; gv = p.fg[wi]; rr = p.fr[wi];
        }
        const float ai = (K == 2 && i >= 2) ? av : 0.0f;
        const float zv = fmaf(-z1, gv, fmaf(-z2, ai, rv)) * rr;
        p.z[w0 + i * ws] = zv;
        z2 = z1;
        z1 = zv;
      }
      if (RING) cp_async_wait<0>();
    }
  }
  if (p.steps) p.steps[s] = k;
  set_status(p.status, s, st);
}

__global__ void __launch_bounds__(32 * kRefWarps) k_refine(const RefArgs p, int kmode) {
  extern __shared__ __align__(16) unsigned char ref_stage[];
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  unsigned char* stage = ref_stage + (threadIdx.x >> 5) * kRefRingBytes;
  const int K = kmode ? kmode : p.L.kband(s);
  const bool ring = !p.L.offsets && p.L.ss == 1;
  if (ring) {
    if (K == 1) refine_one<1, true>(p, s, stage);
    else refine_one<2, true>(p, s, stage);
  } else {
    if (K == 1) refine_one<1, false>(p, s, stage);
    else refine_one<2, false>(p, s, stage);
  }
}

struct RefWs {
  float *fa, *fb, *fg, *fr, *z, *r;
};
RefWs carve_refine(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  RefWs w;
  const size_t rows = (size_t)spill_rows(d) * sizeof(float);
  w.fa = (float*)c.take(rows);
  w.fb = (float*)c.take(rows);
  w.fg = (float*)c.take(rows);
  w.fr = (float*)c.take(rows);
  w.z = (float*)c.take(rows);
  w.r = (float*)c.take(rows);
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

extern "C" band_status band_refine_solve(const band_desc* desc32, const void* const diag32[5],
                                         const double* f, double* x, double rel_stop,
                                         int32_t max_steps, int32_t* steps, int32_t* sys_status,
                                         void* ws, size_t ws_bytes, void* stream) {
  if (!desc_ok(desc32) || desc32->dtype != BAND_F32 || desc32->systems) return BAND_ERR_ARG;
  if (max_steps < 0 || !(rel_stop >= 0.0)) return BAND_ERR_ARG;
  if (desc32->nsys == 0) return BAND_OK;
  if (!diag32 || !f || !x) return BAND_ERR_ARG;
  if (!diag32[1] || !diag32[2] || !diag32[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc32) && (!diag32[0] || !diag32[4])) return BAND_ERR_ARG;
  size_t need = 0;
  carve_refine(desc32, nullptr, &need);
  if (!ws || ws_bytes < need) return BAND_ERR_WORKSPACE;
  const RefWs w = carve_refine(desc32, ws, &need);
  RefArgs p{layout_of(desc32), spill_of(desc32),
            (const float*)diag32[0], (const float*)diag32[1], (const float*)diag32[2],
            (const float*)diag32[3], (const float*)diag32[4], f, x,
            w.fa, w.fb, w.fg, w.fr, w.z, w.r, rel_stop, max_steps, steps, sys_status};
  const int kmode = desc32->hbw ? 0 : desc32->half_bw;
  const size_t smem = (size_t)kRefWarps * kRefRingBytes;
  if (cudaFuncSetAttribute(k_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return BAND_ERR_CUDA;
  const int tb = 32 * kRefWarps;
  k_refine<<<(unsigned)((desc32->nsys + tb - 1) / tb), tb, smem,
             static_cast<cudaStream_t>(stream)>>>(p, kmode);
  return cuda_status(cudaGetLastError());
}
