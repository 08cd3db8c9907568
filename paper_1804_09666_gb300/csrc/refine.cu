// refine.cu -- FP32 factor/solve with FP64 iterative refinement.
//
// The systems are stored in FP32; the right-hand side and the solution are FP64.
// x_0 = solve32(f); then per step
//   r = f - A x            (FP64, A = the FP64 values of the FP32 diagonals)
//   s = max |r|,  delta = s * solve32(r / s)   (scaling keeps FP32 in range)
//   x = x + delta          (FP64)
// until max|delta| <= rel_stop * max|x| or max_steps steps.  solve32 is the NPDM /
// NTDM recurrence (Veneva & Ayriyan, Sec. 1) in single precision, refactored from the
// FP32 diagonals on every call (they are read anyway for the residual).
// One thread per system.
#include "api_util.h"
#include "kernels.h"

namespace band {
namespace {

struct RefArgs {
  Layout L;
  Spill W;
  const float *a, *b, *c, *d, *e;
  const double* f;
  double* x;
  double* r;          // residual rows (workspace)
  float *al, *be, *zs;
  double rel_stop;
  int max_steps;
  int32_t *steps, *status;
};

// FP32 NPDM/NTDM solve of A32 y = rhs(i) * scale, y written through out(i, y).
template <int K, class Rhs, class Out>
__device__ __forceinline__ bool solve32(const RefArgs& p, int64_t n, int64_t q0, int64_t es,
                                        int64_t w0, int64_t ws, Rhs rhs, Out out) {
  float al1 = 0, al2 = 0, be1 = 0, be2 = 0, z1 = 0, z2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es, w = w0 + i * ws;
    const float bi = (i >= 1) ? ldro(p.b + q) : 0.0f;
    const float ci = ldro(p.c + q);
    const float di = (i + 1 < n) ? ldro(p.d + q) : 0.0f;
    const float fi = rhs(i, q);
    float ai = 0.0f, ei = 0.0f;
    if (K == 2) {
      ai = (i >= 2) ? ldro(p.a + q) : 0.0f;
      ei = (i + 2 < n) ? ldro(p.e + q) : 0.0f;
    }
    const float g = fmaf(-al2, ai, bi);
    const float m = fmaf(-al1, g, fmaf(-be2, ai, ci));
    if (m == 0.0f) return false;
    const float rr = __frcp_rn(m);
    const float alv = fmaf(-be1, g, di) * rr;
    const float bev = ei * rr;
    const float zv = fmaf(-z1, g, fmaf(-z2, ai, fi)) * rr;
    p.al[w] = alv;
    p.be[w] = bev;
    p.zs[w] = zv;
    al2 = al1; al1 = alv; be2 = be1; be1 = bev; z2 = z1; z1 = zv;
  }
  float x1 = 0, x2 = 0;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t w = w0 + i * ws;
    float xi = fmaf(-p.al[w], x1, p.zs[w]);
    if (K == 2) xi = fmaf(-p.be[w], x2, xi);
    out(i, q0 + i * es, xi);
    x2 = x1;
    x1 = xi;
  }
  return true;
}

template <int K>
__device__ void refine_one(const RefArgs& p, int64_t s) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  int32_t st = BAND_OK;
  int k = 0;
  if (!solve32<K>(p, n, q0, es, w0, ws, [&](int64_t, int64_t q) { return (float)p.f[q]; },
                  [&](int64_t, int64_t q, float v) { p.x[q] = (double)v; })) {
    st = BAND_ERR_ZERO_PIVOT;
  }
  while (st == BAND_OK && k < p.max_steps) {
    // r = f - A x in FP64
    double smax = 0.0;
    bool nan_seen = false;
    double xm2 = 0, xm1 = 0, x0 = p.x[q0], xp1 = n > 1 ? p.x[q0 + es] : 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t q = q0 + i * es;
      const double xp2 = (i + 2 < n) ? p.x[q + 2 * es] : 0.0;
      double ax = (double)ldro(p.c + q) * x0;
      if (i >= 1) ax = fma((double)ldro(p.b + q), xm1, ax);
      if (i + 1 < n) ax = fma((double)ldro(p.d + q), xp1, ax);
      if (K == 2) {
        if (i >= 2) ax = fma((double)ldro(p.a + q), xm2, ax);
        if (i + 2 < n) ax = fma((double)ldro(p.e + q), xp2, ax);
      }
      const double r = p.f[q] - ax;
      p.r[w0 + i * ws] = r;
      nan_seen |= (r != r);
      smax = fmax(smax, fabs(r));
      xm2 = xm1; xm1 = x0; x0 = xp1; xp1 = xp2;
    }
    if (nan_seen || !isfinite(smax)) { st = BAND_ERR_NONFINITE; break; }
    if (smax == 0.0) break;
    const double inv = 1.0 / smax;
    double dmax = 0.0, xmax = 0.0;
    const bool ok = solve32<K>(
        p, n, q0, es, w0, ws, [&](int64_t i, int64_t) { return (float)(p.r[w0 + i * ws] * inv); },
        [&](int64_t, int64_t q, float v) {
          const double dl = smax * (double)v;
          const double xn = p.x[q] + dl;
          p.x[q] = xn;
          dmax = fmax(dmax, fabs(dl));
          xmax = fmax(xmax, fabs(xn));
        });
    if (!ok) { st = BAND_ERR_ZERO_PIVOT; break; }
    ++k;
    if (dmax <= p.rel_stop * xmax) break;
  }
  if (st == BAND_OK) {
    for (int64_t i = 0; i < n; ++i)
      if (!isfinite(p.x[q0 + i * es])) { st = BAND_ERR_NONFINITE; break; }
  }
  if (p.steps) p.steps[s] = k;
  set_status(p.status, s, st);
}

__global__ void __launch_bounds__(128) k_refine(const RefArgs p, int kmode) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  const int K = kmode ? kmode : p.L.kband(s);
  if (K == 1) refine_one<1>(p, s);
  else refine_one<2>(p, s);
}

struct RefWs {
  void *r, *al, *be, *zs;
};
RefWs carve_refine(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  RefWs w;
  const size_t rows = (size_t)spill_rows(d);
  w.r = c.take(rows * sizeof(double));
  w.al = c.take(rows * sizeof(float));
  w.be = c.take(rows * sizeof(float));
  w.zs = c.take(rows * sizeof(float));
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
  if (!desc_ok(desc32) || desc32->dtype != BAND_F32) return BAND_ERR_ARG;
  if (max_steps < 0 || !(rel_stop >= 0.0)) return BAND_ERR_ARG;
  if (desc32->nsys == 0) return BAND_OK;
  if (!diag32 || !f || !x) return BAND_ERR_ARG;
  if (!diag32[1] || !diag32[2] || !diag32[3]) return BAND_ERR_ARG;
  if (may_be_pd(desc32) && (!diag32[0] || !diag32[4])) return BAND_ERR_ARG;
  if (max_steps < 0 || !(rel_stop >= 0.0)) return BAND_ERR_ARG;
  size_t need = 0;
  carve_refine(desc32, nullptr, &need);
  if (!ws || ws_bytes < need) return BAND_ERR_WORKSPACE;
  const RefWs w = carve_refine(desc32, ws, &need);
  RefArgs p{layout_of(desc32), spill_of(desc32),
            (const float*)diag32[0], (const float*)diag32[1], (const float*)diag32[2],
            (const float*)diag32[3], (const float*)diag32[4], f, x, (double*)w.r,
            (float*)w.al, (float*)w.be, (float*)w.zs, rel_stop, max_steps, steps, sys_status};
  const int kmode = desc32->hbw ? 0 : desc32->half_bw;
  k_refine<<<(unsigned)((desc32->nsys + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      p, kmode);
  return cuda_status(cudaGetLastError());
}
