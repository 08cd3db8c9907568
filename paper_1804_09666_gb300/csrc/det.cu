// det.cu -- band_det: the determinant of every system of a batch in O(N) operations
// (Veneva & Ayriyan, arXiv:1804.09666, Sec. 3.2, Remark 1: the symbolic algorithm
// gives det A as the limit of the product of its pivots).
//
// A numeric pass runs the NPDM / NTDM factor recurrence (gamma, mu, alpha, beta; no
// right-hand side) and keeps the product of the pivots as mantissa * 2^exponent, the
// mantissa renormalised every row so that no product overflows.  A system whose pass
// meets a pivot that is exactly zero (or within rounding residue of zero, as for the
// numeric sweep of STDM / SPDM: residue_pivot in sweeps.cuh) is handed to the
// Laurent-series fix-up (symbolic.cuh) in its determinant-only form: V = the sum of
// the pivots' valuations decides SINGULAR (V > 0), and for V = 0 the product of the
// leading coefficients is the determinant.
#include <cstdint>

#include "api_util.h"
#include "kernels.h"
#include "sweeps.cuh"
#include "symbolic.cuh"

namespace band {

struct DetArgs {
  Layout L;
  const double *a, *b, *c, *d, *e;
  double* mant;
  long long* ex;
  int32_t* status;
  unsigned long long* fix_count;
  int64_t* fix_list;
};

// One thread per system: the numeric pass.
template <int K>
__global__ void __launch_bounds__(128) k_det(const DetArgs p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.L.nsys) return;
  const int64_t s = p.L.sys(t);
  const int kb = K ? K : p.L.kband(s);
  const int64_t n = p.L.rows(s);
  const int64_t q0 = p.L.base(s), es = p.L.stride();
  double al1 = 0.0, al2 = 0.0, be1 = 0.0, be2 = 0.0;
  double mant = 1.0;
  long long ex = 0;
  bool zero = false;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es;
    const double ai = (kb == 2 && i >= 2) ? ldro(p.a + q) : 0.0;
    const double bi = i >= 1 ? ldro(p.b + q) : 0.0;
    const double ci = ldro(p.c + q);
    const double di = i + 1 < n ? ldro(p.d + q) : 0.0;
    const double ei = (kb == 2 && i + 2 < n) ? ldro(p.e + q) : 0.0;
    const double g = fma(-al2, ai, bi);
    const double m = fma(-al1, g, fma(-be2, ai, ci));
    if (is_zero(m) || residue_pivot<double>(m, ai, bi, ci, al1, al2, be2, g)) {
      zero = true;
      break;
    }
    int e2;
    mant *= frexp(m, &e2);
    ex += e2;
    int e3;
    mant = frexp(mant, &e3);
    ex += e3;
    const double r = rcp64(m);
    const double alv = fma(-be1, g, di) * r;
    const double bev = ei * r;
    al2 = al1;
    al1 = alv;
    be2 = be1;
    be1 = bev;
  }
  if (zero) {
    const unsigned long long k = atomicAdd(p.fix_count, 1ull);
    p.fix_list[k] = t;
    return;
  }
  const bool ok = !not_finite(mant);
  p.mant[s] = mant;
  p.ex[s] = ex;
  set_status(p.status, s, ok ? BAND_OK : BAND_ERR_NONFINITE);
}

// The fix-up in its determinant-only form needs no series rows: one warp per flagged
// system, min(nsys, kFixSlotsMax) warps.
constexpr int kDetFixWarps = 4;
__global__ void __launch_bounds__(32 * kDetFixWarps) k_det_fixup(const SymArgs p) {
  __shared__ lser::dd stage[kDetFixWarps][128];
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= p.nslots) return;
  const unsigned long long count = *p.fix_count;
  const lser::SlotView none{nullptr, nullptr, p.nmax};
  for (unsigned long long item = w; item < count; item += p.nslots)
    lser::symbolic_warp(p, p.fix_list[item], none, stage[threadIdx.x >> 5]);
}

// Workspace of band_det: the flagged-system counter and list.
static size_t carve_det(const band_desc* d, void* base, void** count, void** list) {
  Carve c(base);
  *count = c.take(sizeof(unsigned long long));
  *list = c.take(sizeof(int64_t) * (size_t)(d->nsys > 0 ? d->nsys : 1));
  return c.size();
}

size_t det_workspace_bytes(const band_desc* d) {
  void *a, *b;
  return carve_det(d, nullptr, &a, &b);
}

}  // namespace band

using namespace band;

extern "C" band_status band_det(const band_desc* desc, const void* const diag[5], double* det_mant,
                                int64_t* det_exp, int32_t* sys_status, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64 || desc->systems) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !diag[1] || !diag[2] || !diag[3] || !det_mant || !det_exp || !sys_status)
    return BAND_ERR_ARG;
  const int kmode = desc->hbw ? 0 : desc->half_bw;
  if (kmode != 0 && kmode != 1 && kmode != 2) return BAND_ERR_ARG;
  if (kmode != 1 && (!diag[0] || !diag[4])) return BAND_ERR_ARG;
  if (!arrays_aligned(BAND_F64, diag, det_mant, det_exp, sys_status)) return BAND_ERR_ARG;
  void *count, *list;
  const size_t need = carve_det(desc, nullptr, &count, &list);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  carve_det(desc, ws, &count, &list);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return BAND_ERR_CUDA;
  const Layout L = layout_of(desc);
  DetArgs p{L, (const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
            (const double*)diag[3], (const double*)diag[4], det_mant, (long long*)det_exp,
            sys_status, (unsigned long long*)count, (int64_t*)list};
  const unsigned grid = (unsigned)((desc->nsys + 127) / 128);
  if (kmode == 1) k_det<1><<<grid, 128, 0, st>>>(p);
  else if (kmode == 2) k_det<2><<<grid, 128, 0, st>>>(p);
  else k_det<0><<<grid, 128, 0, st>>>(p);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  SymArgs sa{};
  sa.L = L;
  sa.a = p.a;
  sa.b = p.b;
  sa.c = p.c;
  sa.d = p.d;
  sa.e = p.e;
  sa.status = sys_status;
  sa.fix_count = (const unsigned long long*)count;
  sa.fix_list = (const int64_t*)list;
  sa.nslots = desc->nsys < kFixSlotsMax ? desc->nsys : kFixSlotsMax;
  sa.nmax = desc->n;
  sa.det_mant = det_mant;
  sa.det_exp = (long long*)det_exp;
  sa.det_only = 1;
  const int tb = 32 * kDetFixWarps;
  k_det_fixup<<<(unsigned)((sa.nslots * 32 + tb - 1) / tb), tb, 0, st>>>(sa);
  return cuda_status(cudaGetLastError());
}
