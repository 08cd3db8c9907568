// adi.cu -- band_adi_step: one time step of a nonlinear parabolic PDE on a square grid
// by the alternating direction implicit method, the use the paper's band solvers are
// for (Sec. 1: an ADI step solves N independent TD or PD systems per direction).
//
//   u_t = u_xx + u_yy + g(u) + s(x, y),   g(u) = lambda u (1 - u),
// on the unit square, u = 0 on the boundary, n x n interior points (h = 1 / (n + 1)),
// u stored row-major (u[y * n + x]).  Second differences along one direction: the
// 3-point stencil (1, -2, 1) / h^2 (half_bw 1: TD systems) or the fourth-order 5-point
// stencil (-1, 16, -30, 16, -1) / (12 h^2) (half_bw 2: PD systems), u = 0 on the
// boundary and, for the 5-point stencil, the point beyond it the odd reflection of the
// first interior point (u(-h) = -u(h): second order at the boundary rows, where zero
// there would be first order).  The nonlinearity stays on the right-hand side (evaluated at the latest values).
// One Peaceman-Rachford step, theta = tau / 2:
//   (I - theta D_x) u* = u + theta (D_y u + g(u) + s)          x-sweep: n systems (rows)
//   (I - theta D_y) u' = u* + theta (D_x u* + g(u*) + s)       y-sweep: n systems (columns)
// The implicit operator I - theta D has constant diagonals (r = theta / h^2):
//   TD: (-r, 1 + 2r, -r);  PD: (r/12, -4r/3, 1 + 5r/2, -4r/3, r/12), the reflection
// making the PD main diagonal 1 + 29r/12 on each system's first and last row,
// written into the workspace (the main diagonal once per sweep); the line systems are
// solved by band_solve (NTDM / NPDM on its automatic schedule: partitioned while the
// grid has fewer than 32 lines per SM, two-sided beyond), x-sweep systems contiguous,
// y-sweep systems interleaved.  The right-hand sides come from one elementwise stencil kernel each.
#include <cstdint>

#include "api_util.h"
#include "kernels.h"

namespace band {

namespace {

// g(u) = lambda u (1 - u)
__device__ __forceinline__ double g_of(double u, double lambda) { return lambda * u * (1.0 - u); }

// F = v + theta (D v + g(v) + s), D along y (axis 1) or x (axis 0) of the row-major grid
template <int K>
__global__ void __launch_bounds__(256) k_adi_rhs(const double* __restrict__ v,
                                                 const double* __restrict__ src,
                                                 double* __restrict__ F, int64_t n, int axis,
                                                 double theta, double inv_h2, double lambda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t y = idx / n, x = idx - y * n;
  const int64_t pos = axis == 1 ? y : x;         // coordinate along the stencil
  const int64_t step = axis == 1 ? n : 1;
  const double c = v[idx];
  auto at = [&](int64_t off) -> double {
    const int64_t p = pos + off;
    if (p == -2 || p == n + 1) return -c;      // the reflected point beyond the boundary
    return (p >= 0 && p < n) ? v[idx + off * step] : 0.0;
  };
  double dv;
  if (K == 1) {
    dv = (at(-1) - 2.0 * c + at(1)) * inv_h2;
  } else {
    dv = (-at(-2) + 16.0 * at(-1) - 30.0 * c + 16.0 * at(1) - at(2)) * (inv_h2 / 12.0);
  }
  const double s = src ? src[idx] : 0.0;
  F[idx] = c + theta * (dv + g_of(c, lambda) + s);
}

// the diagonals: a, b, d, e constant; the main diagonal of the x-sweep (position x) and
// of the y-sweep (position y), c_edge on each system's first and last row
__global__ void __launch_bounds__(256) k_adi_diags(double* a, double* b, double* d, double* e,
                                                   double* cx, double* cy, int64_t n, double va,
                                                   double vb, double vc, double vedge) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int64_t y = i / n, x = i - y * n;
  a[i] = va;
  b[i] = vb;
  d[i] = vb;
  e[i] = va;
  cx[i] = (x == 0 || x == n - 1) ? vedge : vc;
  cy[i] = (y == 0 || y == n - 1) ? vedge : vc;
}

struct AdiWs {
  void *diag[5], *cy, *F, *ustar, *solve;
  size_t solve_bytes;
};

// the two sweeps' descriptors: x-sweep systems are rows (contiguous), y-sweep systems
// columns (interleaved)
void sweep_descs(const band_desc* g, band_desc* dx, band_desc* dy) {
  *dx = band_desc{};
  dx->half_bw = g->half_bw;
  dx->dtype = BAND_F64;
  dx->nsys = g->n;
  dx->n = g->n;
  dx->sys_stride = g->n;
  dx->elem_stride = 1;
  *dy = *dx;
  dy->sys_stride = 1;
  dy->elem_stride = g->n;
}

AdiWs carve_adi(const band_desc* g, void* base, size_t* bytes) {
  Carve c(base);
  AdiWs w{};
  const size_t plane = (size_t)g->n * (size_t)g->n * sizeof(double);
  for (int q = 0; q < 5; ++q) w.diag[q] = c.take(plane);    // diag[2]: the x-sweep's c
  w.cy = c.take(plane);
  w.F = c.take(plane);
  w.ustar = c.take(plane);
  band_desc dx, dy;
  sweep_descs(g, &dx, &dy);
  const int32_t m = g->half_bw == 1 ? BAND_NTDM : BAND_NPDM;
  const size_t bx = single_solve_bytes(&dx, m), by = single_solve_bytes(&dy, m);  // band_solve's
  w.solve_bytes = bx > by ? bx : by;
  w.solve = c.take(w.solve_bytes);
  *bytes = c.size();
  return w;
}

bool grid_ok(const band_desc* g) {
  return g && g->dtype == BAND_F64 && (g->half_bw == 1 || g->half_bw == 2) && !g->hbw &&
         !g->offsets && g->n >= 3 && g->nsys == g->n && g->schedule == BAND_SCHED_AUTO &&
         g->chunks == 0;
}

}  // namespace

size_t adi_workspace_bytes(const band_desc* g) {
  if (!grid_ok(g)) return 0;
  size_t b = 0;
  carve_adi(g, nullptr, &b);
  return b;
}

}  // namespace band

using namespace band;

extern "C" band_status band_adi_step(const band_desc* grid, double tau, double lambda,
                                     const double* source, double* u, int32_t* sys_status,
                                     void* ws, size_t ws_bytes, void* stream) {
  if (!grid_ok(grid) || !u || !(tau > 0.0) || !(lambda == lambda)) return BAND_ERR_ARG;
  if (!aligned_all(8, {u, source}) || !aligned_to(sys_status, 4)) return BAND_ERR_ARG;
  size_t need = 0;
  carve_adi(grid, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const AdiWs w = carve_adi(grid, ws, &need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = grid->n, cells = n * n;
  const double h = 1.0 / (double)(n + 1);
  const double theta = 0.5 * tau, inv_h2 = 1.0 / (h * h), r = theta * inv_h2;
  const int K = grid->half_bw;
  // the implicit operator's diagonals (a, b, c, d, e)
  const double va = K == 2 ? r / 12.0 : 0.0, vb = K == 2 ? -4.0 * r / 3.0 : -r;
  const double vc = K == 2 ? 1.0 + 2.5 * r : 1.0 + 2.0 * r;
  const double vedge = K == 2 ? 1.0 + 29.0 * r / 12.0 : vc;
  const unsigned blocks = (unsigned)((cells + 255) / 256);
  k_adi_diags<<<blocks, 256, 0, st>>>((double*)w.diag[0], (double*)w.diag[1], (double*)w.diag[3],
                                      (double*)w.diag[4], (double*)w.diag[2], (double*)w.cy, n,
                                      va, vb, vc, vedge);
  band_desc dx, dy;
  sweep_descs(grid, &dx, &dy);
  const int32_t m = K == 1 ? BAND_NTDM : BAND_NPDM;
  const void* diag_x[5] = {w.diag[0], w.diag[1], w.diag[2], w.diag[3], w.diag[4]};
  const void* diag_y[5] = {w.diag[0], w.diag[1], w.cy, w.diag[3], w.diag[4]};
  // x-sweep: F = u + theta (D_y u + g(u) + s), solve along x into u*
  if (K == 1) k_adi_rhs<1><<<blocks, 256, 0, st>>>(u, source, (double*)w.F, n, 1, theta, inv_h2, lambda);
  else k_adi_rhs<2><<<blocks, 256, 0, st>>>(u, source, (double*)w.F, n, 1, theta, inv_h2, lambda);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  band_status v = band_solve(&dx, m, nullptr, diag_x, w.F, w.ustar, sys_status, w.solve,
                             w.solve_bytes, stream);
  if (v != BAND_OK) return v;
  // y-sweep: F = u* + theta (D_x u* + g(u*) + s), solve along y into u
  if (K == 1) k_adi_rhs<1><<<blocks, 256, 0, st>>>((double*)w.ustar, source, (double*)w.F, n, 0, theta, inv_h2, lambda);
  else k_adi_rhs<2><<<blocks, 256, 0, st>>>((double*)w.ustar, source, (double*)w.F, n, 0, theta, inv_h2, lambda);
  if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
  return band_solve(&dy, m, nullptr, diag_y, w.F, u, sys_status ? sys_status + n : nullptr, w.solve,
                    w.solve_bytes, stream);
}
