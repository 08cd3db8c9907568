// adjoint.cu -- gradients of x = A^{-1} f through the NPDM / NTDM factorisation.
//
// For a loss L(x) with w = dL/dx:  A^T lambda = w,  dL/df = lambda,
// dL/dA[i][j] = -lambda_i x_j, i.e. on the row-aligned diagonals
//   ga_i = -lambda_i x_{i-2}, gb_i = -lambda_i x_{i-1}, gc_i = -lambda_i x_i,
//   gd_i = -lambda_i x_{i+1}, ge_i = -lambda_i x_{i+2}  (0 outside the matrix).
// With A = L U (L lower with diagonals a_i, gamma_i, mu_i; U unit upper with alpha_i,
// beta_i -- the NPDM factorisation of Veneva & Ayriyan, Sec. 1):
//   U^T v = w:       v_i = w_i - alpha_{i-1} v_{i-1} - beta_{i-2} v_{i-2}
//   L^T lambda = v:  lambda_i = (v_i - gamma_{i+1} lambda_{i+1} - a_{i+2} lambda_{i+2}) / mu_i
// With stored factors (band_factor's buffer), or for ragged batches, one thread per
// system runs these two sweeps and forms the gradients in the second.
//
// Otherwise A^T lambda = w is solved as a band system of its own: A^T's row-aligned
// diagonals are (e_{i-2}, d_{i-1}, c_i, b_{i+1}, a_{i+2}), copied into the workspace
// by an elementwise kernel; the NPDM / NTDM sweep then runs on them as band_solve would
// on the schedule band_desc asks for (on AUTO: partitioned for a batch too small to fill
// the GPU, two-sided otherwise), writing lambda straight into dL/df; an elementwise
// kernel forms the five gradient diagonals.  The two copies are memory traffic at full
// bandwidth; the solve is the part bound by its chains.
#include "api_util.h"
#include "kernels.h"

namespace band {
namespace {

struct AdjArgs {
  Layout L;
  Spill W;
  const double *a, *b, *c, *d, *e;
  const double *x, *w;
  const double *fg, *fr, *fa, *fb;  // stored factors (gamma, 1/mu, alpha, beta) or null
  double *ga, *gb, *gc, *gd, *ge, *gf;
  double *sg, *sr, *sv;             // workspace rows: gamma, 1/mu, v
  int32_t* status;
};

template <int K>
__device__ void adjoint_one(const AdjArgs& p, int64_t s) {
  const int64_t n = p.L.rows(s), q0 = p.L.base(s), es = p.L.stride();
  const int64_t w0 = p.W.base(s), ws = p.W.stride();
  const bool stored = p.fr != nullptr;
  double al1 = 0, al2 = 0, be1 = 0, be2 = 0, v1 = 0, v2 = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t q = q0 + i * es, wi = w0 + i * ws;
    double g, r, alv, bev;
    if (stored) {
      g = p.fg[wi];
      r = p.fr[wi];
      alv = p.fa[wi];
      bev = p.fb[wi];
    } else {
      const double bi = (i >= 1) ? ldro(p.b + q) : 0.0;
      const double ci = ldro(p.c + q);
      const double di = (i + 1 < n) ? ldro(p.d + q) : 0.0;
      double ai = 0.0, ei = 0.0;
      if (K == 2) {
        ai = (i >= 2) ? ldro(p.a + q) : 0.0;
        ei = (i + 2 < n) ? ldro(p.e + q) : 0.0;
      }
      g = fma(-al2, ai, bi);
      const double m = fma(-al1, g, fma(-be2, ai, ci));
      if (m == 0.0) {
        set_status(p.status, s, BAND_ERR_ZERO_PIVOT);
        return;
      }
      r = rcp64(m);
      alv = fma(-be1, g, di) * r;
      bev = ei * r;
    }
    double v = fma(-al1, v1, p.w[q]);
    if (K == 2) v = fma(-be2, v2, v);
    p.sg[wi] = g;
    p.sr[wi] = r;
    p.sv[wi] = v;
    al2 = al1; al1 = alv; be2 = be1; be1 = bev; v2 = v1; v1 = v;
  }
  double l1 = 0, l2 = 0;       // lambda_{i+1}, lambda_{i+2}
  double g1 = 0;               // gamma_{i+1}
  double a1 = 0, a2 = 0;       // a_{i+1}, a_{i+2}
  double xp1 = 0, xp2 = 0;     // x_{i+1}, x_{i+2}
  bool bad = false;
  for (int64_t i = n - 1; i >= 0; --i) {
    const int64_t q = q0 + i * es, wi = w0 + i * ws;
    double t = fma(-g1, l1, p.sv[wi]);
    if (K == 2) t = fma(-a2, l2, t);
    const double lam = t * p.sr[wi];
    const double xi = p.x[q];
    const double xm1 = (i >= 1) ? p.x[q - es] : 0.0;
    p.gf[q] = lam;
    p.gc[q] = -lam * xi;
    p.gb[q] = (i >= 1) ? -lam * xm1 : 0.0;
    p.gd[q] = (i + 1 < n) ? -lam * xp1 : 0.0;
    if (K == 2) {
      const double xm2 = (i >= 2) ? p.x[q - 2 * es] : 0.0;
      p.ga[q] = (i >= 2) ? -lam * xm2 : 0.0;
      p.ge[q] = (i + 2 < n) ? -lam * xp2 : 0.0;
    } else {
      if (p.ga) p.ga[q] = 0.0;
      if (p.ge) p.ge[q] = 0.0;
    }
    bad |= !isfinite(lam);
    l2 = l1; l1 = lam;
    g1 = p.sg[wi];
    a2 = a1;
    a1 = (K == 2 && i >= 2) ? ldro(p.a + q) : 0.0;
    xp2 = xp1; xp1 = xi;
  }
  set_status(p.status, s, bad ? BAND_ERR_NONFINITE : BAND_OK);
}

__global__ void __launch_bounds__(128) k_adjoint(const AdjArgs p, int kmode) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.L.nsys) return;
  const int K = kmode ? kmode : p.L.kband(s);
  if (K == 1) adjoint_one<1>(p, s);
  else adjoint_one<2>(p, s);
}

struct AdjWs {
  double *g, *r, *v;
};
AdjWs carve_adjoint(const band_desc* d, void* base, size_t* bytes) {
  Carve c(base);
  const size_t rows = (size_t)spill_rows(d) * sizeof(double);
  AdjWs w;
  w.g = (double*)c.take(rows);
  w.r = (double*)c.take(rows);
  w.v = (double*)c.take(rows);
  *bytes = c.size();
  return w;
}

// Elements of one strided array that a uniform batch spans.
int64_t span_of(const band_desc* d) {
  return (d->n - 1) * d->elem_stride + (d->nsys - 1) * d->sys_stride + 1;
}

// Workspace of the transposed path: A^T's diagonals in A's layout, then the solve's.
struct AdjTWs {
  double* t[5];
  void* solve;
  size_t solve_bytes;
};
AdjTWs carve_adjoint_t(const band_desc* d, int32_t method, void* base, size_t* bytes) {
  Carve c(base);
  AdjTWs w{};
  const size_t arr = (size_t)span_of(d) * sizeof(double);
  for (int k = 0; k < 5; ++k) w.t[k] = (double*)c.take(arr);
  const size_t sb = single_solve_bytes(d, method);    // band_solve's workspace for A^T
  w.solve = c.take(sb);
  w.solve_bytes = sb;
  *bytes = c.size();
  return w;
}

// (i, s) of the idx-th element, running along the unit-stride index first
__device__ __forceinline__ void elem_of(const Layout& L, int64_t idx, int64_t& i, int64_t& s) {
  if (L.ss == 1) { s = idx % L.nsys; i = idx / L.nsys; }
  else { i = idx % L.n; s = idx / L.n; }
}

template <int K>
__global__ void __launch_bounds__(256) k_transpose_band(const Layout L, const double* a,
                                                        const double* b, const double* c,
                                                        const double* d, const double* e,
                                                        double* ta, double* tb, double* tc,
                                                        double* td, double* te) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.nsys * L.n) return;
  int64_t i, s;
  elem_of(L, idx, i, s);
  const int64_t n = L.n, es = L.es, q = s * L.ss + i * es;
  tc[q] = ldro(c + q);
  tb[q] = (i >= 1) ? ldro(d + q - es) : 0.0;
  td[q] = (i + 1 < n) ? ldro(b + q + es) : 0.0;
  if (K == 2) {
    ta[q] = (i >= 2) ? ldro(e + q - 2 * es) : 0.0;
    te[q] = (i + 2 < n) ? ldro(a + q + 2 * es) : 0.0;
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_adjoint_grad(const Layout L, const double* x,
                                                      const double* lam, double* ga, double* gb,
                                                      double* gc, double* gd, double* ge) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L.nsys * L.n) return;
  int64_t i, s;
  elem_of(L, idx, i, s);
  const int64_t n = L.n, es = L.es, q = s * L.ss + i * es;
  const double l = lam[q];
  gc[q] = -l * x[q];
  gb[q] = (i >= 1) ? -l * x[q - es] : 0.0;
  gd[q] = (i + 1 < n) ? -l * x[q + es] : 0.0;
  if (K == 2) {
    ga[q] = (i >= 2) ? -l * x[q - 2 * es] : 0.0;
    ge[q] = (i + 2 < n) ? -l * x[q + 2 * es] : 0.0;
  } else {
    if (ga) ga[q] = 0.0;
    if (ge) ge[q] = 0.0;
  }
}

}  // namespace

size_t adjoint_workspace_bytes(const band_desc* d) {
  size_t b = 0, bt = 0;
  carve_adjoint(d, nullptr, &b);
  if (!d->offsets && d->nsys > 0 && d->n > 0) {
    carve_adjoint_t(d, d->half_bw == 1 ? BAND_NTDM : BAND_NPDM, nullptr, &bt);
  }
  return b > bt ? b : bt;
}

}  // namespace band

using namespace band;

extern "C" band_status band_adjoint(const band_desc* desc, int32_t method, const void* factors,
                                    const void* const diag[5], const void* x, const void* w,
                                    void* const grad_diag[5], void* grad_f, int32_t* sys_status,
                                    void* ws, size_t ws_bytes, void* stream) {
  if (!desc_ok(desc) || desc->dtype != BAND_F64 || desc->systems) return BAND_ERR_ARG;
  const int kmode = kmode_for(desc, method);
  if (kmode < 0 || is_symbolic(method)) return BAND_ERR_ARG;
  if (desc->nsys == 0) return BAND_OK;
  if (!diag || !x || !w || !grad_diag || !grad_f) return BAND_ERR_ARG;
  if (!diag[1] || !diag[2] || !diag[3]) return BAND_ERR_ARG;
  if (!grad_diag[1] || !grad_diag[2] || !grad_diag[3]) return BAND_ERR_ARG;
  const bool pd = may_be_pd(desc) && kmode != 1;
  if (pd && (!diag[0] || !diag[4] || !grad_diag[0] || !grad_diag[4])) return BAND_ERR_ARG;
  if (!arrays_aligned(BAND_F64, diag, x, w, sys_status) ||
      !arrays_aligned(BAND_F64, grad_diag, grad_f, nullptr, nullptr))
    return BAND_ERR_ARG;
  if (!aligned_to(factors, kWsAlign)) return BAND_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!factors && !desc->offsets && kmode > 0) {
    // the transposed system solved as a band system of its own
    const int32_t m = kmode == 1 ? BAND_NTDM : BAND_NPDM;
    size_t need = 0;
    carve_adjoint_t(desc, m, nullptr, &need);
    if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
    const AdjTWs tw = carve_adjoint_t(desc, m, ws, &need);
    const Layout L = layout_of(desc);
    const int64_t total = desc->nsys * desc->n;
    const unsigned grid = (unsigned)((total + 255) / 256);
    const double* A[5] = {(const double*)diag[0], (const double*)diag[1], (const double*)diag[2],
                          (const double*)diag[3], (const double*)diag[4]};
    if (kmode == 2)
      k_transpose_band<2><<<grid, 256, 0, st>>>(L, A[0], A[1], A[2], A[3], A[4], tw.t[0], tw.t[1],
                                                tw.t[2], tw.t[3], tw.t[4]);
    else
      k_transpose_band<1><<<grid, 256, 0, st>>>(L, A[0], A[1], A[2], A[3], A[4], tw.t[0], tw.t[1],
                                                tw.t[2], tw.t[3], tw.t[4]);
    if (cudaGetLastError() != cudaSuccess) return BAND_ERR_CUDA;
    const void* dt[5] = {tw.t[0], tw.t[1], tw.t[2], tw.t[3], tw.t[4]};
    // A^T solved as band_solve would (its automatic schedule included)
    const band_status v = run_single(desc, m, dt, w, grad_f, sys_status, tw.solve,
                                     tw.solve_bytes, st);
    if (v != BAND_OK) return v;
    double* G[5] = {(double*)grad_diag[0], (double*)grad_diag[1], (double*)grad_diag[2],
                    (double*)grad_diag[3], (double*)grad_diag[4]};
    if (kmode == 2)
      k_adjoint_grad<2><<<grid, 256, 0, st>>>(L, (const double*)x, (const double*)grad_f, G[0],
                                              G[1], G[2], G[3], G[4]);
    else
      k_adjoint_grad<1><<<grid, 256, 0, st>>>(L, (const double*)x, (const double*)grad_f, G[0],
                                              G[1], G[2], G[3], G[4]);
    return cuda_status(cudaGetLastError());
  }
  size_t need = 0;
  carve_adjoint(desc, nullptr, &need);
  if (!ws_fits(ws, ws_bytes, need)) return BAND_ERR_WORKSPACE;
  const AdjWs wk = carve_adjoint(desc, ws, &need);
  AdjArgs p{};
  p.L = layout_of(desc);
  p.W = spill_of(desc);
  p.a = (const double*)diag[0]; p.b = (const double*)diag[1]; p.c = (const double*)diag[2];
  p.d = (const double*)diag[3]; p.e = (const double*)diag[4];
  p.x = (const double*)x;
  p.w = (const double*)w;
  if (factors) {
    const FactorPtrs fp = factor_ptrs(desc, factors);
    p.fg = (const double*)fp.gam; p.fr = (const double*)fp.rmu;
    p.fa = (const double*)fp.al; p.fb = (const double*)fp.be;
  }
  p.ga = (double*)grad_diag[0]; p.gb = (double*)grad_diag[1]; p.gc = (double*)grad_diag[2];
  p.gd = (double*)grad_diag[3]; p.ge = (double*)grad_diag[4];
  p.gf = (double*)grad_f;
  p.sg = wk.g; p.sr = wk.r; p.sv = wk.v;
  p.status = sys_status;
  k_adjoint<<<(unsigned)((desc->nsys + 127) / 128), 128, 0, st>>>(p, kmode);
  return cuda_status(cudaGetLastError());
}
